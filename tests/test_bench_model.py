"""The byte and flop bookkeeping bench.py reports its rooflines on (CPU only).

At 128 x 128 x 32 (padded 256 x 256 x 64) the per-evaluation figures follow
from the array sizes: 3 x 129 x 128 x 32 complex spectrum rows (12.68 MB), a
y-transformed buffer twice as long in y (25.37 MB), a 6 x 129 x 129 x 33
float octant (13.18 MB) and 12 bytes per cell for a float32 3-vector field.
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_1406_7635_gb300.workloads import WORKLOADS  # noqa: E402

N = 128 * 128 * 32
SPEC = 3 * 8 * 129 * 128 * 32          # spectrum rows that carry data
T = SPEC // 128 * 256                  # y-transformed rows (py = 256)
OCT = 6 * 4 * 129 * 129 * 33           # kernel octant
ARR = 12 * N                           # one float32 3-vector field


@pytest.fixture(scope="module")
def c3():
    return WORKLOADS["ellipsoid_128x128x32"]()


def test_five_pass_bytes(c3):
    passes = bench.five_pass_passes(c3)
    assert passes == [N * 14 + SPEC, SPEC + T, 2 * T + OCT, T + SPEC, SPEC + ARR]
    assert round(sum(passes) / 1e6, 1) == 179.0
    fused, floor = bench.yz_kernel_bytes(c3)
    assert fused == 2 * (SPEC + T) + 2 * T + OCT and round(fused / 1e6, 1) == 140.0
    assert floor == 2 * SPEC + OCT and round(floor / 1e6, 1) == 38.5
    assert bench.algorithmic_demag_bytes(c3) == N * 26 + OCT


def test_row_and_partial_kernel_bytes(c3):
    # per launch: spectrum rows in, stage input and codes in, the earlier
    # stages' arrays, k_s out, then the next stage input and its spectrum
    # (five launches) or the candidate m (the last)
    earlier = [2, 3, 4, 5, 5, 5]
    base = [SPEC + ARR + 4 * N + ARR + (ARR + SPEC if i < 5 else ARR) for i in range(6)]
    full = sum(b + e * ARR for b, e in zip(base, earlier)) / 6
    part = sum(b + ARR for b in base) / 6
    assert bench.row_kernel_bytes(c3) == pytest.approx(full)
    assert bench.row_kernel_bytes(c3, partial=True) == pytest.approx(part)
    assert bench.partial_kernel_bytes(c3) == pytest.approx(sum((e + 1) * ARR for e in earlier) / 6)
    assert round(full / 1e6, 1) == 69.4 and round(part / 1e6, 1) == 50.5


def test_sources_hash_ignores_comments_only(tmp_path, monkeypatch):
    a = tmp_path / "a.cu"
    b = tmp_path / "b.cu"
    c = tmp_path / "c.cu"
    a.write_text("int f(int x) {\n  return x + 1;   // one more\n}\n")
    b.write_text("// a header line\nint f(int x) {\n\n  return x + 1;   // plus one\n}\n")
    c.write_text("int f(int x) {\n  return x + 2;\n}\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.sources_sha(["a.cu"]) == bench.sources_sha(["b.cu"])
    assert bench.sources_sha(["a.cu"]) != bench.sources_sha(["c.cu"])
