"""Batched multi-instance RK45 (many independent grids in one graph launch):
each instance against the float64 oracle replaying that instance's own step
sizes, and against the single-instance CUDA path."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.rk45 import RK45  # noqa: E402
from paper_1406_7635_gb300.workloads import batch_instances, problem_from_instance  # noqa: E402

M_TOL = 1e-5


@pytest.fixture(scope="module")
def mm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1406_7635_gb300.build import build
    build()
    from paper_1406_7635_gb300 import mm as _mm
    return _mm


SMALL_SHAPES = ((32, 32, 1), (64, 32, 1), (48, 24, 3), (17, 20, 2))


@pytest.fixture(scope="module")
def batch_run(mm):
    specs, m0s = batch_instances(16, shapes=SMALL_SHAPES, seed=77)
    b = mm.Batch(specs)
    assert b.num_classes() == len({(s["nx"], s["ny"], s["nz"]) for s in specs})
    tiles = [b.class_info(c) for c in range(b.num_classes())]
    for i, m in enumerate(m0s):
        b.set_m(i, m)
    t_end = 4e-12
    b.run(t_end)
    out = {"specs": specs, "m0s": m0s, "t_end": t_end,
           "m": [b.get_m(i) for i in range(len(specs))],
           "dts": [b.get_dt_history(i) for i in range(len(specs))],
           "stats": [b.get_stats(i) for i in range(len(specs))], "tiles": tiles}
    b.close()
    return out


def test_every_instance_reaches_t_end(batch_run):
    for st in batch_run["stats"]:
        assert st["status"] == 0
        assert st["t"] == batch_run["t_end"]
        assert st["accepted"] >= 1
    # instances take different numbers of steps (their own adaptive dt)
    assert len({st["accepted"] for st in batch_run["stats"]}) > 1


@pytest.mark.parametrize("i", range(0, 16, 3))
def test_instance_vs_oracle_replay(batch_run, i):
    spec, m0 = batch_run["specs"][i], batch_run["m0s"][i]
    p = problem_from_instance(spec, m0)
    ora = RK45(p, m=p.m0.astype(np.float32).astype(np.float64))
    ora.run_fixed(batch_run["dts"][i])
    assert abs(ora.t - batch_run["t_end"]) <= 1e-9 * batch_run["t_end"]
    assert np.abs(batch_run["m"][i].astype(np.float64) - ora.m).max() <= M_TOL


@pytest.mark.parametrize("i", [0, 5, 10])
def test_instance_vs_single_context(mm, batch_run, i):
    spec, m0 = batch_run["specs"][i], batch_run["m0s"][i]
    p = problem_from_instance(spec, m0)
    ctx = mm.Context.from_problem(p)
    ctx.set_fixed_dt_sequence(batch_run["dts"][i])
    ctx.step(len(batch_run["dts"][i]))
    m = ctx.get_m()
    ctx.close()
    # two float32 paths that round in different orders
    assert np.abs(m.astype(np.float64) - batch_run["m"][i].astype(np.float64)).max() <= 5e-6


def test_batch_nonfinite_instance_reports_error(mm):
    specs, m0s = batch_instances(3, shapes=((32, 32, 1),), seed=5)
    b = mm.Batch(specs)
    for i, m in enumerate(m0s):
        mm_ = m.copy()
        if i == 1:
            mm_[0, 0, 3, 3] = np.nan
        b.set_m(i, mm_)
    with pytest.raises(mm.MMError) as ei:
        b.run(1e-12)
    assert ei.value.code == -4
    assert b.get_stats(1)["status"] == -4
    assert b.get_stats(0)["status"] == 0
    b.close()


def test_autotuned_tiles_are_valid(batch_run):
    """The FFT-tile autotuner picks, per shape class, a residue split whose
    class transform still holds the grid (py / cly >= ny, pz / clz >= nz, at
    most 4096 points per block) and an x-row block size among the offered
    ones, and reports the timed convolution; the instances then run with those
    tiles (the parity tests above)."""
    def pad(n):
        return 1 if n == 1 else 1 << (2 * n - 2).bit_length()
    seen = {(s["nx"], s["ny"], s["nz"]): 0 for s in batch_run["specs"]}
    for s in batch_run["specs"]:
        seen[(s["nx"], s["ny"], s["nz"])] += 1
    assert len(batch_run["tiles"]) == len(seen)
    for t in batch_run["tiles"]:
        nx, ny, nz = t["grid"]
        assert seen[(nx, ny, nz)] == t["instances"]
        py, pz = pad(ny), pad(nz)
        assert t["cly"] in (1, 2) and t["clz"] in (1, 2)
        assert py // t["cly"] >= ny and pz // t["clz"] >= nz
        assert (py // t["cly"]) * (pz // t["clz"]) <= 4096
        lx = pad(nx) // 2
        default = 2 if lx >= 512 else (4 if lx >= 256 else 8)
        assert t["xrows"] in (max(default // 2, 1), default, 2 * default)
        assert t["conv_us"] > 0


# The batched workload's own shape classes (128 x 64 x 2 and 96 x 96 x 4, 4 nm
# cells), each run with every residue split its fused plan offers, pinned in
# turn: no split (one block per kx plane), y split, z split (the shared-y
# cluster kernel for 96 x 96 x 4) and both.
C4_SHAPES = ((128, 64, 2), (96, 96, 4))


@pytest.mark.parametrize("split", [(1, 1), (2, 1), (1, 2), (2, 2)])
def test_c4_shape_classes_every_split_vs_oracle(mm, split):
    specs, m0s = batch_instances(4, shapes=C4_SHAPES, seed=91)
    b = mm.Batch(specs)
    assert b.num_classes() == 2
    for c in range(b.num_classes()):
        info = b.class_info(c)
        b.set_tiles(c, split[0], split[1], info["xrows"])
        pinned = b.class_info(c)
        assert (pinned["cly"], pinned["clz"]) == split
    for i, m in enumerate(m0s):
        b.set_m(i, m)
    t_end = 2e-12
    b.run(t_end)
    for i in range(len(specs)):
        st = b.get_stats(i)
        assert st["status"] == 0 and st["t"] == t_end
        p = problem_from_instance(specs[i], m0s[i])
        ora = RK45(p, m=p.m0.astype(np.float32).astype(np.float64))
        ora.run_fixed(b.get_dt_history(i))
        assert np.abs(b.get_m(i).astype(np.float64) - ora.m).max() <= M_TOL
    b.close()


def test_set_tiles_rejects_splits_the_plan_does_not_offer(mm):
    specs, m0s = batch_instances(2, shapes=((32, 32, 1),), seed=3)
    b = mm.Batch(specs)
    info = b.class_info(0)
    with pytest.raises(mm.MMError):
        b.set_tiles(0, 1, 2, info["xrows"])     # a 2-D grid has no z split
    with pytest.raises(mm.MMError):
        b.set_tiles(0, 1, 1, 3)                 # not an offered x-row block size
    b.close()
