"""mm_demag_field_noalloc: the demag field for callers that cannot allocate
device memory (frameworks whose GPU memory all comes from their own pool,
applications that forbid device allocation after start-up).  It keeps its
scratch in a static device array; its field must match the context path
(mm_demag_apply) on the same magnetisation, on two calls in a row."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FIELD_TOL = 5e-6   # same float32 tolerance as the other field comparisons


@pytest.fixture(scope="module")
def mm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1406_7635_gb300.build import build
    build()
    from paper_1406_7635_gb300 import mm as _mm
    return _mm


@pytest.mark.parametrize("shape,cell", [
    ((1, 48, 64), (2e-9, 2e-9, 1e-9)),
    ((6, 20, 24), (3e-9, 3e-9, 3e-9)),
    ((3, 1, 7), (1e-9, 2e-9, 0.5e-9)),
    ((1, 1, 1), (1e-9, 1e-9, 1e-9)),
])
def test_noalloc_matches_context_path(mm, shape, cell):
    nz, ny, nx = shape
    rng = np.random.default_rng(nx * 131 + ny * 7 + nz)
    M = (8e5 * rng.standard_normal((3,) + shape)).astype(np.float32)
    Md = torch.tensor(M, device="cuda").contiguous()
    ctx = mm.Context(nx, ny, nz, *cell)
    ctx.set_material(0, msat=1.0, aex=0.0, alpha=0.0)   # Msat = 1 A/m: the context convolves M itself
    Bref = torch.empty_like(Md)
    ctx.demag_apply(Md, Bref)
    ref = Bref.cpu().numpy().astype(np.float64)
    ctx.close()
    scale = np.abs(ref).max()
    for _ in range(2):
        B = torch.full_like(Md, float("nan"))
        mm.demag_field_noalloc(Md, B, nx, ny, nz, *cell)
        torch.cuda.synchronize()
        out = B.cpu().numpy().astype(np.float64)
        assert np.isfinite(out).all()
        assert np.abs(out - ref).max() <= FIELD_TOL * scale


def test_noalloc_rejects_grids_beyond_its_scratch(mm):
    Md = torch.zeros(3 * 8, device="cuda")
    Bd = torch.zeros_like(Md)
    with pytest.raises(mm.MMError) as ei:
        mm.demag_field_noalloc(Md, Bd, 1024, 512, 1, 1e-9, 1e-9, 1e-9)
    assert ei.value.code == -1 and "scratch" in str(ei.value)
