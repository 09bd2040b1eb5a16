"""mm_demag_field_noalloc: the demag field for callers that cannot allocate
device memory (frameworks whose GPU memory all comes from their own pool,
applications that forbid device allocation after start-up).  It keeps its
scratch in a static device array.  Its field must match the float64 oracle's
FFT convolution (Sec. III.B) and the context path (mm_demag_apply) on the same
magnetisation, on two calls in a row; grids beyond the array are rejected
before any device call.

This file is collected last, so that a run stopping at the first failure has
run every other test before it."""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")

FIELD_TOL = 5e-6   # same float32 tolerance as the other field comparisons


@pytest.fixture(scope="module")
def mm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1406_7635_gb300.build import build
    build()
    from paper_1406_7635_gb300 import mm as _mm
    return _mm


def _context_field(mm, Md, shape, cell):
    nz, ny, nx = shape
    ctx = mm.Context(nx, ny, nz, *cell)
    ctx.set_material(0, msat=1.0, aex=0.0, alpha=0.0)   # Msat = 1 A/m: the context convolves M itself
    Bref = torch.empty_like(Md)
    ctx.demag_apply(Md, Bref)
    ref = Bref.cpu().numpy().astype(np.float64)
    ctx.close()
    return ref


@pytest.mark.gpu
@pytest.mark.parametrize("shape,cell", [
    ((1, 48, 64), (2e-9, 2e-9, 1e-9)),
    ((6, 20, 24), (3e-9, 3e-9, 3e-9)),
    ((3, 1, 7), (1e-9, 2e-9, 0.5e-9)),
    ((1, 1, 1), (1e-9, 1e-9, 1e-9)),
])
def test_noalloc_matches_oracle_and_context_path(mm, shape, cell):
    from oracle.demag import demag_fft
    nz, ny, nx = shape
    rng = np.random.default_rng(nx * 131 + ny * 7 + nz)
    M = (8e5 * rng.standard_normal((3,) + shape)).astype(np.float32)
    Md = torch.tensor(M, device="cuda").contiguous()
    ref = _context_field(mm, Md, shape, cell)
    ora = demag_fft(M.astype(np.float64), *cell)
    scale = np.abs(ora).max()
    for _ in range(2):
        B = torch.full_like(Md, float("nan"))
        mm.demag_field_noalloc(Md, B, nx, ny, nz, *cell)
        torch.cuda.synchronize()
        out = B.cpu().numpy().astype(np.float64)
        assert np.isfinite(out).all()
        assert np.abs(out - ora).max() <= FIELD_TOL * scale
        assert np.abs(out - ref).max() <= FIELD_TOL * scale


@pytest.mark.gpu
@pytest.mark.parametrize("fits,too_large", [((1, 256, 512), (1, 257, 512)), ((32, 64, 64), (33, 64, 64))])
def test_noalloc_largest_fitting_grid_runs_next_size_is_rejected(mm, fits, too_large):
    cell = (2e-9, 2e-9, 2e-9)
    nz, ny, nx = fits
    rng = np.random.default_rng(nx + ny + nz)
    M = (8e5 * rng.standard_normal((3,) + fits)).astype(np.float32)
    Md = torch.tensor(M, device="cuda").contiguous()
    ref = _context_field(mm, Md, fits, cell)
    scale = np.abs(ref).max()
    for _ in range(2):
        B = torch.full_like(Md, float("nan"))
        mm.demag_field_noalloc(Md, B, nx, ny, nz, *cell)
        torch.cuda.synchronize()
        assert np.abs(B.cpu().numpy().astype(np.float64) - ref).max() <= FIELD_TOL * scale
    nz, ny, nx = too_large
    Md2 = torch.zeros(3 * nx * ny * nz, device="cuda")
    with pytest.raises(mm.MMError) as ei:
        mm.demag_field_noalloc(Md2, torch.zeros_like(Md2), nx, ny, nz, *cell)
    assert ei.value.code == -1 and "scratch" in str(ei.value)


@pytest.mark.parametrize("shape", [(512, 512, 1), (1024, 256, 1), (512, 257, 1), (128, 64, 32),
                                   (128, 128, 16), (64, 64, 33)])
def test_noalloc_size_check_comes_before_any_device_call(shape):
    """Grids beyond the static array are rejected from the sizes alone: the
    check runs before the entry point touches the device, so it is safe with
    placeholder pointers and on a machine without a GPU."""
    from paper_1406_7635_gb300.build import build
    build()
    from paper_1406_7635_gb300 import mm as _mm
    nx, ny, nz = shape
    dummy = C.c_void_p(16)   # never dereferenced: the call returns before any device work
    rc = _mm.mm_demag_field_noalloc(nx, ny, nz, 1e-9, 1e-9, 1e-9, dummy, dummy, None)
    assert rc == -1
    msg = _mm.mm_last_error().decode()
    assert "scratch" in msg and f"{nx}x{ny}x{nz}" in msg
