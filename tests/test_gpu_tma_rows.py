"""The row-stage kernels' tensor-copy (TMA) path against the float64 oracle:
replayed RK45 step sequences on grids that take it (rows of 32 and of 128
cells, 8 per block, with a ragged last block, nx below the row length and a
periodic z axis) and on grids that fall back to the asynchronous-copy path
(odd ny, periodic y).
Tolerance as in test_gpu_parity (m 1e-5)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.rk45 import RK45  # noqa: E402
from paper_1406_7635_gb300.workloads import Problem, normalise  # noqa: E402

M_TOL = 1e-5


@pytest.fixture(scope="module")
def mm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1406_7635_gb300.build import build
    build()
    from paper_1406_7635_gb300 import mm as _mm
    return _mm


def rows_problem(shape, cell, pbc, seed):
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape
    p = Problem(nx, ny, nz, *cell)
    p.pbc = pbc
    p.region = rng.integers(0, 3, size=shape).astype(np.uint8)
    for r in range(3):
        p.msat[r] = rng.uniform(6e5, 1.1e6)
        p.aex[r] = rng.uniform(1.0e-11, 1.6e-11)
        p.alpha[r] = rng.uniform(0.05, 0.3)
        p.ku1[r] = rng.uniform(-1e5, 3e5)
        u = rng.standard_normal(3)
        p.anis_u[r] = u / np.linalg.norm(u)
        p.b0[r] = rng.uniform(-0.03, 0.03, 3)
    p.mask = (rng.uniform(size=shape) > 0.05).astype(np.uint8)
    p.m0 = normalise(rng.standard_normal((3,) + shape), p.magnetic())
    return p


@pytest.mark.parametrize("shape,pbc,nsteps", [
    ((4, 30, 20), (0, 0, 0), 12),     # rows 32, 8 per block: last block ragged, nx < 32
    ((4, 30, 20), (0, 0, 2), 12),     # the same with a periodic z (wrapped neighbour planes)
    ((32, 78, 68), (0, 0, 0), 2),     # rows 128, 8 per block: ragged last block, nx < 128
    ((4, 29, 20), (0, 0, 0), 12),     # odd ny: asynchronous-copy path
    ((4, 32, 20), (0, 2, 0), 12),     # periodic y: asynchronous-copy path
])
def test_row_kernels_vs_oracle(mm, shape, pbc, nsteps):
    p = rows_problem(shape, (2e-9, 2e-9, 2e-9), pbc, seed=sum(shape) + sum(pbc))
    ctx = mm.Context.from_problem(p)
    ctx.step(nsteps)
    m_gpu = ctx.get_m().astype(np.float64)
    dts = ctx.get_dt_history()
    ctx.close()
    ora = RK45(p, m=p.m0.astype(np.float32).astype(np.float64))
    ora.run_fixed(dts)
    assert np.abs(m_gpu - ora.m).max() <= M_TOL
