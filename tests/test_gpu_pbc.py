"""Periodic boundary conditions on the GPU (C ABI) against the float64 oracle
(whose PBC demag is pinned by Tables tabPBC1/tabPBC2 and brute-force image
sums): the macro-geometry convolution on the general and fused paths, the
wrapped exchange and DMI stencils, and replayed step sequences (general stage
kernels for periodic x, row-stage kernels with wrapped halo rows for
periodic y and z).  Tolerances as in test_gpu_parity."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.demag import demag_fft  # noqa: E402
from oracle.energy import energies as ora_energies  # noqa: E402
from oracle.field import Field, ll_torque  # noqa: E402
from oracle.rk45 import RK45  # noqa: E402
from paper_1406_7635_gb300.workloads import Problem, normalise  # noqa: E402

FIELD_TOL = 5e-6
M_TOL = 1e-5


@pytest.fixture(scope="module")
def mm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1406_7635_gb300.build import build
    build()
    from paper_1406_7635_gb300 import mm as _mm
    return _mm


def pbc_problem(shape, cell, pbc, seed, mask_frac=0.0, dmi=False):
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape
    p = Problem(nx, ny, nz, *cell)
    p.pbc = pbc
    p.region = rng.integers(0, 2, size=shape).astype(np.uint8)
    for r in range(2):
        p.msat[r] = rng.uniform(6e5, 1.1e6)
        p.aex[r] = rng.uniform(1.0e-11, 1.8e-11)
        p.alpha[r] = rng.uniform(0.05, 0.3)
        p.ku1[r] = rng.uniform(-1e5, 3e5)
        u = rng.standard_normal(3)
        p.anis_u[r] = u / np.linalg.norm(u)
        p.b0[r] = rng.uniform(-0.03, 0.03, 3)
        if dmi:
            p.dind[r] = rng.uniform(-2e-3, 2e-3)
    if mask_frac > 0:
        p.mask = (rng.uniform(size=shape) > mask_frac).astype(np.uint8)
    p.m0 = normalise(rng.standard_normal((3,) + shape), p.magnetic())
    return p


PBC_GRIDS = [
    ((1, 16, 8), (2e-9, 2e-9, 1e-9), (2, 0, 0)),      # general path, periodic x
    ((2, 8, 16), (1e-9, 1e-9, 1e-9), (3, 2, 0)),      # general path, periodic x and y
    ((1, 24, 64), (1e-9, 1e-9, 1e-9), (3, 0, 0)),     # fused path, periodic x (no padding)
    ((4, 32, 20), (2e-9, 2e-9, 1e-9), (0, 2, 0)),     # fused path, periodic y
    ((8, 16, 40), (1e-9, 1e-9, 1e-9), (0, 0, 2)),     # fused path, periodic z
    ((4, 1, 32), (1e-9, 2e-9, 1e-9), (1, 3, 0)),      # a periodic axis of one cell
]


@pytest.mark.parametrize("shape,cell,pbc", PBC_GRIDS)
def test_pbc_demag_vs_oracle(mm, shape, cell, pbc):
    p = pbc_problem(shape, cell, pbc, seed=sum(shape) + sum(pbc), mask_frac=0.1)
    ctx = mm.Context.from_problem(p)
    b_gpu = ctx.get_bdemag().astype(np.float64)
    ctx.close()
    msat = np.where(p.magnetic(), p.msat[p.region], 0.0)
    m32 = p.m0.astype(np.float32).astype(np.float64)
    b_ora = demag_fft(msat[None] * m32, *cell, pbc=pbc)
    assert np.abs(b_gpu - b_ora).max() <= FIELD_TOL * np.abs(b_ora).max()


@pytest.mark.parametrize("shape,cell,pbc", [((2, 8, 16), (1e-9, 1e-9, 1e-9), (3, 2, 0)),
                                            ((4, 32, 20), (2e-9, 2e-9, 1e-9), (0, 2, 1))])
def test_pbc_fields_torque_energy_vs_oracle(mm, shape, cell, pbc):
    """Exchange and DMI wrap around the periodic axes (no ghosts there)."""
    p = pbc_problem(shape, cell, pbc, seed=5, mask_frac=0.05, dmi=True)
    ctx = mm.Context.from_problem(p)
    B = ctx.get_beff().astype(np.float64)
    tau = ctx.get_torque().astype(np.float64)
    e = ctx.get_energies()
    ctx.close()
    m32 = p.m0.astype(np.float32).astype(np.float64)
    f = Field(p)
    Bo = f.terms(m32, 0.0)["total"]
    to = ll_torque(p, m32, Bo)
    assert np.abs(B - Bo).max() <= FIELD_TOL * np.abs(Bo).max()
    assert np.abs(tau - to).max() <= FIELD_TOL * np.abs(to).max()
    eo = ora_energies(p, m32, 0.0, f)
    scale = max(abs(eo[k]) for k in ("demag", "exch", "anis", "zeeman", "dmi"))
    for k in ("demag", "exch", "anis", "zeeman", "dmi", "total"):
        assert abs(e[k] - eo[k]) <= 1e-5 * scale, (k, e[k], eo[k])


@pytest.mark.parametrize("shape,cell,pbc,nsteps", [
    ((1, 32, 64), (2e-9, 2e-9, 1e-9), (4, 4, 0), 40),    # periodic x: general stage kernels
    ((4, 32, 40), (2e-9, 2e-9, 2e-9), (0, 3, 2), 15),    # periodic y, z: row-stage kernels, wrapped halos
])
def test_pbc_lockstep_vs_oracle(mm, shape, cell, pbc, nsteps):
    p = pbc_problem(shape, cell, pbc, seed=2, mask_frac=0.05, dmi=True)
    ctx = mm.Context.from_problem(p)
    ctx.step(nsteps)
    m_gpu = ctx.get_m().astype(np.float64)
    dts = ctx.get_dt_history()
    ctx.close()
    ora = RK45(p, m=p.m0.astype(np.float32).astype(np.float64))
    ora.run_fixed(dts)
    assert np.abs(m_gpu - ora.m).max() <= M_TOL


def test_pbc_argument_errors(mm):
    ctx = mm.Context(12, 8, 1, 1e-9, 1e-9, 1e-9)
    with pytest.raises(mm.MMError):
        ctx.set_pbc(1, 0, 0)          # 12 cells: not a power of two
    with pytest.raises(mm.MMError):
        ctx.set_pbc(0, -1, 0)
    ctx.set_pbc(0, 2, 5)              # 8 cells along y, 1 along z: allowed
    ctx.close()
