"""Interfacial DMI with the Rohart boundary conditions on the GPU (C ABI)
against the float64 oracle: fields, torques and energies (general stage
kernels, getters) and replayed step sequences (the fused row-stage kernels
in 2-D and 3-D).  Tolerances as in test_gpu_parity: fields 5e-6 of their
maximum, m after a replayed sequence 1e-5, energies 1e-5 of the largest term."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

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


def dmi_problem(shape, cell, seed, regions=2, mask_frac=0.0, exch=True):
    """Co/Pt-like perpendicular films (Msat ~ 1.1e6, Aex ~ 1.6e-11, Ku1 ~
    1.3e6 along z, D of either sign), random m, optional vacuum holes (whose
    edges use the ghost values too)."""
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape
    p = Problem(nx, ny, nz, *cell)
    p.region = rng.integers(0, regions, size=shape).astype(np.uint8)
    for r in range(regions):
        p.msat[r] = rng.uniform(0.9e6, 1.2e6)
        p.aex[r] = rng.uniform(1.2e-11, 2e-11)
        p.alpha[r] = rng.uniform(0.1, 0.4)
        p.ku1[r] = rng.uniform(0.8e6, 1.3e6)
        p.anis_u[r] = (0.0, 0.0, 1.0)
        p.dind[r] = rng.uniform(-3e-3, 3e-3)
        p.b0[r] = rng.uniform(-0.05, 0.05, 3)
    p.exch = exch
    if mask_frac > 0:
        p.mask = (rng.uniform(size=shape) > mask_frac).astype(np.uint8)
    m = rng.standard_normal((3,) + shape)
    p.m0 = normalise(m, p.magnetic())
    return p


@pytest.mark.parametrize("shape,cell,mask,exch", [
    ((1, 20, 33), (1e-9, 1e-9, 0.6e-9), 0.0, True),
    ((1, 24, 40), (1.5e-9, 1e-9, 1e-9), 0.2, True),
    ((3, 10, 13), (2e-9, 2e-9, 1e-9), 0.15, True),
    ((1, 16, 16), (1e-9, 1e-9, 1e-9), 0.0, False),     # DMI without Heisenberg exchange
])
def test_dmi_fields_vs_oracle(mm, shape, cell, mask, exch):
    p = dmi_problem(shape, cell, seed=11 + shape[2], mask_frac=mask, exch=exch)
    ctx = mm.Context.from_problem(p)
    B = ctx.get_beff().astype(np.float64)
    tau = ctx.get_torque().astype(np.float64)
    e = ctx.get_energies()
    ctx.close()
    m32 = p.m0.astype(np.float32).astype(np.float64)
    f = Field(p)
    terms = f.terms(m32, 0.0)
    Bo = terms["total"]
    to = ll_torque(p, m32, Bo)
    # the DMI field is far above the comparison tolerance (the term is exercised)
    assert np.abs(terms["dmi"]).max() > 1e3 * FIELD_TOL * np.abs(Bo).max()
    assert np.abs(B - Bo).max() <= FIELD_TOL * np.abs(Bo).max()
    assert np.abs(tau - to).max() <= FIELD_TOL * np.abs(to).max()
    eo = ora_energies(p, m32, 0.0, f)
    scale = max(abs(eo[k]) for k in ("demag", "exch", "anis", "zeeman", "dmi"))
    for k in ("demag", "exch", "anis", "zeeman", "dmi", "total"):
        assert abs(e[k] - eo[k]) <= 1e-5 * scale, (k, e[k], eo[k])
    assert abs(e["dmi"] - eo["dmi"]) <= 1e-4 * abs(eo["dmi"])


@pytest.mark.parametrize("shape,cell,nsteps", [
    ((1, 48, 64), (1e-9, 1e-9, 0.6e-9), 60),      # 2-D fused path, row-stage kernels
    ((4, 32, 32), (1e-9, 1e-9, 1e-9), 25),        # 3-D fused path
])
def test_dmi_lockstep_vs_oracle(mm, shape, cell, nsteps):
    """GPU adaptive RK45 with DMI for n steps; the oracle replays the accepted
    step sizes; m agrees to 1e-5."""
    p = dmi_problem(shape, cell, seed=3, regions=2, mask_frac=0.05)
    ctx = mm.Context.from_problem(p)
    ctx.step(nsteps)
    m_gpu = ctx.get_m().astype(np.float64)
    dts = ctx.get_dt_history()
    ctx.close()
    ora = RK45(p, m=p.m0.astype(np.float32).astype(np.float64))
    ora.run_fixed(dts)
    assert np.abs(m_gpu - ora.m).max() <= M_TOL


def test_dmi_off_leaves_path_unchanged(mm):
    """Setting D back to zero switches the DMI term off: the trajectory is
    bit-identical to a context that never had DMI."""
    p = dmi_problem((1, 32, 32), (1e-9, 1e-9, 1e-9), seed=8, regions=1)
    q = dmi_problem((1, 32, 32), (1e-9, 1e-9, 1e-9), seed=8, regions=1)
    q.dind[0] = 0.0
    a = mm.Context.from_problem(p)
    a.set_material(0, p.msat[0], p.aex[0], p.alpha[0], p.gamma[0], p.ku1[0], p.ku2[0], p.anis_u[0], 0.0)
    a.step(10)
    b = mm.Context.from_problem(q)
    b.step(10)
    assert np.array_equal(a.get_m(), b.get_m())
    a.close()
    b.close()
