"""Zhang-Li and Slonczewski spin-transfer torques on the GPU (C ABI) against
the float64 oracle: torques at random states, replayed step sequences (a
context with spin-transfer torques steps with the general stage kernels, on
the fused convolution layout), and the closed forms the oracle is pinned by
(macrospin Slonczewski, periodic Zhang-Li cycloid).
Tolerances as in test_gpu_parity (torques 5e-6 of their maximum, m 1e-5)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.field import Field  # noqa: E402
from oracle.rk45 import RK45  # noqa: E402
from oracle.stt import E_CHARGE, HBAR, MU_B  # noqa: E402
from paper_1406_7635_gb300.workloads import GAMMA_LL, Problem, normalise  # noqa: E402

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


def stt_problem(shape, cell, seed, mask_frac=0.05, zl=True, sl=True):
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape
    p = Problem(nx, ny, nz, *cell)
    p.region = rng.integers(0, 2, size=shape).astype(np.uint8)
    for r in range(2):
        p.msat[r] = rng.uniform(6e5, 1.0e6)
        p.aex[r] = rng.uniform(1.0e-11, 1.5e-11)
        p.alpha[r] = rng.uniform(0.02, 0.2)
        p.b0[r] = rng.uniform(-0.02, 0.02, 3)
        p.jcur[r] = rng.uniform(-2e12, 2e12, 3)
        p.xi[r] = rng.uniform(0.0, 0.4)
        p.pol[r] = rng.uniform(0.3, 0.7)
        p.lam[r] = rng.uniform(1.0, 2.5)
        p.epsp[r] = rng.uniform(0.0, 1.0)
        v = rng.standard_normal(3)
        p.mp[r] = v / np.linalg.norm(v)
        p.tfree[r] = 2e-9
    p.anis = False
    p.zhang_li, p.slonczewski = zl, sl
    if mask_frac > 0:
        p.mask = (rng.uniform(size=shape) > mask_frac).astype(np.uint8)
    p.m0 = normalise(rng.standard_normal((3,) + shape), p.magnetic())
    return p


@pytest.mark.parametrize("shape,cell,zl,sl", [((3, 10, 13), (2e-9, 2e-9, 1e-9), True, True),
                                              ((1, 20, 24), (1e-9, 1.5e-9, 2e-9), True, False),
                                              ((2, 9, 11), (1e-9, 1e-9, 1e-9), False, True)])
def test_stt_torque_vs_oracle(mm, shape, cell, zl, sl):
    """Exchange and demag off (with random m they dwarf the spin torques);
    the Zhang-Li stencil and the Slonczewski terms against the oracle."""
    p = stt_problem(shape, cell, seed=sum(shape), zl=zl, sl=sl)
    p.exch = p.demag = False
    ctx = mm.Context.from_problem(p)
    tau = ctx.get_torque().astype(np.float64)
    ctx.close()
    m32 = p.m0.astype(np.float32).astype(np.float64)
    to = Field(p).torque(m32, 0.0)
    from oracle.field import ll_torque
    ll = ll_torque(p, m32, Field(p).terms(m32, 0.0)["total"])
    assert np.abs(to - ll).max() > 1e3 * FIELD_TOL * np.abs(to).max()   # the STT part is exercised
    assert np.abs(tau - to).max() <= FIELD_TOL * np.abs(to).max()


@pytest.mark.parametrize("shape,cell,nsteps", [((1, 48, 64), (2e-9, 2e-9, 2e-9), 40),     # 2-D fused layout
                                               ((4, 24, 20), (2e-9, 2e-9, 2e-9), 25)])   # 3-D fused layout
def test_stt_lockstep_vs_oracle(mm, shape, cell, nsteps):
    p = stt_problem(shape, cell, seed=7)
    ctx = mm.Context.from_problem(p)
    ctx.step(nsteps)
    m_gpu = ctx.get_m().astype(np.float64)
    dts = ctx.get_dt_history()
    ctx.close()
    ora = RK45(p, m=p.m0.astype(np.float32).astype(np.float64))
    ora.run_fixed(dts)
    assert np.abs(m_gpu - ora.m).max() <= M_TOL


def test_stt_off_keeps_row_stage_path(mm):
    """Switching the torques on and off again: a context whose torques were
    switched off steps bit-identically to one that never had them (the
    row-stage kernels are back in use)."""
    p = stt_problem((1, 32, 32), (2e-9, 2e-9, 2e-9), seed=11, mask_frac=0.0)
    q = stt_problem((1, 32, 32), (2e-9, 2e-9, 2e-9), seed=11, mask_frac=0.0, zl=False, sl=False)
    a = mm.Context.from_problem(p)
    a.enable_stt(False, False)
    a.step(10)
    b = mm.Context.from_problem(q)
    b.step(10)
    assert np.array_equal(a.get_m(), b.get_m())
    a.close()
    b.close()


def test_slonczewski_macrospin_closed_form_gpu(mm):
    """Lambda = 1, eps' = 0, alpha = 0: tan(theta/2) grows as
    exp(gamma beta (P/2) t) (the oracle's pin), on the GPU to the float32
    floor."""
    p = Problem(1, 1, 1, 2e-9, 2e-9, 2e-9)
    p.msat[0] = 8e5
    p.demag = p.exch = p.anis = p.zeeman = False
    p.slonczewski = True
    p.jcur[0] = (0.0, 0.0, 2e11)
    p.pol[0], p.lam[0], p.tfree[0] = 0.6, 1.0, 2e-9
    p.mp[0] = (0.0, 0.0, 1.0)
    p.m0 = np.array([np.sin(0.7), 0.0, np.cos(0.7)]).reshape(3, 1, 1, 1)
    p.max_err = 1e-7
    beta = 2e11 * HBAR / (8e5 * E_CHARGE * 2e-9)
    ctx = mm.Context.from_problem(p)
    t = 0.2e-9
    ctx.run(t)
    m = ctx.get_m()[:, 0, 0, 0].astype(np.float64)
    ctx.close()
    expect = 2 * np.arctan(np.tan(0.35) * np.exp(GAMMA_LL * beta * 0.3 * t))
    assert abs(np.arccos(np.clip(m[2], -1, 1)) - expect) < 1e-5


def test_zhang_li_periodic_cycloid_gpu(mm):
    """xi = alpha, periodic chain: the cycloid's phase advances at
    u sin(k d)/d (the oracle's pin), on the GPU."""
    n, d, xi, j = 32, 1e-9, 0.1, 1e12
    p = Problem(n, 1, 1, d, d, d)
    p.msat[0], p.alpha[0], p.xi[0] = 8e5, xi, xi
    p.demag = p.exch = p.anis = p.zeeman = False
    p.zhang_li = True
    p.jcur[0] = (j, 0.0, 0.0)
    p.pbc = (1, 1, 1)
    k = 2 * np.pi * 3 / (n * d)
    x = (np.arange(n) + 0.5) * d
    m = np.zeros((3, 1, 1, n))
    m[0, 0, 0] = np.sin(k * x)
    m[2, 0, 0] = np.cos(k * x)
    p.m0 = m
    p.max_err = 1e-7
    u = MU_B * j / (2 * E_CHARGE * 8e5 * (1 + xi * xi))
    ctx = mm.Context.from_problem(p)
    t = 0.3e-9
    ctx.run(t)
    mg = ctx.get_m()[:, 0, 0, :].astype(np.float64)
    ctx.close()
    phi = k * x + u * np.sin(k * d) / d * t
    expect = np.stack([np.sin(phi), np.zeros_like(phi), np.cos(phi)])
    assert np.abs(mg - expect).max() < 1e-5
