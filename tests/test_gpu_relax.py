"""RK23 and relax() on the GPU (C ABI) against the float64 oracle.

Tolerances: m after a replayed RK23 step sequence 1e-5 (the RK45 lockstep
bar); relaxed states 1e-3 (each side stops at its own noise floor, the
oracle's in float64, the GPU's in float32); the maximum-torque getter agrees
with the maximum over the torque array to float32 rounding."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.relax import RK23, relax as ora_relax  # noqa: E402
from paper_1406_7635_gb300.workloads import GAMMA_LL, Problem, ellipsoid_vortex, film_sp4  # noqa: E402

M_TOL = 1e-5
RELAX_TOL = 1e-3


@pytest.fixture(scope="module")
def mm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1406_7635_gb300.build import build
    build()
    from paper_1406_7635_gb300 import mm as _mm
    return _mm


@pytest.mark.parametrize("which,nsteps", [("film", 150), ("ellipsoid", 20)])
def test_rk23_lockstep_vs_oracle(mm, which, nsteps):
    """Adaptive RK23 on the GPU, then the oracle's RK23 replays exactly the
    accepted step sizes: m agrees to 1e-5.  The ellipsoid runs the general
    stage kernels on the fused convolution layout."""
    p = film_sp4(64, 16) if which == "film" else ellipsoid_vortex(16, 16, 4, c=3e-9)
    ctx = mm.Context.from_problem(p)
    ctx.set_integrator("rk23")
    assert ctx.get_integrator() == mm.MM_RK23
    ctx.step(nsteps)
    st = ctx.get_stats()
    assert st["evals"] == 3 * (st["accepted"] + st["rejected"])     # new evaluations per attempt
    m_gpu = ctx.get_m().astype(np.float64)
    dts = ctx.get_dt_history()
    ctx.close()
    ora = RK23(p, m=p.m0.astype(np.float32).astype(np.float64))
    ora.run_fixed(dts)
    assert np.abs(m_gpu - ora.m).max() <= M_TOL


def test_rk23_third_order_on_gpu(mm):
    """One undamped precession period in 0.1 T with fixed steps: the float32
    path shows the third-order slope above its rounding floor."""
    p = Problem(1, 1, 1, 1e-9, 1e-9, 1e-9)
    p.msat[0] = 1.0 / (4e-7 * np.pi)
    p.b0[0] = (0.0, 0.0, 0.1)
    p.demag = p.exch = p.anis = False
    p.m0 = (np.array([1.0, 0.0, 1.0]) / np.sqrt(2)).reshape(3, 1, 1, 1)
    T = 2 * np.pi / (GAMMA_LL * 0.1)
    ns = np.array([8, 12, 16, 24])
    errs = []
    for n in ns:
        ctx = mm.Context.from_problem(p)
        ctx.set_integrator("rk23")
        ctx.set_fixed_dt_sequence(np.full(n, T / n))
        ctx.step(n)
        errs.append(np.linalg.norm(ctx.get_m()[:, 0, 0, 0] - p.m0[:, 0, 0, 0]))
        ctx.close()
    slope = -np.polyfit(np.log(ns), np.log(errs), 1)[0]
    assert abs(slope - 3.0) < 0.3, (slope, errs)


def test_max_torque_getter(mm):
    p = film_sp4(32, 8)
    ctx = mm.Context.from_problem(p)
    ctx.step(3)
    tq = ctx.get_torque().astype(np.float64)
    ref = np.sqrt((tq * tq).sum(axis=0)).max()
    assert abs(ctx.get_max_torque() - ref) <= 1e-6 * ref
    ctx.close()


def test_relax_stoner_wohlfarth_gpu(mm):
    """One cell, easy axis x, B = 0.5 T along z: relaxed m_z = Msat B/(2 Ku1)."""
    p = Problem(1, 1, 1, 2e-9, 2e-9, 2e-9)
    p.msat[0], p.aex[0], p.alpha[0] = 8e5, 1.3e-11, 0.5
    p.ku1[0] = 5e5
    p.b0[0] = (0.0, 0.0, 0.5)
    p.m0 = np.array([0.8, 0.6, 0.0]).reshape(3, 1, 1, 1)
    ctx = mm.Context.from_problem(p)
    n = ctx.relax()
    assert n > 0
    m = ctx.get_m()[:, 0, 0, 0].astype(np.float64)
    sz = 8e5 * 0.5 / (2 * 5e5)
    assert abs(m[2] - sz) < 1e-5 and abs(m[1]) < 1e-5
    # integrator and precession restored: ordinary RK45 stepping continues
    assert ctx.get_integrator() == mm.MM_RK45
    ctx.step(2)
    ctx.close()


@pytest.mark.parametrize("b", [(10e-3, 20e-3, 0.0), (-24.6e-3, 4.3e-3, 0.0)])
def test_relaxed_state_vs_oracle(mm, b):
    """Relaxed-state parity: the 32 x 8 SP4-like film
    (alpha 1) relaxed by relax() on the GPU and by the oracle agree to 1e-3
    in every cell."""
    p = film_sp4(32, 8)
    p.alpha[0] = 1.0
    p.b0[0] = b
    ctx = mm.Context.from_problem(p)
    n_gpu = ctx.relax()
    m_gpu = ctx.get_m().astype(np.float64)
    e_gpu = ctx.get_energies()["total"]
    ctx.close()
    s, log = ora_relax(p, m=p.m0.astype(np.float32).astype(np.float64))
    err = np.abs(m_gpu - s.m).max()
    assert err <= RELAX_TOL, (err, n_gpu, s.accepted)
    from oracle.energy import energies
    e_ora = energies(p, s.m, s.t, s.field)["total"]
    assert abs(e_gpu - e_ora) <= 1e-4 * abs(e_ora)


def test_relax_step_limit_and_state_errors(mm):
    p = film_sp4(32, 8)
    p.alpha[0] = 1.0
    ctx = mm.Context.from_problem(p)
    with pytest.raises(mm.MMError) as ei:
        ctx.relax(max_steps=5)
    assert ei.value.code == -6
    # settings restored after the failed call
    assert ctx.get_integrator() == mm.MM_RK45
    ctx.set_fixed_dt_sequence(np.full(3, 1e-13))
    with pytest.raises(mm.MMError):
        ctx.relax()
    ctx.close()
