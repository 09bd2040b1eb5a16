"""Trajectories against the float64 oracle beyond a single replayed step:

* the 64 x 16 x 1 SP4-like film run freely to 0.5 ns, the GPU and the oracle
  each with its own adaptive Dormand-Prince controller (Sec. IV, MaxErr
  1e-5): <m>(t) compared at 5 ps samples, the final m and the energies;
* energy conservation at alpha = 0 on the same film: the GPU's drift of the
  total energy is at most twice the oracle's own drift + 1e-6 |E|;
* the 128 x 128 x 32 ellipsoid in the benchmark's configuration: 20 adaptive
  steps on the GPU replayed by the oracle with the GPU's step sizes.

Bars: <m> within 1e-3 (free-running, each side its own controller), m within
1e-5 after replayed steps (the spec bar)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.energy import energies  # noqa: E402
from oracle.rk45 import RK45  # noqa: E402
from paper_1406_7635_gb300.workloads import WORKLOADS  # noqa: E402

M_AVG_TOL = 1e-3
M_TOL = 1e-5


@pytest.fixture(scope="module")
def mm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1406_7635_gb300.build import build
    build()
    from paper_1406_7635_gb300 import mm as _mm
    return _mm


def test_free_adaptive_film_to_half_a_nanosecond(mm):
    p = WORKLOADS["film_64x16x1"]()
    mag = p.magnetic()
    ctx = mm.Context.from_problem(p)
    ora = RK45(p, m=p.m0.astype(np.float32).astype(np.float64))
    samples = np.arange(1, 101) * 5e-12
    worst = 0.0
    for t in samples:
        ctx.run(t)
        ora.run(t)
        m_gpu = np.array(ctx.get_energies()["m_avg"])
        m_ora = np.array([ora.m[c][mag].mean() for c in range(3)])
        worst = max(worst, float(np.abs(m_gpu - m_ora).max()))
    assert ctx.get_time()[0] == pytest.approx(0.5e-9, rel=1e-12)
    e_gpu = ctx.get_energies()
    e_ora = energies(p, ora.m, ora.t)
    m_final = float(np.abs(ctx.get_m().astype(np.float64) - ora.m).max())
    e_rel = abs(e_gpu["total"] - e_ora["total"]) / abs(e_ora["total"])
    st = ctx.get_stats()
    print(f"\nfree-adaptive 64x16x1 to 0.5 ns: max |<m>_gpu - <m>_oracle| = {worst:.3e} over 100 samples; "
          f"final max |m_gpu - m_oracle| = {m_final:.3e}; total energy rel. diff {e_rel:.3e}; "
          f"steps GPU {st['accepted']} (+{st['rejected']} rejected), oracle {ora.accepted} (+{ora.rejected})")
    ctx.close()
    assert worst <= M_AVG_TOL
    assert e_rel <= M_AVG_TOL
    for k in ("demag", "exch", "zeeman"):
        assert abs(e_gpu[k] - e_ora[k]) <= M_AVG_TOL * abs(e_ora["total"]), k


def test_energy_drift_at_zero_damping_within_twice_the_oracle(mm):
    p = WORKLOADS["film_64x16x1"]()
    p.alpha[0] = 0.0
    ctx = mm.Context.from_problem(p)
    ora = RK45(p, m=p.m0.astype(np.float32).astype(np.float64))
    e0_gpu = ctx.get_energies()["total"]
    e0_ora = energies(p, ora.m, 0.0, field=ora.field)["total"]
    drift_gpu = drift_ora = 0.0
    for t in np.arange(1, 21) * 5e-12:
        ctx.run(t)
        ora.run(t)
        drift_gpu = max(drift_gpu, abs(ctx.get_energies()["total"] - e0_gpu))
        drift_ora = max(drift_ora, abs(energies(p, ora.m, ora.t, field=ora.field)["total"] - e0_ora))
    ctx.close()
    print(f"\nenergy drift over 0.1 ns at alpha = 0: GPU {drift_gpu:.3e} J, oracle {drift_ora:.3e} J, "
          f"|E| = {abs(e0_ora):.3e} J")
    assert drift_gpu <= 2.0 * drift_ora + 1e-6 * abs(e0_ora)


def test_ellipsoid_twenty_steps_replayed(mm):
    p = WORKLOADS["ellipsoid_128x128x32"]()
    ctx = mm.Context.from_problem(p)
    ctx.step(20)
    m_gpu = ctx.get_m().astype(np.float64)
    dts = ctx.get_dt_history()
    ctx.close()
    assert len(dts) == 20
    ora = RK45(p, m=p.m0.astype(np.float32).astype(np.float64))
    ora.run_fixed(dts)
    err = float(np.abs(m_gpu - ora.m).max())
    print(f"\n128x128x32 ellipsoid, 20 replayed steps: max |m_gpu - m_oracle| = {err:.3e}")
    assert err <= M_TOL


def test_grain_film_twenty_steps_replayed(mm):
    """The 256 x 256 x 1 grain film on its default path (the one-kernel 2-D
    (y, z) part with the row kernel started as its programmatic dependent):
    20 accepted steps replayed by the oracle."""
    p = WORKLOADS["grains_256x256x1"]()
    ctx = mm.Context.from_problem(p)
    ctx.step(20)
    m_gpu = ctx.get_m().astype(np.float64)
    dts = ctx.get_dt_history()
    ctx.close()
    assert len(dts) == 20
    ora = RK45(p, m=p.m0.astype(np.float32).astype(np.float64))
    ora.run_fixed(dts)
    err = float(np.abs(m_gpu - ora.m).max())
    print(f"\n256x256x1 grain film, 20 replayed steps: max |m_gpu - m_oracle| = {err:.3e}")
    assert err <= M_TOL
