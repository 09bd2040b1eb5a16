"""Pins for the oracle's spin-transfer torques (Sec. III, Zhang-Li and
Slonczewski): closed-form macrospin and cycloid dynamics, and the
angle-dependent Slonczewski efficiency against scipy's ODE solver."""
import numpy as np
import pytest

from oracle.rk45 import RK45
from oracle.stt import E_CHARGE, HBAR, MU_B, stt_torque
from paper_1406_7635_gb300.workloads import GAMMA_LL, Problem


def macrospin(jz=2e11, P=0.6, lam=1.0, epsp=0.0, alpha=0.0, theta0=0.7):
    p = Problem(1, 1, 1, 2e-9, 2e-9, 2e-9)
    p.msat[0], p.alpha[0] = 8e5, alpha
    p.demag = p.exch = p.anis = p.zeeman = False
    p.slonczewski = True
    p.jcur[0] = (0.0, 0.0, jz)
    p.pol[0], p.lam[0], p.epsp[0], p.tfree[0] = P, lam, epsp, 2e-9
    p.mp[0] = (0.0, 0.0, 1.0)
    p.m0 = np.array([np.sin(theta0), 0.0, np.cos(theta0)]).reshape(3, 1, 1, 1)
    p.max_err = 1e-9
    beta = jz * HBAR / (8e5 * E_CHARGE * 2e-9)
    return p, beta


def theta_of(m):
    return np.arccos(np.clip(m[2, 0, 0, 0], -1, 1))


def test_slonczewski_damping_like_closed_form():
    """Lambda = 1 (eps = P/2), eps' = 0, alpha = 0, m_P = z: dm/dt =
    -gamma beta eps (m_P - (m.m_P) m), so the polar angle obeys
    d theta/dt = gamma beta eps sin(theta): tan(theta/2) grows as
    exp(gamma beta eps t)."""
    p, beta = macrospin()
    s = RK45(p)
    rate = GAMMA_LL * beta * 0.3
    for t in (0.05e-9, 0.1e-9, 0.2e-9):
        s.run(t)
        expect = 2 * np.arctan(np.tan(0.35) * np.exp(rate * t))
        assert abs(theta_of(s.m) - expect) < 1e-6, (t, theta_of(s.m), expect)
    assert abs(s.m[1, 0, 0, 0]) < 1e-9   # no azimuthal motion


def test_slonczewski_field_like_precession():
    """P = 0 (eps = 0), eps' != 0, alpha = 0: dm/dt = gamma beta eps' m x m_P,
    a rotation about m_P = z by -gamma beta eps' t at fixed polar angle."""
    p, beta = macrospin(P=0.0, epsp=0.8)
    s = RK45(p)
    w = GAMMA_LL * beta * 0.8
    t = 0.2e-9
    s.run(t)
    m = s.m[:, 0, 0, 0]
    phi = np.arctan2(m[1], m[0])
    expect = np.angle(np.exp(-1j * w * t))
    assert abs(np.angle(np.exp(1j * (phi - expect)))) < 1e-6
    assert abs(theta_of(s.m) - 0.7) < 1e-9


def test_slonczewski_angle_dependence_vs_scipy():
    """Lambda = 2: eps depends on m.m_P, and d theta/dt = gamma beta
    eps(cos theta) sin(theta); scipy's solve_ivp integrates that 1-D law."""
    solve_ivp = pytest.importorskip("scipy.integrate").solve_ivp
    p, beta = macrospin(lam=2.0, theta0=0.5)
    s = RK45(p)
    lam2 = 4.0

    def rhs(t, th):
        eps = 0.6 * lam2 / ((lam2 + 1) + (lam2 - 1) * np.cos(th[0]))
        return [GAMMA_LL * beta * eps * np.sin(th[0])]
    t_end = 0.15e-9
    ref = solve_ivp(rhs, (0, t_end), [0.5], rtol=1e-11, atol=1e-13).y[0, -1]
    s.run(t_end)
    assert abs(theta_of(s.m) - ref) < 1e-6


def cycloid_problem(n=32, d=1e-9, xi=0.1, alpha=0.1, j=1e12, k_per=3):
    p = Problem(n, 1, 1, d, d, d)
    p.msat[0], p.alpha[0], p.xi[0] = 8e5, alpha, xi
    p.demag = p.exch = p.anis = p.zeeman = False
    p.zhang_li = True
    p.jcur[0] = (j, 0.0, 0.0)
    p.pbc = (1, 1, 1)
    k = 2 * np.pi * k_per / (n * d)
    x = (np.arange(n) + 0.5) * d
    m = np.zeros((3, 1, 1, n))
    m[0, 0, 0] = np.sin(k * x)
    m[2, 0, 0] = np.cos(k * x)
    p.m0 = m
    u = MU_B * j / (2 * E_CHARGE * 8e5 * (1 + xi * xi))
    return p, k, x, u


def test_zhang_li_adiabatic_cycloid_advection():
    """xi = alpha: dm/dt = -m x (m x h) = h for the cycloid (h is
    perpendicular to m), so on a periodic chain the cycloid's phase advances
    uniformly at u sin(k d)/d: m = (sin phi, 0, cos phi), phi = k x + u
    (sin(k d)/d) t -- the texture moves opposite to j."""
    p, k, x, u = cycloid_problem(xi=0.1, alpha=0.1)
    p.max_err = 1e-9
    s = RK45(p)
    t = 0.3e-9
    s.run(t)
    phi = k * x + u * np.sin(k * p.dx) / p.dx * t
    expect = np.stack([np.sin(phi), np.zeros_like(phi), np.cos(phi)])
    assert np.abs(s.m[:, 0, 0, :] - expect).max() < 1e-6


def test_zhang_li_non_adiabatic_initial_rate():
    """xi != alpha, the same cycloid at t = 0: m x dm/dphi = y, so
    dm/dt = (1 + xi alpha)/(1 + alpha^2) h - (xi - alpha)/(1 + alpha^2)
    u (sin(k d)/d) y in every cell."""
    xi, alpha = 0.3, 0.05
    p, k, x, u = cycloid_problem(xi=xi, alpha=alpha)
    tq = stt_torque(p, p.m0)
    f = u * np.sin(k * p.dx) / p.dx
    h = f * np.stack([np.cos(k * x), np.zeros_like(x), -np.sin(k * x)])
    expect = (1 + xi * alpha) / (1 + alpha ** 2) * h
    expect[1] -= (xi - alpha) / (1 + alpha ** 2) * f
    assert np.abs(tq[:, 0, 0, :] - expect).max() < 1e-12 * np.abs(expect).max()
