"""Pins for the oracle's Dormand-Prince integrator and controller (Sec. IV)."""
from fractions import Fraction as F

import numpy as np
import pytest

from oracle.energy import energies
from oracle.rk45 import A, B4, B5, C, RK45
from paper_1406_7635_gb300.workloads import GAMMA_LL, Problem, film_sp4


def _sums(b):
    """Butcher order conditions (rooted trees up to order 5): (lhs, rhs)."""
    s = len(b)
    a = [[A[i][j] if j < len(A[i]) else F(0) for j in range(s)] for i in range(s)]
    c = C
    ac = [sum(a[i][j] * c[j] for j in range(s)) for i in range(s)]
    ac2 = [sum(a[i][j] * c[j] ** 2 for j in range(s)) for i in range(s)]
    ac3 = [sum(a[i][j] * c[j] ** 3 for j in range(s)) for i in range(s)]
    aac = [sum(a[i][j] * ac[j] for j in range(s)) for i in range(s)]
    aac2 = [sum(a[i][j] * ac2[j] for j in range(s)) for i in range(s)]
    acac = [sum(a[i][j] * c[j] * ac[j] for j in range(s)) for i in range(s)]
    aaac = [sum(a[i][j] * aac[j] for j in range(s)) for i in range(s)]
    S = lambda v: sum(b[i] * v[i] for i in range(s))
    one = [F(1)] * s
    cond = {
        1: [(S(one), F(1))],
        2: [(S(c), F(1, 2))],
        3: [(S([x ** 2 for x in c]), F(1, 3)), (S(ac), F(1, 6))],
        4: [(S([x ** 3 for x in c]), F(1, 4)), (S([c[i] * ac[i] for i in range(s)]), F(1, 8)),
            (S(ac2), F(1, 12)), (S(aac), F(1, 24))],
        5: [(S([x ** 4 for x in c]), F(1, 5)), (S([c[i] ** 2 * ac[i] for i in range(s)]), F(1, 10)),
            (S([ac[i] ** 2 for i in range(s)]), F(1, 20)), (S([c[i] * ac2[i] for i in range(s)]), F(1, 15)),
            (S(ac3), F(1, 20)), (S([c[i] * aac[i] for i in range(s)]), F(1, 30)),
            (S(acac), F(1, 40)), (S(aac2), F(1, 60)), (S(aaac), F(1, 120))],
    }
    return cond


def test_tableau_order_conditions():
    """The tableau must satisfy every order condition up to 5 for the
    propagating weights and up to 4 for the embedded ones, with the row-sum
    condition c_i = sum_j a_ij; exact rational arithmetic."""
    for i in range(7):
        assert sum(A[i]) == C[i]
    for order, conds in _sums(B5).items():
        for lhs, rhs in conds:
            assert lhs == rhs, (order, lhs, rhs)
    for order, conds in _sums(B4).items():
        if order <= 4:
            for lhs, rhs in conds:
                assert lhs == rhs, ("embedded", order, lhs, rhs)
    # the embedded method is genuinely of lower order (the error estimate is non-zero)
    assert any(lhs != rhs for lhs, rhs in _sums(B4)[5])
    # FSAL: the last row of A equals the propagating weights
    assert A[6] + [F(0)] == B5


def spin(b=0.1, alpha=0.0, m=(1.0, 0.0, 0.0)):
    p = Problem(1, 1, 1, 1e-9, 1e-9, 1e-9)
    p.msat[0] = 1.0 / (4e-7 * np.pi)
    p.alpha[0] = alpha
    p.b0[0] = (0.0, 0.0, b)
    p.demag = p.exch = p.anis = False
    v = np.array(m, dtype=float)
    p.m0 = (v / np.linalg.norm(v)).reshape(3, 1, 1, 1)
    return p


def test_larmor_precession():
    """E1 (Fig. figtqLL): 0.1 T along z, no damping, 3 ns: m_x = cos(gamma B t)
    and, with the damping-sign reading, m_y = +sin(gamma B t).  The global
    error is bounded by (accepted steps) x MaxErr."""
    p = spin()
    p.max_err = 1e-6
    s = RK45(p)
    w = GAMMA_LL * 0.1
    for t_end in np.linspace(0.25e-9, 3e-9, 12):
        s.run(t_end)
        m = s.m[:, 0, 0, 0]
        exact = np.array([np.cos(w * t_end), np.sin(w * t_end), 0.0])
        assert np.linalg.norm(m - exact) <= s.accepted * p.max_err
    assert s.t == 3e-9


def _period_error(p, n):
    T = 2 * np.pi / (GAMMA_LL * 0.1)
    s = RK45(p)
    s.run_fixed([T / n] * n)
    return np.linalg.norm(s.m[:, 0, 0, 0] - p.m0[:, 0, 0, 0])


def test_fifth_order_convergence():
    """E11 (Fig. figConvergence): one period of precession from (1,0,1)/sqrt(2)
    with fixed steps; the error falls with slope 5."""
    p = spin(m=(1.0, 0.0, 1.0))
    ns = np.array([12, 16, 24, 32, 48])
    errs = np.array([_period_error(p, n) for n in ns])
    slope = -np.polyfit(np.log(ns), np.log(errs), 1)[0]
    assert abs(slope - 5.0) < 0.3, (slope, errs)


def test_error_linear_in_maxerr():
    """E12 (Fig. figMaxErr): the error after one period scales linearly with
    MaxErr."""
    T = 2 * np.pi / (GAMMA_LL * 0.1)
    errs, tols = [], np.array([1e-7, 1e-6, 1e-5, 1e-4])
    for tol in tols:
        p = spin(m=(1.0, 0.0, 1.0))
        p.max_err = tol
        s = RK45(p)
        s.run(T)
        errs.append(np.linalg.norm(s.m[:, 0, 0, 0] - p.m0[:, 0, 0, 0]))
    slope = np.polyfit(np.log(tols), np.log(errs), 1)[0]
    assert 0.7 < slope < 1.3, (slope, errs)


def test_energy_conserved_without_damping():
    """alpha = 0 in a static field: the LL flow conserves the total energy."""
    p = film_sp4(16, 4)
    p.alpha[0] = 0.0
    p.max_err = 1e-6
    s = RK45(p)
    e0 = energies(p, s.m, 0.0, s.field)["total"]
    es = []
    for _ in range(10):
        s.steps(10)
        es.append(energies(p, s.m, s.t, s.field)["total"])
    drift = max(abs(e - e0) for e in es)
    assert drift < 1e-4 * abs(e0), (drift, e0)


def test_energy_decreases_with_damping():
    """alpha > 0 in a static field: energy is non-increasing along the run."""
    p = film_sp4(16, 4)
    p.alpha[0] = 0.5
    s = RK45(p)
    prev = energies(p, s.m, 0.0, s.field)["total"]
    for _ in range(40):
        s.steps(2)
        e = energies(p, s.m, s.t, s.field)["total"]
        assert e <= prev + 1e-9 * abs(prev)
        prev = e


@pytest.mark.parametrize("k", [1, 3, 6])
def test_exchange_spin_wave_dispersion(k):
    """Linear spin waves on an open chain (Neumann): the mode
    cos(pi k (i + 1/2) / N) precesses about B0 z at
    omega_k = gamma (B0 + (2 Aex/Msat)(2 - 2 cos(pi k / N)) / Delta^2)."""
    n, d, A, ms, b0 = 16, 2e-9, 1.3e-11, 8e5, 0.05
    p = Problem(n, 1, 1, d, d, d)
    p.msat[0], p.aex[0], p.alpha[0] = ms, A, 0.0
    p.b0[0] = (0.0, 0.0, b0)
    p.demag = p.anis = False
    amp = 1e-5
    mode = np.cos(np.pi * k * (np.arange(n) + 0.5) / n)
    m = np.zeros((3, 1, 1, n))
    m[0, 0, 0] = amp * mode
    m[2, 0, 0] = 1.0
    p.m0 = m / np.sqrt((m * m).sum(axis=0))
    omega = GAMMA_LL * (b0 + (2 * A / ms) * (2 - 2 * np.cos(np.pi * k / n)) / d ** 2)
    T = 2 * np.pi / omega
    p.max_err = 1e-12
    s = RK45(p)
    s.run(2.25 * T)
    # after 2.25 periods the transverse part has turned counter-clockwise
    # (x towards y) by 4.5 pi, i.e. it points along +y
    c = s.m[0, 0, 0] + 1j * s.m[1, 0, 0]
    phase = np.angle(np.sum(c * mode))
    assert abs(phase - 0.5 * np.pi) / (4.5 * np.pi) < 1e-4
    assert abs(np.abs(np.sum(c * mode)) / (amp * np.sum(mode * mode)) - 1) < 1e-4
