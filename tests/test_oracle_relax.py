"""Pins for the oracle's RK23 (Bogacki-Shampine) solver and relax() (Sec. IV,
"Dynamics" and "Energy minimization")."""
from fractions import Fraction as F

import numpy as np
import pytest

from oracle.energy import energies
from oracle.field import Field, cross
from oracle.relax import A23, B2, B3, C23, RK23, max_torque, relax
from paper_1406_7635_gb300.workloads import GAMMA_LL, Problem, film_sp4, normalise


def test_bogacki_shampine_order_conditions():
    """Row sums c_i = sum_j a_ij; the propagating weights satisfy every order
    condition up to 3, the embedded ones up to 2 but not 3 (so the error
    estimate is of order 2); FSAL: the last row of A is the propagating
    weights.  Exact rational arithmetic."""
    s = 4
    a = [[A23[i][j] if j < len(A23[i]) else F(0) for j in range(s)] for i in range(s)]
    c = C23
    for i in range(s):
        assert sum(a[i]) == c[i]
    ac = [sum(a[i][j] * c[j] for j in range(s)) for i in range(s)]

    def conds(b):
        S = lambda v: sum(b[i] * v[i] for i in range(s))
        return {1: [(S([F(1)] * s), F(1))], 2: [(S(c), F(1, 2))],
                3: [(S([x * x for x in c]), F(1, 3)), (S(ac), F(1, 6))]}
    for order, cs in conds(B3).items():
        for lhs, rhs in cs:
            assert lhs == rhs, (order, lhs, rhs)
    for order, cs in conds(B2).items():
        if order <= 2:
            for lhs, rhs in cs:
                assert lhs == rhs, ("embedded", order)
    assert any(lhs != rhs for lhs, rhs in conds(B2)[3])
    assert A23[3] + [F(0)] == B3


def spin(m=(1.0, 0.0, 1.0), b=0.1):
    p = Problem(1, 1, 1, 1e-9, 1e-9, 1e-9)
    p.msat[0] = 1.0 / (4e-7 * np.pi)
    p.b0[0] = (0.0, 0.0, b)
    p.demag = p.exch = p.anis = False
    v = np.array(m, dtype=float)
    p.m0 = (v / np.linalg.norm(v)).reshape(3, 1, 1, 1)
    return p


def test_third_order_convergence():
    """Fig. figConvergence for RK23: one undamped precession period with
    fixed steps; the error falls with slope 3."""
    p = spin()
    T = 2 * np.pi / (GAMMA_LL * 0.1)
    ns = np.array([24, 32, 48, 64, 96])
    errs = []
    for n in ns:
        s = RK23(p)
        s.run_fixed([T / n] * n)
        errs.append(np.linalg.norm(s.m[:, 0, 0, 0] - p.m0[:, 0, 0, 0]))
    slope = -np.polyfit(np.log(ns), np.log(errs), 1)[0]
    assert abs(slope - 3.0) < 0.3, (slope, errs)


def test_larmor_adaptive_rk23():
    """Adaptive RK23 follows m = (cos wt, sin wt, 0) within (steps) x MaxErr."""
    p = spin(m=(1.0, 0.0, 0.0))
    p.max_err = 1e-7
    s = RK23(p)
    w = GAMMA_LL * 0.1
    s.run(1e-9)
    exact = np.array([np.cos(w * 1e-9), np.sin(w * 1e-9), 0.0])
    assert np.linalg.norm(s.m[:, 0, 0, 0] - exact) <= s.accepted * p.max_err
    assert s.t == 1e-9


def test_relax_stoner_wohlfarth_closed_form():
    """One cell, easy axis x (Ku1), field B along z below the anisotropy
    field: E/V = -Ku1 cos^2(phi) - Msat B sin(phi) is minimal at
    sin(phi) = Msat B / (2 Ku1) (the cube's demag energy is isotropic)."""
    p = Problem(1, 1, 1, 2e-9, 2e-9, 2e-9)
    p.msat[0], p.aex[0], p.alpha[0] = 8e5, 1.3e-11, 0.5
    p.ku1[0] = 5e5
    p.b0[0] = (0.0, 0.0, 0.5)
    p.m0 = np.array([0.8, 0.6, 0.0]).reshape(3, 1, 1, 1)
    s, log = relax(p)
    m = s.m[:, 0, 0, 0]
    sz = 8e5 * 0.5 / (2 * 5e5)
    assert abs(m[2] - sz) < 1e-7
    assert abs(m[0] - np.sqrt(1 - sz * sz)) < 1e-7
    assert abs(m[1]) < 1e-7
    assert log["final_max_err"] <= 1e-9 and log["levels"] == 27
    # the solver settings and the precession switch are restored
    assert p.precession and p.max_err == 1e-5


def _grain(seed=2):
    p = Problem(4, 2, 1, 3e-9, 3e-9, 2e-9)
    p.msat[0], p.aex[0], p.alpha[0] = 8e5, 1.3e-11, 0.5
    p.ku1[0], p.ku2[0] = 2e5, 3e4
    p.anis_u[0] = (1.0, 1.0, 0.0)
    p.b0[0] = (10e-3, -30e-3, 20e-3)
    rng = np.random.default_rng(seed)
    p.m0 = normalise(rng.standard_normal((3,) + p.shape), p.magnetic())
    return p


def test_relax_matches_library_energy_minimiser():
    """4 x 2 x 1 cells with demag, exchange, both anisotropy terms and a
    tilted field: relax() ends at the local energy minimum that BFGS (scipy,
    finite-difference gradients of the oracle's energy over the cells'
    spherical angles) finds from the same start."""
    minimize = pytest.importorskip("scipy.optimize").minimize
    p = _grain()
    s, _ = relax(p)
    f = Field(p)
    e0 = abs(energies(p, p.m0, 0.0, f)["total"])

    def m_of(x):
        th, ph = x[:8], x[8:]
        return np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)]).reshape(3, 1, 2, 4)

    m0 = p.m0.reshape(3, -1)
    x0 = np.concatenate([np.arccos(np.clip(m0[2], -1, 1)), np.arctan2(m0[1], m0[0])])
    r = minimize(lambda x: energies(p, m_of(x), 0.0, f)["total"] / e0, x0, method="BFGS",
                 options={"gtol": 1e-10})
    assert np.abs(m_of(r.x) - s.m).max() < 1e-6
    # a stationary point: m x B_eff vanishes
    B = f.terms(s.m, 0.0)["total"]
    assert np.sqrt((cross(s.m, B) ** 2).sum(axis=0)).max() < 1e-6


def test_relax_lowers_energy_and_is_independent_of_damping():
    """The relaxed state of a 16 x 4 film does not depend on alpha (which
    only sets the speed of the precession-free flow); the energy is lower
    than at the start and the residual torque is at the noise floor."""
    out = []
    for alpha in (0.5, 1.0):
        p = film_sp4(16, 4)
        p.alpha[0] = alpha
        p.b0[0] = (10e-3, 20e-3, 0.0)
        s, log = relax(p)
        e = energies(p, s.m, s.t, s.field)["total"]
        assert e < energies(p, p.m0, 0.0)["total"]
        B = s.field.terms(s.m, s.t)["total"]
        assert np.sqrt((cross(s.m, B) ** 2).sum(axis=0))[p.magnetic()].max() < 1e-5
        out.append(s.m)
    assert np.abs(out[0] - out[1]).max() < 1e-6
