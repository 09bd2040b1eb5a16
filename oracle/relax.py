"""Energy minimisation: relax() of Sec. IV ("Energy minimization") with the
Bogacki-Shampine RK23 solver of Sec. IV ("Dynamics").  Test infrastructure
only.

RK23 (Bogacki & Shampine 1989): 4 stages, the last one evaluated at the
3rd-order solution and reused as the next first stage (FSAL, like RK45); the
embedded 2nd-order solution gives the error estimate, so the step factor uses
the exponent 1/3.

relax(): the precession term is switched off, so that the torque points
down the energy gradient; the solver is RK23.  Time is advanced while the
total energy still decreases; after it stops decreasing (it has reached its
noise floor) the torque magnitude is watched instead, and each time the
torque stops decreasing MaxErr is lowered, until MaxErr reaches 1e-9.

Readings where the paper is silent:
* the energy and the torque are compared between blocks of 3 accepted steps;
* "torque magnitude" is the maximum over the magnetic cells of |tau| (the
  relaxation torque, precession off) at the current m and time;
* MaxErr is divided by sqrt(2) at each level; the level on which it first
  falls to 1e-9 or below is the last one;
* "stops decreasing" means the new value is >= the previous one;
* the solver, MaxErr and the precession switch are restored afterwards; t
  advances as in any run.
"""
from fractions import Fraction as F
from math import sqrt

import numpy as np

from .energy import energies
from .rk45 import RK45

C23 = [F(0), F(1, 2), F(3, 4), F(1)]
A23 = [
    [],
    [F(1, 2)],
    [F(0), F(3, 4)],
    [F(2, 9), F(1, 3), F(4, 9)],
]
B3 = [F(2, 9), F(1, 3), F(4, 9), F(0)]
B2 = [F(7, 24), F(1, 4), F(1, 3), F(1, 8)]
E23 = [b - bh for b, bh in zip(B3, B2)]


class RK23(RK45):
    """Bogacki-Shampine 3(2) pair with the same controller as RK45."""

    C, A, E = C23, A23, E23
    EXPONENT = 1.0 / 3.0


def max_torque(solver):
    """max over magnetic cells of |tau(m, t)| at the solver's state."""
    tq = solver.field.torque(solver.m, solver.t)
    n = np.sqrt((tq * tq).sum(axis=0))
    mag = solver.mag
    return float(n[mag].max()) if mag.any() else 0.0


def relax(p, m=None, t=0.0, block=3, min_err=1e-9, max_steps=200000):
    """Relax p's magnetisation (from m, default p.m0).  Returns the RK23
    solver at the end (its m, t, counters) and a log of the phases."""
    saved = (p.precession, p.max_err)
    p.precession = False
    s = RK23(p, m=m)
    s.t = t
    log = {"energy_blocks": 0, "torque_blocks": 0, "levels": 0}
    try:
        e0 = energies(p, s.m, s.t, s.field)["total"]
        while s.accepted < max_steps:
            s.steps(block)
            log["energy_blocks"] += 1
            e1 = energies(p, s.m, s.t, s.field)["total"]
            if e1 >= e0:
                break
            e0 = e1
        t0 = max_torque(s)
        while s.accepted < max_steps:
            s.steps(block)
            log["torque_blocks"] += 1
            t1 = max_torque(s)
            if t1 < t0:
                t0 = t1
                continue
            if p.max_err <= min_err:
                break
            p.max_err /= sqrt(2.0)
            log["levels"] += 1
            t0 = t1
        log["final_max_err"] = p.max_err
        log["final_torque"] = t0
    finally:
        p.precession, p.max_err = saved
    return s, log
