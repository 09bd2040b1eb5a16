"""Dormand-Prince RK45 with adaptive step control (Sec. IV, "Dynamics").

The 5th-order solution advances m; the embedded 4th-order one gives the error
per step eps = max over cells |tau_high - tau_low| * dt (Sec. IV, "Adaptive
time step"), here the Euclidean norm per cell of dt * sum_i (b_i - bhat_i) k_i.
Coefficients are Dormand & Prince's 1980 tableau (7 stages, the last stage is
evaluated at the new solution and reused as the next first stage: FSAL).

Readings where the paper is silent:
* accept iff eps <= MaxErr; new dt = dt * clamp(headroom (MaxErr/eps)^(1/5),
  0.2, 5) (factor 5 when eps == 0), then limited to [dt_min, dt_max]; a
  rejected step whose new dt would fall below dt_min is an underflow error;
* stage s is evaluated at t + c_s dt (time-dependent excitations);
* the 7th stage is evaluated at the un-normalised 5th-order solution and kept
  as the next k1; only then is m normalised per cell (m has unit length);
* run(t_end) shortens the last step to land on t_end exactly; the step size the
  controller proposes after it is kept for the next call.

Float64 test infrastructure only: tests, smoke() and the benchmark's CPU
legs use it; the product path never does.
"""
from fractions import Fraction as F

import numpy as np

from .field import Field

C = [F(0), F(1, 5), F(3, 10), F(4, 5), F(8, 9), F(1), F(1)]
A = [
    [],
    [F(1, 5)],
    [F(3, 40), F(9, 40)],
    [F(44, 45), F(-56, 15), F(32, 9)],
    [F(19372, 6561), F(-25360, 2187), F(64448, 6561), F(-212, 729)],
    [F(9017, 3168), F(-355, 33), F(46732, 5247), F(49, 176), F(-5103, 18656)],
    [F(35, 384), F(0), F(500, 1113), F(125, 192), F(-2187, 6784), F(11, 84)],
]
B5 = [F(35, 384), F(0), F(500, 1113), F(125, 192), F(-2187, 6784), F(11, 84), F(0)]
B4 = [F(5179, 57600), F(0), F(7571, 16695), F(393, 640), F(-92097, 339200),
      F(187, 2100), F(1, 40)]
E = [b - bh for b, bh in zip(B5, B4)]


class DtUnderflow(RuntimeError):
    pass


class NonFinite(RuntimeError):
    pass


class RK45:
    """Integrates dm/dt = tau(m, t) from the problem's m0 at t = 0.

    The tableau is read from the class attributes (nodes C, stage rows A,
    error weights E = b_high - b_low, step-factor exponent 1/(q+1) for an
    error estimate of order q), so that an embedded pair with the same
    FSAL structure only overrides them."""

    C, A, E = C, A, E
    EXPONENT = 0.2

    def __init__(self, p, demag_method="fft", m=None):
        self.p = p
        self.field = Field(p, demag_method)
        self.mag = p.magnetic()
        self.m = (p.m0 if m is None else m).astype(np.float64).copy()
        self.t = 0.0
        self.dt = p.dt0
        self.k1 = None
        self.accepted = 0
        self.rejected = 0
        self.last_err = 0.0
        self.dt_history = []

    def _attempt(self, h):
        """One trial step of size h from (m, t): returns (y_new, k7, eps)."""
        tau = self.field.torque
        if self.k1 is None:
            self.k1 = tau(self.m, self.t)
        k = [self.k1]
        for s in range(1, len(self.C)):
            ys = self.m.copy()
            for j, a in enumerate(self.A[s]):
                if a != 0:
                    ys = ys + h * float(a) * k[j]
            k.append(tau(ys, self.t + float(self.C[s]) * h))
        y_new = ys                      # the last stage point is the high-order solution
        err = np.zeros_like(self.m)
        for j, e in enumerate(self.E):
            err = err + h * float(e) * k[j]
        norm = np.sqrt((err * err).sum(axis=0))
        eps = float(norm[self.mag].max()) if self.mag.any() else 0.0
        return y_new, k[-1], eps

    def _accept(self, y_new, k7, h):
        n = np.sqrt((y_new * y_new).sum(axis=0))
        self.m = np.where(self.mag[None], y_new / np.where(n > 0, n, 1.0)[None], 0.0)
        self.k1 = k7
        self.t += h
        self.accepted += 1
        self.dt_history.append(h)

    def _factor(self, eps):
        p = self.p
        if eps == 0.0:
            return 5.0
        return min(5.0, max(0.2, p.headroom * (p.max_err / eps) ** self.EXPONENT))

    def adaptive_step(self, h_limit=None):
        """Attempts until one is accepted; returns the accepted step size."""
        p = self.p
        while True:
            h = self.dt if h_limit is None else min(self.dt, h_limit)
            y_new, k7, eps = self._attempt(h)
            if not np.isfinite(eps):
                raise NonFinite("non-finite error estimate")
            self.last_err = eps
            new_dt = min(h * self._factor(eps), p.dt_max)
            if eps <= p.max_err:
                self._accept(y_new, k7, h)
                self.dt = max(new_dt, p.dt_min)
                return h
            self.rejected += 1
            if new_dt < p.dt_min:
                raise DtUnderflow("time step below dt_min")
            self.dt = new_dt

    def steps(self, n):
        """n accepted adaptive steps (the paper's steps(n))."""
        for _ in range(n):
            self.adaptive_step()

    def run(self, t_end):
        """Advance to t_end exactly (the paper's run(t))."""
        while self.t < t_end:
            h = self.adaptive_step(h_limit=t_end - self.t)
            if self.t + 1e-6 * h >= t_end:   # landed (rounding of t += h)
                self.t = t_end
        return self.t

    def run_fixed(self, dts):
        """Replay a given step sequence: every step accepted (lockstep mode)."""
        for h in dts:
            y_new, k7, eps = self._attempt(float(h))
            self.last_err = eps
            self._accept(y_new, k7, float(h))
