"""Spin-transfer torques (Sec. III, "Zhang-Li spin-transfer torque" and
"Slonczewski spin-transfer torque"), float64, test infrastructure only.

Zhang-Li, with u = mu_B mu_0 j / (2 e gamma_0 B_sat (1 + xi^2)) and
h = (u . grad) m:
    tau_ZL = 1/(1 + alpha^2) ((1 + xi alpha) m x (m x h) + (xi - alpha) m x h)
Slonczewski, with beta = j_z hbar / (Msat e d) and
eps = P Lambda^2 / ((Lambda^2 + 1) + (Lambda^2 - 1) (m . m_P)):
    tau_SL = beta (eps - alpha eps') / (1 + alpha^2) m x (m_P x m)
           - beta (eps' - alpha eps) / (1 + alpha^2) m x m_P

Readings where the paper is silent or garbled:
* both expressions are in tesla (u carries 1/gamma_0, beta is a field) and
  are read in the sign convention of the Landau-Lifshitz torque (the reading
  of Eq. eqLLG's sign): dm/dt = -gamma_LL tau.  So gamma_0 cancels in the
  Zhang-Li term, dm/dt_ZL = -(...)(u_v) with the velocity
  u_v = mu_B j / (2 e Msat (1 + xi^2)) (B_sat = mu_0 Msat), and a cycloid is
  advected opposite to j, with the electron flow;
* the Zhang-Li expression has no polarisation factor (none is printed);
* h uses central differences (m_{i+1} - m_{i-1}) / (2 Delta); a missing
  neighbour (outside the grid or vacuum) is replaced by the cell's own m, as
  for exchange; periodic axes wrap;
* j, xi, P, Lambda, eps', m_P and d are per-region parameters (of the cell's
  region); the Slonczewski current is j_z, the z component of j.
"""
import numpy as np

from .field import cross, msat_cells, neighbour_of, periodic_axes

MU_B = 9.2740100783e-24     # J/T
E_CHARGE = 1.602176634e-19  # C
HBAR = 1.054571817e-34      # J s


def zl_h(p, m):
    """h = (u_v . grad) m with central differences (velocity units, 1/s)."""
    mag = p.magnetic()
    ms = np.where(mag, msat_cells(p), 1.0)
    xi = p.xi[p.region]
    j = p.jcur[p.region].transpose(3, 0, 1, 2)                     # (3, nz, ny, nx)
    u = np.where(mag[None], MU_B * j / (2 * E_CHARGE * ms[None] * (1 + xi * xi)[None]), 0.0)
    per = periodic_axes(p)
    h = np.zeros_like(m)
    for comp, axis, delta in ((0, 2, p.dx), (1, 1, p.dy), (2, 0, p.dz)):
        nxt, prv = [], []
        for step, store in ((1, nxt), (-1, prv)):
            nmag, valid = neighbour_of(mag, axis, step, per[axis])
            present = nmag & valid
            vals = np.stack([neighbour_of(m[c], axis, step, per[axis])[0] for c in range(3)])
            store.append(np.where(present[None], vals, m))
        d = (nxt[0] - prv[0]) / (2.0 * delta)
        h += u[comp][None] * d
    return h * mag[None]


def stt_torque(p, m):
    """dm/dt of the enabled spin-transfer terms (zero in vacuum)."""
    mag = p.magnetic()
    a = p.alpha[p.region]
    g = p.gamma[p.region]
    out = np.zeros_like(m)
    if p.zhang_li:
        h = zl_h(p, m)
        xi = p.xi[p.region]
        c1 = (1 + xi * a) / (1 + a * a)
        c2 = (xi - a) / (1 + a * a)
        out -= c1[None] * cross(m, cross(m, h)) + c2[None] * cross(m, h)
    if p.slonczewski:
        ms = np.where(mag, msat_cells(p), 1.0)
        d = np.where(p.tfree[p.region] > 0, p.tfree[p.region], 1.0)
        jz = p.jcur[p.region][..., 2]
        beta = np.where(p.tfree[p.region] > 0, jz * HBAR / (ms * E_CHARGE * d), 0.0)
        mp = p.mp[p.region].transpose(3, 0, 1, 2)
        lam2 = p.lam[p.region] ** 2
        eps = p.pol[p.region] * lam2 / ((lam2 + 1) + (lam2 - 1) * (m * mp).sum(axis=0))
        epsp = p.epsp[p.region]
        t1 = beta * (eps - a * epsp) / (1 + a * a)
        t2 = beta * (epsp - a * eps) / (1 + a * a)
        tau = t1[None] * cross(m, cross(mp, m)) - t2[None] * cross(m, mp)
        out -= g[None] * tau
    return out * mag[None]
