"""Interfacial Dzyaloshinskii-Moriya field and the boundary conditions it
imposes (Sec. III, "Dzyaloshinskii-Moriya interaction"), float64, test
infrastructure only.

  B_DM = (2D/Msat) (dmz/dx, dmz/dy, -dmx/dx - dmy/dy)

with central differences dm/di = (m_{i+1} - m_{i-1}) / (2 Delta_i).  A
neighbour that is missing (outside the grid, or not magnetic) is replaced by
the ghost value m + n Delta_i dm/di|_boundary, n = +1 on the high face and -1
on the low face of axis i, with the boundary derivatives
  x faces: dm/dx = ( -D/(2A) mz, 0, D/(2A) mx )
  y faces: dm/dy = ( 0, -D/(2A) mz, D/(2A) my )
  z faces: dm/dz = 0.
Where D != 0 the Heisenberg exchange field uses the same ghosts (a ghost
couples with the cell's own 2 Aex/Msat).  Energy: -1/2 M.B_DM per cell
volume.

Readings where the paper is silent:
* D, Aex and Msat are those of the central cell's region; a magnetic
  neighbour of another region enters the differences with its own m;
* with Aex = 0 the boundary derivative is taken as zero (no ghost tilt).
"""
import numpy as np

from .field import exchange_lut, msat_cells, neighbour_of, periodic_axes


def _neighbour(p, m, axis, step):
    """Neighbour values along `axis` (2 = x, 1 = y, 0 = z of the (z, y, x)
    arrays) in direction `step` (+1 / -1): the neighbour's m where it exists
    and is magnetic (wrapping around along a periodic axis), else the ghost
    value of the central cell.  Returns (values (3, nz, ny, nx), present
    mask)."""
    mag = p.magnetic()
    per = periodic_axes(p)[axis]
    nmag, valid = neighbour_of(mag, axis, step, per)
    present = nmag & valid
    nb = np.stack([neighbour_of(m[c], axis, step, per)[0] for c in range(3)])
    # ghosts: m + step * Delta * dm/d(axis) at the boundary
    d = p.dind[p.region]
    a = p.aex[p.region]
    cbc = np.where(a > 0, d / (2.0 * np.where(a > 0, a, 1.0)), 0.0)
    g = m.copy()
    if axis == 2:
        g[0] = m[0] + step * p.dx * (-cbc * m[2])
        g[2] = m[2] + step * p.dx * (cbc * m[0])
    elif axis == 1:
        g[1] = m[1] + step * p.dy * (-cbc * m[2])
        g[2] = m[2] + step * p.dy * (cbc * m[1])
    nb = np.where(present[None], nb, g)
    return nb, present


def dmi_field(p, m):
    """B_DM at every magnetic cell (zero elsewhere)."""
    mag = p.magnetic()
    ms = msat_cells(p)
    pref = np.where(mag, 2.0 * p.dind[p.region] / np.where(mag, ms, 1.0), 0.0)
    xp, _ = _neighbour(p, m, 2, 1)
    xm, _ = _neighbour(p, m, 2, -1)
    yp, _ = _neighbour(p, m, 1, 1)
    ym, _ = _neighbour(p, m, 1, -1)
    dmz_dx = (xp[2] - xm[2]) / (2.0 * p.dx)
    dmz_dy = (yp[2] - ym[2]) / (2.0 * p.dy)
    dmx_dx = (xp[0] - xm[0]) / (2.0 * p.dx)
    dmy_dy = (yp[1] - ym[1]) / (2.0 * p.dy)
    B = np.stack([dmz_dx, dmz_dy, -dmx_dx - dmy_dy]) * pref[None]
    return B * mag[None]


def exchange_field_bc(p, m):
    """Exchange field with the DMI boundary conditions: as the plain 6-point
    stencil, but a missing neighbour is the ghost value (coupling 2 Aex/Msat
    of the central cell) instead of the cell itself."""
    mag = p.magnetic()
    lut = exchange_lut(p)
    reg = p.region.astype(np.int64)
    own = lut[reg, reg]
    B = np.zeros_like(m)
    for axis, delta in ((2, p.dx), (1, p.dy), (0, p.dz)):
        n = m.shape[1 + axis]
        for step in (1, -1):
            nb, present = _neighbour(p, m, axis, step)
            # coupling to a present neighbour: the inter-region table
            nreg = np.roll(reg, -step, axis=axis)
            coupling = np.where(present, lut[reg, nreg], own)
            for c in range(3):
                B[c] += coupling * (nb[c] - m[c]) / delta ** 2
    return B * mag[None]
