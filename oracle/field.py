"""Effective field and Landau-Lifshitz torque (Sec. III), float64.

B_eff = B_ext + B_demag + B_exch + B_anis + B_DM (the interfacial DMI term
and its boundary conditions are in dmi.py; thermal and spin-transfer terms
are outside this path).  Non-magnetic cells (mask 0 or Msat 0) carry m = 0,
B_eff = 0 and zero torque.

Float64 test infrastructure only: tests, smoke() and the benchmark's CPU
legs use it; the product path never does.
"""
import numpy as np

from .demag import MU0, demag_direct, demag_fft, magnetisation


def msat_cells(p):
    return np.where(p.magnetic(), p.msat[p.region], 0.0)


def exchange_lut(p):
    """2 S(r1, r2) * harmonic mean of Aex/Msat of the two regions (Eq. for
    inter-region exchange).  Within one region the harmonic mean of a with
    itself is a, so the table reduces to 2 Aex/Msat (Eq. for B_exch).  A pair
    whose Aex/Msat values sum to zero couples with 0."""
    a = np.where(p.msat > 0, p.aex / np.where(p.msat > 0, p.msat, 1.0), 0.0)
    s = a[:, None] + a[None, :]
    h = np.where(s != 0, 2.0 * a[:, None] * a[None, :] / np.where(s != 0, s, 1.0), 0.0)
    return 2.0 * p.exch_scale * h


def periodic_axes(p):
    """Periodic flags per array axis (0 = z, 1 = y, 2 = x) of the (z, y, x)
    arrays, from p.pbc = (Px, Py, Pz)."""
    px, py, pz = getattr(p, "pbc", (0, 0, 0))
    return (pz > 0, py > 0, px > 0)


def neighbour_of(a, axis, step, periodic):
    """a shifted so that entry i holds a[i + step] along `axis`, wrapping
    around on a periodic axis; returns (values, valid) where valid marks the
    entries that have a neighbour (all of them on a periodic axis)."""
    n = a.shape[axis]
    if periodic:
        return np.roll(a, -step, axis=axis), np.ones(a.shape, dtype=bool)
    out = np.zeros_like(a)
    valid = np.zeros(a.shape, dtype=bool)
    sl_c = [slice(None)] * a.ndim
    sl_n = [slice(None)] * a.ndim
    if step == 1:
        sl_c[axis], sl_n[axis] = slice(0, n - 1), slice(1, n)
    else:
        sl_c[axis], sl_n[axis] = slice(1, n), slice(0, n - 1)
    out[tuple(sl_c)] = a[tuple(sl_n)]
    valid[tuple(sl_c)] = True
    return out, valid


def exchange_field(p, m):
    """6-neighbour exchange: sum over neighbours of lut * (m_i - m) / Delta_i^2.

    A neighbour outside the grid or not magnetic is missing; using the cell's
    own m in its place (Neumann condition, Sec. III.C) makes its term zero.
    Along a periodic axis the grid wraps around (the paper's PBC are felt by
    the stencils), so the first and last cells are neighbours.
    """
    mag = p.magnetic()
    lut = exchange_lut(p)
    reg = p.region.astype(np.int64)
    per = periodic_axes(p)
    B = np.zeros_like(m)
    for axis, delta in ((2, p.dx), (1, p.dy), (0, p.dz)):
        for step in (1, -1):
            nreg, valid = neighbour_of(reg, axis, step, per[axis])
            nmag, _ = neighbour_of(mag, axis, step, per[axis])
            both = mag & nmag & valid
            coupling = np.where(both, lut[reg, nreg], 0.0)
            for c in range(3):
                nm, _ = neighbour_of(m[c], axis, step, per[axis])
                B[c] += coupling * (nm - m[c]) / delta ** 2
    return B * mag[None]


def anisotropy_field_parts(p, m):
    """Uniaxial anisotropy, Sec. III.E: (2 Ku1/Msat)(u.m)u and (4 Ku2/Msat)(u.m)^3 u.

    The paper prints Bsat in the denominators; J/m^3 divided by T is A/m, not
    T, and the energy identity E = -1/2 B(Ku1).M - 1/4 B(Ku2).M only holds with
    Msat, so Msat is used.
    """
    mag = p.magnetic()
    ms = msat_cells(p)
    safe = np.where(mag, ms, 1.0)
    u = p.anis_u[p.region].transpose(3, 0, 1, 2)          # (3, nz, ny, nx)
    um = (u * m).sum(axis=0)
    k1 = np.where(mag, 2.0 * p.ku1[p.region] / safe, 0.0)
    k2 = np.where(mag, 4.0 * p.ku2[p.region] / safe, 0.0)
    return k1 * um * u, k2 * um ** 3 * u


def zeeman_field(p, t):
    """B_ext = b0 + b1 sin(2 pi f t + phase) by region (Sec. II.A excitations)."""
    s = np.sin(2.0 * np.pi * p.freq * t + p.phase)
    b = p.b0 + p.b1 * s                                      # (256, 3)
    return b[p.region].transpose(3, 0, 1, 2) * p.magnetic()[None]


def effective_field(p, m, t, demag_method="fft", spectrum=None):
    """All enabled terms of B_eff (a dict) and their sum under key 'total'."""
    mag = p.magnetic()
    zero = np.zeros_like(m)
    terms = {}
    if p.demag:
        M = magnetisation(msat_cells(p), m)
        pbc = getattr(p, "pbc", (0, 0, 0))
        if demag_method == "direct":
            terms["demag"] = demag_direct(M, p.dx, p.dy, p.dz, pbc)
        else:
            terms["demag"] = demag_fft(M, p.dx, p.dy, p.dz, spectrum=spectrum, pbc=pbc)
    else:
        terms["demag"] = zero
    has_dmi = bool(np.any(p.dind[np.unique(p.region)] != 0))
    if has_dmi:
        from .dmi import dmi_field, exchange_field_bc
        terms["exch"] = exchange_field_bc(p, m) if p.exch else zero
        terms["dmi"] = dmi_field(p, m)
    else:
        terms["exch"] = exchange_field(p, m) if p.exch else zero
        terms["dmi"] = zero
    if p.anis:
        a1, a2 = anisotropy_field_parts(p, m)
        terms["anis1"], terms["anis2"] = a1, a2
    else:
        terms["anis1"] = terms["anis2"] = zero
    terms["zeeman"] = zeeman_field(p, t) if p.zeeman else zero
    total = (terms["demag"] + terms["exch"] + terms["anis1"] + terms["anis2"]
             + terms["zeeman"] + terms["dmi"])
    terms["total"] = total * mag[None]
    return terms


def cross(a, b):
    return np.stack([a[1] * b[2] - a[2] * b[1],
                     a[2] * b[0] - a[0] * b[2],
                     a[0] * b[1] - a[1] * b[0]])


def ll_torque(p, m, B):
    """Landau-Lifshitz torque, Eq. (eqLLG), with the sign that damps.

    tau = -gamma/(1 + alpha^2) (m x B + alpha m x (m x B)).  The paper prints
    a + sign with gamma > 0; with that sign the damping term would drive m away
    from B and raise the energy, so the sign is read as minus (a spin at +x in
    B = +z then turns to +y).  With precession disabled (relaxation) the
    m x B term is dropped.
    """
    mag = p.magnetic()
    g = p.gamma[p.region]
    a = p.alpha[p.region]
    pref = np.where(mag, -g / (1.0 + a * a), 0.0)
    mxB = cross(m, B)
    mxmxB = cross(m, mxB)
    prec = mxB if p.precession else 0.0
    return pref[None] * (prec + a[None] * mxmxB)


class Field:
    """Torque evaluator with the kernel spectrum computed once per grid."""

    def __init__(self, p, demag_method="fft"):
        self.p = p
        self.method = demag_method
        self.spectrum = None
        if p.demag and demag_method == "fft":
            from .demag import kernel_spectrum
            self.spectrum = kernel_spectrum(p.nx, p.ny, p.nz, p.dx, p.dy, p.dz, getattr(p, "pbc", (0, 0, 0)))
        self.evals = 0

    def terms(self, m, t):
        return effective_field(self.p, m, t, self.method, self.spectrum)

    def torque(self, m, t):
        self.evals += 1
        tq = ll_torque(self.p, m, self.terms(m, t)["total"])
        if getattr(self.p, "zhang_li", False) or getattr(self.p, "slonczewski", False):
            from .stt import stt_torque
            tq = tq + stt_torque(self.p, m)
        return tq
