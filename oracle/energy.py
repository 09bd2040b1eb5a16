"""Energies computed from the effective field (Sec. III).

E_demag = -1/2 sum M.B_demag V           (energy density of the demag term)
E_exch  = -1/2 sum M.B_exch V            (Eq. eqEdensExch)
E_anis  = -1/2 sum M.B_anis(Ku1) V - 1/4 sum M.B_anis(Ku2) V   (Eq. EaniUM)
E_Z     = -sum M.B_ext V                 (Zeeman energy density -M.B)
E_DM    = -1/2 sum M.B_DM V              (Eq. eqEdensDMI)
<m>     = average of m over the magnetic cells.

Float64 test infrastructure only: tests, smoke() and the benchmark's CPU
legs use it; the product path never does.
"""
import numpy as np

from .field import Field, msat_cells


def energies(p, m, t, field=None):
    f = field if field is not None else Field(p)
    terms = f.terms(m, t)
    mag = p.magnetic()
    M = msat_cells(p)[None] * m
    V = p.dx * p.dy * p.dz

    def dot(B):
        return float((M * B).sum()) * V

    e = {
        "demag": -0.5 * dot(terms["demag"]),
        "exch": -0.5 * dot(terms["exch"]),
        "anis": -0.5 * dot(terms["anis1"]) - 0.25 * dot(terms["anis2"]),
        "zeeman": -dot(terms["zeeman"]),
        "dmi": -0.5 * dot(terms["dmi"]),
    }
    e["total"] = e["demag"] + e["exch"] + e["anis"] + e["zeeman"] + e["dmi"]
    nmag = int(mag.sum())
    e["m_avg"] = [float(m[c][mag].sum()) / nmag if nmag else 0.0 for c in range(3)]
    return e
