"""Pins for the oracle's interfacial DMI field, energy and boundary
conditions (Sec. III, "Dzyaloshinskii-Moriya interaction")."""
import numpy as np
import pytest

from oracle.dmi import dmi_field
from oracle.energy import energies
from oracle.field import cross, effective_field
from paper_1406_7635_gb300.workloads import Problem


W = 5   # strip width (cells) across the profile; the middle line is checked,
        # away from the strip's own side edges (where the ghosts also act)


def chain(n, axis="x", d=1e-9, D=3e-3, A=1.5e-11, ms=1.1e6):
    shape = {"x": (n, W, 1), "y": (W, n, 1)}[axis]
    p = Problem(*shape, d, d, d)
    p.msat[0], p.aex[0], p.dind[0] = ms, A, D
    p.alpha[0] = 0.5
    p.demag = p.anis = p.zeeman = False
    return p


@pytest.mark.parametrize("axis,sense", [("x", 1), ("x", -1), ("y", 1), ("y", -1)])
def test_cycloid_interior_closed_form(axis, sense):
    """A cycloid m = (s sin kx, 0, cos kx) (or its y analogue): the central
    differences of sin/cos give exactly sin(k d)/d times the derivative, so
    in the interior B_DM = -s (2D/Msat) (sin(k d)/d) m, and the DMI energy
    density -1/2 M.B_DM is s D sin(k d)/d (the discrete form of
    D (mz div m - (m.grad) mz) = s D k)."""
    n, d, D, ms = 64, 1e-9, 3e-3, 1.1e6
    p = chain(n, axis, d, D, ms=ms)
    k = 2 * np.pi / (23.0 * d)
    x = (np.arange(n) + 0.5) * d
    m = np.zeros((3,) + p.shape)
    comp = 0 if axis == "x" else 1
    if axis == "x":
        m[comp, 0] = sense * np.sin(k * x)[None, :]
        m[2, 0] = np.cos(k * x)[None, :]
    else:
        m[comp, 0] = sense * np.sin(k * x)[:, None]
        m[2, 0] = np.cos(k * x)[:, None]
    B = dmi_field(p, m)
    f = np.sin(k * d) / d
    inner = slice(1, n - 1)
    inner_idx = (slice(None), 0, inner, W // 2) if axis == "y" else (slice(None), 0, W // 2, inner)
    expect = -sense * (2 * D / ms) * f * m[inner_idx]
    assert np.abs(B[inner_idx] - expect).max() < 1e-9 * (2 * D / ms) * f
    dens = -0.5 * ms * (m[inner_idx] * B[inner_idx]).sum(axis=0)
    assert np.allclose(dens, sense * D * f, rtol=1e-12)


def test_energy_gradient_is_minus_field_in_the_interior():
    """The central-difference DMI operator is symmetric, so away from the
    boundary B_DM = -(1/(Msat V)) dE_DM/dm (central finite differences of the
    oracle's own energy), for every component of interior cells of a 2-D
    patch of one material (with the central cell's D, an interface between
    regions of different D is not variational)."""
    rng = np.random.default_rng(4)
    p = Problem(7, 6, 1, 1e-9, 1.5e-9, 1e-9)
    p.msat[0], p.aex[0], p.dind[0], p.alpha[0] = 1.1e6, 1.5e-11, 2e-3, 0.3
    p.demag = p.anis = p.zeeman = p.exch = False
    m = rng.standard_normal((3,) + p.shape)
    m /= np.sqrt((m * m).sum(axis=0))[None]
    B = dmi_field(p, m)
    V = p.dx * p.dy * p.dz
    h = 1e-6
    for (y, x) in [(2, 2), (3, 4), (2, 3)]:
        for c in range(3):
            mp, mm_ = m.copy(), m.copy()
            mp[c, 0, y, x] += h
            mm_[c, 0, y, x] -= h
            ep = energies(p, mp, 0.0)["dmi"]
            em = energies(p, mm_, 0.0)["dmi"]
            grad = (ep - em) / (2 * h)
            ms = p.msat[p.region[0, y, x]]
            assert abs(-grad / (ms * V) - B[c, 0, y, x]) <= 1e-6 * np.abs(B).max()


def _edge_profile(n, d, A, K, D):
    """Continuum edge state of a chain along x with perpendicular anisotropy
    K and interfacial DMI: the energy density A th'^2 + K sin^2 th + D th'
    (m = (sin th, 0, cos th)) has the first integral A th'^2 = K sin^2 th and
    the natural boundary condition 2 A th' + D = 0 at both ends, so the left
    edge tilts by sin th0 = D / (2 sqrt(A K)) and the right edge by -th0,
    with tan(th/2) = tan(th0/2) exp(-dist / sqrt(A/K))."""
    lam = np.sqrt(A / K)
    th0 = np.arcsin(D / (2 * np.sqrt(A * K)))
    x = (np.arange(n) + 0.5) * d
    L = n * d
    th = 2 * np.arctan(np.tan(th0 / 2) * np.exp(-x / lam)) - 2 * np.arctan(np.tan(th0 / 2) * np.exp(-(L - x) / lam))
    return th


def test_rohart_boundary_condition_converges():
    """Sampling the continuum edge state on chains of finer cells, the
    largest residual torque |m x B_eff| (exchange + DMI with the ghost
    boundary values + anisotropy) falls at least linearly with the cell size
    -- the boundary cells included.  A Neumann edge (ghost = the cell itself)
    would leave a residual of about D / (2 K d) there (0.75 at d = 1 nm,
    growing as 1/d).  Relative to the anisotropy field 2K/Msat."""
    A, K, D, ms, Lx = 1.6e-11, 1.0e6, 1.5e-3, 1.1e6, 64e-9
    res = []
    for n in (64, 128, 256):
        d = Lx / n
        p = chain(n, "x", d, D, A, ms)
        p.anis = True
        p.ku1[0] = K
        p.anis_u[0] = (0.0, 0.0, 1.0)
        th = _edge_profile(n, d, A, K, D)
        m = np.zeros((3,) + p.shape)
        m[0, 0] = np.sin(th)[None, :]
        m[2, 0] = np.cos(th)[None, :]
        B = effective_field(p, m, 0.0)["total"]
        tq = np.sqrt((cross(m, B) ** 2).sum(axis=0))[0, W // 2]
        res.append(tq.max() / (2 * K / ms))
    assert res[0] < 5e-3, res
    assert res[1] < 0.7 * res[0] and res[2] < 0.7 * res[1], res
