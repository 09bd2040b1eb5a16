"""Pins for the oracle's exchange, anisotropy, Zeeman terms, torque, energies."""
import numpy as np
import pytest

from oracle.energy import energies
from oracle.field import Field, anisotropy_field_parts, exchange_field, exchange_lut, ll_torque
from paper_1406_7635_gb300.workloads import Problem, film_sp4, grain_film


def chain(n, dx=1e-9, aex=1e-11, msat=1e6):
    p = Problem(n, 1, 1, dx, dx, dx)
    p.msat[0], p.aex[0], p.alpha[0] = msat, aex, 0.0
    p.demag = p.anis = p.zeeman = False
    return p


@pytest.mark.parametrize("theta_deg", [1.0, 5.0, 20.0, 45.0, 90.0, 170.0])
def test_spiral_exchange_energy(theta_deg):
    """E5 (Fig. figExchE) without PBC: a planar spiral with angle theta between
    neighbours on an open chain of N cells has, from the 6-neighbour field and
    E = -1/2 M.B V, exactly E = 2 Aex (N - 1)(1 - cos theta) Delta; for small
    theta this tends to the continuum Aex theta^2 / Delta^2 per bond volume."""
    n, d, A = 64, 1e-9, 1e-11
    p = chain(n, d, A)
    th = np.deg2rad(theta_deg) * np.arange(n)
    m = np.zeros((3, 1, 1, n))
    m[1, 0, 0] = np.sin(th)
    m[2, 0, 0] = np.cos(th)
    e = energies(p, m, 0.0)["exch"]
    exact = 2 * A * (n - 1) * (1 - np.cos(np.deg2rad(theta_deg))) * d
    assert abs(e - exact) < 1e-12 * exact
    if theta_deg <= 5.0:
        cont = (n - 1) * d ** 3 * A * np.deg2rad(theta_deg) ** 2 / d ** 2
        assert abs(e / cont - 1) < 1e-3


def test_exchange_uniform_is_zero_and_neumann_edges():
    p = film_sp4(8, 4)
    m = np.zeros((3,) + p.shape)
    m[0] = 1.0
    assert np.abs(exchange_field(p, m)).max() == 0.0
    # a vacuum cell next to a magnetic one contributes nothing
    p.mask[0, 1, 3] = 0
    m[:, 0, 1, 3] = 0.0
    B = exchange_field(p, m)
    assert np.abs(B).max() == 0.0


def test_harmonic_mean_between_regions():
    """Eq. for inter-region exchange: two cells of different materials couple
    with 2 S * 2 a1 a2 / (a1 + a2), a = Aex/Msat; by hand on a 2-cell chain."""
    p = Problem(2, 1, 1, 2e-9, 1e-9, 1e-9)
    p.region[0, 0, 1] = 1
    p.msat[0], p.aex[0] = 8e5, 1.3e-11
    p.msat[1], p.aex[1] = 1.2e6, 2.0e-11
    p.exch_scale[0, 1] = p.exch_scale[1, 0] = 0.85
    m = np.zeros((3, 1, 1, 2))
    m[0, 0, 0, 0] = 1.0
    m[1, 0, 0, 1] = 1.0
    a0, a1 = 1.3e-11 / 8e5, 2.0e-11 / 1.2e6
    c = 2 * 0.85 * 2 * a0 * a1 / (a0 + a1)
    B = exchange_field(p, m)
    expect0 = c * (m[:, 0, 0, 1] - m[:, 0, 0, 0]) / (2e-9) ** 2
    assert np.allclose(B[:, 0, 0, 0], expect0, rtol=1e-14, atol=0)
    assert np.allclose(B[:, 0, 0, 1], -expect0, rtol=1e-14, atol=0)
    assert abs(exchange_lut(p)[0, 0] - 2 * a0) < 1e-14 * a0


@pytest.mark.parametrize("ku1,ku2", [(1e6, 0.0), (-1e6, 0.0), (0.0, 1e6), (0.0, -1e6), (3e5, -2e5)])
def test_uniaxial_energy_sweep(ku1, ku2):
    """E7 (Fig. figAnis): single spin with u = x swept in the xy-plane; the
    field route E = -1/2 B(Ku1).M - 1/4 B(Ku2).M equals the closed form
    -Ku1 cos^2 - Ku2 cos^4 (Eq. EanisUA)."""
    p = Problem(1, 1, 1, 1e-9, 1e-9, 1e-9)
    p.msat[0] = 1e6
    p.ku1[0], p.ku2[0] = ku1, ku2
    p.anis_u[0] = (1.0, 0.0, 0.0)
    p.demag = p.exch = p.zeeman = False
    V = 1e-27
    for th in np.deg2rad(np.arange(0, 361, 7)):
        m = np.array([np.cos(th), np.sin(th), 0.0]).reshape(3, 1, 1, 1)
        e = energies(p, m, 0.0)["anis"] / V
        exact = -ku1 * np.cos(th) ** 2 - ku2 * np.cos(th) ** 4
        assert abs(e - exact) < 1e-9 * max(abs(ku1), abs(ku2))


def test_zeeman_energy_and_time_function():
    p = grain_film(8, 8, 4)
    t = 0.3e-9
    m = p.m0
    e = energies(p, m, t)
    V = p.dx * p.dy * p.dz
    bx = 10e-3 * np.sin(2 * np.pi * 1e9 * t)
    assert abs(e["zeeman"] - (-(1e6 * m[0] * bx).sum() * V)) < 1e-12 * abs(e["zeeman"])


def test_torque_sign_and_orthogonality():
    """A spin at +x in B = +z turns to +y (damping sign reading of Eq. eqLLG),
    the torque is perpendicular to m, and with damping it has a component
    along B (towards the field)."""
    p = Problem(1, 1, 1, 1e-9, 1e-9, 1e-9)
    p.msat[0], p.alpha[0] = 1e6, 0.1
    m = np.array([1.0, 0.0, 0.0]).reshape(3, 1, 1, 1)
    B = np.array([0.0, 0.0, 0.1]).reshape(3, 1, 1, 1)
    tau = ll_torque(p, m, B)[:, 0, 0, 0]
    g = 1.7595e11 / (1 + 0.01)
    assert np.allclose(tau, [0.0, g * 0.1, g * 0.1 * 0.1], rtol=1e-14)
    rng = np.random.default_rng(3)
    p2 = film_sp4(8, 4)
    f = Field(p2)
    tau = f.torque(p2.m0, 0.0)
    assert np.abs((tau * p2.m0).sum(axis=0)).max() < 1e-6 * np.abs(tau).max()


def test_demag_energy_of_uniform_cube():
    """E_demag of a uniformly magnetised cube = 1/2 mu0 (1/3) Ms^2 V."""
    p = Problem(4, 4, 4, 1e-9, 1e-9, 1e-9)
    p.msat[0] = 8e5
    p.exch = p.anis = p.zeeman = False
    m = np.zeros((3,) + p.shape)
    m[2] = 1.0
    e = energies(p, m, 0.0)["demag"]
    exact = 0.5 * 4e-7 * np.pi / 3.0 * 8e5 ** 2 * (4e-9) ** 3
    assert abs(e / exact - 1) < 1e-10


def test_anisotropy_field_is_energy_gradient():
    """B_anis = -dE/dM: a finite difference of the closed-form energy density
    along a random tangent direction matches the field."""
    p = Problem(1, 1, 1, 1e-9, 1e-9, 1e-9)
    p.msat[0], p.ku1[0], p.ku2[0] = 7e5, 4e5, -1.5e5
    p.anis_u[0] = np.array([1.0, 2.0, -0.5]) / np.linalg.norm([1.0, 2.0, -0.5])
    m = np.array([0.3, -0.2, 0.9])
    m /= np.linalg.norm(m)
    u = p.anis_u[0]

    def edens(v):
        c = u @ v
        return -4e5 * c * c + 1.5e5 * c ** 4

    h = 1e-6
    grad = np.array([(edens(m + h * e) - edens(m - h * e)) / (2 * h) for e in np.eye(3)])
    a1, a2 = anisotropy_field_parts(p, m.reshape(3, 1, 1, 1))
    B = (a1 + a2)[:, 0, 0, 0]
    assert np.allclose(B, -grad / 7e5, rtol=1e-7)
