"""Pins for the oracle's periodic boundary conditions (Sec. III.B, "Periodic
boundary conditions"): the macro-geometry demag against brute-force image
sums and against the printed PBC columns of Tables tabPBC1 and tabPBC2, and
the stencils' wrap-around against closed forms."""
import os

import numpy as np
import pytest

from oracle.demag import MU0, demag_direct, demag_fft
from oracle.dmi import dmi_field
from oracle.energy import energies
from oracle.field import exchange_field
from paper_1406_7635_gb300.workloads import Problem

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def read_table(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


@pytest.mark.parametrize("shape,pbc", [((2, 3, 4), (1, 0, 0)), ((2, 3, 4), (2, 1, 0)),
                                       ((3, 2, 2), (1, 2, 1)), ((1, 3, 5), (3, 2, 0)),
                                       ((4, 1, 1), (0, 0, 2))])
def test_periodic_fft_equals_image_sum(shape, pbc):
    """Brute force: every image of every source cell whose offset lies in the
    window -P N < D < P N, summed pair by pair, equals the cyclic FFT
    convolution with the image-summed tensor (1e-12 relative)."""
    rng = np.random.default_rng(sum(shape) + sum(pbc))
    M = rng.standard_normal((3,) + shape)
    a = demag_direct(M, 1e-9, 1.5e-9, 0.8e-9, pbc)
    b = demag_fft(M, 1e-9, 1.5e-9, 0.8e-9, pbc=pbc)
    assert np.abs(a - b).max() <= 1e-12 * np.abs(a).max()


@pytest.mark.parametrize("row", read_table("table_film_pbc.txt"))
def test_film_pbc_table(row):
    """Table tabPBC1, PBC column: 2 x 2 x 1 film, P images each side in x and
    y.  Within 1.5e-3, the deviation of the paper's numerically integrated
    kernel from the exact one (the same bound as the no-PBC column)."""
    P, nzz = int(row[0]), float(row[1])
    M = np.zeros((3, 1, 2, 2))
    M[2] = 1.0
    B = demag_fft(M, 1e-9, 1e-9, 1e-9, pbc=(P, P, 0))
    assert abs(B[2].mean() / MU0 - nzz) < 1.5e-3


@pytest.mark.parametrize("row", read_table("table_rod_pbc.txt"))
def test_rod_pbc_table(row):
    """Table tabPBC2, PBC column: rod periodic along z, m along x."""
    P, nxx = int(row[0]), float(row[1])
    M = np.zeros((3, 1, 2, 2))
    M[0] = 1.0
    B = demag_fft(M, 1e-9, 1e-9, 1e-9, pbc=(0, 0, P))
    assert abs(B[0].mean() / MU0 - nxx) < 5e-4


def test_periodic_exchange_spiral_energy():
    """A planar spiral closing on itself around a periodic chain (angle
    theta = 2 pi k / N per cell): every one of the N bonds is a bulk bond, so
    the exchange energy is exactly N Delta^3 2 Aex (1 - cos theta) / Delta^2,
    and every cell feels the same field (2 Aex/Msat)(2 cos theta - 2) m /
    Delta^2."""
    n, d, A, ms, k = 12, 1e-9, 1.3e-11, 8e5, 5
    p = Problem(n, 1, 1, d, d, d)
    p.msat[0], p.aex[0] = ms, A
    p.pbc = (1, 0, 0)
    th = 2 * np.pi * k / n
    phi = th * np.arange(n)
    m = np.zeros((3, 1, 1, n))
    m[0, 0, 0] = np.cos(phi)
    m[1, 0, 0] = np.sin(phi)
    B = exchange_field(p, m)
    expect = (2 * A / ms) * (2 * np.cos(th) - 2) * m / d ** 2
    assert np.abs(B - expect).max() <= 1e-12 * np.abs(expect).max()
    p.demag = p.anis = p.zeeman = False
    e = energies(p, m, 0.0)["exch"]
    assert abs(e - n * d ** 3 * 2 * A * (1 - np.cos(th)) / d ** 2) < 1e-12 * abs(e)


def test_periodic_dmi_cycloid_everywhere():
    """With x and y periodic there is no boundary: a cycloid closing on
    itself has the interior closed form B_DM = -(2D/Msat)(sin(k d)/d) m in
    every cell."""
    n, d, D, ms = 16, 1e-9, 3e-3, 1.1e6
    p = Problem(n, 1, 1, d, d, d)
    p.msat[0], p.aex[0], p.dind[0] = ms, 1.5e-11, D
    p.pbc = (1, 1, 0)
    k = 2 * np.pi * 3 / (n * d)
    x = (np.arange(n) + 0.5) * d
    m = np.zeros((3, 1, 1, n))
    m[0, 0, 0] = np.sin(k * x)
    m[2, 0, 0] = np.cos(k * x)
    B = dmi_field(p, m)
    expect = -(2 * D / ms) * (np.sin(k * d) / d) * m
    assert np.abs(B - expect).max() < 1e-9 * (2 * D / ms) * np.sin(k * d) / d
