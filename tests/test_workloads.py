"""The seeded input recipes keep the properties the benchmark and the tests
rely on: grid and cell sizes, material ranges, masks and regions, unit
magnetisation on magnetic cells (zero elsewhere), the vortex sense, and
determinism (the same arrays on every call)."""
import numpy as np
import pytest

from paper_1406_7635_gb300.workloads import BATCH_SHAPES, WORKLOADS, batch_instances


def unit_on_magnet(p):
    mag = p.magnetic()
    n = np.sqrt((p.m0 ** 2).sum(axis=0))
    return np.allclose(n[mag], 1.0, atol=1e-12) and np.all(p.m0[:, ~mag] == 0)


@pytest.mark.parametrize("name", sorted(WORKLOADS))
def test_recipes_are_deterministic_and_unit(name):
    a, b = WORKLOADS[name](), WORKLOADS[name]()
    assert np.array_equal(a.m0, b.m0)
    assert np.array_equal(a.region, b.region) and np.array_equal(a.mask, b.mask)
    assert unit_on_magnet(a)
    assert a.m0.shape == (3, a.nz, a.ny, a.nx)


def test_ellipsoid_mask_and_vortex():
    p = WORKLOADS["ellipsoid_128x128x32"]()
    assert (p.nx, p.ny, p.nz) == (128, 128, 32) and p.dx == p.dy == p.dz == 3e-9
    mag = p.magnetic()
    # inscribed ellipsoid: pi / 6 of the box up to the staircase (274 352 cells)
    assert int(mag.sum()) == 274352
    assert abs(mag.mean() - np.pi / 6) < 2e-3
    # circulation +1: m_y > 0 on the +x side of the centre plane, m_x < 0 on +y
    zc, yc, xc = 16, 64, 64
    assert p.m0[1, zc, yc, xc + 30] > 0.9 and p.m0[0, zc, yc + 30, xc] < -0.9
    # polarity +1 at the core
    assert p.m0[2, zc, yc, xc] > 0.8
    assert p.msat[0] == 8e5 and p.aex[0] == 1.3e-11 and p.alpha[0] == 0.01
    assert not p.zeeman and not p.anis


def test_grain_film_regions_and_materials():
    p = WORKLOADS["grains_256x256x1"]()
    assert (p.nx, p.ny, p.nz) == (256, 256, 1)
    g = np.unique(p.region)
    assert g.min() == 0 and g.max() <= 63 and len(g) >= 60   # 64 seeded centres, almost all own a cell
    assert np.all(p.ku1[:64] >= 0.5e5) and np.all(p.ku1[:64] <= 1.5e5)
    u = p.anis_u[:64]
    assert np.allclose(np.linalg.norm(u, axis=1), 1.0) and np.all(u[:, 2] == 0)
    S = p.exch_scale[:64, :64]
    off = ~np.eye(64, dtype=bool)
    assert np.array_equal(S, S.T) and np.all(np.diag(S) == 1.0)
    assert S[off].min() >= 0.8 and S[off].max() <= 1.0
    assert p.freq == 1e9 and np.allclose(p.b1[:64], [10e-3, 0.0, 0.0])


def test_sp4_film():
    p = WORKLOADS["film_64x16x1"]()
    assert (p.nx, p.ny, p.nz, p.dx, p.dy, p.dz) == (64, 16, 1, 4e-9, 4e-9, 3e-9)
    assert p.magnetic().all()
    mean = p.m0.reshape(3, -1).mean(axis=1)
    base = np.array([1.0, 1.0, 0.1]) / np.linalg.norm([1.0, 1.0, 0.1])
    assert np.dot(mean / np.linalg.norm(mean), base) > 0.999
    assert np.allclose(p.b0[0], [-24.6e-3, 4.3e-3, 0.0])


def test_batch_instances():
    specs, m0s = batch_instances()
    assert len(specs) == 512 and len(m0s) == 512
    shapes = {(s["nx"], s["ny"], s["nz"]) for s in specs}
    assert shapes == set(BATCH_SHAPES)   # every size is drawn
    for s, m in zip(specs, m0s):
        assert 4e5 <= s["msat"] <= 1.2e6 and 0.8e-11 <= s["aex"] <= 2e-11 and 0.005 <= s["alpha"] <= 0.5
        assert np.linalg.norm(s["bext"]) <= 50e-3
        assert m.shape == (3, s["nz"], s["ny"], s["nx"])
    assert np.allclose((m0s[0] ** 2).sum(axis=0), 1.0)
    again, _ = batch_instances()
    assert again == specs
