"""Seeded synthetic inputs: problem descriptions and initial magnetisations.

This module builds inputs only -- grids, geometry masks, region maps,
per-region parameter tables and initial states -- and holds none of the
method's arithmetic (no fields, torques or time stepping).  It is the one
module that both the CUDA path's tests/bench and the CPU oracle read.

The workloads mirror the paper's own synthetic set-ups: an SP4-like permalloy
film (Sec. V, standard problem 4), a grainy film with Voronoi regions
(Sec. VI, "Voronoi tessellation") and a 3-D ellipsoid in a vortex state.
Random draws use numpy's PCG64 generator, whose stream is identical on every
platform.
"""
from dataclasses import dataclass, field
import numpy as np

MU0 = 4e-7 * np.pi
GAMMA_LL = 1.7595e11           # rad/(T s), the paper's default gyromagnetic ratio
SEED_BASE = 1406763500


def _zeros256(*shape):
    return np.zeros((256,) + shape, dtype=np.float64)


@dataclass
class Problem:
    """A finite-difference micromagnet: grid, materials, excitation, state.

    Arrays are in (z, y, x) order with x fastest; vectors carry a leading
    component axis of length 3.  Per-region tables have 256 entries (region
    indices 0..255).  B_ext(region, t) = b0 + b1 * sin(2 pi freq t + phase).
    """
    nx: int
    ny: int
    nz: int
    dx: float
    dy: float
    dz: float
    mask: np.ndarray = None        # uint8 (nz, ny, nx); 0 = vacuum
    region: np.ndarray = None      # uint8 (nz, ny, nx)
    msat: np.ndarray = field(default_factory=lambda: _zeros256())
    aex: np.ndarray = field(default_factory=lambda: _zeros256())
    alpha: np.ndarray = field(default_factory=lambda: _zeros256())
    gamma: np.ndarray = field(default_factory=lambda: np.full(256, GAMMA_LL))
    ku1: np.ndarray = field(default_factory=lambda: _zeros256())
    ku2: np.ndarray = field(default_factory=lambda: _zeros256())
    dind: np.ndarray = field(default_factory=lambda: _zeros256())   # interfacial DMI constant D (J/m^2)
    # spin-transfer torque parameters per region: current density (A/m^2),
    # Zhang-Li non-adiabaticity xi; Slonczewski polarisation P, Lambda,
    # secondary parameter eps', fixed-layer direction and free-layer thickness
    jcur: np.ndarray = field(default_factory=lambda: _zeros256(3))
    xi: np.ndarray = field(default_factory=lambda: _zeros256())
    pol: np.ndarray = field(default_factory=lambda: _zeros256())
    lam: np.ndarray = field(default_factory=lambda: np.ones(256))
    epsp: np.ndarray = field(default_factory=lambda: _zeros256())
    mp: np.ndarray = field(default_factory=lambda: np.tile([0.0, 0.0, 1.0], (256, 1)))
    tfree: np.ndarray = field(default_factory=lambda: _zeros256())
    zhang_li: bool = False
    slonczewski: bool = False
    anis_u: np.ndarray = field(default_factory=lambda: np.tile([1.0, 0.0, 0.0], (256, 1)))
    exch_scale: np.ndarray = field(default_factory=lambda: np.ones((256, 256)))
    b0: np.ndarray = field(default_factory=lambda: _zeros256(3))
    b1: np.ndarray = field(default_factory=lambda: _zeros256(3))
    freq: float = 0.0
    phase: float = 0.0
    demag: bool = True
    exch: bool = True
    anis: bool = True
    zeeman: bool = True
    precession: bool = True
    pbc: tuple = (0, 0, 0)         # periodic images on each side along x, y, z (0 = open)
    m0: np.ndarray = None          # float64 (3, nz, ny, nx), unit or zero
    # solver settings (Sec. IV: MaxErr default 1e-5, headroom 0.8)
    max_err: float = 1e-5
    headroom: float = 0.8
    dt0: float = 1e-14
    dt_min: float = 1e-20
    dt_max: float = 1e-10

    def __post_init__(self):
        shp = (self.nz, self.ny, self.nx)
        if self.mask is None:
            self.mask = np.ones(shp, dtype=np.uint8)
        if self.region is None:
            self.region = np.zeros(shp, dtype=np.uint8)
        if self.m0 is None:
            self.m0 = np.zeros((3,) + shp)
            self.m0[0] = 1.0

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def ncells(self):
        return self.nx * self.ny * self.nz

    def magnetic(self):
        """Cells that carry a magnetisation: inside the mask with Msat > 0."""
        return (self.mask != 0) & (self.msat[self.region] > 0)


def normalise(v, keep):
    """Unit vectors where ``keep``; zero elsewhere (input construction)."""
    n = np.sqrt((v * v).sum(axis=0))
    out = np.where(keep[None] & (n[None] > 0), v / np.where(n > 0, n, 1.0)[None], 0.0)
    return out


def random_unit(rng, shape):
    """Uniform directions on the unit sphere (normalised Gaussian triples)."""
    v = rng.standard_normal((3,) + shape)
    return v / np.sqrt((v * v).sum(axis=0))[None]


# ---------------------------------------------------------------------------
# The three plain-method workloads.
# ---------------------------------------------------------------------------
def film_sp4(nx=64, ny=16, seed=SEED_BASE + 0):
    """SP4-like permalloy film: nx x ny x 1 cells of 4 x 4 x 3 nm.

    Msat 8e5 A/m, Aex 1.3e-11 J/m, alpha 0.02, no anisotropy, static field
    (-24.6, 4.3, 0) mT.  m0 = (1, 1, 0.1) normalised plus N(0, 0.05) noise per
    component, renormalised.
    """
    rng = np.random.default_rng(seed)
    p = Problem(nx, ny, 1, 4e-9, 4e-9, 3e-9)
    p.msat[0], p.aex[0], p.alpha[0] = 8e5, 1.3e-11, 0.02
    p.anis = False
    p.b0[0] = (-24.6e-3, 4.3e-3, 0.0)
    base = np.array([1.0, 1.0, 0.1]) / np.linalg.norm([1.0, 1.0, 0.1])
    m = base[:, None, None, None] + 0.05 * rng.standard_normal((3,) + p.shape)
    p.m0 = normalise(m, p.magnetic())
    return p


def voronoi_regions(nx, ny, dx, dy, ngrains, rng):
    """Nearest-centre grain map of an nx x ny film (no wrap; ties to lower index)."""
    cx = rng.uniform(0.0, nx * dx, ngrains)
    cy = rng.uniform(0.0, ny * dy, ngrains)
    x = (np.arange(nx) + 0.5) * dx
    y = (np.arange(ny) + 0.5) * dy
    d2 = (x[None, None, :] - cx[:, None, None]) ** 2 + (y[None, :, None] - cy[:, None, None]) ** 2
    return np.argmin(d2, axis=0).astype(np.uint8)   # argmin returns the first minimum


def grain_film(nx=256, ny=256, ngrains=64, seed=SEED_BASE + 1):
    """Film of nx x ny x 1 cells of 2 x 2 x 1 nm with Voronoi grains.

    Per grain: Ku1 ~ U[0.5, 1.5]e5 J/m^3, in-plane easy axis at a uniform
    angle.  Msat 1e6 A/m, Aex 1.5e-11 J/m, alpha 0.1; the exchange between two
    different grains is scaled by a factor ~ U[0.8, 1].  m0 uniform on the unit
    sphere per cell; B_ext = 10 mT sin(2 pi 1 GHz t) along x.
    """
    rng = np.random.default_rng(seed)
    p = Problem(nx, ny, 1, 2e-9, 2e-9, 1e-9)
    p.region = voronoi_regions(nx, ny, p.dx, p.dy, ngrains, rng)[None]
    g = np.arange(ngrains)
    p.msat[g], p.aex[g], p.alpha[g] = 1e6, 1.5e-11, 0.1
    p.ku1[g] = rng.uniform(0.5e5, 1.5e5, ngrains)
    phi = rng.uniform(0.0, 2 * np.pi, ngrains)
    p.anis_u[g] = np.stack([np.cos(phi), np.sin(phi), np.zeros(ngrains)], axis=1)
    S = np.ones((256, 256))
    iu = np.triu_indices(ngrains, k=1)
    s = rng.uniform(0.8, 1.0, iu[0].size)
    S[iu] = s
    S[(iu[1], iu[0])] = s
    p.exch_scale = S
    p.b1[g] = (10e-3, 0.0, 0.0)
    p.freq = 1e9
    p.m0 = normalise(random_unit(rng, p.shape), p.magnetic())
    return p


def ellipsoid_vortex(nx=128, ny=128, nz=32, c=3e-9, seed=SEED_BASE + 2):
    """3-D grid of c-sized cubes with an inscribed ellipsoid mask, vortex state.

    Semi-axes are half the box (192, 192, 48 nm at 128 x 128 x 32, 3 nm).
    Msat 8e5 A/m, Aex 1.3e-11 J/m, alpha 0.01, no field.  m0: circulation +1,
    polarity +1 vortex m ~ (-y, x, r_c) / |.| about the box centre with
    r_c = 2 cells, plus N(0, 0.02) noise per component, renormalised.
    """
    rng = np.random.default_rng(seed)
    p = Problem(nx, ny, nz, c, c, c)
    x = (np.arange(nx) + 0.5) * c - 0.5 * nx * c
    y = (np.arange(ny) + 0.5) * c - 0.5 * ny * c
    z = (np.arange(nz) + 0.5) * c - 0.5 * nz * c
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    ax, ay, az = 0.5 * nx * c, 0.5 * ny * c, 0.5 * nz * c
    p.mask = ((X / ax) ** 2 + (Y / ay) ** 2 + (Z / az) ** 2 <= 1.0).astype(np.uint8)
    p.msat[0], p.aex[0], p.alpha[0] = 8e5, 1.3e-11, 0.01
    p.anis = False
    p.zeeman = False
    rc = 2 * c
    m = np.stack([-Y, X, np.full_like(X, rc)])
    m = m / np.sqrt((m * m).sum(axis=0))[None]
    m = m + 0.02 * rng.standard_normal(m.shape)
    p.m0 = normalise(m, p.magnetic())
    return p


def film_surrogate(nx=512, ny=512, seed=SEED_BASE + 4):
    """Film of nx x ny x 1 cells of 2 x 2 x 2 nm for the learned demag
    surrogate: Msat 8e5 A/m, Aex 1.3e-11 J/m, alpha 0.02, no anisotropy, a
    static 20 mT field along (1, 1, 0)/sqrt 2; m0 uniform on the sphere."""
    rng = np.random.default_rng(seed)
    p = Problem(nx, ny, 1, 2e-9, 2e-9, 2e-9)
    p.msat[0], p.aex[0], p.alpha[0] = 8e5, 1.3e-11, 0.02
    p.anis = False
    p.b0[0] = (20e-3 / np.sqrt(2.0), 20e-3 / np.sqrt(2.0), 0.0)
    p.m0 = normalise(random_unit(rng, p.shape), p.magnetic())
    return p


WORKLOADS = {
    "film_64x16x1": lambda: film_sp4(64, 16),
    "grains_256x256x1": lambda: grain_film(256, 256, 64),
    "ellipsoid_128x128x32": lambda: ellipsoid_vortex(128, 128, 32),
    "film_512x512x1": lambda: film_surrogate(512, 512),
}


# ---------------------------------------------------------------------------
# Batched workload: many independent instances of uneven sizes.
# ---------------------------------------------------------------------------
BATCH_SHAPES = ((32, 32, 1), (64, 32, 1), (128, 64, 2), (96, 96, 4))


def batch_instances(n=512, shapes=BATCH_SHAPES, cell=4e-9, seed=SEED_BASE + 3):
    """n instance descriptions: grid drawn uniformly from `shapes` (nx, ny,
    nz) with cubic cells; Msat ~ U[4e5, 1.2e6] A/m, Aex ~ U[0.8, 2]e-11 J/m,
    alpha ~ U[0.005, 0.5]; a static field of uniform direction and magnitude
    ~ U[0, 50] mT; m0 uniform on the unit sphere per cell.  Returns (specs,
    m0s): dicts for the batched API and float64 arrays (3, nz, ny, nx)."""
    rng = np.random.default_rng(seed)
    specs, m0s = [], []
    for _ in range(n):
        nx, ny, nz = shapes[rng.integers(len(shapes))]
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        spec = {"nx": int(nx), "ny": int(ny), "nz": int(nz), "dx": cell, "dy": cell, "dz": cell,
                "msat": float(rng.uniform(4e5, 1.2e6)), "aex": float(rng.uniform(0.8e-11, 2e-11)),
                "alpha": float(rng.uniform(0.005, 0.5)), "gamma_ll": GAMMA_LL,
                "bext": (d * rng.uniform(0.0, 50e-3)).tolist()}
        specs.append(spec)
        m0s.append(random_unit(rng, (nz, ny, nx)))
    return specs, m0s


def problem_from_instance(spec, m0):
    """The single-grid Problem equivalent to one batched instance."""
    p = Problem(spec["nx"], spec["ny"], spec["nz"], spec["dx"], spec["dy"], spec["dz"])
    p.msat[0], p.aex[0], p.alpha[0] = spec["msat"], spec["aex"], spec["alpha"]
    p.gamma[0] = spec.get("gamma_ll", GAMMA_LL)
    p.b0[0] = spec["bext"]
    p.anis = False
    p.m0 = np.asarray(m0, dtype=np.float64)
    return p
