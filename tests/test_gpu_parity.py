"""GPU (CUDA path through the C ABI) vs the float64 oracle, element by element.

Tolerances (float32 path against float64):
* fields: the float32 FFT convolution has a rounding error of order
  eps32 log2(N) relative to the largest field value (eps32 = 6e-8, N up to
  2^22), so fields and torques are compared with 5e-6 of their maximum;
* m after a replayed step sequence: 1e-5 (absolute, m has unit length);
* energies: 1e-5 relative to the largest energy term.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.demag import MU0, demag_fft  # noqa: E402
from oracle.energy import energies as ora_energies  # noqa: E402
from oracle.field import Field, effective_field, ll_torque  # noqa: E402
from oracle.newell import demag_tensor  # noqa: E402
from oracle.rk45 import RK45  # noqa: E402
from paper_1406_7635_gb300.workloads import Problem, ellipsoid_vortex, film_sp4, grain_film  # noqa: E402

FIELD_TOL = 5e-6
M_TOL = 1e-5


@pytest.fixture(scope="module")
def mm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1406_7635_gb300.build import build
    build()
    from paper_1406_7635_gb300 import mm as _mm
    return _mm


def random_problem(shape, cell, seed, regions=1, mask_frac=0.0):
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape
    p = Problem(nx, ny, nz, *cell)
    p.region = rng.integers(0, regions, size=shape).astype(np.uint8)
    for r in range(regions):
        p.msat[r] = rng.uniform(4e5, 1.2e6)
        p.aex[r] = rng.uniform(0.8e-11, 2e-11)
        p.alpha[r] = rng.uniform(0.01, 0.3)
        p.ku1[r] = rng.uniform(-2e5, 2e5)
        p.ku2[r] = rng.uniform(-5e4, 5e4)
        u = rng.standard_normal(3)
        p.anis_u[r] = u / np.linalg.norm(u)
        p.b0[r] = rng.uniform(-0.05, 0.05, 3)
        p.b1[r] = rng.uniform(-0.02, 0.02, 3)
    for r1 in range(regions):
        for r2 in range(r1 + 1, regions):
            p.exch_scale[r1, r2] = p.exch_scale[r2, r1] = rng.uniform(0.5, 1.0)
    p.freq, p.phase = 2.3e9, 0.7
    if mask_frac > 0:
        p.mask = (rng.uniform(size=shape) > mask_frac).astype(np.uint8)
    m = rng.standard_normal((3,) + shape)
    mag = p.magnetic()
    p.m0 = np.where(mag[None], m / np.sqrt((m * m).sum(0))[None], 0.0)
    return p


GRIDS = [
    ((1, 1, 1), (1e-9, 1e-9, 1e-9)),
    ((1, 1, 7), (2e-9, 1e-9, 1e-9)),
    ((2, 5, 3), (1e-9, 2e-9, 0.7e-9)),
    ((3, 1, 7), (3e-9, 3e-9, 3e-9)),
    ((1, 16, 64), (4e-9, 4e-9, 3e-9)),
    ((5, 9, 17), (2e-9, 3e-9, 4e-9)),
    ((4, 1, 1), (1e-9, 1e-9, 2e-9)),
    ((1, 33, 1), (1e-9, 1e-9, 1e-9)),
    ((6, 12, 20), (5e-9, 5e-9, 5e-9)),
    ((20, 64, 24), (3e-9, 3e-9, 3e-9)),     # fused path, residue split in z (2 blocks)
    ((3, 300, 20), (2e-9, 2e-9, 4e-9)),     # fused path, residue split in y (2 blocks)
    ((20, 100, 40), (3e-9, 3e-9, 2e-9)),    # fused path, split in y and z (4 blocks)
    ((40, 30, 9), (2e-9, 2e-9, 2e-9)),      # general path (pz too large for the fused plane)
    ((1, 3, 1024), (1e-9, 2e-9, 1e-9)),     # maximum nx (px = 2048, the twiddle table's length)
    ((1, 512, 6), (2e-9, 1e-9, 1e-9)),      # maximum ny
    ((512, 2, 3), (1e-9, 1e-9, 0.5e-9)),    # maximum nz
    ((2, 512, 512), (2e-9, 2e-9, 1e-9)),    # largest fused plane side (lx = 512, ly = 1024)
]


def test_demag_tensor_fp64_vs_oracle(mm):
    """a1: float64 tensor on the GPU against the oracle's float64 tensor,
    near (Newell) and far (quadrature) offsets, several cell shapes."""
    rng = np.random.default_rng(11)
    for cell in [(1e-9, 1e-9, 1e-9), (2e-9, 3e-9, 0.5e-9), (4e-9, 4e-9, 40e-9), (1.0, 1.0, 1 / 64)]:
        off = np.concatenate([rng.integers(-6, 7, (60, 3)), rng.integers(-200, 201, (60, 3)),
                              np.array([[0, 0, 0], [1, 0, 0], [0, 9, 0], [40, 0, 3], [7, 7, 7]])])
        g = mm.demag_tensor(off, *cell)
        o = np.stack(demag_tensor(off[:, 0], off[:, 1], off[:, 2], *cell), axis=1)
        scale = np.abs(o).max()
        assert np.abs(g - o).max() < 1e-11 * scale, np.abs(g - o).max() / scale


@pytest.mark.parametrize("shape,cell", GRIDS)
def test_bdemag_vs_oracle(mm, shape, cell):
    """a2-a4: the pruned R2C/C2R FFT convolution with the octant kernel
    against the oracle's zero-padded float64 FFT convolution (random M, some
    vacuum cells)."""
    p = random_problem(shape, cell, seed=sum(shape), regions=3, mask_frac=0.2)
    ctx = mm.Context.from_problem(p)
    b_gpu = ctx.get_bdemag().astype(np.float64)
    ctx.close()
    msat = np.where(p.magnetic(), p.msat[p.region], 0.0)
    m32 = p.m0.astype(np.float32).astype(np.float64)
    b_ora = demag_fft(msat[None] * m32, *cell)
    scale = np.abs(b_ora).max()
    assert np.abs(b_gpu - b_ora).max() <= FIELD_TOL * scale


@pytest.mark.parametrize("p6", range(0, 7))
def test_cube_demag_factor_gpu(mm, p6):
    """E2 (Table tabCube) on the GPU: a cube in 2^p x 2^p x 1 cells, -1/3."""
    a = 2 ** p6
    p = Problem(a, a, 1, 1.0 / a, 1.0 / a, 1.0)
    p.msat[0] = 1.0 / MU0
    ctx = mm.Context.from_problem(p)
    for comp in range(3):
        m = np.zeros((3, 1, a, a))
        m[comp] = 1.0
        ctx.set_m(m)
        b = ctx.get_bdemag()[comp].astype(np.float64).mean()
        assert abs(b + 1.0 / 3.0) < 2e-6
    ctx.close()


@pytest.mark.parametrize("i,n,nzz", [(1, 4, -0.76368), (4, 16, -0.94224), (16, 64, -0.98460),
                                      (64, 256, -0.99515), (128, 512, None)])
def test_film_table_gpu(mm, i, n, nzz):
    """E4a (Table tabPBC1, no-PBC column) on the GPU against the oracle's exact
    value and the printed value (within the paper's 1.3e-3 integration error)."""
    p = Problem(n, n, 1, 1e-9, 1e-9, 1e-9)
    p.msat[0] = 1.0 / MU0
    m = np.zeros((3, 1, n, n))
    m[2] = 1.0
    p.m0 = m
    ctx = mm.Context.from_problem(p)
    h = n // 2
    b = ctx.get_bdemag()[2, 0, h - 1:h + 1, h - 1:h + 1].astype(np.float64).mean()
    ctx.close()
    if n <= 256:
        M = np.zeros((3, 1, n, n))
        M[2] = 1.0 / MU0
        exact = demag_fft(M, 1e-9, 1e-9, 1e-9)[2, 0, h - 1:h + 1, h - 1:h + 1].mean()
        assert abs(b - exact) < 2e-6
    if nzz is not None:
        assert abs(b - nzz) < 1.5e-3


def test_long_range_dipole_gpu(mm):
    """E3 (Fig. figLong): single 1 nm cell, Bsat = 1 T on 512 x 1 x 1; the
    float32 field tracks the point dipole down to the ~1e-8 T noise floor."""
    n = 512
    p = Problem(n, 1, 1, 1e-9, 1e-9, 1e-9)
    p.mask = np.zeros((1, 1, n), dtype=np.uint8)
    p.mask[0, 0, 0] = 1
    p.msat[0] = 1.0 / MU0
    ctx = mm.Context.from_problem(p)
    b = ctx.get_bdemag()[0, 0, 0].astype(np.float64)
    ctx.close()
    r = np.arange(1, n) * 1e-9
    dip = 2e-27 / (4 * np.pi * r ** 3)
    err = np.abs(b[1:] - dip)
    assert np.all(err < 0.45 * (1e-9 / r) ** 4 * dip + 2e-8)


@pytest.mark.parametrize("which", ["film", "grains", "ellipsoid", "random"])
def test_beff_torque_energy_vs_oracle(mm, which):
    """a5-a7, a9: B_eff, torque and energies at a time with a non-zero
    excitation, against the oracle."""
    if which == "film":
        p = film_sp4(64, 16)
    elif which == "grains":
        p = grain_film(48, 40, 9)
    elif which == "ellipsoid":
        p = ellipsoid_vortex(24, 20, 8, c=3e-9)
        p.zeeman, p.anis = True, True
        p.b0[0] = (0.01, -0.02, 0.005)
        p.ku1[0] = 5e4
        p.anis_u[0] = (0.0, 0.6, 0.8)
    else:
        p = random_problem((3, 10, 13), (2e-9, 2e-9, 3e-9), seed=5, regions=4, mask_frac=0.15)
    t = 0.37e-9
    ctx = mm.Context.from_problem(p)
    ctx.set_time(t, 1e-13)
    B = ctx.get_beff().astype(np.float64)
    tau = ctx.get_torque().astype(np.float64)
    e = ctx.get_energies()
    ctx.close()
    m32 = p.m0.astype(np.float32).astype(np.float64)
    f = Field(p)
    terms = f.terms(m32, t)
    Bo = terms["total"]
    to = ll_torque(p, m32, Bo)
    assert np.abs(B - Bo).max() <= FIELD_TOL * np.abs(Bo).max()
    assert np.abs(tau - to).max() <= FIELD_TOL * np.abs(to).max()
    eo = ora_energies(p, m32, t, f)
    scale = max(abs(eo[k]) for k in ("demag", "exch", "anis", "zeeman"))
    for k in ("demag", "exch", "anis", "zeeman", "total"):
        assert abs(e[k] - eo[k]) <= 1e-5 * scale, (k, e[k], eo[k])
    assert np.allclose(e["m_avg"], eo["m_avg"], atol=1e-6)


def test_larmor_precession_gpu(mm):
    """E1: single spin in 0.1 T, alpha = 0, 3 ns of adaptive RK45: the error
    stays within (accepted steps) x MaxErr plus the float32 floor."""
    p = Problem(1, 1, 1, 1e-9, 1e-9, 1e-9)
    p.msat[0] = 1.0 / MU0
    p.b0[0] = (0.0, 0.0, 0.1)
    p.demag = p.exch = p.anis = False
    p.max_err = 1e-6
    ctx = mm.Context.from_problem(p)
    w = 1.7595e11 * 0.1
    for t_end in np.linspace(0.5e-9, 3e-9, 6):
        ctx.run(t_end)
        t, _ = ctx.get_time()
        assert t == t_end
        m = ctx.get_m()[:, 0, 0, 0].astype(np.float64)
        steps = ctx.get_stats()["accepted"]
        exact = np.array([np.cos(w * t_end), np.sin(w * t_end), 0.0])
        assert np.linalg.norm(m - exact) <= steps * p.max_err + 1e-5
    ctx.close()


@pytest.mark.parametrize("which,nsteps", [("film", 200), ("grains", 60), ("ellipsoid", 30), ("random", 60)])
def test_lockstep_vs_oracle(mm, which, nsteps):
    """Trajectory parity: GPU adaptive RK45 for n steps, then the oracle
    replays exactly the GPU's accepted step sizes; m must agree to 1e-5."""
    if which == "film":
        p = film_sp4(64, 16)
    elif which == "grains":
        p = grain_film(32, 32, 8)
    elif which == "ellipsoid":
        p = ellipsoid_vortex(16, 16, 4, c=3e-9)
    else:
        p = random_problem((2, 9, 11), (2e-9, 2e-9, 2e-9), seed=9, regions=3, mask_frac=0.1)
    ctx = mm.Context.from_problem(p)
    ctx.step(nsteps)
    m_gpu = ctx.get_m().astype(np.float64)
    dts = ctx.get_dt_history()
    t_gpu, _ = ctx.get_time()
    ctx.close()
    assert dts.size == nsteps
    ora = RK45(p, m=p.m0.astype(np.float32).astype(np.float64))
    ora.run_fixed(dts)
    assert abs(ora.t - t_gpu) <= 1e-12 * t_gpu
    assert np.abs(m_gpu - ora.m).max() <= M_TOL


def test_fixed_sequence_mode(mm):
    """mm_set_fixed_dt_sequence replays given steps; replaying the GPU's own
    adaptive history on a fresh context reproduces m bit for bit."""
    p = film_sp4(32, 8)
    a = mm.Context.from_problem(p)
    a.step(25)
    dts = a.get_dt_history()
    ma = a.get_m()
    a.close()
    b = mm.Context.from_problem(p)
    b.set_fixed_dt_sequence(dts)
    b.step(1000)     # stops when the sequence is used up
    assert b.get_stats()["accepted"] == 25
    assert np.array_equal(b.get_m(), ma)
    b.close()


def test_checkpoint_resume_bit_exact(mm):
    p = grain_film(32, 24, 6)
    a = mm.Context.from_problem(p)
    a.step(10)
    blob = a.get_state()
    a.step(15)
    m1, t1 = a.get_m(), a.get_time()
    a.set_state(blob)
    a.step(15)
    assert np.array_equal(a.get_m(), m1) and a.get_time() == t1
    b = mm.Context.from_problem(p)
    b.set_state(blob)
    b.step(15)
    assert np.array_equal(b.get_m(), m1)
    a.close()
    b.close()


def test_energy_conservation_and_dissipation_gpu(mm):
    p = film_sp4(32, 8)
    p.alpha[0] = 0.0
    p.max_err = 1e-6
    ctx = mm.Context.from_problem(p)
    e0 = ctx.get_energies()["total"]
    drift = 0.0
    for _ in range(10):
        ctx.step(20)
        drift = max(drift, abs(ctx.get_energies()["total"] - e0))
    assert drift < 1e-4 * abs(e0)
    ctx.close()
    p.alpha[0] = 0.5
    ctx = mm.Context.from_problem(p)
    prev = ctx.get_energies()["total"]
    for _ in range(20):
        ctx.step(3)
        e = ctx.get_energies()["total"]
        assert e <= prev + 1e-6 * abs(prev)
        prev = e
    ctx.close()


def test_failure_paths_return_status(mm):
    """Non-finite m -> MM_ERR_NONFINITE; an impossible dt_min ->
    MM_ERR_DT_UNDERFLOW; stepping before m is set -> MM_ERR_STATE.  All
    detected from device state without faulting the GPU."""
    p = film_sp4(16, 4)
    ctx = mm.Context(16, 4, 1, 4e-9, 4e-9, 3e-9)
    with pytest.raises(mm.MMError) as ei:
        ctx.step(1)
    assert ei.value.code == -7
    ctx.close()
    ctx = mm.Context.from_problem(p)
    m = p.m0.copy()
    m[0, 0, 1, 1] = np.nan
    ctx.set_m(m)
    with pytest.raises(mm.MMError) as ei:
        ctx.step(3)
    assert ei.value.code == -4
    ctx.close()
    ctx = mm.Context.from_problem(p)
    ctx.set_solver(max_err=1e-12, headroom=0.8, dt0=1e-12, dt_min=1e-13, dt_max=1e-10)
    with pytest.raises(mm.MMError) as ei:
        ctx.step(5)
    assert ei.value.code == -5
    ctx.close()


def test_device_pointer_variants(mm):
    p = film_sp4(16, 8)
    ctx = mm.Context.from_problem(p)
    t = torch.tensor(p.m0.astype(np.float32), device="cuda").contiguous()
    ctx.set_m_device(t)
    ctx.step(5)
    out = torch.empty_like(t)
    ctx.get_m_device(out)
    assert np.array_equal(out.cpu().numpy(), ctx.get_m())
    ctx.close()
