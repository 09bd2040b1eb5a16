"""The two implementations of the (y, z) part of the fused demag convolution
(Sec. III.B) against the float64 oracle: the cluster kernel (one
thread-block cluster per kx plane, residue classes across the cluster) and
the register-resident kernels (3-D: y forward into a y-transformed buffer;
per (kx, ky) column z forward, kernel product and z inverse in registers; y
inverse.  2-D: y forward, product and y inverse of a kx plane in one
block).

Grids cover every z class length of the column kernel (pz = 16, 32, 64),
y rows of 64, 128 and 256 padded points, ny and nz below their class
lengths (pruned inputs, cropped outputs), odd ny, vacuum cells and three
regions.  Bars: fields 5e-6 of the maximum, m 1e-5 after replayed steps."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.field import Field  # noqa: E402
from oracle.rk45 import RK45  # noqa: E402
from paper_1406_7635_gb300.workloads import Problem, normalise  # noqa: E402

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


def grid_problem(shape, seed):
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape
    p = Problem(nx, ny, nz, 2e-9, 2.5e-9, 1.5e-9)
    p.pbc = (0, 0, 0)
    p.region = rng.integers(0, 3, size=shape).astype(np.uint8)
    for r in range(3):
        p.msat[r] = rng.uniform(6e5, 1.1e6)
        p.aex[r] = rng.uniform(1.0e-11, 1.6e-11)
        p.alpha[r] = rng.uniform(0.05, 0.3)
        p.ku1[r] = rng.uniform(-1e5, 3e5)
        u = rng.standard_normal(3)
        p.anis_u[r] = u / np.linalg.norm(u)
        p.b0[r] = rng.uniform(-0.03, 0.03, 3)
    p.mask = (rng.uniform(size=shape) > 0.05).astype(np.uint8)
    p.m0 = normalise(rng.standard_normal((3,) + shape), p.magnetic())
    return p


# (nz, ny, nx): pz = 16 with py = 64; pz = 32 with py = 128 and odd ny; pz = 64
# with py = 256 and ny below 128 (the smoke grid); nz = 20 < 32 with pz = 64;
# py = 512 (rows of 256 points per parity class) with ny = 130
SHAPES = [(8, 20, 24), (12, 47, 40), (32, 78, 68), (20, 64, 36), (16, 130, 24),
          # 2-D films: the one-kernel (y, K, y^-1) path with rows of 64, 128
          # and 256 points per class (odd ny, ny below the class length)
          (1, 60, 100), (1, 97, 64), (1, 256, 256)]


@pytest.mark.parametrize("shape", SHAPES)
def test_both_yz_paths_match_oracle_field(mm, shape):
    p = grid_problem(shape, seed=sum(shape))
    f = Field(p)
    m32 = p.m0.astype(np.float32).astype(np.float64)
    ref = f.terms(m32, 0.0)["demag"]
    scale = np.abs(ref).max()
    out = {}
    for which in (1, 2):
        ctx = mm.Context.from_problem(p)
        assert ctx.set_yz_kernels(which) == which
        out[which] = ctx.get_bdemag().astype(np.float64)
        ctx.close()
        assert np.abs(out[which] - ref).max() <= FIELD_TOL * scale, which
    assert np.abs(out[1] - out[2]).max() <= FIELD_TOL * scale


@pytest.mark.parametrize("shape", SHAPES)
def test_three_kernel_path_replayed_steps(mm, shape):
    p = grid_problem(shape, seed=7 + sum(shape))
    ctx = mm.Context.from_problem(p)
    assert ctx.set_yz_kernels(2) == 2
    n = 6 if shape[0] * shape[1] * shape[2] < 40000 else 2
    ctx.step(n)
    m_gpu = ctx.get_m().astype(np.float64)
    dts = ctx.get_dt_history()
    ctx.close()
    ora = RK45(p, m=p.m0.astype(np.float32).astype(np.float64))
    ora.run_fixed(dts)
    assert np.abs(m_gpu - ora.m).max() <= M_TOL


def test_default_path_and_availability(mm):
    """3-D grids with 16 <= pz <= 64 step with the three kernels by default;
    thinner grids keep the cluster kernel and refuse the three-kernel path."""
    p = grid_problem((12, 47, 40), seed=3)
    ctx = mm.Context.from_problem(p)
    assert ctx.set_yz_kernels(0) == 2
    assert ctx.set_yz_kernels(1) == 1
    assert ctx.set_yz_kernels(0) == 2
    ctx.close()
    q = grid_problem((4, 30, 20), seed=4)     # pz = 8
    ctx = mm.Context.from_problem(q)
    assert ctx.set_yz_kernels(0) == 1
    with pytest.raises(mm.MMError) as ei:
        ctx.set_yz_kernels(2)
    assert ei.value.code == -1
    ctx.close()


def test_switching_paths_between_steps_keeps_the_trajectory(mm):
    """Stepping with one path, switching, stepping on: the same trajectory as
    one path throughout, within float32 rounding of the two transforms."""
    p = grid_problem((12, 47, 40), seed=11)
    a = mm.Context.from_problem(p)
    a.set_yz_kernels(1)
    a.step(8)                      # adaptive; b replays the same step sizes
    b = mm.Context.from_problem(p)
    b.set_fixed_dt_sequence(a.get_dt_history())
    b.set_yz_kernels(2)
    b.step(4)
    b.set_yz_kernels(1)
    b.step(4)
    assert np.abs(a.get_m().astype(np.float64) - b.get_m().astype(np.float64)).max() <= 5e-6
    a.close()
    b.close()
