"""Failure detection on the GPU without a fault: the row-stage kernels' bounded
waits on their tensor copies.  With the context's wait limit at 0 cycles the
first wait gives up at once, the kernel records MM_ERR_TIMEOUT, waits for its
copies still in flight with the default limit and returns; mm_step reports
the error, m, t and dt are those before the abandoned attempt, and with the
default limit restored the context continues bit for bit as one that never
timed out."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1406_7635_gb300.workloads import Problem, normalise  # noqa: E402

MM_ERR_TIMEOUT = -6
DEFAULT_WAIT = 1 << 30


@pytest.fixture(scope="module")
def mm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1406_7635_gb300.build import build
    build()
    from paper_1406_7635_gb300 import mm as _mm
    return _mm


def tensor_copy_problem():
    """20 x 30 x 4 cells of 2 nm, three regions with vacuum: rows of 32
    complex values, 8 rows per block, ny even and nx a multiple of 4, so the
    row kernels move the spectrum box and the stencil rows by tensor copies."""
    rng = np.random.default_rng(4242)
    shape = (4, 30, 20)
    p = Problem(20, 30, 4, 2e-9, 2e-9, 2e-9)
    p.pbc = (0, 0, 0)
    p.region = rng.integers(0, 3, size=shape).astype(np.uint8)
    for r in range(3):
        p.msat[r] = rng.uniform(6e5, 1.1e6)
        p.aex[r] = rng.uniform(1.0e-11, 1.6e-11)
        p.alpha[r] = rng.uniform(0.05, 0.3)
        p.b0[r] = rng.uniform(-0.03, 0.03, 3)
    p.mask = (rng.uniform(size=shape) > 0.05).astype(np.uint8)
    p.m0 = normalise(rng.standard_normal((3,) + shape), p.magnetic())
    return p


def test_wait_limit_argument_and_default(mm):
    p = tensor_copy_problem()
    ctx = mm.Context.from_problem(p)
    assert ctx.get_wait_limit() == DEFAULT_WAIT
    with pytest.raises(mm.MMError) as ei:
        ctx.set_wait_limit(-1)
    assert ei.value.code == -1
    assert ctx.get_wait_limit() == DEFAULT_WAIT
    ctx.close()


def test_expired_wait_reports_timeout_and_context_stays_usable(mm):
    p = tensor_copy_problem()
    ref = mm.Context.from_problem(p)
    ref.step(3)
    m_ref, t_ref, s_ref = ref.get_m(), ref.get_time(), ref.get_stats()
    ref.close()

    ctx = mm.Context.from_problem(p)
    ctx.step(1)
    m1, t1, s1 = ctx.get_m(), ctx.get_time(), ctx.get_stats()
    ctx.set_wait_limit(0)
    for _ in range(2):   # the error path twice in a row
        with pytest.raises(mm.MMError) as ei:
            ctx.step(1)
        assert ei.value.code == MM_ERR_TIMEOUT
        assert "wait" in str(ei.value)
        assert np.array_equal(ctx.get_m(), m1)
        assert ctx.get_time() == t1
        s = ctx.get_stats()
        assert (s["accepted"], s["rejected"]) == (s1["accepted"], s1["rejected"])
    ctx.set_wait_limit(DEFAULT_WAIT)
    ctx.step(2)
    assert np.array_equal(ctx.get_m(), m_ref)
    assert ctx.get_time() == t_ref
    s = ctx.get_stats()
    assert (s["accepted"], s["rejected"]) == (s_ref["accepted"], s_ref["rejected"])
    ctx.close()
