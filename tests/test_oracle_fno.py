"""Pins for the float64 FNO oracle: the truncated spectral operator reproduces
band-limited inputs exactly and equals numpy's FFT truncation on any input,
GELU matches the tabulated normal distribution, and every analytic gradient
matches central finite differences of the oracle's own loss."""
import numpy as np
import pytest

from oracle.fno import backward, dft_mats, forward, init_params, loss, spectral


def test_spectral_operator_passes_band_limited_modes():
    """With R = identity per mode, a real plane wave inside the kept modes
    comes out unchanged (DFT signs, 1/N scaling, the factor 2 on kx > 0 and
    the real part are all exercised); a mode outside is removed."""
    H, W, Mx, My, C = 16, 12, 4, 3, 2
    mats = dft_mats(H, W, Mx, My)
    R = np.zeros((C, C, 2 * My, Mx), dtype=complex)
    for i in range(C):
        R[i, i] = 1.0
    y, x = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    for (ky, kx) in [(0, 0), (1, 2), (-2, 3), (2, 0), (0, 3)]:
        v = np.stack([np.cos(2 * np.pi * (kx * x / W + ky * y / H) + 0.3),
                      np.sin(2 * np.pi * (kx * x / W + ky * y / H))])
        out, _ = spectral(v, R, mats)
        assert np.abs(out - v).max() < 1e-12, (ky, kx)
    v = np.cos(2 * np.pi * (5 * x / W))[None].repeat(C, 0)
    out, _ = spectral(v, R, mats)
    assert np.abs(out).max() < 1e-12


@pytest.fixture(scope="module")
def tiny():
    C, L, H, W, Mx, My = 4, 2, 8, 8, 3, 3
    rng = np.random.default_rng(3)
    params = init_params(C, L, Mx, My, seed=1)
    for k in list(params):
        if k.startswith("b") or k in ("p", "q"):
            params[k] = 0.1 * rng.standard_normal(params[k].shape)
    u = rng.standard_normal((3, H, W))
    y = rng.standard_normal((3, H, W))
    mats = dft_mats(H, W, Mx, My)
    return params, u, y, L, mats


def test_gradients_match_finite_differences(tiny):
    params, u, y, L, mats = tiny
    yhat, cache = forward(params, u, L, mats)
    g = backward(params, cache, yhat, y, L, mats)
    rng = np.random.default_rng(9)
    h = 1e-6
    for name, val in params.items():
        for _ in range(4):
            idx = tuple(rng.integers(s) for s in val.shape)
            for part in ((1.0,) if not np.iscomplexobj(val) else (1.0, 1j)):
                p2 = {k: v.copy() for k, v in params.items()}
                p2[name][idx] += h * part
                lp = loss(forward(p2, u, L, mats)[0], y)
                p2[name][idx] -= 2 * h * part
                lm = loss(forward(p2, u, L, mats)[0], y)
                fd = (lp - lm) / (2 * h)
                an = g[name][idx].real if part == 1.0 else g[name][idx].imag
                assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)) + 1e-9, (name, idx, part, fd, an)


def test_spectral_operator_is_the_fft_truncation():
    """With R = identity per mode, K v of any real input equals numpy's 2-D
    FFT with every mode outside {kx < Mx} x {ky < My or ky >= H - My} zeroed,
    the kept kx > 0 columns doubled (they stand for their conjugate
    partners), inverted and the real part taken."""
    H, W, Mx, My, C = 12, 10, 4, 3, 3
    mats = dft_mats(H, W, Mx, My)
    R = np.zeros((C, C, 2 * My, Mx), dtype=complex)
    for i in range(C):
        R[i, i] = 1.0
    v = np.random.default_rng(5).standard_normal((C, H, W))
    out, V = spectral(v, R, mats)
    mask = np.zeros((H, W))
    rows = list(range(My)) + list(range(H - My, H))
    for ky in rows:
        mask[ky, 0] = 1.0
        mask[ky, 1:Mx] = 2.0
    ref = np.real(np.fft.ifft2(np.fft.fft2(v) * mask[None]))
    assert np.abs(out - ref).max() < 1e-12
    # the cached coefficients are the FFT's at the kept modes
    assert np.abs(V - np.fft.fft2(v)[:, rows, :Mx]).max() < 1e-10


def test_gelu_against_the_normal_distribution():
    """GELU(x) = x Phi(x) with tabulated Phi(1) = 0.8413447460685429 and
    Phi(3) = 0.9986501019683699; its derivative matches central differences."""
    from oracle.fno import gelu, gelu_grad
    x = np.array([1.0, -1.0, 0.0, 3.0])
    want = np.array([0.8413447460685429, -(1 - 0.8413447460685429), 0.0, 3 * 0.9986501019683699])
    assert np.abs(gelu(x) - want).max() < 1e-15
    xs = np.linspace(-4, 4, 33)
    h = 1e-6
    fd = (gelu(xs + h) - gelu(xs - h)) / (2 * h)
    assert np.abs(gelu_grad(xs) - fd).max() < 1e-8
