"""Pins for the float64 FNO oracle: the truncated spectral operator reproduces
band-limited inputs exactly, and every analytic gradient matches central
finite differences of the oracle's own loss."""
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
