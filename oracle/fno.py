"""Float64 oracle of the Fourier-neural-operator demag surrogate (forward and
backward), test infrastructure only.

The surrogate approximates u = m (3 channels on an H x W film) -> y =
B_demag / (mu0 Msat).  Architecture (a reading of the FNO named for the
learned form of the demag field; the paper has none):

  v_0 = P u + p                                   (lift, 3 -> C)
  v_{l+1} = act_l( W_l v_l + b_l + K_l v_l )      l = 0 .. L-1
  y = Q v_L + q                                   (project, C -> 3)

act_l = GELU (exact, with erf) for l < L-1, identity for the last layer.
K_l is the truncated spectral convolution, written with explicit partial DFT
matrices so that it is one well-defined real linear operator:

  V[i]   = Fy v[i] Fx^T          Fx[kx, x] = exp(-2 pi i kx x / W), kx < Mx
                                 Fy[j, y]  = exp(-2 pi i ky_j y / H),
                                 ky_j in {0..My-1} U {H-My..H-1}
  O[o]   = sum_i R[o, i] * V[i]  (per mode, complex weights)
  (K v)[o] = Re( Gy^T O[o] Gx )  Gx[kx, x] = c_kx exp(+2 pi i kx x / W) / W,
                                 c_0 = 1, c_kx = 2 (kx > 0),
                                 Gy[j, y] = exp(+2 pi i ky_j y / H) / H.

Loss: relative squared L2 over a batch, sum |yhat - y|^2 / sum |y|^2.
"""
import numpy as np
from math import erf, sqrt, pi

_erf = np.vectorize(erf)


def gelu(x):
    return 0.5 * x * (1.0 + _erf(x / sqrt(2.0)))


def gelu_grad(x):
    return 0.5 * (1.0 + _erf(x / sqrt(2.0))) + x * np.exp(-0.5 * x * x) / sqrt(2.0 * pi)


def ky_list(H, My):
    return np.concatenate([np.arange(My), np.arange(H - My, H)])


def dft_mats(H, W, Mx, My):
    x = np.arange(W)
    y = np.arange(H)
    kx = np.arange(Mx)
    ky = ky_list(H, My)
    Fx = np.exp(-2j * np.pi * np.outer(kx, x) / W)
    Fy = np.exp(-2j * np.pi * np.outer(ky, y) / H)
    c = np.where(kx == 0, 1.0, 2.0)
    Gx = c[:, None] * np.exp(2j * np.pi * np.outer(kx, x) / W) / W
    Gy = np.exp(2j * np.pi * np.outer(ky, y) / H) / H
    return Fx, Fy, Gx, Gy


def init_params(C, L, Mx, My, seed=0):
    """Random initial parameters (scaled so activations stay O(1))."""
    rng = np.random.default_rng(seed)
    p = {"P": rng.standard_normal((C, 3)) / np.sqrt(3), "p": np.zeros(C),
         "Q": rng.standard_normal((3, C)) / np.sqrt(C), "q": np.zeros(3)}
    for l in range(L):
        p[f"W{l}"] = rng.standard_normal((C, C)) / np.sqrt(C)
        p[f"b{l}"] = np.zeros(C)
        s = 1.0 / C
        p[f"R{l}"] = s * (rng.standard_normal((C, C, 2 * My, Mx)) + 1j * rng.standard_normal((C, C, 2 * My, Mx)))
    return p


def spectral(v, R, mats):
    Fx, Fy, Gx, Gy = mats
    V = np.einsum("jy,iyx,kx->ijk", Fy, v, Fx)           # (C, 2My, Mx)
    O = np.einsum("oijk,ijk->ojk", R, V)
    return np.real(np.einsum("jy,ojk,kx->oyx", Gy, O, Gx)), V


def forward(params, u, L, mats):
    """u: (3, H, W).  Returns yhat and the cache for backward."""
    cache = {"u": u}
    v = np.einsum("ci,ihw->chw", params["P"], u) + params["p"][:, None, None]
    cache["v0"] = v
    for l in range(L):
        s, V = spectral(v, params[f"R{l}"], mats)
        z = np.einsum("oi,ihw->ohw", params[f"W{l}"], v) + params[f"b{l}"][:, None, None] + s
        cache[f"V{l}"], cache[f"z{l}"] = V, z
        v = gelu(z) if l < L - 1 else z
        cache[f"v{l + 1}"] = v
    y = np.einsum("oc,chw->ohw", params["Q"], v) + params["q"][:, None, None]
    return y, cache


def loss(yhat, y):
    return float(np.sum((yhat - y) ** 2) / np.sum(y * y))


def backward(params, cache, yhat, y, L, mats):
    """Gradients of loss(yhat, y) with respect to every parameter."""
    Fx, Fy, Gx, Gy = mats
    g = {}
    dy = 2.0 * (yhat - y) / np.sum(y * y)
    vL = cache[f"v{L}"]
    g["Q"] = np.einsum("ohw,chw->oc", dy, vL)
    g["q"] = dy.sum(axis=(1, 2))
    dv = np.einsum("oc,ohw->chw", params["Q"], dy)
    for l in reversed(range(L)):
        z = cache[f"z{l}"]
        dz = dv * gelu_grad(z) if l < L - 1 else dv
        v = cache[f"v{l}"]
        g[f"W{l}"] = np.einsum("ohw,ihw->oi", dz, v)
        g[f"b{l}"] = dz.sum(axis=(1, 2))
        # s = Re(Gy^T O Gx): dO = conj(Gy) dz conj(Gx)^T (adjoint of Re-linear map)
        dO = np.einsum("jy,oyx,kx->ojk", np.conj(Gy), dz, np.conj(Gx))
        V = cache[f"V{l}"]
        # O = sum_i R V  ->  dR = dO conj(V), dV = sum_o conj(R) dO
        g[f"R{l}"] = np.einsum("ojk,ijk->oijk", dO, np.conj(V))
        dV = np.einsum("oijk,ojk->ijk", np.conj(params[f"R{l}"]), dO)
        # V = Fy v Fx^T (v real): dv = Re(Fy^H dV conj(Fx))
        dv = np.einsum("oi,ohw->ihw", params[f"W{l}"], dz)
        dv = dv + np.real(np.einsum("jy,ijk,kx->iyx", np.conj(Fy), dV, np.conj(Fx)))
    g["P"] = np.einsum("chw,ihw->ci", dv, cache["u"])
    g["p"] = dv.sum(axis=(1, 2))
    return g
