"""Magnetostatic field B_demag = K * M (Sec. III.B, "Magnetostatic convolution").

B_demag,i(r) = -mu0 * sum_r' N_ij(r - r') M_j(r'),  M = Msat * m,

with N the positive cell-averaged tensor of ``oracle.newell`` (B = -mu0 N M for
a uniformly magnetised body).  Two evaluations of the same discrete sum:

* ``demag_direct``: the O(N^2) double loop written out (tiny grids only);
* ``demag_fft``: the convolution theorem on a zero-padded grid.  Each axis of
  length n is padded to 2n - 1 (n = 1 stays 1), the smallest size at which the
  cyclic convolution equals the linear one; numpy's FFT is the library
  primitive.
"""
import numpy as np

from .newell import demag_tensor, demag_tensor_full

MU0 = 4e-7 * np.pi   # T m / A, the value used throughout the paper's scripts

# component pairs (i, j) -> index into the 6-component tensor
_IDX = {(0, 0): 0, (1, 1): 1, (2, 2): 2, (0, 1): 3, (1, 0): 3,
        (0, 2): 4, (2, 0): 4, (1, 2): 5, (2, 1): 5}


def magnetisation(msat_cell, m):
    """M = Msat m per cell; m has shape (3, nz, ny, nx), msat_cell (nz, ny, nx)."""
    return msat_cell[None] * m


def demag_direct(M, dx, dy, dz):
    """Direct O(N^2) summation of -mu0 N(r_i - r_j) M_j over every cell pair."""
    _, nz, ny, nx = M.shape
    zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    pos = np.stack([xx.ravel(), yy.ravel(), zz.ravel()], axis=1)        # (N, 3)
    d = pos[:, None, :] - pos[None, :, :]                                 # (N, N, 3)
    Nt = demag_tensor(d[..., 0], d[..., 1], d[..., 2], dx, dy, dz)     # 6 x (N, N)
    Mf = M.reshape(3, -1)
    B = np.zeros_like(Mf)
    for i in range(3):
        for j in range(3):
            B[i] -= MU0 * (Nt[_IDX[(i, j)]] @ Mf[j])
    return B.reshape(M.shape)


def padded_sizes(nx, ny, nz):
    return tuple(2 * n - 1 for n in (nx, ny, nz))


def kernel_spectrum(nx, ny, nz, dx, dy, dz):
    """FFT of the zero-padded tensor, offset (X,Y,Z) stored at index mod P."""
    Px, Py, Pz = padded_sizes(nx, ny, nz)
    full = demag_tensor_full(nx, ny, nz, dx, dy, dz)   # offsets -(n-1)..(n-1)
    # move offset 0 to index 0 (negative offsets wrap to the top of the axis)
    wrapped = np.roll(full, shift=(-(nz - 1), -(ny - 1), -(nx - 1)), axis=(1, 2, 3))
    assert wrapped.shape[1:] == (Pz, Py, Px)
    return np.fft.fftn(wrapped, axes=(1, 2, 3))


def demag_fft(M, dx, dy, dz, spectrum=None):
    """Zero-padded FFT convolution; returns B_demag with the shape of M."""
    _, nz, ny, nx = M.shape
    Px, Py, Pz = padded_sizes(nx, ny, nz)
    K = kernel_spectrum(nx, ny, nz, dx, dy, dz) if spectrum is None else spectrum
    Mh = np.fft.fftn(M, s=(Pz, Py, Px), axes=(1, 2, 3))
    B = np.zeros_like(M)
    for i in range(3):
        acc = np.zeros(Mh.shape[1:], dtype=complex)
        for j in range(3):
            acc += K[_IDX[(i, j)]] * Mh[j]
        B[i] = -MU0 * np.fft.ifftn(acc, axes=(0, 1, 2)).real[:nz, :ny, :nx]
    return B
