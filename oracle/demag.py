"""Magnetostatic field B_demag = K * M (Sec. III.B, "Magnetostatic convolution").

B_demag,i(r) = -mu0 * sum_r' N_ij(r - r') M_j(r'),  M = Msat * m,

with N the positive cell-averaged tensor of ``oracle.newell`` (B = -mu0 N M for
a uniformly magnetised body).  Two evaluations of the same discrete sum:

* ``demag_direct``: the O(N^2) double loop written out (tiny grids only);
* ``demag_fft``: the convolution theorem on a zero-padded grid.  Each axis of
  length n is padded to 2n - 1 (n = 1 stays 1), the smallest size at which the
  cyclic convolution equals the linear one; numpy's FFT is the library
  primitive.

Periodic boundary conditions (Sec. III.B, "Periodic boundary conditions"):
P additional images of the box on each side of a periodic axis (the macro
geometry).  Reading: a source image contributes when its offset D from the
target cell along that axis lies in the window -P N < D < P N (N cells along
the axis), i.e. every offset of the 2 P N - 1 cells centred on the target;
this reading reproduces the film column of Table tabPBC1 within its printed
accuracy.  The convolution along a periodic axis is then cyclic with period
N (no padding), with the tensor summed over the offsets D = d mod N.

Float64 test infrastructure only: tests, smoke() and the benchmark's CPU
legs use it; the product path never does.
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


def demag_direct(M, dx, dy, dz, pbc=(0, 0, 0)):
    """Direct O(N^2) summation of -mu0 N(r_i - r_j) M_j over every cell pair
    (and, along periodic axes, over every image of the source whose offset
    lies in the window -P N < D < P N)."""
    _, nz, ny, nx = M.shape
    zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    pos = np.stack([xx.ravel(), yy.ravel(), zz.ravel()], axis=1)        # (N, 3)
    d = pos[None, :, :] - pos[:, None, :]                                 # (target, source, 3): r_j - r_i
    sizes = (nx, ny, nz)
    shifts = [np.arange(-p, p + 1) if p > 0 else np.array([0]) for p in pbc]
    Mf = M.reshape(3, -1)
    B = np.zeros_like(Mf)
    for kx in shifts[0]:
        for ky in shifts[1]:
            for kz in shifts[2]:
                D = d + np.array([kx * nx, ky * ny, kz * nz])
                inside = np.ones(D.shape[:2], dtype=bool)
                for a in range(3):
                    if pbc[a] > 0:
                        inside &= np.abs(D[..., a]) < pbc[a] * sizes[a]
                if not inside.any():
                    continue
                # the tensor depends on the source-to-target offset r_i - r_j = -D
                Nt = demag_tensor(-D[..., 0], -D[..., 1], -D[..., 2], dx, dy, dz)
                for i in range(3):
                    for j in range(3):
                        B[i] -= MU0 * ((Nt[_IDX[(i, j)]] * inside) @ Mf[j])
    return B.reshape(M.shape)


def padded_sizes(nx, ny, nz, pbc=(0, 0, 0)):
    """Transform length per axis: n along a periodic axis, else 2n - 1."""
    return tuple(n if p > 0 else 2 * n - 1 for n, p in zip((nx, ny, nz), pbc))


def kernel_spectrum(nx, ny, nz, dx, dy, dz, pbc=(0, 0, 0)):
    """FFT of the tensor on the transform grid: offset (X, Y, Z) stored at
    index (X mod Px, Y mod Py, Z mod Pz); along a periodic axis every offset
    of the window -P n < X < P n adds into X mod n."""
    Px, Py, Pz = padded_sizes(nx, ny, nz, pbc)
    if not any(pbc):
        full = demag_tensor_full(nx, ny, nz, dx, dy, dz)   # offsets -(n-1)..(n-1)
        # move offset 0 to index 0 (negative offsets wrap to the top of the axis)
        wrapped = np.roll(full, shift=(-(nz - 1), -(ny - 1), -(nx - 1)), axis=(1, 2, 3))
        assert wrapped.shape[1:] == (Pz, Py, Px)
        return np.fft.fftn(wrapped, axes=(1, 2, 3))
    ranges = [np.arange(-(p * n - 1), p * n) if p > 0 else np.arange(-(n - 1), n)
              for n, p in zip((nx, ny, nz), pbc)]
    X, Y, Z = np.meshgrid(ranges[0], ranges[1], ranges[2], indexing="ij")
    T = demag_tensor(X, Y, Z, dx, dy, dz)
    K = np.zeros((6, Pz, Py, Px))
    for c in range(6):
        np.add.at(K[c], (Z % Pz, Y % Py, X % Px), T[c])
    return np.fft.fftn(K, axes=(1, 2, 3))


def demag_fft(M, dx, dy, dz, spectrum=None, pbc=(0, 0, 0)):
    """FFT convolution (zero-padded, cyclic along periodic axes); returns
    B_demag with the shape of M."""
    _, nz, ny, nx = M.shape
    Px, Py, Pz = padded_sizes(nx, ny, nz, pbc)
    K = kernel_spectrum(nx, ny, nz, dx, dy, dz, pbc) if spectrum is None else spectrum
    Mh = np.fft.fftn(M, s=(Pz, Py, Px), axes=(1, 2, 3))
    B = np.zeros_like(M)
    for i in range(3):
        acc = np.zeros(Mh.shape[1:], dtype=complex)
        for j in range(3):
            acc += K[_IDX[(i, j)]] * Mh[j]
        B[i] = -MU0 * np.fft.ifftn(acc, axes=(0, 1, 2)).real[:nz, :ny, :nx]
    return B
