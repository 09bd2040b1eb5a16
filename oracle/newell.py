"""Cell-averaged demagnetising tensor N_ij of two equal orthorhombic cells.

Sec. III.B ("Magnetostatic kernel"): each cell carries a constant
magnetisation and the field it produces is averaged over the destination cell.
The paper integrates numerically with a distance-dependent number of points;
here the same definite integral is evaluated two ways:

* near the source, exactly, with Newell, Williams & Dunlop's closed-form
  antiderivatives f (diagonal) and g (off-diagonal) combined by the
  second-difference stencil in every axis (J. Geophys. Res. 98, 9551, 1993);
* far from the source, where that stencil cancels catastrophically, by
  Gauss-Legendre quadrature of the point-dipole tensor.  Averaging over a
  source box and a destination box of the same size equals one integral of the
  dipole tensor against the "tent" (d_k - |u_k|) in every axis, so the far
  field is a 3-D integral, split at u_k = 0 where the tent has its kink.

Convention (reading of the sign used by the tables of Sec. III.B, which print
N = H/M < 0): N is stored positive, so that the self term of a cube is +1/3,
the trace of every self term is 1, and B_demag = -mu0 * N * M.

Float64 test infrastructure only: tests, smoke() and the benchmark's CPU
legs use it; the product path never does.
"""
import numpy as np

FOUR_PI = 4.0 * np.pi


# ---------------------------------------------------------------------------
# Newell's antiderivatives.  Every singular sub-term (0/0 inside asinh or
# atan) carries a prefactor that vanishes there, so it is set to zero.
# ---------------------------------------------------------------------------
def _asinh_ratio(num, den):
    """asinh(num/den), 0 where den == 0."""
    out = np.zeros(np.broadcast(num, den).shape, dtype=np.result_type(num, den))
    ok = den != 0
    out[ok] = np.arcsinh(num[ok] / den[ok])
    return out


def _atan_ratio(num, den):
    """atan(num/den), 0 where den == 0."""
    out = np.zeros(np.broadcast(num, den).shape, dtype=np.result_type(num, den))
    ok = den != 0
    out[ok] = np.arctan(num[ok] / den[ok])
    return out


def newell_f(x, y, z):
    """Newell's f(x, y, z), whose 27-point second difference gives N_xx."""
    x2, y2, z2 = x * x, y * y, z * z
    R = np.sqrt(x2 + y2 + z2)
    t1 = 0.5 * y * (z2 - x2) * _asinh_ratio(y, np.sqrt(x2 + z2))
    t2 = 0.5 * z * (y2 - x2) * _asinh_ratio(z, np.sqrt(x2 + y2))
    t3 = -x * y * z * _atan_ratio(y * z, x * R)
    t4 = (2.0 * x2 - y2 - z2) * R / 6.0
    return t1 + t2 + t3 + t4


def newell_g(x, y, z):
    """Newell's g(x, y, z), whose 27-point second difference gives N_xy."""
    x2, y2, z2 = x * x, y * y, z * z
    R = np.sqrt(x2 + y2 + z2)
    t1 = x * y * z * _asinh_ratio(z, np.sqrt(x2 + y2))
    t2 = y * (3.0 * z2 - y2) * _asinh_ratio(x, np.sqrt(y2 + z2)) / 6.0
    t3 = x * (3.0 * z2 - x2) * _asinh_ratio(y, np.sqrt(x2 + z2)) / 6.0
    t4 = -z2 * z * _atan_ratio(x * y, z * R) / 6.0
    t5 = -0.5 * z * y2 * _atan_ratio(x * z, y * R)
    t6 = -0.5 * z * x2 * _atan_ratio(y * z, x * R)
    t7 = -x * y * R / 3.0
    return t1 + t2 + t3 + t4 + t5 + t6 + t7


_W = {-1: -1.0, 0: 2.0, 1: -1.0}   # second-difference weights per axis


def _stencil(fun, X, Y, Z, dx, dy, dz, dtype):
    X = np.asarray(X, dtype=dtype)
    Y = np.asarray(Y, dtype=dtype)
    Z = np.asarray(Z, dtype=dtype)
    dx, dy, dz = (np.asarray(v, dtype=dtype) for v in (dx, dy, dz))
    acc = np.zeros(np.broadcast(X, Y, Z).shape, dtype=dtype)
    for i in (-1, 0, 1):
        for j in (-1, 0, 1):
            for k in (-1, 0, 1):
                w = _W[i] * _W[j] * _W[k]
                acc = acc + w * fun(X + i * dx, Y + j * dy, Z + k * dz)
    return acc / (FOUR_PI * dx * dy * dz)


def newell_tensor(X, Y, Z, dx, dy, dz, dtype=np.float64):
    """Exact cell-averaged tensor at offset (X, Y, Z) (metres) via Newell.

    Returns (Nxx, Nyy, Nzz, Nxy, Nxz, Nyz) as arrays of ``dtype``.  The
    diagonal terms are f with the axes permuted, the off-diagonal ones g with
    the axes permuted (the tensor is symmetric).
    """
    nxx = _stencil(newell_f, X, Y, Z, dx, dy, dz, dtype)
    nyy = _stencil(newell_f, Y, X, Z, dy, dx, dz, dtype)
    nzz = _stencil(newell_f, Z, Y, X, dz, dy, dx, dtype)
    nxy = _stencil(newell_g, X, Y, Z, dx, dy, dz, dtype)
    nxz = _stencil(newell_g, X, Z, Y, dx, dz, dy, dtype)
    nyz = _stencil(newell_g, Y, Z, X, dy, dz, dx, dtype)
    return nxx, nyy, nzz, nxy, nxz, nyz


# ---------------------------------------------------------------------------
# Far field: Gauss-Legendre quadrature of the point-dipole tensor against the
# tent weight.  D_ij(r) = (delta_ij r^2 - 3 r_i r_j) / (4 pi r^5).
# ---------------------------------------------------------------------------
def _tent_rule(d, n):
    """Nodes/weights integrating g(u)(d - |u|) over [-d, d] (n GL points per half)."""
    xi, wi = np.polynomial.legendre.leggauss(n)
    u = 0.5 * d * (1.0 + xi)            # nodes on (0, d)
    w = 0.5 * d * wi * (d - u)          # tent weight folded in
    return np.concatenate([-u, u]), np.concatenate([w, w])


def gl_points_for(dist_over_cell):
    """GL points per half-axis for a given distance / largest cell edge.

    The integrand is analytic within a Bernstein ellipse of parameter rho ~
    4 r/d around each half-interval, so the error falls like rho^(-2n); these
    choices keep it below ~1e-13 relative.
    """
    if dist_over_cell < 16:
        return 6
    if dist_over_cell < 32:
        return 5
    if dist_over_cell < 128:
        return 4
    return 3


def dipole_tensor_avg(X, Y, Z, dx, dy, dz, n):
    """Cell-averaged tensor by quadrature (float64); X, Y, Z 1-D arrays."""
    ux, wx = _tent_rule(dx, n)
    uy, wy = _tent_rule(dy, n)
    uz, wz = _tent_rule(dz, n)
    X = np.asarray(X, dtype=np.float64)[:, None, None, None]
    Y = np.asarray(Y, dtype=np.float64)[:, None, None, None]
    Z = np.asarray(Z, dtype=np.float64)[:, None, None, None]
    rx = X + ux[None, :, None, None]
    ry = Y + uy[None, None, :, None]
    rz = Z + uz[None, None, None, :]
    w = (wx[:, None, None] * wy[None, :, None] * wz[None, None, :])[None]
    r2 = rx * rx + ry * ry + rz * rz
    inv5 = 1.0 / (FOUR_PI * r2 * r2 * np.sqrt(r2))
    V = dx * dy * dz
    out = []
    for a, b in (("x", "x"), ("y", "y"), ("z", "z"), ("x", "y"), ("x", "z"), ("y", "z")):
        ra = {"x": rx, "y": ry, "z": rz}[a]
        rb = {"x": rx, "y": ry, "z": rz}[b]
        d = (r2 if a == b else 0.0) - 3.0 * ra * rb
        out.append(np.sum(w * d * inv5, axis=(1, 2, 3)) / V)
    return tuple(out)


NEAR_RADIUS = 8.0   # cell edges: inside, Newell; outside, quadrature


def demag_tensor(IX, IY, IZ, dx, dy, dz, near_dtype=np.float64):
    """N_ij for integer cell offsets (IX, IY, IZ) of a grid with cells dx*dy*dz.

    Offsets whose centre distance is below NEAR_RADIUS times the largest cell
    edge use Newell's closed form (in ``near_dtype``); the others use the
    dipole quadrature.  Returns six float64 arrays shaped like the offsets.
    """
    IX, IY, IZ = np.broadcast_arrays(np.asarray(IX), np.asarray(IY), np.asarray(IZ))
    shape = IX.shape
    X = IX.ravel() * dx
    Y = IY.ravel() * dy
    Z = IZ.ravel() * dz
    dmax = max(dx, dy, dz)
    dist = np.sqrt(X * X + Y * Y + Z * Z) / dmax
    out = [np.zeros(X.shape) for _ in range(6)]
    near = dist < NEAR_RADIUS
    if near.any():
        vals = newell_tensor(X[near], Y[near], Z[near], dx, dy, dz, dtype=near_dtype)
        for c in range(6):
            out[c][near] = np.asarray(vals[c], dtype=np.float64)
    far_idx = np.nonzero(~near)[0]
    if far_idx.size:
        npts = np.array([gl_points_for(v) for v in dist[far_idx]])
        for n in np.unique(npts):
            sel = far_idx[npts == n]
            for s in range(0, sel.size, 4096):
                chunk = sel[s:s + 4096]
                vals = dipole_tensor_avg(X[chunk], Y[chunk], Z[chunk], dx, dy, dz, int(n))
                for c in range(6):
                    out[c][chunk] = vals[c]
    # An off-diagonal component odd in an axis vanishes at zero offset along
    # it (exactly, by the mirror symmetry); remove rounding residue.
    for c in range(3, 6):
        for axis, I in enumerate((IX.ravel(), IY.ravel(), IZ.ravel())):
            if PARITY[c][axis] < 0:
                out[c][I == 0] = 0.0
    return tuple(o.reshape(shape) for o in out)


# Parity of each component under a sign flip of (X, Y, Z): +1 even, -1 odd.
# N_xy is odd in X and Y, N_xz in X and Z, N_yz in Y and Z; diagonals even.
PARITY = {
    0: (1, 1, 1), 1: (1, 1, 1), 2: (1, 1, 1),
    3: (-1, -1, 1), 4: (-1, 1, -1), 5: (1, -1, -1),
}


def demag_tensor_full(nx, ny, nz, dx, dy, dz):
    """N_ij for every offset in [-(n-1), n-1]^3, shape (6, 2nz-1, 2ny-1, 2nx-1).

    The first octant (offsets >= 0) is evaluated and mirrored with the parities
    above: the mirror symmetries the paper uses to shrink the kernel (Sec.
    III.B).  Index [c, Z + nz - 1, Y + ny - 1, X + nx - 1] holds offset (X, Y, Z).
    """
    IZ, IY, IX = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    octant = demag_tensor(IX, IY, IZ, dx, dy, dz)
    full = np.zeros((6, 2 * nz - 1, 2 * ny - 1, 2 * nx - 1))
    for c in range(6):
        px, py, pz = PARITY[c]
        o = octant[c]
        for sz in (1, -1):
            for sy in (1, -1):
                for sx in (1, -1):
                    sign = (px if sx < 0 else 1) * (py if sy < 0 else 1) * (pz if sz < 0 else 1)
                    zi = nz - 1 + sz * np.arange(nz)
                    yi = ny - 1 + sy * np.arange(ny)
                    xi = nx - 1 + sx * np.arange(nx)
                    full[c][np.ix_(zi, yi, xi)] = sign * o
    return full
