// Demagnetising kernel precompute, float64 on the device (Sec. III.B,
// "Magnetostatic kernel"): the field of a uniformly magnetised cell averaged
// over a destination cell, initialised in double precision and only rounded to
// single precision at the end.
//
// Near the source the cell-averaged tensor is evaluated exactly with Newell,
// Williams & Dunlop's antiderivatives f and g (J. Geophys. Res. 98, 9551,
// 1993) under the second-difference stencil in each axis.  Far from it that
// stencil cancels catastrophically (the terms grow like r^3 while the result
// falls like r^-3), so the same average is integrated numerically: the double
// average over two equal boxes is one integral of the point-dipole tensor
// against the tent sum_k (d_k - |u_k|), done with Gauss-Legendre rules on each
// half of every axis -- the paper's route (numerical integration whose point
// count depends on the distance).
//
// The spectrum: the zero-padded kernel is real and, per component, even or
// odd in each axis (the mirror symmetries of Sec. III.B), so its DFT is real
// and is stored on one octant only.  It is computed as three separable
// cosine/sine transforms of the first octant, in float64.
#include <cmath>
#include <vector>

#include "mm_internal.h"

namespace mm {
namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr double kMu0 = 4e-7 * kPi;
constexpr double kNearRadius = 8.0;   // in largest cell edges

// Gauss-Legendre rules with n = 3..6 points on [-1, 1].
struct GLRules {
  double x[4][6];
  double w[4][6];
};

GLRules make_gl_rules() {
  GLRules R{};
  for (int n = 3; n <= 6; ++n) {
    for (int i = 0; i < n; ++i) {
      // Newton iteration on P_n from the Chebyshev-like initial guess
      double z = std::cos(kPi * (i + 0.75) / (n + 0.5));
      double dp = 1.0;
      for (int it = 0; it < 100; ++it) {
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= n; ++k) {
          const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
          p0 = p1;
          p1 = p2;
        }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        const double dz = p1 / dp;
        z -= dz;
        if (std::fabs(dz) < 1e-16) break;
      }
      R.x[n - 3][i] = z;
      R.w[n - 3][i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
  }
  return R;
}

__device__ double asinh_ratio(double num, double den) { return den != 0.0 ? asinh(num / den) : 0.0; }
__device__ double atan_ratio(double num, double den) { return den != 0.0 ? atan(num / den) : 0.0; }

__device__ double newell_f(double x, double y, double z) {
  const double x2 = x * x, y2 = y * y, z2 = z * z;
  const double R = sqrt(x2 + y2 + z2);
  double r = 0.5 * y * (z2 - x2) * asinh_ratio(y, sqrt(x2 + z2));
  r += 0.5 * z * (y2 - x2) * asinh_ratio(z, sqrt(x2 + y2));
  r -= x * y * z * atan_ratio(y * z, x * R);
  r += (2.0 * x2 - y2 - z2) * R * (1.0 / 6.0);
  return r;
}

__device__ double newell_g(double x, double y, double z) {
  const double x2 = x * x, y2 = y * y, z2 = z * z;
  const double R = sqrt(x2 + y2 + z2);
  double r = x * y * z * asinh_ratio(z, sqrt(x2 + y2));
  r += y * (3.0 * z2 - y2) * asinh_ratio(x, sqrt(y2 + z2)) * (1.0 / 6.0);
  r += x * (3.0 * z2 - x2) * asinh_ratio(y, sqrt(x2 + z2)) * (1.0 / 6.0);
  r -= z2 * z * atan_ratio(x * y, z * R) * (1.0 / 6.0);
  r -= 0.5 * z * y2 * atan_ratio(x * z, y * R);
  r -= 0.5 * z * x2 * atan_ratio(y * z, x * R);
  r -= x * y * R * (1.0 / 3.0);
  return r;
}

// sum over the 27 stencil points of w_i w_j w_k F(X + i a, Y + j b, Z + k c),
// w_0 = 2, w_{+-1} = -1, divided by 4 pi a b c
template <bool G>
__device__ double stencil(double X, double Y, double Z, double a, double b, double c) {
  double acc = 0.0;
  for (int i = -1; i <= 1; ++i)
    for (int j = -1; j <= 1; ++j)
      for (int k = -1; k <= 1; ++k) {
        const double w = (i ? -1.0 : 2.0) * (j ? -1.0 : 2.0) * (k ? -1.0 : 2.0);
        const double v = G ? newell_g(X + i * a, Y + j * b, Z + k * c)
                           : newell_f(X + i * a, Y + j * b, Z + k * c);
        acc = fma(w, v, acc);
      }
  return acc / (4.0 * kPi * a * b * c);
}

// Tensor at one offset (metres): out = Nxx, Nyy, Nzz, Nxy, Nxz, Nyz.
__device__ void tensor_at(double X, double Y, double Z, double dx, double dy, double dz,
                          const GLRules& gl, double out[6]) {
  const double dmax = fmax(dx, fmax(dy, dz));
  const double dist = sqrt(X * X + Y * Y + Z * Z) / dmax;
  if (dist < kNearRadius) {
    out[0] = stencil<false>(X, Y, Z, dx, dy, dz);
    out[1] = stencil<false>(Y, X, Z, dy, dx, dz);
    out[2] = stencil<false>(Z, Y, X, dz, dy, dx);
    out[3] = stencil<true>(X, Y, Z, dx, dy, dz);
    out[4] = stencil<true>(X, Z, Y, dx, dz, dy);
    out[5] = stencil<true>(Y, Z, X, dy, dz, dx);
  } else {
    // error of an n-point rule on a half-axis ~ (4 dist)^(-2n)
    const int n = dist < 16.0 ? 6 : (dist < 32.0 ? 5 : (dist < 128.0 ? 4 : 3));
    const double* xs = gl.x[n - 3];
    const double* ws = gl.w[n - 3];
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int a = 0; a < 2 * n; ++a) {
      const double ua = 0.5 * dx * (1.0 + xs[a % n]);
      const double wa = 0.5 * dx * ws[a % n] * (dx - ua);
      const double rx = X + (a < n ? -ua : ua);
      for (int b = 0; b < 2 * n; ++b) {
        const double ub = 0.5 * dy * (1.0 + xs[b % n]);
        const double wb = wa * 0.5 * dy * ws[b % n] * (dy - ub);
        const double ry = Y + (b < n ? -ub : ub);
        for (int c = 0; c < 2 * n; ++c) {
          const double uc = 0.5 * dz * (1.0 + xs[c % n]);
          const double w = wb * 0.5 * dz * ws[c % n] * (dz - uc);
          const double rz = Z + (c < n ? -uc : uc);
          const double r2 = rx * rx + ry * ry + rz * rz;
          const double s = w / (r2 * r2 * sqrt(r2));
          acc[0] += s * (r2 - 3.0 * rx * rx);
          acc[1] += s * (r2 - 3.0 * ry * ry);
          acc[2] += s * (r2 - 3.0 * rz * rz);
          acc[3] -= s * 3.0 * rx * ry;
          acc[4] -= s * 3.0 * rx * rz;
          acc[5] -= s * 3.0 * ry * rz;
        }
      }
    }
    const double norm = 1.0 / (4.0 * kPi * dx * dy * dz);
    for (int i = 0; i < 6; ++i) out[i] = acc[i] * norm;
  }
  // off-diagonal components odd in an axis vanish at zero offset along it
  if (X == 0.0 || Y == 0.0) out[3] = 0.0;
  if (X == 0.0 || Z == 0.0) out[4] = 0.0;
  if (Y == 0.0 || Z == 0.0) out[5] = 0.0;
}

__global__ void k_tensor_offsets(int n, const int32_t* __restrict__ off, double dx, double dy,
                                 double dz, GLRules gl, double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double v[6];
  tensor_at(off[3 * i] * dx, off[3 * i + 1] * dy, off[3 * i + 2] * dz, dx, dy, dz, gl, v);
  for (int c = 0; c < 6; ++c) out[6 * i + c] = v[c];
}

// First octant: w[c][Z][Y][X] for 0 <= X < nx etc.
__global__ void k_tensor_octant(int nx, int ny, int nz, double dx, double dy, double dz,
                                GLRules gl, double* __restrict__ w) {
  const long long n = (long long)nx * ny * nz;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int X = (int)(i % nx), Y = (int)((i / nx) % ny), Z = (int)(i / ((long long)nx * ny));
  double v[6];
  tensor_at(X * dx, Y * dy, Z * dz, dx, dy, dz, gl, v);
  for (int c = 0; c < 6; ++c) w[c * n + i] = v[c];
}

// First octant of the periodic (macro-geometry) kernel, Sec. III.B: extents
// (mx, my, mz) = n/2 + 1 along a periodic axis, n along an open one; along a
// periodic axis of n cells with P images per side the value at offset X is
// the tensor summed over the offsets D = X + k n with |D| < P n.
__global__ void k_tensor_octant_pbc(int mx, int my, int mz, int nx, int ny, int nz, int pbx, int pby, int pbz,
                                    double dx, double dy, double dz, GLRules gl, double* __restrict__ w) {
  const long long n = (long long)mx * my * mz;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int X = (int)(i % mx), Y = (int)((i / mx) % my), Z = (int)(i / ((long long)mx * my));
  double acc[6] = {0, 0, 0, 0, 0, 0};
  const int kx = pbx > 0 ? pbx : 0, ky = pby > 0 ? pby : 0, kz = pbz > 0 ? pbz : 0;
  for (int a = -kx; a <= kx; ++a) {
    const long long DX = X + (long long)a * nx;
    if (pbx > 0 && !(DX > -(long long)pbx * nx && DX < (long long)pbx * nx)) continue;
    for (int b = -ky; b <= ky; ++b) {
      const long long DY = Y + (long long)b * ny;
      if (pby > 0 && !(DY > -(long long)pby * ny && DY < (long long)pby * ny)) continue;
      for (int c = -kz; c <= kz; ++c) {
        const long long DZ = Z + (long long)c * nz;
        if (pbz > 0 && !(DZ > -(long long)pbz * nz && DZ < (long long)pbz * nz)) continue;
        double v[6];
        tensor_at(DX * dx, DY * dy, DZ * dz, dx, dy, dz, gl, v);
        for (int t = 0; t < 6; ++t) acc[t] += v[t];
      }
    }
  }
  for (int t = 0; t < 6; ++t) w[t * n + i] = acc[t];
}

// Parity (odd = 1) of component c along axis a (0 x, 1 y, 2 z).
__host__ __device__ inline int odd_axis(int c, int a) {
  // Nxy odd in x,y; Nxz odd in x,z; Nyz odd in y,z; diagonals even
  const int tbl[6][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}, {1, 1, 0}, {1, 0, 1}, {0, 1, 1}};
  return tbl[c][a];
}

// One separable transform along the innermost axis of in[c][outer][n] into
// out[c][outer][h]:  out[k] = sum_X t[k][X] in[X], with tcos (even
// components) or tsin (odd components) tables of shape [h][n].
__global__ void k_axis_transform(int n, int h, long long outer, int axis,
                                 const double* __restrict__ in, double* __restrict__ out,
                                 const double* __restrict__ tcos, const double* __restrict__ tsin) {
  const long long total = 6LL * outer * h;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  const int k = (int)(i % h);
  const long long o = (i / h) % outer;
  const int c = (int)(i / (h * outer));
  const double* src = in + ((long long)c * outer + o) * n;
  const double* t = (odd_axis(c, axis) ? tsin : tcos) + (long long)k * n;
  double acc = 0.0;
  for (int X = 0; X < n; ++X) acc = fma(t[X], src[X], acc);
  out[i] = acc;
}

// Reorders w[c][A][B][C] (C fastest) into w[c][C][A][B] so the next axis is
// innermost.
__global__ void k_rotate(int A, int B, int C, const double* __restrict__ in, double* __restrict__ out) {
  const long long per = (long long)A * B * C;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 6 * per) return;
  const int cc = (int)(i / per);
  const long long r = i % per;
  const int c = (int)(r % C), b = (int)((r / C) % B), a = (int)(r / ((long long)B * C));
  out[cc * per + ((long long)c * A + a) * B + b] = in[i];
}

__global__ void k_finish(long long per, double scale, const double* __restrict__ in, float* __restrict__ kt) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 6 * per) return;
  const int c = (int)(i / per);
  // two odd axes: (-i 2 sin)(-i 2 sin) = -(2 sin)(2 sin)
  const double sign = c >= 3 ? -1.0 : 1.0;
  kt[i] = (float)(sign * scale * in[i]);
}

// cos/sin tables for one axis: t[k][X] = wgt * cos(2 pi k X / P) and 2 sin(...)
void axis_tables(int n, int P, int h, std::vector<double>& tc, std::vector<double>& ts) {
  tc.assign((size_t)h * n, 0.0);
  ts.assign((size_t)h * n, 0.0);
  for (int k = 0; k < h; ++k)
    for (int X = 0; X < n; ++X) {
      const long long num = (2LL * k * X) % (2LL * P);   // angle = pi * num / P
      const double ang = kPi * (double)num / (double)P;
      // offsets X and -X are distinct points of the cyclic axis unless
      // X = 0 or X = P/2 (a periodic axis reaches its Nyquist offset)
      tc[(size_t)k * n + X] = (X == 0 || 2 * X == P ? 1.0 : 2.0) * std::cos(ang);
      ts[(size_t)k * n + X] = 2.0 * std::sin(ang);
    }
}

// Device-side version of axis_tables (float64 cospi/sinpi of the exactly
// reduced angle), for callers that must not stage tables from the host.
__global__ void k_axis_tables(int n, int P, int h, double* __restrict__ tc, double* __restrict__ ts) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * h) return;
  const int k = i / n, X = i % n;
  const long long num = (2LL * k * X) % (2LL * P);   // angle = pi * num / P
  const double a = (double)num / (double)P;
  tc[i] = (X == 0 || 2 * X == P ? 1.0 : 2.0) * cospi(a);
  ts[i] = 2.0 * sinpi(a);
}

}  // namespace

cudaError_t demag_tensor_offsets(int n, const int32_t* d_off, double dx, double dy, double dz,
                                 double* d_out, cudaStream_t s) {
  const GLRules gl = make_gl_rules();
  if (n > 0) k_tensor_offsets<<<(n + 127) / 128, 128, 0, s>>>(n, d_off, dx, dy, dz, gl, d_out);
  return cudaGetLastError();
}

cudaError_t build_kernel_spectrum(const Geom& g, double dx, double dy, double dz, float* kt,
                                  cudaStream_t s) {
  const GLRules gl = make_gl_rules();
  // octant extents: n along an open axis, n/2 + 1 along a periodic one
  const bool pbc = g.pbcx > 0 || g.pbcy > 0 || g.pbcz > 0;
  const int nx = g.pbcx > 0 ? g.hkx : g.nx, ny = g.pbcy > 0 ? g.hky : g.ny, nz = g.pbcz > 0 ? g.hkz : g.nz;
  const long long n = (long long)nx * ny * nz;
  const int hx = g.hkx, hy = g.hky, hz = g.hkz;
  // work buffers sized for the largest intermediate
  const long long cap = 6LL * std::max<long long>(
      std::max<long long>(n, (long long)hx * ny * nz),
      std::max<long long>((long long)hx * hy * nz, (long long)hx * hy * hz));
  double *w0 = nullptr, *w1 = nullptr, *tab = nullptr;
  cudaError_t e = cudaMalloc(&w0, cap * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&w1, cap * sizeof(double));
  const int maxn = std::max(nx, std::max(ny, nz)), maxh = std::max(hx, std::max(hy, hz));
  if (e == cudaSuccess) e = cudaMalloc(&tab, 2ULL * maxn * maxh * sizeof(double));
  if (e != cudaSuccess) {
    cudaFree(w0); cudaFree(w1); cudaFree(tab);
    return e;
  }
  const int T = 128;
  auto blocks = [&](long long tot) { return (unsigned)((tot + T - 1) / T); };
  if (pbc)
    k_tensor_octant_pbc<<<blocks(n), T, 0, s>>>(nx, ny, nz, g.nx, g.ny, g.nz, g.pbcx, g.pbcy, g.pbcz, dx, dy, dz,
                                                 gl, w0);
  else
    k_tensor_octant<<<blocks(n), T, 0, s>>>(nx, ny, nz, dx, dy, dz, gl, w0);

  std::vector<double> tc, ts;
  auto transform = [&](int len, int P, int h, long long outer, int axis, double* in, double* out) {
    axis_tables(len, P, h, tc, ts);
    cudaMemcpyAsync(tab, tc.data(), tc.size() * sizeof(double), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(tab + tc.size(), ts.data(), ts.size() * sizeof(double), cudaMemcpyHostToDevice, s);
    k_axis_transform<<<blocks(6 * outer * h), T, 0, s>>>(len, h, outer, axis, in, out, tab, tab + tc.size());
    cudaStreamSynchronize(s);   // tables are reused by the next axis
  };
  // x: w0[c][z][y][x] -> w1[c][z][y][kx]
  transform(nx, g.px, hx, (long long)nz * ny, 0, w0, w1);
  // rotate to [c][kx][z][y], transform y -> [c][kx][z][ky]
  k_rotate<<<blocks(6LL * nz * ny * hx), T, 0, s>>>(nz, ny, hx, w1, w0);
  transform(ny, g.py, hy, (long long)hx * nz, 1, w0, w1);
  // rotate [c][kx][z][ky] -> [c][ky][kx][z], transform z -> [c][ky][kx][kz]
  k_rotate<<<blocks(6LL * hx * nz * hy), T, 0, s>>>(hx, nz, hy, w1, w0);
  transform(nz, g.pz, hz, (long long)hy * hx, 2, w0, w1);
  // rotate [c][ky][kx][kz] -> [c][kz][ky][kx]
  k_rotate<<<blocks(6LL * hy * hx * hz), T, 0, s>>>(hy * hx, 1, hz, w1, w0);
  // B = -mu0 N * M, and the inverse transforms are unnormalised: divide by
  // lx * py * pz (lx = px / 2 complex points along x, or 1)
  const double scale = -kMu0 / ((double)g.lx * g.py * g.pz);
  k_finish<<<blocks(6LL * hx * hy * hz), T, 0, s>>>((long long)hx * hy * hz, scale, w0, kt);
  e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaFree(w0);
  cudaFree(w1);
  cudaFree(tab);
  return e;
}

// Same computation as build_kernel_spectrum, on caller-provided work space
// and without host round trips: w0, w1 hold 6 * kernel_work_doubles(g)
// doubles each, tab holds 2 * max(n) * max(h) doubles.
size_t kernel_work_doubles(const Geom& g) {
  const long long n = g.n;
  return 6ULL * std::max<long long>(std::max<long long>(n, (long long)g.hkx * g.ny * g.nz),
                                    std::max<long long>((long long)g.hkx * g.hky * g.nz,
                                                        (long long)g.hkx * g.hky * g.hkz));
}
size_t kernel_table_doubles(const Geom& g) {
  const int maxn = std::max(g.nx, std::max(g.ny, g.nz)), maxh = std::max(g.hkx, std::max(g.hky, g.hkz));
  return 2ULL * maxn * maxh;
}

cudaError_t build_kernel_spectrum_ws(const Geom& g, double dx, double dy, double dz, float* kt, double* w0,
                                     double* w1, double* tab, cudaStream_t s) {
  const GLRules gl = make_gl_rules();
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const int hx = g.hkx, hy = g.hky, hz = g.hkz;
  const int T = 128;
  auto blocks = [&](long long tot) { return (unsigned)((tot + T - 1) / T); };
  k_tensor_octant<<<blocks(g.n), T, 0, s>>>(nx, ny, nz, dx, dy, dz, gl, w0);
  auto transform = [&](int len, int P, int h, long long outer, int axis, double* in, double* out) {
    double* tc = tab;
    double* ts = tab + (size_t)len * h;
    k_axis_tables<<<blocks((long long)len * h), T, 0, s>>>(len, P, h, tc, ts);
    k_axis_transform<<<blocks(6 * outer * h), T, 0, s>>>(len, h, outer, axis, in, out, tc, ts);
  };
  transform(nx, g.px, hx, (long long)nz * ny, 0, w0, w1);
  k_rotate<<<blocks(6LL * nz * ny * hx), T, 0, s>>>(nz, ny, hx, w1, w0);
  transform(ny, g.py, hy, (long long)hx * nz, 1, w0, w1);
  k_rotate<<<blocks(6LL * hx * nz * hy), T, 0, s>>>(hx, nz, hy, w1, w0);
  transform(nz, g.pz, hz, (long long)hy * hx, 2, w0, w1);
  k_rotate<<<blocks(6LL * hy * hx * hz), T, 0, s>>>(hy * hx, 1, hz, w1, w0);
  const double scale = -kMu0 / ((double)g.lx * g.py * g.pz);
  k_finish<<<blocks(6LL * hx * hy * hz), T, 0, s>>>((long long)hx * hy * hz, scale, w0, kt);
  return cudaGetLastError();
}

}  // namespace mm
