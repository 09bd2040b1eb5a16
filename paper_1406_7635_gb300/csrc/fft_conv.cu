// Zero-padded FFT convolution B_demag = K * M (Sec. III.B "Magnetostatic
// convolution"), M = Msat m, with the kernel spectrum stored as a real octant.
//
// Passes (all in place in one spectrum buffer; see Geom in mm_internal.h):
//   FX   rows along x: real M (nx values, the zero half is never read) ->
//        half spectrum X_k, k = 0..px/2, via one complex FFT of length px/2
//        on even/odd-packed samples;
//   FY   columns along y: ny non-zero inputs -> py outputs        (3-D only)
//   FZMI pencils along z: nz inputs -> FFT -> multiply by the 3x3 kernel ->
//        inverse FFT -> nz outputs                                  (3-D)
//   FYMI in 2-D the y pass does forward, multiply and inverse in one kernel
//   IY   columns along y: py inputs -> ny outputs                  (3-D only)
//   IX   rows along x: half spectrum -> nx real outputs (C2R, cropped).
// The inverse transforms are unnormalised; the kernel spectrum carries the
// 1/(lx py pz) factor and -mu0.
#include <algorithm>

#include "fft.cuh"
#include "mm_internal.h"

namespace mm {
namespace {
using namespace mmfft;

__device__ __forceinline__ float cell_msat(const RegionLUT* __restrict__ lut, const uint8_t* __restrict__ mask,
                                           const uint8_t* __restrict__ region, long long i) {
  return mask[i] ? __ldg(&lut->msat[region[i]]) : 0.0f;
}

// ----------------------------------------------------------------------------
// FX: real rows -> half spectrum
// ----------------------------------------------------------------------------
template <int L, int ROWS, int NT>
__global__ void __launch_bounds__(NT) k_fx(Geom g, const float* __restrict__ m, const uint8_t* __restrict__ mask,
                                           const uint8_t* __restrict__ region, const RegionLUT* __restrict__ lut,
                                           float2* __restrict__ spec, const float2* __restrict__ tw,
                                           const DevState* __restrict__ st) {
  if (st && st->done) return;
  constexpr int PST = L + 1;
  __shared__ float2 s[ROWS * PST];
  const int nrows = 3 * g.nz * g.ny;
  const int row0 = blockIdx.x * ROWS;
  for (int e = threadIdx.x; e < ROWS * L; e += NT) {
    const int r = e / L, n = e % L, row = row0 + r;
    float2 v = make_float2(0.f, 0.f);
    if (row < nrows) {
      const int c = row / (g.nz * g.ny), zy = row % (g.nz * g.ny);
      const long long cell0 = (long long)zy * g.nx;
      const int x0 = 2 * n, x1 = 2 * n + 1;
      if (x0 < g.nx) v.x = cell_msat(lut, mask, region, cell0 + x0) * m[c * g.n + cell0 + x0];
      if (x1 < g.nx) v.y = cell_msat(lut, mask, region, cell0 + x1) * m[c * g.n + cell0 + x1];
    }
    s[r * PST + n] = v;
  }
  __syncthreads();
  Fft<L, -1, ROWS, NT, PST>::run(s, tw);
  // X_k = E_k + W_P^k O_k with E = (Z_k + Z*_{L-k}) / 2, O = (Z_k - Z*_{L-k}) / (2i)
  for (int e = threadIdx.x; e < ROWS * (L + 1); e += NT) {
    const int r = e / (L + 1), k = e % (L + 1), row = row0 + r;
    if (row >= nrows) continue;
    const float2 zk = s[r * PST + (k & (L - 1))];
    const float2 zc = cconj(s[r * PST + ((L - k) & (L - 1))]);
    const float2 E = cscale(cadd(zk, zc), 0.5f);
    const float2 d = csub(zk, zc);
    const float2 O = make_float2(0.5f * d.y, -0.5f * d.x);
    const float2 w = __ldg(&tw[k * (kTwN / (2 * L))]);
    const int c = row / (g.nz * g.ny), zy = row % (g.nz * g.ny);
    const int z = zy / g.ny, y = zy % g.ny;
    spec[c * g.sc + ((long long)z * g.srows + y) * g.hxs + k] = cadd(E, cmul(w, O));
  }
}

// nx == 1: the x "transform" is the identity
__global__ void k_fx_copy(Geom g, const float* __restrict__ m, const uint8_t* __restrict__ mask,
                          const uint8_t* __restrict__ region, const RegionLUT* __restrict__ lut,
                          float2* __restrict__ spec, const DevState* __restrict__ st) {
  if (st && st->done) return;
  const int nrows = 3 * g.nz * g.ny;
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= nrows) return;
  const int c = row / (g.nz * g.ny), zy = row % (g.nz * g.ny);
  const int z = zy / g.ny, y = zy % g.ny;
  spec[c * g.sc + ((long long)z * g.srows + y) * g.hxs] =
      make_float2(cell_msat(lut, mask, region, zy) * m[c * g.n + zy], 0.f);
}

// ----------------------------------------------------------------------------
// IX: half spectrum -> real rows (cropped to nx)
// ----------------------------------------------------------------------------
template <int L, int ROWS, int NT>
__global__ void __launch_bounds__(NT) k_ix(Geom g, const float2* __restrict__ spec, float* __restrict__ out,
                                           const float2* __restrict__ tw, const DevState* __restrict__ st) {
  if (st && st->done) return;
  constexpr int PST = L + 1;
  __shared__ float2 s[ROWS * PST];
  const int nrows = 3 * g.nz * g.ny;
  const int row0 = blockIdx.x * ROWS;
  for (int e = threadIdx.x; e < ROWS * (L + 1); e += NT) {
    const int r = e / (L + 1), k = e % (L + 1), row = row0 + r;
    float2 v = make_float2(0.f, 0.f);
    if (row < nrows) {
      const int c = row / (g.nz * g.ny), zy = row % (g.nz * g.ny);
      const int z = zy / g.ny, y = zy % g.ny;
      v = spec[c * g.sc + ((long long)z * g.srows + y) * g.hxs + k];
    }
    s[r * PST + k] = v;
  }
  __syncthreads();
  // Z_k = E_k + i O_k,  E = (X_k + X*_{L-k}) / 2,  O = (X_k - X*_{L-k}) W_P^{-k} / 2;
  // one thread owns the pair (k, L - k), so the update is in place
  for (int e = threadIdx.x; e < ROWS * (L / 2 + 1); e += NT) {
    const int r = e / (L / 2 + 1), k = e % (L / 2 + 1);
    const float2 xa = s[r * PST + k], xb = s[r * PST + L - k];
    float2 za, zb;
    {
      const float2 E = cscale(cadd(xa, cconj(xb)), 0.5f);
      const float2 w = cconj(__ldg(&tw[k * (kTwN / (2 * L))]));
      const float2 O = cmul(cscale(csub(xa, cconj(xb)), 0.5f), w);
      za = make_float2(E.x - O.y, E.y + O.x);
    }
    {
      const int kb = L - k;
      const float2 E = cscale(cadd(xb, cconj(xa)), 0.5f);
      const float2 w = cconj(__ldg(&tw[kb * (kTwN / (2 * L))]));
      const float2 O = cmul(cscale(csub(xb, cconj(xa)), 0.5f), w);
      zb = make_float2(E.x - O.y, E.y + O.x);
    }
    s[r * PST + k] = za;
    if (k != 0 && k != L / 2) s[r * PST + L - k] = zb;
  }
  __syncthreads();
  Fft<L, 1, ROWS, NT, PST>::run(s, tw);
  for (int e = threadIdx.x; e < ROWS * L; e += NT) {
    const int r = e / L, n = e % L, row = row0 + r;
    if (row >= nrows) continue;
    const int c = row / (g.nz * g.ny), zy = row % (g.nz * g.ny);
    const long long cell0 = (long long)zy * g.nx;
    const float2 v = s[r * PST + n];
    if (2 * n < g.nx) out[c * g.n + cell0 + 2 * n] = v.x;
    if (2 * n + 1 < g.nx) out[c * g.n + cell0 + 2 * n + 1] = v.y;
  }
}

__global__ void k_ix_copy(Geom g, const float2* __restrict__ spec, float* __restrict__ out,
                          const DevState* __restrict__ st) {
  if (st && st->done) return;
  const int nrows = 3 * g.nz * g.ny;
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= nrows) return;
  const int c = row / (g.nz * g.ny), zy = row % (g.nz * g.ny);
  const int z = zy / g.ny, y = zy % g.ny;
  out[c * g.n + zy] = spec[c * g.sc + ((long long)z * g.srows + y) * g.hxs].x;
}

// ----------------------------------------------------------------------------
// Kernel multiply: B = K M with K real symmetric; octant lookup with mirror
// signs (Nxy odd in y, Nxz odd in z, Nyz odd in y and z; x never mirrors in
// the half spectrum).
// ----------------------------------------------------------------------------
__device__ __forceinline__ void kernel_multiply(const Geom& g, const float* __restrict__ kt, int kx, int ky, int kz,
                                                float2& X, float2& Y, float2& Z) {
  int iy = ky, iz = kz;
  float sy = 1.f, sz = 1.f;
  if (ky > g.py / 2) { iy = g.py - ky; sy = -1.f; }
  if (kz > g.pz / 2) { iz = g.pz - kz; sz = -1.f; }
  const long long per = (long long)g.hkx * g.hky * g.hkz;
  const long long o = ((long long)iz * g.hky + iy) * g.hkx + kx;
  const float kxx = __ldg(&kt[o]), kyy = __ldg(&kt[per + o]), kzz = __ldg(&kt[2 * per + o]);
  const float kxy = sy * __ldg(&kt[3 * per + o]);
  const float kxz = sz * __ldg(&kt[4 * per + o]);
  const float kyz = sy * sz * __ldg(&kt[5 * per + o]);
  const float2 bx = make_float2(kxx * X.x + kxy * Y.x + kxz * Z.x, kxx * X.y + kxy * Y.y + kxz * Z.y);
  const float2 by = make_float2(kxy * X.x + kyy * Y.x + kyz * Z.x, kxy * X.y + kyy * Y.y + kyz * Z.y);
  const float2 bz = make_float2(kxz * X.x + kyz * Y.x + kzz * Z.x, kxz * X.y + kyz * Y.y + kzz * Z.y);
  X = bx;
  Y = by;
  Z = bz;
}

// ----------------------------------------------------------------------------
// Column passes along y (axis 1) or z (axis 2) on TK consecutive kx columns,
// all three components per block.
// ----------------------------------------------------------------------------
enum { MODE_FWD = 0, MODE_INV = 1, MODE_FMI = 2 };

template <int L, int MODE, int AXIS, int TK, int NT>
__global__ void __launch_bounds__(NT) k_col(Geom g, float2* __restrict__ spec, const float* __restrict__ kt,
                                            const float2* __restrict__ tw, const DevState* __restrict__ st) {
  if (st && st->done) return;
  constexpr int PST = L + 1;
  constexpr int NP = 3 * TK;
  extern __shared__ float2 s[];
  const int kx0 = blockIdx.x * TK;
  const int other = blockIdx.y;     // z plane (AXIS 1) or ky row (AXIS 2)
  long long base, estride;
  int n_in, n_out;
  if (AXIS == 1) {
    base = (long long)other * g.srows * g.hxs + kx0;
    estride = g.hxs;
    n_in = MODE == MODE_INV ? L : g.ny;
    n_out = MODE == MODE_FWD ? L : g.ny;
  } else {
    base = (long long)other * g.hxs + kx0;
    estride = (long long)g.srows * g.hxs;
    n_in = MODE == MODE_INV ? L : g.nz;
    n_out = MODE == MODE_FWD ? L : g.nz;
  }
  for (int e = threadIdx.x; e < 3 * TK * L; e += NT) {
    const int t = e % TK, i = (e / TK) % L, c = e / (TK * L);
    float2 v = make_float2(0.f, 0.f);
    if (i < n_in && kx0 + t < g.hx) v = spec[c * g.sc + base + i * estride + t];
    s[(c * TK + t) * PST + i] = v;
  }
  __syncthreads();
  if (MODE == MODE_INV) {
    Fft<L, 1, NP, NT, PST>::run(s, tw);
  } else {
    Fft<L, -1, NP, NT, PST>::run(s, tw);
  }
  if (MODE == MODE_FMI) {
    for (int e = threadIdx.x; e < TK * L; e += NT) {
      const int t = e % TK, i = e / TK;
      const int kx = kx0 + t;
      if (kx >= g.hx) continue;
      float2 X = s[(0 * TK + t) * PST + i], Y = s[(1 * TK + t) * PST + i], Z = s[(2 * TK + t) * PST + i];
      if (AXIS == 1) kernel_multiply(g, kt, kx, i, 0, X, Y, Z);
      else kernel_multiply(g, kt, kx, other, i, X, Y, Z);
      s[(0 * TK + t) * PST + i] = X;
      s[(1 * TK + t) * PST + i] = Y;
      s[(2 * TK + t) * PST + i] = Z;
    }
    __syncthreads();
    Fft<L, 1, NP, NT, PST>::run(s, tw);
  }
  for (int e = threadIdx.x; e < 3 * TK * n_out; e += NT) {
    const int t = e % TK, i = (e / TK) % n_out, c = e / (TK * n_out);
    if (kx0 + t < g.hx) spec[c * g.sc + base + i * estride + t] = s[(c * TK + t) * PST + i];
  }
}

// py == pz == 1: multiply the single row in place
__global__ void k_mul_row(Geom g, float2* __restrict__ spec, const float* __restrict__ kt,
                          const DevState* __restrict__ st) {
  if (st && st->done) return;
  const int kx = blockIdx.x * blockDim.x + threadIdx.x;
  if (kx >= g.hx) return;
  float2 X = spec[kx], Y = spec[g.sc + kx], Z = spec[2 * g.sc + kx];
  kernel_multiply(g, kt, kx, 0, 0, X, Y, Z);
  spec[kx] = X;
  spec[g.sc + kx] = Y;
  spec[2 * g.sc + kx] = Z;
}

// ----------------------------------------------------------------------------
// dispatch
// ----------------------------------------------------------------------------
template <int L>
struct RowCfg {
  static constexpr int ROWS = L >= 1024 ? 1 : 1024 / L;
  static constexpr int NT = 128;
};

template <int L>
void run_fx(const Geom& g, const Buffers& b, const float* m, cudaStream_t s) {
  using C = RowCfg<L>;
  const int nrows = 3 * g.nz * g.ny;
  k_fx<L, C::ROWS, C::NT><<<(nrows + C::ROWS - 1) / C::ROWS, C::NT, 0, s>>>(g, m, b.mask, b.region, b.lut,
                                                                          b.spec, b.tw, b.st);
}
template <int L>
void run_ix(const Geom& g, const Buffers& b, cudaStream_t s) {
  using C = RowCfg<L>;
  const int nrows = 3 * g.nz * g.ny;
  k_ix<L, C::ROWS, C::NT><<<(nrows + C::ROWS - 1) / C::ROWS, C::NT, 0, s>>>(g, b.spec, b.bd, b.tw, b.st);
}

template <int L>
struct ColCfg {
  static constexpr int TK = L >= 2048 ? 1 : (2048 / L > 16 ? 16 : 2048 / L);
  static constexpr int NT0 = 3 * TK * L / 16;
  static constexpr int NT = NT0 < 64 ? 64 : (NT0 > 512 ? 512 : NT0);
  static constexpr size_t SMEM = sizeof(float2) * 3 * TK * (L + 1);
};

template <int L, int MODE, int AXIS>
void run_col(const Geom& g, const Buffers& b, cudaStream_t s) {
  using C = ColCfg<L>;
  auto kern = k_col<L, MODE, AXIS, C::TK, C::NT>;
  // (a function attribute belongs to the current device's context: set on
  // every launch, a host-side call that enqueues nothing)
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
  const int others = AXIS == 1 ? g.nz : g.py;
  dim3 grid((g.hx + C::TK - 1) / C::TK, others);
  kern<<<grid, C::NT, C::SMEM, s>>>(g, b.spec, b.kt, b.tw, b.st);
}

#define MM_DISPATCH_L(LEN, CALL)          \
  switch (LEN) {                          \
    case 2: CALL(2); break;               \
    case 4: CALL(4); break;               \
    case 8: CALL(8); break;               \
    case 16: CALL(16); break;             \
    case 32: CALL(32); break;             \
    case 64: CALL(64); break;             \
    case 128: CALL(128); break;           \
    case 256: CALL(256); break;           \
    case 512: CALL(512); break;           \
    case 1024: CALL(1024); break;         \
    default: break;                       \
  }

}  // namespace

void launch_demag(const Geom& g, const Buffers& b, const float* m, cudaStream_t s) {
  if (g.fused) {
    launch_demag_fused(g, b, m, s);
    return;
  }
  const int nrows = 3 * g.nz * g.ny;
  // FX
  if (g.px == 1) {
    k_fx_copy<<<(nrows + 127) / 128, 128, 0, s>>>(g, m, b.mask, b.region, b.lut, b.spec, b.st);
  } else {
#define CALL_FX(LL) run_fx<LL>(g, b, m, s)
    MM_DISPATCH_L(g.lx, CALL_FX)
#undef CALL_FX
  }
  // middle passes
  if (g.pz > 1) {
    if (g.py > 1) {
#define CALL_FY(LL) run_col<LL, MODE_FWD, 1>(g, b, s)
      MM_DISPATCH_L(g.py, CALL_FY)
#undef CALL_FY
    }
#define CALL_FZ(LL) run_col<LL, MODE_FMI, 2>(g, b, s)
    MM_DISPATCH_L(g.pz, CALL_FZ)
#undef CALL_FZ
    if (g.py > 1) {
#define CALL_IY(LL) run_col<LL, MODE_INV, 1>(g, b, s)
      MM_DISPATCH_L(g.py, CALL_IY)
#undef CALL_IY
    }
  } else if (g.py > 1) {
#define CALL_FYMI(LL) run_col<LL, MODE_FMI, 1>(g, b, s)
    MM_DISPATCH_L(g.py, CALL_FYMI)
#undef CALL_FYMI
  } else {
    k_mul_row<<<(g.hx + 127) / 128, 128, 0, s>>>(g, b.spec, b.kt, b.st);
  }
  // IX
  if (g.px == 1) {
    k_ix_copy<<<(nrows + 127) / 128, 128, 0, s>>>(g, b.spec, b.bd, b.st);
  } else {
#define CALL_IX(LL) run_ix<LL>(g, b, s)
    MM_DISPATCH_L(g.lx, CALL_IX)
#undef CALL_IX
  }
}

}  // namespace mm
