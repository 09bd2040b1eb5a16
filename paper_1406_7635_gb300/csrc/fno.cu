// Fourier-neural-operator surrogate of the demag field: forward, backward and
// Adam on the GPU (the learned form of the demag convolution of Sec. III.B).
//
//   v_0 = P u + p,  v_{l+1} = act_l(W_l v_l + b_l + K_l v_l),  y = Q v_L + q
//
// u = M / Ms_ref (3 channels on an H x W film), y = B_demag / (mu0 Ms_ref).
// K_l is the truncated spectral convolution written with explicit partial DFT
// matrices (kx < Mx; ky in {0..My-1} U {H-My..H-1}):
//   V = Fy v Fx^T,  O[o] = sum_i R[o,i] V[i] (per mode),  K v = Re(Gy^T O Gx),
// Gx = c_kx exp(+2 pi i kx x / W) / W (c_0 = 1, else 2), Gy = exp(+...)/H.
// act = exact GELU except after the last layer.  Loss: sum |yhat - y|^2 /
// sum |y|^2 over the batch.
//
// Activations are float32, channel-major [C][H][W].  The dense products (lift,
// project, pointwise W, the x-direction partial DFTs and their adjoints) run
// on the tensor cores: operands rounded to bfloat16 while staged in shared
// memory, float32 accumulation (mma m16n8k16).  The y-direction partial DFTs
// and the per-mode channel mixing are small complex products on the FP32
// cores.  Parameters are float32 masters (Adam), used in bfloat16 by the
// tensor-core products.
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_bf16.h>

#include "../../include/mm.h"
#include "mm_internal.h"

namespace mm {
namespace {

__device__ __forceinline__ float gelu_f(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_df(float x) {
  return 0.5f * (1.f + erff(x * 0.70710678118654752f)) + x * 0.3989422804014327f * __expf(-0.5f * x * x);
}

// 4-, 8- and 16-byte asynchronous global -> shared copies (complete at
// cp.async.wait_all; both addresses aligned to the copy size)
__device__ __forceinline__ void cp_async_4(float* dst, const float* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_8(float2* dst, const float2* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_16(float* dst, const float* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}

// ---------------------------------------------------------------------------
// bfloat16 tensor-core GEMM: C[b] = alpha op(A[b]) op(B[b]) + beta C[b]
// (+ bias[m]).  op(A)(m, k) = TA ? A[k lda + m] : A[m lda + k];
// op(B)(k, n) = TB ? B[n ldb + k] : B[k ldb + n].  Split-K (gridDim.z =
// batch * splits) adds alpha * partial into C with atomics (C prepared by the
// caller), or, with sPart > 0, writes split s's partial to C + s sPart (the
// consumer sums the slices in a fixed order: deterministic).  With act set,
// the result is also written to act at the same offset, through the exact
// GELU when act_gelu.  Block tile 64 x 64 x 32, four warps of 32 x 32.
// ---------------------------------------------------------------------------
struct GemmArgs {
  int M, N, K;
  const float* A;
  long long lda, sA;   // leading dimension, batch stride
  const float* B;
  long long ldb, sB;
  float* C;
  long long ldc, sC;
  float alpha, beta;
  const float* bias;   // per-row bias or null
  int splits;          // split-K factor
  int atomic;          // add alpha * product into C with atomics (C prepared by the caller)
  long long sPart;     // > 0: split s writes its partial product to C + s sPart (no bias, beta 0)
  float* act;          // optional second output: act_gelu ? GELU(C) : C
  int act_gelu;
};

constexpr int BM = 64, BN = 64, BK = 32, APITCH = BK + 8;

__device__ __forceinline__ unsigned pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const unsigned*>(&v);
}

template <bool TA, bool TB>
__global__ void __launch_bounds__(128) k_gemm(GemmArgs a) {
  __shared__ __align__(16) __nv_bfloat16 As[BM][APITCH];
  __shared__ __align__(16) __nv_bfloat16 Bs[BN][APITCH];
  const int batch = blockIdx.z / a.splits, split = blockIdx.z % a.splits;
  const float* __restrict__ A = a.A + batch * a.sA;
  const float* __restrict__ B = a.B + batch * a.sB;
  float* __restrict__ Cm = a.C + batch * a.sC + split * a.sPart;
  float* __restrict__ Am = a.act ? a.act + batch * a.sC : nullptr;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int kchunk = ((a.K + a.splits - 1) / a.splits + BK - 1) / BK * BK;
  const int kbeg = split * kchunk, kend = min(a.K, kbeg + kchunk);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
  const int g = lane >> 2, t = lane & 3;
  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.f;

  // operand pairs of one BK step in registers: the next step's global loads
  // are in flight while the tensor cores work on the current one
  constexpr int PA = BM * BK / 2 / 128, PB = BN * BK / 2 / 128;
  float ra[PA][2], rb[PB][2];
  auto load = [&](int k0) {
#pragma unroll
    for (int u = 0; u < PA; ++u) {
      const int e = tid + u * 128;
      int mm_, kk;
      if (TA) { mm_ = (2 * e) % BM; kk = (2 * e) / BM; } else { mm_ = (2 * e) / BK; kk = (2 * e) % BK; }
      const int gm = m0 + mm_, gk = k0 + kk;
      float v0 = 0.f, v1 = 0.f;
      if (TA) {
        if (gk < kend) {
          if (gm < a.M) v0 = A[(long long)gk * a.lda + gm];
          if (gm + 1 < a.M) v1 = A[(long long)gk * a.lda + gm + 1];
        }
      } else if (gm < a.M) {
        if (gk < kend) v0 = A[(long long)gm * a.lda + gk];
        if (gk + 1 < kend) v1 = A[(long long)gm * a.lda + gk + 1];
      }
      ra[u][0] = v0;
      ra[u][1] = v1;
    }
#pragma unroll
    for (int u = 0; u < PB; ++u) {
      const int e = tid + u * 128;
      int nn, kk;
      if (TB) { nn = (2 * e) / BK; kk = (2 * e) % BK; } else { nn = (2 * e) % BN; kk = (2 * e) / BN; }
      const int gn = n0 + nn, gk = k0 + kk;
      float v0 = 0.f, v1 = 0.f;
      if (TB) {
        if (gn < a.N) {
          if (gk < kend) v0 = B[(long long)gn * a.ldb + gk];
          if (gk + 1 < kend) v1 = B[(long long)gn * a.ldb + gk + 1];
        }
      } else if (gk < kend) {
        if (gn < a.N) v0 = B[(long long)gk * a.ldb + gn];
        if (gn + 1 < a.N) v1 = B[(long long)gk * a.ldb + gn + 1];
      }
      rb[u][0] = v0;
      rb[u][1] = v1;
    }
  };
  // stage A (BM x BK) and B (BN x BK), k contiguous in shared memory
  auto store = [&]() {
#pragma unroll
    for (int u = 0; u < PA; ++u) {
      const int e = tid + u * 128;
      if (TA) {
        const int mm_ = (2 * e) % BM, kk = (2 * e) / BM;
        As[mm_][kk] = __float2bfloat16_rn(ra[u][0]);
        As[mm_ + 1][kk] = __float2bfloat16_rn(ra[u][1]);
      } else {
        const int mm_ = (2 * e) / BK, kk = (2 * e) % BK;
        *reinterpret_cast<unsigned*>(&As[mm_][kk]) = pack_bf16(ra[u][0], ra[u][1]);
      }
    }
#pragma unroll
    for (int u = 0; u < PB; ++u) {
      const int e = tid + u * 128;
      if (TB) {
        const int nn = (2 * e) / BK, kk = (2 * e) % BK;
        *reinterpret_cast<unsigned*>(&Bs[nn][kk]) = pack_bf16(rb[u][0], rb[u][1]);
      } else {
        const int nn = (2 * e) % BN, kk = (2 * e) / BN;
        Bs[nn][kk] = __float2bfloat16_rn(rb[u][0]);
        Bs[nn + 1][kk] = __float2bfloat16_rn(rb[u][1]);
      }
    }
  };

  if (kbeg < kend) load(kbeg);
  for (int k0 = kbeg; k0 < kend; k0 += BK) {
    store();
    __syncthreads();
    if (k0 + BK < kend) load(k0 + BK);
#pragma unroll
    for (int ks = 0; ks < BK; ks += 16) {
      unsigned af[2][4], bfr[4][2];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const int r = wm + 16 * i + g;
        af[i][0] = *reinterpret_cast<const unsigned*>(&As[r][ks + 2 * t]);
        af[i][1] = *reinterpret_cast<const unsigned*>(&As[r + 8][ks + 2 * t]);
        af[i][2] = *reinterpret_cast<const unsigned*>(&As[r][ks + 2 * t + 8]);
        af[i][3] = *reinterpret_cast<const unsigned*>(&As[r + 8][ks + 2 * t + 8]);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int c = wn + 8 * j + g;
        bfr[j][0] = *reinterpret_cast<const unsigned*>(&Bs[c][ks + 2 * t]);
        bfr[j][1] = *reinterpret_cast<const unsigned*>(&Bs[c][ks + 2 * t + 8]);
      }
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
          asm volatile(
              "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
              "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
              : "+f"(acc[i][j][0]), "+f"(acc[i][j][1]), "+f"(acc[i][j][2]), "+f"(acc[i][j][3])
              : "r"(af[i][0]), "r"(af[i][1]), "r"(af[i][2]), "r"(af[i][3]), "r"(bfr[j][0]), "r"(bfr[j][1]));
    }
    __syncthreads();
  }
  // epilogue
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int row = m0 + wm + 16 * i + g + (r >= 2 ? 8 : 0);
        const int col = n0 + wn + 8 * j + 2 * t + (r & 1);
        if (row >= a.M || col >= a.N) continue;
        const long long o = (long long)row * a.ldc + col;
        float* dst = Cm + o;
        const float v = a.alpha * acc[i][j][r];
        if (a.atomic) {
          atomicAdd(dst, v);
        } else {
          float out = v + (a.bias ? a.bias[row] : 0.f);
          if (a.beta != 0.f) out += a.beta * *dst;
          *dst = out;
          if (Am) Am[o] = a.act_gelu ? gelu_f(out) : out;
        }
      }
}

void gemm(cudaStream_t s, bool ta, bool tb, int batch, const GemmArgs& a) {
  dim3 grid((a.N + BN - 1) / BN, (a.M + BM - 1) / BM, batch * a.splits);
  if (!ta && !tb) k_gemm<false, false><<<grid, 128, 0, s>>>(a);
  else if (ta && !tb) k_gemm<true, false><<<grid, 128, 0, s>>>(a);
  else if (!ta && tb) k_gemm<false, true><<<grid, 128, 0, s>>>(a);
  else k_gemm<true, true><<<grid, 128, 0, s>>>(a);
}

GemmArgs gargs(int M, int N, int K, const float* A, long long lda, long long sA, const float* B, long long ldb,
               long long sB, float* C, long long ldc, long long sC, float alpha = 1.f, float beta = 0.f,
               const float* bias = nullptr, int splits = 1, int atomic = 0) {
  return GemmArgs{M, N, K, A, lda, sA, B, ldb, sB, C, ldc, sC, alpha, beta, bias, splits, atomic || splits > 1,
                  0, nullptr, 0};
}

// split-K into `parts` slices part_stride floats apart (see GemmArgs::sPart)
GemmArgs sliced(GemmArgs a, int parts, long long part_stride) {
  a.splits = parts;
  a.atomic = 0;
  a.sPart = part_stride;
  return a;
}

// second output through GELU (gelu) or as is
GemmArgs with_act(GemmArgs a, float* act, bool gelu) {
  a.act = act;
  a.act_gelu = gelu ? 1 : 0;
  return a;
}

// ---------------------------------------------------------------------------
// small complex kernels (FP32 cores)
// ---------------------------------------------------------------------------
// Y[c][j][k] = sum_y F[j][y] * X[c][y][k]; X blocked real [c][y][re Mx | im Mx]
// (if xin_blocked) or complex [c][y][k]; conj_f conjugates F.  Output complex.
__global__ void k_ysum(int S, int C, int H, int J, int Mx, const float* __restrict__ X, bool x_blocked,
                       const float2* __restrict__ F, bool conj_f, float2* __restrict__ Y) {
  const long long total = (long long)S * C * J * Mx;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  const int k = (int)(i % Mx), j = (int)((i / Mx) % J);
  const long long sc = i / ((long long)Mx * J);   // sample * C + c
  float re = 0.f, im = 0.f;
  for (int y = 0; y < H; ++y) {
    float2 f = F[(long long)j * H + y];
    if (conj_f) f.y = -f.y;
    float xr, xi;
    if (x_blocked) {
      const float* row = X + (sc * H + y) * 2 * Mx;
      xr = row[k];
      xi = row[Mx + k];
    } else {
      const float2 v = reinterpret_cast<const float2*>(X)[(sc * H + y) * Mx + k];
      xr = v.x;
      xi = v.y;
    }
    re = fmaf(f.x, xr, fmaf(-f.y, xi, re));
    im = fmaf(f.x, xi, fmaf(f.y, xr, im));
  }
  Y[i] = make_float2(re, im);
}

// Z[c][y][re k | im k] = sum_j F[j][y] * O[c][j][k] (conj_f: conj(F)), blocked real output
__global__ void k_yexpand(int S, int C, int H, int J, int Mx, const float2* __restrict__ O,
                          const float2* __restrict__ F, bool conj_f, float* __restrict__ Z) {
  const long long total = (long long)S * C * H * Mx;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  const int k = (int)(i % Mx), y = (int)((i / Mx) % H);
  const long long sc = i / ((long long)Mx * H);
  float re = 0.f, im = 0.f;
  for (int j = 0; j < J; ++j) {
    float2 f = F[(long long)j * H + y];
    if (conj_f) f.y = -f.y;
    const float2 o = O[(sc * J + j) * Mx + k];
    re = fmaf(f.x, o.x, fmaf(-f.y, o.y, re));
    im = fmaf(f.x, o.y, fmaf(f.y, o.x, im));
  }
  float* row = Z + (sc * H + y) * 2 * Mx;
  row[k] = re;
  row[Mx + k] = im;
}

// The same two products tiled through shared memory (one block per sample and
// channel and group of frequencies, or of rows): the one-thread-per-output
// kernels above walk a whole column of global memory per thread, which is
// latency-bound.  Same summation order per output (y, resp. j, ascending).
constexpr int kYNT = 256;
constexpr int kXParts = 4;   // most split-K slices of the x partial DFT products
constexpr int kYSplit = 8;   // most row ranges of the tiled y product

// as k_ysum; blocked X may be split-K partials: the sum of `parts` slices
// part_stride floats apart (slice 0 first).  Block (j group, sc, row range):
// JB frequencies x Mx columns over rows [z YR, (z + 1) YR), staged YC rows
// at a time; range z writes its partial sums to Y + z y_stride (one range:
// the result itself).
__global__ void __launch_bounds__(kYNT) k_ysum_t(int H, int J, int Mx, int JB, int YC, int YR,
                                               const float* __restrict__ X, bool x_blocked, int parts,
                                               long long part_stride, const float2* __restrict__ F, bool conj_f,
                                               float2* __restrict__ Y, long long y_stride) {
  extern __shared__ float2 ysh[];
  float2* xs = ysh;             // [YC][Mx]
  float2* fs = ysh + YC * Mx;   // [JB][YC]
  const long long sc = blockIdx.y;
  const int j0 = blockIdx.x * JB, jn = min(JB, J - j0);
  const int tid = threadIdx.x, jj = tid / Mx, k = tid % Mx;
  const bool mine = jj < jn;
  float re = 0.f, im = 0.f;
  const int ybeg = blockIdx.z * YR, yend = min(H, ybeg + YR);
  Y += blockIdx.z * y_stride;
  for (int y0 = ybeg; y0 < yend; y0 += YC) {
    const int yn = min(YC, yend - y0);
    for (int e = tid; e < yn * Mx; e += kYNT) {
      const int yy = e / Mx, kk = e % Mx;
      const long long ri = sc * H + y0 + yy;
      float2 v;
      if (x_blocked) {
        const float* row = X + ri * 2 * Mx;
        v = make_float2(row[kk], row[Mx + kk]);
        for (int q = 1; q < parts; ++q) {
          v.x += row[q * part_stride + kk];
          v.y += row[q * part_stride + Mx + kk];
        }
      } else {
        v = reinterpret_cast<const float2*>(X)[ri * Mx + kk];
      }
      xs[yy * Mx + kk] = v;
    }
    for (int e = tid; e < jn * yn; e += kYNT) {
      const int a = e / yn, yy = e % yn;
      float2 f = F[(long long)(j0 + a) * H + y0 + yy];
      if (conj_f) f.y = -f.y;
      fs[a * YC + yy] = f;
    }
    __syncthreads();
    if (mine) {
      for (int yy = 0; yy < yn; ++yy) {
        const float2 f = fs[jj * YC + yy], x = xs[yy * Mx + k];
        re = fmaf(f.x, x.x, fmaf(-f.y, x.y, re));
        im = fmaf(f.x, x.y, fmaf(f.y, x.x, im));
      }
    }
    __syncthreads();
  }
  if (mine) Y[(sc * J + j0 + jj) * Mx + k] = make_float2(re, im);
}

// dst[i] = sum_z src[z stride + i] over z < parts (ascending)
__global__ void k_sum_parts(long long n, int parts, long long stride, const float2* __restrict__ src,
                            float2* __restrict__ dst) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float2 a = src[i];
  for (int z = 1; z < parts; ++z) {
    const float2 b = src[z * stride + i];
    a.x += b.x;
    a.y += b.y;
  }
  dst[i] = a;
}

// as k_yexpand; block (row group, sc): O[sc] (J x Mx) and F[:, y0 .. y0+YB)
// staged by asynchronous copies (conj_f applied at use), YB x Mx outputs
__global__ void __launch_bounds__(kYNT) k_yexpand_t(int H, int J, int Mx, int YB, const float2* __restrict__ O,
                                                  const float2* __restrict__ F, bool conj_f, float* __restrict__ Z) {
  extern __shared__ float2 ysh[];
  float2* os = ysh;             // [J][Mx]
  float2* fs = ysh + J * Mx;    // [J][YB]
  const long long sc = blockIdx.y;
  const int y0 = blockIdx.x * YB, yn = min(YB, H - y0);
  const int tid = threadIdx.x;
  for (int e = tid; e < J * Mx; e += kYNT) cp_async_8(&os[e], &O[sc * J * Mx + e]);
  for (int e = tid; e < J * yn; e += kYNT) {
    const int j = e / yn, yy = e % yn;
    cp_async_8(&fs[j * YB + yy], &F[(long long)j * H + y0 + yy]);
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  __syncthreads();
  const float cs = conj_f ? -1.f : 1.f;
  for (int e = tid; e < yn * Mx; e += kYNT) {
    const int yy = e / Mx, k = e % Mx;
    float re = 0.f, im = 0.f;
    for (int j = 0; j < J; ++j) {
      float2 f = fs[j * YB + yy];
      f.y *= cs;
      const float2 o = os[j * Mx + k];
      re = fmaf(f.x, o.x, fmaf(-f.y, o.y, re));
      im = fmaf(f.x, o.y, fmaf(f.y, o.x, im));
    }
    float* row = Z + (sc * H + y0 + yy) * 2 * Mx;
    row[k] = re;
    row[Mx + k] = im;
  }
}

// tile shapes of the two (shared memory <= 48 KB)
struct YTile {
  int JB, YC;   // ysum: frequencies per block, rows per stage
  int YB;       // yexpand: rows per block (0: untiled kernel)
  bool ysum;    // ysum tiled
  int ysplit;   // ysum: row ranges (partials summed by k_sum_parts)
};
YTile ytile(int S, int C, int H, int J, int Mx, int sms) {
  YTile t{};
  t.ysum = Mx <= kYNT && (long long)S * C <= 65535;
  t.ysplit = 1;
  if (t.ysum) {
    t.JB = std::min(J, std::min(64, kYNT / Mx));
    t.YC = std::max(1, std::min(64, 2048 / Mx));
    // row ranges until about four blocks per multiprocessor, at least a stage each
    const long long blocks = (long long)((J + t.JB - 1) / t.JB) * S * C;
    const long long want = (4LL * sms + blocks - 1) / blocks;
    t.ysplit = (int)std::max<long long>(1, std::min<long long>(std::min<long long>(want, kYSplit),
                                                                 (H + t.YC - 1) / t.YC));
  }
  t.YB = 0;
  if ((long long)S * C <= 65535 && J * Mx <= 4096) {
    const int yb = (6144 - J * Mx) / J;   // (J Mx + J YB) float2 <= 48 KB
    t.YB = std::min(H, std::min(64, yb));
    if (t.YB < 1) t.YB = 0;
  }
  return t;
}

// (Yp: kYSplit S C J Mx float2 of scratch for the row-range partials)
void ysum(cudaStream_t s, const YTile& t, int S, int C, int H, int J, int Mx, const float* X, bool blocked, int parts,
          long long part_stride, const float2* F, bool conj_f, float2* Y, float2* Yp) {
  if (!t.ysum) {   // (parts == 1 here: sliced products are only made for the tiled kernel)
    k_ysum<<<(unsigned)(((long long)S * C * J * Mx + 255) / 256), 256, 0, s>>>(S, C, H, J, Mx, X, blocked, F, conj_f, Y);
    return;
  }
  const int YR = (H + t.ysplit - 1) / t.ysplit;
  const dim3 grid((J + t.JB - 1) / t.JB, S * C, t.ysplit);
  const size_t smem = (size_t)(t.YC * Mx + t.JB * t.YC) * sizeof(float2);
  const long long n = (long long)S * C * J * Mx;
  k_ysum_t<<<grid, kYNT, smem, s>>>(H, J, Mx, t.JB, t.YC, YR, X, blocked, parts, part_stride, F, conj_f,
                                    t.ysplit > 1 ? Yp : Y, n);
  if (t.ysplit > 1) k_sum_parts<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, t.ysplit, n, Yp, Y);
}

void yexpand(cudaStream_t s, const YTile& t, int S, int C, int H, int J, int Mx, const float2* O, const float2* F,
             bool conj_f, float* Z) {
  if (t.YB == 0) {
    k_yexpand<<<(unsigned)(((long long)S * C * H * Mx + 255) / 256), 256, 0, s>>>(S, C, H, J, Mx, O, F, conj_f, Z);
    return;
  }
  const dim3 grid((H + t.YB - 1) / t.YB, S * C);
  const size_t smem = (size_t)(J * Mx + J * t.YB) * sizeof(float2);
  k_yexpand_t<<<grid, kYNT, smem, s>>>(H, J, Mx, t.YB, O, F, conj_f, Z);
}

// Pointwise channel products on the FP32 cores, one thread per pixel (these
// are memory-bound: a tensor-core GEMM with M = C rows leaves most of its
// tile idle and needs a second pass for the activation):
//   out[s][o][p] = bias[o] + (SPEC: sum_k Zb[s][o][y][k] G[k][x]) + sum_i A[o][i] in[s][i][p]
// with p = y W + x; ACT 1 also writes GELU(out) to act, ACT 2 a copy.  The
// spectral part is the inverse x partial DFT of the layer (Zb blocked
// [re Mx | im Mx] rows, G = Gblk).  A block is kPwNT pixels of one image
// row; it stages A, that row of Zb (as [i][o] and [k][o]: pitch a multiple of
// 4 plus 4 floats, aligned float4 reads) and its columns of G ([k][pixel])
// in shared memory with asynchronous copies, all in flight together.
constexpr int kPwNT = 128;
__host__ __device__ constexpr int pw_pitch(int co) { return (co + 3) / 4 * 4 + 4; }


template <int CI, int CO, bool SPEC, int ACT>
__global__ void __launch_bounds__(kPwNT) k_pointwise(int H, int W, int K2, const float* __restrict__ A,
                                                   const float* __restrict__ bias, const float* __restrict__ in,
                                                   const float* __restrict__ Zb, const float* __restrict__ G,
                                                   float* __restrict__ out, float* __restrict__ act) {
  constexpr int P = pw_pitch(CO);
  extern __shared__ __align__(16) float pws[];
  float* As = pws;                  // [CI][P]
  float* Zs = pws + CI * P;         // [K2][P]
  float* Gs = Zs + K2 * P;          // [K2][kPwNT]
  const int x0 = blockIdx.x * kPwNT, x = x0 + threadIdx.x, y = blockIdx.y, s = blockIdx.z;
  for (int e = threadIdx.x; e < CI * CO; e += kPwNT) cp_async_4(&As[(e % CI) * P + e / CI], &A[e]);
  if (SPEC) {
    const float* zrow = Zb + ((long long)s * CO * H + y) * K2;   // + o H K2 + k
    for (int e = threadIdx.x; e < K2 * CO; e += kPwNT) {
      const int o = e / K2, k = e % K2;
      cp_async_4(&Zs[k * P + o], &zrow[(long long)o * H * K2 + k]);
    }
    if (x < W)
      for (int k = 0; k < K2; ++k) cp_async_4(&Gs[k * kPwNT + threadIdx.x], &G[(long long)k * W + x]);
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  __syncthreads();
  if (x >= W) return;
  const long long N = (long long)H * W, px = (long long)y * W + x;
  float vi[CI];
#pragma unroll
  for (int i = 0; i < CI; ++i) vi[i] = in[((long long)s * CI + i) * N + px];
  float acc[CO];
#pragma unroll
  for (int o = 0; o < CO; ++o) acc[o] = __ldg(&bias[o]);
  if (SPEC) {
#pragma unroll 4
    for (int k = 0; k < K2; ++k) {
      const float g = Gs[k * kPwNT + threadIdx.x];
      const float* zr = Zs + k * P;
#pragma unroll
      for (int o = 0; o < CO; o += 4) {
        const float4 z4 = *reinterpret_cast<const float4*>(zr + o);
        acc[o] = fmaf(z4.x, g, acc[o]);
        if (o + 1 < CO) acc[o + 1] = fmaf(z4.y, g, acc[o + 1]);
        if (o + 2 < CO) acc[o + 2] = fmaf(z4.z, g, acc[o + 2]);
        if (o + 3 < CO) acc[o + 3] = fmaf(z4.w, g, acc[o + 3]);
      }
    }
  }
#pragma unroll
  for (int i = 0; i < CI; ++i) {
    const float* ar = As + i * P;
#pragma unroll
    for (int o = 0; o < CO; o += 4) {
      const float4 a4 = *reinterpret_cast<const float4*>(ar + o);
      acc[o] = fmaf(a4.x, vi[i], acc[o]);
      if (o + 1 < CO) acc[o + 1] = fmaf(a4.y, vi[i], acc[o + 1]);
      if (o + 2 < CO) acc[o + 2] = fmaf(a4.z, vi[i], acc[o + 2]);
      if (o + 3 < CO) acc[o + 3] = fmaf(a4.w, vi[i], acc[o + 3]);
    }
  }
#pragma unroll
  for (int o = 0; o < CO; ++o) {
    const long long oi = ((long long)s * CO + o) * N + px;
    out[oi] = acc[o];
    if (ACT == 1) act[oi] = gelu_f(acc[o]);
    if (ACT == 2) act[oi] = acc[o];
  }
}

// The layer output for C a multiple of 8, register-blocked: thread (g, q)
// computes channels 8g .. 8g + 7 at pixels 4q .. 4q + 3 of the block's
// kPwNT pixels (C / 8 warps; channel group uniform per warp), so one float4
// of Zs / A (broadcast) and one of G / v feed 32 FMAs.  A, Zb's row, G's
// columns and v's pixels are staged with asynchronous copies; with W a
// multiple of 4 (every row and pixel quad 16-byte aligned) G and v move in
// 16-byte copies and the outputs in float4 stores.
template <int C, int ACT>
__global__ void __launch_bounds__(C * 4) k_layer_pw(int H, int W, int K2, const float* __restrict__ A,
                                                   const float* __restrict__ bias, const float* __restrict__ in,
                                                   const float* __restrict__ Zb, const float* __restrict__ G,
                                                   float* __restrict__ out, float* __restrict__ act) {
  constexpr int NT = C * 4, P = pw_pitch(C);
  static_assert(C % 8 == 0, "channel groups of 8");
  extern __shared__ __align__(16) float pws[];
  float* As = pws;                 // [C][P]      A[o][i] at [i][o]
  float* Zs = As + C * P;          // [K2][P]     Zb[s][o][y][k] at [k][o]
  float* Gs = Zs + K2 * P;         // [K2][kPwNT] G[k][x0 + px]
  float* Vs = Gs + K2 * kPwNT;     // [C][kPwNT]  in[s][i][y][x0 + px]
  const int tid = threadIdx.x, x0 = blockIdx.x * kPwNT, y = blockIdx.y, s = blockIdx.z;
  const long long N = (long long)H * W, row = (long long)y * W + x0;
  const int nx = min(kPwNT, W - x0);
  for (int e = tid; e < C * C; e += NT) cp_async_4(&As[(e % C) * P + e / C], &A[e]);
  const float* zrow = Zb + ((long long)s * C * H + y) * K2;   // + o H K2 + k
  for (int e = tid; e < K2 * C; e += NT) {
    const int o = e / K2, k = e % K2;
    cp_async_4(&Zs[k * P + o], &zrow[(long long)o * H * K2 + k]);
  }
  const float* vin = in + (long long)s * C * N + row;
  const bool vec = (W & 3) == 0;   // (then nx is a multiple of 4 too)
  if (vec) {
    constexpr int Q = kPwNT / 4;
    for (int e = tid; e < K2 * Q; e += NT) {
      const int k = e / Q, px = 4 * (e % Q);
      if (px < nx) cp_async_16(&Gs[k * kPwNT + px], &G[(long long)k * W + x0 + px]);
    }
    for (int e = tid; e < C * Q; e += NT) {
      const int i = e / Q, px = 4 * (e % Q);
      if (px < nx) cp_async_16(&Vs[i * kPwNT + px], &vin[(long long)i * N + px]);
    }
  } else {
    for (int e = tid; e < K2 * kPwNT; e += NT) {
      const int k = e / kPwNT, px = e % kPwNT;
      if (px < nx) cp_async_4(&Gs[e], &G[(long long)k * W + x0 + px]);
    }
    for (int e = tid; e < C * kPwNT; e += NT) {
      const int i = e / kPwNT, px = e % kPwNT;
      if (px < nx) cp_async_4(&Vs[e], &vin[(long long)i * N + px]);
    }
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  __syncthreads();
  const int g = tid / (kPwNT / 4), q = tid % (kPwNT / 4);
  if (4 * q >= nx) return;
  float acc[8][4];
#pragma unroll
  for (int o = 0; o < 8; ++o) {
    const float b = __ldg(&bias[8 * g + o]);
#pragma unroll
    for (int p = 0; p < 4; ++p) acc[o][p] = b;
  }
#pragma unroll 2
  for (int k = 0; k < K2; ++k) {
    const float4 gv = *reinterpret_cast<const float4*>(&Gs[k * kPwNT + 4 * q]);
    const float4 z0 = *reinterpret_cast<const float4*>(&Zs[k * P + 8 * g]);
    const float4 z1 = *reinterpret_cast<const float4*>(&Zs[k * P + 8 * g + 4]);
    const float zz[8] = {z0.x, z0.y, z0.z, z0.w, z1.x, z1.y, z1.z, z1.w}, gg[4] = {gv.x, gv.y, gv.z, gv.w};
#pragma unroll
    for (int o = 0; o < 8; ++o)
#pragma unroll
      for (int p = 0; p < 4; ++p) acc[o][p] = fmaf(zz[o], gg[p], acc[o][p]);
  }
#pragma unroll 4
  for (int i = 0; i < C; ++i) {
    const float4 vv = *reinterpret_cast<const float4*>(&Vs[i * kPwNT + 4 * q]);
    const float4 a0 = *reinterpret_cast<const float4*>(&As[i * P + 8 * g]);
    const float4 a1 = *reinterpret_cast<const float4*>(&As[i * P + 8 * g + 4]);
    const float aa[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w}, vq[4] = {vv.x, vv.y, vv.z, vv.w};
#pragma unroll
    for (int o = 0; o < 8; ++o)
#pragma unroll
      for (int p = 0; p < 4; ++p) acc[o][p] = fmaf(aa[o], vq[p], acc[o][p]);
  }
#pragma unroll
  for (int o = 0; o < 8; ++o) {
    const long long ob = ((long long)s * C + 8 * g + o) * N + row + 4 * q;
    if (vec) {
      *reinterpret_cast<float4*>(out + ob) = make_float4(acc[o][0], acc[o][1], acc[o][2], acc[o][3]);
      if (ACT == 1)
        *reinterpret_cast<float4*>(act + ob) =
            make_float4(gelu_f(acc[o][0]), gelu_f(acc[o][1]), gelu_f(acc[o][2]), gelu_f(acc[o][3]));
      if (ACT == 2) *reinterpret_cast<float4*>(act + ob) = make_float4(acc[o][0], acc[o][1], acc[o][2], acc[o][3]);
      continue;
    }
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      if (4 * q + p >= nx) break;
      out[ob + p] = acc[o][p];
      if (ACT == 1) act[ob + p] = gelu_f(acc[o][p]);
      if (ACT == 2) act[ob + p] = acc[o][p];
    }
  }
}

size_t layer_pw_smem(int C, int K2) {
  return ((size_t)(C + K2) * pw_pitch(C) + (size_t)(K2 + C) * kPwNT) * sizeof(float);
}

// (the shared-memory limit is raised by layer_pw_prepare, outside any graph capture)
template <int C, int ACT>
void launch_layer_pw(cudaStream_t s, int S, int H, int W, int K2, const float* A, const float* bias, const float* in,
                     const float* Zb, const float* G, float* out, float* act) {
  const dim3 grid((W + kPwNT - 1) / kPwNT, H, S);
  k_layer_pw<C, ACT><<<grid, C * 4, layer_pw_smem(C, K2), s>>>(H, W, K2, A, bias, in, Zb, G, out, act);
}

// The limit is raised to the fixed cap, not to one network's need, so that a
// later network of the same width never lowers it below an earlier one's.
constexpr int kLayerPwSmemCap = 200 * 1024;
template <int C>
bool layer_pw_attr(size_t smem) {
  return smem <= 48 * 1024 ||
         (cudaFuncSetAttribute(k_layer_pw<C, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kLayerPwSmemCap) ==
              cudaSuccess &&
          cudaFuncSetAttribute(k_layer_pw<C, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kLayerPwSmemCap) ==
              cudaSuccess);
}

// whether the register-blocked layer kernel serves this width and mode count
// (raises its shared-memory limit where needed; called at creation, outside
// any graph capture)
bool layer_pw_prepare(int C, int K2) {
  const size_t smem = layer_pw_smem(C, K2);
  if (smem > (size_t)kLayerPwSmemCap) return false;
  bool ok = false;
  switch (C) {
    case 8: ok = layer_pw_attr<8>(smem); break;
    case 16: ok = layer_pw_attr<16>(smem); break;
    case 32: ok = layer_pw_attr<32>(smem); break;
    default: return false;
  }
  if (!ok) (void)cudaGetLastError();   // (a refused limit is not an error of the context)
  return ok;
}

template <int CI, int CO, bool SPEC, int ACT>
void launch_pw(cudaStream_t s, int S, int H, int W, int K2, const float* A, const float* bias, const float* in,
               const float* Zb, const float* G, float* out, float* act) {
  const size_t smem = ((size_t)(CI + (SPEC ? K2 : 0)) * pw_pitch(CO) + (SPEC ? (size_t)K2 * kPwNT : 0)) * sizeof(float);
  const dim3 grid((W + kPwNT - 1) / kPwNT, H, S);
  k_pointwise<CI, CO, SPEC, ACT><<<grid, kPwNT, smem, s>>>(H, W, K2, A, bias, in, Zb, G, out, act);
}

// The pointwise passes: the layer output (CI = CO = C, spectral part, act 1
// GELU / 2 copy), the lift (CI = 3) and the projection (CO = 3).
enum PwKind { kPwLayer, kPwLift, kPwProject };
// (the register-blocked layer kernel exists for C a multiple of 8; its
// template argument is clamped so that the untaken branch still compiles
// for C = 4)
template <int C>
void pw_c(PwKind kind, bool layer_pw, cudaStream_t s, int S, int H, int W, int K2, const float* A, const float* bias,
          const float* in, const float* Zb, const float* G, float* out, float* act, int act_kind) {
  if (kind == kPwLift) launch_pw<3, C, false, 0>(s, S, H, W, 0, A, bias, in, nullptr, nullptr, out, nullptr);
  else if (kind == kPwProject) launch_pw<C, 3, false, 0>(s, S, H, W, 0, A, bias, in, nullptr, nullptr, out, nullptr);
  else if (layer_pw && C % 8 == 0 && act_kind == 1)
    launch_layer_pw<(C % 8 == 0 ? C : 8), 1>(s, S, H, W, K2, A, bias, in, Zb, G, out, act);
  else if (layer_pw && C % 8 == 0)
    launch_layer_pw<(C % 8 == 0 ? C : 8), 2>(s, S, H, W, K2, A, bias, in, Zb, G, out, act);
  else if (act_kind == 1) launch_pw<C, C, true, 1>(s, S, H, W, K2, A, bias, in, Zb, G, out, act);
  else launch_pw<C, C, true, 2>(s, S, H, W, K2, A, bias, in, Zb, G, out, act);
}
// Launches one pointwise pass for C in {4, 8, 16, 32}; false where there is
// no instantiation or the staged tables exceed 48 KB (the caller then takes
// the GEMM path).  layer_pw: layer_pw_prepare(C, K2) succeeded (the
// register-blocked layer kernel serves the layer output).
bool pointwise(PwKind kind, bool layer_pw, cudaStream_t s, int S, int C, int H, int W, int K2, const float* A,
               const float* bias, const float* in, const float* Zb, const float* G, float* out, float* act,
               int act_kind) {
  if (H > 65535 || S > 65535) return false;
  if (C != 4 && C != 8 && C != 16 && C != 32) return false;
  const int ci = kind == kPwLift ? 3 : C, co = kind == kPwProject ? 3 : C;
  if (!(kind == kPwLayer && layer_pw) &&
      ((long long)(ci + (kind == kPwLayer ? K2 : 0)) * pw_pitch(co) + (kind == kPwLayer ? (long long)K2 * kPwNT : 0)) *
              4 > 49152)
    return false;
  switch (C) {
    case 4: pw_c<4>(kind, layer_pw, s, S, H, W, K2, A, bias, in, Zb, G, out, act, act_kind); break;
    case 8: pw_c<8>(kind, layer_pw, s, S, H, W, K2, A, bias, in, Zb, G, out, act, act_kind); break;
    case 16: pw_c<16>(kind, layer_pw, s, S, H, W, K2, A, bias, in, Zb, G, out, act, act_kind); break;
    default: pw_c<32>(kind, layer_pw, s, S, H, W, K2, A, bias, in, Zb, G, out, act, act_kind); break;
  }
  return true;
}

// O[s][o][m] = sum_i R[o][i][m] V[s][i][m]   (conj: sum_o conj(R[o][i][m]) V[s][o][m] -> O[s][i][m])
// Four lanes per output (kMixLanes consecutive threads), each summing
// i = part, part + 4, ..., then a fixed two-step shuffle sum.  Launch with
// kMixLanes * S * C * NM threads in blocks of a multiple of 32.
constexpr int kMixLanes = 4;
__global__ void k_mix(int S, int C, int NM, const float2* __restrict__ R, const float2* __restrict__ V,
                      float2* __restrict__ O, bool adjoint) {
  const long long total = (long long)S * C * NM;
  const long long gt = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long idx = gt / kMixLanes;
  const int part = (int)(gt % kMixLanes);
  const bool on = idx < total;   // (every lane stays for the shuffles)
  float re = 0.f, im = 0.f;
  if (on) {
    const int m = (int)(idx % NM), o = (int)((idx / NM) % C);
    const long long s = idx / ((long long)NM * C);
#pragma unroll 4
    for (int i = part; i < C; i += kMixLanes) {
      float2 r = adjoint ? R[((long long)i * C + o) * NM + m] : R[((long long)o * C + i) * NM + m];
      if (adjoint) r.y = -r.y;
      const float2 v = V[(s * C + i) * NM + m];
      re = fmaf(r.x, v.x, fmaf(-r.y, v.y, re));
      im = fmaf(r.x, v.y, fmaf(r.y, v.x, im));
    }
  }
  re += __shfl_xor_sync(0xffffffffu, re, 1);
  im += __shfl_xor_sync(0xffffffffu, im, 1);
  re += __shfl_xor_sync(0xffffffffu, re, 2);
  im += __shfl_xor_sync(0xffffffffu, im, 2);
  if (on && part == 0) O[idx] = make_float2(re, im);
}
unsigned mix_blocks(long long outputs) { return (unsigned)((outputs * kMixLanes + 255) / 256); }

// dR[o][i][m] += sum_s dO[s][o][m] conj(V[s][i][m])
__global__ void k_dR(int S, int C, int NM, const float2* __restrict__ dO, const float2* __restrict__ V,
                     float2* __restrict__ dR) {
  const long long total = (long long)C * C * NM;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  const int m = (int)(idx % NM), i = (int)((idx / NM) % C), o = (int)(idx / ((long long)NM * C));
  float re = 0.f, im = 0.f;
  for (int s = 0; s < S; ++s) {
    const float2 d = dO[((long long)s * C + o) * NM + m];
    const float2 v = V[((long long)s * C + i) * NM + m];
    re += d.x * v.x + d.y * v.y;
    im += d.y * v.x - d.x * v.y;
  }
  dR[idx].x += re;
  dR[idx].y += im;
}

__global__ void k_gelu_back(long long n, const float* __restrict__ z, float* __restrict__ dv) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dv[i] *= gelu_df(z[i]);
}

// sum over pixels per (row) for bias gradients: out[r] += sum_{s,p} d[s][r][p]
__global__ void k_rowsum(int S, int R, long long P, const float* __restrict__ d, float* __restrict__ out) {
  const int r = blockIdx.x;
  float acc = 0.f;
  for (int s = 0; s < S; ++s)
    for (long long p = threadIdx.x; p < P; p += blockDim.x) acc += d[((long long)s * R + r) * P + p];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  __shared__ float red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float v = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[w];
    out[r] += v;
  }
}

// loss pieces: acc[0] += sum (yhat - y)^2, acc[1] += sum y^2
__global__ void k_loss(long long n, const float* __restrict__ yh, const float* __restrict__ y, double* acc) {
  double a = 0.0, b = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double d = (double)yh[i] - (double)y[i];
    a += d * d;
    b += (double)y[i] * y[i];
  }
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&acc[0], a);
    atomicAdd(&acc[1], b);
  }
}

__global__ void k_dloss(long long n, const float* __restrict__ yh, const float* __restrict__ y,
                        const double* __restrict__ acc, float* __restrict__ dy) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dy[i] = (float)(2.0 * ((double)yh[i] - (double)y[i]) / acc[1]);
}

__global__ void k_adam(long long n, float* __restrict__ p, const float* __restrict__ gr, float* __restrict__ m1,
                       float* __restrict__ m2, float lr, float b1, float b2, float eps, float c1, float c2) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float g = gr[i];
  const float a = b1 * m1[i] + (1.f - b1) * g;
  const float b = b2 * m2[i] + (1.f - b2) * g * g;
  m1[i] = a;
  m2[i] = b;
  p[i] -= lr * (a / c1) / (sqrtf(b / c2) + eps);
}

// u = (Msat(cell) / ms_ref) m  and  B = mu0 ms_ref y
__global__ void k_to_u(long long n, const float* __restrict__ m, const uint8_t* __restrict__ mask,
                       const uint8_t* __restrict__ region, const RegionLUT* __restrict__ lut, float inv_ref,
                       float* __restrict__ u) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float s = mask[i] ? lut->msat[region[i]] * inv_ref : 0.f;
  u[i] = s * m[i];
  u[n + i] = s * m[n + i];
  u[2 * n + i] = s * m[2 * n + i];
}

__global__ void k_scale(long long n, const float* __restrict__ x, float s, float* __restrict__ y) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = s * x[i];
}

__global__ void k_rel_err(long long n, const float* __restrict__ a, const float* __restrict__ b, double* acc) {
  double x = 0.0, y = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double d = (double)a[i] - (double)b[i];
    x += d * d;
    y += (double)b[i] * b[i];
  }
  for (int o = 16; o > 0; o >>= 1) {
    x += __shfl_xor_sync(0xffffffffu, x, o);
    y += __shfl_xor_sync(0xffffffffu, y, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&acc[0], x);
    atomicAdd(&acc[1], y);
  }
}

unsigned nb(long long n, int t = 256) { return (unsigned)((n + t - 1) / t); }

}  // namespace
}  // namespace mm

using namespace mm;

struct mm_fno {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int C = 0, L = 0, Mx = 0, My = 0, H = 0, W = 0, J = 0, Smax = 0;
  int sms = 1;                  // multiprocessors of the device
  bool layer_pw = false;        // the register-blocked layer kernel serves (C, 2 Mx)
  long long N = 0, nparam = 0;
  long long xslice = 0;         // floats between the split-K slices of X and Z
  std::vector<long long> off;   // P, p, {W, b, R} per layer, Q, q
  float *prm = nullptr, *grd = nullptr, *m1 = nullptr, *m2 = nullptr;
  long long adam_t = 0;
  // constant partial-DFT matrices
  float *Fblk = nullptr, *Gblk = nullptr;   // [W][2Mx], [2Mx][W]
  float2 *Fy = nullptr, *Gy = nullptr;      // [J][H]
  // activations and caches for Smax samples
  float *u = nullptr, *yh = nullptr, *dy = nullptr;
  std::vector<float*> v, z;                 // L+1 and L
  std::vector<float2*> V;                   // L
  float *X = nullptr, *Z = nullptr, *dv = nullptr, *dv2 = nullptr, *dz = nullptr;
  float2 *O = nullptr, *dO = nullptr, *dV = nullptr;
  float2* Yp = nullptr;                     // row-range partials of the y product
  double* acc = nullptr;
};

namespace {

int ffail(int code, const std::string& msg) {
  mm::set_last_error(msg);
  return code;
}

#define MMF_CUDA(call)                                                                        \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess)                                                                    \
      return ffail(e_ == cudaErrorMemoryAllocation ? MM_ERR_OOM : MM_ERR_CUDA,                \
                   std::string(#call) + ": " + cudaGetErrorString(e_));                       \
  } while (0)

float* P_(mm_fno* f, int k) { return f->prm + f->off[k]; }
float* G_(mm_fno* f, int k) { return f->grd + f->off[k]; }
// parameter slots: 0 P, 1 p, 2 + 3l W_l, 3 + 3l b_l, 4 + 3l R_l, 2 + 3L Q, 3 + 3L q
int sW(int l) { return 2 + 3 * l; }
int sb(int l) { return 3 + 3 * l; }
int sR(int l) { return 4 + 3 * l; }

// Slices of the x partial DFT products (M = C H rows, N = 2 Mx, K = W): split
// K until there are about four blocks per multiprocessor; the tiled y
// product sums the slices.
int xparts(const mm_fno* f, int S, const YTile& t) {
  if (!t.ysum) return 1;
  const long long blocks = (long long)((2 * f->Mx + BN - 1) / BN) * ((f->C * f->H + BM - 1) / BM) * S;
  long long p = (4LL * f->sms + blocks - 1) / blocks;
  p = std::min<long long>(p, kXParts);
  p = std::min<long long>(p, (f->W + BK - 1) / BK);
  return (int)std::max<long long>(1, p);
}

// forward for S samples whose inputs are already in f->u; output in f->yh
void fwd(mm_fno* f, int S) {
  cudaStream_t s = f->stream;
  const int C = f->C, H = f->H, W = f->W, Mx = f->Mx, J = f->J;
  const long long N = f->N, CN = (long long)C * N;
  const int L = f->L;
  const int q = sW(L) , qq = sb(L);
  const YTile yt = ytile(S, C, H, J, Mx, f->sms);
  const int xp = xparts(f, S, yt);
  // lift: v0[C x N] = P[C x 3] u[3 x N] + p
  if (!pointwise(kPwLift, f->layer_pw, s, S, C, H, W, 0, P_(f, 0), P_(f, 1), f->u, nullptr, nullptr, f->v[0], nullptr, 0))
    gemm(s, false, false, S, gargs(C, (int)N, 3, P_(f, 0), 3, 0, f->u, N, 3 * N, f->v[0], N, CN, 1.f, 0.f, P_(f, 1)));
  for (int l = 0; l < L; ++l) {
    float* vin = f->v[l];
    // X = v [C H x W] . Fblk [W x 2Mx]
    gemm(s, false, false, S, sliced(gargs(C * H, 2 * Mx, W, vin, W, CN, f->Fblk, 2 * Mx, 0, f->X, 2 * Mx,
                                          (long long)C * H * 2 * Mx), xp, f->xslice));
    ysum(s, yt, S, C, H, J, Mx, f->X, true, xp, f->xslice, f->Fy, false, f->V[l], f->Yp);
    k_mix<<<mix_blocks((long long)S * C * J * Mx), 256, 0, s>>>(S, C, J * Mx, reinterpret_cast<const float2*>(P_(f, sR(l))),
                                                      f->V[l], f->O, false);
    yexpand(s, yt, S, C, H, J, Mx, f->O, f->Gy, false, f->Z);
    // z = Z_blk [C H x 2Mx] . Gblk [2Mx x W] (spectral part) + W v + b, and
    // v_{l+1} = GELU(z) (z after the last layer)
    if (!pointwise(kPwLayer, f->layer_pw, s, S, C, H, W, 2 * Mx, P_(f, sW(l)), P_(f, sb(l)), vin, f->Z, f->Gblk, f->z[l],
                   f->v[l + 1], l < L - 1 ? 1 : 2)) {
      gemm(s, false, false, S, gargs(C * H, W, 2 * Mx, f->Z, 2 * Mx, (long long)C * H * 2 * Mx, f->Gblk, W, 0,
                                     f->z[l], W, CN));
      gemm(s, false, false, S, with_act(gargs(C, (int)N, C, P_(f, sW(l)), C, 0, vin, N, CN, f->z[l], N, CN, 1.f, 1.f,
                                              P_(f, sb(l))), f->v[l + 1], l < L - 1));
    }
  }
  // project: y[3 x N] = Q[3 x C] v_L + q
  if (!pointwise(kPwProject, f->layer_pw, s, S, C, H, W, 0, P_(f, q), P_(f, qq), f->v[L], nullptr, nullptr, f->yh, nullptr, 0))
    gemm(s, false, false, S, gargs(3, (int)N, C, P_(f, q), C, 0, f->v[L], N, CN, f->yh, N, 3 * N, 1.f, 0.f, P_(f, qq)));
}

// gradients of the batch loss into f->grd (zeroed here); loss pieces in acc
void bwd(mm_fno* f, int S, const float* y) {
  cudaStream_t s = f->stream;
  const int C = f->C, H = f->H, W = f->W, Mx = f->Mx, J = f->J, L = f->L;
  const long long N = f->N, CN = (long long)C * N;
  const int splits = (int)std::min<long long>(64, std::max<long long>(1, N / 4096));
  const YTile yt = ytile(S, C, H, J, Mx, f->sms);
  const int xp = xparts(f, S, yt);
  cudaMemsetAsync(f->grd, 0, f->nparam * sizeof(float), s);
  cudaMemsetAsync(f->acc, 0, 2 * sizeof(double), s);
  k_loss<<<1024, 256, 0, s>>>(S * 3 * N, f->yh, y, f->acc);
  k_dloss<<<nb(S * 3 * N), 256, 0, s>>>(S * 3 * N, f->yh, y, f->acc, f->dy);
  // project
  for (int b = 0; b < S; ++b)
    gemm(s, false, true, 1, gargs(3, C, (int)N, f->dy + b * 3 * N, N, 0, f->v[L] + b * CN, N, 0, G_(f, sW(L)), C, 0,
                                  1.f, 0.f, nullptr, splits, 1));
  k_rowsum<<<3, 256, 0, s>>>(S, 3, N, f->dy, G_(f, sb(L)));
  gemm(s, true, false, S, gargs(C, (int)N, 3, P_(f, sW(L)), C, 0, f->dy, N, 3 * N, f->dv, N, CN));
  for (int l = L - 1; l >= 0; --l) {
    if (l < L - 1) k_gelu_back<<<nb(S * CN), 256, 0, s>>>(S * CN, f->z[l], f->dv);
    float* dzl = f->dv;   // dz
    for (int b = 0; b < S; ++b)
      gemm(s, false, true, 1, gargs(C, C, (int)N, dzl + b * CN, N, 0, f->v[l] + b * CN, N, 0, G_(f, sW(l)), C, 0, 1.f,
                                    0.f, nullptr, splits, 1));
    k_rowsum<<<C, 256, 0, s>>>(S, C, N, dzl, G_(f, sb(l)));
    // dv2 = W^T dz
    gemm(s, true, false, S, gargs(C, (int)N, C, P_(f, sW(l)), C, 0, dzl, N, CN, f->dv2, N, CN));
    // spectral adjoint: dZ_blk = dz [C H x W] . Gblk^T
    gemm(s, false, true, S, sliced(gargs(C * H, 2 * Mx, W, dzl, W, CN, f->Gblk, W, 0, f->Z, 2 * Mx,
                                         (long long)C * H * 2 * Mx), xp, f->xslice));
    ysum(s, yt, S, C, H, J, Mx, f->Z, true, xp, f->xslice, f->Gy, true, f->dO, f->Yp);
    k_dR<<<nb((long long)C * C * J * Mx), 256, 0, s>>>(S, C, J * Mx, f->dO, f->V[l],
                                                      reinterpret_cast<float2*>(G_(f, sR(l))));
    k_mix<<<mix_blocks((long long)S * C * J * Mx), 256, 0, s>>>(S, C, J * Mx, reinterpret_cast<const float2*>(P_(f, sR(l))),
                                                      f->dO, f->dV, true);
    yexpand(s, yt, S, C, H, J, Mx, f->dV, f->Fy, true, f->X);
    // dv2 += dX_blk [C H x 2Mx] . Fblk^T [2Mx x W]
    gemm(s, false, true, S, gargs(C * H, W, 2 * Mx, f->X, 2 * Mx, (long long)C * H * 2 * Mx, f->Fblk, 2 * Mx, 0, f->dv2,
                                  W, CN, 1.f, 1.f));
    std::swap(f->dv, f->dv2);
  }
  // lift
  for (int b = 0; b < S; ++b)
    gemm(s, false, true, 1, gargs(C, 3, (int)N, f->dv + b * CN, N, 0, f->u + b * 3 * N, N, 0, G_(f, 0), 3, 0, 1.f, 0.f,
                                  nullptr, splits, 1));
  k_rowsum<<<C, 256, 0, s>>>(S, C, N, f->dv, G_(f, 1));
}

}  // namespace

extern "C" {

int mm_fno_create(mm_fno** out, int H, int W, const mm_fno_cfg* cfg, int device, void* stream) {
  if (!out || !cfg) return ffail(MM_ERR_ARG, "NULL argument");
  *out = nullptr;
  const int C = cfg->width, L = cfg->layers, Mx = cfg->modes_x, My = cfg->modes_y, Smax = cfg->max_batch;
  if (H < 2 || W < 2 || C < 1 || L < 1 || Mx < 1 || My < 1 || Smax < 1 || Mx > W / 2 || 2 * My > H)
    return ffail(MM_ERR_ARG, "need H, W >= 2, width, layers, batch >= 1, modes_x <= W/2, 2 modes_y <= H");
  MMF_CUDA(cudaSetDevice(device));
  int sms = 1;
  MMF_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
  mm_fno* f = new mm_fno();
  f->device = device;
  f->sms = sms;
  f->layer_pw = layer_pw_prepare(C, 2 * Mx);
  f->C = C; f->L = L; f->Mx = Mx; f->My = My; f->H = H; f->W = W; f->J = 2 * My; f->Smax = Smax;
  f->N = (long long)H * W;
  auto cleanup = [&](int code) { mm_fno_destroy(f); return code; };
  // parameter layout
  long long o = 0;
  auto add = [&](long long n) { f->off.push_back(o); o += n; };
  add((long long)C * 3);
  add(C);
  for (int l = 0; l < L; ++l) {
    add((long long)C * C);
    add(C);
    add(2LL * C * C * f->J * Mx);
  }
  add(3LL * C);
  add(3);
  f->nparam = o;
  cudaError_t e = cudaSuccess;
  if (stream) f->stream = (cudaStream_t)stream;
  else { e = cudaStreamCreateWithFlags(&f->stream, cudaStreamNonBlocking); f->own_stream = e == cudaSuccess; }
  auto alloc = [&](void** p, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) e = cudaMemsetAsync(*p, 0, bytes, f->stream);
  };
  alloc((void**)&f->prm, o * sizeof(float));
  alloc((void**)&f->grd, o * sizeof(float));
  alloc((void**)&f->m1, o * sizeof(float));
  alloc((void**)&f->m2, o * sizeof(float));
  alloc((void**)&f->Fblk, (size_t)W * 2 * Mx * sizeof(float));
  alloc((void**)&f->Gblk, (size_t)2 * Mx * W * sizeof(float));
  alloc((void**)&f->Fy, (size_t)f->J * H * sizeof(float2));
  alloc((void**)&f->Gy, (size_t)f->J * H * sizeof(float2));
  const long long CN = (long long)C * f->N;
  alloc((void**)&f->u, (size_t)Smax * 3 * f->N * sizeof(float));
  alloc((void**)&f->yh, (size_t)Smax * 3 * f->N * sizeof(float));
  alloc((void**)&f->dy, (size_t)Smax * 3 * f->N * sizeof(float));
  f->v.assign(L + 1, nullptr);
  f->z.assign(L, nullptr);
  f->V.assign(L, nullptr);
  for (int l = 0; l <= L; ++l) alloc((void**)&f->v[l], (size_t)Smax * CN * sizeof(float));
  for (int l = 0; l < L; ++l) alloc((void**)&f->z[l], (size_t)Smax * CN * sizeof(float));
  for (int l = 0; l < L; ++l) alloc((void**)&f->V[l], (size_t)Smax * C * f->J * Mx * sizeof(float2));
  f->xslice = (long long)Smax * C * H * 2 * Mx;
  alloc((void**)&f->X, (size_t)kXParts * f->xslice * sizeof(float));
  alloc((void**)&f->Z, (size_t)kXParts * f->xslice * sizeof(float));
  alloc((void**)&f->dv, (size_t)Smax * CN * sizeof(float));
  alloc((void**)&f->dv2, (size_t)Smax * CN * sizeof(float));
  alloc((void**)&f->O, (size_t)Smax * C * f->J * Mx * sizeof(float2));
  alloc((void**)&f->dO, (size_t)Smax * C * f->J * Mx * sizeof(float2));
  alloc((void**)&f->dV, (size_t)Smax * C * f->J * Mx * sizeof(float2));
  alloc((void**)&f->Yp, (size_t)kYSplit * Smax * C * f->J * Mx * sizeof(float2));
  alloc((void**)&f->acc, 4 * sizeof(double));
  if (e != cudaSuccess) return cleanup(ffail(e == cudaErrorMemoryAllocation ? MM_ERR_OOM : MM_ERR_CUDA, cudaGetErrorString(e)));
  // partial DFT matrices (float64 on the host, rounded once)
  const double pi = 3.14159265358979323846;
  std::vector<float> Fb((size_t)W * 2 * Mx), Gb((size_t)2 * Mx * W);
  for (int x = 0; x < W; ++x)
    for (int k = 0; k < Mx; ++k) {
      const double a = 2.0 * pi * (double)((long long)k * x % W) / W;
      Fb[(size_t)x * 2 * Mx + k] = (float)std::cos(a);
      Fb[(size_t)x * 2 * Mx + Mx + k] = (float)-std::sin(a);
      const double c = (k == 0 ? 1.0 : 2.0) / W;
      Gb[(size_t)k * W + x] = (float)(c * std::cos(a));           // Re(Z Gx) = Zr Gr - Zi Gi
      Gb[(size_t)(Mx + k) * W + x] = (float)(-c * std::sin(a));
    }
  std::vector<float2> fy((size_t)f->J * H), gy((size_t)f->J * H);
  for (int j = 0; j < f->J; ++j) {
    const int ky = j < My ? j : H - 2 * My + j;
    for (int y = 0; y < H; ++y) {
      const double a = 2.0 * pi * (double)((long long)ky * y % H) / H;
      fy[(size_t)j * H + y] = make_float2((float)std::cos(a), (float)-std::sin(a));
      gy[(size_t)j * H + y] = make_float2((float)(std::cos(a) / H), (float)(std::sin(a) / H));
    }
  }
  e = cudaMemcpyAsync(f->Fblk, Fb.data(), Fb.size() * sizeof(float), cudaMemcpyHostToDevice, f->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(f->Gblk, Gb.data(), Gb.size() * sizeof(float), cudaMemcpyHostToDevice, f->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(f->Fy, fy.data(), fy.size() * sizeof(float2), cudaMemcpyHostToDevice, f->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(f->Gy, gy.data(), gy.size() * sizeof(float2), cudaMemcpyHostToDevice, f->stream);
  // initial parameters: scaled normal draws from a seeded generator
  std::vector<float> p0(o, 0.0f);
  unsigned long long st = cfg->seed * 0x9E3779B97F4A7C15ULL + 1;
  auto unif = [&]() {   // splitmix64 -> (0, 1)
    st += 0x9E3779B97F4A7C15ULL;
    unsigned long long z = st;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    z ^= z >> 31;
    return ((z >> 11) + 0.5) * (1.0 / 9007199254740992.0);
  };
  auto normal = [&]() { return std::sqrt(-2.0 * std::log(unif())) * std::cos(2.0 * pi * unif()); };
  auto fill = [&](int slot, long long n, double scale) {
    for (long long i = 0; i < n; ++i) p0[f->off[slot] + i] = (float)(scale * normal());
  };
  fill(0, 3LL * C, 1.0 / std::sqrt(3.0));
  for (int l = 0; l < L; ++l) {
    fill(sW(l), (long long)C * C, 1.0 / std::sqrt((double)C));
    fill(sR(l), 2LL * C * C * f->J * Mx, 1.0 / C);
  }
  fill(sW(L), 3LL * C, 1.0 / std::sqrt((double)C));
  if (e == cudaSuccess) e = cudaMemcpyAsync(f->prm, p0.data(), o * sizeof(float), cudaMemcpyHostToDevice, f->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(f->stream);
  if (e != cudaSuccess) return cleanup(ffail(MM_ERR_CUDA, cudaGetErrorString(e)));
  *out = f;
  return MM_OK;
}

int mm_fno_destroy(mm_fno* f) {
  if (!f) return MM_OK;
  cudaSetDevice(f->device);
  if (f->stream) cudaStreamSynchronize(f->stream);
  void* ptrs[] = {f->prm, f->grd, f->m1, f->m2, f->Fblk, f->Gblk, f->Fy, f->Gy, f->u, f->yh, f->dy,
                  f->X, f->Z, f->dv, f->dv2, f->O, f->dO, f->dV, f->Yp, f->acc};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  for (float* p : f->v) if (p) cudaFree(p);
  for (float* p : f->z) if (p) cudaFree(p);
  for (float2* p : f->V) if (p) cudaFree(p);
  if (f->own_stream && f->stream) cudaStreamDestroy(f->stream);
  delete f;
  return MM_OK;
}

long long mm_fno_param_count(mm_fno* f) { return f ? f->nparam : 0; }

int mm_fno_get_params(mm_fno* f, float* host, long long n) {
  if (!f || !host || n != f->nparam) return ffail(MM_ERR_ARG, "bad arguments");
  MMF_CUDA(cudaMemcpyAsync(host, f->prm, n * sizeof(float), cudaMemcpyDeviceToHost, f->stream));
  MMF_CUDA(cudaStreamSynchronize(f->stream));
  return MM_OK;
}

int mm_fno_set_params(mm_fno* f, const float* host, long long n) {
  if (!f || !host || n != f->nparam) return ffail(MM_ERR_ARG, "bad arguments");
  MMF_CUDA(cudaMemcpyAsync(f->prm, host, n * sizeof(float), cudaMemcpyHostToDevice, f->stream));
  MMF_CUDA(cudaMemsetAsync(f->m1, 0, n * sizeof(float), f->stream));
  MMF_CUDA(cudaMemsetAsync(f->m2, 0, n * sizeof(float), f->stream));
  MMF_CUDA(cudaStreamSynchronize(f->stream));
  f->adam_t = 0;
  return MM_OK;
}

int mm_fno_forward(mm_fno* f, const float* u, float* y, int S) {
  if (!f || !u || !y || S < 1 || S > f->Smax) return ffail(MM_ERR_ARG, "bad arguments");
  MMF_CUDA(cudaMemcpyAsync(f->u, u, (size_t)S * 3 * f->N * sizeof(float), cudaMemcpyDeviceToDevice, f->stream));
  fwd(f, S);
  MMF_CUDA(cudaMemcpyAsync(y, f->yh, (size_t)S * 3 * f->N * sizeof(float), cudaMemcpyDeviceToDevice, f->stream));
  MMF_CUDA(cudaGetLastError());
  MMF_CUDA(cudaStreamSynchronize(f->stream));
  return MM_OK;
}

int mm_fno_grad(mm_fno* f, const float* u, const float* y, int S, float* grad_host, double* loss) {
  if (!f || !u || !y || S < 1 || S > f->Smax) return ffail(MM_ERR_ARG, "bad arguments");
  MMF_CUDA(cudaMemcpyAsync(f->u, u, (size_t)S * 3 * f->N * sizeof(float), cudaMemcpyDeviceToDevice, f->stream));
  fwd(f, S);
  bwd(f, S, y);
  MMF_CUDA(cudaGetLastError());
  double acc[2];
  MMF_CUDA(cudaMemcpyAsync(acc, f->acc, sizeof(acc), cudaMemcpyDeviceToHost, f->stream));
  if (grad_host) MMF_CUDA(cudaMemcpyAsync(grad_host, f->grd, f->nparam * sizeof(float), cudaMemcpyDeviceToHost, f->stream));
  MMF_CUDA(cudaStreamSynchronize(f->stream));
  if (loss) *loss = acc[0] / acc[1];
  return MM_OK;
}

int mm_fno_train_step(mm_fno* f, const float* u, const float* y, int S, double lr, double* loss) {
  int rc = mm_fno_grad(f, u, y, S, nullptr, loss);
  if (rc) return rc;
  f->adam_t++;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - std::pow(b1, (float)f->adam_t), c2 = 1.f - std::pow(b2, (float)f->adam_t);
  k_adam<<<nb(f->nparam), 256, 0, f->stream>>>(f->nparam, f->prm, f->grd, f->m1, f->m2, (float)lr, b1, b2, 1e-8f, c1, c2);
  MMF_CUDA(cudaGetLastError());
  MMF_CUDA(cudaStreamSynchronize(f->stream));
  return MM_OK;
}

}  // extern "C"

namespace mm {
// surrogate demag field for a context: u from m, FNO forward, B = mu0 ms_ref y
void launch_fno_demag(mm_fno* f, const Geom& g, const Buffers& b, const float* m, float inv_ref, float mu0_ref,
                      float* bd, cudaStream_t s) {
  cudaStream_t keep = f->stream;
  f->stream = s;
  k_to_u<<<nb(g.n), 256, 0, s>>>(g.n, m, b.mask, b.region, b.lut, inv_ref, f->u);
  fwd(f, 1);
  k_scale<<<nb(3 * g.n), 256, 0, s>>>(3 * g.n, f->yh, mu0_ref, bd);
  f->stream = keep;
}
void launch_rel_err(long long n, const float* a, const float* b, double* acc, cudaStream_t s) {
  cudaMemsetAsync(acc, 0, 2 * sizeof(double), s);
  k_rel_err<<<512, 256, 0, s>>>(n, a, b, acc);
}
bool fno_matches(mm_fno* f, const Geom& g) { return f && f->H == g.ny && f->W == g.nx && g.nz == 1; }
void launch_to_u(const Geom& g, const Buffers& b, const float* m, float inv_ref, float* u, cudaStream_t s) {
  k_to_u<<<nb(g.n), 256, 0, s>>>(g.n, m, b.mask, b.region, b.lut, inv_ref, u);
}
void launch_scale(long long n, const float* x, float a, float* y, cudaStream_t s) {
  k_scale<<<nb(n), 256, 0, s>>>(n, x, a, y);
}
}  // namespace mm
