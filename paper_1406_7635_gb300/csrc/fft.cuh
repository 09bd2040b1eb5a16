// Complex FFT building blocks for the demag convolution (Sec. III.B: the
// convolution is FFT-accelerated by the convolution theorem).
//
// Power-of-two lengths only.  A length-L transform is a sequence of Stockham
// radix passes (radices 16, 8, 4, 2 -- see radix_of) over pencils held in
// shared memory; each pass reads every element into registers, synchronises,
// then writes the butterflies' outputs in place, so no second buffer is needed.
// Twiddles come from one table W[k] = exp(-2 pi i k / 2048) (k < 2048), built
// on the host in float64 and rounded once to float32.
#pragma once
#include <cuda_runtime.h>

#include <type_traits>

namespace mmfft {

constexpr int kTwN = 2048;   // twiddle table length: largest supported L

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// multiply by DIR * i  (DIR = -1 forward, +1 inverse)
template <int DIR>
__device__ __forceinline__ float2 mul_dir_i(float2 a) {
  return DIR < 0 ? make_float2(a.y, -a.x) : make_float2(-a.y, a.x);
}

// exp(DIR * 2 pi i k / 16) for k = 0..7, as constants
__device__ __forceinline__ float2 w16(int k, int dir) {
  const float c1 = 0.92387953251128674f, s1 = 0.38268343236508978f, h = 0.70710678118654752f;
  float c, s;
  switch (k) {
    case 0: c = 1.f; s = 0.f; break;
    case 1: c = c1; s = s1; break;
    case 2: c = h; s = h; break;
    case 3: c = s1; s = c1; break;
    case 4: c = 0.f; s = 1.f; break;
    case 5: c = -s1; s = c1; break;
    case 6: c = -h; s = h; break;
    default: c = -c1; s = s1; break;
  }
  return make_float2(c, dir < 0 ? -s : s);
}

// o * exp(DIR 2 pi i k / 16) with the trivial factors done without multiplies
template <int K, int DIR>
__device__ __forceinline__ float2 rot16(float2 o) {
  constexpr float h = 0.70710678118654752f;
  if (K == 0) return o;
  if (K == 4) return mul_dir_i<DIR>(o);
  if (K == 2) {   // (1 + DIR i) h
    const float2 t = mul_dir_i<DIR>(o);
    return make_float2((o.x + t.x) * h, (o.y + t.y) * h);
  }
  if (K == 6) {   // (-1 + DIR i) h
    const float2 t = mul_dir_i<DIR>(o);
    return make_float2((t.x - o.x) * h, (t.y - o.y) * h);
  }
  return cmul(o, w16(K, DIR));
}

// In-register DFT of length R (R = 1, 2, 4, 8, 16), natural order in and out,
// by recursive even/odd splitting.
template <int R, int DIR>
struct Dft {
  __device__ __forceinline__ static void run(float2 (&x)[R]) {
    float2 e[R / 2], o[R / 2];
#pragma unroll
    for (int i = 0; i < R / 2; ++i) { e[i] = x[2 * i]; o[i] = x[2 * i + 1]; }
    Dft<R / 2, DIR>::run(e);
    Dft<R / 2, DIR>::run(o);
    combine<0>(x, e, o);
  }
  template <int K>
  __device__ __forceinline__ static void combine(float2 (&x)[R], const float2 (&e)[R / 2], const float2 (&o)[R / 2]) {
    if constexpr (K < R / 2) {
      const float2 t = rot16<K * (16 / R), DIR>(o[K]);
      x[K] = cadd(e[K], t);
      x[K + R / 2] = csub(e[K], t);
      combine<K + 1>(x, e, o);
    }
  }
};
template <int DIR>
struct Dft<1, DIR> {
  __device__ __forceinline__ static void run(float2 (&)[1]) {}
};
template <int DIR>
struct Dft<2, DIR> {
  __device__ __forceinline__ static void run(float2 (&x)[2]) {
    const float2 a = x[0];
    x[0] = cadd(a, x[1]);
    x[1] = csub(a, x[1]);
  }
};
template <int DIR>
struct Dft<4, DIR> {
  __device__ __forceinline__ static void run(float2 (&x)[4]) {
    const float2 a0 = cadd(x[0], x[2]), a1 = csub(x[0], x[2]);
    const float2 a2 = cadd(x[1], x[3]), a3 = mul_dir_i<DIR>(csub(x[1], x[3]));
    x[0] = cadd(a0, a2);
    x[2] = csub(a0, a2);
    x[1] = cadd(a1, a3);
    x[3] = csub(a1, a3);
  }
};

// Radix of pass `p` for length L (a power of two): as few passes as radix 16
// allows, with the factors balanced so no pass is a thin radix-2/4 tail
// (32 = 8 x 4, 64 = 8 x 8, 128 = 16 x 8, 512 = 8 x 8 x 8, 2048 = 16 x 16 x 8).
__host__ __device__ constexpr int radix_of(int L, int p) {
  int lg = 0;
  while ((1 << lg) < L) ++lg;
  const int passes = (lg + 3) / 4;   // ceil(lg / 4) passes of at most radix 16
  if (passes == 0) return 1;
  const int base = lg / passes, extra = lg % passes;   // first `extra` passes get one more bit
  return 1 << (base + (p < extra ? 1 : 0));
}
__host__ __device__ constexpr int npasses(int L) {
  int ns = 1, n = 0;
  while (ns < L) { ns *= radix_of(L, n); ++n; }
  return n;
}
__host__ __device__ constexpr int ns_of(int L, int p) {
  int ns = 1;
  for (int i = 0; i < p; ++i) ns *= radix_of(L, i);
  return ns;
}

// One Stockham pass of radix R on NP pencils of length L in shared memory.
// Element i of pencil q sits at s[(q / INNER) * BS + (q % INNER) + i * ES]:
// rows (INNER = 1, BS = pitch, ES = 1) or columns of a row-major plane
// (INNER = row length, BS = plane size, ES = pitch).  NT threads cooperate;
// butterfly b belongs to pencil b % NP, so consecutive threads touch
// consecutive pencils (with an odd row pitch this avoids bank conflicts).
// tw holds W_TWL^i = exp(-2 pi i i / TWL) for i < TWL (TWL a multiple of L):
// the global 2048-entry table, or a per-length copy in shared memory.
// pre (first pass only, may be null): input element i is multiplied by pre[i]
// as it is loaded.
// WARP: the pencils belong to one warp (NT = 32, lanes share the butterflies,
// __syncwarp() orders reads before writes) instead of the whole block.
// IS: stride between the pencils of one group (default 1), so that
// base = (q / INNER) * BS + (q % INNER) * IS.
// nin (first pass only): input elements i >= nin are zero and not read
// (a pruned transform of a zero-padded row); nout (last pass only): output
// elements i >= nout are not needed and not written (a cropped transform).
template <int L, int R, int NS, int DIR, int NP, int NT, int INNER, int BS, int ES, int TWL, bool WARP = false,
          int IS = 1>
__device__ __forceinline__ void stockham_pass(float2* s, const float2* __restrict__ tw,
                                              const float2* __restrict__ pre = nullptr, int nin = L, int nout = L) {
  constexpr int NB = L / R;
  constexpr int TOT = NB * NP;
  constexpr int PER = (TOT + NT - 1) / NT;
  const int tid = WARP ? (int)(threadIdx.x & 31) : (int)threadIdx.x;
  float2 v[PER][R];
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int b = tid + q * NT;
    if (TOT % NT == 0 || b < TOT) {
      const int p = b % NP, j = b / NP;
      const int base = (p / INNER) * BS + (p % INNER) * IS;
#pragma unroll
      for (int r = 0; r < R; ++r)
        v[q][r] = (NS > 1 || j + r * NB < nin) ? s[base + (j + r * NB) * ES] : make_float2(0.f, 0.f);
      if (NS == 1 && pre != nullptr) {
#pragma unroll
        for (int r = 0; r < R; ++r) v[q][r] = cmul(v[q][r], pre[j + r * NB]);
      }
    }
  }
  if (WARP) __syncwarp();
  else __syncthreads();
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int b = tid + q * NT;
    if (TOT % NT == 0 || b < TOT) {
      const int p = b % NP, j = b / NP;
      const int base = (p / INNER) * BS + (p % INNER) * IS;
      const int k = j % NS;
      if (NS > 1) {
#pragma unroll
        for (int r = 1; r < R; ++r) {
          // exp(DIR 2 pi i r k / (NS R)) = W[r k (TWL / (NS R))] (conjugated if DIR > 0)
          float2 w = tw[(r * k * (TWL / (NS * R))) & (TWL - 1)];
          if (DIR > 0) w.y = -w.y;
          v[q][r] = cmul(v[q][r], w);
        }
      }
      Dft<R, DIR>::run(v[q]);
      const int o = (j - k) * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r)
        if (NS * R < L || o + r * NS < nout) s[base + (o + r * NS) * ES] = v[q][r];
    }
  }
  if (WARP) __syncwarp();
  else __syncthreads();
}

// Full length-L complex transform of NP shared-memory pencils (in place,
// natural order), addressed as in stockham_pass.  Callers synchronise before
// (data written); the last pass ends with __syncthreads().
template <int L, int DIR, int NP, int NT, int INNER, int BS, int ES, int TWL = kTwN, int IS = 1, int P = 0,
          bool DONE = (P >= npasses(L))>
struct FftG;
// (nin: the first pass reads only input elements i < nin, the rest are zero;
// nout: the last pass writes only output elements i < nout)
template <int L, int DIR, int NP, int NT, int INNER, int BS, int ES, int TWL, int IS, int P>
struct FftG<L, DIR, NP, NT, INNER, BS, ES, TWL, IS, P, false> {
  __device__ __forceinline__ static void run(float2* s, const float2* __restrict__ tw,
                                             const float2* __restrict__ pre = nullptr, int nin = L, int nout = L) {
    stockham_pass<L, radix_of(L, P), ns_of(L, P), DIR, NP, NT, INNER, BS, ES, TWL, false, IS>(
        s, tw, P == 0 ? pre : nullptr, P == 0 ? nin : L, P + 1 == npasses(L) ? nout : L);
    FftG<L, DIR, NP, NT, INNER, BS, ES, TWL, IS, P + 1>::run(s, tw, nullptr, L, nout);
  }
};
template <int L, int DIR, int NP, int NT, int INNER, int BS, int ES, int TWL, int IS, int P>
struct FftG<L, DIR, NP, NT, INNER, BS, ES, TWL, IS, P, true> {
  __device__ __forceinline__ static void run(float2*, const float2* __restrict__, const float2* __restrict__ = nullptr,
                                             int = L, int = L) {}
};

// In-register DFT of length N, natural order in and out: Dft for N <= 16;
// N = 32 as two 16-point halves (even / odd samples) combined with W_32^k,
// read from tw32[k] = exp(-2 pi i k / 32) (conjugated for DIR > 0).
template <int N, int DIR>
struct RegDft {
  __device__ __forceinline__ static void run(float2 (&x)[N], const float2* __restrict__) { Dft<N, DIR>::run(x); }
};
template <int DIR>
struct RegDft<32, DIR> {
  __device__ __forceinline__ static void run(float2 (&x)[32], const float2* __restrict__ tw32) {
    float2 e[16], o[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      e[i] = x[2 * i];
      o[i] = x[2 * i + 1];
    }
    Dft<16, DIR>::run(e);
    Dft<16, DIR>::run(o);
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      float2 w = tw32[k];
      if (DIR > 0) w.y = -w.y;
      const float2 t = cmul(o[k], w);
      x[k] = cadd(e[k], t);
      x[k + 16] = csub(e[k], t);
    }
  }
};

// pencils stored as rows with pitch PST, twiddles from the global table
template <int L, int DIR, int NP, int NT, int PST>
using Fft = FftG<L, DIR, NP, NT, 1, PST, 1>;

// A shared-memory pencil layout: element i of pencil p at
// (p / INNER) * BS + (p % INNER) + i * ES.
template <int INNER_, int BS_, int ES_>
struct Lay {
  static constexpr int INNER = INNER_, BS = BS_, ES = ES_;
  __device__ __forceinline__ static int at(int p, int i) { return (p / INNER) * BS + (p % INNER) + i * ES; }
};

// A Stockham pass as stockham_pass, reading its inputs in layout LI and
// writing its outputs in layout LO over the same buffer (every read of the
// pass completes before the barrier, every write comes after it).
template <int L, int R, int NS, int DIR, int NP, int NT, class LI, class LO, int TWL>
__device__ __forceinline__ void stockham_pass_x(float2* s, const float2* __restrict__ tw, int nin = L, int nout = L) {
  constexpr int NB = L / R;
  constexpr int TOT = NB * NP;
  constexpr int PER = (TOT + NT - 1) / NT;
  float2 v[PER][R];
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int b = threadIdx.x + q * NT;
    if (TOT % NT == 0 || b < TOT) {
      const int p = b % NP, j = b / NP;
#pragma unroll
      for (int r = 0; r < R; ++r)
        v[q][r] = (NS > 1 || j + r * NB < nin) ? s[LI::at(p, j + r * NB)] : make_float2(0.f, 0.f);
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int b = threadIdx.x + q * NT;
    if (TOT % NT == 0 || b < TOT) {
      const int p = b % NP, j = b / NP;
      const int k = j % NS;
      if (NS > 1) {
#pragma unroll
        for (int r = 1; r < R; ++r) {
          float2 w = tw[(r * k * (TWL / (NS * R))) & (TWL - 1)];
          if (DIR > 0) w.y = -w.y;
          v[q][r] = cmul(v[q][r], w);
        }
      }
      Dft<R, DIR>::run(v[q]);
      const int o = (j - k) * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r)
        if (NS * R < L || o + r * NS < nout) s[LO::at(p, o + r * NS)] = v[q][r];
    }
  }
  __syncthreads();
}

// Full length-L transform of NP pencils whose first pass reads layout LI,
// whose last pass writes layout LO and whose other passes use layout LM.
// nin: the first pass reads only input elements i < nin (the rest are zero);
// nout: the last pass writes only output elements i < nout.
// Callers synchronise before; ends with __syncthreads().
template <int L, int DIR, int NP, int NT, class LI, class LM, class LO, int TWL, int P = 0,
          bool DONE = (P >= npasses(L))>
struct FftX;
template <int L, int DIR, int NP, int NT, class LI, class LM, class LO, int TWL, int P>
struct FftX<L, DIR, NP, NT, LI, LM, LO, TWL, P, false> {
  __device__ __forceinline__ static void run(float2* s, const float2* __restrict__ tw, int nin = L, int nout = L) {
    using In = typename std::conditional<P == 0, LI, LM>::type;
    using Out = typename std::conditional<P + 1 == npasses(L), LO, LM>::type;
    stockham_pass_x<L, radix_of(L, P), ns_of(L, P), DIR, NP, NT, In, Out, TWL>(s, tw, P == 0 ? nin : L,
                                                                                P + 1 == npasses(L) ? nout : L);
    FftX<L, DIR, NP, NT, LI, LM, LO, TWL, P + 1>::run(s, tw, L, nout);
  }
};
template <int L, int DIR, int NP, int NT, class LI, class LM, class LO, int TWL, int P>
struct FftX<L, DIR, NP, NT, LI, LM, LO, TWL, P, true> {
  __device__ __forceinline__ static void run(float2*, const float2* __restrict__, int = L, int = L) {}
};

// copy W_L^i (i < L) out of the global 2048-entry table into shared memory
template <int L, int NT>
__device__ __forceinline__ void load_twiddles(float2* dst, const float2* __restrict__ tw) {
  for (int i = threadIdx.x; i < L; i += NT) dst[i] = __ldg(&tw[i * (kTwN / L)]);
}

// 8-byte asynchronous global -> shared copy (completes with the caller's
// next cp.async.commit_group / wait)
__device__ __forceinline__ void cp_async_f2(float2* dst, const float2* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}

// W_TWN^(i * stride mod TWN) for i < n, as asynchronous copies: the per-length
// table (stride kTwN / L) or a residue-class twiddle (stride kTwN / P)
template <int NT>
__device__ __forceinline__ void twiddles_async(float2* dst, const float2* __restrict__ tw, int n, int stride) {
  for (int i = threadIdx.x; i < n; i += NT) cp_async_f2(dst + i, tw + ((i * stride) & (kTwN - 1)));
}

}  // namespace mmfft
