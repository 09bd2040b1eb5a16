// Fused RK45 stage kernels for the fused convolution layout (spec as
// [c][kx][z][y]): per attempt, one prep kernel and, per stage, the y/z
// transform kernel (k_yz2 / k_yz) plus one row kernel, instead of five
// kernels per stage.  Where the shape allows, the row kernel moves its
// spectrum box and stencil rows with tensor copies (TMA).  On 3-D grids with
// the z-split (y, z) part and on 2-D grids with the one-kernel (y, z) path it
// is launched as a programmatic dependent of its predecessor: its stencil
// copies, table loads and (where they are summed in the kernel) earlier-stage
// sums run before the wait.
//
// A block owns ROWS complete x-rows (one z plane) of all three components.
//   k_rs_prep  stage input m_s = m + dt sum_j a_sj k_j for its cells, written
//              for the neighbours' stencils, then M = Msat m_s -> x R2C into
//              the spectrum rows it owns;
//   k_rs_row   x C2R of the demag spectrum of stage s (B_demag stays in
//              shared memory) -> effective field and LL torque k_s of its
//              cells -> next stage input m_{s+1} and its x R2C, or, after the
//              last stage, the error estimate, the candidate m and (last
//              block) the step controller (Sec. IV);
//   k_rs_partial  the part of that stage input (or error estimate) without
//              k_s, an elementwise sum over m and the earlier k's that runs
//              beside the (y, z) part of stage s, so that the row kernel
//              reads one array instead of up to six.
// Stage inputs alternate between two buffers (ms for even stages, ms2 for odd
// ones), because a stage's stencil reads neighbours owned by other blocks.
#include <algorithm>
#include <cstring>

#include "fft.cuh"
#include "llg_device.cuh"

namespace mm {
namespace {
using namespace mmfft;

enum { ROW_K1 = 0, ROW_NEXT = 1, ROW_LAST = 2 };

__device__ __forceinline__ float* stage_buf(const Buffers& b, int s) { return (s & 1) ? b.ms2 : b.ms; }

// 32-bit indices: the fused layout has nz <= 32 and at most 2^28 cells
__device__ __forceinline__ int tix(const Geom& g, int c, int kx, int z, int y) {
  return ((c * g.hx + kx) * g.nz + z) * g.ny + y;
}

// x R2C of the packed rows in s (3 * ROWS pencils) into the spectrum; the
// complex inputs n >= (nx + 1) / 2 are the zero padding and are not read
template <int L, int ROWS, int NT>
__device__ __forceinline__ void rows_fx(const Geom& g, float2* s, const float2* twl, const float2* tw2, float2* spec,
                                        int y0, int z) {
  constexpr int PST = L + 1;
  FftG<L, -1, 3 * ROWS, NT, 1, PST, 1, L>::run(s, twl, nullptr, (g.nx + 1) / 2);
  for (int e = threadIdx.x; e < 3 * ROWS * (L + 1); e += NT) {
    const int r = e % ROWS, k = (e / ROWS) % (L + 1), c = e / (ROWS * (L + 1));
    const int y = y0 + r;
    if (y >= g.ny) continue;
    const float2* row = s + (c * ROWS + r) * PST;
    const float2 zk = row[k & (L - 1)];
    const float2 zc = cconj(row[(L - k) & (L - 1)]);
    const float2 E = cscale(cadd(zk, zc), 0.5f);
    const float2 d = csub(zk, zc);
    const float2 O = make_float2(0.5f * d.y, -0.5f * d.x);
    spec[tix(g, c, k, z, y)] = cadd(E, cmul(tw2[k], O));
  }
}

// ---------------------------------------------------------------------------
// TMA (cp.async.bulk.tensor) path: the spectrum box of a block is one tensor
// copy each way, the stencil rows twelve; completion through mbarriers that a
// single thread waits on with a time limit.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// Waits for phase 0 of bar to complete; false once `limit` SM cycles have
// passed (the context's wait limit, by default 2^30 cycles: half a second),
// so that a lost transfer ends the kernel with an error instead of a hang.
// The limit is checked before each poll: with limit 0 the wait gives up
// without polling.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, long long limit) {
  const long long t0 = clock64();
  for (;;) {
    if (clock64() - t0 >= limit) return false;
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(bar))
        : "memory");
    if (done) return true;
  }
}
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
      "[%6];\n" ::"r"(smem_u32(dst)),
      "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int c0, int c1, int c2,
                                            unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];\n" ::
          "r"(smem_u32(dst)),
      "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tma_store_4d(const CUtensorMap* map, int c0, int c1, int c2, int c3, const void* src) {
  asm volatile("cp.async.bulk.tensor.4d.global.shared::cta.bulk_group [%0, {%1, %2, %3, %4}], [%5];\n" ::"l"(map),
               "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(src))
               : "memory");
  asm volatile("cp.async.bulk.commit_group;\n" ::: "memory");
}
// the block's own bulk stores have finished reading shared memory (the
// global writes complete with the grid, before the next kernel in the stream)
__device__ __forceinline__ void tma_store_drain() { asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory"); }
// generic-proxy shared-memory writes become visible to the tensor copies
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

// Pencil layouts of the block's spectrum rows: the tensor box [c][k][r]
// (A: element k of pencil (c, r) at (c (L + 1) + k) ROWS + r) and rows of
// pitch L + 1 (B, the layout the field code reads and the stage input is
// written in).
template <int L, int ROWS>
using LayA = Lay<ROWS, (L + 1) * ROWS, ROWS>;
template <int L>
using LayB = Lay<1, L + 1, 1>;

// x R2C of the packed rows in s (layout B) into the spectrum by one tensor
// store: the first pass moves the rows into the box layout A, the post-pass
// X_k = E_k + W_2L^k O_k runs on the pairs (k, L - k) in place (X_L beside),
// rows past the grid are clipped by the store.
template <int L, int ROWS, int NT>
__device__ __forceinline__ void rows_fx_tma(const Geom& g, float2* s, const float2* twl, const float2* tw2,
                                            const CUtensorMap* map, int y0, int z) {
  using A = LayA<L, ROWS>;
  FftX<L, -1, 3 * ROWS, NT, LayB<L>, A, A, L>::run(s, twl, (g.nx + 1) / 2);
  for (int e = threadIdx.x; e < 3 * ROWS * (L / 2 + 1); e += NT) {
    const int pen = e % (3 * ROWS), k = e / (3 * ROWS);
    const int ia = A::at(pen, k), ib = A::at(pen, (L - k) & (L - 1));
    const float2 zk = s[ia], zl = s[ib];
    {
      const float2 zc = cconj(zl);
      const float2 E = cscale(cadd(zk, zc), 0.5f);
      const float2 d = csub(zk, zc);
      s[ia] = cadd(E, cmul(tw2[k], make_float2(0.5f * d.y, -0.5f * d.x)));
    }
    {
      const float2 zc = cconj(zk);
      const float2 E = cscale(cadd(zl, zc), 0.5f);
      const float2 d = csub(zl, zc);
      const float2 X = cadd(E, cmul(tw2[L - k], make_float2(0.5f * d.y, -0.5f * d.x)));
      if (k == 0) s[A::at(pen, L)] = X;
      else if (k != L / 2) s[ib] = X;
    }
  }
  fence_async_smem();
  __syncthreads();
  if (threadIdx.x == 0) {
    tma_store_4d(map, y0, z, 0, 0, s);
    tma_store_drain();
  }
}

// the x-transform tables W_L^i (i < L) and W_2L^k (k <= L), as asynchronous
// copies (awaited with the caller's next cp.async wait)
template <int L, int NT>
__device__ __forceinline__ void load_tables(float2* twl, float2* tw2, const float2* __restrict__ tw) {
  twiddles_async<NT>(twl, tw, L, kTwN / L);
  twiddles_async<NT>(tw2, tw, L + 1, kTwN / (2 * L));
}

template <int L, int ROWS, int NT, bool SS>
__global__ void __launch_bounds__(NT) k_rs_prep(Geom g, Buffers b, Ptrs p, const DevState* __restrict__ st,
                                               const StageCoef* __restrict__ sc, int s,
                                               const __grid_constant__ RsMaps maps) {
  if (st->done) return;
  constexpr int PST = L + 1;
  __shared__ __align__(128) float2 sm[3 * ROWS * PST];
  __shared__ float2 twl[L], tw2[L + 1];
  const int y0 = blockIdx.x * ROWS, z = blockIdx.y;
  load_tables<L, NT>(twl, tw2, b.tw);
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  float* sf = reinterpret_cast<float*>(sm);
  const int par = st->parity;
  const float* __restrict__ m = par ? p.m1 : p.m0;
  float* __restrict__ out = stage_buf(b, s);
  // (x >= nx rounded up to even is zero padding, never read by the transform)
  const int xw = (g.nx + 1) & ~1;
  for (int e = threadIdx.x; e < ROWS * xw; e += NT) {
    const int x = e % xw, r = e / xw, y = y0 + r;
    float v[3] = {0.f, 0.f, 0.f};
    if (y < g.ny && x < g.nx) {
      const int n = (int)g.n, i = (z * g.ny + y) * g.nx + x;
      float a0 = m[i], a1 = m[n + i], a2 = m[2 * n + i];
      for (int j = 0; j < s; ++j) {
        const float a = sc->ah[s][j];
        if (a == 0.0f) continue;
        const float* __restrict__ k = pick_k(p, k_role(j, par));
        a0 = fmaf(a, k[i], a0);
        a1 = fmaf(a, k[n + i], a1);
        a2 = fmaf(a, k[2 * n + i], a2);
      }
      out[i] = a0;
      out[n + i] = a1;
      out[2 * n + i] = a2;
      const int ci = b.code[i];
      const float ms = ci != kVacuum ? __ldg(&b.lut->msat[ci]) : 0.f;
      v[0] = ms * a0;
      v[1] = ms * a1;
      v[2] = ms * a2;
    }
    for (int c = 0; c < 3; ++c) sf[2 * (c * ROWS + r) * PST + x] = v[c];
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  __syncthreads();
  if constexpr (SS) rows_fx_tma<L, ROWS, NT>(g, sm, twl, tw2, &maps.spec, y0, z);
  else rows_fx<L, ROWS, NT>(g, sm, twl, tw2, b.spec, y0, z);
}

// Shared-memory layout of the row kernel (dynamic, base rounded up to 128
// bytes): the demag rows of the block (3 ROWS pencils of L + 1 complex,
// padded to 128 bytes), then the stencil rows of the stage input [3][NR][L]
// and their cell codes [NR][L].
// Local stencil rows: 0 .. ROWS+1 are y0-1 .. y0+ROWS of plane z, then ROWS
// rows y0 .. of plane z-1, then ROWS rows of plane z+1.
template <int L, int ROWS>
struct RsSmem {
  static constexpr int PST = L + 1;
  static constexpr int NR = 3 * ROWS + 2;
  static constexpr int SPEC = ((3 * ROWS * PST * 8) + 127) / 128 * 128;
  static constexpr int STEN = 3 * NR * L * 4;
  static constexpr int CODE = NR * L * 4;
  // (+128: the base is rounded up to 128 bytes, the alignment of tensor copies)
  static constexpr int BYTES = SPEC + STEN + CODE + 128;
};

// Which copies go through the tensor engine where the shape allows it: the
// row kernel's spectrum box load (SL) and store (SS), its stencil rows (TT),
// and the prep kernel's spectrum store (PS).  Measured on the 128 x 128 x 32
// step (same GPU, ms per step): all four 0.5516, PS off 0.5472, SS and PS off
// 0.5485, TT off 0.5643; the prep kernel's blocks are short and waiting for
// their store to drain costs more than the scattered stores.  Re-measured
// with the current (y, z) kernels and the earlier-stage sums branch: PS on
// makes the prep kernel 15.5 -> 14.6 us and leaves the step where it is
// (0.433-0.435 ms either way), so it stays off.
constexpr bool kRsSL = true;
constexpr bool kRsSS = true;
constexpr bool kRsTT = true;
constexpr bool kRsPS = false;

// Spectrum boxes: rows of 32..128 complex values with at least 8 rows per
// block (box dimension L + 1 <= 256, conflict-free box layout A).
template <int L, int ROWS>
constexpr bool rs_spec_shape() {
  return L >= 32 && L <= 128 && ROWS >= 8;
}
// Stencil rows: 32..256 floats (row starts 128-byte aligned, box <= 256).
template <int L>
constexpr bool rs_sten_shape() {
  return L >= 32 && L <= 256;
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}

// asynchronous copies of the block's stencil rows (stage input and codes);
// rows outside the grid are not copied and never read
template <int L, int ROWS, int NT>
__device__ __forceinline__ void stage_stencil(const Geom& g, const float* __restrict__ ms, const int* __restrict__ code,
                                              float* sten, int* scode, int y0, int z) {
  constexpr int NR = RsSmem<L, ROWS>::NR;
  const bool vec = (g.nx & 3) == 0;      // rows start on 16-byte boundaries
  const int n = (int)g.n;
  if (vec) {
    constexpr int CPR = L / 4;             // 16-byte chunks per (padded) row
    for (int e = threadIdx.x; e < NR * 4 * CPR; e += NT) {
      const int ch = e % CPR, t = e / CPR, a = t & 3, lr = t >> 2;
      int yy = y0 + lr - 1, zz = z;
      if (lr >= ROWS + 2) {
        const int q = lr - (ROWS + 2);
        yy = y0 + (q % ROWS);
        zz = q < ROWS ? z - 1 : z + 1;
      } else if (g.pbcy) {
        yy = (yy + g.ny) % g.ny;          // halo rows wrap around a periodic y
      }
      if (g.pbcz) zz = (zz + g.nz) % g.nz;
      if (4 * ch >= g.nx || yy < 0 || yy >= g.ny || zz < 0 || zz >= g.nz) continue;
      const int row = (zz * g.ny + yy) * g.nx + 4 * ch;
      const void* src = a < 3 ? (const void*)(ms + a * n + row) : (const void*)(code + row);
      void* dst = a < 3 ? (void*)(sten + (a * NR + lr) * L + 4 * ch) : (void*)(scode + lr * L + 4 * ch);
      cp_async16(dst, src);
    }
  } else {
    for (int e = threadIdx.x; e < NR * 4 * L; e += NT) {
      const int ch = e % L, t = e / L, a = t & 3, lr = t >> 2;
      int yy = y0 + lr - 1, zz = z;
      if (lr >= ROWS + 2) {
        const int q = lr - (ROWS + 2);
        yy = y0 + (q % ROWS);
        zz = q < ROWS ? z - 1 : z + 1;
      } else if (g.pbcy) {
        yy = (yy + g.ny) % g.ny;
      }
      if (g.pbcz) zz = (zz + g.nz) % g.nz;
      if (ch >= g.nx || yy < 0 || yy >= g.ny || zz < 0 || zz >= g.nz) continue;
      const int row = (zz * g.ny + yy) * g.nx + ch;
      const void* src = a < 3 ? (const void*)(ms + a * n + row) : (const void*)(code + row);
      void* dst = a < 3 ? (void*)(sten + (a * NR + lr) * L + ch) : (void*)(scode + lr * L + ch);
      cp_async4(dst, src);
    }
  }
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}

// SL / SS: the spectrum box loaded / stored by tensor copies, TT: the stencil
// rows by tensor copies; otherwise asynchronous copies and plain stores
template <int L, int ROWS, int NT, bool SL, bool SS, bool TT>
__global__ void __launch_bounds__(NT, 2) k_rs_row(Geom g, Buffers b, Terms T, Ptrs p, DevState* __restrict__ st,
                                                 StageCoef* __restrict__ sc, int s, int mode, double freq,
                                                 double phase_over_pi, const __grid_constant__ RsMaps maps) {
  // The done flag is read once per block: the controller runs after every
  // block of this launch, but a block that gave up a wait on its copies sets
  // the flag while others may be starting, and the block must agree.
  __shared__ int blk_done;
  if (threadIdx.x == 0) blk_done = st->done;
  __syncthreads();
  if (blk_done) return;
  using SM = RsSmem<L, ROWS>;
  constexpr int PST = SM::PST, NR = SM::NR;
  // real cells per thread: ROWS rows of at most L cells (nx <= 2L, and the
  // x-padding cells are not visited)
  constexpr int CPT = (ROWS * L + NT - 1) / NT;
  constexpr int NCELL = ROWS * L;   // cell slots: x < L of each row (x >= nx idle)
  extern __shared__ float4 rs_dyn[];
  char* const base = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(rs_dyn) + 127) & ~uintptr_t(127));
  float2* sm = reinterpret_cast<float2*>(base);
  float* sten = reinterpret_cast<float*>(base + SM::SPEC);
  int* scode = reinterpret_cast<int*>(base + SM::SPEC + SM::STEN);
  __shared__ float2 twl[L], tw2[L + 1];
  __shared__ float wmax[32];
  __shared__ __align__(8) unsigned long long bars[2];   // TMA: spectrum, stencil
  __shared__ int tma_ok;
  const int y0 = blockIdx.x * ROWS, z = blockIdx.y;
  const float* __restrict__ ms = stage_buf(b, s);
  // 0. copies in flight: the demag spectrum rows and the twiddle tables, then
  //    the stencil rows of the stage input (awaited only after the x
  //    transform).  Tensor copies are issued by thread 0: the spectrum box
  //    (layout A) and twelve boxes of stencil rows.
  if constexpr (SL || TT) {
    if (threadIdx.x == 0) {
      mbar_init(&bars[0]);
      mbar_init(&bars[1]);
      mbar_init_fence();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      if constexpr (TT) {
        mbar_expect_tx(&bars[1], 16 * NR * L);
        const CUtensorMap* own = (s & 1) ? &maps.ms2_own : &maps.ms_own;
        const CUtensorMap* pl = (s & 1) ? &maps.ms2_pl : &maps.ms_pl;
        // neighbour planes: wrapped on a periodic z, else out of range (zero
        // filled, never read)
        const int zm = g.pbcz ? (z + g.nz - 1) % g.nz : z - 1, zp = g.pbcz ? (z + 1) % g.nz : z + 1;
        for (int c = 0; c < 3; ++c) {
          tma_load_4d(sten + (c * NR) * L, own, 0, y0 - 1, z, c, &bars[1]);
          tma_load_4d(sten + (c * NR + ROWS + 2) * L, pl, 0, y0, zm, c, &bars[1]);
          tma_load_4d(sten + (c * NR + 2 * ROWS + 2) * L, pl, 0, y0, zp, c, &bars[1]);
        }
        tma_load_3d(scode, &maps.code_own, 0, y0 - 1, z, &bars[1]);
        tma_load_3d(scode + (ROWS + 2) * L, &maps.code_pl, 0, y0, zm, &bars[1]);
        tma_load_3d(scode + (2 * ROWS + 2) * L, &maps.code_pl, 0, y0, zp, &bars[1]);
      }
    }
  }
  load_tables<L, NT>(twl, tw2, b.tw);
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  if constexpr (!TT) stage_stencil<L, ROWS, NT>(g, ms, b.code, sten, scode, y0, z);
  const int par = st->parity;
  const int n = (int)g.n;
  // 1. the earlier-stage sums at the block's cells: next stage
  //    m + dt sum_{j<s} a_{s+1,j} k_j, or the error dt sum_{j<6} e_j k_j.
  //    With b.part they come from k_rs_partial (a graph branch beside the
  //    (y, z) part; loaded below, after the dependency wait, while the
  //    spectrum copy is in flight); otherwise they are summed here from
  //    global memory while the asynchronous copies are in flight, the stage
  //    loop unrolled (a zero coefficient skips its loads) so that all loads
  //    of a cell are issued before the first is used.  Same operation order
  //    on both paths.
  float av[CPT][3];
#pragma unroll
  for (int q = 0; q < CPT; ++q) av[q][0] = av[q][1] = av[q][2] = 0.f;
  if (!b.part && mode != ROW_K1) {
    float cj[6];
#pragma unroll
    for (int j = 0; j < 6; ++j) cj[j] = mode == ROW_NEXT ? (j < s ? sc->ah[s + 1][j] : 0.f) : sc->eh[j];
    const float* __restrict__ m = par ? p.m1 : p.m0;
#pragma unroll
    for (int q = 0; q < CPT; ++q) {
      const int e = threadIdx.x + q * NT;
      if (e >= NCELL) continue;
      const int x = e % L, r = e / L, y = y0 + r;
      if (x >= g.nx || y >= g.ny) continue;
      const int i = (z * g.ny + y) * g.nx + x;
      float kj[6][3];
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        kj[j][0] = kj[j][1] = kj[j][2] = 0.f;
        if (cj[j] != 0.0f) {
          const float* __restrict__ k = pick_k(p, k_role(j, par));
          kj[j][0] = k[i];
          kj[j][1] = k[n + i];
          kj[j][2] = k[2 * n + i];
        }
      }
      float a0 = 0.f, a1 = 0.f, a2 = 0.f;
      if (mode == ROW_NEXT) {
        a0 = m[i];
        a1 = m[n + i];
        a2 = m[2 * n + i];
      }
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        if (cj[j] != 0.0f) {
          a0 = fmaf(cj[j], kj[j][0], a0);
          a1 = fmaf(cj[j], kj[j][1], a1);
          a2 = fmaf(cj[j], kj[j][2], a2);
        }
      }
      av[q][0] = a0;
      av[q][1] = a1;
      av[q][2] = a2;
    }
  }
  // the spectrum is the previous kernel's output (programmatic dependent
  // launch: everything above overlaps its last blocks)
  grid_dependency_wait();
  if constexpr (SL) {
    if (threadIdx.x == 0) {
      mbar_expect_tx(&bars[0], 3 * (L + 1) * ROWS * 8);
      tma_load_4d(sm, &maps.spec, y0, z, 0, 0, &bars[0]);
    }
  } else {
    for (int e = threadIdx.x; e < 3 * ROWS * (L + 1); e += NT) {
      const int r = e % ROWS, k = (e / ROWS) % (L + 1), c = e / (ROWS * (L + 1));
      const int y = y0 + r;
      float2* dst = sm + (c * ROWS + r) * PST + k;
      if (y < g.ny) cp_async8(dst, b.spec + tix(g, c, k, z, y));
      else *dst = make_float2(0.f, 0.f);
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  }
  // (1. continued: the precomputed sums, used after the field)
  if (b.part && mode != ROW_K1) {
#pragma unroll
    for (int q = 0; q < CPT; ++q) {
      const int e = threadIdx.x + q * NT;
      if (e >= NCELL) continue;
      const int x = e % L, r = e / L, y = y0 + r;
      if (x >= g.nx || y >= g.ny) continue;
      const int i = (z * g.ny + y) * g.nx + x;
      av[q][0] = b.part[i];
      av[q][1] = b.part[n + i];
      av[q][2] = b.part[2 * n + i];
    }
  }
  // 2. x C2R of the demag spectrum rows (3 components); the output is in
  //    rows of pitch L + 1 (layout B) on both paths
  using A = LayA<L, ROWS>;
  using Bl = LayB<L>;
  using LIn = typename std::conditional<SL, A, Bl>::type;
  // (groups: tables, then the stencil rows unless TT, then the spectrum
  // unless SL; only the stencil group may stay in flight)
  if constexpr (TT || !SL) asm volatile("cp.async.wait_all;\n" ::: "memory");
  else asm volatile("cp.async.wait_group 1;\n" ::: "memory");
  // (a wait that gives up records MM_ERR_TIMEOUT and ends the attempt; the
  // copies still in flight are then awaited with the default limit, so that
  // they land before the block's shared memory is released)
  if constexpr (SL) {
    if (threadIdx.x == 0) tma_ok = mbar_wait(&bars[0], st->wait_cycles);
    __syncthreads();
    if (!tma_ok) {   // uniform; the copies in flight land before the block ends
      if (threadIdx.x == 0) {
        st->status = -6;   // MM_ERR_TIMEOUT
        st->done = 1;
        mbar_wait(&bars[0], kWaitCycles);
        if (TT) mbar_wait(&bars[1], kWaitCycles);
      }
      return;
    }
  } else {
    __syncthreads();
  }
  for (int e = threadIdx.x; e < 3 * ROWS * (L / 2 + 1); e += NT) {
    // (consecutive threads on consecutive pencils in layout A)
    const int pen = SL ? e % (3 * ROWS) : e / (L / 2 + 1), k = SL ? e / (3 * ROWS) : e % (L / 2 + 1);
    const int ia = LIn::at(pen, k), ib = LIn::at(pen, L - k);
    const float2 xa = sm[ia], xb = sm[ib];
    float2 za, zb;
    {
      const float2 E = cscale(cadd(xa, cconj(xb)), 0.5f);
      const float2 O = cmul(cscale(csub(xa, cconj(xb)), 0.5f), cconj(tw2[k]));
      za = make_float2(E.x - O.y, E.y + O.x);
    }
    {
      const float2 E = cscale(cadd(xb, cconj(xa)), 0.5f);
      const float2 O = cmul(cscale(csub(xb, cconj(xa)), 0.5f), cconj(tw2[L - k]));
      zb = make_float2(E.x - O.y, E.y + O.x);
    }
    sm[ia] = za;
    if (k != 0 && k != L / 2) sm[ib] = zb;
  }
  __syncthreads();
  // (outputs 2n >= nx are cropped: the field code reads x < nx)
  FftX<L, 1, 3 * ROWS, NT, LIn, LIn, Bl, L>::run(sm, twl, L, (g.nx + 1) / 2);
  if constexpr (TT) {
    if (threadIdx.x == 0) tma_ok = mbar_wait(&bars[1], st->wait_cycles);
    __syncthreads();
    if (!tma_ok) {
      if (threadIdx.x == 0) {
        st->status = -6;   // MM_ERR_TIMEOUT
        st->done = 1;
        mbar_wait(&bars[1], kWaitCycles);
      }
      return;
    }
  } else {
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    __syncthreads();
  }
  // 3. field and torque of the block's cells, stencil from shared memory
  const float* sf = reinterpret_cast<const float*>(sm);
  const RegionLUT* __restrict__ lut = b.lut;
  float* __restrict__ kout = pick_k(p, k_role(s, par));
  const float sinft = T.zeeman ? excitation(freq, phase_over_pi, st->stage_t[s]) : 0.0f;
  float kv[CPT][3], mv[CPT][3];
  int cv[CPT];
#pragma unroll
  for (int q = 0; q < CPT; ++q) {
    const int e = threadIdx.x + q * NT;
    kv[q][0] = kv[q][1] = kv[q][2] = 0.f;
    mv[q][0] = mv[q][1] = mv[q][2] = 0.f;
    cv[q] = kVacuum;
    if (e >= NCELL) continue;
    const int x = e % L, r = e / L, y = y0 + r;
    if (x >= g.nx || y >= g.ny) continue;
    const int C = (r + 1) * L + x;
    const int ci = scode[C];
    cv[q] = ci;
    const float3 mi = f3(sten[C], sten[NR * L + C], sten[2 * NR * L + C]);
    mv[q][0] = mi.x;
    mv[q][1] = mi.y;
    mv[q][2] = mi.z;
    if (ci == kVacuum) continue;
    FieldParts P;
    P.demag = T.demag ? f3(sf[2 * (0 * ROWS + r) * PST + x], sf[2 * (1 * ROWS + r) * PST + x],
                           sf[2 * (2 * ROWS + r) * PST + x])
                      : f3(0, 0, 0);
    float3 ex = f3(0, 0, 0);
    P.dmi = f3(0, 0, 0);
    if (T.exch || T.dmi) {
      // same neighbour order and arithmetic as field_at
      const float* __restrict__ xl = b.xlut + ci * kXStride;
      // periodic axes wrap: the staged halo rows/planes hold the wrapped data
      const int nb[6] = {x > 0 ? C - 1 : (g.pbcx ? C + g.nx - 1 : C),
                         x < g.nx - 1 ? C + 1 : (g.pbcx ? C - (g.nx - 1) : C),
                         (y > 0 || g.pbcy) ? C - L : C,
                         (y < g.ny - 1 || g.pbcy) ? C + L : C,
                         (z > 0 || g.pbcz) ? (ROWS + 2 + r) * L + x : C,
                         (z < g.nz - 1 || g.pbcz) ? (2 * ROWS + 2 + r) * L + x : C};
      const bool per[6] = {g.pbcx > 0, g.pbcx > 0, g.pbcy > 0, g.pbcy > 0, g.pbcz > 0, g.pbcz > 0};
      const float id2[6] = {g.idx2, g.idx2, g.idy2, g.idy2, g.idz2, g.idz2};
      if (!T.dmi) {
#pragma unroll
        for (int d = 0; d < 6; ++d) {
          const int j = nb[d];
          const float c = __ldg(&xl[scode[j]]) * id2[d];
          ex.x += c * (sten[j] - mi.x);
          ex.y += c * (sten[NR * L + j] - mi.y);
          ex.z += c * (sten[2 * NR * L + j] - mi.z);
        }
      } else {
        // missing neighbours (grid edge or vacuum) are the DMI ghost values
        const float cbc = __ldg(&lut->dbc[ci]);
        float3 v[4];
#pragma unroll
        for (int d = 0; d < 6; ++d) {
          const int j = nb[d];
          const int cj = scode[j];
          const bool present = (j != C || per[d]) && cj != kVacuum;
          const float3 mj = present ? f3(sten[j], sten[NR * L + j], sten[2 * NR * L + j])
                                    : dmi_ghost(mi, d, cbc, g.cdx, g.cdy);
          const float c = T.exch ? __ldg(&xl[present ? cj : ci]) * id2[d] : 0.0f;
          ex.x += c * (mj.x - mi.x);
          ex.y += c * (mj.y - mi.y);
          ex.z += c * (mj.z - mi.z);
          if (d < 4) v[d] = mj;
        }
        P.dmi = dmi_field(__ldg(&lut->dmi[ci]), v[0], v[1], v[2], v[3], g.cdx, g.cdy);
      }
    }
    P.exch = ex;
    field_local(lut, T, ci, mi, sinft, P);
    const float3 tq = llg_torque(mi, total(P), __ldg(&lut->gfac[ci]), __ldg(&lut->alpha[ci]), st->precession);
    kv[q][0] = tq.x;
    kv[q][1] = tq.y;
    kv[q][2] = tq.z;
  }
#pragma unroll
  for (int q = 0; q < CPT; ++q) {
    const int e = threadIdx.x + q * NT;
    if (e >= NCELL) continue;
    const int x = e % L, r = e / L, y = y0 + r;
    if (x >= g.nx || y >= g.ny) continue;
    const int i = (z * g.ny + y) * g.nx + x;
    kout[i] = kv[q][0];
    kout[n + i] = kv[q][1];
    kout[2 * n + i] = kv[q][2];
  }
  if (mode == ROW_K1) return;
  if (mode == ROW_NEXT) {
    // 4. next stage input and its x R2C
    __syncthreads();   // every thread is done reading B_demag from sm
    float* sw = reinterpret_cast<float*>(sm);
    float* __restrict__ nxt = stage_buf(b, s + 1);
    // the transform reads x < nx rounded up to even: with an odd nx the
    // element x = nx is padding and must be zero (rows past the grid are
    // transformed but never stored)
    if (g.nx & 1)
      for (int row = threadIdx.x; row < 3 * ROWS; row += NT) sw[2 * row * PST + g.nx] = 0.f;
    const float a = sc->ah[s + 1][s];
#pragma unroll
    for (int q = 0; q < CPT; ++q) {
      const int e = threadIdx.x + q * NT;
      if (e >= NCELL) continue;
      const int x = e % L, r = e / L, y = y0 + r;
      if (x >= g.nx || y >= g.ny) continue;
      const int i = (z * g.ny + y) * g.nx + x;
      const float n0 = fmaf(a, kv[q][0], av[q][0]);
      const float n1 = fmaf(a, kv[q][1], av[q][1]);
      const float n2 = fmaf(a, kv[q][2], av[q][2]);
      nxt[i] = n0;
      nxt[n + i] = n1;
      nxt[2 * n + i] = n2;
      const float msat = cv[q] != kVacuum ? __ldg(&lut->msat[cv[q]]) : 0.f;
      sw[2 * (0 * ROWS + r) * PST + x] = msat * n0;
      sw[2 * (1 * ROWS + r) * PST + x] = msat * n1;
      sw[2 * (2 * ROWS + r) * PST + x] = msat * n2;
    }
    __syncthreads();
    if constexpr (SS) rows_fx_tma<L, ROWS, NT>(g, sm, twl, tw2, &maps.spec, y0, z);
    else rows_fx<L, ROWS, NT>(g, sm, twl, tw2, b.spec, y0, z);
    return;
  }
  // 4'. last stage: error estimate, candidate m, block max, controller
  float emax = 0.f;
  float* __restrict__ mnew = par ? p.m0 : p.m1;
  const float e6 = sc->eh[6];
#pragma unroll
  for (int q = 0; q < CPT; ++q) {
    const int e = threadIdx.x + q * NT;
    if (e >= NCELL) continue;
    const int x = e % L, r = e / L, y = y0 + r;
    if (x >= g.nx || y >= g.ny) continue;
    const int i = (z * g.ny + y) * g.nx + x;
    if (cv[q] != kVacuum) {
      const float ex = fmaf(e6, kv[q][0], av[q][0]);
      const float ey = fmaf(e6, kv[q][1], av[q][1]);
      const float ez = fmaf(e6, kv[q][2], av[q][2]);
      float err = sqrtf(ex * ex + ey * ey + ez * ez);
      if (!(err <= FLT_MAX)) err = __int_as_float(0x7f800000);
      emax = fmaxf(emax, err);
      const float mx = mv[q][0], my = mv[q][1], mz = mv[q][2];
      const float inv = rsqrtf(mx * mx + my * my + mz * mz);
      mnew[i] = mx * inv;
      mnew[n + i] = my * inv;
      mnew[2 * n + i] = mz * inv;
    } else {
      mnew[i] = mnew[n + i] = mnew[2 * n + i] = 0.0f;
    }
  }
  for (int o = 16; o > 0; o >>= 1) emax = fmaxf(emax, __shfl_xor_sync(0xffffffffu, emax, o));
  if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = emax;
  __syncthreads();
  if (threadIdx.x < 32) {
    float v = threadIdx.x < (NT >> 5) ? wmax[threadIdx.x] : 0.0f;
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (threadIdx.x == 0) {
      atomicMax(&st->err_bits, __float_as_uint(v));
      __threadfence();
      const unsigned int t = atomicAdd(&st->ticket, 1u);
      if (t == gridDim.x * gridDim.y - 1) {
        __threadfence();
        controller(st, sc, b.hist, b.fixed);
      }
    }
  }
}

Ptrs rs_ptrs(const Buffers& b) {
  Ptrs p;
  p.m0 = b.m[0];
  p.m1 = b.m[1];
  for (int j = 0; j < 7; ++j) p.k[j] = b.k[j];
  return p;
}

// Earlier-stage sums of the row kernel of stage s, elementwise over the 3 n
// values of the component-major arrays (16-byte vectors, then the tail):
// ROW_NEXT  P = m + sum_{j<s} a_{s+1,j} k_j   (the next stage input of the
//           Dormand-Prince tableau without its k_s term, Sec. IV),
// ROW_LAST  P = sum_{j<6} e_j k_j             (the error estimate without k_6),
// the coefficients carrying dt; m first, then j ascending, one fused
// multiply-add each (the row kernel adds the k_s term).  It reads only
// k_0 .. k_{s-1}, all complete once the row kernel of stage s - 1 is, and
// runs as a graph branch beside the (y, z) part of stage s.
constexpr int kPartNT = 256;

__global__ void __launch_bounds__(kPartNT) k_rs_partial(float* __restrict__ out, Ptrs p,
                                                        const DevState* __restrict__ st,
                                                        const StageCoef* __restrict__ sc, int s, int mode, int n3) {
  if (st->done) return;
  const int par = st->parity;
  float cj[6];
  const float* kp[6];
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    cj[j] = mode == ROW_NEXT ? (j < s ? sc->ah[s + 1][j] : 0.f) : sc->eh[j];
    kp[j] = pick_k(p, k_role(j, par));
  }
  const float* __restrict__ m = mode == ROW_NEXT ? (par ? p.m1 : p.m0) : nullptr;
  const int n4 = n3 >> 2, stride = gridDim.x * kPartNT;
  for (int e = blockIdx.x * kPartNT + threadIdx.x; e < n4; e += stride) {
    // (every load of the element issued before the first use)
    float4 v[6];
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 a = m ? reinterpret_cast<const float4*>(m)[e] : z4;
#pragma unroll
    for (int j = 0; j < 6; ++j) v[j] = cj[j] != 0.0f ? reinterpret_cast<const float4*>(kp[j])[e] : z4;
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      if (cj[j] != 0.0f) {
        a.x = fmaf(cj[j], v[j].x, a.x);
        a.y = fmaf(cj[j], v[j].y, a.y);
        a.z = fmaf(cj[j], v[j].z, a.z);
        a.w = fmaf(cj[j], v[j].w, a.w);
      }
    }
    reinterpret_cast<float4*>(out)[e] = a;
  }
  for (int e = 4 * n4 + blockIdx.x * kPartNT + threadIdx.x; e < n3; e += stride) {
    float a = m ? m[e] : 0.f;
#pragma unroll
    for (int j = 0; j < 6; ++j)
      if (cj[j] != 0.0f) a = fmaf(cj[j], kp[j][e], a);
    out[e] = a;
  }
}

// ROWS * L = 1024 points per block, or 256 when that leaves too few blocks.
// Threads: one per radix-8 butterfly of the three components' rows (at
// least one per cell up to 256 was measured slower on the 256 x 256 film:
// 0.162 -> 0.174 ms per step).
template <int L, int ROWS>
struct RsCfg {
  static constexpr int NT0 = 3 * ROWS * L / 8;
  static constexpr int NT1 = NT0 < 64 ? 64 : (NT0 > 512 ? 512 : NT0);
  static constexpr int NT = NT1;
};

template <int L, int ROWS, bool SL, bool SS, bool TT>
void launch_row(const Geom& g, const Buffers& b, const Terms& T, const RsMaps& maps, int s, int mode, double freq,
                double ph, cudaStream_t st, bool dep) {
  using C = RsCfg<L, ROWS>;
  StageCoef* sc = reinterpret_cast<StageCoef*>(b.st + 1);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((g.ny + ROWS - 1) / ROWS, g.nz);
  cfg.blockDim = dim3(C::NT);
  cfg.dynamicSmemBytes = RsSmem<L, ROWS>::BYTES;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = dep ? 1 : 0;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k_rs_row<L, ROWS, C::NT, SL, SS, TT>, g, b, T, rs_ptrs(b), b.st, sc, s, mode, freq, ph,
                     maps);
}

template <int L, int ROWS>
void launch_rs(const Geom& g, const Buffers& b, const Terms& T, const RsMaps& maps, int kind, int s, int mode,
               double freq, double phase, cudaStream_t st, bool dep) {
  using C = RsCfg<L, ROWS>;
  constexpr bool SPEC = rs_spec_shape<L, ROWS>(), STEN = rs_sten_shape<L>();
  const bool spec = SPEC && maps.ok_spec, sten = STEN && maps.ok_sten;
  const double ph = phase / 3.14159265358979323846;
  if (kind == 0) {
    dim3 grid((g.ny + ROWS - 1) / ROWS, g.nz);
    StageCoef* sc = reinterpret_cast<StageCoef*>(b.st + 1);
    if constexpr (SPEC && kRsPS) {
      if (spec) {
        k_rs_prep<L, ROWS, C::NT, true><<<grid, C::NT, 0, st>>>(g, b, rs_ptrs(b), b.st, sc, s, maps);
        return;
      }
    }
    k_rs_prep<L, ROWS, C::NT, false><<<grid, C::NT, 0, st>>>(g, b, rs_ptrs(b), b.st, sc, s, maps);
    return;
  }
  if constexpr (SPEC && STEN) {
    if (spec && sten) return launch_row<L, ROWS, kRsSL, kRsSS, kRsTT>(g, b, T, maps, s, mode, freq, ph, st, dep);
  }
  if constexpr (STEN) {
    if (sten) return launch_row<L, ROWS, false, false, kRsTT>(g, b, T, maps, s, mode, freq, ph, st, dep);
  }
  launch_row<L, ROWS, false, false, false>(g, b, T, maps, s, mode, freq, ph, st, dep);
}

template <int L, int ROWS, bool SL, bool SS, bool TT>
cudaError_t prepare_row() {
  return cudaFuncSetAttribute(k_rs_row<L, ROWS, RsCfg<L, ROWS>::NT, SL, SS, TT>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, RsSmem<L, ROWS>::BYTES);
}

template <int L, int ROWS>
cudaError_t prepare_rs() {
  cudaError_t e = prepare_row<L, ROWS, false, false, false>();
  if constexpr (rs_sten_shape<L>()) {
    if (e == cudaSuccess) e = prepare_row<L, ROWS, false, false, kRsTT>();
  }
  if constexpr (rs_spec_shape<L, ROWS>() && rs_sten_shape<L>()) {
    if (e == cudaSuccess) e = prepare_row<L, ROWS, kRsSL, kRsSS, kRsTT>();
  }
  return e;
}

template <int L>
struct RsRows {
  static constexpr int R1 = L >= 1024 ? 1 : 1024 / L;
  static constexpr int R2 = L >= 256 ? 1 : 256 / L;
  static bool big(const Geom& g) { return (long long)((g.ny + R1 - 1) / R1) * g.nz >= 300; }
  static int rows(const Geom& g) { return big(g) ? R1 : R2; }
};

template <int L>
void launch_rs_l(const Geom& g, const Buffers& b, const Terms& T, const RsMaps& maps, int kind, int s, int mode,
                 double freq, double phase, cudaStream_t st, bool dep) {
  if (RsRows<L>::big(g)) launch_rs<L, RsRows<L>::R1>(g, b, T, maps, kind, s, mode, freq, phase, st, dep);
  else launch_rs<L, RsRows<L>::R2>(g, b, T, maps, kind, s, mode, freq, phase, st, dep);
}

template <int L>
cudaError_t prepare_rs_l(const Geom& g) {
  return RsRows<L>::big(g) ? prepare_rs<L, RsRows<L>::R1>() : prepare_rs<L, RsRows<L>::R2>();
}

// rows per block of the row kernels for this grid
int rs_rows(const Geom& g) {
  switch (g.lx) {
    case 16: return RsRows<16>::rows(g);
    case 32: return RsRows<32>::rows(g);
    case 64: return RsRows<64>::rows(g);
    case 128: return RsRows<128>::rows(g);
    case 256: return RsRows<256>::rows(g);
    case 512: return RsRows<512>::rows(g);
    default: return 0;
  }
}

// the driver's tensor-map encoder, fetched once through the runtime (no link
// against the driver library)
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled() {
  // (a function-local static: initialised once, thread-safe)
  static const EncodeTiledFn fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return reinterpret_cast<EncodeTiledFn>(f);
    return EncodeTiledFn(nullptr);
  }();
  return fn;
}

// one tiled map of `rank` dimensions (innermost first); strides in bytes of
// dimensions 1..rank-1; zero fill out of range
bool encode(CUtensorMap* m, CUtensorMapDataType t, int rank, void* base, const cuuint64_t* dims,
            const cuuint64_t* strides, const cuuint32_t* box) {
  EncodeTiledFn fn = encode_tiled();
  if (!fn) return false;
  const cuuint32_t es[5] = {1, 1, 1, 1, 1};
  return fn(m, t, (cuuint32_t)rank, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

}  // namespace

cudaError_t prepare_rowstage(const Geom& g) {
  switch (g.lx) {
    case 16: return prepare_rs_l<16>(g);
    case 32: return prepare_rs_l<32>(g);
    case 64: return prepare_rs_l<64>(g);
    case 128: return prepare_rs_l<128>(g);
    case 256: return prepare_rs_l<256>(g);
    case 512: return prepare_rs_l<512>(g);
    default: return cudaSuccess;
  }
}

// Tensor-copy conditions.  Spectrum box: a shape with rs_spec_shape (32 <=
// L <= 128, >= 8 rows per block) and rows of ny complex values whose stride
// is a multiple of 16 bytes (ny even).  Stencil rows: 32 <= L <= 256, rows of
// nx floats with a 16-byte multiple stride (nx % 4 == 0), y not periodic (the
// halo rows would wrap).
void rowstage_maps(const Geom& g, const Buffers& b, RsMaps* m) {
  std::memset(m, 0, sizeof(RsMaps));
  const int L = g.lx, rows = rs_rows(g);
  if (!g.fused || g.pbcx || !b.spec || !b.ms || !b.ms2 || !b.code) return;
  if (L >= 32 && L <= 128 && rows >= 8 && g.ny % 2 == 0) {
    const cuuint64_t dims[4] = {(cuuint64_t)g.ny, (cuuint64_t)g.nz, (cuuint64_t)g.hx, 3};
    const cuuint64_t st[3] = {(cuuint64_t)g.ny * 8, (cuuint64_t)g.nz * g.ny * 8, (cuuint64_t)g.hx * g.nz * g.ny * 8};
    const cuuint32_t box[4] = {(cuuint32_t)rows, 1, (cuuint32_t)(L + 1), 3};
    m->ok_spec = encode(&m->spec, CU_TENSOR_MAP_DATA_TYPE_UINT64, 4, b.spec, dims, st, box) ? 1 : 0;
  }
  if (L >= 32 && L <= 256 && g.nx % 4 == 0 && !g.pbcy) {
    bool ok = true;
    {
      const cuuint64_t dims[4] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz, 3};
      const cuuint64_t st[3] = {(cuuint64_t)g.nx * 4, (cuuint64_t)g.ny * g.nx * 4, (cuuint64_t)g.n * 4};
      const cuuint32_t own[4] = {(cuuint32_t)L, (cuuint32_t)(rows + 2), 1, 1};
      const cuuint32_t pl[4] = {(cuuint32_t)L, (cuuint32_t)rows, 1, 1};
      ok = ok && encode(&m->ms_own, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, b.ms, dims, st, own);
      ok = ok && encode(&m->ms_pl, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, b.ms, dims, st, pl);
      ok = ok && encode(&m->ms2_own, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, b.ms2, dims, st, own);
      ok = ok && encode(&m->ms2_pl, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, b.ms2, dims, st, pl);
    }
    {
      const cuuint64_t dims[3] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz};
      const cuuint64_t st[2] = {(cuuint64_t)g.nx * 4, (cuuint64_t)g.ny * g.nx * 4};
      const cuuint32_t own[3] = {(cuuint32_t)L, (cuuint32_t)(rows + 2), 1};
      const cuuint32_t pl[3] = {(cuuint32_t)L, (cuuint32_t)rows, 1};
      ok = ok && encode(&m->code_own, CU_TENSOR_MAP_DATA_TYPE_INT32, 3, b.code, dims, st, own);
      ok = ok && encode(&m->code_pl, CU_TENSOR_MAP_DATA_TYPE_INT32, 3, b.code, dims, st, pl);
    }
    m->ok_sten = ok ? 1 : 0;
  }
}

// Up to two blocks per multiprocessor: the kernel shares the GPU with the
// (y, z) kernels of the same stage and has their whole duration to finish.
void launch_rs_partial(const Geom& g, const Buffers& b, int s, int mode, cudaStream_t st) {
  const int n3 = 3 * (int)g.n;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 1;
  const int blocks = std::max(1, std::min((n3 / 4 + kPartNT - 1) / kPartNT, 2 * sms));
  StageCoef* sc = reinterpret_cast<StageCoef*>(b.st + 1);
  k_rs_partial<<<blocks, kPartNT, 0, st>>>(b.part, rs_ptrs(b), b.st, sc, s, mode, n3);
}

// kind 0: prep of stage s; kind 1: row kernel of stage s with mode 0 (first
// stage only), 1 (next stage), 2 (last stage: error and controller); the row
// kernel is a programmatic dependent of its predecessor where pdl_row(g) or
// `dep` says so
void launch_rowstage(const Geom& g, const Buffers& b, const Terms& T, const RsMaps& maps, int kind, int s, int mode,
                     double freq, double phase, cudaStream_t st, bool dep) {
  dep = dep || pdl_row(g);
  switch (g.lx) {
    case 16: launch_rs_l<16>(g, b, T, maps, kind, s, mode, freq, phase, st, dep); break;
    case 32: launch_rs_l<32>(g, b, T, maps, kind, s, mode, freq, phase, st, dep); break;
    case 64: launch_rs_l<64>(g, b, T, maps, kind, s, mode, freq, phase, st, dep); break;
    case 128: launch_rs_l<128>(g, b, T, maps, kind, s, mode, freq, phase, st, dep); break;
    case 256: launch_rs_l<256>(g, b, T, maps, kind, s, mode, freq, phase, st, dep); break;
    case 512: launch_rs_l<512>(g, b, T, maps, kind, s, mode, freq, phase, st, dep); break;
    default: break;
  }
}

}  // namespace mm
