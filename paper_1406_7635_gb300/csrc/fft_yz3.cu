// The (y, z) part of the fused demag convolution (Sec. III.B) for 3-D grids
// as three kernels over a y-transformed buffer T instead of one cluster per
// kx plane:
//
//   k_yf  y forward: spectrum rows spec[c][kx][z][y] (y < ny, the rest is
//         zero padding and never read) -> T[kx][c][z][ky], ky < py;
//   k_zk  one (kx, ky) column of all three components per 6 threads: z
//         forward (nz inputs, pz points), the kernel product B_i = K_ij M_j
//         with the octant's mirror signs, z inverse cropped to z < nz, in
//         place in T;
//   k_yi  y inverse: T rows -> spectrum rows, cropped to y < ny;
//
// and, for 2-D grids (pz = 1), k_y2d: y forward, kernel product and y
// inverse of one kx plane in one block.
//
// Both transforms split their padded length by frequency parity: with
// k = 2 j + r, the padded DFT restricted to class r is the half-length DFT of
// x[n] W_P^(r n), exact because the inputs fill at most half the padded
// length.  The y classes are two pencils per row: for 64..256 points per
// class each pencil is held in the registers of PH / 16 lanes of one warp
// (k_yf3 / k_yi3 / k_y2d), otherwise it is transformed by Stockham passes in
// shared memory (k_yf / k_yi).  The z classes are held in registers (pz / 2
// points per thread), one thread per (column, component, class), so the z
// transforms need no shared-memory passes at all: the threads of a column
// exchange only the spectra the product needs and, after the inverse, the
// halves of the two classes (a lane-pair shuffle).
//
// Every global access is contiguous: rows of y in and out of the spectrum,
// rows of ky in T (16-byte pairs (2j, 2j + 1) of the two classes), and in the
// column kernel runs of consecutive ky for each (component, z).  The kernels
// are launched with programmatic dependent launch and wait for their
// predecessor before reading its output; the inverse transforms are
// unnormalised (the kernel octant carries the 1 / (lx py pz) factor and
// -mu0).
#include <algorithm>

#include "fft.cuh"
#include "mm_internal.h"

namespace mm {
namespace {
using namespace mmfft;

// Threads of the y kernels.  Small blocks (two warps, 8 rows of up to 128
// points) keep every block of the 128 x 128 x 32 grid (4 z chunks x 3
// components x 129 kx planes) resident at once: 12 blocks per SM.
constexpr int kYNT = 64;
constexpr int y_min_blocks(int PH) { return PH >= 512 ? 8 : 12; }   // (rows of 512: more registers)

// spectrum rows (z) per block of the y kernels: 8 (16 pencils of up to 128
// points), fewer for longer rows so that a thread holds at most 32 values
// per pass
template <int PH>
struct YCfg {
  static constexpr int ROWS = PH <= 128 ? 8 : 1024 / PH;
  static constexpr int NP = 2 * ROWS;         // pencils: class r = p / ROWS, row p % ROWS
  static constexpr int P = PH + 1;            // pencil pitch (odd: conflict-free columns of pencils)
  static constexpr size_t SMEM = sizeof(float2) * NP * P;
};

// y forward of ROWS rows (z0 ..) of one (kx, c) plane.  The rows land in
// the class-0 pencils by asynchronous copies (all in flight at once); the
// class-1 pencils are x W_(2 PH)^y of them.
template <int PH>
__global__ void __launch_bounds__(kYNT, y_min_blocks(PH)) k_yf(Geom g, const float2* __restrict__ spec, float2* __restrict__ T,
                                             const float2* __restrict__ tw, const DevState* __restrict__ st) {
  using Y = YCfg<PH>;
  constexpr int ROWS = Y::ROWS, P = Y::P;
  extern __shared__ float2 sm[];
  __shared__ float2 twh[PH], twc[PH];   // W_PH^i and the class-1 twiddle W_(2 PH)^y
  const int z0 = blockIdx.x * ROWS, c = blockIdx.y, kx = blockIdx.z;
  twiddles_async<kYNT>(twh, tw, PH, kTwN / PH);
  twiddles_async<kYNT>(twc, tw, PH, kTwN / (2 * PH));
  const int ny = g.ny, nz = g.nz;
  // the (c, kx) plane [z][y] of the spectrum (32-bit offsets: 3 hx nz ny < 2^31)
  const float2* __restrict__ src = spec + (c * g.hx + kx) * nz * ny;
  grid_dependency_wait();   // the spectrum comes from the previous kernel
  // (the done flag is read once the predecessor, which may set it, has
  // completed: every thread sees one value)
  if (st && st->done) {
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    return;
  }
  for (int e = threadIdx.x; e < ROWS * PH; e += kYNT) {
    const int i = e / PH, y = e % PH, z = z0 + i;
    if (y >= ny) continue;   // zero padding: the first pass reads y < ny only
    if (z < nz) cp_async_f2(&sm[i * P + y], src + z * ny + y);
    else sm[i * P + y] = make_float2(0.f, 0.f);
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  __syncthreads();
  for (int e = threadIdx.x; e < ROWS * PH; e += kYNT) {
    const int i = e / PH, y = e % PH;
    if (y < ny) sm[(ROWS + i) * P + y] = cmul(sm[i * P + y], twc[y]);
  }
  __syncthreads();
  FftG<PH, -1, Y::NP, kYNT, 1, P, 1, PH>::run(sm, twh, nullptr, ny);
  // ky = 2 j + r: the two classes' values at j are the pair (2 j, 2 j + 1)
  float4* __restrict__ dst = reinterpret_cast<float4*>(T) + ((kx * 3 + c) * nz) * PH;
  for (int e = threadIdx.x; e < ROWS * PH; e += kYNT) {
    const int i = e / PH, j = e % PH, z = z0 + i;
    if (z >= nz) continue;
    const float2 a = sm[i * P + j], b = sm[(ROWS + i) * P + j];
    dst[z * PH + j] = make_float4(a.x, a.y, b.x, b.y);
  }
}

// y inverse of ROWS rows of one (kx, c) plane, cropped to y < ny; the T rows
// land de-interleaved in the two class pencils by asynchronous copies
template <int PH>
__global__ void __launch_bounds__(kYNT, y_min_blocks(PH)) k_yi(Geom g, const float2* __restrict__ T, float2* __restrict__ spec,
                                             const float2* __restrict__ tw, const DevState* __restrict__ st) {
  using Y = YCfg<PH>;
  constexpr int ROWS = Y::ROWS, P = Y::P;
  extern __shared__ float2 sm[];
  __shared__ float2 twh[PH], twc[PH];
  const int z0 = blockIdx.x * ROWS, c = blockIdx.y, kx = blockIdx.z;
  twiddles_async<kYNT>(twh, tw, PH, kTwN / PH);
  twiddles_async<kYNT>(twc, tw, PH, kTwN / (2 * PH));
  const int ny = g.ny, nz = g.nz;
  const float2* __restrict__ src = T + ((kx * 3 + c) * nz) * (2 * PH);
  grid_dependency_wait();   // T comes from the column kernel
  if (st && st->done) {      // (after the predecessor: one value for all threads)
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    return;
  }
  for (int e = threadIdx.x; e < ROWS * PH; e += kYNT) {
    const int i = e / PH, j = e % PH, z = z0 + i;
    if (z < nz) {
      cp_async_f2(&sm[i * P + j], src + z * (2 * PH) + 2 * j);
      cp_async_f2(&sm[(ROWS + i) * P + j], src + z * (2 * PH) + 2 * j + 1);
    } else {
      sm[i * P + j] = sm[(ROWS + i) * P + j] = make_float2(0.f, 0.f);
    }
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  __syncthreads();
  FftG<PH, 1, Y::NP, kYNT, 1, P, 1, PH>::run(sm, twh, nullptr, PH, ny);   // outputs y >= ny cropped
  // x[y] = X_0[y] + conj(W_(2 PH)^y) X_1[y]
  float2* __restrict__ out = spec + (c * g.hx + kx) * nz * ny;
  for (int e = threadIdx.x; e < ROWS * PH; e += kYNT) {
    const int i = e / PH, y = e % PH, z = z0 + i;
    if (z >= nz || y >= ny) continue;
    out[z * ny + y] = cadd(sm[i * P + y], cmul(sm[(ROWS + i) * P + y], cconj(twc[y])));
  }
}

// (kx, ky) columns per block of the column kernel and its threads: 3
// components x 2 classes x 16 columns.  Blocks of three warps (25 KB of
// shared memory at pz = 64) leave 7 per SM resident; the 128 x 128 x 32 grid
// has 16 x 129 of them, just under two rounds.
constexpr int kZCols = 16;
constexpr int kZNT = 96;
constexpr int kZMinBlocks = 7;

template <int LZH>
struct ZCfg {
  static constexpr int PZ = 2 * LZH;
  static constexpr int CP = kZCols;   // complex values per kz row of the block's columns
  static constexpr size_t SMEM = sizeof(float2) * 3 * PZ * CP;
};

// Thread (warp w, lane): component c = w, class rz = lane / 16, column
// lane % 16 of the block (a half-warp holds 16 consecutive columns of one
// class: conflict-free rows of the shared spectra).
template <int LZH>
__global__ void __launch_bounds__(kZNT, kZMinBlocks) k_zk(Geom g, float2* __restrict__ T, const float* __restrict__ kt,
                                             const float2* __restrict__ tw, const DevState* __restrict__ st) {
  using Z = ZCfg<LZH>;
  constexpr int PZ = Z::PZ, CP = Z::CP;
  extern __shared__ float2 sA[];        // [component][kz][column]: the forward spectra
  __shared__ float2 twz[PZ];            // W_PZ^z
  __shared__ float2 twl[LZH];           // W_LZH^l (the 32-point register transform)
  twiddles_async<kZNT>(twz, tw, PZ, kTwN / PZ);
  twiddles_async<kZNT>(twl, tw, LZH, kTwN / LZH);
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int c = threadIdx.x >> 5, rz = lane >> 4, col = lane & 15;
  const int kx = blockIdx.y, ky = blockIdx.x * kZCols + col;
  const int nz = g.nz, PY = g.py;
  // column (kx, c, ., ky) of T, z stride PY (32-bit offsets: 3 hx nz py < 2^31)
  float2* __restrict__ cp = T + (kx * 3 + c) * nz * PY + ky;
  // the block's kernel-octant rows (6 components x (PZ/2 + 1) kz rows of its
  // 16 columns, read in the product below) do not depend on the previous
  // kernel: ask for them in L2 while it drains
  {
    const int my = blockIdx.x * kZCols > PY / 2;
    const int iy0 = my ? PY - (blockIdx.x * kZCols + kZCols - 1) : blockIdx.x * kZCols;
    const int per = g.hky * g.hkz;
    for (int e = threadIdx.x; e < 6 * (PZ / 2 + 1); e += kZNT) {
      const int t = e / (PZ / 2 + 1), iz = e % (PZ / 2 + 1);
      asm volatile("prefetch.global.L2 [%0];\n" ::"l"(kt + kx * 6 * per + t * per + iz * g.hky + iy0));
    }
  }
  grid_dependency_wait();   // T comes from the y kernel
  if (st && st->done) return;   // (after the predecessor: one value for all threads)
  // 1. class rz of component c: the LZH-point DFT of a[z] W_PZ^(rz z)
  float2 v[LZH];
#pragma unroll
  for (int z = 0; z < LZH; ++z) v[z] = z < nz ? cp[z * PY] : make_float2(0.f, 0.f);
  if (rz) {
#pragma unroll
    for (int z = 0; z < LZH; ++z) v[z] = cmul(v[z], twz[z]);
  }
  RegDft<LZH, -1>::run(v, twl);   // v[l] = A_c(kz = 2 l + rz)
#pragma unroll
  for (int l = 0; l < LZH; ++l) sA[(c * PZ + 2 * l + rz) * CP + col] = v[l];
  __syncthreads();
  // 2. the kernel product B_i = sum_j K_ij A_j at every (kz, column) point of
  //    the block, all three components per point, in place in sA.  Thread t
  //    takes column t % 16 and kz = t / 16 + KZS k (KZS = threads / 16), so
  //    the column, its mirror sign and octant row are per-thread constants;
  //    a half-warp covers 16 consecutive columns (conflict-free shared
  //    memory, 64-byte octant rows).  The octant holds K at (|ky|, |kz|):
  //    Kxy is odd in ky, Kxz in kz, Kyz in both.
  {
    constexpr int KZS = kZNT / kZCols;              // kz stride between a thread's points
    constexpr int NPT = (PZ + KZS - 1) / KZS;       // points per thread (the last may be empty)
    constexpr int CH = 4;                           // points whose loads are issued together
    const int pc = threadIdx.x % kZCols, kz0 = threadIdx.x / kZCols;
    const int pky = blockIdx.x * kZCols + pc;
    const bool my = pky > PY / 2;
    const float sgy = my ? -1.f : 1.f;
    const int per = g.hky * g.hkz;                  // octant: 6 hkx hky hkz < 2^31 floats
    const float* __restrict__ kb = kt + kx * 6 * per + (my ? PY - pky : pky);
#pragma unroll
    for (int k0 = 0; k0 < NPT; k0 += CH) {
      float kc[CH][6];
      float2 A[CH][3];
#pragma unroll
      for (int u = 0; u < CH; ++u) {
        const int kz = kz0 + (k0 + u) * KZS;
        if (k0 + u >= NPT || (PZ % KZS != 0 && kz >= PZ)) continue;
        const float* __restrict__ kq = kb + (kz > PZ / 2 ? PZ - kz : kz) * g.hky;
#pragma unroll
        for (int t = 0; t < 6; ++t) kc[u][t] = __ldg(kq + t * per);
#pragma unroll
        for (int j = 0; j < 3; ++j) A[u][j] = sA[(j * PZ + kz) * CP + pc];
      }
#pragma unroll
      for (int u = 0; u < CH; ++u) {
        const int kz = kz0 + (k0 + u) * KZS;
        if (k0 + u >= NPT || (PZ % KZS != 0 && kz >= PZ)) continue;
        const float sgz = kz > PZ / 2 ? -1.f : 1.f;
        const float kxx = kc[u][0], kyy = kc[u][1], kzz = kc[u][2];
        const float kxy = sgy * kc[u][3], kxz = sgz * kc[u][4], kyz = sgy * sgz * kc[u][5];
        const float2 X = A[u][0], Y = A[u][1], Zc = A[u][2];
        sA[kz * CP + pc] = make_float2(kxx * X.x + kxy * Y.x + kxz * Zc.x, kxx * X.y + kxy * Y.y + kxz * Zc.y);
        sA[(PZ + kz) * CP + pc] =
            make_float2(kxy * X.x + kyy * Y.x + kyz * Zc.x, kxy * X.y + kyy * Y.y + kyz * Zc.y);
        sA[(2 * PZ + kz) * CP + pc] =
            make_float2(kxz * X.x + kyz * Y.x + kzz * Zc.x, kxz * X.y + kyz * Y.y + kzz * Zc.y);
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int l = 0; l < LZH; ++l) v[l] = sA[(c * PZ + 2 * l + rz) * CP + col];
  // 3. inverse class transform: v[z] = sum_l B_c(2 l + rz) W_LZH^(-z l)
  RegDft<LZH, 1>::run(v, twl);
  // 4. b[z] = V_0[z] + conj(W_PZ^z) V_1[z]: the class-0 lane writes z < LZH / 2,
  //    the class-1 lane (16 lanes up) the rest, each with the partner's half
  //    by a shuffle
  constexpr int HH = LZH / 2;
#pragma unroll
  for (int i = 0; i < HH; ++i) {
    const float2 send = rz ? v[i] : v[i + HH];
    const float2 recv =
        make_float2(__shfl_xor_sync(0xffffffffu, send.x, 16), __shfl_xor_sync(0xffffffffu, send.y, 16));
    const int z = rz ? i + HH : i;
    const float2 w = cconj(twz[z]);
    const float2 b = rz ? cadd(recv, cmul(v[i + HH], w)) : cadd(v[i], cmul(recv, w));
    if (z < nz) cp[z * PY] = b;
  }
}

// ---------------------------------------------------------------------------
// Register-resident y kernels for rows of PH = 64, 128, 256 points: a row of
// one parity class is held by G = PH / 16 lanes, 16 values each (y = j + G r,
// lane j), so the PH-point transform is one 16-point DFT per lane over r, a
// twiddle, a transpose through a per-warp shared buffer, and 16 / G G-point
// DFTs per lane:
//   X[k1 + 16 k2] = sum_j W_G^(j k2) W_PH^(j k1) sum_r x[j + G r] W_16^(r k1).
// No block barrier: the lanes of a row belong to one warp.  The two classes
// of a row go to neighbouring lanes (lane = 2 j + class within the row's 2 G
// lanes; the class-1 input is x W_(2 PH)^y), so each 16-byte (2j, 2j + 1)
// pair of T is written and read by a lane pair in one instruction, and the
// y inverse combines its classes by a lane shuffle.  Lane j ends with the
// outputs k1 = j + G h (h < 16 / G), k2 < G.  Measured against the same
// transforms with the two classes one after the other in the same lanes
// (half the lanes, 0.85 waves, 8-byte accesses at a 16-byte stride): 128 x
// 128 x 32 step 0.448 -> 0.435 ms.
// ---------------------------------------------------------------------------
constexpr int kY2NT = 64;   // two warps per block

template <int PH>
struct Y3Cfg {
  static constexpr int G = PH / 16;          // lanes per (row, class)
  static constexpr int H = 16 / G;           // k1 values per lane
  static constexpr int RPW = 16 / G;         // rows per warp
  static constexpr int ROWS = RPW * (kY2NT / 32);
  static constexpr int EP = 17;              // exchange pitch of one lane's 16 values
  static constexpr int EW = RPW * 2 * G * EP;   // exchange buffer per warp (complex values)
};
constexpr int kY3MinBlocks = 16;

template <int PH>
__global__ void __launch_bounds__(kY2NT, kY3MinBlocks) k_yf3(Geom g, const float2* __restrict__ spec,
                                                             float2* __restrict__ T, const float2* __restrict__ tw,
                                                             const DevState* __restrict__ st) {
  using Y = Y3Cfg<PH>;
  constexpr int G = Y::G, H = Y::H, EP = Y::EP;
  __shared__ float2 twh[PH], twc[PH];   // W_PH^i and the class-1 twiddle W_(2 PH)^y
  __shared__ float2 ex[(kY2NT / 32) * Y::EW];
  twiddles_async<kY2NT>(twh, tw, PH, kTwN / PH);
  twiddles_async<kY2NT>(twc, tw, PH, kTwN / (2 * PH));
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rw = lane / (2 * G), j = (lane % (2 * G)) >> 1, cls = lane & 1;
  const int c = blockIdx.y, kx = blockIdx.z;
  const int z = blockIdx.x * Y::ROWS + warp * Y::RPW + rw;
  const int ny = g.ny, nz = g.nz;
  float2* e = ex + warp * Y::EW + (2 * rw + cls) * G * EP;   // this (row, class)'s exchange area [j][k1]
  grid_dependency_wait();   // the spectrum comes from the previous kernel
  if (st && st->done) return;   // (after the predecessor: one value for all threads)
  const float2* __restrict__ src = spec + ((c * g.hx + kx) * nz + (z < nz ? z : 0)) * ny;
  float2* __restrict__ dst = T + ((kx * 3 + c) * nz + (z < nz ? z : 0)) * (2 * PH);
  float2 v[16];
#pragma unroll
  for (int r = 0; r < 16; ++r) {
    const int y = j + G * r;
    const float2 x = (z < nz && y < ny) ? src[y] : make_float2(0.f, 0.f);
    v[r] = cls ? cmul(x, twc[y]) : x;
  }
  Dft<16, -1>::run(v);                                    // v[k1] = sum_r x W_16^(r k1)
#pragma unroll
  for (int k1 = 1; k1 < 16; ++k1) v[k1] = cmul(v[k1], twh[(j * k1) & (PH - 1)]);
#pragma unroll
  for (int k1 = 0; k1 < 16; ++k1) e[j * EP + k1] = v[k1];
  __syncwarp();
  float2 w[H][G];
#pragma unroll
  for (int h = 0; h < H; ++h)
#pragma unroll
    for (int jj = 0; jj < G; ++jj) w[h][jj] = e[jj * EP + j + G * h];
#pragma unroll
  for (int h = 0; h < H; ++h) {
    Dft<G, -1>::run(w[h]);                                // w[h][k2] = X(k1 + 16 k2), k1 = j + G h
    if (z < nz) {
#pragma unroll
      for (int k2 = 0; k2 < G; ++k2) dst[2 * (j + G * h + 16 * k2) + cls] = w[h][k2];
    }
  }
}

template <int PH>
__global__ void __launch_bounds__(kY2NT, kY3MinBlocks) k_yi3(Geom g, const float2* __restrict__ T,
                                                             float2* __restrict__ spec, const float2* __restrict__ tw,
                                                             const DevState* __restrict__ st) {
  using Y = Y3Cfg<PH>;
  constexpr int G = Y::G, H = Y::H, EP = Y::EP;
  __shared__ float2 twh[PH], twc[PH];
  __shared__ float2 ex[(kY2NT / 32) * Y::EW];
  twiddles_async<kY2NT>(twh, tw, PH, kTwN / PH);
  twiddles_async<kY2NT>(twc, tw, PH, kTwN / (2 * PH));
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rw = lane / (2 * G), j = (lane % (2 * G)) >> 1, cls = lane & 1;
  const int c = blockIdx.y, kx = blockIdx.z;
  const int z = blockIdx.x * Y::ROWS + warp * Y::RPW + rw;
  const int ny = g.ny, nz = g.nz;
  float2* e = ex + warp * Y::EW + (2 * rw + cls) * G * EP;
  grid_dependency_wait();   // T comes from the column kernel
  if (st && st->done) return;   // (after the predecessor: one value for all threads)
  const float2* __restrict__ src = T + ((kx * 3 + c) * nz + (z < nz ? z : 0)) * (2 * PH);
  // lane j of class cls holds X(k1 + 16 k2) for k1 = j + G h: inverse over k2 first
  float2 w[H][G];
#pragma unroll
  for (int h = 0; h < H; ++h)
#pragma unroll
    for (int k2 = 0; k2 < G; ++k2)
      w[h][k2] = z < nz ? src[2 * (j + G * h + 16 * k2) + cls] : make_float2(0.f, 0.f);
#pragma unroll
  for (int h = 0; h < H; ++h) {
    Dft<G, 1>::run(w[h]);                                 // w[h][jj] = V(jj, k1)
#pragma unroll
    for (int jj = 0; jj < G; ++jj) {
      const int k1 = j + G * h;
      e[jj * EP + k1] = (jj && k1) ? cmul(w[h][jj], cconj(twh[(jj * k1) & (PH - 1)])) : w[h][jj];
    }
  }
  __syncwarp();
  float2 v[16];
#pragma unroll
  for (int k1 = 0; k1 < 16; ++k1) v[k1] = e[j * EP + k1];
  Dft<16, 1>::run(v);                                     // v[r] = x_cls(j + G r)
  // y = j + G r: x_0 + conj(W_(2 PH)^y) x_1; the class-0 lane writes r < 8,
  // the class-1 lane (its neighbour) r >= 8, each with the partner's half
  float2* __restrict__ out = spec + ((c * g.hx + kx) * nz + (z < nz ? z : 0)) * ny;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const float2 send = cls ? v[i] : v[i + 8];
    const float2 recv =
        make_float2(__shfl_xor_sync(0xffffffffu, send.x, 1), __shfl_xor_sync(0xffffffffu, send.y, 1));
    const int y = j + G * (cls ? i + 8 : i);
    const float2 t = cconj(twc[y]);
    const float2 b = cls ? cadd(recv, cmul(v[i + 8], t)) : cadd(v[i], cmul(recv, t));
    if (z < nz && y < ny) out[y] = b;
  }
}

template <int PH>
void run_y3(const Geom& g, const Buffers& b, float2* T, bool forward, cudaStream_t s) {
  using Y = Y3Cfg<PH>;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((g.nz + Y::ROWS - 1) / Y::ROWS, 3, g.hx);
  cfg.blockDim = dim3(kY2NT);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (forward) cudaLaunchKernelEx(&cfg, k_yf3<PH>, g, (const float2*)b.spec, T, (const float2*)b.tw, (const DevState*)b.st);
  else cudaLaunchKernelEx(&cfg, k_yi3<PH>, g, (const float2*)T, b.spec, (const float2*)b.tw, (const DevState*)b.st);
}

// ---------------------------------------------------------------------------
// 2-D grids (pz = 1): the y transform, the kernel product and the inverse y
// transform of one kx plane in one block, with the register-resident y
// transforms above.  Six rows (3 components x 2 parity classes) of G = PH/16
// lanes each; the forward spectra meet in shared memory for the product,
// and the two classes of a component (G lanes apart) combine by a shuffle.
// ---------------------------------------------------------------------------
template <int PH>
struct Y2dCfg {
  static constexpr int G = PH / 16, H = 16 / G, RPW = 32 / G, EP = 17;
  static constexpr int NT = (6 * G + 31) / 32 * 32;   // rows 6 and up (G = 8: 16 lanes) idle
  static constexpr int NW = NT / 32;
};

template <int PH>
__global__ void __launch_bounds__(Y2dCfg<PH>::NT) k_y2d(Geom g, float2* __restrict__ spec,
                                                        const float* __restrict__ kt,
                                                        const float2* __restrict__ tw,
                                                        const DevState* __restrict__ st) {
  using Y = Y2dCfg<PH>;
  constexpr int G = Y::G, H = Y::H, EP = Y::EP, PY = 2 * PH;
  __shared__ float2 twh[PH], twc[PH];
  __shared__ float2 ex[Y::NW * Y::RPW * G * EP];
  __shared__ float2 S[3 * PY];   // [component][class][k]: the spectrum at ky = 2 k + class
  twiddles_async<Y::NT>(twh, tw, PH, kTwN / PH);
  twiddles_async<Y::NT>(twc, tw, PH, kTwN / PY);
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = threadIdx.x / G, j = threadIdx.x % G;   // row = 2 c + class
  const bool act = row < 6;
  const int c = act ? row >> 1 : 0, cls = row & 1;
  const int kx = blockIdx.x, ny = g.ny;
  float2* e = ex + (warp * Y::RPW + lane / G) * G * EP;
  grid_dependency_wait();   // the spectrum comes from the previous kernel
  if (st && st->done) return;   // (after the predecessor: one value for all threads)
  float2* __restrict__ rowp = spec + (c * g.hx + kx) * ny;   // nz = 1: row (c, kx)
  // 1. forward y of class cls of component c: X(k1 + 16 k2), k1 = j + G h
  {
    float2 v[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      const int y = j + G * r;
      const float2 x = (act && y < ny) ? rowp[y] : make_float2(0.f, 0.f);
      v[r] = cls ? cmul(x, twc[y]) : x;
    }
    Dft<16, -1>::run(v);
#pragma unroll
    for (int k1 = 1; k1 < 16; ++k1) v[k1] = cmul(v[k1], twh[(j * k1) & (PH - 1)]);
#pragma unroll
    for (int k1 = 0; k1 < 16; ++k1) e[j * EP + k1] = v[k1];
    __syncwarp();
    float2 w[H][G];
#pragma unroll
    for (int h = 0; h < H; ++h)
#pragma unroll
      for (int jj = 0; jj < G; ++jj) w[h][jj] = e[jj * EP + j + G * h];
    __syncwarp();
#pragma unroll
    for (int h = 0; h < H; ++h) {
      Dft<G, -1>::run(w[h]);
      if (act) {
#pragma unroll
        for (int k2 = 0; k2 < G; ++k2) S[row * PH + j + G * h + 16 * k2] = w[h][k2];
      }
    }
  }
  __syncthreads();
  // 2. kernel product at every ky (kz = 0): Kxy is odd in ky; Kxz and Kyz
  //    (odd in kz) enter with their stored values
  {
    const int per = g.hky * g.hkz;   // octant: 6 hkx hky hkz < 2^31 floats
    const float* __restrict__ kb = kt + kx * 6 * per;
    for (int q = threadIdx.x; q < PY; q += Y::NT) {
      const int qc = q / PH, k = q % PH, ky = 2 * k + qc;
      const int iy = ky > PH ? PY - ky : ky;
      const float sy = ky > PH ? -1.f : 1.f;
      float kc[6];
#pragma unroll
      for (int t = 0; t < 6; ++t) kc[t] = __ldg(kb + t * per + iy);
      const float kxx = kc[0], kyy = kc[1], kzz = kc[2], kxy = sy * kc[3], kxz = kc[4], kyz = sy * kc[5];
      const float2 X = S[(0 + qc) * PH + k], Yv = S[(2 + qc) * PH + k], Z = S[(4 + qc) * PH + k];
      S[(0 + qc) * PH + k] = make_float2(kxx * X.x + kxy * Yv.x + kxz * Z.x, kxx * X.y + kxy * Yv.y + kxz * Z.y);
      S[(2 + qc) * PH + k] = make_float2(kxy * X.x + kyy * Yv.x + kyz * Z.x, kxy * X.y + kyy * Yv.y + kyz * Z.y);
      S[(4 + qc) * PH + k] = make_float2(kxz * X.x + kyz * Yv.x + kzz * Z.x, kxz * X.y + kyz * Yv.y + kzz * Z.y);
    }
  }
  __syncthreads();
  // 3. inverse y of the class, then x[y] = x_0[y] + conj(W_PY^y) x_1[y]: the
  //    class-0 lane writes r < 8, the class-1 lane (G lanes up) r >= 8
  float2 v[16];
  {
    float2 w[H][G];
#pragma unroll
    for (int h = 0; h < H; ++h)
#pragma unroll
      for (int k2 = 0; k2 < G; ++k2) w[h][k2] = act ? S[row * PH + j + G * h + 16 * k2] : make_float2(0.f, 0.f);
#pragma unroll
    for (int h = 0; h < H; ++h) {
      Dft<G, 1>::run(w[h]);
#pragma unroll
      for (int jj = 0; jj < G; ++jj) {
        const int k1 = j + G * h;
        e[jj * EP + k1] = (jj && k1) ? cmul(w[h][jj], cconj(twh[(jj * k1) & (PH - 1)])) : w[h][jj];
      }
    }
    __syncwarp();
#pragma unroll
    for (int k1 = 0; k1 < 16; ++k1) v[k1] = e[j * EP + k1];
    Dft<16, 1>::run(v);   // v[r] = x_class(j + G r)
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const float2 send = cls ? v[i] : v[i + 8];
    const float2 recv =
        make_float2(__shfl_xor_sync(0xffffffffu, send.x, G), __shfl_xor_sync(0xffffffffu, send.y, G));
    const int r = cls ? i + 8 : i, y = j + G * r;
    const float2 w = cconj(twc[y]);
    const float2 out = cls ? cadd(recv, cmul(v[i + 8], w)) : cadd(v[i], cmul(recv, w));
    if (act && y < ny) rowp[y] = out;
  }
}

template <int PH>
void run_y(const Geom& g, const float2* spec_in, float2* T, float2* spec_out, const float2* tw, const DevState* st,
           cudaStream_t s, bool forward) {
  using Y = YCfg<PH>;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((g.nz + Y::ROWS - 1) / Y::ROWS, 3, g.hx);
  cfg.blockDim = dim3(kYNT);
  cfg.dynamicSmemBytes = Y::SMEM;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (forward) {
    cudaFuncSetAttribute(k_yf<PH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Y::SMEM);
    cudaLaunchKernelEx(&cfg, k_yf<PH>, g, spec_in, T, tw, st);
  } else {
    cudaFuncSetAttribute(k_yi<PH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Y::SMEM);
    cudaLaunchKernelEx(&cfg, k_yi<PH>, g, (const float2*)T, spec_out, tw, st);
  }
}

template <int LZH>
void run_z(const Geom& g, float2* T, const float* ktf, const float2* tw, const DevState* st, cudaStream_t s) {
  using Z = ZCfg<LZH>;
  cudaFuncSetAttribute(k_zk<LZH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Z::SMEM);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(g.py / kZCols, g.hx);
  cfg.blockDim = dim3(kZNT);
  cfg.dynamicSmemBytes = Z::SMEM;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k_zk<LZH>, g, T, ktf, tw, st);
}

void launch_y(const Geom& g, const Buffers& b, float2* T, bool forward, cudaStream_t s) {
  const float2* in = b.spec;
  switch (g.py / 2) {
    case 16: run_y<16>(g, in, T, b.spec, b.tw, b.st, s, forward); break;
    case 32: run_y<32>(g, in, T, b.spec, b.tw, b.st, s, forward); break;
    case 64: run_y3<64>(g, b, T, forward, s); break;
    case 128: run_y3<128>(g, b, T, forward, s); break;
    case 256: run_y3<256>(g, b, T, forward, s); break;
    case 512: run_y<512>(g, in, T, b.spec, b.tw, b.st, s, forward); break;
    default: break;
  }
}

}  // namespace

// The one-kernel 2-D plan: a fused spectrum layout of a single layer with an
// open y axis padded to 128, 256 or 512 points.
bool y2d_plan(const Geom& g) {
  return g.fused && g.pz == 1 && g.nz == 1 && g.pbcy == 0 && (g.py == 128 || g.py == 256 || g.py == 512);
}

void launch_demag_y2d(const Geom& g, const Buffers& b, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(g.hx);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  switch (g.py) {
    case 128:
      cfg.blockDim = dim3(Y2dCfg<64>::NT);
      cudaLaunchKernelEx(&cfg, k_y2d<64>, g, b.spec, (const float*)b.ktf, (const float2*)b.tw, (const DevState*)b.st);
      break;
    case 256:
      cfg.blockDim = dim3(Y2dCfg<128>::NT);
      cudaLaunchKernelEx(&cfg, k_y2d<128>, g, b.spec, (const float*)b.ktf, (const float2*)b.tw, (const DevState*)b.st);
      break;
    case 512:
      cfg.blockDim = dim3(Y2dCfg<256>::NT);
      cudaLaunchKernelEx(&cfg, k_y2d<256>, g, b.spec, (const float*)b.ktf, (const float2*)b.tw, (const DevState*)b.st);
      break;
    default: break;
  }
}

// The three-kernel plan: a fused spectrum layout, open (padded) y and z axes
// with 32 <= py <= 1024 and 16 <= pz <= 64 (z classes of 8, 16 or 32 points).
bool yz3_plan(const Geom& g) {
  return g.fused && g.pbcy == 0 && g.pbcz == 0 && g.py >= 32 && g.py <= 1024 && g.pz >= 16 && g.pz <= 64;
}

size_t yz3_bytes(const Geom& g) { return sizeof(float2) * (size_t)g.hx * 3 * g.nz * g.py; }

void launch_yz3_part(const Geom& g, const Buffers& b, float2* T, int part, cudaStream_t s) {
  if (part == 0) {
    launch_y(g, b, T, true, s);
  } else if (part == 1) {
    switch (g.pz / 2) {
      case 8: run_z<8>(g, T, b.ktf, b.tw, b.st, s); break;
      case 16: run_z<16>(g, T, b.ktf, b.tw, b.st, s); break;
      case 32: run_z<32>(g, T, b.ktf, b.tw, b.st, s); break;
      default: break;
    }
  } else {
    launch_y(g, b, T, false, s);
  }
}

void launch_demag_yz3(const Geom& g, const Buffers& b, float2* T, cudaStream_t s) {
  for (int part = 0; part < 3; ++part) launch_yz3_part(g, b, T, part, s);
}

}  // namespace mm
