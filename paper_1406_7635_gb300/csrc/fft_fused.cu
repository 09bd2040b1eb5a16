// Fused demag convolution for grids whose padded (y, z) plane is small
// enough: three kernels per convolution instead of five, every global access
// contiguous, and the zero-padded half of the spectrum never materialised.
//
//   k_fx_t  x rows: real M -> half spectrum (as k_fx), written transposed to
//           spec[c][kx][z][y] (y fastest) so one kx plane is contiguous;
//   k_yz    one kx plane per thread-block cluster: y and z transforms, the
//           kernel multiply and the inverse transforms;
//   k_ix_t  x rows back to real B (as k_ix), reading the transposed layout.
//
// k_yz splits the padded (py x pz) transform by frequency residue class:
// with ky = CLY j + ry and kz = CLZ l + rz, the padded DFT restricted to one
// class is an unpadded (py/CLY x pz/CLZ) DFT of the input multiplied by
// exp(-2 pi i (y ry / py + z rz / pz)) (valid because ny <= py/CLY and
// nz <= pz/CLZ, so no folding is needed).  Each block of a cluster of
// CLY*CLZ blocks owns one class: it twiddles the input, transforms it,
// multiplies by the kernel at its (kx, ky, kz), transforms back, undoes the
// twiddle, and the cluster sums the CLY*CLZ contributions through
// distributed shared memory.
#include <cooperative_groups.h>

#include "fft.cuh"
#include "mm_internal.h"

namespace cg = cooperative_groups;

namespace mm {
namespace {
using namespace mmfft;

__device__ __forceinline__ float cell_msat_f(const RegionLUT* __restrict__ lut, const uint8_t* __restrict__ mask,
                                             const uint8_t* __restrict__ region, int i) {
  return mask[i] ? __ldg(&lut->msat[region[i]]) : 0.0f;
}

// offset in one instance's spectrum (3 hx nz ny < 2^31 points: nz <= 32)
__device__ __forceinline__ int tidx(const Geom& g, int c, int kx, int z, int y) {
  return ((c * g.hx + kx) * g.nz + z) * g.ny + y;
}

// ----------------------------------------------------------------------------
// x rows, transposed spectrum
// ----------------------------------------------------------------------------
// Batches: blockIdx.z = 3 * instance + component; instance i reads m + 3 n i,
// writes spec + 3 hx nz ny i, takes Msat from inst_msat[i] (all cells
// magnetic) when inst_msat is given, and is skipped once inst_done[i] is set.
template <int L, int ROWS, int NT>
__global__ void __launch_bounds__(NT) k_fx_t(Geom g, const float* __restrict__ m, const uint8_t* __restrict__ mask,
                                             const uint8_t* __restrict__ region, const RegionLUT* __restrict__ lut,
                                             float2* __restrict__ spec, const float2* __restrict__ tw,
                                             const DevState* __restrict__ st, BatchArgs ba) {
  if (st && st->done) return;
  const int inst = blockIdx.z / 3;
  if (ba.done && ba.done[(long long)inst * ba.done_stride]) return;
  m += (long long)inst * 3 * g.n;
  spec += (long long)inst * 3 * g.hx * g.nz * g.ny;
  const float inst_ms = ba.msat ? ba.msat[inst] : 0.0f;
  constexpr int PST = L + 1;
  __shared__ float2 s[ROWS * PST];
  __shared__ float2 twl[L], tw2[L + 1];   // W_L^i and W_2L^k
  const int y0 = blockIdx.x * ROWS, z = blockIdx.y, c = blockIdx.z % 3;
  twiddles_async<NT>(twl, tw, L, kTwN / L);
  twiddles_async<NT>(tw2, tw, L + 1, kTwN / (2 * L));
  const bool even = (g.nx & 1) == 0;
  const int nin = (g.nx + 1) / 2;   // complex inputs n >= nin are zero padding (not stored, not read)
  const float* __restrict__ mc = m + c * (int)g.n;   // this component (3 n < 2^31)
  for (int e = threadIdx.x; e < ROWS * L; e += NT) {
    const int r = e / L, n = e % L, y = y0 + r;
    float2 v = make_float2(0.f, 0.f);
    if (y < g.ny) {
      const int cell0 = (z * g.ny + y) * g.nx;
      const int x0 = 2 * n, x1 = 2 * n + 1;
      if (ba.msat) {
        if (x0 < g.nx) v.x = inst_ms * mc[cell0 + x0];
        if (x1 < g.nx) v.y = inst_ms * mc[cell0 + x1];
      } else if (even && x1 < g.nx) {
        // cell0 + x0 is even: aligned pair loads
        const float2 mv = *reinterpret_cast<const float2*>(mc + cell0 + x0);
        const uchar2 mk = *reinterpret_cast<const uchar2*>(mask + cell0 + x0);
        const uchar2 rg = *reinterpret_cast<const uchar2*>(region + cell0 + x0);
        v.x = mk.x ? __ldg(&lut->msat[rg.x]) * mv.x : 0.f;
        v.y = mk.y ? __ldg(&lut->msat[rg.y]) * mv.y : 0.f;
      } else {
        if (x0 < g.nx) v.x = cell_msat_f(lut, mask, region, cell0 + x0) * mc[cell0 + x0];
        if (x1 < g.nx) v.y = cell_msat_f(lut, mask, region, cell0 + x1) * mc[cell0 + x1];
      }
    }
    if (n < nin) s[r * PST + n] = v;
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  __syncthreads();
  FftG<L, -1, ROWS, NT, 1, PST, 1, L>::run(s, twl, nullptr, nin);
  // X_k = E_k + W_P^k O_k; store with consecutive threads on consecutive y
  for (int e = threadIdx.x; e < ROWS * (L + 1); e += NT) {
    const int r = e % ROWS, k = e / ROWS, y = y0 + r;
    if (y >= g.ny) continue;
    const float2 zk = s[r * PST + (k & (L - 1))];
    const float2 zc = cconj(s[r * PST + ((L - k) & (L - 1))]);
    const float2 E = cscale(cadd(zk, zc), 0.5f);
    const float2 d = csub(zk, zc);
    const float2 O = make_float2(0.5f * d.y, -0.5f * d.x);
    spec[tidx(g, c, k, z, y)] = cadd(E, cmul(tw2[k], O));
  }
}

template <int L, int ROWS, int NT>
__global__ void __launch_bounds__(NT) k_ix_t(Geom g, const float2* __restrict__ spec, float* __restrict__ out,
                                             const float2* __restrict__ tw, const DevState* __restrict__ st,
                                             BatchArgs ba) {
  if (st && st->done) return;
  const int inst = blockIdx.z / 3;
  if (ba.done && ba.done[(long long)inst * ba.done_stride]) return;
  out += (long long)inst * 3 * g.n;
  spec += (long long)inst * 3 * g.hx * g.nz * g.ny;
  constexpr int PST = L + 1;
  __shared__ float2 s[ROWS * PST];
  __shared__ float2 twl[L], tw2[L + 1];   // W_L^i and W_2L^k
  const int y0 = blockIdx.x * ROWS, z = blockIdx.y, c = blockIdx.z % 3;
  twiddles_async<NT>(twl, tw, L, kTwN / L);
  twiddles_async<NT>(tw2, tw, L + 1, kTwN / (2 * L));
  grid_dependency_wait();   // the spectrum comes from the y/z kernel
  for (int e = threadIdx.x; e < ROWS * (L + 1); e += NT) {
    const int r = e % ROWS, k = e / ROWS, y = y0 + r;
    if (y < g.ny) cp_async_f2(&s[r * PST + k], spec + tidx(g, c, k, z, y));
    else s[r * PST + k] = make_float2(0.f, 0.f);
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  __syncthreads();
  for (int e = threadIdx.x; e < ROWS * (L / 2 + 1); e += NT) {
    const int r = e / (L / 2 + 1), k = e % (L / 2 + 1);
    const float2 xa = s[r * PST + k], xb = s[r * PST + L - k];
    float2 za, zb;
    {
      const float2 E = cscale(cadd(xa, cconj(xb)), 0.5f);
      const float2 w = cconj(tw2[k]);
      const float2 O = cmul(cscale(csub(xa, cconj(xb)), 0.5f), w);
      za = make_float2(E.x - O.y, E.y + O.x);
    }
    {
      const int kb = L - k;
      const float2 E = cscale(cadd(xb, cconj(xa)), 0.5f);
      const float2 w = cconj(tw2[kb]);
      const float2 O = cmul(cscale(csub(xb, cconj(xa)), 0.5f), w);
      zb = make_float2(E.x - O.y, E.y + O.x);
    }
    s[r * PST + k] = za;
    if (k != 0 && k != L / 2) s[r * PST + L - k] = zb;
  }
  __syncthreads();
  FftG<L, 1, ROWS, NT, 1, PST, 1, L>::run(s, twl, nullptr, L, (g.nx + 1) / 2);   // outputs 2n >= nx cropped
  float* __restrict__ oc = out + c * (int)g.n;
  for (int e = threadIdx.x; e < ROWS * L; e += NT) {
    const int r = e / L, n = e % L, y = y0 + r;
    if (y >= g.ny) continue;
    const int cell0 = (z * g.ny + y) * g.nx;
    const float2 v = s[r * PST + n];
    if ((g.nx & 1) == 0 && 2 * n + 1 < g.nx) {
      *reinterpret_cast<float2*>(oc + cell0 + 2 * n) = v;
    } else {
      if (2 * n < g.nx) oc[cell0 + 2 * n] = v.x;
      if (2 * n + 1 < g.nx) oc[cell0 + 2 * n + 1] = v.y;
    }
  }
}

// Kernel multiply at the points (j, l) of columns j0 .. j0 + YW - 1 of the
// plane (NTH threads, thread index tid): frequency (ky, kz) = (CLY j + ry,
// CLZ l + rz); ktf holds the octant per kx plane, ky fastest
// (ktf[kx][c][iz][iy]); mirror signs: Nxy odd in y, Nxz odd in z, Nyz odd in
// both.  The coefficient loads of CH points are issued together.
template <int LY, int LZ, int RP, int CS, int YW, int NTH, int CHMAX>
__device__ __forceinline__ void kernel_mul(float2* s, const float* __restrict__ kt, const Geom& g, int kx, int ry,
                                           int rz, int j0, int tid) {
  constexpr int PW = YW * LZ;
  constexpr int PPT = (PW + NTH - 1) / NTH;   // points per thread
  constexpr int CH = PPT < CHMAX ? PPT : CHMAX;
  const int per = g.hky * g.hkz;   // octant: 6 hkx hky hkz < 2^31 floats
#pragma unroll
  for (int q0 = 0; q0 < PPT; q0 += CH) {
    float kc[CH][6];
    float sgn[CH][2];
#pragma unroll
    for (int q = 0; q < CH; ++q) {
      const int e = tid + (q0 + q) * NTH;
      if (e >= PW) continue;
      const int j = j0 + e % YW, l = e / YW;
      const int ky = g.cly * j + ry, kz = g.clz * l + rz;
      int iy = ky, iz = kz;
      float sy = 1.f, sz = 1.f;
      if (ky > g.py / 2) { iy = g.py - ky; sy = -1.f; }
      if (kz > g.pz / 2) { iz = g.pz - kz; sz = -1.f; }
      const int o = kx * 6 * per + iz * g.hky + iy;
#pragma unroll
      for (int t = 0; t < 6; ++t) kc[q][t] = __ldg(&kt[t * per + o]);
      sgn[q][0] = sy;
      sgn[q][1] = sz;
    }
#pragma unroll
    for (int q = 0; q < CH; ++q) {
      const int e = tid + (q0 + q) * NTH;
      if (e >= PW) continue;
      const int j = j0 + e % YW, l = e / YW;
      const int a = l * RP + j;
      const float kxx = kc[q][0], kyy = kc[q][1], kzz = kc[q][2];
      const float kxy = sgn[q][0] * kc[q][3], kxz = sgn[q][1] * kc[q][4], kyz = sgn[q][0] * sgn[q][1] * kc[q][5];
      const float2 X = s[a], Y = s[CS + a], Z = s[2 * CS + a];
      s[a] = make_float2(kxx * X.x + kxy * Y.x + kxz * Z.x, kxx * X.y + kxy * Y.y + kxz * Z.y);
      s[CS + a] = make_float2(kxy * X.x + kyy * Y.x + kyz * Z.x, kxy * X.y + kyy * Y.y + kyz * Z.y);
      s[2 * CS + a] = make_float2(kxz * X.x + kyz * Y.x + kzz * Z.x, kxz * X.y + kyz * Y.y + kzz * Z.y);
    }
  }
}

// radix of the last forward / first inverse z pass in z_mid (4 at most, so
// that three components and their kernel coefficients fit in registers)
__host__ __device__ constexpr int zmid_radix(int lz) { return lz >= 4 ? 4 : lz; }

// split cluster barrier: arrive without memory ordering, and the wait
__device__ __forceinline__ void cluster_arrive_relaxed() {
  asm volatile("barrier.cluster.arrive.relaxed.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.aligned;\n" ::: "memory"); }

// The middle of the z transforms of all three components, fused (LZ =
// R0 R1 with R1 = zmid_radix(LZ) the radix of the last forward pass, R0 = 1
// for one pass):
// for butterfly j of column p it runs the last forward pass on the R1
// values at z = j + R0 r, multiplies the three components by the kernel at
// those R1 frequencies and runs the first inverse pass (radix R1, no
// twiddle), writing back to the positions it read -- so butterflies never
// touch each other's data and need no barrier.  The standard first inverse
// pass would store output r of butterfly j at j R1 + r; z_inv_tail reads
// that transposed order.
template <int LY, int LZ, int NT, int RP, int CS>
__device__ __forceinline__ void z_mid(float2* s, const float2* __restrict__ twz, const float2* __restrict__ rtz,
                                      const float* __restrict__ kt, const Geom& g, int kx, int ry, int rz) {
  constexpr int R1 = zmid_radix(LZ);
  constexpr int R0 = LZ / R1;
  constexpr int TOT = R0 * LY;
  constexpr int PER = (TOT + NT - 1) / NT;
  const int per = g.hky * g.hkz;   // octant: 6 hkx hky hkz < 2^31 floats
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int b = threadIdx.x + q * NT;
    if (TOT % NT != 0 && b >= TOT) continue;
    const int p = b % LY, j = b / LY;
    const int ky = g.cly * p + ry;
    int iy = ky;
    float sy = 1.f;
    if (ky > g.py / 2) { iy = g.py - ky; sy = -1.f; }
    float kc[R1][6], sz[R1];
#pragma unroll
    for (int r = 0; r < R1; ++r) {
      const int kz = g.clz * (j + R0 * r) + rz;
      int iz = kz;
      sz[r] = 1.f;
      if (kz > g.pz / 2) { iz = g.pz - kz; sz[r] = -1.f; }
      const int o = kx * 6 * per + iz * g.hky + iy;
#pragma unroll
      for (int t = 0; t < 6; ++t) kc[r][t] = __ldg(&kt[t * per + o]);
    }
    float2 v[3][R1];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int r = 0; r < R1; ++r) v[c][r] = s[c * CS + (j + R0 * r) * RP + p];
    if (R0 == 1) {
      if (rz) {
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int r = 0; r < R1; ++r) v[c][r] = cmul(v[c][r], rtz[r]);
      }
    } else {
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int r = 1; r < R1; ++r) v[c][r] = cmul(v[c][r], twz[(r * j) & (LZ - 1)]);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) Dft<R1, -1>::run(v[c]);
#pragma unroll
    for (int r = 0; r < R1; ++r) {
      const float kxx = kc[r][0], kyy = kc[r][1], kzz = kc[r][2];
      const float kxy = sy * kc[r][3], kxz = sz[r] * kc[r][4], kyz = sy * sz[r] * kc[r][5];
      const float2 X = v[0][r], Y = v[1][r], Z = v[2][r];
      v[0][r] = make_float2(kxx * X.x + kxy * Y.x + kxz * Z.x, kxx * X.y + kxy * Y.y + kxz * Z.y);
      v[1][r] = make_float2(kxy * X.x + kyy * Y.x + kyz * Z.x, kxy * X.y + kyy * Y.y + kyz * Z.y);
      v[2][r] = make_float2(kxz * X.x + kyz * Y.x + kzz * Z.x, kxz * X.y + kyz * Y.y + kzz * Z.y);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) Dft<R1, 1>::run(v[c]);
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int r = 0; r < R1; ++r) s[c * CS + (j + R0 * r) * RP + p] = v[c][r];
  }
}

// Second (last) inverse z pass after z_mid, for NC consecutive components
// (component stride CS): radix R0, butterfly j2 < R1 reads element r2 at the
// transposed position r2 + R0 j2 and writes the natural order j2 + R1 r2.
// Ends with __syncthreads().
template <int LY, int LZ, int NT, int RP, int CS, int NC>
__device__ __forceinline__ void z_inv_tail(float2* sc, const float2* __restrict__ twz) {
  constexpr int R1 = zmid_radix(LZ);
  constexpr int R0 = LZ / R1;
  if constexpr (R0 > 1) {
    constexpr int TOT = R1 * LY * NC;
    constexpr int PER = (TOT + NT - 1) / NT;
    float2 v[PER][R0];
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int b = threadIdx.x + q * NT;
      if (TOT % NT == 0 || b < TOT) {
        const int p = b % LY, cc = (b / LY) % NC, j2 = b / (LY * NC);
#pragma unroll
        for (int r = 0; r < R0; ++r) v[q][r] = sc[cc * CS + (r + R0 * j2) * RP + p];
      }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int b = threadIdx.x + q * NT;
      if (TOT % NT == 0 || b < TOT) {
        const int p = b % LY, cc = (b / LY) % NC, j2 = b / (LY * NC);
#pragma unroll
        for (int r = 1; r < R0; ++r) v[q][r] = cmul(v[q][r], cconj(twz[(r * j2) & (LZ - 1)]));
        Dft<R0, 1>::run(v[q]);
#pragma unroll
        for (int r = 0; r < R0; ++r) sc[cc * CS + (j2 + R1 * r) * RP + p] = v[q][r];
      }
    }
  }
  __syncthreads();
}

// ----------------------------------------------------------------------------
// k_yz: plane [3][LZ][LY] in shared memory, y fastest, rows padded to an
// odd pitch RP = LY + 1 (conflict-free row and column transforms)
// ----------------------------------------------------------------------------
template <int LY, int LZ, int NT>
__global__ void __launch_bounds__(NT, 2) k_yz(Geom g, float2* __restrict__ spec, const float* __restrict__ kt,
                                           const float2* __restrict__ tw, const DevState* __restrict__ st,
                                           BatchArgs ba) {
  // blocks of one cluster share (instance, kx), so these exits are uniform
  // across the cluster: all its blocks leave together (the device state's
  // done flag is read after the predecessor has completed, see below)
  const int inst = blockIdx.x / (g.hx * g.cly * g.clz);
  if (ba.done && ba.done[(long long)inst * ba.done_stride]) return;
  spec += (long long)inst * 3 * g.hx * g.nz * g.ny;
  extern __shared__ float2 s[];
  constexpr int RP = LY + 1;
  constexpr int PL = LY * LZ;   // points per component
  constexpr int CS = LZ * RP;   // component stride in shared memory
  // twiddle tables after the plane: W_LY^i, W_LZ^i, and the residue twiddles
  // W_py^y (y < LY), W_pz^z (z < LZ)
  float2* twy = s + 3 * CS;
  float2* twz = twy + LY;
  float2* rty = twz + LZ;
  float2* rtz = rty + LY;
  // (asynchronous copies, completed with the plane's)
  twiddles_async<NT>(twy, tw, LY, kTwN / LY);
  twiddles_async<NT>(twz, tw, LZ, kTwN / LZ);
  twiddles_async<NT>(rty, tw, LY, kTwN / g.py);
  twiddles_async<NT>(rtz, tw, LZ, kTwN / g.pz);
  const int CL = g.cly * g.clz;
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = CL > 1 ? (int)cluster.block_rank() : 0;
  const int ry = rank % g.cly, rz = rank / g.cly;
  const int kx = (blockIdx.x / CL) % g.hx;
  // the spectrum comes from the previous kernel (programmatic dependent
  // launch: wait for it, then let the next kernel's blocks be scheduled)
  grid_dependency_wait();
  // (a row kernel that gave up a wait sets the done flag while it runs: read
  // it once the predecessor has completed, so every block sees one value;
  // the twiddle copies land before the block leaves)
  if (st && st->done) {
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    return;
  }
  // 1. load the plane (asynchronous copies, all in flight at once); rows
  //    past the grid are zero; columns y >= ny are never read (the first y
  //    pass is pruned to y < ny)
  // (32-bit offsets: one instance's spectrum, 3 hx nz ny < 2^31 points)
  const int cstride = g.hx * g.nz * g.ny;              // component stride of spec
  float2* const plane = spec + kx * g.nz * g.ny;       // this kx plane, component 0
  for (int e = threadIdx.x; e < 3 * PL; e += NT) {
    const int y = e % LY, z = (e / LY) % LZ, c = e / PL;
    if (y >= g.ny) continue;
    float2* dst = s + c * CS + z * RP + y;
    if (z < g.nz) {
      const unsigned saddr = (unsigned)__cvta_generic_to_shared(dst);
      asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(saddr),
                   "l"(plane + c * cstride + z * g.ny + y));
    } else {
      *dst = make_float2(0.f, 0.f);
    }
  }
  asm volatile("cp.async.wait_all;\n" ::);
  __syncthreads();
  // 2. forward transforms along y (LZ rows) and the first z pass (LY
  //    columns), one component at a time; the class twiddle exp(-2 pi i
  //    (y ry / py + z rz / pz)) is applied as the first pass loads its inputs
  if constexpr (LZ > 1) {
    constexpr int R0 = LZ / zmid_radix(LZ);
    // (the three components' rows are one array of 3 LZ rows at pitch RP:
    // components 0 and 1 are transformed together, then component 2)
    FftG<LY, -1, 2 * LZ, NT, 1, RP, 1, LY>::run(s, twy, ry ? rty : nullptr, g.ny);
    FftG<LY, -1, LZ, NT, 1, RP, 1, LY>::run(s + 2 * CS, twy, ry ? rty : nullptr, g.ny);
    if constexpr (R0 > 1) {
      stockham_pass<LZ, R0, 1, -1, 2 * LY, NT, LY, CS, RP, LZ>(s, twz, rz ? rtz : nullptr);
      stockham_pass<LZ, R0, 1, -1, LY, NT, LY, CS, RP, LZ>(s + 2 * CS, twz, rz ? rtz : nullptr);
    }
    // 3. last forward z pass, kernel multiply at (kx, ky = CLY j + ry,
    //    kz = CLZ l + rz), first inverse z pass, all in registers
    z_mid<LY, LZ, NT, RP, CS>(s, twz, rtz, kt, g, kx, ry, rz);
    __syncthreads();
    // 4. rest of the inverse transforms
    z_inv_tail<LY, LZ, NT, RP, CS, 2>(s, twz);
    z_inv_tail<LY, LZ, NT, RP, CS, 1>(s + 2 * CS, twz);
    // (outputs y >= ny are cropped: never stored nor read by the class sum)
    FftG<LY, 1, 2 * LZ, NT, 1, RP, 1, LY>::run(s, twy, nullptr, LY, g.ny);
    FftG<LY, 1, LZ, NT, 1, RP, 1, LY>::run(s + 2 * CS, twy, nullptr, LY, g.ny);
  } else {
    // 2-D: the three components are three rows at pitch RP, transformed together
    FftG<LY, -1, 3, NT, 1, RP, 1, LY>::run(s, twy, ry ? rty : nullptr, g.ny);
    kernel_mul<LY, LZ, RP, CS, LY, NT, 2>(s, kt, g, kx, ry, rz, 0, threadIdx.x);
    __syncthreads();
    FftG<LY, 1, 3, NT, 1, RP, 1, LY>::run(s, twy, nullptr, LY, g.ny);
  }
  // 5. sum the class contributions across the cluster, each multiplied by
  //    the conjugate of its class twiddle; each block stores one contiguous
  //    1/CL share of the plane
  if (CL > 1) cluster.sync();
  else __syncthreads();
  // output points o = (c LZ + z) LY + y of the padded class plane (points
  // with z >= nz or y >= ny are skipped); each block takes 1/CL of them
  constexpr int NOUT = 3 * PL;
  const int chunk = (NOUT + CL - 1) / CL;
  const int o_end = min(NOUT, (rank + 1) * chunk);
  // the (at most 4) blocks' planes; a batch of RB points per thread issues
  // all its distributed-shared-memory loads before combining them
  const float2* part[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) part[q] = (q < CL && q != rank) ? cluster.map_shared_rank(s, q) : s;
  constexpr int RB = 3;
  for (int ob = rank * chunk + threadIdx.x; ob < o_end; ob += RB * NT) {
    float2 val[RB][4];
#pragma unroll
    for (int u = 0; u < RB; ++u) {
      const int o = ob + u * NT;
      const int y = o % LY, z = (o / LY) % LZ, c = o / PL;
      if (o >= o_end || y >= g.ny || z >= g.nz) continue;
      const int e = c * CS + z * RP + y;
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (q < CL) val[u][q] = part[q][e];
    }
#pragma unroll
    for (int u = 0; u < RB; ++u) {
      const int o = ob + u * NT;
      const int y = o % LY, z = (o / LY) % LZ, c = o / PL;
      if (o >= o_end || y >= g.ny || z >= g.nz) continue;
      const float2 ty = cconj(rty[y]), tz = cconj(rtz[z]), tyz = cmul(ty, tz);
      float2 v = val[u][0];   // class (0, 0): no twiddle
#pragma unroll
      for (int q = 1; q < 4; ++q) {
        if (q >= CL) continue;
        const int qy = q % g.cly, qz = q / g.cly;
        const float2 w = qy ? (qz ? tyz : ty) : tz;
        v = cadd(v, cmul(val[u][q], w));
      }
      plane[c * cstride + z * g.ny + y] = v;
    }
  }
  if (CL > 1) cluster.sync();   // keep shared memory alive until every peer has read it
}

// k_yz for clusters split in z (clz = 2): the y transform commutes with the
// z-class twiddle (a per-row factor), so the two blocks of a z-class pair
// (same ry) share it.  Each block loads and y-transforms one half of the z
// rows (its half h = rz) and stores it into its partner's shared memory
// (distributed shared memory), which receives the other half the same way;
// after the inverse z pass each block sums the pair's
// two classes (conjugate z twiddle) for its half of the rows, so the inverse
// y transform also runs on half the rows.  The last step adds the y classes
// (cly = 2) as before.  Same shared-memory layout as k_yz.
template <int LY, int LZ, int NT>
__global__ void __launch_bounds__(NT, 2) k_yz2(Geom g, float2* __restrict__ spec, const float* __restrict__ kt,
                                            const float2* __restrict__ tw, const DevState* __restrict__ st,
                                            BatchArgs ba) {
  const int inst = blockIdx.x / (g.hx * g.cly * 2);
  if (ba.done && ba.done[(long long)inst * ba.done_stride]) return;
  spec += (long long)inst * 3 * g.hx * g.nz * g.ny;
  extern __shared__ float2 s[];
  constexpr int RP = LY + 1;
  constexpr int CS = LZ * RP;
  constexpr int H = LZ / 2;          // rows per z half
  constexpr int PH = LY * H;         // points of one component's half
  float2* twy = s + 3 * CS;
  float2* twz = twy + LY;
  float2* rty = twz + LZ;
  float2* rtz = rty + LY;
  // (asynchronous copies, completed with the plane's)
  twiddles_async<NT>(twy, tw, LY, kTwN / LY);
  twiddles_async<NT>(twz, tw, LZ, kTwN / LZ);
  twiddles_async<NT>(rty, tw, LY, kTwN / g.py);
  twiddles_async<NT>(rtz, tw, LZ, kTwN / g.pz);
  const int CL = g.cly * 2;
  cg::cluster_group cluster = cg::this_cluster();
  cluster_arrive_relaxed();   // "started": awaited before the first remote store
  const int rank = (int)cluster.block_rank();
  const int ry = rank % g.cly, rz = rank / g.cly;
  const int zpart = ry + g.cly * (1 - rz);   // same ry, other z class
  const int kx = (blockIdx.x / CL) % g.hx;
  const int h0 = rz * H;                     // first row of my half
  const int cstride = g.hx * g.nz * g.ny;
  float2* const plane = spec + kx * g.nz * g.ny;
  grid_dependency_wait();   // the spectrum comes from the previous kernel
  // the done flag, read once the predecessor has completed: uniform across
  // the cluster (same instance and kx); the twiddle copies land and the
  // cluster's arrive is matched before the blocks leave
  if (st && st->done) {
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    cluster_wait();
    return;
  }
  // 1. load my half of the rows (columns y >= ny are never read: the first
  //    y pass is pruned to y < ny)
  for (int e = threadIdx.x; e < 3 * PH; e += NT) {
    const int y = e % LY, i = (e / LY) % H, c = e / PH, z = h0 + i;
    if (y >= g.ny) continue;
    float2* dst = s + c * CS + z * RP + y;
    if (z < g.nz) {
      const unsigned saddr = (unsigned)__cvta_generic_to_shared(dst);
      asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(saddr),
                   "l"(plane + c * cstride + z * g.ny + y));
    } else {
      *dst = make_float2(0.f, 0.f);
    }
  }
  asm volatile("cp.async.wait_all;\n" ::);
  __syncthreads();
  // 2. forward y on my half of the rows of all three components (pencil q:
  //    component q / H, row h0 + q % H), y-class twiddle on load
  FftG<LY, -1, 3 * H, NT, H, CS, 1, LY, RP>::run(s + h0 * RP, twy, ry ? rty : nullptr, g.ny);
  // 3. my half into the partner's rows at the same positions, which the
  //    partner neither loaded nor transformed (remote stores, no round trip)
  cluster_wait();
  {
    float2* pd = cluster.map_shared_rank(s, zpart);
    constexpr int NB = 3 * PH;
#pragma unroll 4
    for (int e = threadIdx.x; e < NB; e += NT) {
      const int y = e % LY, i = (e / LY) % H, c = e / PH;
      const int a = c * CS + (h0 + i) * RP + y;
      pd[a] = s[a];
    }
  }
  cluster.sync();   // the pushed rows are complete before anyone transforms in z
  // 4. z: first pass (z-class twiddle on load), fused middle, last inverse pass
  constexpr int R0 = LZ / zmid_radix(LZ);
  if constexpr (R0 > 1) {
    stockham_pass<LZ, R0, 1, -1, 2 * LY, NT, LY, CS, RP, LZ>(s, twz, rz ? rtz : nullptr);
    stockham_pass<LZ, R0, 1, -1, LY, NT, LY, CS, RP, LZ>(s + 2 * CS, twz, rz ? rtz : nullptr);
  }
  z_mid<LY, LZ, NT, RP, CS>(s, twz, rtz, kt, g, kx, ry, rz);
  __syncthreads();
  z_inv_tail<LY, LZ, NT, RP, CS, 2>(s, twz);
  z_inv_tail<LY, LZ, NT, RP, CS, 1>(s + 2 * CS, twz);
  // 5. my half of the rows: sum of the pair's two z classes (conjugate z
  //    twiddle; class 0 has none), in place
  cluster.sync();
  {
    const float2* ps = cluster.map_shared_rank(s, zpart);
    constexpr int NB = 3 * PH;
    constexpr int PER = (NB + NT - 1) / NT;
    float2 v[PER];
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int e = threadIdx.x + q * NT;
      if (NB % NT == 0 || e < NB) {
        const int y = e % LY, i = (e / LY) % H, c = e / PH;
        v[q] = ps[c * CS + (h0 + i) * RP + y];
      }
    }
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int e = threadIdx.x + q * NT;
      if (NB % NT == 0 || e < NB) {
        const int y = e % LY, i = (e / LY) % H, c = e / PH, z = h0 + i;
        const int a = c * CS + z * RP + y;
        const float2 w = cconj(rtz[z]);   // the z class 1 twiddle at row z
        s[a] = rz ? cadd(cmul(s[a], w), v[q]) : cadd(s[a], cmul(v[q], w));
      }
    }
  }
  __syncthreads();
  // 6. inverse y on my half of the rows
  FftG<LY, 1, 3 * H, NT, H, CS, 1, LY, RP>::run(s + h0 * RP, twy, nullptr, LY, g.ny);   // y >= ny cropped
  // 7. sum over the y classes (cly = 2: the block with the other ry and the
  //    same half) and store; with cly = 2 each block stores half of its rows
  if (g.cly > 1) cluster.sync();
  {
    const float2* yp = g.cly > 1 ? cluster.map_shared_rank(s, (1 - ry) + g.cly * rz) : s;
    const int n_rows = g.cly > 1 ? H / 2 : H;           // rows of my half that I store
    const int r0 = h0 + (g.cly > 1 ? ry * (H / 2) : 0);
    const int nb = 3 * n_rows * LY;
    for (int e = threadIdx.x; e < nb; e += NT) {
      const int y = e % LY, i = (e / LY) % n_rows, c = e / (LY * n_rows), z = r0 + i;
      if (y >= g.ny || z >= g.nz) continue;
      const int a = c * CS + z * RP + y;
      float2 v = s[a];
      if (g.cly > 1) {
        const float2 o = yp[a];
        const float2 w = cconj(rty[y]);   // the y class 1 twiddle
        v = ry ? cadd(cmul(v, w), o) : cadd(v, cmul(o, w));
      }
      plane[c * cstride + z * g.ny + y] = v;
    }
  }
  // keep shared memory alive until every peer has read it (the reads have
  // been consumed before each peer arrives, so no memory ordering is needed)
  cluster_arrive_relaxed();
  cluster_wait();
}

// rows per block of the x-row kernels: the default rule (enough blocks to
// fill the GPU: 8 rows of <= 128 points), or half / twice it
template <int L>
struct RowCfgT {
  static constexpr int ROWS = L >= 512 ? 2 : (L >= 256 ? 4 : 8);
  static constexpr int RH = ROWS > 1 ? ROWS / 2 : 1;
  static constexpr int R2 = 2 * ROWS;
};
template <int L, int ROWS>
struct RowNT {
  static constexpr int NT = ROWS * L / 8 < 64 ? 64 : ROWS * L / 8;
};

template <int L, int ROWS>
void run_fx_rows(const Geom& g, const Buffers& b, const float* m, cudaStream_t s, const BatchArgs& ba) {
  constexpr int NT = RowNT<L, ROWS>::NT;
  dim3 grid((g.ny + ROWS - 1) / ROWS, g.nz, 3 * ba.count);
  k_fx_t<L, ROWS, NT><<<grid, NT, 0, s>>>(g, m, b.mask, b.region, b.lut, b.spec, b.tw, b.st, ba);
}
template <int L, int ROWS>
void run_ix_rows(const Geom& g, const Buffers& b, cudaStream_t s, const BatchArgs& ba) {
  constexpr int NT = RowNT<L, ROWS>::NT;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((g.ny + ROWS - 1) / ROWS, g.nz, 3 * ba.count);
  cfg.blockDim = dim3(NT);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k_ix_t<L, ROWS, NT>, g, (const float2*)b.spec, b.bd, (const float2*)b.tw,
                     (const DevState*)b.st, ba);
}
template <int L>
void run_fx_t(const Geom& g, const Buffers& b, const float* m, cudaStream_t s, const BatchArgs& ba) {
  using C = RowCfgT<L>;
  if (g.xrows == C::RH && C::RH != C::ROWS) run_fx_rows<L, C::RH>(g, b, m, s, ba);
  else if (g.xrows == C::R2) run_fx_rows<L, C::R2>(g, b, m, s, ba);
  else run_fx_rows<L, C::ROWS>(g, b, m, s, ba);
}
template <int L>
void run_ix_t(const Geom& g, const Buffers& b, cudaStream_t s, const BatchArgs& ba) {
  using C = RowCfgT<L>;
  if (g.xrows == C::RH && C::RH != C::ROWS) run_ix_rows<L, C::RH>(g, b, s, ba);
  else if (g.xrows == C::R2) run_ix_rows<L, C::R2>(g, b, s, ba);
  else run_ix_rows<L, C::ROWS>(g, b, s, ba);
}
template <int L>
int xrow_options(int* out) {
  using C = RowCfgT<L>;
  int n = 0;
  if (C::RH != C::ROWS) out[n++] = C::RH;
  out[n++] = C::ROWS;
  out[n++] = C::R2;
  return n;
}

template <int LY, int LZ>
struct YzCfg {
  // radix-8 butterflies per component (2-D: of all three components)
  static constexpr int B0 = LZ == 1 ? 3 * LY / 8 : LY * LZ / 8;
  static constexpr int NT = B0 < 64 ? 64 : (B0 > 512 ? 512 : B0);
  static constexpr size_t SMEM = sizeof(float2) * (3 * LZ * (LY + 1) + 2 * (LY + LZ));
};

// one cluster launch of a (y, z) kernel: CLY*CLZ blocks per kx plane and
// instance; the kernel's shared-memory limit is set on every launch (a
// function attribute belongs to the current device's context; the call is
// host-side and enqueues nothing)
template <typename K>
void launch_yz_cluster(K kern, size_t smem, int nt, const Geom& g, const Buffers& b, cudaStream_t s,
                       const BatchArgs& ba, bool pdl) {
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const int CL = g.cly * g.clz;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(g.hx * CL * ba.count);
  cfg.blockDim = dim3(nt);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CL;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = pdl ? 1 : 0;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  cudaLaunchKernelEx(&cfg, kern, g, b.spec, (const float*)b.ktf, (const float2*)b.tw, (const DevState*)b.st, ba);
}

template <int LY, int LZ>
void run_yz(const Geom& g, const Buffers& b, cudaStream_t s, const BatchArgs& ba, bool pdl) {
  using C = YzCfg<LY, LZ>;
  if constexpr (LZ >= 4) {
    // z-split clusters share the y transforms between the two z classes
    if (g.clz == 2) {
      launch_yz_cluster(k_yz2<LY, LZ, C::NT>, C::SMEM, C::NT, g, b, s, ba, pdl);
      return;
    }
  }
  launch_yz_cluster(k_yz<LY, LZ, C::NT>, C::SMEM, C::NT, g, b, s, ba, pdl);
}

__global__ void k_kt_transpose(Geom g, const float* __restrict__ kt, float* __restrict__ ktf) {
  const int per = g.hky * g.hkz;   // octant: 6 hkx hky hkz < 2^31 floats
  const long long total = 6LL * g.hkx * per;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  // destination index i = (kx * 6 + c) * per + iz * hky + iy
  const int iy = (int)(i % g.hky);
  const int iz = (int)((i / g.hky) % g.hkz);
  const int c = (int)((i / per) % 6);
  const int kx = (int)(i / (6 * per));
  ktf[i] = kt[(long long)c * g.hkx * per + ((long long)iz * g.hky + iy) * g.hkx + kx];
}

}  // namespace

void launch_kt_transpose(const Geom& g, const float* kt, float* ktf, cudaStream_t s) {
  const long long total = 6LL * g.hkx * g.hky * g.hkz;
  k_kt_transpose<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(g, kt, ktf);
}

#define MM_ROWL(LEN, CALL) \
  switch (LEN) {           \
    case 16: CALL(16); break; \
    case 32: CALL(32); break; \
    case 64: CALL(64); break; \
    case 128: CALL(128); break; \
    case 256: CALL(256); break; \
    case 512: CALL(512); break; \
    default: break;        \
  }

// Residue splits for the fused path: py/cly >= ny, pz/clz >= nz,
// 3 (py/cly)(pz/clz) complex values in at most 96 KB of shared memory,
// clusters of at most 4 blocks; the smallest cluster first.
int fused_splits(const Geom& g, int (*out)[2], int max) {
  if (g.px < 32 || g.lx > 512) return 0;
  int n = 0;
  for (int clz = 1; clz <= (g.pz > 1 ? 2 : 1); ++clz)
    for (int cly = 1; cly <= (g.py > 1 ? 2 : 1); ++cly) {
      const int ly = g.py / cly, lz = g.pz / clz;
      if (ly < g.ny || lz < g.nz) continue;
      if (ly < 16 || ly > 1024 || lz > 32) continue;
      if ((long long)ly * lz > 4096) continue;
      if (n < max) {
        out[n][0] = cly;
        out[n][1] = clz;
      }
      ++n;
    }
  return n < max ? n : max;
}

void fused_set_split(Geom& g, int cly, int clz) {
  g.cly = cly;
  g.clz = clz;
  g.ly = g.py / cly;
  g.lz = g.pz / clz;
  g.fused = 1;
}

int fused_xrows(const Geom& g, int* out, int max) {
  int tmp[3];
  int n = 0;
#define XR(LL) n = xrow_options<LL>(tmp)
  MM_ROWL(g.lx, XR)
#undef XR
  n = n < max ? n : max;
  for (int i = 0; i < n; ++i) out[i] = tmp[i];
  return n;
}

// The default plan: the first (smallest) split.
bool fused_plan(Geom& g) {
  g.fused = 0;
  int sp[4][2];
  if (fused_splits(g, sp, 4) == 0) return false;
  fused_set_split(g, sp[0][0], sp[0][1]);
  return true;
}


void launch_demag_fused(const Geom& g, const Buffers& b, const float* m, cudaStream_t s) {
  launch_demag_fused_batch(g, b, m, s, BatchArgs{1, nullptr, nullptr, 0});
}

static void launch_yz_batch(const Geom& g, const Buffers& b, cudaStream_t s, const BatchArgs& ba, bool pdl);

void launch_demag_yz(const Geom& g, const Buffers& b, cudaStream_t s) {
  launch_yz_batch(g, b, s, BatchArgs{1, nullptr, nullptr, 0}, pdl_yz(g));
}

void launch_demag_fused_batch(const Geom& g, const Buffers& b, const float* m, cudaStream_t s, const BatchArgs& ba) {
#define CALL_FX(LL) run_fx_t<LL>(g, b, m, s, ba)
  MM_ROWL(g.lx, CALL_FX)
#undef CALL_FX
  // (the y/z and x C2R kernels start while their predecessor drains)
  launch_yz_batch(g, b, s, ba, true);
#define CALL_IX(LL) run_ix_t<LL>(g, b, s, ba)
  MM_ROWL(g.lx, CALL_IX)
#undef CALL_IX
}

void launch_demag_fused3(const Geom& g, const Buffers& b, const float* m, float2* T, cudaStream_t s) {
  const BatchArgs ba{1, nullptr, nullptr, 0};
#define CALL_FX(LL) run_fx_t<LL>(g, b, m, s, ba)
  MM_ROWL(g.lx, CALL_FX)
#undef CALL_FX
  launch_demag_yz3(g, b, T, s);
#define CALL_IX(LL) run_ix_t<LL>(g, b, s, ba)
  MM_ROWL(g.lx, CALL_IX)
#undef CALL_IX
}

void launch_demag_fused2d(const Geom& g, const Buffers& b, const float* m, cudaStream_t s) {
  const BatchArgs ba{1, nullptr, nullptr, 0};
#define CALL_FX(LL) run_fx_t<LL>(g, b, m, s, ba)
  MM_ROWL(g.lx, CALL_FX)
#undef CALL_FX
  launch_demag_y2d(g, b, s);
#define CALL_IX(LL) run_ix_t<LL>(g, b, s, ba)
  MM_ROWL(g.lx, CALL_IX)
#undef CALL_IX
}

static void launch_yz_batch(const Geom& g, const Buffers& b, cudaStream_t s, const BatchArgs& ba, bool pdl) {
  const int key = g.ly * 100 + g.lz;
  switch (key) {
#define YZ(LY, LZ) \
  case LY * 100 + LZ: run_yz<LY, LZ>(g, b, s, ba, pdl); break;
    YZ(16, 1) YZ(32, 1) YZ(64, 1) YZ(128, 1) YZ(256, 1) YZ(512, 1) YZ(1024, 1)
    YZ(16, 2) YZ(32, 2) YZ(64, 2) YZ(128, 2) YZ(256, 2) YZ(512, 2) YZ(1024, 2)
    YZ(16, 4) YZ(32, 4) YZ(64, 4) YZ(128, 4) YZ(256, 4) YZ(512, 4) YZ(1024, 4)
    YZ(16, 8) YZ(32, 8) YZ(64, 8) YZ(128, 8) YZ(256, 8) YZ(512, 8)
    YZ(16, 16) YZ(32, 16) YZ(64, 16) YZ(128, 16) YZ(256, 16)
    YZ(16, 32) YZ(32, 32) YZ(64, 32) YZ(128, 32)
#undef YZ
    default: break;
  }
}

}  // namespace mm
