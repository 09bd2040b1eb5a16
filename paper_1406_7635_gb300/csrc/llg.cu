// Effective field, Landau-Lifshitz torque and the Dormand-Prince RK45 step
// with a device-resident step controller (Sec. III and Sec. IV).
//
//   B_eff = B_demag + B_exch + B_anis + B_ext
//   B_exch = sum_i C(r, r_i) (m_i - m) / Delta_i^2, C = 2 S * harmonic mean of
//            Aex/Msat (Eq. for inter-region exchange; Neumann: a missing
//            neighbour contributes nothing)
//   B_anis = (2 Ku1/Msat)(u.m)u + (4 Ku2/Msat)(u.m)^3 u
//   tau    = -gamma/(1+alpha^2) (m x B + alpha m x (m x B))   (Eq. eqLLG)
//
// One RK45 attempt is a fixed launch sequence (stage input, demag
// convolution, torque for stages 2..7, then the error kernel whose last block
// runs the controller), so it can be captured once in a CUDA graph and
// replayed: every launch reads the step size and the buffer roles from
// DevState, and returns at once when the controller has marked the call done.
#include "llg_device.cuh"

namespace mm {
namespace {

// ----------------------------------------------------------------------------
// kernels
// ----------------------------------------------------------------------------
__global__ void k_stage_input(Geom g, Ptrs p, float* __restrict__ ms, const DevState* __restrict__ st,
                              const StageCoef* __restrict__ sc, int s) {
  if (st->done) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;   // cells < 2^28, 3 n < 2^31
  const int n = (int)g.n;
  if (i >= g.n) return;
  const int par = st->parity;
  const float* __restrict__ m = par ? p.m1 : p.m0;
  float acc[3] = {m[i], m[n + i], m[2 * n + i]};
  for (int j = 0; j < s; ++j) {
    const float a = sc->ah[s][j];
    if (a == 0.0f) continue;
    const float* __restrict__ k = pick_k(p, k_role(j, par));
    acc[0] = fmaf(a, k[i], acc[0]);
    acc[1] = fmaf(a, k[n + i], acc[1]);
    acc[2] = fmaf(a, k[2 * n + i], acc[2]);
  }
  ms[i] = acc[0];
  ms[n + i] = acc[1];
  ms[2 * n + i] = acc[2];
}

__global__ void k_torque(Geom g, Buffers b, Terms T, Stt S, Ptrs p, const DevState* __restrict__ st, int s,
                         double freq, double phase_over_pi) {
  if (st->done) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;   // cells < 2^28, 3 n < 2^31
  const int n = (int)g.n;
  if (i >= g.n) return;
  const int par = st->parity;
  const float* __restrict__ m = s == 0 ? (par ? p.m1 : p.m0) : b.ms;
  float* __restrict__ k = pick_k(p, k_role(s, par));
  const int x = i % g.nx, y = (i / g.nx) % g.ny, z = i / (g.nx * g.ny);
  const int r = b.code[i];
  if (r == kVacuum) {
    k[i] = k[n + i] = k[2 * n + i] = 0.0f;
    return;
  }
  const float3 mi = f3(m[i], m[n + i], m[2 * n + i]);
  const float sinft = T.zeeman ? excitation(freq, phase_over_pi, st->stage_t[s]) : 0.0f;
  FieldParts P;
  field_at(g, b, T, m, i, x, y, z, r, mi, sinft, f3(b.bd[i], b.bd[n + i], b.bd[2 * n + i]), P);
  const float3 tq = add_stt(g, b, S, m, i, x, y, z, r, mi,
                            llg_torque(mi, total(P), b.lut->gfac[r], b.lut->alpha[r], st->precession));
  k[i] = tq.x;
  k[n + i] = tq.y;
  k[2 * n + i] = tq.z;
}

__global__ void k_begin(DevState* st, StageCoef* sc, const double* __restrict__ fixed, int mode, long long nsteps,
                        double t_end) {
  // (on a local copy: one bulk read and one bulk write of the state)
  DevState s = *st;
  s.status = 0;
  s.done = 0;
  s.call_attempts = 0;
  s.err_bits = 0;
  s.ticket = 0;
  s.mode = mode;
  s.target = s.accepted + nsteps;
  s.t_end = t_end;
  if (mode == 2 && s.fixed_idx >= s.fixed_n) s.done = 1;
  check_done(&s);
  if (nsteps <= 0 && mode != 1) s.done = 1;
  if (!s.done) prepare_attempt(&s, sc, fixed);
  *st = s;
}

// error estimate, candidate m (normalised 5th-order solution), block max,
// controller in the last block
__global__ void k_error_control(Geom g, Buffers b, Ptrs p, DevState* __restrict__ st, StageCoef* __restrict__ sc) {
  if (st->done) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;   // cells < 2^28, 3 n < 2^31
  const int n = (int)g.n;
  const int par = st->parity;
  float e = 0.0f;
  if (i < g.n) {
    float* __restrict__ mnew = par ? p.m0 : p.m1;
    const bool mag = is_magnetic(b.mask, b.region, b.lut, i);
    if (mag) {
      float ex = 0.f, ey = 0.f, ez = 0.f;
      for (int j = 0; j < 7; ++j) {
        const float c = sc->eh[j];
        if (c == 0.0f) continue;
        const float* __restrict__ k = pick_k(p, k_role(j, par));
        ex = fmaf(c, k[i], ex);
        ey = fmaf(c, k[n + i], ey);
        ez = fmaf(c, k[2 * n + i], ez);
      }
      e = sqrtf(ex * ex + ey * ey + ez * ez);
      if (!(e <= FLT_MAX)) e = __int_as_float(0x7f800000);
      const float mx = b.ms[i], my = b.ms[n + i], mz = b.ms[2 * n + i];
      const float inv = rsqrtf(mx * mx + my * my + mz * mz);
      mnew[i] = mx * inv;
      mnew[n + i] = my * inv;
      mnew[2 * n + i] = mz * inv;
    } else {
      mnew[i] = mnew[n + i] = mnew[2 * n + i] = 0.0f;
    }
  }
  // block max (non-negative floats order like their bit patterns)
  for (int o = 16; o > 0; o >>= 1) e = fmaxf(e, __shfl_xor_sync(0xffffffffu, e, o));
  __shared__ float wmax[32];
  if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = e;
  __syncthreads();
  if (threadIdx.x < 32) {
    float v = threadIdx.x < (blockDim.x >> 5) ? wmax[threadIdx.x] : 0.0f;
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (threadIdx.x == 0) {
      atomicMax(&st->err_bits, __float_as_uint(v));
      __threadfence();
      const unsigned int t = atomicAdd(&st->ticket, 1u);
      if (t == gridDim.x - 1) {
        __threadfence();
        controller(st, sc, b.hist, b.fixed);
      }
    }
  }
}

// Getters: mode 0 writes B_eff, mode 1 the torque, mode 2 accumulates energies
// (float64) into acc[0..8] = {demag, exch, anis, zeeman, mx, my, mz, ncells, dmi}
// (M.B sums; the host multiplies by the cell volume), mode 4 the maximum of
// |torque| over the magnetic cells into the first 4 bytes of acc (float bits,
// atomicMax; the host zeroes them first).
__global__ void k_field_out(Geom g, Buffers b, Terms T, Stt S, const float* __restrict__ m,
                            const DevState* __restrict__ st, int mode, double freq, double phase_over_pi) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;   // cells < 2^28, 3 n < 2^31
  const int n = (int)g.n;
  double acc[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  float tmax = 0.0f;
  if (i < g.n) {
    const int x = i % g.nx, y = (i / g.nx) % g.ny, z = i / (g.nx * g.ny);
    const int r = b.code[i];
    const bool mag = r != kVacuum;
    float3 out = f3(0, 0, 0);
    if (mag) {
      const float3 mi = f3(m[i], m[n + i], m[2 * n + i]);
      const float sinft = T.zeeman ? excitation(freq, phase_over_pi, st->t) : 0.0f;
      FieldParts P;
      field_at(g, b, T, m, i, x, y, z, r, mi, sinft, f3(b.bd[i], b.bd[n + i], b.bd[2 * n + i]), P);
      const float3 B = total(P);
      if (mode == 0) out = B;
      else if (mode == 1)
        out = add_stt(g, b, S, m, i, x, y, z, r, mi, llg_torque(mi, B, b.lut->gfac[r], b.lut->alpha[r], st->precession));
      else if (mode == 4) {
        const float3 tq =
            add_stt(g, b, S, m, i, x, y, z, r, mi, llg_torque(mi, B, b.lut->gfac[r], b.lut->alpha[r], st->precession));
        tmax = sqrtf(tq.x * tq.x + tq.y * tq.y + tq.z * tq.z);
        if (!(tmax <= FLT_MAX)) tmax = __int_as_float(0x7f800000);
      } else {
        const double ms = b.lut->msat[r];
        auto dot = [&](float3 v) { return ms * ((double)mi.x * v.x + (double)mi.y * v.y + (double)mi.z * v.z); };
        acc[0] = -0.5 * dot(P.demag);
        acc[1] = -0.5 * dot(P.exch);
        acc[2] = -0.5 * dot(P.anis1) - 0.25 * dot(P.anis2);
        acc[3] = -dot(P.zee);
        acc[4] = mi.x;
        acc[5] = mi.y;
        acc[6] = mi.z;
        acc[7] = 1.0;
        acc[8] = -0.5 * dot(P.dmi);
      }
    }
    if (mode < 2) {
      b.out[i] = out.x;
      b.out[n + i] = out.y;
      b.out[2 * n + i] = out.z;
    }
  }
  if (mode == 4) {
    for (int o = 16; o > 0; o >>= 1) tmax = fmaxf(tmax, __shfl_xor_sync(0xffffffffu, tmax, o));
    if ((threadIdx.x & 31) == 0) atomicMax(reinterpret_cast<unsigned int*>(b.acc), __float_as_uint(tmax));
  }
  if (mode == 2) {
    __shared__ double red[9][32];
    for (int c = 0; c < 9; ++c) {
      double v = acc[c];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if ((threadIdx.x & 31) == 0) red[c][threadIdx.x >> 5] = v;
    }
    __syncthreads();
    if (threadIdx.x < 9) {
      double v = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[threadIdx.x][w];
      atomicAdd(&b.acc[threadIdx.x], v);
    }
  }
}

__global__ void k_normalize(Geom g, const uint8_t* __restrict__ mask, const uint8_t* __restrict__ region,
                            const RegionLUT* __restrict__ lut, float* __restrict__ m) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;   // cells < 2^28, 3 n < 2^31
  const int n = (int)g.n;
  if (i >= g.n) return;
  const bool mag = is_magnetic(mask, region, lut, i);
  const float x = m[i], y = m[n + i], z = m[2 * n + i];
  const float n2 = x * x + y * y + z * z;
  const float inv = (mag && n2 > 0.0f) ? rsqrtf(n2) : 0.0f;
  m[i] = x * inv;
  m[n + i] = y * inv;
  m[2 * n + i] = z * inv;
}

// *flag = 1 if the 3 n floats of a and b differ in any bit (the flag is
// zeroed by the caller; every writer stores the same value)
__global__ void k_m_differs(long long n3, const float* __restrict__ a, const float* __restrict__ b,
                            int* __restrict__ flag) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n3) return;
  if (__float_as_uint(a[i]) != __float_as_uint(b[i])) *flag = 1;
}

__global__ void k_codes(Geom g, const uint8_t* __restrict__ mask, const uint8_t* __restrict__ region,
                        const RegionLUT* __restrict__ lut, int* __restrict__ code) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;   // cells < 2^28
  if (i >= g.n) return;
  code[i] = is_magnetic(mask, region, lut, i) ? (int)region[i] : kVacuum;
}

__global__ void k_copy_cur(Geom g, const float* __restrict__ m0, const float* __restrict__ m1,
                           const DevState* __restrict__ st, float* __restrict__ dst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;   // 3 n < 2^31
  if (i >= 3 * g.n) return;
  dst[i] = st->parity ? m1[i] : m0[i];
}

Ptrs ptrs(const Buffers& b) {
  Ptrs p;
  p.m0 = b.m[0];
  p.m1 = b.m[1];
  for (int j = 0; j < 7; ++j) p.k[j] = b.k[j];
  return p;
}

constexpr int kT = 256;
unsigned blocks(long long n) { return (unsigned)((n + kT - 1) / kT); }

}  // namespace

// StageCoef lives right after DevState in the same allocation
static StageCoef* coef(const Buffers& b) { return reinterpret_cast<StageCoef*>(b.st + 1); }
size_t devstate_bytes() { return sizeof(DevState) + sizeof(StageCoef); }

void launch_begin_mode(const Buffers& b, int mode, long long nsteps, double t_end, cudaStream_t s) {
  k_begin<<<1, 1, 0, s>>>(b.st, coef(b), b.fixed, mode, nsteps, t_end);
}

void launch_stage_input(const Geom& g, const Buffers& b, int stage, cudaStream_t s) {
  k_stage_input<<<blocks(g.n), kT, 0, s>>>(g, ptrs(b), b.ms, b.st, coef(b), stage);
}

void launch_torque_t(const Geom& g, const Buffers& b, const Terms& T, const Stt& S, int stage, double freq,
                     double phase, cudaStream_t s) {
  k_torque<<<blocks(g.n), kT, 0, s>>>(g, b, T, S, ptrs(b), b.st, stage, freq, phase / 3.14159265358979323846);
}

void launch_error_control(const Geom& g, const Buffers& b, cudaStream_t s) {
  k_error_control<<<blocks(g.n), kT, 0, s>>>(g, b, ptrs(b), b.st, coef(b));
}

void launch_field_out_t(const Geom& g, const Buffers& b, const Terms& T, const Stt& S, const float* m, int mode,
                        double freq, double phase, cudaStream_t s) {
  k_field_out<<<blocks(g.n), kT, 0, s>>>(g, b, T, S, m, b.st, mode, freq, phase / 3.14159265358979323846);
}

void launch_m_differs(const Geom& g, const float* a, const float* b, int* flag, cudaStream_t s) {
  k_m_differs<<<blocks(3 * g.n), kT, 0, s>>>(3 * g.n, a, b, flag);
}

void launch_normalize(const Geom& g, const Buffers& b, float* m, cudaStream_t s) {
  k_normalize<<<blocks(g.n), kT, 0, s>>>(g, b.mask, b.region, b.lut, m);
}

void launch_codes(const Geom& g, const Buffers& b, cudaStream_t s) {
  k_codes<<<blocks(g.n), kT, 0, s>>>(g, b.mask, b.region, b.lut, b.code);
}

void launch_copy_mcur(const Geom& g, const Buffers& b, float* dst, cudaStream_t s) {
  k_copy_cur<<<blocks(3 * g.n), kT, 0, s>>>(g, b.m[0], b.m[1], b.st, dst);
}

}  // namespace mm
