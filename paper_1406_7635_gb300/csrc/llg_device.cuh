// Per-cell effective field, Landau-Lifshitz torque and the RK45 step
// controller, shared by the stage kernels (llg.cu) and the fused row kernel
// (rowstage.cu).  Sec. III (field terms, Eq. eqLLG) and Sec. IV (controller).
#pragma once
#include <cfloat>

#include "mm_internal.h"

namespace mm {
namespace {

// Dormand & Prince (1980) tableau: nodes, stage weights, 5th-order weights
// minus embedded 4th-order weights (error estimate).
__constant__ double kC[7] = {0.0, 1.0 / 5.0, 3.0 / 10.0, 4.0 / 5.0, 8.0 / 9.0, 1.0, 1.0};
__constant__ double kA[7][6] = {
    {0, 0, 0, 0, 0, 0},
    {1.0 / 5.0, 0, 0, 0, 0, 0},
    {3.0 / 40.0, 9.0 / 40.0, 0, 0, 0, 0},
    {44.0 / 45.0, -56.0 / 15.0, 32.0 / 9.0, 0, 0, 0},
    {19372.0 / 6561.0, -25360.0 / 2187.0, 64448.0 / 6561.0, -212.0 / 729.0, 0, 0},
    {9017.0 / 3168.0, -355.0 / 33.0, 46732.0 / 5247.0, 49.0 / 176.0, -5103.0 / 18656.0, 0},
    {35.0 / 384.0, 0.0, 500.0 / 1113.0, 125.0 / 192.0, -2187.0 / 6784.0, 11.0 / 84.0}};
__constant__ double kE[7] = {71.0 / 57600.0,      0.0,           -71.0 / 16695.0, 71.0 / 1920.0,
                             -17253.0 / 339200.0, 22.0 / 525.0, -1.0 / 40.0};

// Bogacki & Shampine (1989) 3(2) pair, the solver of relax() (Sec. IV).  Its
// four stages occupy the RK45 stage slots 0, 1, 2 and 6, so the last stage
// takes part in the same FSAL buffer swap (slot 6 <-> slot 0) and the stage
// kernels serve both methods unchanged: row = slot of the stage, column =
// slot of the earlier stage it reads.
__device__ __forceinline__ int slot23(int s) { return s == 3 ? 6 : s; }
__constant__ double kC23[4] = {0.0, 0.5, 0.75, 1.0};
__constant__ double kA23[4][3] = {{0, 0, 0}, {0.5, 0, 0}, {0.0, 0.75, 0}, {2.0 / 9.0, 1.0 / 3.0, 4.0 / 9.0}};
// 3rd-order weights (2/9, 1/3, 4/9, 0) minus 2nd-order weights (7/24, 1/4, 1/3, 1/8)
__constant__ double kE23[4] = {-5.0 / 72.0, 1.0 / 12.0, 1.0 / 9.0, -1.0 / 8.0};

// stage coefficients of the current attempt, h * a_sj and h * e_j, in float
struct StageCoef {
  float ah[7][6];
  float eh[7];
};

__device__ __forceinline__ int k_role(int j, int parity) {
  // FSAL: after an accepted step the 7th stage becomes the next 1st stage;
  // instead of copying, buffers 0 and 6 swap roles
  return j == 0 ? (parity ? 6 : 0) : (j == 6 ? (parity ? 0 : 6) : j);
}

struct Ptrs {
  float* m0;
  float* m1;
  float* k[7];
};

// k buffer j of a by-value pointer set, selected without indexing the
// parameter array at run time (which would copy it to local memory)
__device__ __forceinline__ float* pick_k(const Ptrs& p, int j) {
  switch (j) {
    case 0: return p.k[0];
    case 1: return p.k[1];
    case 2: return p.k[2];
    case 3: return p.k[3];
    case 4: return p.k[4];
    case 5: return p.k[5];
    default: return p.k[6];
  }
}

__device__ __forceinline__ bool is_magnetic(const uint8_t* __restrict__ mask, const uint8_t* __restrict__ region,
                                            const RegionLUT* __restrict__ lut, int i) {
  return mask[i] != 0 && __ldg(&lut->msat[region[i]]) > 0.0f;
}

// ----------------------------------------------------------------------------
// effective field at one cell
// ----------------------------------------------------------------------------
struct FieldParts {
  float3 demag, exch, anis1, anis2, zee, dmi;
};

__device__ __forceinline__ float3 f3(float a, float b, float c) { return make_float3(a, b, c); }

// uniaxial anisotropy (Ku1 and Ku2 parts) and Zeeman field of region r
__device__ __forceinline__ void field_local(const RegionLUT* __restrict__ lut, const Terms& T, int r, float3 mi,
                                            float sinft, FieldParts& P) {
  if (T.anis) {
    const float ux = __ldg(&lut->u[0][r]), uy = __ldg(&lut->u[1][r]), uz = __ldg(&lut->u[2][r]);
    const float um = ux * mi.x + uy * mi.y + uz * mi.z;
    const float a1 = __ldg(&lut->k1[r]) * um;
    const float a2 = __ldg(&lut->k2[r]) * um * um * um;
    P.anis1 = f3(a1 * ux, a1 * uy, a1 * uz);
    P.anis2 = f3(a2 * ux, a2 * uy, a2 * uz);
  } else {
    P.anis1 = P.anis2 = f3(0, 0, 0);
  }
  if (T.zeeman) {
    P.zee = f3(__ldg(&lut->b0[0][r]) + __ldg(&lut->b1[0][r]) * sinft,
               __ldg(&lut->b0[1][r]) + __ldg(&lut->b1[1][r]) * sinft,
               __ldg(&lut->b0[2][r]) + __ldg(&lut->b1[2][r]) * sinft);
  } else {
    P.zee = f3(0, 0, 0);
  }
}

// Ghost value of a missing neighbour in direction d (0 x-, 1 x+, 2 y-, 3 y+,
// 4 z-, 5 z+) under the boundary conditions of the interfacial DMI (Sec. III,
// "Dzyaloshinskii-Moriya interaction"): m + n Delta dm/di with the outward
// normal n and dm/dx = (-c mz, 0, c mx), dm/dy = (0, -c mz, c my), dm/dz = 0,
// c = D / (2 Aex).  With c = 0 it is m itself (the plain Neumann edge).
__device__ __forceinline__ float3 dmi_ghost(float3 m, int d, float c, float dx, float dy) {
  switch (d) {
    case 0: return f3(m.x + dx * c * m.z, m.y, m.z - dx * c * m.x);
    case 1: return f3(m.x - dx * c * m.z, m.y, m.z + dx * c * m.x);
    case 2: return f3(m.x, m.y + dy * c * m.z, m.z - dy * c * m.y);
    case 3: return f3(m.x, m.y - dy * c * m.z, m.z + dy * c * m.y);
    default: return m;
  }
}

// B_DM = (2D/Msat)(dmz/dx, dmz/dy, -dmx/dx - dmy/dy), central differences
// over the x-, x+, y-, y+ neighbour values (present or ghost)
__device__ __forceinline__ float3 dmi_field(float pref, float3 xm, float3 xp, float3 ym, float3 yp, float dx,
                                            float dy) {
  const float hx = 0.5f / dx, hy = 0.5f / dy;
  return f3(pref * (xp.z - xm.z) * hx, pref * (yp.z - ym.z) * hy,
            -pref * ((xp.x - xm.x) * hx + (yp.y - ym.y) * hy));
}

// Effective field at cell i of code ci (a magnetic cell: ci < kVacuum).
// Exchange: the six neighbours are read unconditionally; a neighbour outside
// the grid is replaced by the cell itself (m_j - m_i = 0) and a vacuum
// neighbour has a zero coupling, so the loads carry no branches.
__device__ __forceinline__ void field_at(const Geom& g, const Buffers& b, const Terms& T, const float* __restrict__ m,
                                         int i, int x, int y, int z, int ci, float3 mi, float sinft,
                                         float3 bdemag, FieldParts& P) {
  const RegionLUT* __restrict__ lut = b.lut;
  const int r = ci & (kRegions - 1);
  P.demag = T.demag ? bdemag : f3(0, 0, 0);
  P.dmi = f3(0, 0, 0);
  float3 ex = f3(0, 0, 0);
  if (T.exch || T.dmi) {
    const float* __restrict__ xl = b.xlut + r * kXStride;
    const int sy = g.nx, sz = g.nx * g.ny, n = (int)g.n;
    // along a periodic axis the grid wraps around (Sec. III.B, PBC)
    const int js[6] = {x > 0 ? i - 1 : (g.pbcx ? i + g.nx - 1 : i),
                       x < g.nx - 1 ? i + 1 : (g.pbcx ? i - (g.nx - 1) : i),
                       y > 0 ? i - sy : (g.pbcy ? i + sy * (g.ny - 1) : i),
                       y < g.ny - 1 ? i + sy : (g.pbcy ? i - sy * (g.ny - 1) : i),
                       z > 0 ? i - sz : (g.pbcz ? i + sz * (g.nz - 1) : i),
                       z < g.nz - 1 ? i + sz : (g.pbcz ? i - sz * (g.nz - 1) : i)};
    const bool per[6] = {g.pbcx > 0, g.pbcx > 0, g.pbcy > 0, g.pbcy > 0, g.pbcz > 0, g.pbcz > 0};
    const float id2[6] = {g.idx2, g.idx2, g.idy2, g.idy2, g.idz2, g.idz2};
    if (!T.dmi) {
#pragma unroll
      for (int d = 0; d < 6; ++d) {
        const int j = js[d];
        const float c = __ldg(&xl[b.code[j]]) * id2[d];
        ex.x += c * (m[j] - mi.x);
        ex.y += c * (m[n + j] - mi.y);
        ex.z += c * (m[2 * n + j] - mi.z);
      }
    } else {
      // a missing neighbour (grid edge or vacuum) is the ghost value, coupled
      // with the cell's own 2 Aex/Msat; the in-plane values feed B_DM
      const float cbc = __ldg(&lut->dbc[r]);
      float3 v[4];
#pragma unroll
      for (int d = 0; d < 6; ++d) {
        const int j = js[d];
        const int cj = b.code[j];
        const bool present = (j != i || per[d]) && cj != kVacuum;
        const float3 mj = present ? f3(m[j], m[n + j], m[2 * n + j]) : dmi_ghost(mi, d, cbc, g.cdx, g.cdy);
        const float c = T.exch ? __ldg(&xl[present ? cj : r]) * id2[d] : 0.0f;
        ex.x += c * (mj.x - mi.x);
        ex.y += c * (mj.y - mi.y);
        ex.z += c * (mj.z - mi.z);
        if (d < 4) v[d] = mj;
      }
      P.dmi = dmi_field(__ldg(&lut->dmi[r]), v[0], v[1], v[2], v[3], g.cdx, g.cdy);
    }
  }
  P.exch = ex;
  field_local(lut, T, r, mi, sinft, P);
}

__device__ __forceinline__ float3 total(const FieldParts& P) {
  return f3(P.demag.x + P.exch.x + P.anis1.x + P.anis2.x + P.zee.x + P.dmi.x,
            P.demag.y + P.exch.y + P.anis1.y + P.anis2.y + P.zee.y + P.dmi.y,
            P.demag.z + P.exch.z + P.anis1.z + P.anis2.z + P.zee.z + P.dmi.z);
}

// ----------------------------------------------------------------------------
// spin-transfer torques (Sec. III), general stage kernels only
// ----------------------------------------------------------------------------
// Zhang-Li h = (u . grad) m at magnetic cell i of region r: central
// differences; a missing neighbour (grid edge or vacuum) is the cell itself,
// periodic axes wrap.
__device__ __forceinline__ float3 zhang_li_h(const Geom& g, const Buffers& b, const Stt& S,
                                             const float* __restrict__ m, int i, int x, int y, int z, int r,
                                             float3 mi) {
  const int sy = g.nx, sz = g.nx * g.ny, n = (int)g.n;
  const int jp[3] = {x < g.nx - 1 ? i + 1 : (g.pbcx ? i - (g.nx - 1) : i),
                     y < g.ny - 1 ? i + sy : (g.pbcy ? i - sy * (g.ny - 1) : i),
                     z < g.nz - 1 ? i + sz : (g.pbcz ? i - sz * (g.nz - 1) : i)};
  const int jm[3] = {x > 0 ? i - 1 : (g.pbcx ? i + g.nx - 1 : i),
                     y > 0 ? i - sy : (g.pbcy ? i + sy * (g.ny - 1) : i),
                     z > 0 ? i - sz : (g.pbcz ? i + sz * (g.nz - 1) : i)};
  const float hd[3] = {S.hx, S.hy, S.hz};
  float3 h = f3(0, 0, 0);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int a1 = jp[a], a0 = jm[a];
    const float3 v1 = b.code[a1] != kVacuum ? f3(m[a1], m[n + a1], m[2 * n + a1]) : mi;
    const float3 v0 = b.code[a0] != kVacuum ? f3(m[a0], m[n + a0], m[2 * n + a0]) : mi;
    const float c = __ldg(&S.lut->zlu[a][r]) * hd[a];
    h.x += c * (v1.x - v0.x);
    h.y += c * (v1.y - v0.y);
    h.z += c * (v1.z - v0.z);
  }
  return h;
}

// Spin-transfer torques of region r at m, read in the sign convention of the
// LL torque (dm/dt = -gamma tau): Zhang-Li -(a m x (m x h) + b m x h);
// Slonczewski -g ((eps - al eps') m x (m_P x m) - (eps' - al eps) m x m_P),
// g = gamma beta / (1 + al^2), eps = P L^2 / ((L^2 + 1) + (L^2 - 1) m.m_P).
__device__ __forceinline__ float3 stt_torque(const Stt& S, int r, float3 m, float3 h) {
  const SttLUT* __restrict__ L = S.lut;
  float3 out = f3(0, 0, 0);
  auto cr = [](float3 a, float3 b) {
    return f3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
  };
  if (S.zl) {
    const float ca = __ldg(&L->zla[r]), cb = __ldg(&L->zlb[r]);
    const float3 mh = cr(m, h), mmh = cr(m, mh);
    out = f3(-(ca * mmh.x + cb * mh.x), -(ca * mmh.y + cb * mh.y), -(ca * mmh.z + cb * mh.z));
  }
  if (S.sl) {
    const float3 mp = f3(__ldg(&L->mp[0][r]), __ldg(&L->mp[1][r]), __ldg(&L->mp[2][r]));
    const float eps =
        __ldg(&L->slp[r]) / (__ldg(&L->sl1[r]) + __ldg(&L->sl2[r]) * (m.x * mp.x + m.y * mp.y + m.z * mp.z));
    const float ep = __ldg(&L->sle[r]), al = __ldg(&L->alpha[r]), gs = __ldg(&L->slg[r]);
    const float t1 = gs * (eps - al * ep), t2 = gs * (ep - al * eps);
    const float3 mpm = cr(mp, m), mmpm = cr(m, mpm), mmp = cr(m, mp);
    out.x -= t1 * mmpm.x - t2 * mmp.x;
    out.y -= t1 * mmpm.y - t2 * mmp.y;
    out.z -= t1 * mmpm.z - t2 * mmp.z;
  }
  return out;
}

// LL torque plus the spin-transfer torques (if any) at magnetic cell i
__device__ __forceinline__ float3 add_stt(const Geom& g, const Buffers& b, const Stt& S,
                                          const float* __restrict__ m, int i, int x, int y, int z, int r, float3 mi,
                                          float3 tq) {
  if (!(S.zl || S.sl)) return tq;
  const float3 h = S.zl ? zhang_li_h(g, b, S, m, i, x, y, z, r, mi) : f3(0, 0, 0);
  const float3 ts = stt_torque(S, r, mi, h);
  return f3(tq.x + ts.x, tq.y + ts.y, tq.z + ts.z);
}


__device__ __forceinline__ float3 llg_torque(float3 m, float3 B, float gfac, float alpha, int precession) {
  const float3 mxB = f3(m.y * B.z - m.z * B.y, m.z * B.x - m.x * B.z, m.x * B.y - m.y * B.x);
  const float3 mxmxB = f3(m.y * mxB.z - m.z * mxB.y, m.z * mxB.x - m.x * mxB.z, m.x * mxB.y - m.y * mxB.x);
  const float p = precession ? 1.0f : 0.0f;
  return f3(gfac * (p * mxB.x + alpha * mxmxB.x), gfac * (p * mxB.y + alpha * mxmxB.y),
            gfac * (p * mxB.z + alpha * mxmxB.z));
}

// sin(2 pi f t + phase), with the phase reduced in float64 before a float
// sinpi (one function of time for the whole excitation)
__device__ __forceinline__ float excitation(double f, double phase_over_pi, double t) {
  double y = 2.0 * (f * t - floor(f * t)) + phase_over_pi;
  y -= 2.0 * floor(0.5 * y);
  return sinpif((float)y);
}

// per-attempt set-up: step size, stage times, stage coefficients
__device__ void prepare_attempt(DevState* st, StageCoef* sc, const double* __restrict__ fixed) {
  double h;
  if (st->mode == 2) h = fixed[st->fixed_idx];
  else if (st->mode == 1) h = fmin(st->dt, st->t_end - st->t);
  else h = st->dt;
  st->h = h;
  if (st->method == 1) {
    for (int s = 0; s < 7; ++s) {
      st->stage_t[s] = st->t;
      for (int j = 0; j < 6; ++j) sc->ah[s][j] = 0.0f;
      sc->eh[s] = 0.0f;
    }
    for (int s = 0; s < 4; ++s) {
      const int r = slot23(s);
      st->stage_t[r] = st->t + kC23[s] * h;
      for (int j = 0; j < s; ++j) sc->ah[r][slot23(j)] = (float)(kA23[s][j] * h);
      sc->eh[r] = (float)(kE23[s] * h);
    }
    return;
  }
  for (int s = 0; s < 7; ++s) {
    st->stage_t[s] = st->t + kC[s] * h;
    for (int j = 0; j < 6; ++j) sc->ah[s][j] = (float)(kA[s][j] * h);
    sc->eh[s] = (float)(kE[s] * h);
  }
}

__device__ void check_done(DevState* st) {
  if (st->mode == 0 && st->accepted >= st->target) st->done = 1;
  if (st->mode == 1 && st->t >= st->t_end) st->done = 1;
  if (st->mode == 2 && (st->fixed_idx >= st->fixed_n || st->accepted >= st->target)) st->done = 1;
}

// The controller (Sec. IV, "Adaptive time step"): eps = max |tau_5 - tau_4| dt
// against MaxErr with headroom 0.8.  Readings: accept iff eps <= MaxErr;
// dt_new = dt clamp(0.8 (MaxErr/eps)^(1/5), 0.2, 5) (exponent 1/3 for RK23,
// whose error estimate is of order 2), bounded by dt_max, and
// at least dt_min after an accepted step; a rejection that would need a step
// below dt_min ends the call with MM_ERR_DT_UNDERFLOW.
__device__ void controller_on(DevState* st, StageCoef* sc, double* __restrict__ hist,
                              const double* __restrict__ fixed) {
  const double eps = (double)__uint_as_float(st->err_bits);
  st->err_bits = 0;
  st->ticket = 0;
  st->evals += st->method == 1 ? 3 : 6;
  st->call_attempts++;
  st->last_err = eps;
  if (!(eps <= DBL_MAX)) {
    st->status = -4;   // MM_ERR_NONFINITE
    st->done = 1;
    return;
  }
  const double h = st->h;
  const bool replay = st->mode == 2;
  const bool accept = replay || eps <= st->max_err;
  // The growth factor in float32: it only scales dt and is clamped to
  // [0.2, 5].  A float64 pow runs on the GPU's FP64 pipe, slow on this part,
  // in one thread at the end of every attempt: measured on the 128 x 128 x 32
  // step, the last row kernel took 35.6 us with it and 31.1 us without.
  const float ex = st->method == 1 ? 1.0f / 3.0f : 0.2f;
  const float ratio = (float)st->max_err / (float)eps;   // eps > 0 below; inf for a tiny eps
  const double factor = eps == 0.0 ? 5.0 : (double)fminf(5.0f, fmaxf(0.2f, (float)st->headroom * powf(ratio, ex)));
  const double ndt = fmin(h * factor, st->dt_max);
  if (accept) {
    st->t += h;
    if (st->mode == 1 && st->t + 1e-6 * h >= st->t_end) st->t = st->t_end;
    st->parity ^= 1;
    if (st->hist_n < kHistCap) hist[st->hist_n] = h;
    st->hist_n++;
    st->accepted++;
    if (replay) st->fixed_idx++;
    else st->dt = fmax(ndt, st->dt_min);
    check_done(st);
  } else {
    st->rejected++;
    if (ndt < st->dt_min) {
      st->status = -5;   // MM_ERR_DT_UNDERFLOW
      st->done = 1;
      return;
    }
    st->dt = ndt;
  }
  if (!st->done) prepare_attempt(st, sc, fixed);
}

// The controller on a local copy of the device state: one bulk read (all of
// its loads in flight at once) and one bulk write, instead of a chain of
// single-field round trips through memory on the attempt's critical path.
// It runs in one thread after every other block of the attempt has finished
// with the state.
__device__ void controller(DevState* st, StageCoef* sc, double* __restrict__ hist,
                           const double* __restrict__ fixed) {
  DevState s = *st;
  controller_on(&s, sc, hist, fixed);
  *st = s;
}

}  // namespace
}  // namespace mm
