// C ABI (include/mm.h): context lifetime, parameters, state transfer, the
// stepping loop and the getters.
//
// The stepping loop: one RK45 attempt (6 stage evaluations + error/controller)
// is captured once into a CUDA graph and replayed.  The controller runs on the
// device and marks the call done; the host only replays the graph and reads the
// device state back at a few check points, so steps are taken without a
// host round trip per step.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/mm.h"
#include "mm_internal.h"

using namespace mm;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

#define MM_CUDA(call)                                                                  \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess)                                                             \
      return fail(e_ == cudaErrorMemoryAllocation ? MM_ERR_OOM : MM_ERR_CUDA,          \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                 \
  } while (0)

constexpr double kPi = 3.14159265358979323846;
constexpr double kGamma = 1.7595e11;

int next_pow2(int v) {
  int p = 1;
  while (p < v) p <<= 1;
  return p;
}

struct StateBlobHeader {
  unsigned magic;
  int nx, ny, nz;
  unsigned devstate_size;
  int k1_valid;
};

}  // namespace

struct mm_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  Geom g{};
  double dx = 0, dy = 0, dz = 0;
  Buffers b{};
  // host-side tables
  mm_material mat[kRegions];
  std::vector<double> S;        // [256][256]
  double b0[kRegions][3]{}, b1[kRegions][3]{};
  double freq = 0, phase = 0;
  Terms T{1, 1, 1, 1, 0};
  int stt_zl = 0, stt_sl = 0;   // switches of mm_enable_stt
  Stt stt{};                     // active spin-transfer torques (set by flush_luts)
  RsMaps maps{};                 // tensor maps of the row-stage kernels (rowstage_maps)
  int yz_req = 0;                // requested (y, z) kernels: 0 default, 1 cluster, 2 three kernels
  bool yz3 = false;              // the three-kernel (y, z) path is active
  bool y2d = false;              // the one-kernel 2-D (y, K, y^-1) path is active
  float2* yzt = nullptr;         // its y-transformed buffer (yz3_bytes)
  // branch of the row-stage path: the earlier-stage sums (k_rs_partial) run
  // on `side`, forked after each row kernel and joined before the next
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  SttLUT* stt_lut = nullptr;     // device table
  int method = 0;                // host copy of DevState::method
  bool lut_dirty = true;
  bool m_set = false;
  bool k1_valid = false;
  // graph of one attempt
  cudaGraphExec_t graph = nullptr;
  bool graph_valid = false;
  DevState* st_host = nullptr;   // pinned mirror
  bool st_fresh = false;         // st_host equals the device state (no stepping kernel since)
  int fixed_cap = 0;
  int fixed_n = 0;   // host copy of the replay length
  long long launches = 0;        // kernels launched (host count)
  long long graph_nodes = 0;     // kernels per captured attempt
  // learned demag surrogate (fno.cu) with the exact path as guard
  mm_fno* sur = nullptr;
  bool sur_active = false;
  int sur_every = 10;
  double sur_tol = 1e-3;
  float sur_inv_ref = 0.f, sur_mu0_ref = 0.f;
  long long sur_steps = 0, sur_checks = 0, sur_fallbacks = 0;
  double sur_last_err = 0.0;
  double* sur_acc = nullptr;   // device, 2 doubles
};

namespace {

int read_state(mm_ctx* c) {
  MM_CUDA(cudaMemcpyAsync(c->st_host, c->b.st, sizeof(DevState), cudaMemcpyDeviceToHost, c->stream));
  MM_CUDA(cudaStreamSynchronize(c->stream));
  c->st_fresh = true;
  return MM_OK;
}

int write_state(mm_ctx* c) {
  MM_CUDA(cudaMemcpyAsync(c->b.st, c->st_host, sizeof(DevState), cudaMemcpyHostToDevice, c->stream));
  MM_CUDA(cudaStreamSynchronize(c->stream));
  c->st_fresh = true;
  return MM_OK;
}

// the host mirror of the device state, read back only if a stepping kernel
// may have changed it since the last transfer
int current_state(mm_ctx* c) { return c->st_fresh ? MM_OK : read_state(c); }

// Derived float tables from the float64 host parameters.
int flush_luts(mm_ctx* c) {
  if (!c->lut_dirty) return MM_OK;
  RegionLUT L{};
  std::vector<float> X((size_t)kRegions * kXStride, 0.0f);
  double a[kRegions];
  int dmi = 0, zl = 0, sl = 0;
  SttLUT SL{};
  for (int r = 0; r < kRegions; ++r) {
    const mm_material& m = c->mat[r];
    L.msat[r] = (float)m.msat;
    L.alpha[r] = (float)m.alpha;
    L.gfac[r] = (float)(-m.gamma_ll / (1.0 + m.alpha * m.alpha));
    L.k1[r] = m.msat > 0 ? (float)(2.0 * m.ku1 / m.msat) : 0.0f;
    L.k2[r] = m.msat > 0 ? (float)(4.0 * m.ku2 / m.msat) : 0.0f;
    double u[3] = {m.anis_u[0], m.anis_u[1], m.anis_u[2]};
    const double nu = std::sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    for (int k = 0; k < 3; ++k) {
      L.u[k][r] = nu > 0 ? (float)(u[k] / nu) : 0.0f;
      L.b0[k][r] = (float)c->b0[r][k];
      L.b1[k][r] = (float)c->b1[r][k];
    }
    a[r] = m.msat > 0 ? m.aex / m.msat : 0.0;
    L.dmi[r] = m.msat > 0 ? (float)(2.0 * m.dind / m.msat) : 0.0f;
    L.dbc[r] = m.aex > 0 ? (float)(m.dind / (2.0 * m.aex)) : 0.0f;
    if (m.msat > 0 && m.dind != 0.0) dmi = 1;
    // spin-transfer torques (Sec. III); constants in SI
    const double muB = 9.2740100783e-24, qe = 1.602176634e-19, hbar = 1.054571817e-34;
    const double a2 = 1.0 + m.alpha * m.alpha;
    for (int k = 0; k < 3; ++k)
      SL.zlu[k][r] = m.msat > 0 ? (float)(muB * m.jcur[k] / (2.0 * qe * m.msat * (1.0 + m.xi * m.xi))) : 0.0f;
    SL.zla[r] = (float)((1.0 + m.xi * m.alpha) / a2);
    SL.zlb[r] = (float)((m.xi - m.alpha) / a2);
    const double beta = (m.msat > 0 && m.tfree > 0) ? m.jcur[2] * hbar / (m.msat * qe * m.tfree) : 0.0;
    SL.slg[r] = (float)(m.gamma_ll * beta / a2);
    const double l2 = m.lambda_sl * m.lambda_sl;
    SL.slp[r] = (float)(m.pol * l2);
    SL.sl1[r] = (float)(l2 + 1.0);
    SL.sl2[r] = (float)(l2 - 1.0);
    SL.sle[r] = (float)m.eps_prime;
    SL.alpha[r] = (float)m.alpha;
    const double np_ = std::sqrt(m.mp[0] * m.mp[0] + m.mp[1] * m.mp[1] + m.mp[2] * m.mp[2]);
    for (int k = 0; k < 3; ++k) SL.mp[k][r] = np_ > 0 ? (float)(m.mp[k] / np_) : 0.0f;
    if (m.msat > 0 && (m.jcur[0] != 0.0 || m.jcur[1] != 0.0 || m.jcur[2] != 0.0)) {
      if (c->stt_zl) zl = 1;
      if (c->stt_sl && m.tfree > 0 && m.jcur[2] != 0.0) sl = 1;
    }
  }
  // 2 S(r1, r2) * harmonic mean of Aex/Msat (inter-region exchange)
  for (int r1 = 0; r1 < kRegions; ++r1)
    for (int r2 = 0; r2 < kRegions; ++r2) {
      const double s = a[r1] + a[r2];
      const double h = s != 0.0 ? 2.0 * a[r1] * a[r2] / s : 0.0;
      X[(size_t)r1 * kXStride + r2] = (float)(2.0 * c->S[(size_t)r1 * kRegions + r2] * h);
    }
  MM_CUDA(cudaMemcpyAsync(c->b.lut, &L, sizeof(L), cudaMemcpyHostToDevice, c->stream));
  MM_CUDA(cudaMemcpyAsync(c->b.xlut, X.data(), X.size() * sizeof(float), cudaMemcpyHostToDevice, c->stream));
  if (zl || sl) {
    if (!c->stt_lut) MM_CUDA(cudaMalloc((void**)&c->stt_lut, sizeof(SttLUT)));
    MM_CUDA(cudaMemcpyAsync(c->stt_lut, &SL, sizeof(SL), cudaMemcpyHostToDevice, c->stream));
  }
  launch_codes(c->g, c->b, c->stream);
  MM_CUDA(cudaGetLastError());
  MM_CUDA(cudaStreamSynchronize(c->stream));
  c->lut_dirty = false;
  if (dmi != c->T.dmi || zl != c->stt.zl || sl != c->stt.sl) {   // terms switch on or off
    c->T.dmi = dmi;
    c->stt.zl = zl;
    c->stt.sl = sl;
    c->graph_valid = false;
    c->k1_valid = false;
  }
  c->stt.lut = c->stt_lut;
  c->stt.hx = (float)(0.5 / c->dx);
  c->stt.hy = (float)(0.5 / c->dy);
  c->stt.hz = (float)(0.5 / c->dz);
  return MM_OK;
}

void invalidate(mm_ctx* c) {
  c->k1_valid = false;
}

// kernels of the (y, z) part on the fused layout
int yz_launches(const mm_ctx* c) { return c->yz3 ? 3 : 1; }

// kernels one demag convolution launches (see launch_demag)
int demag_launches(const mm_ctx* c) {
  const Geom& g = c->g;
  if (g.fused) return 2 + yz_launches(c);
  int mid = g.pz > 1 ? (g.py > 1 ? 3 : 1) : 1;
  return 2 + mid;
}

// the exact demag convolution of m into nb.bd (nb: the context's buffers,
// possibly without the device state)
void demag_exact(mm_ctx* c, const Buffers& nb, const float* m) {
  if (c->yz3) launch_demag_fused3(c->g, nb, m, c->yzt, c->stream);
  else if (c->y2d) launch_demag_fused2d(c->g, nb, m, c->stream);
  else launch_demag(c->g, nb, m, c->stream);
}

// the (y, z) part of the convolution inside the row-stage path
void demag_yz(mm_ctx* c) {
  if (c->yz3) launch_demag_yz3(c->g, c->b, c->yzt, c->stream);
  else if (c->y2d) launch_demag_y2d(c->g, c->b, c->stream);
  else launch_demag_yz(c->g, c->b, c->stream);
}

// Applies the requested (y, z) kernels: the three-kernel path where the grid
// allows it (default, or asked for), its buffer allocated or freed to match.
int apply_yz_choice(mm_ctx* c) {
  const bool want = yz3_plan(c->g) && c->yz_req != 1;
  if (want && !c->yzt) {
    cudaError_t e = cudaMalloc((void**)&c->yzt, yz3_bytes(c->g));
    if (e != cudaSuccess) {
      c->yzt = nullptr;
      return fail(e == cudaErrorMemoryAllocation ? MM_ERR_OOM : MM_ERR_CUDA,
                  std::string("(y, z) buffer: ") + cudaGetErrorString(e));
    }
  }
  if (!want && c->yzt) {
    cudaStreamSynchronize(c->stream);
    cudaFree(c->yzt);
    c->yzt = nullptr;
  }
  if (want != c->yz3) c->graph_valid = false;
  c->yz3 = want;
  const bool want2d = y2d_plan(c->g) && c->yz_req != 1;
  if (want2d != c->y2d) c->graph_valid = false;
  c->y2d = want2d;
  return MM_OK;
}

// demag field of the stage input: exact convolution, or the surrogate
void enqueue_demag(mm_ctx* c) {
  if (!c->T.demag) return;
  if (c->sur_active)
    launch_fno_demag(c->sur, c->g, c->b, c->b.ms, c->sur_inv_ref, c->sur_mu0_ref, c->b.bd, c->stream);
  else
    demag_exact(c, c->b, c->b.ms);
}

// The row-stage path (fused convolution layout, exact demag): per attempt one
// prep kernel, then per stage the (y, z) transform and one row kernel.
// (a periodic x axis has no padding, so its rows do not fit the row
// kernels' shared-memory stencil, which holds px / 2 cells per row)
// (the spin-transfer torques are evaluated by the general torque kernel only)
bool rowstage_path(const mm_ctx* c) {
  return c->g.fused && !c->sur_active && c->method == 0 && c->g.pbcx == 0 && !c->stt.zl && !c->stt.sl;
}

// The row kernel also starts as a programmatic dependent of the one-kernel
// 2-D (y, z) path (besides the grids of pdl_row).  Same-GPU A/B on the 256 x
// 256 film, ms per step: 0.160 -> 0.140.  (The flag travels as a launch
// argument: the context keeps the Geom layout unchanged.)
bool row_dep(const mm_ctx* c) { return c->y2d; }

// stage-1 torque at the current m (FSAL start)
void enqueue_k1(mm_ctx* c) {
  if (rowstage_path(c)) {
    c->launches += 2 + (c->T.demag ? yz_launches(c) : 0);
    launch_rowstage(c->g, c->b, c->T, c->maps, 0, 0, 0, c->freq, c->phase, c->stream);
    if (c->T.demag) demag_yz(c);
    launch_rowstage(c->g, c->b, c->T, c->maps, 1, 0, 0, c->freq, c->phase, c->stream, row_dep(c));
    return;
  }
  c->launches += 2 + (c->T.demag ? demag_launches(c) : 0);
  launch_copy_mcur(c->g, c->b, c->b.ms, c->stream);
  enqueue_demag(c);
  launch_torque_t(c->g, c->b, c->T, c->stt, 0, c->freq, c->phase, c->stream);
}

// Whether the earlier-stage sums of the row kernels run as a graph branch
// (k_rs_partial beside the (y, z) part) or inside the row kernels.  Same-GPU
// A/B (ms per step, in-kernel -> branch): 128 x 128 x 32, row kernel in 1.7
// waves, 0.4589 -> 0.4470 (row kernel 34.0 -> 27.8 us); 256 x 256 x 1 film,
// one wave and a single short (y, z) kernel, 0.1609 -> 0.1649.  The rule is
// the one of the row kernel's programmatic dependent launch: grids whose
// (y, z) part runs in several waves.
bool partial_branch(const mm_ctx* c) { return c->b.part && pdl_row(c->g); }

// the buffers the row kernels get: without the branch, no partial sums
Buffers row_buffers(const mm_ctx* c) {
  Buffers b = c->b;
  if (!partial_branch(c)) b.part = nullptr;
  return b;
}

// The earlier-stage sums of stage s on the side stream, after everything
// enqueued so far on the context's stream; the row kernel of stage s waits
// for them (join_partial).
void fork_partial(mm_ctx* c, int s) {
  cudaEventRecord(c->ev_fork, c->stream);
  cudaStreamWaitEvent(c->side, c->ev_fork, 0);
  launch_rs_partial(c->g, c->b, s, s < 6 ? 1 : 2, c->side);
  cudaEventRecord(c->ev_join, c->side);
}
void join_partial(mm_ctx* c) { cudaStreamWaitEvent(c->stream, c->ev_join, 0); }

void enqueue_attempt(mm_ctx* c) {
  if (rowstage_path(c)) {
    // stage s: [sums of stage s] beside [(y, z) part], then the row kernel
    const bool br = partial_branch(c);
    const Buffers rb = row_buffers(c);
    if (br) fork_partial(c, 1);
    launch_rowstage(c->g, rb, c->T, c->maps, 0, 1, 0, c->freq, c->phase, c->stream);
    for (int s = 1; s < 7; ++s) {
      if (br && s > 1) fork_partial(c, s);
      if (c->T.demag) demag_yz(c);
      if (br) join_partial(c);
      launch_rowstage(c->g, rb, c->T, c->maps, 1, s, s < 6 ? 1 : 2, c->freq, c->phase, c->stream, row_dep(c));
    }
    return;
  }
  // stage slots of the attempt: RK45 uses 1..6; RK23 its stages 2..4 in
  // slots 1, 2 and 6 (the slot of the FSAL stage)
  static const int kRK45[6] = {1, 2, 3, 4, 5, 6}, kRK23[3] = {1, 2, 6};
  const int* slots = c->method == 1 ? kRK23 : kRK45;
  const int ns = c->method == 1 ? 3 : 6;
  for (int i = 0; i < ns; ++i) {
    launch_stage_input(c->g, c->b, slots[i], c->stream);
    enqueue_demag(c);
    launch_torque_t(c->g, c->b, c->T, c->stt, slots[i], c->freq, c->phase, c->stream);
  }
  launch_error_control(c->g, c->b, c->stream);
}

int build_graph(mm_ctx* c) {
  if (c->graph_valid) return MM_OK;
  if (c->graph) {
    cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
  }
  cudaGraph_t gr = nullptr;
  MM_CUDA(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
  enqueue_attempt(c);
  MM_CUDA(cudaStreamEndCapture(c->stream, &gr));
  size_t nodes = 0;
  cudaGraphGetNodes(gr, nullptr, &nodes);
  c->graph_nodes = (long long)nodes;
  cudaError_t e = cudaGraphInstantiate(&c->graph, gr, 0);
  cudaGraphDestroy(gr);
  if (e != cudaSuccess) return fail(MM_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  c->graph_valid = true;
  return MM_OK;
}

int status_to_code(int status) {
  if (status == MM_ERR_NONFINITE) return fail(MM_ERR_NONFINITE, "non-finite step error (NaN/Inf in m or torque)");
  if (status == MM_ERR_DT_UNDERFLOW) return fail(MM_ERR_DT_UNDERFLOW, "time step fell below dt_min");
  if (status == MM_ERR_TIMEOUT)
    return fail(MM_ERR_TIMEOUT, "a kernel's bounded wait on its tensor copies expired (the attempt was abandoned; m, t "
                                "and dt are those before it)");
  if (status != 0) return fail(status, "device status error");
  return MM_OK;
}

// The stepping loop shared by mm_step and mm_run.  Launches are queued
// without waiting: the begin kernel, the first-stage evaluation and a first
// batch of attempts; the device state is read back only at check points.
int drive(mm_ctx* c, int mode, long long nsteps, double t_end) {
  if (!c->m_set) return fail(MM_ERR_STATE, "m has not been set");
  int rc = flush_luts(c);
  if (rc) return rc;
  rc = build_graph(c);
  if (rc) return rc;
  c->st_fresh = false;   // the stepping kernels write the device state
  launch_begin_mode(c->b, mode, nsteps, t_end, c->stream);
  c->launches += 1;
  if (!c->k1_valid) enqueue_k1(c);   // no-op on the device if begin found nothing to do
  MM_CUDA(cudaGetLastError());
  const bool k1_was_valid = c->k1_valid;
  // at least one attempt per remaining step; then re-check
  long long batch = mode == 1 ? 4 : std::max<long long>(1, nsteps);
  for (int guard = 0; guard < 1000000; ++guard) {
    batch = std::min<long long>(batch, 4096);
    for (long long i = 0; i < batch; ++i) MM_CUDA(cudaGraphLaunch(c->graph, c->stream));
    c->launches += batch * c->graph_nodes;
    rc = read_state(c);
    if (rc) return rc;
    const DevState& s = *c->st_host;
    // the first-stage torque was evaluated iff an attempt ran in this call
    c->k1_valid = k1_was_valid || s.call_attempts > 0;
    if (s.done) return status_to_code(s.status);
    const long long att = s.accepted + s.rejected;
    const double rej = att > 0 ? (double)s.rejected / att : 0.0;
    long long left;
    if (mode == 1) left = (long long)std::ceil((s.t_end - s.t) / std::max(s.dt, 1e-300)) + 1;
    else left = s.target - s.accepted;
    batch = std::max<long long>(1, (long long)std::ceil(left * (1.0 + 2.0 * rej)));
  }
  return fail(MM_ERR_STATE, "stepping loop did not finish");
}

int eval_field(mm_ctx* c, int mode) {
  int rc = flush_luts(c);
  if (rc) return rc;
  rc = read_state(c);
  if (rc) return rc;
  Buffers nb = c->b;
  nb.st = nullptr;    // getters ignore the stepping loop's done flag
  launch_copy_mcur(c->g, c->b, c->b.ms, c->stream);
  if (c->T.demag || mode == 3) demag_exact(c, nb, c->b.ms);
  if (mode == 3) return MM_OK;
  if (mode == 2 || mode == 4) MM_CUDA(cudaMemsetAsync(c->b.acc, 0, 9 * sizeof(double), c->stream));
  Terms T = c->T;
  launch_field_out_t(c->g, c->b, T, c->stt, c->b.ms, mode, c->freq, c->phase, c->stream);
  MM_CUDA(cudaGetLastError());
  return MM_OK;
}

}  // namespace

namespace mm {
void set_last_error(const std::string& msg) { g_err = msg; }

// Grid and padded-FFT geometry of an nx x ny x nz grid (the fused-path
// fields are filled in by fused_plan).
Geom make_geom(int nx, int ny, int nz, double dx, double dy, double dz, const int* pbc) {
  Geom g{};
  if (pbc) {
    g.pbcx = pbc[0];
    g.pbcy = pbc[1];
    g.pbcz = pbc[2];
  }
  g.nx = nx;
  g.ny = ny;
  g.nz = nz;
  g.n = (long long)nx * ny * nz;
  g.idx2 = (float)(1.0 / (dx * dx));
  g.cdx = (float)dx;
  g.cdy = (float)dy;
  g.idy2 = (float)(1.0 / (dy * dy));
  g.idz2 = (float)(1.0 / (dz * dz));
  // transform lengths: a periodic axis is cyclic with period n (Sec. III.B,
  // periodic boundary conditions), an open axis zero-padded to 2n - 1 or more
  g.px = nx == 1 ? 1 : (g.pbcx > 0 ? nx : next_pow2(2 * nx - 1));
  g.py = ny == 1 ? 1 : (g.pbcy > 0 ? ny : next_pow2(2 * ny - 1));
  g.pz = nz == 1 ? 1 : (g.pbcz > 0 ? nz : next_pow2(2 * nz - 1));
  g.lx = g.px == 1 ? 1 : g.px / 2;
  g.hx = g.px == 1 ? 1 : g.lx + 1;
  g.hxs = (g.hx + 7) / 8 * 8;
  g.srows = g.pz > 1 ? g.py : ny;
  g.sc = (long long)nz * g.srows * g.hxs;
  g.hkx = g.px == 1 ? 1 : g.px / 2 + 1;
  g.hky = g.py == 1 ? 1 : g.py / 2 + 1;
  g.hkz = g.pz == 1 ? 1 : g.pz / 2 + 1;
  return g;
}
}  // namespace mm

extern "C" {

const char* mm_last_error(void) { return g_err.c_str(); }

int mm_create(mm_ctx** out, int nx, int ny, int nz, double dx, double dy, double dz, int device, void* stream) {
  if (!out) return fail(MM_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (nx < 1 || ny < 1 || nz < 1) return fail(MM_ERR_ARG, "grid sizes must be >= 1");
  if (nx > 1024 || ny > 512 || nz > 512)
    return fail(MM_ERR_ARG, "grid too large: nx <= 1024, ny <= 512, nz <= 512");
  if (!(dx > 0) || !(dy > 0) || !(dz > 0)) return fail(MM_ERR_ARG, "cell sizes must be > 0");
  MM_CUDA(cudaSetDevice(device));
  mm_ctx* c = new mm_ctx();
  c->device = device;
  c->dx = dx;
  c->dy = dy;
  c->dz = dz;
  c->g = make_geom(nx, ny, nz, dx, dy, dz);
  Geom& g = c->g;
  fused_plan(g);
  for (int r = 0; r < kRegions; ++r) {
    std::memset(&c->mat[r], 0, sizeof(mm_material));
    c->mat[r].gamma_ll = kGamma;
    c->mat[r].anis_u[0] = 1.0;
    c->mat[r].lambda_sl = 1.0;
    c->mat[r].mp[2] = 1.0;
  }
  c->S.assign((size_t)kRegions * kRegions, 1.0);

  auto cleanup = [&](int code) {
    mm_destroy(c);
    return code;
  };
  cudaError_t e = cudaSuccess;
  if (stream) {
    c->stream = (cudaStream_t)stream;
  } else {
    e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cleanup(fail(MM_ERR_CUDA, cudaGetErrorString(e)));
    c->own_stream = true;
  }
  e = cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming);
  if (e != cudaSuccess) return cleanup(fail(MM_ERR_CUDA, cudaGetErrorString(e)));
  const size_t vec = 3 * (size_t)g.n * sizeof(float);
  Buffers& b = c->b;
  auto alloc = [&](void** p, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) e = cudaMemsetAsync(*p, 0, bytes, c->stream);
  };
  alloc((void**)&b.m[0], vec);
  alloc((void**)&b.m[1], vec);
  for (int j = 0; j < 7; ++j) alloc((void**)&b.k[j], vec);
  alloc((void**)&b.ms, vec);
  if (g.fused) alloc((void**)&b.ms2, vec);
  if (g.fused) alloc((void**)&b.part, vec);
  alloc((void**)&b.bd, vec);
  alloc((void**)&b.out, vec);
  alloc((void**)&b.spec, 3 * (size_t)g.sc * sizeof(float2));
  alloc((void**)&b.kt, 6 * (size_t)g.hkx * g.hky * g.hkz * sizeof(float));
  if (g.fused) alloc((void**)&b.ktf, 6 * (size_t)g.hkx * g.hky * g.hkz * sizeof(float));
  alloc((void**)&b.tw, 2048 * sizeof(float2));
  alloc((void**)&b.mask, (size_t)g.n);
  alloc((void**)&b.region, (size_t)g.n);
  alloc((void**)&b.lut, sizeof(RegionLUT));
  alloc((void**)&b.xlut, (size_t)kRegions * kXStride * sizeof(float));
  alloc((void**)&b.code, (size_t)g.n * sizeof(int));
  alloc((void**)&b.st, devstate_bytes());
  alloc((void**)&b.hist, (size_t)kHistCap * sizeof(double));
  alloc((void**)&b.acc, 16 * sizeof(double));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&c->st_host, sizeof(DevState));
  if (e != cudaSuccess)
    return cleanup(fail(e == cudaErrorMemoryAllocation ? MM_ERR_OOM : MM_ERR_CUDA, cudaGetErrorString(e)));
  // twiddles
  std::vector<float2> tw(2048);
  for (int k = 0; k < 2048; ++k) {
    const double a = -2.0 * kPi * k / 2048.0;
    tw[k] = make_float2((float)std::cos(a), (float)std::sin(a));
  }
  e = cudaMemcpyAsync(b.tw, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice, c->stream);
  std::vector<uint8_t> ones((size_t)g.n, 1);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b.mask, ones.data(), ones.size(), cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cleanup(fail(MM_ERR_CUDA, cudaGetErrorString(e)));
  // demag kernel (float64 on the device)
  e = build_kernel_spectrum(g, dx, dy, dz, b.kt, c->stream);
  if (e == cudaSuccess && g.fused) {
    launch_kt_transpose(g, b.kt, b.ktf, c->stream);
    e = cudaStreamSynchronize(c->stream);
  }
  if (e != cudaSuccess)
    return cleanup(fail(e == cudaErrorMemoryAllocation ? MM_ERR_OOM : MM_ERR_CUDA,
                        std::string("kernel precompute: ") + cudaGetErrorString(e)));
  // device state defaults (Sec. IV: MaxErr 1e-5, headroom 0.8)
  DevState& s = *c->st_host;
  std::memset(&s, 0, sizeof(DevState));
  s.dt = 1e-14;
  s.max_err = 1e-5;
  s.headroom = 0.8;
  s.dt_min = 1e-20;
  s.dt_max = 1e-10;
  s.precession = 1;
  s.done = 1;
  s.wait_cycles = kWaitCycles;
  int rc = write_state(c);
  if (rc) return cleanup(rc);
  rc = flush_luts(c);
  if (rc) return cleanup(rc);
  rc = apply_yz_choice(c);
  if (rc) return cleanup(rc);
  // one convolution outside any capture: sets per-kernel launch attributes
  Buffers nb = b;
  nb.st = nullptr;
  demag_exact(c, nb, b.ms);
  e = cudaStreamSynchronize(c->stream);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess && g.fused) e = prepare_rowstage(g);
  if (e == cudaSuccess) rowstage_maps(g, b, &c->maps);
  if (e != cudaSuccess) return cleanup(fail(MM_ERR_CUDA, std::string("warm-up: ") + cudaGetErrorString(e)));
  *out = c;
  return MM_OK;
}

int mm_destroy(mm_ctx* c) {
  if (!c) return MM_OK;
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  if (c->graph) cudaGraphExecDestroy(c->graph);
  Buffers& b = c->b;
  void* ptrs[] = {b.m[0], b.m[1], b.k[0], b.k[1], b.k[2], b.k[3], b.k[4], b.k[5], b.k[6], b.ms, b.ms2, b.bd, b.out,
                  b.spec, b.kt, b.ktf, b.tw, b.mask, b.region, b.lut, b.xlut, b.code, b.st, b.hist, b.acc,
                  b.fixed, c->sur_acc, c->stt_lut, c->yzt, b.part};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (c->st_host) cudaFreeHost(c->st_host);
  if (c->side) {
    cudaStreamSynchronize(c->side);
    cudaStreamDestroy(c->side);
  }
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
  return MM_OK;
}

int mm_set_geometry(mm_ctx* c, const uint8_t* mask) {
  if (!c) return fail(MM_ERR_ARG, "ctx is NULL");
  std::vector<uint8_t> v((size_t)c->g.n, 1);
  if (mask)
    for (long long i = 0; i < c->g.n; ++i) v[i] = mask[i] ? 1 : 0;
  MM_CUDA(cudaMemcpyAsync(c->b.mask, v.data(), v.size(), cudaMemcpyHostToDevice, c->stream));
  MM_CUDA(cudaStreamSynchronize(c->stream));
  c->lut_dirty = true;   // cell codes
  invalidate(c);
  return MM_OK;
}

int mm_set_regions(mm_ctx* c, const uint8_t* region) {
  if (!c) return fail(MM_ERR_ARG, "ctx is NULL");
  std::vector<uint8_t> v((size_t)c->g.n, 0);
  if (region) std::memcpy(v.data(), region, v.size());
  MM_CUDA(cudaMemcpyAsync(c->b.region, v.data(), v.size(), cudaMemcpyHostToDevice, c->stream));
  MM_CUDA(cudaStreamSynchronize(c->stream));
  c->lut_dirty = true;   // cell codes
  invalidate(c);
  return MM_OK;
}

int mm_set_region_material(mm_ctx* c, int region, const mm_material* mat) {
  if (!c || !mat) return fail(MM_ERR_ARG, "NULL argument");
  if (region < 0 || region >= kRegions) return fail(MM_ERR_ARG, "region must be 0..255");
  if (mat->msat < 0 || mat->aex < 0 || mat->alpha < 0 || !std::isfinite(mat->gamma_ll) || !std::isfinite(mat->dind))
    return fail(MM_ERR_ARG, "msat, aex, alpha must be >= 0 and gamma_ll, dind finite");
  c->mat[region] = *mat;
  c->lut_dirty = true;
  invalidate(c);
  return MM_OK;
}

int mm_set_exchange_scale(mm_ctx* c, int r1, int r2, double S) {
  if (!c) return fail(MM_ERR_ARG, "ctx is NULL");
  if (r1 < 0 || r1 >= kRegions || r2 < 0 || r2 >= kRegions) return fail(MM_ERR_ARG, "region must be 0..255");
  c->S[(size_t)r1 * kRegions + r2] = S;
  c->S[(size_t)r2 * kRegions + r1] = S;
  c->lut_dirty = true;
  invalidate(c);
  return MM_OK;
}

int mm_set_bext(mm_ctx* c, int region, const double b0[3], const double b1[3]) {
  if (!c || !b0) return fail(MM_ERR_ARG, "NULL argument");
  if (region < -1 || region >= kRegions) return fail(MM_ERR_ARG, "region must be -1..255");
  const int lo = region < 0 ? 0 : region, hi = region < 0 ? kRegions : region + 1;
  for (int r = lo; r < hi; ++r)
    for (int k = 0; k < 3; ++k) {
      c->b0[r][k] = b0[k];
      c->b1[r][k] = b1 ? b1[k] : 0.0;
    }
  c->lut_dirty = true;
  invalidate(c);
  return MM_OK;
}

int mm_set_bext_timefn(mm_ctx* c, double freq, double phase) {
  if (!c) return fail(MM_ERR_ARG, "ctx is NULL");
  c->freq = freq;
  c->phase = phase;
  c->graph_valid = false;
  invalidate(c);
  return MM_OK;
}

int mm_enable_terms(mm_ctx* c, int demag, int exch, int anis, int zeeman, int precession) {
  if (!c) return fail(MM_ERR_ARG, "ctx is NULL");
  c->T = Terms{demag != 0, exch != 0, anis != 0, zeeman != 0, c->T.dmi};
  int rc = read_state(c);
  if (rc) return rc;
  c->st_host->precession = precession != 0;
  rc = write_state(c);
  if (rc) return rc;
  c->graph_valid = false;
  invalidate(c);
  return MM_OK;
}

// Setting m to the value it already has (bit for bit, e.g. a host loop that
// writes back what it read) changes nothing: the cached first RK stage stays
// valid.  The data go to a scratch buffer first and are compared on the
// device; otherwise they replace m, are normalised and the cache is dropped.
static int set_m_common(mm_ctx* c, const float* src, cudaMemcpyKind kind) {
  int rc = flush_luts(c);
  if (rc) return rc;
  rc = current_state(c);
  if (rc) return rc;
  float* dst = c->b.m[c->st_host->parity];
  const size_t bytes = 3 * (size_t)c->g.n * sizeof(float);
  if (c->m_set && c->k1_valid) {
    int* flag = reinterpret_cast<int*>(c->b.acc + 15);   // (acc[15]: not used by the getters)
    MM_CUDA(cudaMemcpyAsync(c->b.out, src, bytes, kind, c->stream));
    MM_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), c->stream));
    launch_m_differs(c->g, c->b.out, dst, flag, c->stream);
    MM_CUDA(cudaGetLastError());
    int differs = 1;
    MM_CUDA(cudaMemcpyAsync(&differs, flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    MM_CUDA(cudaStreamSynchronize(c->stream));
    if (!differs) return MM_OK;
    MM_CUDA(cudaMemcpyAsync(dst, c->b.out, bytes, cudaMemcpyDeviceToDevice, c->stream));
  } else {
    MM_CUDA(cudaMemcpyAsync(dst, src, bytes, kind, c->stream));
  }
  launch_normalize(c->g, c->b, dst, c->stream);
  MM_CUDA(cudaGetLastError());
  MM_CUDA(cudaStreamSynchronize(c->stream));
  c->m_set = true;
  invalidate(c);
  return MM_OK;
}

int mm_set_m(mm_ctx* c, const float* m) {
  if (!c || !m) return fail(MM_ERR_ARG, "NULL argument");
  return set_m_common(c, m, cudaMemcpyHostToDevice);
}

int mm_set_m_device(mm_ctx* c, const float* m) {
  if (!c || !m) return fail(MM_ERR_ARG, "NULL argument");
  return set_m_common(c, m, cudaMemcpyDeviceToDevice);
}

static int get_m_common(mm_ctx* c, float* dst, cudaMemcpyKind kind) {
  int rc = current_state(c);
  if (rc) return rc;
  MM_CUDA(cudaMemcpyAsync(dst, c->b.m[c->st_host->parity], 3 * (size_t)c->g.n * sizeof(float), kind, c->stream));
  MM_CUDA(cudaStreamSynchronize(c->stream));
  return MM_OK;
}

int mm_get_m(mm_ctx* c, float* m) {
  if (!c || !m) return fail(MM_ERR_ARG, "NULL argument");
  return get_m_common(c, m, cudaMemcpyDeviceToHost);
}

int mm_get_m_device(mm_ctx* c, float* m) {
  if (!c || !m) return fail(MM_ERR_ARG, "NULL argument");
  return get_m_common(c, m, cudaMemcpyDeviceToDevice);
}

int mm_set_solver(mm_ctx* c, double max_err, double headroom, double dt0, double dt_min, double dt_max) {
  if (!c) return fail(MM_ERR_ARG, "ctx is NULL");
  if (!(max_err > 0) || !(headroom > 0) || !(dt0 > 0) || !(dt_min > 0) || !(dt_max >= dt_min))
    return fail(MM_ERR_ARG, "solver settings must be positive with dt_min <= dt_max");
  int rc = read_state(c);
  if (rc) return rc;
  DevState& s = *c->st_host;
  s.max_err = max_err;
  s.headroom = headroom;
  s.dt = std::min(std::max(dt0, dt_min), dt_max);
  s.dt_min = dt_min;
  s.dt_max = dt_max;
  return write_state(c);
}

int mm_set_wait_limit(mm_ctx* c, long long cycles) {
  if (!c) return fail(MM_ERR_ARG, "ctx is NULL");
  if (cycles < 0) return fail(MM_ERR_ARG, "the wait limit must be >= 0 cycles");
  int rc = read_state(c);
  if (rc) return rc;
  c->st_host->wait_cycles = cycles;
  return write_state(c);
}

int mm_get_wait_limit(mm_ctx* c, long long* cycles) {
  if (!c || !cycles) return fail(MM_ERR_ARG, "ctx and cycles must not be NULL");
  int rc = current_state(c);
  if (rc) return rc;
  *cycles = c->st_host->wait_cycles;
  return MM_OK;
}

int mm_set_fixed_dt_sequence(mm_ctx* c, const double* dts, int n) {
  if (!c) return fail(MM_ERR_ARG, "ctx is NULL");
  if (n < 0 || (n > 0 && !dts)) return fail(MM_ERR_ARG, "bad sequence");
  for (int i = 0; i < n; ++i)
    if (!(dts[i] > 0) || !std::isfinite(dts[i])) return fail(MM_ERR_ARG, "step sizes must be finite and > 0");
  if (n > c->fixed_cap) {
    if (c->b.fixed) cudaFree(c->b.fixed);
    c->b.fixed = nullptr;
    c->fixed_cap = 0;
    MM_CUDA(cudaMalloc((void**)&c->b.fixed, (size_t)n * sizeof(double)));
    c->fixed_cap = n;
    c->graph_valid = false;   // the error kernel's pointer changed
  }
  if (n > 0)
    MM_CUDA(cudaMemcpyAsync(c->b.fixed, dts, (size_t)n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  int rc = read_state(c);
  if (rc) return rc;
  c->st_host->fixed_idx = 0;
  c->st_host->fixed_n = n;
  c->fixed_n = n;
  return write_state(c);
}

// Exact-path check of the surrogate: relative L2 difference of the two
// demag fields at the current m; above the tolerance the context falls back
// to the exact convolution for the rest of its life.
static int surrogate_check(mm_ctx* c) {
  Buffers nb = c->b;
  nb.st = nullptr;
  launch_copy_mcur(c->g, c->b, c->b.ms, c->stream);
  demag_exact(c, nb, c->b.ms);                                     // exact -> bd
  launch_fno_demag(c->sur, c->g, c->b, c->b.ms, c->sur_inv_ref, c->sur_mu0_ref, c->b.out, c->stream);
  launch_rel_err(3 * c->g.n, c->b.out, c->b.bd, c->sur_acc, c->stream);
  double acc[2];
  MM_CUDA(cudaMemcpyAsync(acc, c->sur_acc, sizeof(acc), cudaMemcpyDeviceToHost, c->stream));
  MM_CUDA(cudaStreamSynchronize(c->stream));
  c->sur_checks++;
  c->sur_last_err = acc[1] > 0 ? std::sqrt(acc[0] / acc[1]) : 0.0;
  if (!(c->sur_last_err <= c->sur_tol)) {
    c->sur_active = false;
    c->sur_fallbacks++;
    c->graph_valid = false;
    c->k1_valid = false;   // the cached first stage used the surrogate field
  }
  return MM_OK;
}

int mm_step(mm_ctx* c, int n) {
  if (!c) return fail(MM_ERR_ARG, "ctx is NULL");
  if (n < 0) return fail(MM_ERR_ARG, "n must be >= 0");
  if (n == 0) return MM_OK;
  const int mode = c->fixed_n > 0 ? 2 : 0;
  if (!c->sur_active) return drive(c, mode, n, 0.0);
  // surrogate mode: chunks of sur_every steps, each judged by the exact path
  int left = n;
  while (left > 0) {
    const int chunk = c->sur_active ? std::min(left, c->sur_every) : left;
    const bool was_active = c->sur_active;
    int rc = drive(c, mode, chunk, 0.0);
    if (rc) return rc;
    if (was_active) c->sur_steps += chunk;
    left -= chunk;
    if (c->sur_active) {
      rc = surrogate_check(c);
      if (rc) return rc;
    }
  }
  return MM_OK;
}

int mm_run(mm_ctx* c, double t_end) {
  if (!c) return fail(MM_ERR_ARG, "ctx is NULL");
  if (!std::isfinite(t_end)) return fail(MM_ERR_ARG, "t_end must be finite");
  if (c->fixed_n > 0) return fail(MM_ERR_STATE, "run() is not available in replay mode");
  if (c->sur_active) return fail(MM_ERR_STATE, "run() is not available with the demag surrogate; use mm_step");
  return drive(c, 1, 0, t_end);
}

int mm_get_time(mm_ctx* c, double* t, double* dt) {
  if (!c) return fail(MM_ERR_ARG, "ctx is NULL");
  int rc = read_state(c);
  if (rc) return rc;
  if (t) *t = c->st_host->t;
  if (dt) *dt = c->st_host->dt;
  return MM_OK;
}

int mm_set_time(mm_ctx* c, double t, double dt) {
  if (!c) return fail(MM_ERR_ARG, "ctx is NULL");
  if (!std::isfinite(t) || !(dt > 0)) return fail(MM_ERR_ARG, "bad time or step");
  int rc = read_state(c);
  if (rc) return rc;
  c->st_host->t = t;
  c->st_host->dt = dt;
  invalidate(c);
  return write_state(c);
}

static int copy_out(mm_ctx* c, const float* src, float* dst) {
  MM_CUDA(cudaMemcpyAsync(dst, src, 3 * (size_t)c->g.n * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
  MM_CUDA(cudaStreamSynchronize(c->stream));
  return MM_OK;
}

int mm_get_beff(mm_ctx* c, float* b) {
  if (!c || !b) return fail(MM_ERR_ARG, "NULL argument");
  int rc = eval_field(c, 0);
  return rc ? rc : copy_out(c, c->b.out, b);
}

int mm_get_torque(mm_ctx* c, float* tau) {
  if (!c || !tau) return fail(MM_ERR_ARG, "NULL argument");
  int rc = eval_field(c, 1);
  return rc ? rc : copy_out(c, c->b.out, tau);
}

int mm_get_bdemag(mm_ctx* c, float* b) {
  if (!c || !b) return fail(MM_ERR_ARG, "NULL argument");
  int rc = eval_field(c, 3);
  return rc ? rc : copy_out(c, c->b.bd, b);
}

int mm_get_energies(mm_ctx* c, mm_energies* out) {
  if (!c || !out) return fail(MM_ERR_ARG, "NULL argument");
  int rc = eval_field(c, 2);
  if (rc) return rc;
  double acc[9];
  MM_CUDA(cudaMemcpyAsync(acc, c->b.acc, sizeof(acc), cudaMemcpyDeviceToHost, c->stream));
  MM_CUDA(cudaStreamSynchronize(c->stream));
  const double V = c->dx * c->dy * c->dz;
  out->demag = acc[0] * V;
  out->exch = acc[1] * V;
  out->anis = acc[2] * V;
  out->zeeman = acc[3] * V;
  out->dmi = acc[8] * V;
  out->total = out->demag + out->exch + out->anis + out->zeeman + out->dmi;
  for (int k = 0; k < 3; ++k) out->m_avg[k] = acc[7] > 0 ? acc[4 + k] / acc[7] : 0.0;
  return MM_OK;
}

int mm_enable_stt(mm_ctx* c, int zhang_li, int slonczewski) {
  if (!c) return fail(MM_ERR_ARG, "ctx is NULL");
  c->stt_zl = zhang_li != 0;
  c->stt_sl = slonczewski != 0;
  c->lut_dirty = true;   // the terms are switched on with the tables
  return MM_OK;
}

int mm_set_pbc(mm_ctx* c, int px, int py, int pz) {
  if (!c) return fail(MM_ERR_ARG, "ctx is NULL");
  const int pbc[3] = {px, py, pz};
  const int n[3] = {c->g.nx, c->g.ny, c->g.nz};
  for (int a = 0; a < 3; ++a) {
    if (pbc[a] < 0 || pbc[a] > 4096) return fail(MM_ERR_ARG, "periodic images must be 0..4096");
    const bool pow2 = (n[a] & (n[a] - 1)) == 0;
    if (pbc[a] > 0 && n[a] != 1 && (n[a] < 4 || !pow2))
      return fail(MM_ERR_ARG, "a periodic axis needs 1 cell or a power of two >= 4 cells");
  }
  Geom g = make_geom(c->g.nx, c->g.ny, c->g.nz, c->dx, c->dy, c->dz, pbc);
  fused_plan(g);
  MM_CUDA(cudaStreamSynchronize(c->stream));
  // buffers whose size depends on the transform lengths
  Buffers& b = c->b;
  void* old[] = {b.spec, b.kt, b.ktf, b.ms2, b.part};
  for (void* p : old)
    if (p) cudaFree(p);
  b.spec = nullptr;
  b.kt = b.ktf = nullptr;
  b.ms2 = nullptr;
  b.part = nullptr;
  c->graph_valid = false;
  c->k1_valid = false;
  const size_t vec = 3 * (size_t)g.n * sizeof(float);
  cudaError_t e = cudaMalloc((void**)&b.spec, 3 * (size_t)g.sc * sizeof(float2));
  if (e == cudaSuccess) e = cudaMemsetAsync(b.spec, 0, 3 * (size_t)g.sc * sizeof(float2), c->stream);
  if (e == cudaSuccess) e = cudaMalloc((void**)&b.kt, 6 * (size_t)g.hkx * g.hky * g.hkz * sizeof(float));
  if (e == cudaSuccess && g.fused) e = cudaMalloc((void**)&b.ktf, 6 * (size_t)g.hkx * g.hky * g.hkz * sizeof(float));
  if (e == cudaSuccess && g.fused) e = cudaMalloc((void**)&b.ms2, vec);
  if (e == cudaSuccess && g.fused) e = cudaMemsetAsync(b.ms2, 0, vec, c->stream);
  if (e == cudaSuccess && g.fused) e = cudaMalloc((void**)&b.part, vec);
  if (e == cudaSuccess && g.fused) e = cudaMemsetAsync(b.part, 0, vec, c->stream);
  if (e == cudaSuccess) e = build_kernel_spectrum(g, c->dx, c->dy, c->dz, b.kt, c->stream);
  if (e == cudaSuccess && g.fused) launch_kt_transpose(g, b.kt, b.ktf, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  c->g = g;
  if (e == cudaSuccess) {
    // the (y, z) buffer's size follows the transform lengths
    if (c->yzt) {
      cudaFree(c->yzt);
      c->yzt = nullptr;
    }
    c->yz3 = false;
    c->y2d = false;
    const int rc = apply_yz_choice(c);
    if (rc) return rc;
    // one convolution outside any capture (launch attributes), as at creation
    Buffers nb = b;
    nb.st = nullptr;
    demag_exact(c, nb, b.ms);
    e = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess) e = cudaGetLastError();
  }
  if (e == cudaSuccess && g.fused && g.pbcx == 0) e = prepare_rowstage(g);
  if (e == cudaSuccess) rowstage_maps(g, b, &c->maps);
  if (e != cudaSuccess)
    return fail(e == cudaErrorMemoryAllocation ? MM_ERR_OOM : MM_ERR_CUDA,
                std::string("set_pbc: ") + cudaGetErrorString(e));
  return MM_OK;
}

int mm_get_max_torque(mm_ctx* c, double* tau_max) {
  if (!c || !tau_max) return fail(MM_ERR_ARG, "NULL argument");
  int rc = eval_field(c, 4);
  if (rc) return rc;
  unsigned int bits = 0;
  MM_CUDA(cudaMemcpyAsync(&bits, c->b.acc, sizeof(bits), cudaMemcpyDeviceToHost, c->stream));
  MM_CUDA(cudaStreamSynchronize(c->stream));
  float v;
  std::memcpy(&v, &bits, sizeof(v));
  *tau_max = (double)v;
  return MM_OK;
}

int mm_set_integrator(mm_ctx* c, int method) {
  if (!c) return fail(MM_ERR_ARG, "ctx is NULL");
  if (method != MM_RK45 && method != MM_RK23) return fail(MM_ERR_ARG, "method must be MM_RK45 or MM_RK23");
  if (method == c->method) return MM_OK;
  int rc = read_state(c);
  if (rc) return rc;
  c->st_host->method = method;
  rc = write_state(c);
  if (rc) return rc;
  c->method = method;
  c->graph_valid = false;     // the cached first stage (torque at m) stays valid
  return MM_OK;
}

int mm_get_integrator(mm_ctx* c, int* method) {
  if (!c || !method) return fail(MM_ERR_ARG, "NULL argument");
  *method = c->method;
  return MM_OK;
}

// relax() (Sec. IV, "Energy minimization"): precession off, RK23; advance in
// blocks of kRelaxBlock accepted steps while the total energy decreases, then
// while the maximum torque decreases, lowering MaxErr by sqrt(2) each time it
// stops, until MaxErr <= 1e-9.  The solver, MaxErr and the precession switch
// are restored on every exit.
namespace {
constexpr int kRelaxBlock = 3;
constexpr double kRelaxMinErr = 1e-9;

int set_precession(mm_ctx* c, int on) {
  int rc = read_state(c);
  if (rc) return rc;
  if (c->st_host->precession == on) return MM_OK;
  c->st_host->precession = on;
  rc = write_state(c);
  if (rc) return rc;
  c->graph_valid = false;
  invalidate(c);              // the cached first-stage torque depends on it
  return MM_OK;
}

int set_max_err(mm_ctx* c, double e) {
  int rc = read_state(c);
  if (rc) return rc;
  c->st_host->max_err = e;
  return write_state(c);
}

int relax_body(mm_ctx* c, long long max_steps, long long* taken) {
  int rc = read_state(c);
  if (rc) return rc;
  const long long a0 = c->st_host->accepted;
  double max_err = c->st_host->max_err;
  auto steps_done = [&]() { return c->st_host->accepted - a0; };
  auto block = [&]() -> int {
    if (steps_done() + kRelaxBlock > max_steps) return fail(MM_ERR_TIMEOUT, "relax: step limit reached");
    int r = drive(c, 0, kRelaxBlock, 0.0);
    if (r) return r;
    *taken = steps_done();
    return MM_OK;
  };
  mm_energies e;
  rc = mm_get_energies(c, &e);
  if (rc) return rc;
  double e0 = e.total;
  for (;;) {
    rc = block();
    if (rc) return rc;
    rc = mm_get_energies(c, &e);
    if (rc) return rc;
    if (!(e.total < e0)) break;
    e0 = e.total;
  }
  double t0;
  rc = mm_get_max_torque(c, &t0);
  if (rc) return rc;
  for (;;) {
    rc = block();
    if (rc) return rc;
    double t1;
    rc = mm_get_max_torque(c, &t1);
    if (rc) return rc;
    if (t1 < t0) {
      t0 = t1;
      continue;
    }
    if (max_err <= kRelaxMinErr) break;
    max_err /= std::sqrt(2.0);
    rc = set_max_err(c, max_err);
    if (rc) return rc;
    t0 = t1;
  }
  return MM_OK;
}
}  // namespace

int mm_relax(mm_ctx* c, long long max_steps, long long* steps_taken) {
  if (!c) return fail(MM_ERR_ARG, "ctx is NULL");
  if (max_steps <= 0) return fail(MM_ERR_ARG, "max_steps must be > 0");
  if (!c->m_set) return fail(MM_ERR_STATE, "m has not been set");
  if (c->fixed_n > 0) return fail(MM_ERR_STATE, "relax() is not available in replay mode");
  if (c->sur_active) return fail(MM_ERR_STATE, "relax() is not available with the demag surrogate");
  int rc = read_state(c);
  if (rc) return rc;
  const int saved_prec = c->st_host->precession, saved_method = c->method;
  const double saved_err = c->st_host->max_err;
  long long taken = 0;
  rc = set_precession(c, 0);
  if (!rc) rc = mm_set_integrator(c, MM_RK23);
  if (!rc) rc = relax_body(c, max_steps, &taken);
  const std::string msg = rc ? g_err : std::string();
  // restore (errors here take precedence only if the relaxation succeeded)
  int r2 = set_max_err(c, saved_err);
  if (!r2) r2 = set_precession(c, saved_prec);
  if (!r2) r2 = mm_set_integrator(c, saved_method);
  if (steps_taken) *steps_taken = taken;
  if (rc) {
    g_err = msg;
    return rc;
  }
  return r2;
}

int mm_get_stats(mm_ctx* c, mm_stats* s) {
  if (!c || !s) return fail(MM_ERR_ARG, "NULL argument");
  int rc = read_state(c);
  if (rc) return rc;
  const DevState& d = *c->st_host;
  s->accepted = d.accepted;
  s->rejected = d.rejected;
  s->evals = d.evals;
  s->last_err = d.last_err;
  s->t = d.t;
  s->dt = d.dt;
  s->launches = c->launches;
  return MM_OK;
}

int mm_get_dt_history(mm_ctx* c, double* dts, int max, int* n) {
  if (!c || !n || (max > 0 && !dts)) return fail(MM_ERR_ARG, "NULL argument");
  int rc = read_state(c);
  if (rc) return rc;
  const int avail = std::min(c->st_host->hist_n, kHistCap);
  const int k = std::min(avail, std::max(max, 0));
  if (k > 0) {
    MM_CUDA(cudaMemcpyAsync(dts, c->b.hist, (size_t)k * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    MM_CUDA(cudaStreamSynchronize(c->stream));
  }
  *n = k;
  return MM_OK;
}

size_t mm_state_bytes(mm_ctx* c) {
  if (!c) return 0;
  return sizeof(StateBlobHeader) + sizeof(DevState) + 4 * 3 * (size_t)c->g.n * sizeof(float);
}

int mm_get_state(mm_ctx* c, void* buf, size_t bytes) {
  if (!c || !buf) return fail(MM_ERR_ARG, "NULL argument");
  if (bytes < mm_state_bytes(c)) return fail(MM_ERR_ARG, "buffer too small");
  int rc = read_state(c);
  if (rc) return rc;
  char* p = (char*)buf;
  StateBlobHeader h{0x6d6d3435u, c->g.nx, c->g.ny, c->g.nz, (unsigned)sizeof(DevState), c->k1_valid ? 1 : 0};
  std::memcpy(p, &h, sizeof(h));
  p += sizeof(h);
  std::memcpy(p, c->st_host, sizeof(DevState));
  p += sizeof(DevState);
  const size_t vb = 3 * (size_t)c->g.n * sizeof(float);
  float* src[4] = {c->b.m[0], c->b.m[1], c->b.k[0], c->b.k[6]};
  for (float* s : src) {
    MM_CUDA(cudaMemcpyAsync(p, s, vb, cudaMemcpyDeviceToHost, c->stream));
    p += vb;
  }
  MM_CUDA(cudaStreamSynchronize(c->stream));
  return MM_OK;
}

int mm_set_state(mm_ctx* c, const void* buf, size_t bytes) {
  if (!c || !buf) return fail(MM_ERR_ARG, "NULL argument");
  if (bytes < mm_state_bytes(c)) return fail(MM_ERR_ARG, "buffer too small");
  const char* p = (const char*)buf;
  StateBlobHeader h;
  std::memcpy(&h, p, sizeof(h));
  if (h.magic != 0x6d6d3435u || h.nx != c->g.nx || h.ny != c->g.ny || h.nz != c->g.nz ||
      h.devstate_size != sizeof(DevState))
    return fail(MM_ERR_ARG, "state blob does not match this context");
  p += sizeof(h);
  DevState s;
  std::memcpy(&s, p, sizeof(DevState));
  p += sizeof(DevState);
  s.done = 1;
  s.ticket = 0;
  s.err_bits = 0;
  s.fixed_idx = s.fixed_n = 0;   // the replay sequence is not part of a checkpoint
  c->fixed_n = 0;
  *c->st_host = s;
  int rc = write_state(c);
  if (rc) return rc;
  const size_t vb = 3 * (size_t)c->g.n * sizeof(float);
  float* dst[4] = {c->b.m[0], c->b.m[1], c->b.k[0], c->b.k[6]};
  for (float* d : dst) {
    MM_CUDA(cudaMemcpyAsync(d, p, vb, cudaMemcpyHostToDevice, c->stream));
    p += vb;
  }
  MM_CUDA(cudaStreamSynchronize(c->stream));
  c->m_set = true;
  c->k1_valid = h.k1_valid != 0;
  if (c->method != s.method) {
    c->method = s.method;
    c->graph_valid = false;
  }
  return MM_OK;
}

int mm_demag_tensor(int device, double dx, double dy, double dz, int n, const int32_t* offsets, double* out) {
  if (n < 0 || (n > 0 && (!offsets || !out))) return fail(MM_ERR_ARG, "bad arguments");
  if (!(dx > 0) || !(dy > 0) || !(dz > 0)) return fail(MM_ERR_ARG, "cell sizes must be > 0");
  if (n == 0) return MM_OK;
  MM_CUDA(cudaSetDevice(device));
  int32_t* d_off = nullptr;
  double* d_out = nullptr;
  cudaError_t e = cudaMalloc(&d_off, (size_t)n * 3 * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMalloc(&d_out, (size_t)n * 6 * sizeof(double));
  if (e == cudaSuccess) e = cudaMemcpy(d_off, offsets, (size_t)n * 3 * sizeof(int32_t), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = demag_tensor_offsets(n, d_off, dx, dy, dz, d_out, 0);
  if (e == cudaSuccess) e = cudaMemcpy(out, d_out, (size_t)n * 6 * sizeof(double), cudaMemcpyDeviceToHost);
  cudaFree(d_off);
  cudaFree(d_out);
  if (e != cudaSuccess) return fail(MM_ERR_CUDA, cudaGetErrorString(e));
  return MM_OK;
}

int mm_demag_apply(mm_ctx* c, const float* m, float* b) {
  if (!c || !m || !b) return fail(MM_ERR_ARG, "NULL argument");
  int rc = flush_luts(c);
  if (rc) return rc;
  Buffers nb = c->b;
  nb.st = nullptr;
  nb.bd = b;
  demag_exact(c, nb, m);
  MM_CUDA(cudaGetLastError());
  MM_CUDA(cudaStreamSynchronize(c->stream));
  return MM_OK;
}

int mm_set_demag_surrogate(mm_ctx* c, mm_fno* net, double ms_ref, int check_every, double fallback_rel_err) {
  if (!c) return fail(MM_ERR_ARG, "ctx is NULL");
  if (!net) {
    c->sur = nullptr;
    c->sur_active = false;
    c->graph_valid = false;
    c->k1_valid = false;
    return MM_OK;
  }
  if (!fno_matches(net, c->g)) return fail(MM_ERR_ARG, "surrogate grid differs from the context (2-D, same nx, ny)");
  if (!(ms_ref > 0) || check_every < 1 || !(fallback_rel_err > 0)) return fail(MM_ERR_ARG, "bad surrogate settings");
  if (!c->sur_acc) MM_CUDA(cudaMalloc((void**)&c->sur_acc, 2 * sizeof(double)));
  c->sur = net;
  c->sur_active = true;
  c->sur_every = check_every;
  c->sur_tol = fallback_rel_err;
  c->sur_inv_ref = (float)(1.0 / ms_ref);
  c->sur_mu0_ref = (float)(4e-7 * kPi * ms_ref);
  c->sur_steps = c->sur_checks = c->sur_fallbacks = 0;
  c->graph_valid = false;
  c->k1_valid = false;
  return MM_OK;
}

// Training pairs from the context's own exact trajectories, then Adam epochs
// on the GPU.  Each trajectory starts from m uniform on the sphere per cell
// under a static field of uniform direction and magnitude U[0, field_max];
// consecutive pairs are steps_between exact RK45 steps apart.  The context's
// m, time, fields and surrogate setting are restored afterwards.
int mm_surrogate_train(mm_ctx* c, mm_fno* net, double ms_ref, int n_pairs, int traj_len, int steps_between,
                       double field_max, int epochs, int batch, double lr, unsigned long long seed,
                       double* final_loss) {
  if (!c || !net) return fail(MM_ERR_ARG, "NULL argument");
  if (!fno_matches(net, c->g)) return fail(MM_ERR_ARG, "surrogate grid differs from the context (2-D, same nx, ny)");
  if (!(ms_ref > 0) || n_pairs < 1 || traj_len < 1 || steps_between < 0 || epochs < 0 || batch < 1 || !(lr > 0))
    return fail(MM_ERR_ARG, "bad training settings");
  const long long n3 = 3 * c->g.n;
  // save state
  std::vector<float> m_save(n3);
  int rc = mm_get_m(c, m_save.data());
  if (rc) return rc;
  double t_save, dt_save;
  rc = mm_get_time(c, &t_save, &dt_save);
  if (rc) return rc;
  double b0_save[kRegions][3], b1_save[kRegions][3];
  std::memcpy(b0_save, c->b0, sizeof(b0_save));
  std::memcpy(b1_save, c->b1, sizeof(b1_save));
  mm_fno* sur_save = c->sur;
  const bool active_save = c->sur_active;
  c->sur_active = false;
  c->graph_valid = false;
  c->k1_valid = false;
  float *U = nullptr, *Y = nullptr;
  cudaError_t e = cudaMalloc((void**)&U, (size_t)n_pairs * n3 * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc((void**)&Y, (size_t)n_pairs * n3 * sizeof(float));
  auto done = [&](int code) {
    cudaFree(U);
    cudaFree(Y);
    std::memcpy(c->b0, b0_save, sizeof(b0_save));
    std::memcpy(c->b1, b1_save, sizeof(b1_save));
    c->lut_dirty = true;
    mm_set_m(c, m_save.data());
    mm_set_time(c, t_save, dt_save);
    c->sur = sur_save;
    c->sur_active = active_save && sur_save;
    c->graph_valid = false;
    c->k1_valid = false;
    return code;
  };
  if (e != cudaSuccess) return done(fail(MM_ERR_OOM, "no room for the training pairs"));
  unsigned long long st = seed * 0x9E3779B97F4A7C15ULL + 7;
  auto unif = [&]() {   // splitmix64 -> (0, 1)
    st += 0x9E3779B97F4A7C15ULL;
    unsigned long long z = st;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    z ^= z >> 31;
    return ((z >> 11) + 0.5) * (1.0 / 9007199254740992.0);
  };
  auto normal = [&]() { return std::sqrt(-2.0 * std::log(unif())) * std::cos(2.0 * kPi * unif()); };
  std::vector<float> m0(n3);
  Buffers nb = c->b;
  nb.st = nullptr;
  const float inv_ref = (float)(1.0 / ms_ref), inv_mu = (float)(1.0 / (4e-7 * kPi * ms_ref));
  for (int p = 0; p < n_pairs; ++p) {
    if (p % traj_len == 0) {
      const long long n = c->g.n;
      for (long long i = 0; i < n; ++i) {
        double v[3] = {normal(), normal(), normal()};
        const double r = std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        for (int k = 0; k < 3; ++k) m0[k * n + i] = (float)(v[k] / r);
      }
      double d[3] = {normal(), normal(), normal()};
      const double r = std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
      const double mag = field_max * unif();
      for (int reg = 0; reg < kRegions; ++reg)
        for (int k = 0; k < 3; ++k) {
          c->b0[reg][k] = mag * d[k] / r;
          c->b1[reg][k] = 0.0;
        }
      c->lut_dirty = true;
      rc = mm_set_m(c, m0.data());
      if (rc == MM_OK) rc = mm_set_time(c, 0.0, 1e-14);
      if (rc) return done(rc);
    } else if (steps_between > 0) {
      rc = mm_step(c, steps_between);
      if (rc) return done(rc);
    }
    // pair: u = Msat m / ms_ref, y = B_demag / (mu0 ms_ref), exact convolution
    launch_copy_mcur(c->g, c->b, c->b.ms, c->stream);
    launch_to_u(c->g, c->b, c->b.ms, inv_ref, U + (size_t)p * n3, c->stream);
    demag_exact(c, nb, c->b.ms);
    launch_scale(n3, c->b.bd, inv_mu, Y + (size_t)p * n3, c->stream);
  }
  MM_CUDA(cudaStreamSynchronize(c->stream));
  // training: shuffled mini-batches, pairs gathered into contiguous staging
  float *ub = nullptr, *yb = nullptr;
  e = cudaMalloc((void**)&ub, (size_t)batch * n3 * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc((void**)&yb, (size_t)batch * n3 * sizeof(float));
  if (e != cudaSuccess) {
    cudaFree(ub);
    cudaFree(yb);
    return done(fail(MM_ERR_OOM, "no room for the training batch"));
  }
  std::vector<int> order(n_pairs);
  for (int i = 0; i < n_pairs; ++i) order[i] = i;
  double last = 0.0;
  for (int ep = 0; ep < epochs && rc == MM_OK; ++ep) {
    for (int i = n_pairs - 1; i > 0; --i) std::swap(order[i], order[(int)(unif() * (i + 1)) % (i + 1)]);
    for (int b0i = 0; b0i < n_pairs && rc == MM_OK; b0i += batch) {
      const int S = std::min(batch, n_pairs - b0i);
      for (int j = 0; j < S; ++j) {
        cudaMemcpyAsync(ub + (size_t)j * n3, U + (size_t)order[b0i + j] * n3, n3 * sizeof(float),
                        cudaMemcpyDeviceToDevice, c->stream);
        cudaMemcpyAsync(yb + (size_t)j * n3, Y + (size_t)order[b0i + j] * n3, n3 * sizeof(float),
                        cudaMemcpyDeviceToDevice, c->stream);
      }
      cudaStreamSynchronize(c->stream);
      rc = mm_fno_train_step(net, ub, yb, S, lr, &last);
    }
  }
  cudaFree(ub);
  cudaFree(yb);
  if (final_loss) *final_loss = last;
  return done(rc);
}

int mm_get_surrogate_stats(mm_ctx* c, long long* steps, long long* checks, long long* fallbacks, double* last_err,
                           int* active) {
  if (!c) return fail(MM_ERR_ARG, "ctx is NULL");
  if (steps) *steps = c->sur_steps;
  if (checks) *checks = c->sur_checks;
  if (fallbacks) *fallbacks = c->sur_fallbacks;
  if (last_err) *last_err = c->sur_last_err;
  if (active) *active = c->sur_active ? 1 : 0;
  return MM_OK;
}

int mm_sync(mm_ctx* c) {
  if (!c) return fail(MM_ERR_ARG, "ctx is NULL");
  MM_CUDA(cudaStreamSynchronize(c->stream));
  return MM_OK;
}

int mm_set_yz_kernels(mm_ctx* c, int which, int* active) {
  if (!c) return fail(MM_ERR_ARG, "ctx is NULL");
  if (which < 0 || which > 2) return fail(MM_ERR_ARG, "which must be 0 (default), 1 (cluster) or 2 (three kernels)");
  if (which == 2 && !yz3_plan(c->g) && !y2d_plan(c->g))
    return fail(MM_ERR_ARG, "the register-resident (y, z) kernels need open y and z axes and, in 3-D, py >= 32 and "
                            "16 <= pz <= 64, in 2-D py of 128, 256 or 512");
  MM_CUDA(cudaStreamSynchronize(c->stream));
  c->yz_req = which;
  c->graph_valid = false;   // the captured attempt holds the previous kernels
  const int rc = apply_yz_choice(c);
  if (rc) return rc;
  if (c->yz3 || c->y2d) {
    // one convolution outside any capture (launch attributes)
    Buffers nb = c->b;
    nb.st = nullptr;
    demag_exact(c, nb, c->b.ms);
    MM_CUDA(cudaStreamSynchronize(c->stream));
    MM_CUDA(cudaGetLastError());
  }
  if (active) *active = c->g.fused ? ((c->yz3 || c->y2d) ? 2 : 1) : 0;
  return MM_OK;
}

int mm_profile_attempts(mm_ctx* c, int attempts, int max, int* kinds, double* us, int* n_out) {
  if (!c || attempts < 1 || max < 1 || !kinds || !us || !n_out) return fail(MM_ERR_ARG, "bad profiling arguments");
  if (!c->m_set) return fail(MM_ERR_STATE, "m has not been set");
  if (!rowstage_path(c)) return fail(MM_ERR_STATE, "profiling covers the fused row-stage path only");
  int rc = flush_luts(c);
  if (rc) return rc;
  // launch positions of one attempt: the prep kernel, then per stage the
  // (y, z) kernel(s) (with demag), the earlier-stage sums (here in line, in
  // the graph a branch beside the (y, z) part) and the row kernel
  std::vector<int> kind;
  kind.push_back(0);
  for (int s = 1; s < 7; ++s) {
    if (c->T.demag) {
      if (c->yz3) {
        kind.push_back(3);
        kind.push_back(4);
        kind.push_back(5);
      } else {
        kind.push_back(1);
      }
    }
    if (partial_branch(c)) kind.push_back(6);
    kind.push_back(2);
  }
  const int P = (int)kind.size();
  std::vector<cudaEvent_t> ev((size_t)P * attempts + 1, nullptr);
  auto destroy = [&]() {
    for (cudaEvent_t e : ev)
      if (e) cudaEventDestroy(e);
  };
  for (auto& e : ev) {
    const cudaError_t er = cudaEventCreate(&e);
    if (er != cudaSuccess) {
      destroy();
      return fail(MM_ERR_CUDA, std::string("cudaEventCreate: ") + cudaGetErrorString(er));
    }
  }
  c->st_fresh = false;
  launch_begin_mode(c->b, 0, attempts, 0.0, c->stream);
  c->launches += 1;
  const bool k1_was_valid = c->k1_valid;
  if (!c->k1_valid) enqueue_k1(c);
  size_t q = 0;
  const Buffers rb = row_buffers(c);
  cudaError_t e = cudaEventRecord(ev[q++], c->stream);
  for (int a = 0; a < attempts && e == cudaSuccess; ++a) {
    launch_rowstage(c->g, c->b, c->T, c->maps, 0, 1, 0, c->freq, c->phase, c->stream);
    e = cudaEventRecord(ev[q++], c->stream);
    for (int s = 1; s < 7 && e == cudaSuccess; ++s) {
      if (c->T.demag && c->yz3) {
        // the three kernels of launch_demag_yz3, one event after each
        launch_yz3_part(c->g, c->b, c->yzt, 0, c->stream);
        e = cudaEventRecord(ev[q++], c->stream);
        launch_yz3_part(c->g, c->b, c->yzt, 1, c->stream);
        if (e == cudaSuccess) e = cudaEventRecord(ev[q++], c->stream);
        launch_yz3_part(c->g, c->b, c->yzt, 2, c->stream);
        if (e == cudaSuccess) e = cudaEventRecord(ev[q++], c->stream);
      } else if (c->T.demag) {
        demag_yz(c);
        e = cudaEventRecord(ev[q++], c->stream);
      }
      if (partial_branch(c)) {
        launch_rs_partial(c->g, c->b, s, s < 6 ? 1 : 2, c->stream);
        if (e == cudaSuccess) e = cudaEventRecord(ev[q++], c->stream);
      }
      launch_rowstage(c->g, rb, c->T, c->maps, 1, s, s < 6 ? 1 : 2, c->freq, c->phase, c->stream, row_dep(c));
      if (e == cudaSuccess) e = cudaEventRecord(ev[q++], c->stream);
    }
  }
  c->launches += (long long)attempts * P;
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  std::vector<double> sum(P, 0.0);
  for (size_t i = 1; i < q && e == cudaSuccess; ++i) {
    float ms = 0.f;
    e = cudaEventElapsedTime(&ms, ev[i - 1], ev[i]);
    sum[(i - 1) % P] += ms * 1e3;
  }
  destroy();
  if (e != cudaSuccess) return fail(MM_ERR_CUDA, std::string("profiled attempts: ") + cudaGetErrorString(e));
  rc = read_state(c);
  if (rc) return rc;
  c->k1_valid = k1_was_valid || c->st_host->call_attempts > 0;
  const int n = std::min(P, max);
  for (int i = 0; i < n; ++i) {
    kinds[i] = kind[i];
    us[i] = sum[i] / attempts;
  }
  *n_out = n;
  return status_to_code(c->st_host->status);
}

}  // extern "C"
