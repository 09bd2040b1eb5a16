// Batched RK45: many independent simulations of uneven grid sizes in one
// graph launch, each with its own adaptive step (Sec. IV) and its own
// material and field.
//
// Instances with the same grid and cell size form a shape class; a class
// shares one demag kernel spectrum and runs every kernel over all its
// instances at once (an instance index in the grid).  Each instance keeps its
// own t, dt, accept/reject decision and FSAL buffer roles (InstState).  One
// "batched attempt" advances every unfinished instance by one RK45 attempt;
// the classes are independent branches of the captured graph.  The whole run
// is a single CUDA graph launch: a conditional while node repeats the batched
// attempt until every instance has reached t_end (or the attempt cap of one
// launch is hit, after which the host launches the graph again).
//
// Instances in this path: one material per instance, every cell magnetic,
// static applied field, demag + exchange + Zeeman (no anisotropy).
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/mm.h"
#include "mm_internal.h"

namespace mm {
namespace {

constexpr int kBatchHist = 4096;
constexpr unsigned kMaxAttemptsPerLaunch = 200000;

// (the instances' fields are static, so the stage nodes c_s are not needed)
__constant__ double bA[7][6] = {
    {0, 0, 0, 0, 0, 0},
    {1.0 / 5.0, 0, 0, 0, 0, 0},
    {3.0 / 40.0, 9.0 / 40.0, 0, 0, 0, 0},
    {44.0 / 45.0, -56.0 / 15.0, 32.0 / 9.0, 0, 0, 0},
    {19372.0 / 6561.0, -25360.0 / 2187.0, 64448.0 / 6561.0, -212.0 / 729.0, 0, 0},
    {9017.0 / 3168.0, -355.0 / 33.0, 46732.0 / 5247.0, 49.0 / 176.0, -5103.0 / 18656.0, 0},
    {35.0 / 384.0, 0.0, 500.0 / 1113.0, 125.0 / 192.0, -2187.0 / 6784.0, 11.0 / 84.0}};
__constant__ double bE[7] = {71.0 / 57600.0,      0.0,           -71.0 / 16695.0, 71.0 / 1920.0,
                             -17253.0 / 339200.0, 22.0 / 525.0, -1.0 / 40.0};

struct InstState {
  double t, dt, h, t_end, last_err;
  double max_err, headroom, dt_min, dt_max;
  long long accepted, rejected;
  int parity, done, status, hist_n;
  unsigned int err_bits, ticket;
  float ah[7][6];
  float eh[7];
};

struct InstParams {
  float msat, alpha, gfac, exch;   // exch = 2 Aex / Msat
  float b[3];
};

struct BPtrs {
  float* m0;
  float* m1;
  float* k[7];
};

__device__ __forceinline__ float* bpick(const BPtrs& p, int j) {
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

__device__ __forceinline__ int role(int j, int parity) {
  return j == 0 ? (parity ? 6 : 0) : (j == 6 ? (parity ? 0 : 6) : j);
}

__device__ void prepare(InstState& s) {
  const double h = fmin(s.dt, s.t_end - s.t);
  s.h = h;
  for (int i = 0; i < 7; ++i) {
    for (int j = 0; j < 6; ++j) s.ah[i][j] = (float)(bA[i][j] * h);
    s.eh[i] = (float)(bE[i] * h);
  }
}

__global__ void k_b_begin(InstState* st, int n, double t_end) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  InstState& s = st[i];
  s.status = 0;
  s.err_bits = 0;
  s.ticket = 0;
  s.t_end = t_end;
  s.done = s.t >= t_end ? 1 : 0;
  if (!s.done) prepare(s);
}

__global__ void k_b_stage_input(Geom g, BPtrs p, float* __restrict__ ms, const InstState* __restrict__ st, int s) {
  const int inst = blockIdx.y;
  const InstState& S = st[inst];
  if (S.done) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;   // in-instance offsets: 3 n < 2^31
  if (i >= g.n) return;
  const long long o = (long long)inst * 3 * g.n;
  const int n = (int)g.n;
  const int par = S.parity;
  const float* __restrict__ m = (par ? p.m1 : p.m0) + o;
  float a0 = m[i], a1 = m[n + i], a2 = m[2 * n + i];
  for (int j = 0; j < s; ++j) {
    const float a = S.ah[s][j];
    if (a == 0.0f) continue;
    const float* __restrict__ k = bpick(p, role(j, par)) + o;
    a0 = fmaf(a, k[i], a0);
    a1 = fmaf(a, k[n + i], a1);
    a2 = fmaf(a, k[2 * n + i], a2);
  }
  float* __restrict__ mso = ms + o;
  mso[i] = a0;
  mso[n + i] = a1;
  mso[2 * n + i] = a2;
}

// effective field (demag + exchange + static Zeeman) and LL torque
__global__ void k_b_torque(Geom g, BPtrs p, const float* __restrict__ ms, const float* __restrict__ bd,
                           const InstParams* __restrict__ prm, const InstState* __restrict__ st, int s) {
  const int inst = blockIdx.y;
  const InstState& S = st[inst];
  if (S.done) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;   // in-instance offsets: 3 n < 2^31
  if (i >= g.n) return;
  const long long o = (long long)inst * 3 * g.n;
  const int n = (int)g.n;
  const float* __restrict__ m = ms + o;
  const float* __restrict__ bdo = bd + o;
  const InstParams P = prm[inst];
  const int x = i % g.nx, y = (i / g.nx) % g.ny, z = i / (g.nx * g.ny);
  const float mx = m[i], my = m[n + i], mz = m[2 * n + i];
  float bx = bdo[i] + P.b[0], by = bdo[n + i] + P.b[1], bz = bdo[2 * n + i] + P.b[2];
  auto nb = [&](int j, float id2) {
    const float c = P.exch * id2;
    bx += c * (m[j] - mx);
    by += c * (m[n + j] - my);
    bz += c * (m[2 * n + j] - mz);
  };
  const int sy = g.nx, sz = g.nx * g.ny;
  if (x > 0) nb(i - 1, g.idx2);
  if (x < g.nx - 1) nb(i + 1, g.idx2);
  if (y > 0) nb(i - sy, g.idy2);
  if (y < g.ny - 1) nb(i + sy, g.idy2);
  if (z > 0) nb(i - sz, g.idz2);
  if (z < g.nz - 1) nb(i + sz, g.idz2);
  const float cx = my * bz - mz * by, cy = mz * bx - mx * bz, cz = mx * by - my * bx;
  const float dx = my * cz - mz * cy, dy = mz * cx - mx * cz, dz = mx * cy - my * cx;
  float* __restrict__ k = bpick(p, role(s, S.parity)) + o;
  k[i] = P.gfac * (cx + P.alpha * dx);
  k[n + i] = P.gfac * (cy + P.alpha * dy);
  k[2 * n + i] = P.gfac * (cz + P.alpha * dz);
}

// Sec. IV controller, per instance (the same readings as the single path).
__device__ void b_controller(InstState& s, double* __restrict__ hist) {
  const double eps = (double)__uint_as_float(s.err_bits);
  s.err_bits = 0;
  s.ticket = 0;
  s.last_err = eps;
  if (!(eps <= DBL_MAX)) {
    s.status = MM_ERR_NONFINITE;
    s.done = 1;
    return;
  }
  const double h = s.h;
  // (the growth factor in float32, as in the single-context controller)
  const float ratio = (float)s.max_err / (float)eps;
  const double factor = eps == 0.0 ? 5.0 : (double)fminf(5.0f, fmaxf(0.2f, (float)s.headroom * powf(ratio, 0.2f)));
  const double ndt = fmin(h * factor, s.dt_max);
  if (eps <= s.max_err) {
    s.t += h;
    if (s.t + 1e-6 * h >= s.t_end) s.t = s.t_end;
    s.parity ^= 1;
    if (s.hist_n < kBatchHist) hist[s.hist_n] = h;
    s.hist_n++;
    s.accepted++;
    s.dt = fmax(ndt, s.dt_min);
    if (s.t >= s.t_end) s.done = 1;
  } else {
    s.rejected++;
    if (ndt < s.dt_min) {
      s.status = MM_ERR_DT_UNDERFLOW;
      s.done = 1;
      return;
    }
    s.dt = ndt;
  }
  if (!s.done) prepare(s);
}

__global__ void k_b_error(Geom g, BPtrs p, const float* __restrict__ ms, InstState* __restrict__ st,
                          double* __restrict__ hist) {
  const int inst = blockIdx.y;
  InstState& S = st[inst];
  if (S.done) return;   // uniform over the instance's blocks
  const int i = blockIdx.x * blockDim.x + threadIdx.x;   // in-instance offsets: 3 n < 2^31
  const long long o = (long long)inst * 3 * g.n;
  const int n = (int)g.n;
  const int par = S.parity;
  float e = 0.0f;
  if (i < n) {
    float ex = 0.f, ey = 0.f, ez = 0.f;
    for (int j = 0; j < 7; ++j) {
      const float c = S.eh[j];
      if (c == 0.0f) continue;
      const float* __restrict__ k = bpick(p, role(j, par)) + o;
      ex = fmaf(c, k[i], ex);
      ey = fmaf(c, k[n + i], ey);
      ez = fmaf(c, k[2 * n + i], ez);
    }
    e = sqrtf(ex * ex + ey * ey + ez * ez);
    if (!(e <= FLT_MAX)) e = __int_as_float(0x7f800000);
    float* __restrict__ mnew = (par ? p.m0 : p.m1) + o;
    const float* __restrict__ mso = ms + o;
    const float mx = mso[i], my = mso[n + i], mz = mso[2 * n + i];
    const float inv = rsqrtf(mx * mx + my * my + mz * mz);
    mnew[i] = mx * inv;
    mnew[n + i] = my * inv;
    mnew[2 * n + i] = mz * inv;
  }
  for (int off = 16; off > 0; off >>= 1) e = fmaxf(e, __shfl_xor_sync(0xffffffffu, e, off));
  __shared__ float wmax[32];
  if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = e;
  __syncthreads();
  if (threadIdx.x < 32) {
    float v = threadIdx.x < (blockDim.x >> 5) ? wmax[threadIdx.x] : 0.0f;
    for (int off = 16; off > 0; off >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, off));
    if (threadIdx.x == 0) {
      atomicMax(&S.err_bits, __float_as_uint(v));
      __threadfence();
      const unsigned int t = atomicAdd(&S.ticket, 1u);
      if (t == gridDim.x - 1) {
        __threadfence();
        b_controller(S, hist + (long long)inst * kBatchHist);
      }
    }
  }
}

// Keeps the while node looping while any instance is unfinished, at most
// kMaxAttemptsPerLaunch batched attempts per graph launch.
__global__ void k_b_cond(cudaGraphConditionalHandle handle, const InstState* __restrict__ st, int n,
                         unsigned int* attempts) {
  __shared__ int active;
  if (threadIdx.x == 0) active = 0;
  __syncthreads();
  int mine = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) mine |= !st[i].done;
  if (mine) atomicOr(&active, 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned int a = ++(*attempts);
    cudaGraphSetConditional(handle, (active && a < kMaxAttemptsPerLaunch) ? 1u : 0u);
  }
}

__global__ void k_b_normalize(float* __restrict__ m, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float x = m[i], y = m[n + i], z = m[2 * n + i];
  const float r2 = x * x + y * y + z * z;
  const float inv = r2 > 0.0f ? rsqrtf(r2) : 0.0f;
  m[i] = x * inv;
  m[n + i] = y * inv;
  m[2 * n + i] = z * inv;
}

constexpr int kT = 256;

}  // namespace

struct BClass {
  Geom g{};
  int B = 0;
  int first = 0;            // offset of its first instance in the state array
  std::vector<int> ids;     // global instance indices
  Buffers b{};
  float* msat = nullptr;
  InstParams* prm = nullptr;
  double* hist = nullptr;
  float conv_us = 0.f;      // autotuned convolution time of the whole class
};

}  // namespace mm

using namespace mm;

struct mm_batch {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int n = 0;
  std::vector<BClass> cls;
  std::vector<int> cls_of, slot_of;   // instance -> class, slot within the state array
  InstState* st = nullptr;            // [n], grouped by class
  unsigned int* attempts = nullptr;
  float2* tw = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<cudaStream_t> side;
  std::vector<cudaEvent_t> ev;
  bool k1_valid = false;
  std::vector<InstState> host_st;
};

namespace {

int bfail(int code, const std::string& msg) {
  mm::set_last_error(msg);
  return code;
}

#define MMB_CUDA(call)                                                                        \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess)                                                                    \
      return bfail(e_ == cudaErrorMemoryAllocation ? MM_ERR_OOM : MM_ERR_CUDA,                \
                   std::string(#call) + ": " + cudaGetErrorString(e_));                       \
  } while (0)

BPtrs bptrs(const BClass& c) {
  BPtrs p;
  p.m0 = c.b.m[0];
  p.m1 = c.b.m[1];
  for (int j = 0; j < 7; ++j) p.k[j] = c.b.k[j];
  return p;
}

BatchArgs bargs(const mm_batch* B, const BClass& c) {
  return BatchArgs{c.B, c.msat, &B->st[c.first].done, (int)(sizeof(InstState) / sizeof(int))};
}

// stage s of every unfinished instance of class c (s = 0: first stage at m)
void enqueue_stage(mm_batch* B, BClass& c, int s, cudaStream_t st) {
  const Geom& g = c.g;
  dim3 grid((unsigned)((g.n + kT - 1) / kT), c.B);
  k_b_stage_input<<<grid, kT, 0, st>>>(g, bptrs(c), c.b.ms, B->st + c.first, s);
  Buffers bb = c.b;
  bb.st = nullptr;
  launch_demag_fused_batch(g, bb, c.b.ms, st, bargs(B, c));
  k_b_torque<<<grid, kT, 0, st>>>(g, bptrs(c), c.b.ms, c.b.bd, c.prm, B->st + c.first, s);
}

void enqueue_attempt(mm_batch* B, BClass& c, cudaStream_t st) {
  for (int s = 1; s < 7; ++s) enqueue_stage(B, c, s, st);
  dim3 grid((unsigned)((c.g.n + kT - 1) / kT), c.B);
  k_b_error<<<grid, kT, 0, st>>>(c.g, bptrs(c), c.b.ms, B->st + c.first, c.hist);
}

int build_batch_graph(mm_batch* B) {
  if (B->exec) return MM_OK;
  cudaGraph_t graph = nullptr;
  MMB_CUDA(cudaGraphCreate(&graph, 0));
  cudaGraphConditionalHandle handle;
  MMB_CUDA(cudaGraphConditionalHandleCreate(&handle, graph, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams prm = {};
  prm.type = cudaGraphNodeTypeConditional;
  prm.conditional.handle = handle;
  prm.conditional.type = cudaGraphCondTypeWhile;
  prm.conditional.size = 1;
  cudaGraphNode_t node;
  MMB_CUDA(cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &prm));
  cudaGraph_t body = prm.conditional.phGraph_out[0];
  // body: one batched attempt, the shape classes as parallel branches
  MMB_CUDA(cudaStreamBeginCaptureToGraph(B->stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  const int nc = (int)B->cls.size();
  MMB_CUDA(cudaEventRecord(B->ev[0], B->stream));
  for (int c = 0; c < nc; ++c) {
    MMB_CUDA(cudaStreamWaitEvent(B->side[c], B->ev[0], 0));
    enqueue_attempt(B, B->cls[c], B->side[c]);
    MMB_CUDA(cudaEventRecord(B->ev[1 + c], B->side[c]));
    MMB_CUDA(cudaStreamWaitEvent(B->stream, B->ev[1 + c], 0));
  }
  k_b_cond<<<1, 256, 0, B->stream>>>(handle, B->st, B->n, B->attempts);
  cudaGraph_t captured = nullptr;
  cudaError_t e = cudaStreamEndCapture(B->stream, &captured);
  if (e != cudaSuccess) {
    cudaGraphDestroy(graph);
    return bfail(MM_ERR_CUDA, std::string("batch capture: ") + cudaGetErrorString(e));
  }
  e = cudaGraphInstantiate(&B->exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return bfail(MM_ERR_CUDA, std::string("batch graph: ") + cudaGetErrorString(e));
  return MM_OK;
}

// FFT tile autotuner: for one class, time the convolution of all its
// instances for every residue split and x-row block size the fused plan
// allows (2 warm-up + 3 timed launches each, on the class's own buffers)
// and keep the fastest.  Runs before any instance is marked done.
int tune_class(mm_batch* B, BClass& C) {
  int sp[4][2];
  const int nsp = fused_splits(C.g, sp, 4);
  int xr[3];
  const int nxr = fused_xrows(C.g, xr, 3);
  cudaEvent_t a = nullptr, z = nullptr;
  MMB_CUDA(cudaEventCreate(&a));
  MMB_CUDA(cudaEventCreate(&z));
  Buffers bb = C.b;
  bb.st = nullptr;
  float best = 1e30f;
  Geom bestg = C.g;
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < nsp && e == cudaSuccess; ++i)
    for (int j = 0; j < nxr && e == cudaSuccess; ++j) {
      Geom g = C.g;
      fused_set_split(g, sp[i][0], sp[i][1]);
      g.xrows = xr[j];
      for (int w = 0; w < 2; ++w) launch_demag_fused_batch(g, bb, C.b.ms, B->stream, bargs(B, C));
      e = cudaEventRecord(a, B->stream);
      for (int r = 0; r < 3; ++r) launch_demag_fused_batch(g, bb, C.b.ms, B->stream, bargs(B, C));
      if (e == cudaSuccess) e = cudaEventRecord(z, B->stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(z);
      if (e == cudaSuccess) e = cudaGetLastError();
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, z);
      if (e == cudaSuccess && ms / 3 < best) {
        best = ms / 3;
        bestg = g;
      }
    }
  cudaEventDestroy(a);
  cudaEventDestroy(z);
  if (e != cudaSuccess) return bfail(MM_ERR_CUDA, std::string("batch autotune: ") + cudaGetErrorString(e));
  C.g = bestg;
  C.conv_us = best * 1e3f;
  return MM_OK;
}

int read_states(mm_batch* B) {
  B->host_st.resize(B->n);
  MMB_CUDA(cudaMemcpyAsync(B->host_st.data(), B->st, B->n * sizeof(InstState), cudaMemcpyDeviceToHost, B->stream));
  MMB_CUDA(cudaStreamSynchronize(B->stream));
  return MM_OK;
}

int write_states(mm_batch* B) {
  MMB_CUDA(cudaMemcpyAsync(B->st, B->host_st.data(), B->n * sizeof(InstState), cudaMemcpyHostToDevice, B->stream));
  MMB_CUDA(cudaStreamSynchronize(B->stream));
  return MM_OK;
}

}  // namespace

extern "C" {

int mm_batch_create(mm_batch** out, int n, const mm_instance_spec* specs, int device, void* stream) {
  if (!out) return bfail(MM_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (n < 1 || !specs) return bfail(MM_ERR_ARG, "need n >= 1 instance specs");
  for (int i = 0; i < n; ++i) {
    const mm_instance_spec& s = specs[i];
    if (s.nx < 1 || s.ny < 1 || s.nz < 1 || s.nx > 1024 || s.ny > 512 || s.nz > 512)
      return bfail(MM_ERR_ARG, "instance grid out of range");
    if (!(s.dx > 0) || !(s.dy > 0) || !(s.dz > 0) || !(s.msat > 0) || s.aex < 0 || s.alpha < 0)
      return bfail(MM_ERR_ARG, "instance cell sizes and Msat must be > 0, Aex and alpha >= 0");
  }
  MMB_CUDA(cudaSetDevice(device));
  mm_batch* B = new mm_batch();
  B->device = device;
  B->n = n;
  auto cleanup = [&](int code) {
    mm_batch_destroy(B);
    return code;
  };
  // group into shape classes
  std::map<std::tuple<int, int, int, double, double, double>, int> key2c;
  B->cls_of.assign(n, 0);
  for (int i = 0; i < n; ++i) {
    const mm_instance_spec& s = specs[i];
    auto key = std::make_tuple(s.nx, s.ny, s.nz, s.dx, s.dy, s.dz);
    auto it = key2c.find(key);
    int c;
    if (it == key2c.end()) {
      c = (int)B->cls.size();
      key2c[key] = c;
      B->cls.emplace_back();
      B->cls[c].g = make_geom(s.nx, s.ny, s.nz, s.dx, s.dy, s.dz);
      if (!fused_plan(B->cls[c].g))
        return cleanup(bfail(MM_ERR_ARG, "batched path needs nx >= 17 and a (y, z) plane that fits one cluster"));
    } else {
      c = it->second;
    }
    B->cls_of[i] = c;
    B->cls[c].ids.push_back(i);
  }
  cudaError_t e = cudaSuccess;
  if (stream) {
    B->stream = (cudaStream_t)stream;
  } else {
    e = cudaStreamCreateWithFlags(&B->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cleanup(bfail(MM_ERR_CUDA, cudaGetErrorString(e)));
    B->own_stream = true;
  }
  const int nc = (int)B->cls.size();
  B->side.assign(nc, nullptr);
  B->ev.assign(nc + 1, nullptr);
  for (int c = 0; c < nc && e == cudaSuccess; ++c) e = cudaStreamCreateWithFlags(&B->side[c], cudaStreamNonBlocking);
  for (int c = 0; c <= nc && e == cudaSuccess; ++c) e = cudaEventCreateWithFlags(&B->ev[c], cudaEventDisableTiming);
  if (e != cudaSuccess) return cleanup(bfail(MM_ERR_CUDA, cudaGetErrorString(e)));
  auto alloc = [&](void** p, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) e = cudaMemsetAsync(*p, 0, bytes, B->stream);
  };
  alloc((void**)&B->st, n * sizeof(InstState));
  alloc((void**)&B->attempts, sizeof(unsigned int));
  alloc((void**)&B->tw, 2048 * sizeof(float2));
  std::vector<float2> tw(2048);
  for (int k = 0; k < 2048; ++k) {
    const double a = -2.0 * 3.14159265358979323846 * k / 2048.0;
    tw[k] = make_float2((float)std::cos(a), (float)std::sin(a));
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(B->tw, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice, B->stream);
  int first = 0;
  B->slot_of.assign(n, 0);
  for (int c = 0; c < nc && e == cudaSuccess; ++c) {
    BClass& C = B->cls[c];
    C.B = (int)C.ids.size();
    C.first = first;
    for (int j = 0; j < C.B; ++j) B->slot_of[C.ids[j]] = first + j;
    first += C.B;
    const Geom& g = C.g;
    const size_t vec = (size_t)C.B * 3 * g.n * sizeof(float);
    alloc((void**)&C.b.m[0], vec);
    alloc((void**)&C.b.m[1], vec);
    for (int j = 0; j < 7; ++j) alloc((void**)&C.b.k[j], vec);
    alloc((void**)&C.b.ms, vec);
    alloc((void**)&C.b.bd, vec);
    alloc((void**)&C.b.spec, (size_t)C.B * 3 * g.hx * g.nz * g.ny * sizeof(float2));
    alloc((void**)&C.b.kt, 6 * (size_t)g.hkx * g.hky * g.hkz * sizeof(float));
    alloc((void**)&C.b.ktf, 6 * (size_t)g.hkx * g.hky * g.hkz * sizeof(float));
    alloc((void**)&C.msat, C.B * sizeof(float));
    alloc((void**)&C.prm, C.B * sizeof(InstParams));
    alloc((void**)&C.hist, (size_t)C.B * kBatchHist * sizeof(double));
    C.b.tw = B->tw;
    if (e != cudaSuccess) break;
    std::vector<float> ms(C.B);
    std::vector<InstParams> pr(C.B);
    for (int j = 0; j < C.B; ++j) {
      const mm_instance_spec& s = specs[C.ids[j]];
      ms[j] = (float)s.msat;
      pr[j].msat = (float)s.msat;
      pr[j].alpha = (float)s.alpha;
      pr[j].gfac = (float)(-(s.gamma_ll > 0 ? s.gamma_ll : 1.7595e11) / (1.0 + s.alpha * s.alpha));
      pr[j].exch = (float)(2.0 * s.aex / s.msat);
      for (int k = 0; k < 3; ++k) pr[j].b[k] = (float)s.bext[k];
    }
    e = cudaMemcpyAsync(C.msat, ms.data(), C.B * sizeof(float), cudaMemcpyHostToDevice, B->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(C.prm, pr.data(), C.B * sizeof(InstParams), cudaMemcpyHostToDevice, B->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(B->stream);
    if (e == cudaSuccess) e = build_kernel_spectrum(g, specs[C.ids[0]].dx, specs[C.ids[0]].dy, specs[C.ids[0]].dz, C.b.kt, B->stream);
    if (e == cudaSuccess) {
      launch_kt_transpose(g, C.b.kt, C.b.ktf, B->stream);
      e = cudaStreamSynchronize(B->stream);
    }
  }
  if (e != cudaSuccess)
    return cleanup(bfail(e == cudaErrorMemoryAllocation ? MM_ERR_OOM : MM_ERR_CUDA, cudaGetErrorString(e)));
  // FFT tiles per class (instances are not yet marked done, buffers are zero)
  for (int c = 0; c < nc; ++c) {
    const int rc = tune_class(B, B->cls[c]);
    if (rc) return cleanup(rc);
  }
  // instance defaults (Sec. IV: MaxErr 1e-5, headroom 0.8); m along +x
  B->host_st.assign(n, InstState{});
  for (auto& s : B->host_st) {
    s.dt = 1e-14;
    s.max_err = 1e-5;
    s.headroom = 0.8;
    s.dt_min = 1e-20;
    s.dt_max = 1e-10;
    s.done = 1;
  }
  int rc = write_states(B);
  if (rc) return cleanup(rc);
  // one pass of every kernel outside any capture (sets launch attributes)
  for (int c = 0; c < nc; ++c) enqueue_stage(B, B->cls[c], 0, B->stream);
  e = cudaStreamSynchronize(B->stream);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return cleanup(bfail(MM_ERR_CUDA, std::string("batch warm-up: ") + cudaGetErrorString(e)));
  *out = B;
  return MM_OK;
}

int mm_batch_destroy(mm_batch* B) {
  if (!B) return MM_OK;
  cudaSetDevice(B->device);
  if (B->stream) cudaStreamSynchronize(B->stream);
  if (B->exec) cudaGraphExecDestroy(B->exec);
  for (BClass& C : B->cls) {
    void* ptrs[] = {C.b.m[0], C.b.m[1], C.b.k[0], C.b.k[1], C.b.k[2], C.b.k[3], C.b.k[4], C.b.k[5], C.b.k[6],
                    C.b.ms,   C.b.bd,   C.b.spec, C.b.kt,   C.b.ktf,  C.msat,   C.prm,    C.hist};
    for (void* p : ptrs)
      if (p) cudaFree(p);
  }
  if (B->st) cudaFree(B->st);
  if (B->attempts) cudaFree(B->attempts);
  if (B->tw) cudaFree(B->tw);
  for (cudaStream_t s : B->side)
    if (s) cudaStreamDestroy(s);
  for (cudaEvent_t v : B->ev)
    if (v) cudaEventDestroy(v);
  if (B->own_stream && B->stream) cudaStreamDestroy(B->stream);
  delete B;
  return MM_OK;
}

static int batch_vec(mm_batch* B, int i, float** dev, size_t* count) {
  if (!B) return bfail(MM_ERR_ARG, "batch is NULL");
  if (i < 0 || i >= B->n) return bfail(MM_ERR_ARG, "instance index out of range");
  BClass& C = B->cls[B->cls_of[i]];
  const int j = B->slot_of[i] - C.first;
  const int par = B->host_st[B->slot_of[i]].parity;
  *dev = C.b.m[par] + (size_t)j * 3 * C.g.n;
  *count = 3 * (size_t)C.g.n;
  return MM_OK;
}

int mm_batch_set_m(mm_batch* B, int i, const float* m) {
  if (!m) return bfail(MM_ERR_ARG, "m is NULL");
  float* d = nullptr;
  size_t cnt = 0;
  int rc = read_states(B);
  if (rc) return rc;
  rc = batch_vec(B, i, &d, &cnt);
  if (rc) return rc;
  MMB_CUDA(cudaMemcpyAsync(d, m, cnt * sizeof(float), cudaMemcpyHostToDevice, B->stream));
  k_b_normalize<<<(unsigned)((cnt / 3 + 255) / 256), 256, 0, B->stream>>>(d, (long long)(cnt / 3));
  MMB_CUDA(cudaGetLastError());
  MMB_CUDA(cudaStreamSynchronize(B->stream));
  B->k1_valid = false;
  return MM_OK;
}

int mm_batch_get_m(mm_batch* B, int i, float* m) {
  if (!m) return bfail(MM_ERR_ARG, "m is NULL");
  float* d = nullptr;
  size_t cnt = 0;
  int rc = read_states(B);
  if (rc) return rc;
  rc = batch_vec(B, i, &d, &cnt);
  if (rc) return rc;
  MMB_CUDA(cudaMemcpyAsync(m, d, cnt * sizeof(float), cudaMemcpyDeviceToHost, B->stream));
  MMB_CUDA(cudaStreamSynchronize(B->stream));
  return MM_OK;
}

int mm_batch_set_solver(mm_batch* B, double max_err, double headroom, double dt0, double dt_min, double dt_max) {
  if (!B) return bfail(MM_ERR_ARG, "batch is NULL");
  if (!(max_err > 0) || !(headroom > 0) || !(dt0 > 0) || !(dt_min > 0) || !(dt_max >= dt_min))
    return bfail(MM_ERR_ARG, "solver settings must be positive with dt_min <= dt_max");
  int rc = read_states(B);
  if (rc) return rc;
  for (auto& s : B->host_st) {
    s.max_err = max_err;
    s.headroom = headroom;
    s.dt = std::min(std::max(dt0, dt_min), dt_max);
    s.dt_min = dt_min;
    s.dt_max = dt_max;
  }
  return write_states(B);
}

int mm_batch_run(mm_batch* B, double t_end) {
  if (!B) return bfail(MM_ERR_ARG, "batch is NULL");
  if (!std::isfinite(t_end)) return bfail(MM_ERR_ARG, "t_end must be finite");
  int rc = build_batch_graph(B);
  if (rc) return rc;
  k_b_begin<<<(B->n + 127) / 128, 128, 0, B->stream>>>(B->st, B->n, t_end);
  MMB_CUDA(cudaGetLastError());
  if (!B->k1_valid) {
    for (BClass& C : B->cls) enqueue_stage(B, C, 0, B->stream);
    MMB_CUDA(cudaGetLastError());
    B->k1_valid = true;
  }
  for (int launch = 0; launch < 1000; ++launch) {
    MMB_CUDA(cudaMemsetAsync(B->attempts, 0, sizeof(unsigned int), B->stream));
    MMB_CUDA(cudaGraphLaunch(B->exec, B->stream));
    rc = read_states(B);
    if (rc) return rc;
    bool all_done = true;
    int bad = 0;
    for (const auto& s : B->host_st) {
      all_done = all_done && s.done;
      if (s.status) bad = s.status;
    }
    if (bad) return bfail(bad, "an instance stopped with an error (see mm_batch_get_stats)");
    if (all_done) return MM_OK;
  }
  return bfail(MM_ERR_STATE, "batched run did not finish");
}

int mm_batch_get_stats(mm_batch* B, int i, mm_stats* out) {
  if (!B || !out) return bfail(MM_ERR_ARG, "NULL argument");
  if (i < 0 || i >= B->n) return bfail(MM_ERR_ARG, "instance index out of range");
  int rc = read_states(B);
  if (rc) return rc;
  const InstState& s = B->host_st[B->slot_of[i]];
  out->accepted = s.accepted;
  out->rejected = s.rejected;
  out->evals = 6 * (s.accepted + s.rejected);
  out->last_err = s.last_err;
  out->t = s.t;
  out->dt = s.dt;
  out->launches = 0;
  return s.status;
}

int mm_batch_get_dt_history(mm_batch* B, int i, double* dts, int max, int* n) {
  if (!B || !n || (max > 0 && !dts)) return bfail(MM_ERR_ARG, "NULL argument");
  if (i < 0 || i >= B->n) return bfail(MM_ERR_ARG, "instance index out of range");
  int rc = read_states(B);
  if (rc) return rc;
  BClass& C = B->cls[B->cls_of[i]];
  const int j = B->slot_of[i] - C.first;
  const int k = std::min(std::min(B->host_st[B->slot_of[i]].hist_n, kBatchHist), std::max(max, 0));
  if (k > 0) {
    MMB_CUDA(cudaMemcpyAsync(dts, C.hist + (size_t)j * kBatchHist, k * sizeof(double), cudaMemcpyDeviceToHost,
                             B->stream));
    MMB_CUDA(cudaStreamSynchronize(B->stream));
  }
  *n = k;
  return MM_OK;
}

int mm_batch_num_classes(mm_batch* B) { return B ? (int)B->cls.size() : 0; }

int mm_batch_set_tiles(mm_batch* B, int c, int cly, int clz, int xrows) {
  if (!B || c < 0 || c >= (int)B->cls.size()) return bfail(MM_ERR_ARG, "bad batch or class index");
  BClass& C = B->cls[c];
  int sp[4][2];
  const int nsp = fused_splits(C.g, sp, 4);
  bool ok_split = false;
  for (int i = 0; i < nsp; ++i) ok_split = ok_split || (sp[i][0] == cly && sp[i][1] == clz);
  int xr[3];
  const int nxr = fused_xrows(C.g, xr, 3);
  bool ok_rows = false;
  for (int i = 0; i < nxr; ++i) ok_rows = ok_rows || xr[i] == xrows;
  if (!ok_split || !ok_rows) return bfail(MM_ERR_ARG, "tiles not offered for this shape class");
  fused_set_split(C.g, cly, clz);
  C.g.xrows = xrows;
  // the captured graph holds the old tiles: capture again at the next run
  if (B->exec) {
    cudaGraphExecDestroy(B->exec);
    B->exec = nullptr;
  }
  return MM_OK;
}

int mm_batch_class_info(mm_batch* B, int c, int info[7], double* conv_us) {
  if (!B || !info || c < 0 || c >= (int)B->cls.size()) return bfail(MM_ERR_ARG, "bad batch or class index");
  const BClass& C = B->cls[c];
  info[0] = C.g.nx;
  info[1] = C.g.ny;
  info[2] = C.g.nz;
  info[3] = C.B;
  info[4] = C.g.cly;
  info[5] = C.g.clz;
  info[6] = C.g.xrows;
  if (conv_us) *conv_us = C.conv_us;
  return MM_OK;
}

}  // extern "C"
