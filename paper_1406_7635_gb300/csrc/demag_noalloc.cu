// mm_demag_field_noalloc: the demagnetising field of a caller-provided
// magnetisation without any device allocation.
//
// Some callers cannot call cudaMalloc: host frameworks whose device memory
// must all come from their own pool (a caching allocator that owns the GPU),
// embedding applications that forbid device allocation after start-up, or
// real-time loops that must never touch the allocator.  A context (mm_create)
// allocates its state and scratch, so it does not serve them.  This entry
// point takes device input and output buffers only and keeps every
// intermediate -- the float64 kernel
// precompute work, the float32 kernel spectrum octant, the FFT spectrum, the
// twiddle table and a trivial region/geometry table -- in one file-scope
// device array of kScratchBytes, which every GPU that loads the library holds
// until the process exits.  There is no counterpart in the paper; the
// arithmetic is the same convolution as mm_demag_apply (Sec. III.B).
#include <cstdio>
#include <mutex>
#include <string>

#include "../../include/mm.h"
#include "mm_internal.h"

namespace {

constexpr size_t kScratchBytes = size_t(32) << 20;   // 32 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Device address of g_scratch per device (the host-side symbol is a
// stand-in, not a device address), looked up with that device current and
// kept with the context it belongs to: a device whose primary context was
// torn down and re-created (cudaDeviceReset) reloads the module, and the
// address is looked up again.
struct ScratchSlot {
  CUcontext ctx;
  unsigned char* ptr;
};
ScratchSlot g_scratch_slot[kMaxDevices] = {};
std::mutex g_scratch_mu;

// the calling thread's current context through the runtime's driver entry
// point (no link against the driver library); null when unavailable
typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
CUcontext current_context() {
  static const CtxGetCurrentFn fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return reinterpret_cast<CtxGetCurrentFn>(f);
    return CtxGetCurrentFn(nullptr);
  }();
  CUcontext c = nullptr;
  if (!fn || fn(&c) != CUDA_SUCCESS) return nullptr;
  return c;
}

int noalloc_fail(int code, const std::string& msg) {
  mm::set_last_error(msg);
  return code;
}

__global__ void k_noalloc_twiddles(float2* tw) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= 2048) return;
  const double a = -2.0 * (double)k / 2048.0;   // angle / pi
  tw[k] = make_float2((float)cospi(a), (float)sinpi(a));
}

// one region (0) with Msat = 1: the convolution then reads M directly
__global__ void k_noalloc_lut(mm::RegionLUT* lut) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= mm::kRegions) return;
  lut->msat[r] = r == 0 ? 1.0f : 0.0f;
}

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

}  // namespace

extern "C" int mm_demag_field_noalloc(int nx, int ny, int nz, double dx, double dy, double dz, const float* M,
                                      float* B, void* stream) {
  if (!M || !B) return noalloc_fail(MM_ERR_ARG, "M and B must be device pointers");
  if (nx < 1 || ny < 1 || nz < 1 || nx > 1024 || ny > 512 || nz > 512)
    return noalloc_fail(MM_ERR_ARG, "grid sizes must be 1..1024 (x), 1..512 (y, z)");
  if (!(dx > 0) || !(dy > 0) || !(dz > 0)) return noalloc_fail(MM_ERR_ARG, "cell sizes must be > 0");
  // the context path's geometry (padding, spectrum strides, octant sizes);
  // the fused-convolution fields stay zero, so the general five-pass
  // convolution runs
  const mm::Geom g = mm::make_geom(nx, ny, nz, dx, dy, dz);

  // carve the scratch array
  const size_t b_tw = align256(2048 * sizeof(float2));
  const size_t b_lut = align256(sizeof(mm::RegionLUT));
  const size_t b_mask = align256((size_t)g.n);
  const size_t b_kt = align256(6 * (size_t)g.hkx * g.hky * g.hkz * sizeof(float));
  const size_t b_spec = align256(3 * (size_t)g.sc * sizeof(float2));
  const size_t b_work = align256(mm::kernel_work_doubles(g) * sizeof(double));
  const size_t b_tab = align256(mm::kernel_table_doubles(g) * sizeof(double));
  const size_t need = b_tw + b_lut + 2 * b_mask + b_kt + b_spec + 2 * b_work + b_tab;
  if (need > kScratchBytes) {
    char msg[256];
    std::snprintf(msg, sizeof msg,
                  "grid %dx%dx%d needs %zu bytes of scratch; mm_demag_field_noalloc has %zu (use a context)",
                  nx, ny, nz, need, kScratchBytes);
    return noalloc_fail(MM_ERR_ARG, msg);
  }

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return noalloc_fail(MM_ERR_CUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(MM_ERR_ARG, "device index out of range");
  unsigned char* base = nullptr;
  {
    // set-up, once per device (and again after that device's context was
    // re-created), with that device current
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    ScratchSlot& slot = g_scratch_slot[dev];
    const CUcontext cur = current_context();
    if (!slot.ptr || !cur || cur != slot.ctx) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_scratch);
      if (e != cudaSuccess) return noalloc_fail(MM_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      slot.ptr = static_cast<unsigned char*>(p);
      slot.ctx = current_context();
    }
    base = slot.ptr;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    unsigned char* p = base + off;
    off += bytes;
    return p;
  };
  mm::Buffers b{};
  b.tw = reinterpret_cast<float2*>(take(b_tw));
  b.lut = reinterpret_cast<mm::RegionLUT*>(take(b_lut));
  b.mask = take(b_mask);
  b.region = take(b_mask);
  b.kt = reinterpret_cast<float*>(take(b_kt));
  b.spec = reinterpret_cast<float2*>(take(b_spec));
  double* w0 = reinterpret_cast<double*>(take(b_work));
  double* w1 = reinterpret_cast<double*>(take(b_work));
  double* tab = reinterpret_cast<double*>(take(b_tab));
  b.st = nullptr;
  b.bd = B;

  // the array keeps the previous call's contents: (re)initialise every table
  // this call reads before it writes
  k_noalloc_twiddles<<<16, 128, 0, s>>>(b.tw);
  e = cudaMemsetAsync(b.lut, 0, sizeof(mm::RegionLUT), s);
  if (e == cudaSuccess) k_noalloc_lut<<<2, 128, 0, s>>>(b.lut);
  if (e == cudaSuccess) e = cudaMemsetAsync(b.mask, 1, (size_t)g.n, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(b.region, 0, (size_t)g.n, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(b.spec, 0, 3 * (size_t)g.sc * sizeof(float2), s);
  if (e == cudaSuccess) e = mm::build_kernel_spectrum_ws(g, dx, dy, dz, b.kt, w0, w1, tab, s);
  if (e != cudaSuccess) return noalloc_fail(MM_ERR_CUDA, cudaGetErrorString(e));
  mm::launch_demag(g, b, M, s);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return noalloc_fail(MM_ERR_CUDA, cudaGetErrorString(e));
  return MM_OK;
}
