// mm_fp32_peak: the float32 FMA throughput of a device, measured.
//
// The demag convolution's transforms and kernel product run on the FP32
// pipes; their roof is this throughput, which the device's specifications do
// not state as a measured number.  The kernel keeps every SM's FP32 pipes busy
// with independent fused multiply-add chains (eight per thread, 32 warps per
// SM) and is timed with CUDA events; the result is 2 x FMAs / time.  No
// counterpart in the paper (a measurement utility).
#include <algorithm>
#include <string>

#include "../../include/mm.h"
#include "mm_internal.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;
constexpr int kBlocksPerSM = 4;
constexpr int kIters = 1 << 15;   // loop trips; 4 x kChains FMAs per trip

__global__ void __launch_bounds__(kThreads) k_fma_chains(float* out, float a, float b) {
  float x[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) x[i] = 1e-3f * (float)threadIdx.x + (float)i;
  for (int it = 0; it < kIters; ++it) {
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int i = 0; i < kChains; ++i) x[i] = fmaf(x[i], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += x[i];
  // (a store the compiler cannot drop; the condition is never true for the
  // contracting map x -> a x + b with |a| < 1)
  if (s == -1.0f) out[blockIdx.x * kThreads + threadIdx.x] = s;
}

int peak_fail(int code, const std::string& msg) {
  mm::set_last_error(msg);
  return code;
}

}  // namespace

extern "C" int mm_fp32_peak(int device, int reps, double* tflops, int* sm_count, int* clock_mhz) {
  if (!tflops || reps < 1) return peak_fail(MM_ERR_ARG, "tflops must not be NULL and reps >= 1");
  int prev = 0;
  cudaError_t e = cudaGetDevice(&prev);
  if (e == cudaSuccess) e = cudaSetDevice(device);
  if (e != cudaSuccess) return peak_fail(MM_ERR_CUDA, std::string("device: ") + cudaGetErrorString(e));
  int sms = 0, khz = 0;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, device);
  cudaStream_t s = nullptr;
  cudaEvent_t a = nullptr, z = nullptr;
  float* out = nullptr;
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&z);
  const int blocks = std::max(1, sms) * kBlocksPerSM;
  if (e == cudaSuccess) e = cudaMalloc(&out, sizeof(float) * blocks * kThreads);
  float best = 1e30f;
  for (int r = 0; r <= reps && e == cudaSuccess; ++r) {   // r = 0: warm-up
    e = cudaEventRecord(a, s);
    k_fma_chains<<<blocks, kThreads, 0, s>>>(out, 0.999999f, 1e-7f);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(z, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(z);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, z);
    if (e == cudaSuccess && r > 0) best = std::min(best, ms);
  }
  if (out) cudaFree(out);
  if (a) cudaEventDestroy(a);
  if (z) cudaEventDestroy(z);
  if (s) cudaStreamDestroy(s);
  cudaSetDevice(prev);
  if (e != cudaSuccess) return peak_fail(MM_ERR_CUDA, std::string("FMA kernel: ") + cudaGetErrorString(e));
  const double fmas = (double)blocks * kThreads * kIters * 4.0 * kChains;
  *tflops = 2.0 * fmas / (best * 1e-3) / 1e12;
  if (sm_count) *sm_count = sms;
  if (clock_mhz) *clock_mhz = khz / 1000;
  return MM_OK;
}
