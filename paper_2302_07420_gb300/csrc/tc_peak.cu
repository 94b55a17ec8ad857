// Measured FMA throughput of the non-tensor arithmetic pipes (tc_alu_peak).
//
// The FFT codelets and pair products of the operator run on the FP32 (or
// FP64) fused multiply-add pipes, not on the tensor cores, so the roofline of
// those kernels is the FMA rate.  This launch measures it: every thread runs
// kChains independent chains x <- a x + b (a, b kernel arguments, so nothing folds
// at compile time), one CTA wave per SM at full occupancy, timed with CUDA
// events.  a = 1 - 2^-20 and b = 2^-20 keep every chain inside [0, 1] (fixed
// point 1): no overflow, no subnormals.
#include <algorithm>
#include <cmath>
#include <string>

#include "tc_ctx.hpp"

namespace {

constexpr int kChains = 16;
constexpr int kThreads = 256;

__device__ __forceinline__ float fma_rn(float x, float a, float b) { return __fmaf_rn(x, a, b); }
__device__ __forceinline__ double fma_rn(double x, double a, double b) { return __fma_rn(x, a, b); }

template <typename T>
__global__ void __launch_bounds__(kThreads) k_fma_peak(T* out, T a, T b, T sentinel, int iters) {
  T x[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) x[i] = T(threadIdx.x % 97 + i) * T(0.0078125);
#pragma unroll 4
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = fma_rn(x[i], a, b);
  }
  T s = T(0);
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += x[i];
  // never true for the chains above (their sum stays below kChains + 2); keeps the work live
  if (s == sentinel) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T> int measure(double target_ms, double* tflops, cudaStream_t st, std::string& err) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_peak<T>, kThreads, 0);
  if (e != cudaSuccess) {
    err = std::string("tc_alu_peak: ") + cudaGetErrorString(e);
    return TC_ERR_CUDA;
  }
  const int blocks = sms * std::max(per_sm, 1);
  T* out = nullptr;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  e = cudaMalloc(&out, sizeof(T) * (size_t)blocks * kThreads);
  if (e == cudaSuccess) e = cudaEventCreate(&ev[0]);
  if (e == cudaSuccess) e = cudaEventCreate(&ev[1]);
  const T a = T(1) - T(1.0 / 1048576.0), b = T(1.0 / 1048576.0), sentinel = T(-1);
  // one launch of `iters` iterations, timed on st; returns ms (< 0 on a CUDA error)
  auto timed = [&](int iters) -> float {
    if (e != cudaSuccess) return -1.f;
    cudaEventRecord(ev[0], st);
    k_fma_peak<T><<<blocks, kThreads, 0, st>>>(out, a, b, sentinel, iters);
    cudaEventRecord(ev[1], st);
    e = cudaEventSynchronize(ev[1]);
    if (e == cudaSuccess) e = cudaGetLastError();
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
    return e == cudaSuccess ? ms : -1.f;
  };
  // calibration by doubling: each launch takes about twice the previous one's time, so no launch
  // runs much longer than target_ms whatever the rate turns out to be
  int iters = 256;
  timed(iters);
  float ms = timed(iters);
  while (ms >= 0.f && ms < 0.5 * target_ms && iters < (1 << 24)) {
    iters *= 2;
    ms = timed(iters);
  }
  double best = 0.0;
  for (int r = 0; r < 3 && e == cudaSuccess; ++r) {   // fastest of three: clocks settle after the first
    const float t = timed(iters);
    if (t > 0.f) best = std::max(best, 2.0 * kChains * (double)iters * blocks * kThreads / (t * 1e-3) / 1e12);
  }
  const cudaError_t e_run = e;
  if (ev[0]) cudaEventDestroy(ev[0]);
  if (ev[1]) cudaEventDestroy(ev[1]);
  if (out) cudaFree(out);
  if (e_run != cudaSuccess) {
    err = std::string("tc_alu_peak: ") + cudaGetErrorString(e_run);
    return TC_ERR_CUDA;
  }
  *tflops = best;
  return TC_OK;
}

}  // namespace

extern "C" tc_status tc_alu_peak(int precision, double target_ms, double* tflops, void* stream) {
  if (!tflops || (precision != TC_FP32 && precision != TC_FP64) || !(target_ms > 0.0 && target_ms <= 1000.0)) {
    tc::set_thread_error("tc_alu_peak: needs precision TC_FP32 or TC_FP64, 0 < target_ms <= 1000 and an output");
    return TC_ERR_ARG;
  }
  std::string err;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int r = precision == TC_FP64 ? measure<double>(target_ms, tflops, st, err)
                                     : measure<float>(target_ms, tflops, st, err);
  if (r != TC_OK) tc::set_thread_error(err);
  return (tc_status)r;
}
