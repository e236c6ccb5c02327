// Throughput probe of the FP64 fused multiply-add pipe: hd_fp64_fma_rate.
//
// The FP64 form of the method is bound by this pipe rather than by HBM on this GPU (each
// element of a reflector stack streamed in FP64 costs at least one dependent FMA per pass),
// so its roofline needs the pipe's rate measured on the device that runs it.  Every thread
// advances kChains independent FMA chains (enough in flight to hide the dependent latency),
// and the launch covers every SM with several resident warps per scheduler.  The result
// feeds nothing in the method itself.
#include <cstdint>

#include <cuda_runtime.h>

#include "hd.h"
#include "hd_state.cuh"

namespace {

constexpr int kChains = 8;
constexpr int kPeakThreads = 256;

__global__ void __launch_bounds__(kPeakThreads) k_dfma_rate(double* sink, int iters, double a, double b) {
  double c[kChains];
#pragma unroll
  for (int i = 0; i < kChains; i++) c[i] = 1e-3 * (double)(threadIdx.x + i);
  for (int it = 0; it < iters; it++) {
#pragma unroll
    for (int i = 0; i < kChains; i++) c[i] = fma(c[i], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < kChains; i++) s += c[i];
  if (s == -1.0) sink[blockIdx.x] = s;   // never true for these inputs; keeps the chains live
}

}  // namespace

extern "C" HD_API int hd_fp64_fma_rate(int32_t iters, int32_t reps, double* tflops_host, void* stream) {
  if (!tflops_host || iters < 1 || reps < 1) return HD_ERR_ARG;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    hd::set_error("hd_fp64_fma_rate", cudaGetLastError());
    return HD_ERR_CUDA;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int blocks = nsm * 8;   // 64 resident warps per SM
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  double best = 0.0;
  for (int r = 0; r < reps + 1 && e == cudaSuccess; r++) {   // the first launch is a warm-up
    e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) {
      k_dfma_rate<<<blocks, kPeakThreads, 0, s>>>(nullptr, iters, 0.9999999, 1e-7);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && r > 0 && ms > 0.f) {
      const double flops = 2.0 * kChains * (double)iters * blocks * kPeakThreads;
      const double tf = flops / (ms * 1e-3) / 1e12;
      if (tf > best) best = tf;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess) {
    hd::set_error("hd_fp64_fma_rate", e);
    return HD_ERR_CUDA;
  }
  *tflops_host = best;
  return HD_OK;
}
