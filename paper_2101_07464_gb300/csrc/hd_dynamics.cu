// Built-in elementwise dynamics f_t of eq. (dynamics) for whole-trajectory runs (hd_run).
//   tanh       x_{t+1} = tanh(y_t)
//   sign_mem   x_{t+1} = sign(y_t) + a x_{t-1}       (sign(0) = 0, x_0 = 0)
//   norm_tanh  x_{t+1} = v / ||v||, v = tanh(y_t) + a x_t
// The caller's own f_t can always be used instead through hd_apply.
#include <cstdint>

#include "hd_common.cuh"
#include "hd_dynamics.cuh"

namespace hd {

template <typename T>
__device__ __forceinline__ T sgn(T v) {
  return (v > T(0)) ? T(1) : ((v < T(0)) ? T(-1) : T(0));
}

// out may alias xprev (elementwise, read before write).
template <typename T>
__global__ void k_dyn(int kind, T a, const T* __restrict__ y, const T* xcur, const T* xprev, T* out,
                      int64_t n, double* sumsq) {
  // y comes from the preceding kernel (programmatic dependent launch): wait, then let the
  // next kernel start
  asm volatile("griddepcontrol.wait;\n" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double s = 0.0;
  if (i < n) {
    const T yi = y[i];
    T v;
    if (kind == kDynTanh) v = tanh(yi);
    else if (kind == kDynSignMem) v = sgn(yi) + a * xprev[i];
    else v = tanh(yi) + a * xcur[i];
    out[i] = v;
    s = (double)v * (double)v;
  }
  if (kind == kDynNormTanh) {
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) atomicAdd(sumsq, s);
  }
}

template <typename T>
__global__ void k_scale_rsqrt(T* x, int64_t n, const double* sumsq) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const double s = *sumsq;
    x[i] = (s > 0.0) ? (T)((double)x[i] / sqrt(s)) : x[i];
  }
}

template <typename T>
cudaError_t launch_dynamics(int kind, double a, const T* y, const T* xcur, const T* xprev, T* out,
                            int64_t n, double* sumsq, cudaStream_t s, bool pdl) {
  const int thr = 256;
  const unsigned blocks = (unsigned)((n + thr - 1) / thr);
  if (kind == kDynNormTanh) {
    cudaError_t e = cudaMemsetAsync(sumsq, 0, sizeof(double), s);
    if (e != cudaSuccess) return e;
    pdl = false;   // the memset sits between the sweep and this kernel
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(thr);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = pdl ? attr : nullptr;
  cfg.numAttrs = pdl ? 1 : 0;
  cudaError_t e = cudaLaunchKernelEx(&cfg, k_dyn<T>, kind, (T)a, y, xcur, xprev, out, n, sumsq);
  if (e != cudaSuccess) return e;
  if (kind == kDynNormTanh) k_scale_rsqrt<T><<<blocks, thr, 0, s>>>(out, n, sumsq);
  return cudaGetLastError();
}

template cudaError_t launch_dynamics<float>(int, double, const float*, const float*, const float*,
                                            float*, int64_t, double*, cudaStream_t, bool);
template cudaError_t launch_dynamics<double>(int, double, const double*, const double*,
                                             const double*, double*, int64_t, double*, cudaStream_t, bool);

}  // namespace hd
