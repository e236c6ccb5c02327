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

// ------------------------------------------------------------------------------------
// AMP (one CTA per trial)
constexpr int kAmpThreads = 256;

__device__ __forceinline__ double amp_block_sum(double v, double* red) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
#pragma unroll
  for (int w = 0; w < kAmpThreads / 32; w++) s += red[w];
  return s;
}

template <typename T>
__global__ void __launch_bounds__(kAmpThreads) k_amp_init(const int64_t* offm, const T* __restrict__ q,
                                                          const T* __restrict__ w, T* ymeas, T* z, double* zsq) {
  __shared__ double red[kAmpThreads / 32];
  const int i = blockIdx.x;
  const int64_t r0 = offm[i], r1 = offm[i + 1];
  double s = 0.0;
  for (int64_t r = r0 + threadIdx.x; r < r1; r += kAmpThreads) {
    const T v = q[r] + w[r];
    ymeas[r] = v;
    z[r] = v;
    s = fma((double)v, (double)v, s);
  }
  s = amp_block_sum(s, red);
  if (threadIdx.x == 0) zsq[i] = s;
}

template <typename T>
__device__ __forceinline__ T soft_thr(T r, T theta) {
  const T a = fabs(r) - theta;
  return (a > T(0)) ? copysign(a, r) : T(0);
}

template <typename T>
__global__ void __launch_bounds__(kAmpThreads) k_amp_x(const int64_t* offn, const int64_t* offm,
                                                       const T* __restrict__ sv, T* x, const double* zsq,
                                                       double a, T tau, int ista, int* nnz) {
  __shared__ double red[kAmpThreads / 32];
  const int i = blockIdx.x;
  const int64_t r0 = offn[i], r1 = offn[i + 1];
  const double mi = (double)(offm[i + 1] - offm[i]);
  const T theta = ista ? (T)a : (T)(a * sqrt(zsq[i] / mi));
  double c = 0.0;
  for (int64_t r = r0 + threadIdx.x; r < r1; r += kAmpThreads) {
    const T v = soft_thr(fma(tau, sv[r], x[r]), theta);
    x[r] = v;
    c += (v != T(0)) ? 1.0 : 0.0;
  }
  c = amp_block_sum(c, red);
  if (threadIdx.x == 0) nnz[i] = (int)c;
}

template <typename T>
__global__ void __launch_bounds__(kAmpThreads) k_amp_z(const int64_t* offm, const T* __restrict__ ymeas,
                                                       const T* __restrict__ q, T* z, const int* nnz, int ista,
                                                       double* zsq) {
  __shared__ double red[kAmpThreads / 32];
  const int i = blockIdx.x;
  const int64_t r0 = offm[i], r1 = offm[i + 1];
  const T ons = ista ? T(0) : (T)((double)nnz[i] / (double)(r1 - r0));
  double s = 0.0;
  for (int64_t r = r0 + threadIdx.x; r < r1; r += kAmpThreads) {
    const T v = fma(z[r], ons, ymeas[r] - q[r]);
    z[r] = v;
    s = fma((double)v, (double)v, s);
  }
  s = amp_block_sum(s, red);
  if (threadIdx.x == 0) zsq[i] = s;
}

template <typename T>
cudaError_t launch_amp_init(int count, const int64_t* offm, const T* q, const T* w, T* ymeas, T* z,
                            double* zsq, cudaStream_t s) {
  k_amp_init<T><<<count, kAmpThreads, 0, s>>>(offm, q, w, ymeas, z, zsq);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_amp_x(int count, const int64_t* offn, const int64_t* offm, const T* sv, T* x,
                         const double* zsq, double a, double tau, int ista, int* nnz, cudaStream_t s) {
  k_amp_x<T><<<count, kAmpThreads, 0, s>>>(offn, offm, sv, x, zsq, a, (T)tau, ista, nnz);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_amp_z(int count, const int64_t* offm, const T* ymeas, const T* q, T* z, const int* nnz,
                         int ista, double* zsq, cudaStream_t s) {
  k_amp_z<T><<<count, kAmpThreads, 0, s>>>(offm, ymeas, q, z, nnz, ista, zsq);
  return cudaGetLastError();
}

#define HD_AMP_INST(T)                                                                               \
  template cudaError_t launch_amp_init<T>(int, const int64_t*, const T*, const T*, T*, T*, double*,  \
                                          cudaStream_t);                                             \
  template cudaError_t launch_amp_x<T>(int, const int64_t*, const int64_t*, const T*, T*,            \
                                       const double*, double, double, int, int*, cudaStream_t);      \
  template cudaError_t launch_amp_z<T>(int, const int64_t*, const T*, const T*, T*, const int*, int, \
                                       double*, cudaStream_t);
HD_AMP_INST(float)
HD_AMP_INST(double)
#undef HD_AMP_INST

template cudaError_t launch_dynamics<float>(int, double, const float*, const float*, const float*,
                                            float*, int64_t, double*, cudaStream_t, bool);
template cudaError_t launch_dynamics<double>(int, double, const double*, const double*,
                                             const double*, double*, int64_t, double*, cudaStream_t, bool);

}  // namespace hd
