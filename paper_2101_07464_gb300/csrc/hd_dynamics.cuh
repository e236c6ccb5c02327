// Built-in elementwise dynamics for hd_run.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace hd {

enum DynKind { kDynNone = 0, kDynTanh = 1, kDynSignMem = 2, kDynNormTanh = 3, kDynAmp = 4, kDynIsta = 5 };

template <typename T>
cudaError_t launch_dynamics(int kind, double a, const T* y, const T* xcur, const T* xprev, T* out,
                            int64_t n, double* sumsq, cudaStream_t s, bool pdl);

// AMP and ISTA on a batch of trials (packed vectors, trial i's m-space rows [offm[i], offm[i+1])
// and n-space rows [offn[i], offn[i+1])); one CTA per trial, FP64 sums in a fixed order.
//   init:  ymeas = z = q + w, zsq_i = ||z_i||^2
//   x:     AMP  x = eta(x + s; a sqrt(zsq_i / m_i)),  ISTA  x = eta(x + tau s; a);  nnz_i = ||x_i||_0
//   z:     AMP  z = ymeas - q + z nnz_i / m_i,        ISTA  z = ymeas - q;        zsq_i = ||z_i||^2
template <typename T>
cudaError_t launch_amp_init(int count, const int64_t* offm, const T* q, const T* w, T* ymeas, T* z,
                            double* zsq, cudaStream_t s);
template <typename T>
cudaError_t launch_amp_x(int count, const int64_t* offn, const int64_t* offm, const T* sv, T* x,
                         const double* zsq, double a, double tau, int ista, int* nnz, cudaStream_t s);
template <typename T>
cudaError_t launch_amp_z(int count, const int64_t* offm, const T* ymeas, const T* q, T* z, const int* nnz,
                         int ista, double* zsq, cudaStream_t s);

}  // namespace hd
