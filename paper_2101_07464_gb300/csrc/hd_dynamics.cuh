// Built-in elementwise dynamics for hd_run.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace hd {

enum DynKind { kDynNone = 0, kDynTanh = 1, kDynSignMem = 2, kDynNormTanh = 3 };

template <typename T>
cudaError_t launch_dynamics(int kind, double a, const T* y, const T* xcur, const T* xprev, T* out,
                            int64_t n, double* sumsq, cudaStream_t s, bool pdl);

}  // namespace hd
