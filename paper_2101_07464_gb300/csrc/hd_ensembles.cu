// Other ensembles built from the Gaussian and Haar ones (section "Other Random Matrix
// Ensembles" of the paper): a GOE product from two products of one square Ginibre state, and
// the product with Q = U Sigma V (eq. inv) from one product of each of two independent Haar
// states.  Both are compositions of the library's own steps plus an elementwise kernel.
#include <cmath>
#include <cstdint>

#include <cuda_runtime.h>

#include "hd.h"
#include "hd_state.cuh"

using namespace hd;

namespace {

// y = (y + yh) / sqrt(2), elementwise (the GOE combination).
template <typename T>
__global__ void __launch_bounds__(256) k_goe_combine(T* __restrict__ y, const T* __restrict__ yh, int64_t len) {
  const T r = (T)0.70710678118654752440;   // 1 / sqrt(2)
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = (y[i] + yh[i]) * r;
}

// out[i] = s[i] in[i] for i < kmin, 0 for kmin <= i < len_out (Sigma, rectangular diagonal).
template <typename T>
__global__ void __launch_bounds__(256) k_sigma(T* __restrict__ out, const T* __restrict__ in,
                                               const double* __restrict__ s, int64_t kmin, int64_t len_out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len_out; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (i < kmin) ? (T)s[i] * in[i] : T(0);
}

unsigned grid_for(const hd_state* st, int64_t len) {
  const int64_t want = (len + 255) / 256;
  const int64_t cap = (int64_t)st->nsm * 8;
  return (unsigned)(want < 1 ? 1 : (want < cap ? want : cap));
}

void* scratch(hd_state* st, int q, int64_t len) {
  if (!st->ens_tmp[q]) st->ens_tmp[q] = dalloc(st, (size_t)round_up(len, 64) * st->esz);
  return st->ens_tmp[q];
}

}  // namespace

HD_API int hd_goe_apply(hd_state* st, const void* x, void* y) {
  if (!st || !x || !y || x == y) return HD_ERR_ARG;
  if (st->ens != HD_GINIBRE) return HD_ERR_ARG;
  for (int i = 0; i < st->count; i++)
    if (st->dims[0][i] != st->dims[1][i]) return HD_ERR_DIM;
  if (st->poisoned) return st->poisoned;
  if (st->t + 2 > st->Tm) return HD_ERR_TMAX;
  if (cudaSetDevice(st->device) != cudaSuccess) return cuda_fail(st, cudaErrorInvalidDevice);
  const int64_t len = st->off[0][st->count];
  void* yh = scratch(st, 0, len);
  if (!yh) return HD_ERR_OOM;
  int rc = hd_apply(st, x, 0, yh);   // yh = Q x
  if (!rc) rc = hd_apply(st, x, 1, y);   // y = Q^T x
  if (rc) return rc;
  if (st->dtype == HD_F64)
    k_goe_combine<double><<<grid_for(st, len), 256, 0, st->stream>>>((double*)y, (const double*)yh, len);
  else
    k_goe_combine<float><<<grid_for(st, len), 256, 0, st->stream>>>((float*)y, (const float*)yh, len);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(st, e);
  st->launches += 1;
  return HD_OK;
}

HD_API int hd_usv_apply(hd_state* U, hd_state* V, const double* s, const void* x, int transpose, void* y) {
  if (!U || !V || !s || !x || !y || U == V) return HD_ERR_ARG;
  if (transpose != 0 && transpose != 1) return HD_ERR_ARG;
  if (U->ens != HD_HAAR || V->ens != HD_HAAR || U->count != 1 || V->count != 1) return HD_ERR_ARG;
  if (U->dtype != V->dtype || U->device != V->device || U->stream != V->stream) return HD_ERR_ARG;
  if (U->poisoned) return U->poisoned;
  if (V->poisoned) return V->poisoned;
  if (U->t >= U->Tm || V->t >= V->Tm) return HD_ERR_TMAX;
  if (cudaSetDevice(U->device) != cudaSuccess) return cuda_fail(U, cudaErrorInvalidDevice);
  const int64_t m = U->dims[0][0], n = V->dims[0][0], kmin = (m < n) ? m : n;
  // M x = U (Sigma (V x)); M^T z = V^T (Sigma^T (U^T z))
  hd_state* first = transpose ? U : V;
  hd_state* second = transpose ? V : U;
  const int64_t len1 = transpose ? m : n, len2 = transpose ? n : m;
  void* t1 = scratch(U, 0, (m > n) ? m : n);
  void* t2 = scratch(U, 1, (m > n) ? m : n);
  if (!t1 || !t2) return HD_ERR_OOM;
  int rc = hd_apply(first, x, transpose, t1);
  if (rc) return rc;
  if (U->dtype == HD_F64)
    k_sigma<double><<<grid_for(U, len2), 256, 0, U->stream>>>((double*)t2, (const double*)t1, s, kmin, len2);
  else
    k_sigma<float><<<grid_for(U, len2), 256, 0, U->stream>>>((float*)t2, (const float*)t1, s, kmin, len2);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(U, e);
  U->launches += 1;
  (void)len1;
  return hd_apply(second, t2, transpose, y);
}
