// Allocation-free first product of a fresh matrix: hd_first_product_noalloc.
//
// The first product of a fresh matrix needs no stored reflectors.  For Q ~ Haar(n) the
// data-side reflector sends x_1 to ||x_1|| e_1 and the random-side reflector sends e_1 to
// g_1 / ||g_1||, so y_1 = ||x_1|| g_1 / ||g_1||, for Q and for Q^T alike.  For Q ~ Gin(m, n)
// the first basis pair is v_1 = x_1 / ||x_1|| and u_1 = g_1, so y_1 = (v_1^T x_1) u_1 =
// ||x_1|| g_1 (g_1 drawn with entry scale sigma, in R^m for Q and R^n for Q^T).  g_1 is the
// same Philox draw that a new state makes for its step 1, so the result equals hd_create +
// hd_apply at step 1 up to rounding.
//
// Two kernels on the caller's stream: per-tile partial sums of ||x_1||^2 (and ||g_1||^2 for
// Haar), the last tile to finish forming the coefficient; then y = coefficient * g_1 with
// g_1 drawn again.  Their scratch (partials, tile counter, coefficient) is one file-scope
// device array whose device address is looked up on every call with cudaGetSymbolAddress
// (cheap once the module is loaded, and never stale after a device reset), so a call
// allocates no device or host memory.  The scratch is shared by every call on a device:
// calls that overlap on the device race on it.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>

#include <cuda_runtime.h>

#include "../../include/hd.h"
#include "hd_common.cuh"

namespace hd {

void record_error_text(const char* msg);   // hd_last_error's text (defined with the C ABI)

namespace {

constexpr int kNaThreads = 256;
constexpr int kNaPerThread = 16;                           // entries per thread and tile
constexpr int64_t kNaTile = kNaThreads * kNaPerThread;      // 4096 entries per CTA
constexpr int kNaMaxTiles = 4096;                           // partial-sum slots
constexpr int64_t kNaMaxDim = kNaTile * kNaMaxTiles;        // 16,777,216 entries
// Layout (doubles): [0, 2 * kNaMaxTiles) partial sums (||x||^2, ||g||^2) per tile;
// [kNaCoef] the coefficient; [kNaCounter] the tile counter (an unsigned int, must be zero
// when kernel 1 starts: every call clears it first, and the last tile resets it).
constexpr int kNaCoef = 2 * kNaMaxTiles;
constexpr int kNaCounter = 2 * kNaMaxTiles + 32;
constexpr int kNaScratchDoubles = 2 * kNaMaxTiles + 64;    // 66,048 bytes

static __device__ __align__(256) double g_na_scratch[kNaScratchDoubles];

__device__ __forceinline__ double na_block_sum(double v, double* red) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
#pragma unroll
  for (int w = 0; w < kNaThreads / 32; w++) s += red[w];
  return s;
}

// One tile per CTA: partial ||x||^2 over [0, nx) and (Haar) ||g||^2 over [0, ng); the last
// CTA sums the partials in tile order and writes the coefficient.
template <typename T, bool kHaar>
__global__ void __launch_bounds__(kNaThreads) k_na_norms(const T* __restrict__ x, int64_t nx,
                                                          int64_t ng, DrawKey key, double gin_scale,
                                                          double* scratch) {
  __shared__ double red[kNaThreads / 32];
  const int64_t base = (int64_t)blockIdx.x * kNaTile;
  double sx = 0.0, sg = 0.0;
#pragma unroll 4
  for (int q = 0; q < kNaPerThread; q++) {
    const int64_t i = base + (int64_t)q * kNaThreads + threadIdx.x;
    if (i < nx) {
      const double v = (double)x[i];
      sx += v * v;
    }
  }
  if (kHaar) {
#pragma unroll 2
    for (int q = 0; q < kNaPerThread / 2; q++) {
      const int64_t j = base / 2 + (int64_t)q * kNaThreads + threadIdx.x;   // normal pair j
      if (2 * j < ng) {
        T a, b;
        normal_pair(key, (uint64_t)j, a, b);
        sg += (double)a * (double)a;
        if (2 * j + 1 < ng) sg += (double)b * (double)b;
      }
    }
  }
  sx = na_block_sum(sx, red);
  sg = na_block_sum(sg, red);
  if (threadIdx.x == 0) {
    scratch[2 * blockIdx.x] = sx;
    scratch[2 * blockIdx.x + 1] = sg;
  }
  unsigned int* counter = reinterpret_cast<unsigned int*>(scratch + kNaCounter);
  if (!elect_last_block(counter)) return;
  double tx = 0.0, tg = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += kNaThreads) {
    tx += __ldcg(scratch + 2 * b);
    tg += __ldcg(scratch + 2 * b + 1);
  }
  tx = na_block_sum(tx, red);
  tg = na_block_sum(tg, red);
  if (threadIdx.x == 0) {
    const double nrm = sqrt(tx);
    scratch[kNaCoef] = kHaar ? (tg > 0.0 ? nrm / sqrt(tg) : 0.0) : nrm * gin_scale;
  }
}

// y[i] = coefficient * g[i], g drawn as in kernel 1 (Haar: unscaled; Gin: unit normals,
// the scale being inside the coefficient).
template <typename T>
__global__ void __launch_bounds__(kNaThreads) k_na_out(T* __restrict__ y, int64_t ny, DrawKey key,
                                                        const double* scratch) {
  const double c = __ldcg(scratch + kNaCoef);
  const int64_t base = (int64_t)blockIdx.x * (kNaTile / 2);
#pragma unroll 2
  for (int q = 0; q < kNaPerThread / 2; q++) {
    const int64_t j = base + (int64_t)q * kNaThreads + threadIdx.x;
    if (2 * j < ny) {
      T a, b;
      normal_pair(key, (uint64_t)j, a, b);
      y[2 * j] = (T)(c * (double)a);
      if (2 * j + 1 < ny) y[2 * j + 1] = (T)(c * (double)b);
    }
  }
}

int na_fail(const char* where, cudaError_t e) {
  char msg[256];
  snprintf(msg, sizeof(msg), "hd_first_product_noalloc %s: %s", where, cudaGetErrorString(e));
  record_error_text(msg);
  return HD_ERR_CUDA;
}

// Device address of the scratch on the current device.  Looked up on every call rather than
// cached: the address belongs to the current context, which a device reset replaces.
int na_scratch(double** out) {
  double* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress((void**)&p, g_na_scratch);
  if (e != cudaSuccess) return na_fail("set-up (cudaGetSymbolAddress)", e);
  *out = p;
  return HD_OK;
}

template <typename T>
int na_run(bool haar, int64_t nx, int64_t ny, DrawKey key, double sigma, const void* x, void* y,
           cudaStream_t s, double* scratch) {
  cudaError_t e = cudaMemsetAsync(scratch + kNaCounter, 0, sizeof(unsigned int), s);
  if (e != cudaSuccess) return na_fail("counter clear", e);
  const int64_t nnorm = haar ? std::max(nx, ny) : nx;
  const unsigned t1 = (unsigned)((nnorm + kNaTile - 1) / kNaTile);
  const unsigned t2 = (unsigned)((ny + kNaTile - 1) / kNaTile);
  if (haar)
    k_na_norms<T, true><<<t1, kNaThreads, 0, s>>>((const T*)x, nx, ny, key, 1.0, scratch);
  else
    k_na_norms<T, false><<<t1, kNaThreads, 0, s>>>((const T*)x, nx, 0, key, sigma, scratch);
  e = cudaGetLastError();
  if (e != cudaSuccess) return na_fail("norm kernel launch", e);
  k_na_out<T><<<t2, kNaThreads, 0, s>>>((T*)y, ny, key, scratch);
  e = cudaGetLastError();
  if (e != cudaSuccess) return na_fail("output kernel launch", e);
  return HD_OK;
}

}  // namespace
}  // namespace hd

using namespace hd;

HD_API int hd_first_product_noalloc(int ensemble, int dtype, int64_t m, int64_t n,
                                               int transpose, uint64_t seed, uint32_t trial,
                                               double sigma, const void* x, void* y, void* stream) {
  if (ensemble != HD_GINIBRE && ensemble != HD_HAAR) return HD_ERR_ARG;
  if (dtype != HD_F64 && dtype != HD_F32) return HD_ERR_ARG;
  if (!x || !y || m <= 0 || n <= 0) return HD_ERR_ARG;
  if (ensemble == HD_GINIBRE && !(std::isfinite(sigma) && sigma > 0.0)) return HD_ERR_ARG;
  if (ensemble == HD_HAAR && m != n) return HD_ERR_DIM;
  if (m > kNaMaxDim || n > kNaMaxDim) {
    char msg[160];
    snprintf(msg, sizeof(msg),
             "hd_first_product_noalloc: max(m, n) = %lld exceeds the scratch limit of %lld entries",
             (long long)std::max(m, n), (long long)kNaMaxDim);
    record_error_text(msg);
    return HD_ERR_DIM;
  }
  double* scratch = nullptr;
  int rc = na_scratch(&scratch);
  if (rc) return rc;
  DrawKey key;
  key.k0 = (uint32_t)(seed & 0xFFFFFFFFu);
  key.k1 = (uint32_t)(seed >> 32);
  key.step = 1;
  key.trial = trial;
  key.stream = 0;
  const int64_t nx = transpose ? m : n;   // Q x: x in R^n, y in R^m; Q^T x: the reverse
  const int64_t ny = transpose ? n : m;
  const bool haar = ensemble == HD_HAAR;
  cudaStream_t s = (cudaStream_t)stream;
  return dtype == HD_F64 ? na_run<double>(haar, nx, ny, key, sigma, x, y, s, scratch)
                         : na_run<float>(haar, nx, ny, key, sigma, x, y, s, scratch);
}
