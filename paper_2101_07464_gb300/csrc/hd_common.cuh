// Device helpers shared by the Householder Dice kernels (sm_103a).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace hd {

constexpr int kThreads = 256;          // threads per CTA of every streaming kernel
constexpr int kWarps = kThreads / 32;
constexpr int kChunkMax = 4;           // 16-byte vectors per thread per sweep (registers)
// Resident CTAs per SM that every sweep kernel is compiled for (registers capped to fit) and
// that the CTA maps are sized to: one wave of kSweepCtasPerSm CTAs of up to 8 warps per SM.
constexpr int kSweepCtasPerSm = 2;
constexpr int kColBlock = 8;           // stack columns per register block in a sweep
constexpr int kFinThreads = 256;       // threads of the single-CTA finalisation
constexpr int kTmaxLimit = 256;        // column owners hold at most 8 columns per lane

// ---------------------------------------------------------------------------------
// 16-byte vectors: 4 floats or 2 doubles per thread access.
template <typename T> struct Vec;
template <> struct Vec<float> {
  static constexpr int N = 4;
  float e[4];
};
template <> struct Vec<double> {
  static constexpr int N = 2;
  double e[2];
};

// Streaming (evict-first) load of data that this kernel does not write.
__device__ __forceinline__ void ld_stream(const float* p, Vec<float>& v) {
  float4 q = __ldcs(reinterpret_cast<const float4*>(p));
  v.e[0] = q.x; v.e[1] = q.y; v.e[2] = q.z; v.e[3] = q.w;
}
__device__ __forceinline__ void ld_stream(const double* p, Vec<double>& v) {
  double2 q = __ldcs(reinterpret_cast<const double2*>(p));
  v.e[0] = q.x; v.e[1] = q.y;
}
__device__ __forceinline__ void st_vec(float* p, const Vec<float>& v) {
  *reinterpret_cast<float4*>(p) = make_float4(v.e[0], v.e[1], v.e[2], v.e[3]);
}
__device__ __forceinline__ void st_vec(double* p, const Vec<double>& v) {
  *reinterpret_cast<double2*>(p) = make_double2(v.e[0], v.e[1]);
}

// Load rows [row, row+N) of a caller vector of length dim: vector load when in range and
// aligned, element loads with zero fill at the ragged end or on unaligned buffers.
template <typename T>
__device__ __forceinline__ void ld_caller(const T* p, int64_t row, int64_t dim, bool aligned,
                                          Vec<T>& v) {
  constexpr int N = Vec<T>::N;
  if (aligned && row + N <= dim) {
    ld_stream(p + row, v);
  } else {
#pragma unroll
    for (int q = 0; q < N; q++) v.e[q] = (row + q < dim) ? p[row + q] : T(0);
  }
}
template <typename T>
__device__ __forceinline__ void st_caller(T* p, int64_t row, int64_t dim, bool aligned,
                                          const Vec<T>& v) {
  constexpr int N = Vec<T>::N;
  if (aligned && row + N <= dim) {
    st_vec(p + row, v);
  } else {
#pragma unroll
    for (int q = 0; q < N; q++)
      if (row + q < dim) p[row + q] = v.e[q];
  }
}

// ---------------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds of
//   (hi0, lo0) = M0*c0, (hi1, lo1) = M1*c2,  c <- (hi1^c1^k0, lo1, hi0^c3^k1, lo0),
// with the key bumped by the Weyl constants between rounds.
struct PhiloxOut {
  uint32_t w[4];
};
__device__ __forceinline__ PhiloxOut philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2,
                                                   uint32_t c3, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; r++) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  PhiloxOut o;
  o.w[0] = c0; o.w[1] = c1; o.w[2] = c2; o.w[3] = c3;
  return o;
}

struct DrawKey {
  uint32_t k0, k1;    // seed
  uint32_t step;      // paper's t (1-based)
  uint32_t trial;
  uint32_t stream;
};

// Normals 2j and 2j+1: u = (53-bit integer + 1) 2^-53 in (0, 1] from two words, then
// Box-Muller r = sqrt(-2 ln u1), (r cos 2 pi u2, r sin 2 pi u2).
__device__ __forceinline__ void normal_pair(const DrawKey& k, uint64_t j, double& z0, double& z1) {
  PhiloxOut o = philox4x32_10((uint32_t)j, k.step, k.trial, k.stream, k.k0, k.k1);
  const double u1 = ((double)((((uint64_t)o.w[0]) << 21) | (o.w[1] >> 11)) + 1.0) * 0x1.0p-53;
  const double u2 = ((double)((((uint64_t)o.w[2]) << 21) | (o.w[3] >> 11)) + 1.0) * 0x1.0p-53;
  const double r = sqrt(-2.0 * log(u1));
  double sn, cs;
  sincospi(2.0 * u2, &sn, &cs);
  z0 = r * cs;
  z1 = r * sn;
}
// The same words through 32-bit arithmetic: u = w_hi 2^-32 + ((w_lo >> 11) + 1) 2^-53 equals
// the 53-bit uniform up to float rounding (relative 2^-24), then Box-Muller in FP32.  Near
// u1 = 1 the rounded u1 would lose the small quantity 1 - u1 that ln u1 depends on (a normal
// near zero would then be off by up to about 2^-12), so for u1 >= 1 - 2^-10 ln u1 is formed
// as log1p(-v) from v = 1 - u1 = (2^53 - 1 - k) 2^-53, which the words give exactly before
// one float rounding.  That branch is taken by about 3% of warps.
__device__ __forceinline__ void normal_pair(const DrawKey& k, uint64_t j, float& z0, float& z1) {
  PhiloxOut o = philox4x32_10((uint32_t)j, k.step, k.trial, k.stream, k.k0, k.k1);
  const float u2 = fmaf((float)o.w[2], 0x1.0p-32f, (float)((o.w[3] >> 11) + 1u) * 0x1.0p-53f);
  float l;
  if (o.w[0] >= 0xFFC00000u) {
    const float v = fmaf((float)(0xFFFFFFFFu - o.w[0]), 0x1.0p-32f, (float)(0x1FFFFFu - (o.w[1] >> 11)) * 0x1.0p-53f);
    l = log1pf(-v);
  } else {
    l = logf(fmaf((float)o.w[0], 0x1.0p-32f, (float)((o.w[1] >> 11) + 1u) * 0x1.0p-53f));
  }
  const float r = sqrtf(-2.0f * l);
  float sn, cs;
  sincospif(2.0f * u2, &sn, &cs);
  z0 = r * cs;
  z1 = r * sn;
}

// Draw rows [row, row+N) (row even, N even) of the step's vector, scaled by sigma, with
// zeros at rows < first (the masked head Z_{1:first}) and rows >= dim.
template <typename T>
__device__ __forceinline__ void draw_vec(const DrawKey& k, int64_t row, int64_t first, int64_t dim,
                                         T sigma, Vec<T>& v) {
  constexpr int N = Vec<T>::N;
  if (row + N <= first || row >= dim) {
#pragma unroll
    for (int q = 0; q < N; q++) v.e[q] = T(0);
    return;
  }
#pragma unroll
  for (int q = 0; q < N; q += 2) {
    T a, b;
    normal_pair(k, (uint64_t)(row + q) >> 1, a, b);
    v.e[q] = (row + q >= first && row + q < dim) ? sigma * a : T(0);
    v.e[q + 1] = (row + q + 1 >= first && row + q + 1 < dim) ? sigma * b : T(0);
  }
}

// ---------------------------------------------------------------------------------
// Reductions.  Per-warp partial sums are formed in the storage type (FP32 in the mixed
// mode: at most 32 * kChunkMax * 4 products), everything above the warp in FP64.
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

// Sum NV per-thread values over the CTA; thread q < NV receives the total of value q in
// out[q] (FP64).  red: shared scratch of kWarps * NV doubles.  Contains __syncthreads.
template <int NV, typename T>
__device__ __forceinline__ void block_sum(const T (&a)[NV], double* red, double* out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NV; q++) {
    T s = warp_sum(a[q]);
    if (lane == 0) red[warp * NV + q] = (double)s;
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < kWarps; w++) s += red[w * NV + threadIdx.x];
    out[threadIdx.x] = s;
  }
  __syncthreads();
}

// Last-block election: every CTA has written its partial sums; the CTA that increments
// the counter last sees all of them (no waiting: the others simply exit).  The elected
// CTA resets the counter for the next launch.
__device__ __forceinline__ bool elect_last_block(unsigned int* counter) {
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned int prev = atomicAdd(counter, 1u);
    last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (last) {
    __threadfence();
    if (threadIdx.x == 0) *counter = 0u;
  }
  return last;
}

// Coherent load of a value written by another CTA of the same launch.
__device__ __forceinline__ double ld_cg(const double* p) { return __ldcg(p); }

}  // namespace hd
