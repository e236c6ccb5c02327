// Device helpers shared by the Householder Dice kernels (sm_103a).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "hd_log_table.cuh"

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

// ---------------------------------------------------------------------------------
// FP64 Box-Muller with few FP64 operations.  On this GPU the FP64 pipe runs at 1/64 of the
// FP32 rate and bounds the FP64 sweeps, so the logarithm and the sine-cosine of the draws
// keep FP64 arithmetic for the terms whose size needs it and take the rest from integer and
// FP32 operations; each result is within a few units in the last place of the FP64 value.
constexpr double kLn2 = 0x1.62e42fefa39efp-1;          // ln 2 rounded to FP64
constexpr double kPiScaled = 0x1.921fb54442d18p-51;    // pi 2^-52 (pi rounded to FP64)

// ln u for u = K 2^-53, K in [1, 2^53].  u = m 2^e with m in [0.75, 1.5) (from the bits of K:
// no cancellation between e ln 2 and ln m near u = 1), and ln m = -ln c_i + ln(1 + r) with
// r = m c_i - 1 (one FMA) for the table entry i = round(256 (m - 1)), |r| <= 0.0026 (table
// method: Tang, ACM TOMS 16, 1990).  ln(1 + r) = r + r^2 (-1/2 + r (1/3 + q)): the series'
// terms beyond r^3 / 3, q = -r/4 + r^2/5 - r^3/6, are below 2^-30 and are formed in FP32.
__device__ __forceinline__ double log_u53(uint64_t K) {
  if (K >= (1ull << 53)) return 0.0;
  const int lz = __clzll((long long)K) - 11;             // K < 2^53: 0 .. 52
  const uint64_t Kp = K << lz;                            // [2^52, 2^53): m_n = Kp 2^-52 in [1, 2)
  const bool half = (Kp >> 51) & 1ull;                    // m_n >= 1.5: take m = m_n / 2
  const uint64_t mant = Kp & ((1ull << 52) - 1ull);
  const double m = __longlong_as_double((long long)(((half ? 0x3FEull : 0x3FFull) << 52) | mant));
  const int e = half ? -lz : -1 - lz;                     // u = m 2^e
  const int i = half ? -(int)(((1ull << 53) - Kp + (1ull << 44)) >> 45)   // m in [0.75, 1): -64 .. 0
                     : (int)((Kp - (1ull << 52) + (1ull << 43)) >> 44);   // m in [1, 1.5): 0 .. 128
  const double2 ct = __ldg(&kLogTab[i - kLogTabLo]);
  const double r = fma(m, ct.x, -1.0);
  const float rf = (float)r;
  const float q = rf * fmaf(rf, fmaf(rf, -1.0f / 6.0f, 0.2f), -0.25f);
  const double inner = fma(r, 0x1.5555555555555p-2 + (double)q, -0.5);   // -1/2 + r (1/3 + q)
  const double lm = fma(r * r, inner, r);                                 // ln(1 + r)
  return fma((double)e, kLn2, ct.y) + lm;
}

// sin(pi x), cos(pi x) for x = K 2^-52, K in [1, 2^53] (x in (0, 2]).  x = n/2 + y with
// n = round(2x) and |y| <= 1/4 exactly in integers; z = pi y; the Taylor series of sin z and
// cos z in w = z^2 keep FP64 for the terms above 4e-8 and FP32 for the rest (the error of the
// FP32 part stays below 2e-16); then the quadrant n mod 4 selects and signs the two.
__device__ __forceinline__ void sincospi_u52(uint64_t K, double& sn, double& cs) {
  const uint64_t n = (K + (1ull << 50)) >> 51;                  // 0 .. 4
  const long long D = (long long)K - (long long)(n << 51);     // 2^52 y, |D| <= 2^50
  const double z = (double)D * kPiScaled;
  const double w = z * z;
  const float wf = (float)w;
  // sin z = z + z^3 S(w): S = -1/3! + w/5! - w^2/7! + w^3/9! + w^4 (-1/11! + w/13! - w^2/15!)
  const float ts = fmaf(wf, fmaf(wf, -0x1.ae7f3ep-41f, 0x1.612462p-33f), -0x1.ae6456p-26f);
  double S = fma(w, (double)ts, 0x1.71de3a556c734p-19);         // 1/9!
  S = fma(w, S, -0x1.a01a01a01a01ap-13);                        // -1/7!
  S = fma(w, S, 0x1.1111111111111p-7);                          // 1/5!
  S = fma(w, S, -0x1.5555555555555p-3);                         // -1/3!
  const double s = fma(z * w, S, z);
  // cos z = 1 + w C(w): C = -1/2! + w/4! - w^2/6! + w^3/8! - w^4/10! + w^5 (1/12! - w/14! + w^2/16!)
  const float tc = fmaf(wf, fmaf(wf, 0x1.ae7f3ep-45f, -0x1.93974ap-37f), 0x1.1eed8ep-29f);
  double C = fma(w, (double)tc, -0x1.27e4fb7789f5cp-22);        // -1/10!
  C = fma(w, C, 0x1.a01a01a01a01ap-16);                         // 1/8!
  C = fma(w, C, -0x1.6c16c16c16c17p-10);                        // -1/6!
  C = fma(w, C, 0x1.5555555555555p-5);                          // 1/4!
  C = fma(w, C, -0.5);
  const double c = fma(w, C, 1.0);
  // theta = n pi / 2 + z
  const unsigned q = (unsigned)n & 3u;
  const double a = (q & 1u) ? c : s;                            // |sin theta|
  const double b = (q & 1u) ? s : c;                            // |cos theta|
  sn = (q >= 2u) ? -a : a;
  cs = (q == 1u || q == 2u) ? -b : b;
}

// Normals 2j and 2j+1: u = (53-bit integer + 1) 2^-53 in (0, 1] from two words, then
// Box-Muller r = sqrt(-2 ln u1), (r cos 2 pi u2, r sin 2 pi u2).
__device__ __forceinline__ void normal_pair(const DrawKey& k, uint64_t j, double& z0, double& z1) {
  PhiloxOut o = philox4x32_10((uint32_t)j, k.step, k.trial, k.stream, k.k0, k.k1);
  const uint64_t K1 = ((((uint64_t)o.w[0]) << 21) | (o.w[1] >> 11)) + 1ull;
  const uint64_t K2 = ((((uint64_t)o.w[2]) << 21) | (o.w[3] >> 11)) + 1ull;
  const double r = sqrt(-2.0 * log_u53(K1));
  double sn, cs;
  sincospi_u52(K2, sn, cs);
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
