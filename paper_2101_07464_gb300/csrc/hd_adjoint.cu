// Reverse mode of Householder Dice: the adjoint of a recorded single-trial trajectory.
//
// With the Gaussian draws held fixed, the outputs y_1..y_T of Algorithms 1 and 2 are a
// deterministic function of the step inputs x_1..x_T.  y_t depends on x_t directly and on the
// earlier inputs through the data-side reflectors they created (R_s = H_s(p_s), eq.
// Householder_e) and, for Ginibre, through the basis vectors built with those reflectors.
// hd_adjoint_step reverses the forward steps one at a time, last first.  Given ybar_t =
// dLoss/dy_t it returns xbar_t = dLoss/dx_t through every product that x_t reaches, i.e. y_t
// itself and all later steps through the reflector built from x_t.
//
// The forward steps are composed of three kinds of operation on the compact WY form
// (I - V S V^T = P_0 ... P_{K-1}, Delta the prefix signs of the reflectors' scalar factors):
//   data product     p = Delta (I - V S^T V^T) x            (z = V^T x, w = S^T z)
//   output product   y = (I - V S V^T) Delta c              (a = V^T Delta c, b = S a)
//   new reflector    u = p[k:] + s alpha e_k, alpha = ||p[k:]||, s = sign(p_k)
//   and S = (strict_upper(G) + diag(G)/2)^{-1} with G = V^T V.
// Their adjoints are accumulated into Vbar (per stack, like V), Sbar (upper triangle only),
// and for Ginibre Bbar (per basis store).  When the reverse pass reaches the step that created
// column j of a stack, every later use of that column has been accounted for: the explicit
// terms are in Vbar[:, j], and the terms through S (Gbar = upper(-S^T Sbar S^T) with half
// diagonal, Vbar += V (Gbar + Gbar^T)) depend only on entries of Sbar in columns >= j, which
// are complete.  The column's adjoint then goes back into p and, through the data product,
// into x and into the older columns.  Forward quantities (z, w, p, alpha) are recomputed from
// the recorded x_t and the final stacks, whose leading blocks are the stacks of step t.
// The sign s and the prefix signs are piecewise constant and carry no derivative; an identity
// reflector (alpha = 0) passes no derivative to p.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>

#include <cuda_runtime.h>

#include "../../include/hd.h"
#include "hd_common.cuh"
#include "hd_state.cuh"

namespace hd {
namespace {

constexpr int kAT = 256;   // threads of every adjoint kernel
constexpr int kSmallT = 1024;   // threads of the small FP64 kernels (FP64 latency wants many warps)

// A pointer with the distance between consecutive trials of a batched state (all trials of
// a batch in reverse mode have the same dimensions, so every per-trial array is evenly
// spaced).  Kernels take the trial from blockIdx.z.
template <typename P>
struct TP {
  P* p;
  int64_t s;
  __host__ __device__ P* at(int tr) const { return p ? p + (int64_t)tr * s : nullptr; }
};
template <typename P>
__host__ __device__ inline TP<P> tp(P* p, int64_t s) { return TP<P>{p, s}; }

// qbar, zbar and E have a second copy: a reverse step uses the copy of its step's parity, so a
// step's data-side update held back for the next call keeps its vectors while that call forms
// its own (the two sides of a Haar reverse step run on two streams).
enum AdjVec { kVp, kVub, kVqb, kVg, kVqb2, kAdjVecs };
enum AdjSmall {
  kSz, kSw, kSh, kSbb, kSb, kScb, kSzb, kSwb, kSE, kSc, kShb, kSau, kSbu, kSbbu, kSabu, kSscal, kSzb2, kSE2,
  kAdjSmall
};

// Precision: the streaming passes over the stacks run in the state's precision T (FP32 for an
// FP32 state, as the forward sweeps do: GB300's FP64 rate would bound them otherwise); every
// sum across threads or CTAs, the small coefficient vectors and Sbar are FP64.

__device__ __forceinline__ double a_block_sum(double v, double* red) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); w++) s += red[w];
  return s;
}

// Partial column dots: CTA (x, y) covers row chunk x and the 8 columns 8y..8y+7, one warp per
// column; part[(x K + j) 2 + v] = sum over the chunk of A[r, j] v_v[r] (per-lane sums in T over
// at most ~100 rows, eight loads in flight per lane, FP64 across lanes).
template <typename T>
__global__ void __launch_bounds__(kAT) k_colpass(TP<const T> A_, int64_t ld, int K, int64_t dim,
                                                 TP<const T> v1_, TP<const T> v2_, TP<double> part_) {
  const int tr = blockIdx.z;
  const T* __restrict__ A = A_.at(tr);
  const T* __restrict__ v1 = v1_.at(tr);
  const T* __restrict__ v2 = v2_.at(tr);
  double* part = part_.at(tr);
  const int64_t per = ((dim + gridDim.x - 1) / gridDim.x + 31) / 32 * 32;
  const int64_t r0 = (int64_t)blockIdx.x * per, r1 = min(dim, r0 + per);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int j = blockIdx.y * 8 + warp;
  if (j >= K) return;
  const T* Aj = A + (int64_t)j * ld;
  T s1 = T(0), s2 = T(0), t1 = T(0), t2 = T(0);
  int64_t r = r0 + lane;
#pragma unroll 4
  for (; r + 32 < r1; r += 64) {
    const T a0 = Aj[r], a1 = Aj[r + 32];
    s1 = fma(a0, v1[r], s1);
    t1 = fma(a1, v1[r + 32], t1);
    if (v2) {
      s2 = fma(a0, v2[r], s2);
      t2 = fma(a1, v2[r + 32], t2);
    }
  }
  if (r < r1) {
    const T a0 = Aj[r];
    s1 = fma(a0, v1[r], s1);
    if (v2) s2 = fma(a0, v2[r], s2);
  }
  const double d1 = warp_sum((double)s1 + (double)t1);
  const double d2 = warp_sum((double)s2 + (double)t2);
  if (lane == 0) {
    part[((int64_t)blockIdx.x * K + j) * 2] = d1;
    part[((int64_t)blockIdx.x * K + j) * 2 + 1] = d2;
  }
}

// out_v[j] = scale_v * sum over the nblk row chunks of the partials: one warp per column, the
// lanes over the chunks, then a shuffle reduction (fixed order: deterministic).
__device__ __forceinline__ void colreduce_col(const double* __restrict__ part, int nblk, int K, int j,
                                              double s1, double* out1, double s2, double* out2) {
  const int lane = threadIdx.x & 31;
  double a0 = 0.0, b0 = 0.0, a1 = 0.0, b1 = 0.0;   // two chains each: the loads overlap
  int q = lane;
  for (; q + 32 < nblk; q += 64) {
    a0 += part[((int64_t)q * K + j) * 2];
    b0 += part[((int64_t)q * K + j) * 2 + 1];
    a1 += part[((int64_t)(q + 32) * K + j) * 2];
    b1 += part[((int64_t)(q + 32) * K + j) * 2 + 1];
  }
  if (q < nblk) {
    a0 += part[((int64_t)q * K + j) * 2];
    b0 += part[((int64_t)q * K + j) * 2 + 1];
  }
  const double a = warp_sum(a0 + a1);
  const double b = warp_sum(b0 + b1);
  if (lane == 0) {
    out1[j] = s1 * a;
    if (out2) out2[j] = s2 * b;
  }
}
__global__ void __launch_bounds__(kAT) k_colreduce(TP<const double> part, int nblk, int K,
                                                   double s1, TP<double> out1, double s2, TP<double> out2) {
  const int tr = blockIdx.z;
  const int j = blockIdx.x * (kAT / 32) + (threadIdx.x >> 5);
  if (j < K) colreduce_col(part.at(tr), nblk, K, j, s1, out1.at(tr), s2, out2.at(tr));
}

// out[r] (+)= sgn(r) (s_in in[r] + c_scale sum_{j<K} A[r, j] c[j]), sgn(r) = dpre[min(r+1, Kd)]
// (or 1); optionally per-CTA FP64 partial sums of out[r]^2 over r >= rnorm.
template <typename T>
__global__ void __launch_bounds__(kAT) k_rowpass(TP<T> out_, TP<const T> in_, double s_in, TP<const T> A_,
                                                 int64_t ld, int K, TP<const double> c_, double c_scale,
                                                 int64_t dim, TP<const double> dpre_, int Kd,
                                                 int accumulate, int64_t rnorm, TP<double> npart_) {
  const int tr = blockIdx.z;
  T* out = out_.at(tr);
  const T* in = in_.at(tr);
  const T* __restrict__ A = A_.at(tr);
  const double* __restrict__ c = c_.at(tr);
  const double* __restrict__ dpre = dpre_.at(tr);
  double* npart = npart_.at(tr);
  __shared__ T cs[kTmaxLimit + 1];
  __shared__ double red[kAT / 32];
  for (int j = threadIdx.x; j < K; j += blockDim.x) cs[j] = (T)(c_scale * c[j]);
  __syncthreads();
  const T si = (T)s_in;
  double ns = 0.0;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < dim; r += (int64_t)gridDim.x * blockDim.x) {
    T v0 = in ? si * in[r] : T(0), v1 = T(0), v2 = T(0), v3 = T(0);
    const T* Ar = A + r;
    int j = 0;
    for (; j + 4 <= K; j += 4) {
      v0 = fma(Ar[(int64_t)j * ld], cs[j], v0);
      v1 = fma(Ar[(int64_t)(j + 1) * ld], cs[j + 1], v1);
      v2 = fma(Ar[(int64_t)(j + 2) * ld], cs[j + 2], v2);
      v3 = fma(Ar[(int64_t)(j + 3) * ld], cs[j + 3], v3);
    }
    for (; j < K; j++) v0 = fma(Ar[(int64_t)j * ld], cs[j], v0);
    T v = (v0 + v1) + (v2 + v3);
    if (dpre) v *= (T)dpre[min(r + 1, (int64_t)Kd)];
    if (accumulate) v += out[r];
    out[r] = v;
    if (r >= rnorm) ns = fma((double)v, (double)v, ns);
  }
  if (npart) {
    ns = a_block_sum(ns, red);
    if (threadIdx.x == 0) npart[blockIdx.x] = ns;
  }
}

// Ab[r, j] += a[r] b[j] + c[r] d[j] + e[r] f[j] for r < dim, j < K (column-major, leading dim
// ld; b, d, f are FP64 coefficient vectors with the scales sb, sd, sf; c, e may be null).
template <typename T>
__global__ void __launch_bounds__(kAT) k_rank(TP<T> Ab_, int64_t ld, int K, int64_t dim, TP<const T> a_,
                                              TP<const double> b_, double sb, TP<const T> c_,
                                              TP<const double> d_, double sd, TP<const T> e_,
                                              TP<const double> f_, double sf, int Kf) {
  const int tr = blockIdx.z;
  T* Ab = Ab_.at(tr);
  const T* __restrict__ a = a_.at(tr);
  const double* __restrict__ b = b_.at(tr);
  const T* __restrict__ c = c_.at(tr);
  const double* __restrict__ d = d_.at(tr);
  const T* __restrict__ e = e_.at(tr);
  const double* __restrict__ f = f_.at(tr);
  __shared__ T bs[8], ds[8], fs[8];
  const int j0 = blockIdx.y * 8;
  if (threadIdx.x < 8) {
    const int j = j0 + threadIdx.x;
    bs[threadIdx.x] = (j < K) ? (T)(sb * b[j]) : T(0);
    ds[threadIdx.x] = (j < K && c) ? (T)(sd * d[j]) : T(0);
    fs[threadIdx.x] = (j < Kf && e) ? (T)(sf * f[j]) : T(0);
  }
  __syncthreads();
  const int jn = min(K, j0 + 8) - j0;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < dim; r += (int64_t)gridDim.x * blockDim.x) {
    const T ar = a[r];
    const T cr = c ? c[r] : T(0);
    const T er = e ? e[r] : T(0);
    for (int q = 0; q < jn; q++) {
      T v = ar * bs[q];
      if (c) v = fma(cr, ds[q], v);
      if (e) v = fma(er, fs[q], v);
      Ab[r + (int64_t)(j0 + q) * ld] += v;
    }
  }
}

// FP32, 16-byte aligned: four rows per thread; every thread loads its rows of a, c, e once and
// walks all K columns, eight column loads in flight at a time.
__global__ void __launch_bounds__(kAT) k_rank4(TP<float> Ab_, int64_t ld, int K, int64_t dim4, TP<const float> a_,
                                               TP<const double> b_, double sb, TP<const float> c_,
                                               TP<const double> d_, double sd, TP<const float> e_,
                                               TP<const double> f_, double sf, int Kf) {
  const int tr = blockIdx.z;
  float* Ab = Ab_.at(tr);
  const float* __restrict__ a = a_.at(tr);
  const double* __restrict__ b = b_.at(tr);
  const float* __restrict__ c = c_.at(tr);
  const double* __restrict__ d = d_.at(tr);
  const float* __restrict__ e = e_.at(tr);
  const double* __restrict__ f = f_.at(tr);
  __shared__ float bs[kTmaxLimit + 1], ds[kTmaxLimit + 1], fs[kTmaxLimit + 1];
  for (int j = threadIdx.x; j < K; j += blockDim.x) {
    bs[j] = (float)(sb * b[j]);
    ds[j] = c ? (float)(sd * d[j]) : 0.f;
    fs[j] = (e && j < Kf) ? (float)(sf * f[j]) : 0.f;
  }
  __syncthreads();
  const int64_t ld4 = ld / 4;
  for (int64_t q4 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q4 < dim4; q4 += (int64_t)gridDim.x * blockDim.x) {
    const float4 ar = reinterpret_cast<const float4*>(a)[q4];
    const float4 cr = c ? reinterpret_cast<const float4*>(c)[q4] : make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 er = e ? reinterpret_cast<const float4*>(e)[q4] : make_float4(0.f, 0.f, 0.f, 0.f);
    float4* col0 = reinterpret_cast<float4*>(Ab) + q4;
    for (int j0 = 0; j0 < K; j0 += 8) {
      const int jn = min(8, K - j0);
      float4 v[8];
#pragma unroll
      for (int jj = 0; jj < 8; jj++)
        if (jj < jn) v[jj] = col0[(int64_t)(j0 + jj) * ld4];
#pragma unroll
      for (int jj = 0; jj < 8; jj++) {
        if (jj < jn) {
          const float bq = bs[j0 + jj], dq = ds[j0 + jj], fq = fs[j0 + jj];
          v[jj].x = fmaf(er.x, fq, fmaf(cr.x, dq, fmaf(ar.x, bq, v[jj].x)));
          v[jj].y = fmaf(er.y, fq, fmaf(cr.y, dq, fmaf(ar.y, bq, v[jj].y)));
          v[jj].z = fmaf(er.z, fq, fmaf(cr.z, dq, fmaf(ar.z, bq, v[jj].z)));
          v[jj].w = fmaf(er.w, fq, fmaf(cr.w, dq, fmaf(ar.w, bq, v[jj].w)));
          col0[(int64_t)(j0 + jj) * ld4] = v[jj];
        }
      }
    }
  }
}

// Up to five rank-one terms in one pass: Ab[:, j] += sum_q v_q (s_q c_q[j]) for j < min(K, K_q).
struct RankTerms {
  const void* v[5];
  const double* c[5];
  double s[5];
  int K[5];
  int64_t sv[5];   // trial strides of v (elements) and c (doubles)
  int64_t sc[5];
  int n;
};
template <typename T>
__global__ void __launch_bounds__(kAT) k_rankN(TP<T> Ab_, int64_t ld, int K, int64_t dim, RankTerms t) {
  const int tr = blockIdx.z;
  T* Ab = Ab_.at(tr);
#pragma unroll
  for (int q = 0; q < 5; q++) {
    if (q < t.n) {
      t.v[q] = (const T*)t.v[q] + (int64_t)tr * t.sv[q];
      t.c[q] = t.c[q] + (int64_t)tr * t.sc[q];
    }
  }
  __shared__ T cs[5][8];
  const int j0 = blockIdx.y * 8;
  if (threadIdx.x < 40) {
    const int q = threadIdx.x >> 3, jj = threadIdx.x & 7, j = j0 + jj;
    cs[q][jj] = (q < t.n && j < K && j < t.K[q]) ? (T)(t.s[q] * t.c[q][j]) : T(0);
  }
  __syncthreads();
  const int jn = min(K, j0 + 8) - j0;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < dim; r += (int64_t)gridDim.x * blockDim.x) {
    T vr[5];
#pragma unroll
    for (int q = 0; q < 5; q++) vr[q] = (q < t.n) ? ((const T*)t.v[q])[r] : T(0);
    for (int jj = 0; jj < jn; jj++) {
      T* col = Ab + (int64_t)(j0 + jj) * ld;
      T v = col[r];
#pragma unroll
      for (int q = 0; q < 5; q++) v = fma(vr[q], cs[q][jj], v);
      col[r] = v;
    }
  }
}
// FP32, 16-byte aligned: four rows per thread; every thread loads its rows of the terms' vectors
// once and walks all K columns, eight column loads in flight at a time.
__global__ void __launch_bounds__(kAT) k_rankN4(TP<float> Ab_, int64_t ld, int K, int64_t dim4, RankTerms t) {
  const int tr = blockIdx.z;
  float* Ab = Ab_.at(tr);
#pragma unroll
  for (int q = 0; q < 5; q++) {
    if (q < t.n) {
      t.v[q] = (const float*)t.v[q] + (int64_t)tr * t.sv[q];
      t.c[q] = t.c[q] + (int64_t)tr * t.sc[q];
    }
  }
  __shared__ float cs[5][kTmaxLimit + 1];
  for (int idx = threadIdx.x; idx < 5 * K; idx += blockDim.x) {
    const int q = idx / K, j = idx % K;
    cs[q][j] = (q < t.n && j < t.K[q]) ? (float)(t.s[q] * t.c[q][j]) : 0.f;
  }
  __syncthreads();
  const int64_t ld4 = ld / 4;
  for (int64_t q4 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q4 < dim4; q4 += (int64_t)gridDim.x * blockDim.x) {
    float4 vr[5];
#pragma unroll
    for (int q = 0; q < 5; q++)
      vr[q] = (q < t.n) ? reinterpret_cast<const float4*>(t.v[q])[q4] : make_float4(0.f, 0.f, 0.f, 0.f);
    float4* col0 = reinterpret_cast<float4*>(Ab) + q4;
    for (int j0 = 0; j0 < K; j0 += 8) {
      const int jn = min(8, K - j0);
      float4 v[8];
#pragma unroll
      for (int jj = 0; jj < 8; jj++)
        if (jj < jn) v[jj] = col0[(int64_t)(j0 + jj) * ld4];
#pragma unroll
      for (int jj = 0; jj < 8; jj++) {
        if (jj < jn) {
#pragma unroll
          for (int q = 0; q < 5; q++) {
            const float cq = cs[q][j0 + jj];
            v[jj].x = fmaf(vr[q].x, cq, v[jj].x);
            v[jj].y = fmaf(vr[q].y, cq, v[jj].y);
            v[jj].z = fmaf(vr[q].z, cq, v[jj].z);
            v[jj].w = fmaf(vr[q].w, cq, v[jj].w);
          }
          col0[(int64_t)(j0 + jj) * ld4] = v[jj];
        }
      }
    }
  }
}

__global__ void __launch_bounds__(kAT) k_rowpass4(TP<float> out_, TP<const float> in_, double s_in,
                                                  TP<const float> A_, int64_t ld, int K, TP<const double> c_,
                                                  double c_scale, int64_t dim4, int accumulate) {
  const int tr = blockIdx.z;
  float* out = out_.at(tr);
  const float* in = in_.at(tr);
  const float* __restrict__ A = A_.at(tr);
  const double* __restrict__ c = c_.at(tr);
  __shared__ float cs[kTmaxLimit + 1];
  for (int j = threadIdx.x; j < K; j += blockDim.x) cs[j] = (float)(c_scale * c[j]);
  __syncthreads();
  const float si = (float)s_in;
  for (int64_t q4 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q4 < dim4; q4 += (int64_t)gridDim.x * blockDim.x) {
    float4 v = in ? reinterpret_cast<const float4*>(in)[q4] : make_float4(0.f, 0.f, 0.f, 0.f);
    v.x *= si; v.y *= si; v.z *= si; v.w *= si;
    const float4* Aq = reinterpret_cast<const float4*>(A) + q4;
    const int64_t ld4 = ld / 4;
    int j = 0;
    for (; j + 4 <= K; j += 4) {   // four column loads in flight
      const float4 a0 = Aq[(int64_t)j * ld4], a1 = Aq[(int64_t)(j + 1) * ld4];
      const float4 a2 = Aq[(int64_t)(j + 2) * ld4], a3 = Aq[(int64_t)(j + 3) * ld4];
      const float c0 = cs[j], c1 = cs[j + 1], c2 = cs[j + 2], c3 = cs[j + 3];
      v.x = fmaf(a3.x, c3, fmaf(a2.x, c2, fmaf(a1.x, c1, fmaf(a0.x, c0, v.x))));
      v.y = fmaf(a3.y, c3, fmaf(a2.y, c2, fmaf(a1.y, c1, fmaf(a0.y, c0, v.y))));
      v.z = fmaf(a3.z, c3, fmaf(a2.z, c2, fmaf(a1.z, c1, fmaf(a0.z, c0, v.z))));
      v.w = fmaf(a3.w, c3, fmaf(a2.w, c2, fmaf(a1.w, c1, fmaf(a0.w, c0, v.w))));
    }
    for (; j < K; j++) {
      const float4 aj = Aq[(int64_t)j * ld4];
      const float cj = cs[j];
      v.x = fmaf(aj.x, cj, v.x);
      v.y = fmaf(aj.y, cj, v.y);
      v.z = fmaf(aj.z, cj, v.z);
      v.w = fmaf(aj.w, cj, v.w);
    }
    if (accumulate) {
      const float4 o = reinterpret_cast<const float4*>(out)[q4];
      v.x += o.x; v.y += o.y; v.z += o.z; v.w += o.w;
    }
    reinterpret_cast<float4*>(out)[q4] = v;
  }
}

// Column pass, float4: CTA (x, y) = row chunk x (a multiple of 128 rows) and columns 8y..8y+7.
__global__ void __launch_bounds__(kAT) k_colpass4(TP<const float> A_, int64_t ld, int K, int64_t dim4,
                                                  TP<const float> v1_, TP<const float> v2_, TP<double> part_) {
  const int tr = blockIdx.z;
  const float* __restrict__ A = A_.at(tr);
  const float* __restrict__ v1 = v1_.at(tr);
  const float* __restrict__ v2 = v2_.at(tr);
  double* part = part_.at(tr);
  const int64_t per = ((dim4 + gridDim.x - 1) / gridDim.x + 31) / 32 * 32;
  const int64_t q0 = (int64_t)blockIdx.x * per, q1 = min(dim4, q0 + per);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int j = blockIdx.y * 8 + warp;
  if (j >= K) return;
  const float4* Aj = reinterpret_cast<const float4*>(A + (int64_t)j * ld);
  const float4* w1 = reinterpret_cast<const float4*>(v1);
  const float4* w2 = reinterpret_cast<const float4*>(v2);
  float s1 = 0.f, s2 = 0.f;
#pragma unroll 4
  for (int64_t q = q0 + lane; q < q1; q += 32) {
    const float4 a = Aj[q];
    const float4 x = w1[q];
    s1 = fmaf(a.x, x.x, fmaf(a.y, x.y, fmaf(a.z, x.z, fmaf(a.w, x.w, s1))));
    if (v2) {
      const float4 y = w2[q];
      s2 = fmaf(a.x, y.x, fmaf(a.y, y.y, fmaf(a.z, y.z, fmaf(a.w, y.w, s2))));
    }
  }
  const double d1 = warp_sum((double)s1);
  const double d2 = warp_sum((double)s2);
  if (lane == 0) {
    part[((int64_t)blockIdx.x * K + j) * 2] = d1;
    part[((int64_t)blockIdx.x * K + j) * 2 + 1] = d2;
  }
}

// Readers of the small matrices of the single-CTA kernels: S's upper triangle and the head
// block of a stack (rows below the diagonal), from global memory or packed in shared memory.
// Staged, each entry is read from global memory once, with coalesced loads, instead of once
// per product term.
struct SGlob {
  const double* p;
  int Tm;
  __device__ __forceinline__ double operator()(int i, int j) const { return p[i + (int64_t)j * Tm]; }
};
struct SUpper {   // column j's rows 0..j at j (j + 1) / 2
  const double* p;
  __device__ __forceinline__ double operator()(int i, int j) const { return p[j * (j + 1) / 2 + i]; }
};
template <typename T>
struct VGlob {
  const T* p;
  int64_t ld;
  __device__ __forceinline__ T operator()(int i, int j) const { return p[i + (int64_t)j * ld]; }
};
template <typename T>
struct VLower {   // column j's rows j..n-1 at j n - j (j - 1) / 2
  const T* p;
  int n;
  __device__ __forceinline__ T operator()(int i, int j) const { return p[j * n - j * (j - 1) / 2 + (i - j)]; }
};
__host__ __device__ __forceinline__ int64_t packed_tri(int n) { return (int64_t)n * (n + 1) / 2; }
// A[i, j] += f(i, j) over the entries of an n_i x n_j block (leading dim ld) with i <= j
// (upper) or j <= i (lower), the CTA's threads over the entries in column order.  The entries
// are distinct, so each thread issues four loads before its four stores instead of waiting for
// a store before every next load.
template <bool UPPER, typename E, typename F>
__device__ __forceinline__ void tri_add(E* A, int64_t ld, int ni, int nj, F f) {
  const int n = ni * nj, step = (int)blockDim.x;
  for (int q0 = threadIdx.x; q0 < n; q0 += 4 * step) {
    E v[4];
    int ii[4], jj[4];
    bool on[4];
#pragma unroll
    for (int u = 0; u < 4; u++) {
      const int q = q0 + u * step;
      ii[u] = q % ni;
      jj[u] = q / ni;
      on[u] = q < n && (UPPER ? ii[u] <= jj[u] : jj[u] <= ii[u]);
      if (on[u]) v[u] = A[ii[u] + (int64_t)jj[u] * ld];
    }
#pragma unroll
    for (int u = 0; u < 4; u++)
      if (on[u]) A[ii[u] + (int64_t)jj[u] * ld] = v[u] + (E)f(ii[u], jj[u]);
  }
}
// Copy the K x K upper triangle of S (leading dim Tm) to dst (SUpper order), a warp per column.
__device__ void stage_upper_sm(const double* __restrict__ S, int Tm, int K, double* dst) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = wid; j < K; j += nw)
    for (int i = lane; i <= j; i += 32) dst[j * (j + 1) / 2 + i] = S[i + (int64_t)j * Tm];
}
// Copy rows j..n-1 of columns j < n of V (leading dim ld) to dst (VLower order).
template <typename T>
__device__ void stage_lower_sm(const T* __restrict__ V, int64_t ld, int n, T* dst) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = wid; j < n; j += nw)
    for (int i = j + lane; i < n; i += 32) dst[j * n - j * (j - 1) / 2 + (i - j)] = V[i + (int64_t)j * ld];
}
// Dynamic shared memory of the staged single-CTA kernels: the packed upper triangle of a K x K
// block of S, then (when sizeof_v > 0) the packed lower triangle of the K x K head of a stack.
inline size_t staged_bytes(int K, int sizeof_v) {
  const size_t s = (size_t)packed_tri(K) * 8;
  return ((s + 15) & ~(size_t)15) + (size_t)packed_tri(K) * (size_t)sizeof_v;
}
constexpr size_t kStagedMax = 200 * 1024;   // larger blocks read S and V from global memory

// Adjoint of the S-column recurrence of column k of a stack: S[:k, k] = c = -tau S_k a with
// a = V_k^T u (recorded) and S[k, k] = tau = 2 / u^T u.  With cbar = Sbar[:k, k] and
// taubar = Sbar[k, k] + cbar . c / tau:  abar = -tau S_k^T cbar (a = V^T u passes it on as
// Vbar_k += u abar^T and ubar += V_k abar), Sbar_k += -tau cbar a^T (upper triangle), and
// tau = 2 / u^T u gives ubar += -tau^2 taubar u.  Writes coef[0..k) = abar, coef[k] =
// -tau^2 taubar (the coefficients of ubar += V[:, 0..k] coef).  An identity column (tau = 0)
// passes nothing.
template <typename SA>
__device__ void rec_col_dev(SA S, double* Sb, int Tm, int k, const double* __restrict__ a, double* coef) {
  __shared__ double cb[kTmaxLimit + 1];
  __shared__ double tb;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const double tau = S(k, k);
  for (int i = threadIdx.x; i < k; i += blockDim.x) cb[i] = (tau != 0.0) ? Sb[i + (int64_t)k * Tm] : 0.0;
  if (wid == 0) {
    double s = 0.0;
    for (int i = lane; i < k; i += 32) s = fma(Sb[i + (int64_t)k * Tm], S(i, k), s);
    s = warp_sum(s);
    if (lane == 0) tb = (tau != 0.0) ? Sb[k + (int64_t)k * Tm] + s / tau : 0.0;
  }
  __syncthreads();
  for (int j = wid; j < k; j += nw) {   // abar_j = -tau sum_{i <= j} S[i, j] cbar_i
    double s = 0.0;
    for (int i = lane; i <= j; i += 32) s = fma(S(i, j), cb[i], s);
    s = warp_sum(s);
    if (lane == 0) coef[j] = -tau * s;
  }
  if (threadIdx.x == 0) coef[k] = -tau * tau * tb;
  tri_add<true>(Sb, Tm, k, k, [&](int i, int j) { return -tau * cb[i] * a[j]; });
}
template <bool STAGED>
__global__ void __launch_bounds__(kSmallT) k_rec_col(TP<const double> S, TP<double> Sb, int Tm, int k,
                                                     TP<const double> a, TP<double> coef) {
  const int tr = blockIdx.z;
  if constexpr (STAGED) {
    extern __shared__ __align__(16) unsigned char adj_dsm[];
    double* Su = (double*)adj_dsm;
    stage_upper_sm(S.at(tr), Tm, k + 1, Su);
    __syncthreads();
    rec_col_dev(SUpper{Su}, Sb.at(tr), Tm, k, a.at(tr), coef.at(tr));
  } else {
    rec_col_dev(SGlob{S.at(tr), Tm}, Sb.at(tr), Tm, k, a.at(tr), coef.at(tr));
  }
}

// out = scale S v (trans = 0) or scale S^T v (trans = 1), leading K x K block of the upper
// triangular S (column-major, leading dim Tm): one warp per output, lanes over the sum.
template <typename SA>
__device__ void tri_dev(SA S, int K, const double* __restrict__ v, double scale, int trans, double* out) {
  const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int i = threadIdx.x >> 5; i < K; i += nw) {
    double s = 0.0;
    if (!trans) {
      for (int j = i + lane; j < K; j += 32) s = fma(S(i, j), v[j], s);
    } else {
      for (int q = lane; q <= i; q += 32) s = fma(S(q, i), v[q], s);
    }
    s = warp_sum(s);
    if (lane == 0) out[i] = scale * s;
  }
}
__global__ void __launch_bounds__(kSmallT) k_tri(TP<const double> S, int Tm, int K, TP<const double> v,
                                                 double scale, int trans, TP<double> out) {
  const int tr = blockIdx.z;
  tri_dev(SGlob{S.at(tr), Tm}, K, v.at(tr), scale, trans, out.at(tr));
}

// Sb[i, j] += a[i] b[j] on the upper triangle i <= j < K (S has no free entries below).
__device__ __forceinline__ void outer_upper_dev(double* Sb, int Tm, int K, const double* __restrict__ a,
                                                const double* __restrict__ b) {
  tri_add<true>(Sb, Tm, K, K, [&](int i, int j) { return a[i] * b[j]; });
}
__global__ void __launch_bounds__(kAT) k_outer_upper(TP<double> Sb, int Tm, int K, TP<const double> a,
                                                     TP<const double> b) {
  const int tr = blockIdx.z;
  outer_upper_dev(Sb.at(tr), Tm, K, a.at(tr), b.at(tr));
}

// c = [p_head[0:k]; alpha] from the step's record
__global__ void k_head_alpha(TP<const double> phead_, int k, TP<const double> rs_, TP<double> c_) {
  const int tr = blockIdx.z;
  const double* phead = phead_.at(tr);
  const double* rs = rs_.at(tr);
  double* c = c_.at(tr);
  for (int i = threadIdx.x; i <= k; i += blockDim.x) c[i] = (i < k) ? phead[i] : rs[1];
}

// Adjoint of the output product y = (I - V S V^T) Delta c for c supported on rows < nc <= Ke
// (Ke reflectors).  Given bb = -V^T ybar (from a column pass) and the head of ybar: writes
// b = S a (for Vbar += -ybar b^T, done by the caller), cbar = Delta (ybar + V S^T bb) on the
// first nc rows, and adds Sbar += bb a^T and Vbar[:nc, :] += (Delta c) (S^T bb)^T.  One warp
// per output, lanes over the sums.
template <typename T, typename VA, typename SA>
__device__ void out_small_dev(VA V, T* Vb, int64_t ld, int Ke, int nc, SA S, int Tm, const double* __restrict__ dpre,
                              const double* __restrict__ c, const double* __restrict__ bb,
                              const T* __restrict__ ybd, double* Sb, double* b_out, double* cbar) {
  __shared__ double cp[kTmaxLimit + 1], a[kTmaxLimit + 1], ab[kTmaxLimit + 1];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = threadIdx.x; i < nc; i += blockDim.x) cp[i] = dpre[i + 1] * c[i];
  __syncthreads();
  for (int j = wid; j < Ke; j += nw) {   // a = V^T Delta c (rows j..nc-1 of column j)
    double s = 0.0;
    for (int i = j + lane; i < nc; i += 32) s = fma((double)V(i, j), cp[i], s);
    s = warp_sum(s);
    if (lane == 0) a[j] = s;
  }
  __syncthreads();
  for (int i = wid; i < Ke; i += nw) {   // b = S a, abar = S^T bb
    double sb = 0.0, sa = 0.0;
    for (int j = i + lane; j < Ke; j += 32) sb = fma(S(i, j), a[j], sb);
    for (int q = lane; q <= i; q += 32) sa = fma(S(q, i), bb[q], sa);
    sb = warp_sum(sb);
    sa = warp_sum(sa);
    if (lane == 0) {
      b_out[i] = sb;
      ab[i] = sa;
    }
  }
  __syncthreads();
  tri_add<true>(Sb, Tm, Ke, Ke, [&](int i, int j) { return bb[i] * a[j]; });
  // Vbar[:nc, :] += (Delta c) abar^T on the stored (lower) part
  tri_add<false>(Vb, ld, nc, Ke, [&](int i, int j) { return cp[i] * ab[j]; });
  // cbar = Delta (ybar + V abar) on rows < nc: a row per thread
  for (int i = threadIdx.x; i < nc; i += blockDim.x) {
    const int jm = min(i, Ke - 1);
    double s0 = 0.0, s1 = 0.0;
    int j = 0;
    for (; j + 1 <= jm; j += 2) {
      s0 = fma((double)V(i, j), ab[j], s0);
      s1 = fma((double)V(i, j + 1), ab[j + 1], s1);
    }
    if (j <= jm) s0 = fma((double)V(i, j), ab[j], s0);
    cbar[i] = dpre[i + 1] * ((double)ybd[i] + (s0 + s1));
  }
}
template <typename T>
__global__ void __launch_bounds__(kSmallT) k_out_small(TP<const T> V, int64_t ld, int Ke, int nc,
                                                       TP<const double> S, int Tm, TP<const double> dpre,
                                                       TP<const double> c, TP<const double> bb, TP<const T> ybd,
                                                       TP<double> Sb, TP<T> Vb, TP<double> b_out, TP<double> cbar) {
  const int tr = blockIdx.z;
  out_small_dev<T>(VGlob<T>{V.at(tr), ld}, Vb.at(tr), ld, Ke, nc, SGlob{S.at(tr), Tm}, Tm, dpre.at(tr), c.at(tr),
                   bb.at(tr), ybd.at(tr), Sb.at(tr), b_out.at(tr), cbar.at(tr));
}

// Haar output side in one CTA: with bb = -V^T ybar (the column pass, reduced over its row blocks
// by k_colreduce), c = [p_head; alpha], the output-product adjoint (k_out_small) and the S
// recurrence of the step's random column (k_rec_col, after the Sbar update it depends on).
template <typename T, bool STAGED>
__global__ void __launch_bounds__(kSmallT) k_out_haar_adj(TP<const T> V_,
                                                          int64_t ld, int Ke, TP<const double> S_, int Tm,
                                                          TP<const double> dpre_, TP<const double> phead_,
                                                          TP<const double> rs_, TP<double> cv_, TP<double> bb_,
                                                          TP<const T> ybd_, TP<double> Sb_, TP<T> Vb_, TP<double> bo_,
                                                          TP<double> cbar_, TP<const double> rag_, TP<double> au_) {
  const int tr = blockIdx.z;
  const T* __restrict__ V = V_.at(tr);
  const double* __restrict__ S = S_.at(tr);
  const double* __restrict__ dpre = dpre_.at(tr);
  const double* __restrict__ phead = phead_.at(tr);
  const double* __restrict__ rs = rs_.at(tr);
  double* cv = cv_.at(tr);
  double* bb = bb_.at(tr);
  const T* __restrict__ ybd = ybd_.at(tr);
  double* Sb = Sb_.at(tr);
  T* Vb = Vb_.at(tr);
  double* bo = bo_.at(tr);
  double* cbar = cbar_.at(tr);
  const double* __restrict__ rag = rag_.at(tr);
  double* au = au_.at(tr);
  const int k = Ke - 1;
  for (int i = threadIdx.x; i <= k; i += blockDim.x) cv[i] = (i < k) ? phead[i] : rs[1];
  if constexpr (STAGED) {   // S's upper triangle and V's head block in shared memory
    extern __shared__ __align__(16) unsigned char adj_dsm[];
    double* Su = (double*)adj_dsm;
    T* Vl = (T*)(adj_dsm + ((packed_tri(Ke) * 8 + 15) & ~(int64_t)15));
    stage_upper_sm(S, Tm, Ke, Su);
    stage_lower_sm<T>(V, ld, Ke, Vl);
    __syncthreads();
    out_small_dev<T>(VLower<T>{Vl, Ke}, Vb, ld, Ke, Ke, SUpper{Su}, Tm, dpre, cv, bb, ybd, Sb, bo, cbar);
    __syncthreads();
    rec_col_dev(SUpper{Su}, Sb, Tm, k, rag, au);
  } else {
    __syncthreads();
    out_small_dev<T>(VGlob<T>{V, ld}, Vb, ld, Ke, Ke, SGlob{S, Tm}, Tm, dpre, cv, bb, ybd, Sb, bo, cbar);
    __syncthreads();
    rec_col_dev(SGlob{S, Tm}, Sb, Tm, k, rag, au);
  }
}

// The step's record (adj_record_after) in one launch: z (nz), w, p_head, V_D^T u (kD each),
// p's pivot entry and alpha, and (Haar) V_N^T u_g (nug).
__global__ void __launch_bounds__(kAT) k_adj_record(TP<double> r_, int64_t L, TP<const double> z_, int nz,
                                                    TP<const double> w_, TP<const double> ph_, int kD,
                                                    TP<const double> scal_, TP<const double> ua_,
                                                    TP<const double> ug_, int nug) {
  const int tr = blockIdx.z;
  double* r = r_.at(tr);
  const double* __restrict__ z = z_.at(tr);
  const double* __restrict__ w = w_.at(tr);
  const double* __restrict__ ph = ph_.at(tr);
  const double* __restrict__ scal = scal_.at(tr);
  const double* __restrict__ ua = ua_.at(tr);
  const double* __restrict__ ug = ug_.at(tr);
  for (int i = threadIdx.x; i < nz; i += blockDim.x) r[i] = z[i];
  for (int i = threadIdx.x; i < kD; i += blockDim.x) {
    r[L + i] = w[i];
    r[2 * L + i] = ph[i];
    r[3 * L + 8 + i] = ua[i];
  }
  if (threadIdx.x < 2) r[3 * L + threadIdx.x] = scal[threadIdx.x];
  for (int i = threadIdx.x; i < nug; i += blockDim.x) r[4 * L + 8 + i] = ug[i];
}

// Data side after the column pass of qbar in one CTA: with wbar = -V^T qbar (reduced by
// k_colreduce), zbar = S wbar, Sbar += z wbar^T.
template <bool STAGED>
__global__ void __launch_bounds__(kSmallT) k_data_small(int K, TP<const double> S_, int Tm, TP<const double> z_,
                                                        TP<const double> wb_, TP<double> zb_, TP<double> Sb_) {
  const int tr = blockIdx.z;
  const double* __restrict__ S = S_.at(tr);
  const double* __restrict__ z = z_.at(tr);
  const double* wb = wb_.at(tr);
  double* zb = zb_.at(tr);
  double* Sb = Sb_.at(tr);
  if constexpr (STAGED) {
    extern __shared__ __align__(16) unsigned char adj_dsm[];
    double* Su = (double*)adj_dsm;
    stage_upper_sm(S, Tm, K, Su);
    __syncthreads();
    tri_dev(SUpper{Su}, K, wb, 1.0, 0, zb);
  } else {
    tri_dev(SGlob{S, Tm}, K, wb, 1.0, 0, zb);
  }
  outer_upper_dev(Sb, Tm, K, z, wb);
}

// qbar = Delta_D pbar with pbar[r] = cb[r] (r < kD) and, on the tail, the adjoint of the new
// column u = p[kD:] + s alpha e_kD and of alpha: (cb[kD] + s ub[kD]) p[r] / alpha + ub[r].  The
// tail of p is read back from the stored column (p[r] = u[r] for r > kD, p[kD] recorded).
// rs = the step's record: rs[0] = p[kD], rs[1] = alpha.
template <typename T>
__global__ void __launch_bounds__(kAT) k_pbar(TP<T> qbar_, TP<const T> u_, TP<const T> ub_, TP<const double> cb_,
                                              TP<const double> rs_, int kD, TP<const double> dpre_, int64_t dim) {
  const int tr = blockIdx.z;
  T* __restrict__ qbar = qbar_.at(tr);
  const T* __restrict__ u = u_.at(tr);
  const T* __restrict__ ub = ub_.at(tr);
  const double* __restrict__ cb = cb_.at(tr);
  const double* __restrict__ rs = rs_.at(tr);
  const double* __restrict__ dpre = dpre_.at(tr);
  __shared__ T coef_s;
  const double ppiv = rs[0], alpha = rs[1];
  if (threadIdx.x == 0) {   // one FP64 division per CTA
    const double s = (ppiv >= 0.0) ? 1.0 : -1.0;
    coef_s = (alpha > 0.0) ? (T)((cb[kD] + s * (double)ub[kD]) / alpha) : T(0);
  }
  __syncthreads();
  const T coef = coef_s;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < dim; r += (int64_t)gridDim.x * blockDim.x) {
    T pb;
    if (r < kD) pb = (T)cb[r];
    else pb = (alpha > 0.0) ? fma(coef, (r == kD) ? (T)ppiv : u[r], ub[r]) : T(0);
    qbar[r] = (T)dpre[min(r + 1, (int64_t)kD)] * pb;
  }
}

// out[r] = sgn * (sigma g_r) for first <= r < dim (the step's draw, in the state's precision),
// 0 elsewhere; sgn = *sgnp.
template <typename T>
__global__ void __launch_bounds__(kAT) k_draw_d(DrawKey key, int64_t first, int64_t dim,
                                                const TrialDesc* __restrict__ desc, TP<const double> sgnp_, TP<T> out_) {
  const int tr = blockIdx.z;
  key.trial = desc[tr].trial;
  const T sigma = (T)desc[tr].sigma;
  T* out = out_.at(tr);
  const T sg = (T)*sgnp_.at(tr);
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < dim; r += (int64_t)gridDim.x * blockDim.x) {
    T v = T(0);
    if (r >= first) {
      T a, b;
      normal_pair(key, (uint64_t)(r >> 1), a, b);
      v = sg * (sigma * ((r & 1) ? b : a));
    }
    out[r] = v;
  }
}

// ------------------------------------------------------------------------------------
// Host side.  Every launch covers all trials of the state (grid z = trial); per-trial arrays
// are addressed through TP (pointer of trial 0, distance between trials).
struct Ctx {
  hd_state* st;
  cudaStream_t s;
  int nz;           // trials
};

template <typename P>
bool al16tp(const TP<P>& t) {
  return t.p == nullptr || (((uintptr_t)t.p & 15u) == 0 && ((t.s * (int64_t)sizeof(P)) & 15) == 0);
}

unsigned rows_grid(const hd_state* st, int64_t dim) {
  const int64_t want = (dim + kAT - 1) / kAT;
  const int64_t cap = std::max<int64_t>(1, (int64_t)st->nsm * 8 / std::max(1, st->count));
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(want, cap));
}

template <typename P>
TP<const P> cst(const TP<P>& t) { return TP<const P>{t.p, t.s}; }

// Column pass o_v = s_v A^T v_v; with o1 null only the partial sums are formed (a following
// single-CTA kernel reduces them).
template <typename T>
void colpass(const Ctx& c, TP<const T> A, int64_t ld, int K, int64_t dim, TP<const T> v1, double s1, TP<double> o1,
             TP<const T> v2 = TP<const T>{nullptr, 0}, double s2 = 0.0, TP<double> o2 = TP<double>{nullptr, 0}) {
  if (K <= 0) return;
  AdjState& A_ = *c.st->adj;
  const TP<double> part = tp(A_.part, A_.part_stride);
  if (sizeof(T) == 4 && dim % 4 == 0 && ld % 4 == 0 && al16tp(A) && al16tp(v1) && al16tp(v2))
    k_colpass4<<<dim3(A_.nblk, (K + 7) / 8, c.nz), kAT, 0, c.s>>>(
        TP<const float>{(const float*)A.p, A.s}, ld, K, dim / 4, TP<const float>{(const float*)v1.p, v1.s},
        TP<const float>{(const float*)v2.p, v2.s}, part);
  else
    k_colpass<T><<<dim3(A_.nblk, (K + 7) / 8, c.nz), kAT, 0, c.s>>>(A, ld, K, dim, v1, v2, part);
  if (o1.p)
    k_colreduce<<<dim3((K + kAT / 32 - 1) / (kAT / 32), 1, c.nz), kAT, 0, c.s>>>(cst(part), A_.nblk, K, s1, o1, s2, o2);
}

template <typename T>
void rowpass(const Ctx& c, TP<T> out, TP<const T> in, double s_in, TP<const T> A, int64_t ld, int K,
             TP<const double> coef, double cscale, int64_t dim, TP<const double> dpre, int Kd, int acc,
             int64_t rnorm = INT64_MAX, TP<double> npart = TP<double>{nullptr, 0}, unsigned grid = 0) {
  const unsigned g = grid ? grid : rows_grid(c.st, dim);
  if (sizeof(T) == 4 && !dpre.p && !npart.p && dim % 4 == 0 && ld % 4 == 0 && al16tp(out) && al16tp(in) &&
      al16tp(A)) {
    k_rowpass4<<<dim3(rows_grid(c.st, dim / 4), 1, c.nz), kAT, 0, c.s>>>(
        TP<float>{(float*)out.p, out.s}, TP<const float>{(const float*)in.p, in.s}, s_in,
        TP<const float>{(const float*)A.p, A.s}, ld, K, coef, cscale, dim / 4, acc);
    return;
  }
  k_rowpass<T><<<dim3(g, 1, c.nz), kAT, 0, c.s>>>(out, in, s_in, A, ld, K, coef, cscale, dim, dpre, Kd, acc, rnorm,
                                                  npart);
}

template <typename T>
void rankN(const Ctx& c, TP<T> Ab, int64_t ld, int K, int64_t dim, const RankTerms& t) {
  if (K <= 0 || t.n <= 0) return;
  bool al = sizeof(T) == 4 && dim % 4 == 0 && ld % 4 == 0 && al16tp(Ab);
  for (int q = 0; q < t.n; q++) al = al && al16tp(TP<const T>{(const T*)t.v[q], t.sv[q]});
  if (al) {
    dim3 g4(rows_grid(c.st, dim / 4), 1, c.nz);
    k_rankN4<<<g4, kAT, 0, c.s>>>(TP<float>{(float*)Ab.p, Ab.s}, ld, K, dim / 4, t);
    return;
  }
  dim3 g(rows_grid(c.st, dim), (unsigned)((K + 7) / 8), c.nz);
  k_rankN<T><<<g, kAT, 0, c.s>>>(Ab, ld, K, dim, t);
}

template <typename T>
void rank(const Ctx& c, TP<T> Ab, int64_t ld, int K, int64_t dim, TP<const T> a, TP<const double> b, double sb,
          TP<const T> cc = TP<const T>{nullptr, 0}, TP<const double> d = TP<const double>{nullptr, 0}, double sd = 0.0,
          TP<const T> e = TP<const T>{nullptr, 0}, TP<const double> f = TP<const double>{nullptr, 0}, double sf = 0.0,
          int Kf = 0) {
  if (K <= 0) return;
  if (sizeof(T) == 4 && dim % 4 == 0 && ld % 4 == 0 && al16tp(Ab) && al16tp(a) && al16tp(cc) && al16tp(e)) {
    dim3 g4(rows_grid(c.st, dim / 4), 1, c.nz);
    k_rank4<<<g4, kAT, 0, c.s>>>(TP<float>{(float*)Ab.p, Ab.s}, ld, K, dim / 4,
                                 TP<const float>{(const float*)a.p, a.s}, b, sb,
                                 TP<const float>{(const float*)cc.p, cc.s}, d, sd,
                                 TP<const float>{(const float*)e.p, e.s}, f, sf, Kf);
    return;
  }
  dim3 g(rows_grid(c.st, dim), (unsigned)((K + 7) / 8), c.nz);
  k_rank<T><<<g, kAT, 0, c.s>>>(Ab, ld, K, dim, a, b, sb, cc, d, sd, e, f, sf, Kf);
}

// Distances between consecutive trials of the state's own arrays (0 for a single trial).
struct Strides {
  int64_t V[2], S, dpre, B[2], ws;
};
Strides state_strides(const hd_state* st) {
  Strides r{};
  if (st->count < 2) return r;
  const TrialDesc& a = st->hdesc[0];
  const TrialDesc& b = st->hdesc[1];
  for (int s = 0; s < 2; s++) {
    r.V[s] = ((const char*)b.st[s].V - (const char*)a.st[s].V) / (int64_t)st->esz;
    r.B[s] = a.basis[s] ? ((const char*)b.basis[s] - (const char*)a.basis[s]) / (int64_t)st->esz : 0;
  }
  r.S = b.st[0].S - a.st[0].S;
  r.dpre = b.st[0].dpre - a.st[0].dpre;
  r.ws = b.ws.z - a.ws.z;
  return r;
}

template <typename T>
int adj_step(hd_state* st, const void* ybar, const void* x_in, void* xbar) {
  AdjState& A = *st->adj;
  const int t = A.rev;                 // 1-based forward step being reversed
  const int tr = A.flag[t - 1], kD = A.kD[t - 1], kN = A.kN[t - 1];
  const int d = tr ? 1 : 0, e = 1 - d;
  const TrialDesc& td = st->hdesc[0];
  const StackDev& Sd = td.st[d];
  const StackDev& Se = td.st[e];
  const int64_t nd = st->dims[d][0], ne = st->dims[e][0];
  const bool haar = st->ens == HD_HAAR;
  const Strides ss = state_strides(st);
  const TP<const T> Vd{(const T*)Sd.V, ss.V[d]};
  const TP<const T> Ve{(const T*)Se.V, ss.V[e]};
  const TP<T> Vbd{(T*)A.Vbar[d], A.vbar_stride[d]};
  const TP<T> Vbe{(T*)A.Vbar[e], A.vbar_stride[e]};
  const TP<const double> SdS{Sd.S, ss.S}, SeS{Se.S, ss.S};
  const TP<const double> Sdp{Sd.dpre, ss.dpre}, Sep{Se.dpre, ss.dpre};
  const TP<double> Sbd{A.Sbar[d], A.sbar_stride}, Sbe{A.Sbar[e], A.sbar_stride};
  const int Tm = st->Sld;   // leading dimension of S and Sbar
  const Ctx c{st, st->stream, st->count};
  const int64_t L = A.dmax;
  T* vec = (T*)A.vec;
  const int par = t & 1;   // the copy of qbar, zbar and E of this step's parity
  const TP<T> ub{vec + kVub * L, A.vec_stride};
  const TP<T> qb{vec + (par ? kVqb2 : kVqb) * L, A.vec_stride};
  const TP<T> gd{vec + kVg * L, A.vec_stride};
  // the step input: the caller's (packed) or the recorded one (slot t - 1, packed)
  const TP<const T> xd = x_in ? TP<const T>{(const T*)x_in, nd}
                              : TP<const T>{(const T*)((const char*)A.X + (size_t)(t - 1) * A.ldx * sizeof(T)), nd};
  const TP<const T> ybd{(const T*)ybar, ne};
  const TP<T> xb{(T*)xbar, nd};
  auto sm = [&](int slot) { return TP<double>{A.small + (int64_t)slot * A.small_ld, A.small_stride}; };
  const TP<double> bb = sm(kSbb), bo = sm(kSb), cb = sm(kScb), zb = sm(par ? kSzb2 : kSzb), wb = sm(kSwb),
                   E = sm(par ? kSE2 : kSE);
  const TP<double> cv = sm(kSc), hb = sm(kShb), au = sm(kSau), bu = sm(kSbu), bbu = sm(kSbbu), abu = sm(kSabu);
  const TP<double> part{A.part, A.part_stride};
  const unsigned gv = rows_grid(st, std::max(nd, ne));
  const TP<double> none{nullptr, 0};
  const TP<const double> cnone{nullptr, 0};
  const TP<const T> tnone{nullptr, 0};

  // forward quantities of step t, recorded after it: z = V_D^T x, (Gin) h = B_D^T x, w, p_head,
  // p's pivot entry and alpha; p's tail is the stored column u of V_D (minus s alpha at the pivot)
  const double* rz = A.rec + (int64_t)(t - 1) * A.rec_ld;
  const int64_t sr = A.rec_stride;
  const TP<const double> z{rz, sr};
  const TP<const double> h{rz + kD, sr};
  const TP<const double> w{rz + st->Sld, sr};
  const TP<const double> phead{rz + 2 * (int64_t)st->Sld, sr};
  const TP<const double> rs{rz + 3 * (int64_t)st->Sld, sr};
  const TP<const double> ra{rz + 3 * (int64_t)st->Sld + 8, sr};    // V_D^T u (new data column)
  const TP<const double> rag{rz + 4 * (int64_t)st->Sld + 8, sr};   // V_N^T u_g (Haar: new random column)
  const TP<const T> ucol{Vd.p + (int64_t)kD * Sd.ld, Vd.s};
  const unsigned gp = rows_grid(st, nd);

  // A data-side update held back by the previous call (the next-later step) joins this
  // step's output-side update when that covers the same stack and columns; otherwise it is
  // applied now, before anything here reads that stack's Vbar.
  AdjState::Pending& pd = A.pend;
  const bool join = haar && pd.on && pd.s == e && pd.K == kD + 1;
  auto pending_terms = [&](RankTerms& rt) {
    for (int q = 0; q < pd.n; q++) {
      rt.v[rt.n] = pd.v[q];
      rt.c[rt.n] = pd.c[q];
      rt.s[rt.n] = pd.sc[q];
      rt.K[rt.n] = pd.Kq[q];
      rt.sv[rt.n] = pd.sv[q];
      rt.sc[rt.n] = pd.scs[q];
      rt.n++;
    }
    pd.on = 0;
  };
  if (pd.on && !join) {
    RankTerms rt{};
    const int s0 = pd.s, K0 = pd.K;
    pending_terms(rt);
    rankN<T>(c, TP<T>{(T*)A.Vbar[s0], A.vbar_stride[s0]}, td.st[s0].ld, K0, st->dims[s0][0], rt);
  }
  // Haar: the data side (cd) runs on the second stream beside the output side (c).  It needs
  // the output side only for cbar (the event ev_mid); the two sides write different stacks'
  // Sbar and Vbar, different small slots, and the partial-sum buffer only after ev_mid.
  const bool two = haar && A.aux != nullptr;
  const Ctx cd = two ? Ctx{st, A.aux, c.nz} : c;
  if (two) {
    cudaEventRecord(A.ev_fork, c.s);
    cudaStreamWaitEvent(A.aux, A.ev_fork, 0);
  }

  // output product
  if (haar) {
    const int Ke = kD + 1;   // the other stack including this step's random reflector
    // bb = -V_N^T ybar, the output-product adjoint, and the S recurrence of this step's random
    // column (L_t = H_t(g_t), column kD of V_N)
    colpass<T>(c, Ve, Se.ld, Ke, ne, ybd, -1.0, bb);
    const size_t sb_out = staged_bytes(Ke, (int)sizeof(T));
    if (sb_out <= kStagedMax)
      k_out_haar_adj<T, true><<<dim3(1, 1, c.nz), kSmallT, sb_out, c.s>>>(Ve, Se.ld, Ke, SeS, Tm, Sep, phead, rs,
                                                                         cv, bb, ybd, Sbe, Vbe, bo, cb, rag, au);
    else
      k_out_haar_adj<T, false><<<dim3(1, 1, c.nz), kSmallT, 0, c.s>>>(Ve, Se.ld, Ke, SeS, Tm, Sep, phead, rs,
                                                                      cv, bb, ybd, Sbe, Vbe, bo, cb, rag, au);
    if (two) cudaEventRecord(A.ev_mid, c.s);   // cbar is ready
    RankTerms rt{};
    rt.v[0] = ybd.p; rt.c[0] = bo.p; rt.s[0] = -1.0; rt.K[0] = Ke; rt.sv[0] = ybd.s; rt.sc[0] = bo.s;
    rt.v[1] = Ve.p + (int64_t)kD * Se.ld; rt.c[1] = au.p; rt.s[1] = 1.0; rt.K[1] = Ke; rt.sv[1] = Ve.s;
    rt.sc[1] = au.s;
    rt.n = 2;
    if (join) pending_terms(rt);
    rankN<T>(c, Vbe, Se.ld, Ke, ne, rt);
  } else {
    if (kN > 0) {
      colpass<T>(c, Ve, Se.ld, kN, ne, ybd, -1.0, bb);
      k_out_small<T><<<dim3(1, 1, c.nz), kSmallT, 0, c.s>>>(Ve, Se.ld, kN, kN, SeS, Tm, Sep, h, cst(bb), ybd, Sbe,
                                                            Vbe, bo, hb);
      rank<T>(c, Vbe, Se.ld, kN, ne, ybd, cst(bo), -1.0);
    }
    const TP<const T> Be{(const T*)td.basis[e], ss.B[e]};
    const int64_t lde = td.ldb[e];
    const TP<T> Bbe{(T*)A.Bbar[e], A.bbar_stride[e]};
    colpass<T>(c, Be, lde, kD + 1, ne, ybd, 1.0, cb);         // [pbar_head; alphabar]
    k_head_alpha<<<dim3(1, 1, c.nz), kAT, 0, c.s>>>(phead, kD, rs, cv);   // [p_head; alpha]
    rank<T>(c, Bbe, lde, kD + 1, ne, ybd, cst(cv), 1.0);
    if (kN > 0) {
      // the basis column built at this step, u = (I - V_N S_N V_N^T) Delta_N g: its adjoint
      // is complete; g is constant
      const TP<const T> ubar_b{(const T*)Bbe.p + (int64_t)kD * lde, Bbe.s};
      DrawKey key = key_for(st, t);
      k_draw_d<T><<<dim3(gv, 1, c.nz), kAT, 0, c.s>>>(key, kN, ne, st->ddesc, TP<const double>{Sep.p + kN, Sep.s},
                                                       gd);
      colpass<T>(c, Ve, Se.ld, kN, ne, ubar_b, -1.0, bbu, cst(gd), 1.0, au);
      k_tri<<<dim3(1, 1, c.nz), kSmallT, 0, c.s>>>(SeS, Tm, kN, cst(au), 1.0, 0, bu);
      k_tri<<<dim3(1, 1, c.nz), kSmallT, 0, c.s>>>(SeS, Tm, kN, cst(bbu), 1.0, 1, abu);
      k_outer_upper<<<dim3(1, 1, c.nz), kAT, 0, c.s>>>(Sbe, Tm, kN, cst(bbu), cst(au));
      rank<T>(c, Vbe, Se.ld, kN, ne, ubar_b, cst(bu), -1.0, cst(gd), cst(abu), 1.0);
    }
  }

  // the data-side reflector of this step (column kD of V_D): ubar = Vbar[:, kD] + the S
  // recurrence's V[:, 0..kD] coef (E = [abar; -tau^2 taubar])
  const size_t sb_rec = staged_bytes(kD + 1, 0);
  if (sb_rec <= kStagedMax)
    k_rec_col<true><<<dim3(1, 1, cd.nz), kSmallT, sb_rec, cd.s>>>(SdS, Sbd, Tm, kD, ra, E);
  else
    k_rec_col<false><<<dim3(1, 1, cd.nz), kSmallT, 0, cd.s>>>(SdS, Sbd, Tm, kD, ra, E);
  rowpass<T>(cd, ub, TP<const T>{(const T*)Vbd.p + (int64_t)kD * Sd.ld, Vbd.s}, 1.0, Vd, Sd.ld, kD + 1, cst(E), 1.0,
             nd, cnone, 0, 0);
  if (two) cudaStreamWaitEvent(cd.s, A.ev_mid, 0);   // k_pbar reads cbar
  k_pbar<T><<<dim3(gp, 1, cd.nz), kAT, 0, cd.s>>>(qb, ucol, cst(ub), cst(cb), rs, kD, Sdp, nd);

  // the data product p = Delta (I - V S^T V^T) x
  if (kD > 0) {   // wbar = -V_D^T qbar, zbar = S wbar, Sbar += z wbar^T
    colpass<T>(cd, Vd, Sd.ld, kD, nd, cst(qb), -1.0, wb);
    const size_t sb_dat = staged_bytes(kD, 0);
    if (sb_dat <= kStagedMax)
      k_data_small<true><<<dim3(1, 1, cd.nz), kSmallT, sb_dat, cd.s>>>(kD, SdS, Tm, z, cst(wb), zb, Sbd);
    else
      k_data_small<false><<<dim3(1, 1, cd.nz), kSmallT, 0, cd.s>>>(kD, SdS, Tm, z, cst(wb), zb, Sbd);
  }
  rowpass<T>(cd, xb, cst(qb), 1.0, Vd, Sd.ld, kD, cst(zb), 1.0, nd, cnone, 0, 0);
  if (!haar && kN > 0) {
    const TP<const T> Bd{(const T*)td.basis[d], ss.B[d]};
    rowpass<T>(cd, xb, tnone, 0.0, Bd, td.ldb[d], kN, cst(hb), 1.0, nd, cnone, 0, 1);
    rank<T>(cd, TP<T>{(T*)A.Bbar[d], A.bbar_stride[d]}, td.ldb[d], kN, nd, xd, cst(hb), 1.0);
  }
  // Vbar_D += -qbar w^T + x zbar^T + u abar^T.  Haar with the recorded x_t and the next reverse
  // step on the other product: held back for that step's output-side pass over this stack
  // (qbar, w, x, zbar, u, abar stay in place until then).
  if (haar && !x_in && t > 1 && A.flag[t - 2] != A.flag[t - 1] && kD > 0) {
    pd.on = 1;
    pd.s = d;
    pd.K = kD;
    pd.n = 3;
    pd.v[0] = qb.p; pd.c[0] = w.p; pd.sc[0] = -1.0; pd.Kq[0] = kD; pd.sv[0] = qb.s; pd.scs[0] = w.s;
    pd.v[1] = xd.p; pd.c[1] = zb.p; pd.sc[1] = 1.0; pd.Kq[1] = kD; pd.sv[1] = xd.s; pd.scs[1] = zb.s;
    pd.v[2] = ucol.p; pd.c[2] = E.p; pd.sc[2] = 1.0; pd.Kq[2] = kD; pd.sv[2] = ucol.s; pd.scs[2] = E.s;
  } else {
    rank<T>(cd, Vbd, Sd.ld, kD, nd, cst(qb), w, -1.0, xd, cst(zb), 1.0, ucol, cst(E), 1.0, kD);   // + u abar^T
  }
  if (two) {   // join: the caller's stream waits for the data side
    cudaEventRecord(A.ev_join, cd.s);
    cudaStreamWaitEvent(c.s, A.ev_join, 0);
  }
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return cuda_fail(st, err);
  A.rev -= 1;
  return HD_OK;
}

int adj_zero(hd_state* st) {
  AdjState& A = *st->adj;
  A.pend.on = 0;
  const int nt = st->count;
  for (int s = 0; s < 2; s++) {
    if (cudaMemsetAsync(A.Vbar[s], 0, (size_t)A.vbar_stride[s] * nt * st->esz, st->stream) != cudaSuccess ||
        cudaMemsetAsync(A.Sbar[s], 0, (size_t)A.sbar_stride * nt * sizeof(double), st->stream) != cudaSuccess)
      return cuda_fail(st, cudaGetLastError());
    if (A.Bbar[s] && cudaMemsetAsync(A.Bbar[s], 0, (size_t)A.bbar_stride[s] * nt * st->esz, st->stream) != cudaSuccess)
      return cuda_fail(st, cudaGetLastError());
  }
  return HD_OK;
}

}  // namespace

// Called by the forward step when reverse mode is on: record the step and its input (the
// packed vector of all trials).
int adj_record_step(hd_state* st, const void* x, int transpose, int kD, int kN) {
  AdjState& A = *st->adj;
  if (A.rev != st->t) return HD_ERR_STATE;   // a reverse pass has started: no more forward steps
  A.flag.push_back((int8_t)(transpose ? 1 : 0));
  A.kD.push_back(kD);
  A.kN.push_back(kN);
  if (A.record_x) {
    const int64_t nin = st->off[transpose ? 1 : 0][st->count];
    cudaError_t e = cudaMemcpyAsync((char*)A.X + (size_t)st->t * A.ldx * st->esz, x, (size_t)nin * st->esz,
                                    cudaMemcpyDeviceToDevice, st->stream);
    if (e != cudaSuccess) return cuda_fail(st, e);
  }
  A.rev = st->t + 1;
  return HD_OK;
}

// Called by the forward step after its launches: copy the step's small vectors from each
// trial's workspace (they are overwritten by the next step).
int adj_record_after(hd_state* st, int kD, int kN) {
  AdjState& A = *st->adj;
  const Ws& ws = st->hdesc[0].ws;
  const int64_t sw = state_strides(st).ws;
  double* r = A.rec + (int64_t)(st->t) * A.rec_ld;   // st->t is still this step's index
  const int nz = (st->ens == HD_GINIBRE) ? kD + kN : kD;   // Haar's K1 forms no basis dots
  const int nug = (st->ens == HD_HAAR) ? kN : 0;            // V_N^T u_g of the new random column
  k_adj_record<<<dim3(1, 1, st->count), kAT, 0, st->stream>>>(
      TP<double>{r, A.rec_stride}, st->Sld, TP<const double>{ws.z, sw}, nz, TP<const double>{ws.w, sw},
      TP<const double>{ws.phead, sw}, kD, TP<const double>{ws.scal, sw},
      TP<const double>{ws.scrb + ws.scr_stride * 1, sw}, TP<const double>{ws.scrb + ws.scr_stride * 2, sw}, nug);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(st, e);
  return HD_OK;
}

// Called by hd_reset: forget the recorded steps and clear the accumulators.
int adj_on_reset(hd_state* st) {
  if (!st->adj || !st->adj->on) return HD_OK;
  AdjState& A = *st->adj;
  A.flag.clear();
  A.kD.clear();
  A.kN.clear();
  A.rev = 0;
  return adj_zero(st);
}

}  // namespace hd

using namespace hd;

HD_API int hd_adjoint_enable(hd_state* st, int flags) {
  if (!st) return HD_ERR_ARG;
  if (st->poisoned) return st->poisoned;
  if (st->t != 0) return HD_ERR_STATE;
  if (flags & ~(HD_ADJ_RECORD_X)) return HD_ERR_ARG;
  // a batch must have trials of one shape (every per-trial array then evenly spaced)
  for (int i = 1; i < st->count; i++)
    if (st->dims[0][i] != st->dims[0][0] || st->dims[1][i] != st->dims[1][0]) return HD_ERR_ARG;
  if (cudaSetDevice(st->device) != cudaSuccess) return cuda_fail(st, cudaErrorInvalidDevice);
  {   // the staged single-CTA kernels take up to kStagedMax bytes of dynamic shared memory
    const int b = (int)kStagedMax;
    cudaError_t e = cudaFuncSetAttribute(k_out_haar_adj<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_out_haar_adj<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_rec_col<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_data_small<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    if (e != cudaSuccess) return cuda_fail(st, e);
  }
  const int nt = st->count;
  if (!st->adj) {
    AdjState* A = new (std::nothrow) AdjState();
    if (!A) return HD_ERR_OOM;
    st->adj = A;
    const TrialDesc& td = st->hdesc[0];
    const int Tm = st->Tm;
    A->sbar_stride = (int64_t)st->Sld * st->Sld;
    for (int s = 0; s < 2; s++) {
      A->vbar_stride[s] = td.st[s].ld * Tm;
      A->Vbar[s] = dalloc(st, (size_t)A->vbar_stride[s] * nt * st->esz);
      A->Sbar[s] = (double*)dalloc(st, (size_t)A->sbar_stride * nt * sizeof(double));
      if (!A->Vbar[s] || !A->Sbar[s]) return HD_ERR_OOM;
      if (st->ens == HD_GINIBRE) {
        A->bbar_stride[s] = td.ldb[s] * Tm;
        A->Bbar[s] = dalloc(st, (size_t)A->bbar_stride[s] * nt * st->esz);
        if (!A->Bbar[s]) return HD_ERR_OOM;
      }
    }
    A->dmax = round_up(std::max(st->dims[0][0], st->dims[1][0]), 256);
    A->ldx = round_up(std::max(st->off[0][nt], st->off[1][nt]), 256);   // one packed input per step
    A->vec_stride = (int64_t)kAdjVecs * A->dmax;
    A->vec = dalloc(st, (size_t)A->vec_stride * nt * st->esz);
    A->small_ld = Tm + 8;
    A->small_stride = (int64_t)kAdjSmall * A->small_ld;
    A->small = (double*)dalloc(st, (size_t)A->small_stride * nt * sizeof(double));
    // row chunks of a column pass per trial: about two CTAs per SM over the whole batch
    A->nblk = std::max(4, 2 * st->nsm / nt);
    const int64_t gmax = (int64_t)st->nsm * 8;
    A->part_stride = std::max<int64_t>((int64_t)A->nblk * (Tm + 1) * 2, gmax);
    A->part = (double*)dalloc(st, (size_t)A->part_stride * nt * sizeof(double));
    A->rec_ld = 5 * (int64_t)st->Sld + 8;
    A->rec_stride = A->rec_ld * Tm;
    A->rec = (double*)dalloc(st, (size_t)A->rec_stride * nt * sizeof(double));
    if (!A->vec || !A->small || !A->part || !A->rec) return HD_ERR_OOM;
  }
  AdjState& A = *st->adj;
  if (!A.aux && st->ens == HD_HAAR) {   // the data side's stream (Haar reverse steps)
    if (cudaStreamCreateWithFlags(&A.aux, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&A.ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&A.ev_mid, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&A.ev_join, cudaEventDisableTiming) != cudaSuccess)
      return cuda_fail(st, cudaGetLastError());
  }
  A.record_x = (flags & HD_ADJ_RECORD_X) ? 1 : 0;
  if (A.record_x && !A.X) {
    A.X = dalloc(st, (size_t)A.ldx * st->Tm * st->esz);
    if (!A.X) return HD_ERR_OOM;
  }
  A.on = 1;
  A.flag.clear();
  A.kD.clear();
  A.kN.clear();
  A.rev = 0;
  return adj_zero(st);
}

HD_API int hd_adjoint_step(hd_state* st, const void* ybar, const void* x_t, void* xbar) {
  if (!st || !ybar || !xbar) return HD_ERR_ARG;
  if (st->poisoned) return st->poisoned;
  if (!st->adj || !st->adj->on) return HD_ERR_STATE;
  AdjState& A = *st->adj;
  if (A.rev < 1) return HD_ERR_STATE;
  if (!x_t && !A.record_x) return HD_ERR_ARG;
  if (cudaSetDevice(st->device) != cudaSuccess) return cuda_fail(st, cudaErrorInvalidDevice);
  return st->dtype == HD_F64 ? adj_step<double>(st, ybar, x_t, xbar) : adj_step<float>(st, ybar, x_t, xbar);
}

HD_API int hd_adjoint_restart(hd_state* st) {
  if (!st) return HD_ERR_ARG;
  if (st->poisoned) return st->poisoned;
  if (!st->adj || !st->adj->on) return HD_ERR_STATE;
  if (cudaSetDevice(st->device) != cudaSuccess) return cuda_fail(st, cudaErrorInvalidDevice);
  st->adj->rev = st->t;
  return adj_zero(st);
}

HD_API int hd_adjoint_position(const hd_state* st, int32_t* remaining) {
  if (!st || !remaining) return HD_ERR_ARG;
  *remaining = (st->adj && st->adj->on) ? st->adj->rev : 0;
  return HD_OK;
}
