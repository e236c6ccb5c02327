// Householder Dice on the unitary group: y_t = M_t x_t for Q ~ Haar(U(n)), M_t in {Q, Q^H}
// (the paper's section "Other Random Matrix Ensembles": the construction carries over to
// complex matrices with M^T replaced by M^H, and the complex reflector of eq. Householder_c).
//
// The complex reflector of v in C^m with v_1 / ||v|| = r e^{i theta} (theta = 0 when v_1 = 0):
//     H(v) = -e^{-i theta} [I - w w^H / (1 + r)],   w = v / ||v|| + e^{i theta} e_1,
// unitary with H(v) v = ||v|| e_1.  With u = ||v|| w = v + ||v|| e^{i theta} e_1 this is
// H = c P,  P = I - tau u u^H,  tau = 1 / (||v|| (||v|| + |v_1|)),  c = -e^{-i theta},
// a Hermitian P times a unit scalar c on the reflector's coordinates.  As in the real case
// (where c = -sign(v_1)) the scalars of later reflectors commute past earlier P's, so for a
// stack of k generalised reflectors H_j = D_j P_j (pivot j, D_j = diag(I_j, c_j I)):
//     H_{k-1} ... H_0       = Delta_k (I - V S^H V^H)      (forward: the data-side product)
//     H_0^H ... H_{k-1}^H   = (I - V S V^H) Delta_k^H      (the output-side product)
// with V = [u_0 .. u_{k-1}] (column j zero above row j), S upper triangular (compact WY,
// S[j][j] = tau_j, S[:j, j] = -tau_j S[:j, :j] (V[:, :j]^H u_j)) and the phase diagonal
// Delta_k[i] = dpre[min(i, k - 1) + 1], dpre[q] = c_0 ... c_{q-1}.
//
// One step with data-side stack D (R for Q, L for Q^H) and the other stack N, both holding k
// reflectors before the step (pivot k of the new ones):
//   colpass(D, x)       z = V_D^H x                        colpass(N, draw)  V_N^H g, ||g||,
//                                                                            g -> column k of N
//   fin1                w = S_D^H z; the random reflector L_t = H_k(g): pivot, tau, phase, S_N
//   rowpass(D)          p = Delta_D (x - V_D w)  (= R_{t-1} ... R_1 x)
//   colpass(D, p)       V_D^H p[k:], ||p[k:]||, p[k:] -> column k of D
//   fin2                R_t = H_k(p): pivot, tau, phase, S_D; the output coefficients
//                       d = Delta_N^H [p_head; alpha; 0] (R_t p = [p_head; alpha; 0]) and
//                       w' = S_N V_N^H d over the head rows
//   rowpass(N)          y = d - V_N w'
// Streaming passes are in the storage type (complex FP32 or FP64); every cross-thread sum,
// S, the phases and the small coefficient vectors are FP64.  Draws: entry i of g_t is
// (N_{2i} + i N_{2i+1}) / sqrt(2), N the normals of step t's Philox stream.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include <cuda_runtime.h>

#include "hd.h"
#include "hd_common.cuh"

namespace hd {
void set_error(const char* where, cudaError_t e);
void record_error_text(const char* msg);
}  // namespace hd

using hd::DrawKey;

namespace {

constexpr int kCThreads = 256;
constexpr int kCRows = 1024;            // rows of a stack per CTA in the streaming passes
constexpr int kCTmax = 256;             // reflectors per stack (S is kCTmax^2 in FP64)

template <typename T>
struct __align__(2 * sizeof(T)) Cx {
  T re, im;
};

struct Cd {
  double re, im;
};

__device__ __forceinline__ Cd cmul(Cd a, Cd b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__device__ __forceinline__ Cd cconj(Cd a) { return {a.re, -a.im}; }
__device__ __forceinline__ Cd cadd(Cd a, Cd b) { return {a.re + b.re, a.im + b.im}; }
__device__ __forceinline__ Cd cscale(Cd a, double s) { return {a.re * s, a.im * s}; }
__device__ __forceinline__ double cabs(Cd a) { return hypot(a.re, a.im); }

template <typename T>
__device__ __forceinline__ Cd to_cd(Cx<T> a) { return {(double)a.re, (double)a.im}; }
template <typename T>
__device__ __forceinline__ Cx<T> from_cd(Cd a) { return {(T)a.re, (T)a.im}; }

// acc += conj(a) * b in T
template <typename T>
__device__ __forceinline__ void cdotacc(Cx<T>& acc, Cx<T> a, Cx<T> b) {
  acc.re = fma(a.re, b.re, fma(a.im, b.im, acc.re));
  acc.im = fma(a.re, b.im, fma(-a.im, b.re, acc.im));
}
// acc -= a * b in T
template <typename T>
__device__ __forceinline__ void cfms(Cx<T>& acc, Cx<T> a, Cx<T> b) {
  acc.re = fma(-a.re, b.re, fma(a.im, b.im, acc.re));
  acc.im = fma(-a.re, b.im, fma(-a.im, b.re, acc.im));
}

// Device state of one stack.
struct CStack {
  void* V;          // Cx<T>, column-major, ld x Tm
  int64_t ld;
  Cd* S;            // Tm x Tm (S[i + j Tm]), upper triangular, diagonal tau
  Cd* dpre;         // Tm + 1 prefix phases, dpre[0] = 1
};

// Workspace of the passes and finalisations (FP64).
struct CWs {
  Cd* part;         // per-CTA partial sums: [cta][Tm + 1] (dots, then the squared norm in .re)
  Cd* z;            // Tm + 1: summed dots
  Cd* w;            // Tm + 1: row-pass coefficients of the data side
  Cd* wout;         // Tm + 1: row-pass coefficients of the output
  Cd* d;            // Tm + 1: the output's head entries
  Cd* s2;           // Tm + 1: summed dots of the random side
  Cd* wg;           // Tm + 1: (Ginibre) coefficients of the new basis vector's row pass
  Cd* c;            // Tm + 1: (Ginibre) coefficients of the stored basis vectors in y
  Cd* h;            // Tm + 1: (Ginibre) dots of x with the data space's stored basis vectors
  void* p;          // Cx<T>, n: p = R_{t-1} ... R_1 x (the data-side product)
};

template <typename T>
__device__ __forceinline__ Cx<T> draw_c(const DrawKey& key, int64_t i) {
  T a, b;
  hd::normal_pair(key, (uint64_t)i, a, b);
  const T s = (T)0.70710678118654752440;
  return {a * s, b * s};
}

// Column pass over rows [blockIdx.x * kCRows, +kCRows): per CTA the partial sums of
// conj(c_j) . r for the k1 columns of the stack st (column j is zero above row j) and then the
// k2 dense columns of B, and of |r|^2 (slot k1 + k2); r is restricted to rows >= lo and is the
// vector src (mode 0) or sigma times the draw of `key` (mode 1).  When wcol is non-null, r
// (rows >= lo) is also stored there (a new stack or basis column; a stack column's pivot entry
// is replaced by the finalisation).
template <typename T>
__global__ void __launch_bounds__(kCThreads) k_c_colpass(CStack st, int k1, const void* B, int64_t ldb, int k2,
                                                         int64_t dim, int mode, const void* src, DrawKey key,
                                                         T sigma, int64_t lo, void* wcol, Cd* part, int P) {
  extern __shared__ __align__(16) unsigned char c_smem[];
  Cx<T>* r = (Cx<T>*)c_smem;
  __shared__ double red[kCThreads / 32];
  const int64_t r0 = (int64_t)blockIdx.x * kCRows;
  const int rows = (int)min((int64_t)kCRows, dim - r0);
  Cx<T>* wc = (Cx<T>*)wcol;
  T nrm = T(0);
  for (int q = threadIdx.x; q < kCRows; q += blockDim.x) {
    const int64_t i = r0 + q;
    Cx<T> v = {T(0), T(0)};
    if (q < rows && i >= lo) {
      if (mode == 0) {
        v = ((const Cx<T>*)src)[i];
      } else {
        v = draw_c<T>(key, i);
        v = {sigma * v.re, sigma * v.im};
      }
      if (wc) wc[i] = v;
      nrm = fma(v.re, v.re, fma(v.im, v.im, nrm));
    }
    r[q] = v;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = warp; j < k1 + k2; j += nw) {
    // a stack column is zero above its pivot row j; basis columns are dense
    const int64_t first = (j < k1) ? max((int64_t)j, lo) : lo;
    const int q0 = (int)max((int64_t)0, first - r0);
    const Cx<T>* col = (j < k1) ? (const Cx<T>*)st.V + (int64_t)j * st.ld + r0
                                : (const Cx<T>*)B + (int64_t)(j - k1) * ldb + r0;
    // four independent accumulators: the dependent FMA latency (long in FP64) is hidden
    Cx<T> a0 = {T(0), T(0)}, a1 = a0, a2 = a0, a3 = a0;
    int q = q0 + lane;
    for (; q + 96 < rows; q += 128) {
      cdotacc(a0, col[q], r[q]);
      cdotacc(a1, col[q + 32], r[q + 32]);
      cdotacc(a2, col[q + 64], r[q + 64]);
      cdotacc(a3, col[q + 96], r[q + 96]);
    }
    for (; q < rows; q += 32) cdotacc(a0, col[q], r[q]);
    double ar = ((double)a0.re + (double)a1.re) + ((double)a2.re + (double)a3.re);
    double ai = ((double)a0.im + (double)a1.im) + ((double)a2.im + (double)a3.im);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      ar += __shfl_xor_sync(0xffffffffu, ar, o);
      ai += __shfl_xor_sync(0xffffffffu, ai, o);
    }
    if (lane == 0) part[(int64_t)blockIdx.x * P + j] = {ar, ai};
  }
  double nd = (double)nrm;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) nd += __shfl_xor_sync(0xffffffffu, nd, o);
  if (lane == 0) red[warp] = nd;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < nw; w++) s += red[w];
    part[(int64_t)blockIdx.x * P + k1 + k2] = {s, 0.0};
  }
}

// Row pass: out[i] = ph_i (a_i - sum_{j < nc} V[i, j] coef[j]) over rows [blockIdx.x * kCRows,
// +kCRows); a_i = src[i] (src non-null) or head[i] for i < nhead (else 0); the phase ph_i is
// dpre[min(i, nc - 1) + 1] when phase_fwd (the data side), else 1.
template <typename T>
__global__ void __launch_bounds__(kCThreads) k_c_rowpass(CStack st, int nc, int64_t dim, const void* src, const Cd* head,
                                                         int nhead, const Cd* coef, int phase_fwd, void* out) {
  __shared__ Cx<T> cf[kCTmax + 1];
  for (int j = threadIdx.x; j < nc; j += blockDim.x) cf[j] = from_cd<T>(coef[j]);
  __syncthreads();
  const Cx<T>* V = (const Cx<T>*)st.V;
  const int64_t r0 = (int64_t)blockIdx.x * kCRows;
  constexpr int R = kCRows / kCThreads;   // rows per thread, interleaved for independent chains
  Cx<T> acc[R];
  int64_t row[R];
#pragma unroll
  for (int m = 0; m < R; m++) {
    row[m] = r0 + threadIdx.x + (int64_t)m * kCThreads;
    const int64_t i = row[m];
    if (i < dim && src) acc[m] = ((const Cx<T>*)src)[i];
    else acc[m] = (i < nhead) ? from_cd<T>(head[i]) : Cx<T>{T(0), T(0)};
  }
  // V[i, j] = 0 for j > i: rows below nc see every column; the few head rows mask the rest
  for (int j = 0; j < nc; j++) {
    const Cx<T> c = cf[j];
    const Cx<T>* col = V + (int64_t)j * st.ld;
#pragma unroll
    for (int m = 0; m < R; m++)
      if (row[m] < dim && row[m] >= j) cfms(acc[m], col[row[m]], c);
  }
#pragma unroll
  for (int m = 0; m < R; m++) {
    const int64_t i = row[m];
    if (i >= dim) continue;
    Cx<T> a = acc[m];
    if (phase_fwd && nc > 0) {
      const Cx<T> ph = from_cd<T>(st.dpre[min(i, (int64_t)nc - 1) + 1]);
      a = {ph.re * a.re - ph.im * a.im, ph.re * a.im + ph.im * a.re};
    }
    ((Cx<T>*)out)[i] = a;
  }
}

// Sum of the per-CTA partials (fixed order) into out[0..P).  Every thread of the CTA calls it.
__device__ void c_sum_parts(const Cd* part, int ncta, int P, Cd* out) {
  for (int j = threadIdx.x; j < P; j += blockDim.x) {
    double re = 0.0, im = 0.0;
    for (int c = 0; c < ncta; c++) {
      re += part[(int64_t)c * P + j].re;
      im += part[(int64_t)c * P + j].im;
    }
    out[j] = {re, im};
  }
  __syncthreads();
}

// Append the reflector H_k(v) to a stack whose column k holds v[k:] (v's pivot at row k):
// given s = V[:, :k]^H v[k:] (sums, k values) and ||v[k:]||^2, set the pivot entry, tau, the
// phase and S's column k.  Returns nothing; alpha_out receives ||v[k:]||.  Single thread
// block; uses scratch tmp (k values).
template <typename T>
__device__ void c_append(CStack st, int k, int Tm, const Cd* s, double nrm2, Cd* tmp, double* alpha_out) {
  __shared__ Cd s_e;
  __shared__ double s_tau, s_alpha;
  Cx<T>* V = (Cx<T>*)st.V;
  if (threadIdx.x == 0) {
    const double alpha = sqrt(nrm2);
    const Cd vk = to_cd(V[k + (int64_t)k * st.ld]);
    const double avk = cabs(vk);
    Cd e = {1.0, 0.0};
    if (avk > 0.0) e = {vk.re / avk, vk.im / avk};
    s_e = e;
    s_alpha = alpha;
    if (alpha > 0.0) {
      s_tau = 1.0 / (alpha * (alpha + avk));
      V[k + (int64_t)k * st.ld] = from_cd<T>(cadd(vk, cscale(e, alpha)));
      st.dpre[k + 1] = cmul(st.dpre[k], Cd{-e.re, e.im});   // c = -e^{-i theta} = -conj(e)
    } else {
      s_tau = 0.0;                                          // H_k = I (zero tail)
      st.dpre[k + 1] = st.dpre[k];
    }
    *alpha_out = alpha;
  }
  __syncthreads();
  const double tau = s_tau;
  // V[:, :k]^H u with u = v[k:] + alpha e e_k: the pivot adds alpha e conj(V[k, j])
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    const Cd vkj = to_cd(V[k + (int64_t)j * st.ld]);
    tmp[j] = cadd(s[j], cmul(cconj(vkj), cscale(s_e, s_alpha)));
  }
  __syncthreads();
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    Cd acc = {0.0, 0.0};
    for (int j = i; j < k; j++) acc = cadd(acc, cmul(st.S[i + (int64_t)j * Tm], tmp[j]));
    st.S[i + (int64_t)k * Tm] = cscale(acc, -tau);
  }
  if (threadIdx.x == 0) st.S[k + (int64_t)k * Tm] = {tau, 0.0};
  __syncthreads();
}

// fin1: z = V_D^H x summed, w = S_D^H z; the random reflector of the other stack.
template <typename T>
__global__ void __launch_bounds__(kCThreads) k_c_fin1(CStack D, CStack N, int k, int Tm, CWs ws, int ncta, int P) {
  __shared__ double nrm2;
  // partials: D's in part[0 .. ncta), N's in part[ncta .. 2 ncta)
  c_sum_parts(ws.part, ncta, P, ws.z);
  Cd* sN = ws.s2;
  c_sum_parts(ws.part + (int64_t)ncta * P, ncta, P, sN);
  if (threadIdx.x == 0) nrm2 = sN[k].re;
  __syncthreads();
  // w_i = sum_{j <= i} conj(S[j, i]) z_j
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    Cd acc = {0.0, 0.0};
    for (int j = 0; j <= i; j++) acc = cadd(acc, cmul(cconj(D.S[j + (int64_t)i * Tm]), ws.z[j]));
    ws.w[i] = acc;
  }
  double beta;
  c_append<T>(N, k, Tm, sN, nrm2, ws.d, &beta);
}

// fin2: the data-side reflector R_t = H_k(p) and the output coefficients.
template <typename T>
__global__ void __launch_bounds__(kCThreads) k_c_fin2(CStack D, CStack N, int k, int Tm, CWs ws, int ncta, int P) {
  __shared__ double nrm2, alpha;
  c_sum_parts(ws.part, ncta, P, ws.z);
  if (threadIdx.x == 0) nrm2 = ws.z[k].re;
  __syncthreads();
  // head of p (rows < k) before the pivot entry is overwritten
  const Cx<T>* p = (const Cx<T>*)ws.p;
  for (int i = threadIdx.x; i < k; i += blockDim.x) ws.d[i] = to_cd(p[i]);
  __syncthreads();
  double a;
  c_append<T>(D, k, Tm, ws.z, nrm2, ws.wout, &a);
  if (threadIdx.x == 0) alpha = a;
  __syncthreads();
  // c = [p_head; alpha]; d = Delta_N^H c with N holding k + 1 reflectors
  const int kn = k + 1;
  for (int i = threadIdx.x; i <= k; i += blockDim.x) {
    const Cd c = (i < k) ? ws.d[i] : Cd{alpha, 0.0};
    ws.d[i] = cmul(cconj(N.dpre[min(i, kn - 1) + 1]), c);
  }
  __syncthreads();
  // v_j = sum_{i <= k} conj(V_N[i, j]) d_i (j <= k), then w' = S_N v
  Cd* v = ws.z;
  const Cx<T>* VN = (const Cx<T>*)N.V;
  for (int j = threadIdx.x; j < kn; j += blockDim.x) {
    Cd acc = {0.0, 0.0};
    for (int i = j; i <= k; i++) acc = cadd(acc, cmul(cconj(to_cd(VN[i + (int64_t)j * N.ld])), ws.d[i]));
    v[j] = acc;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kn; i += blockDim.x) {
    Cd acc = {0.0, 0.0};
    for (int j = i; j < kn; j++) acc = cadd(acc, cmul(N.S[i + (int64_t)j * Tm], v[j]));
    ws.wout[i] = acc;
  }
}

// ---- complex Ginibre (Algorithm 1 with adjoints) ----------------------------------------
// A step with data space d and output space o (Q: d = the n-space; Q^H: the m-space): the data
// stack D holds kD reflectors, the other stack N holds kN; the basis store of the data space
// (Bd) holds kN columns (v_i of the other-type steps for Q, u_i for Q^H) and the one of the
// output space (Bo) kD columns.  Only D and Bo grow.
//   colpass(D-space, x)      z = V_D^H x, h = Bd^H x
//   colpass(o-space, draw)   V_N^H (sigma Z g); sigma Z g -> Bo column kD
//   fin1                     w = S_D^H z, w_g = S_N Delta_N^H V_N^H (Z g)  (the new basis vector
//                            u = Delta_N^H Z g - V_N w_g = N_1^H ... N_kN^H Z g)
//   rowpass(D), colpass(D, p), fin2   as for Haar; then w_h = S_N V_N^H Delta_N^H h over the head
//   out                      u as above -> Bo column kD;
//                            y = Bo[:, :kD] p_head + alpha u + Delta_N^H h - V_N w_h
// (the coefficients of the earlier same-type basis vectors are entries of p, eq. Gaussian_t).

// fin1 (Ginibre): partials of colpass(D-space) in part[0 .. ncD) with P slots (kD + kN dots),
// of colpass(o-space) in part[ncD .. ncD + ncN).
template <typename T>
__global__ void __launch_bounds__(kCThreads) k_cg_fin1(CStack D, CStack N, int kD, int kN, int Tm, CWs ws, int ncD,
                                                       int ncN, int P) {
  c_sum_parts(ws.part, ncD, P, ws.z);
  c_sum_parts(ws.part + (int64_t)ncD * P, ncN, P, ws.s2);
  for (int i = threadIdx.x; i < kN; i += blockDim.x) ws.h[i] = ws.z[kD + i];
  for (int i = threadIdx.x; i < kD; i += blockDim.x) {
    Cd acc = {0.0, 0.0};
    for (int j = 0; j <= i; j++) acc = cadd(acc, cmul(cconj(D.S[j + (int64_t)i * Tm]), ws.z[j]));
    ws.w[i] = acc;
  }
  // Delta_N^H on the draw's rows (>= kN) is the constant conj(dpre[kN])
  const Cd ph = cconj(N.dpre[kN]);
  for (int i = threadIdx.x; i < kN; i += blockDim.x) {
    Cd acc = {0.0, 0.0};
    for (int j = i; j < kN; j++) acc = cadd(acc, cmul(N.S[i + (int64_t)j * Tm], ws.s2[j]));
    ws.wg[i] = cmul(acc, ph);
  }
}

// fin2 (Ginibre): the data-side reflector, then the output coefficients.
template <typename T>
__global__ void __launch_bounds__(kCThreads) k_cg_fin2(CStack D, CStack N, int kD, int kN, int Tm, CWs ws, int ncta,
                                                       int P, double* alpha_out) {
  __shared__ double nrm2;
  c_sum_parts(ws.part, ncta, P, ws.z);
  if (threadIdx.x == 0) nrm2 = ws.z[kD].re;
  const Cx<T>* p = (const Cx<T>*)ws.p;
  for (int i = threadIdx.x; i < kD; i += blockDim.x) ws.c[i] = to_cd(p[i]);
  __syncthreads();
  c_append<T>(D, kD, Tm, ws.z, nrm2, ws.d, alpha_out);
  // w_h = S_N v, v_j = sum_{j <= i < kN} conj(V_N[i, j]) conj(dpre_N[i + 1]) h_i
  const Cx<T>* VN = (const Cx<T>*)N.V;
  Cd* v = ws.d;
  for (int j = threadIdx.x; j < kN; j += blockDim.x) {
    Cd acc = {0.0, 0.0};
    for (int i = j; i < kN; i++)
      acc = cadd(acc, cmul(cconj(to_cd(VN[i + (int64_t)j * N.ld])), cmul(cconj(N.dpre[i + 1]), ws.h[i])));
    v[j] = acc;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kN; i += blockDim.x) {
    Cd acc = {0.0, 0.0};
    for (int j = i; j < kN; j++) acc = cadd(acc, cmul(N.S[i + (int64_t)j * Tm], v[j]));
    ws.wout[i] = acc;
  }
}

// Output rows of a Ginibre step (rows [blockIdx.x * kCRows, +kCRows) of the output space):
// u = (rows >= kN: conj(dpre_N[kN]) g) - V_N w_g, stored over g in Bo column kD;
// y = Bo[:, :kD] c + alpha u + (rows < kN: conj(dpre_N[i + 1]) h_i) - V_N w_h.
template <typename T>
__global__ void __launch_bounds__(kCThreads) k_cg_out(CStack N, int kN, void* Bo, int64_t ldb, int kD, int64_t dim,
                                                      CWs ws, const double* alpha, void* out) {
  __shared__ Cx<T> cg[kCTmax], chh[kCTmax], cc[kCTmax];
  for (int j = threadIdx.x; j < kN; j += blockDim.x) {
    cg[j] = from_cd<T>(ws.wg[j]);
    chh[j] = from_cd<T>(ws.wout[j]);
  }
  for (int j = threadIdx.x; j < kD; j += blockDim.x) cc[j] = from_cd<T>(ws.c[j]);
  __syncthreads();
  const Cx<T>* VN = (const Cx<T>*)N.V;
  Cx<T>* B = (Cx<T>*)Bo;
  const T a = (T)(*alpha);
  const Cx<T> ph = from_cd<T>(cconj(N.dpre[kN]));
  const int64_t r0 = (int64_t)blockIdx.x * kCRows;
  constexpr int R = kCRows / kCThreads;
  Cx<T> u[R], y[R];
  int64_t row[R];
#pragma unroll
  for (int m = 0; m < R; m++) {
    const int64_t i = r0 + threadIdx.x + (int64_t)m * kCThreads;
    row[m] = i;
    u[m] = {T(0), T(0)};
    y[m] = {T(0), T(0)};
    if (i < dim) {
      if (i >= kN) {
        const Cx<T> g = B[i + (int64_t)kD * ldb];
        u[m] = {ph.re * g.re - ph.im * g.im, ph.re * g.im + ph.im * g.re};
      } else {
        const Cx<T> hp = from_cd<T>(cmul(cconj(N.dpre[i + 1]), ws.h[i]));
        y[m] = hp;
      }
    }
  }
  for (int j = 0; j < kN; j++) {
    const Cx<T> wgj = cg[j], whj = chh[j];
    const Cx<T>* col = VN + (int64_t)j * N.ld;
#pragma unroll
    for (int m = 0; m < R; m++) {
      if (row[m] < dim && row[m] >= j) {
        const Cx<T> vv = col[row[m]];
        cfms(u[m], vv, wgj);
        cfms(y[m], vv, whj);
      }
    }
  }
  for (int j = 0; j < kD; j++) {
    const Cx<T> cj = cc[j];
    const Cx<T>* col = B + (int64_t)j * ldb;
#pragma unroll
    for (int m = 0; m < R; m++) {
      if (row[m] < dim) {
        const Cx<T> b = col[row[m]];
        y[m].re = fma(b.re, cj.re, fma(-b.im, cj.im, y[m].re));
        y[m].im = fma(b.re, cj.im, fma(b.im, cj.re, y[m].im));
      }
    }
  }
#pragma unroll
  for (int m = 0; m < R; m++) {
    const int64_t i = row[m];
    if (i >= dim) continue;
    B[i + (int64_t)kD * ldb] = u[m];
    ((Cx<T>*)out)[i] = {fma(a, u[m].re, y[m].re), fma(a, u[m].im, y[m].im)};
  }
}

// y = (y + yh) / sqrt(2), elementwise (the GUE combination), complex.
template <typename T>
__global__ void __launch_bounds__(256) k_c_gue_combine(Cx<T>* y, const Cx<T>* yh, int64_t len) {
  const T r = (T)0.70710678118654752440;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = {(y[i].re + yh[i].re) * r, (y[i].im + yh[i].im) * r};
}

}  // namespace

struct hd_cstate {
  int ens = HD_HAAR;
  int dtype = HD_F64;
  int64_t dim[2] = {0, 0};   // 0: the n-space (R, input of Q), 1: the m-space (L)
  int Tm = 0;
  uint64_t seed = 0;
  uint32_t trial = 0;
  double sigma = 1.0;        // Ginibre entry scale
  cudaStream_t stream = nullptr;
  int device = 0;
  int t = 0;
  int cnt[2] = {0, 0};       // Ginibre: reflectors per stack (Q steps, Q^H steps)
  int poisoned = 0;
  size_t esz = 16;           // bytes of one complex element
  int ncta[2] = {1, 1};
  CStack st[2];              // 0: R (acts on the n-space), 1: L (the m-space)
  void* B[2] = {nullptr, nullptr};   // Ginibre basis stores per space (dim x Tm)
  int64_t ldb[2] = {0, 0};
  double* alpha = nullptr;   // Ginibre: the step's alpha (device)
  void* tmp = nullptr;       // GUE: the Q^H product
  CWs ws;
  std::vector<void*> allocs;
};

namespace {

void* c_alloc(hd_cstate* s, size_t bytes) {
  void* p = nullptr;
  bytes = (bytes + 255) & ~(size_t)255;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  s->allocs.push_back(p);
  return p;
}

void c_free(hd_cstate* s) {
  for (void* p : s->allocs) cudaFree(p);
  s->allocs.clear();
}

int c_fail(hd_cstate* s, const char* where, cudaError_t e) {
  hd::set_error(where, e);
  if (s) s->poisoned = HD_ERR_CUDA;
  return HD_ERR_CUDA;
}

// zero S and the phases, dpre[0] = 1 (stack and basis columns are rewritten by the step that
// creates them, and the passes never read a stack column above its pivot)
int c_clear(hd_cstate* s) {
  const size_t sb = (size_t)s->Tm * s->Tm * sizeof(Cd);
  const size_t db = (size_t)(s->Tm + 1) * sizeof(Cd);
  const Cd one = {1.0, 0.0};
  for (int q = 0; q < 2; q++) {
    cudaError_t e = cudaMemsetAsync(s->st[q].S, 0, sb, s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->st[q].dpre, 0, db, s->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->st[q].dpre, &one, sizeof(Cd), cudaMemcpyHostToDevice, s->stream);
    if (e != cudaSuccess) return c_fail(s, "hd_complex state clear", e);
  }
  // the host value `one` must outlive the copy
  if (cudaStreamSynchronize(s->stream) != cudaSuccess) return c_fail(s, "hd_complex state clear", cudaGetLastError());
  s->t = 0;
  s->cnt[0] = s->cnt[1] = 0;
  return HD_OK;
}

DrawKey c_key(const hd_cstate* s) {
  DrawKey key;
  key.k0 = (uint32_t)(s->seed & 0xFFFFFFFFu);
  key.k1 = (uint32_t)(s->seed >> 32);
  key.step = (uint32_t)(s->t + 1);
  key.trial = s->trial;
  key.stream = 0;
  return key;
}

template <typename T>
int c_step(hd_cstate* s, const void* x, int adjoint, void* y) {
  const int k = s->t;
  const int d = adjoint ? 1 : 0;
  const CStack D = s->st[d], N = s->st[1 - d];
  const DrawKey key = c_key(s);
  const int64_t n = s->dim[0];
  const int P = s->Tm + 1;
  const int nc = s->ncta[0];
  const size_t smem = (size_t)kCRows * sizeof(Cx<T>);
  cudaStream_t q = s->stream;
  Cd* partN = s->ws.part + (int64_t)nc * P;
  Cx<T>* colD = (Cx<T>*)D.V + (int64_t)k * D.ld;
  Cx<T>* colN = (Cx<T>*)N.V + (int64_t)k * N.ld;
  k_c_colpass<T><<<nc, kCThreads, smem, q>>>(D, k, nullptr, 0, 0, n, 0, x, key, T(1), 0, nullptr, s->ws.part, P);
  k_c_colpass<T><<<nc, kCThreads, smem, q>>>(N, k, nullptr, 0, 0, n, 1, nullptr, key, T(1), k, colN, partN, P);
  k_c_fin1<T><<<1, kCThreads, 0, q>>>(D, N, k, s->Tm, s->ws, nc, P);
  k_c_rowpass<T><<<nc, kCThreads, 0, q>>>(D, k, n, x, nullptr, 0, s->ws.w, 1, s->ws.p);
  k_c_colpass<T><<<nc, kCThreads, smem, q>>>(D, k, nullptr, 0, 0, n, 0, s->ws.p, key, T(1), k, colD, s->ws.part, P);
  k_c_fin2<T><<<1, kCThreads, 0, q>>>(D, N, k, s->Tm, s->ws, nc, P);
  k_c_rowpass<T><<<nc, kCThreads, 0, q>>>(N, k + 1, n, nullptr, s->ws.d, k + 1, s->ws.wout, 0, y);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return c_fail(s, "hd_complex_apply launch", e);
  s->t += 1;
  return HD_OK;
}

// One product of the complex Ginibre ensemble (see the kernels above).
template <typename T>
int c_step_gin(hd_cstate* s, const void* x, int adjoint, void* y) {
  const int d = adjoint ? 1 : 0, o = 1 - d;
  const int kD = s->cnt[d], kN = s->cnt[o];
  const CStack D = s->st[d], N = s->st[o];
  const DrawKey key = c_key(s);
  const int P = s->Tm + 1;
  const int ncD = s->ncta[d], ncN = s->ncta[o];
  const size_t smem = (size_t)kCRows * sizeof(Cx<T>);
  cudaStream_t q = s->stream;
  Cd* partN = s->ws.part + (int64_t)ncD * P;
  Cx<T>* colD = (Cx<T>*)D.V + (int64_t)kD * D.ld;
  Cx<T>* colBo = (Cx<T>*)s->B[o] + (int64_t)kD * s->ldb[o];
  k_c_colpass<T><<<ncD, kCThreads, smem, q>>>(D, kD, s->B[d], s->ldb[d], kN, s->dim[d], 0, x, key, T(1), 0, nullptr,
                                             s->ws.part, P);
  k_c_colpass<T><<<ncN, kCThreads, smem, q>>>(N, kN, nullptr, 0, 0, s->dim[o], 1, nullptr, key, (T)s->sigma, kN,
                                             colBo, partN, P);
  k_cg_fin1<T><<<1, kCThreads, 0, q>>>(D, N, kD, kN, s->Tm, s->ws, ncD, ncN, P);
  k_c_rowpass<T><<<ncD, kCThreads, 0, q>>>(D, kD, s->dim[d], x, nullptr, 0, s->ws.w, 1, s->ws.p);
  k_c_colpass<T><<<ncD, kCThreads, smem, q>>>(D, kD, nullptr, 0, 0, s->dim[d], 0, s->ws.p, key, T(1), kD, colD,
                                             s->ws.part, P);
  k_cg_fin2<T><<<1, kCThreads, 0, q>>>(D, N, kD, kN, s->Tm, s->ws, ncD, P, s->alpha);
  k_cg_out<T><<<ncN, kCThreads, 0, q>>>(N, kN, s->B[o], s->ldb[o], kD, s->dim[o], s->ws, s->alpha, y);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return c_fail(s, "hd_complex_apply launch", e);
  s->t += 1;
  s->cnt[d] += 1;
  return HD_OK;
}

int c_product(hd_cstate* s, const void* x, int adjoint, void* y) {
  if (s->ens == HD_HAAR)
    return (s->dtype == HD_F64) ? c_step<double>(s, x, adjoint, y) : c_step<float>(s, x, adjoint, y);
  return (s->dtype == HD_F64) ? c_step_gin<double>(s, x, adjoint, y) : c_step_gin<float>(s, x, adjoint, y);
}

}  // namespace

extern "C" {

HD_API int hd_complex_create(int ensemble, int64_t m, int64_t n, int32_t T_max, uint64_t seed, int dtype,
                             hd_cstate** out) {
  if (!out) return HD_ERR_ARG;
  *out = nullptr;
  if (ensemble != HD_HAAR && ensemble != HD_GINIBRE) return HD_ERR_ARG;
  if (dtype != HD_F64 && dtype != HD_F32) return HD_ERR_ARG;
  if (m <= 0 || n <= 0 || m > ((int64_t)1 << 36) || n > ((int64_t)1 << 36)) return HD_ERR_DIM;
  if (ensemble == HD_HAAR && m != n) return HD_ERR_DIM;
  if (T_max <= 0 || T_max > kCTmax || (int64_t)T_max > std::min(m, n)) return HD_ERR_TMAX;
  hd_cstate* s = new (std::nothrow) hd_cstate();
  if (!s) return HD_ERR_OOM;
  s->ens = ensemble;
  s->dtype = dtype;
  s->dim[0] = n;
  s->dim[1] = m;
  s->Tm = T_max;
  s->seed = seed;
  s->esz = (dtype == HD_F64) ? 16 : 8;
  if (cudaGetDevice(&s->device) != cudaSuccess) {
    hd::set_error("cudaGetDevice", cudaGetLastError());
    delete s;
    return HD_ERR_CUDA;
  }
  const int P = T_max + 1;
  int64_t ldmax = 0;
  bool ok = true;
  for (int q = 0; q < 2 && ok; q++) {
    s->ncta[q] = (int)((s->dim[q] + kCRows - 1) / kCRows);
    const int64_t ld = (s->dim[q] + 63) / 64 * 64;
    ldmax = std::max(ldmax, ld);
    s->st[q].ld = ld;
    s->st[q].V = c_alloc(s, (size_t)ld * T_max * s->esz);
    s->st[q].S = (Cd*)c_alloc(s, (size_t)T_max * T_max * sizeof(Cd));
    s->st[q].dpre = (Cd*)c_alloc(s, (size_t)(T_max + 1) * sizeof(Cd));
    ok = s->st[q].V && s->st[q].S && s->st[q].dpre;
    if (ok) ok = cudaMemset(s->st[q].V, 0, (size_t)ld * T_max * s->esz) == cudaSuccess;
    if (ok && ensemble == HD_GINIBRE) {
      s->ldb[q] = ld;
      s->B[q] = c_alloc(s, (size_t)ld * T_max * s->esz);
      ok = s->B[q] && cudaMemset(s->B[q], 0, (size_t)ld * T_max * s->esz) == cudaSuccess;
    }
  }
  if (ok) {
    const int nmax = std::max(s->ncta[0], s->ncta[1]);
    s->ws.part = (Cd*)c_alloc(s, (size_t)2 * nmax * P * sizeof(Cd));
    Cd* small = (Cd*)c_alloc(s, (size_t)8 * P * sizeof(Cd));
    s->ws.p = c_alloc(s, (size_t)ldmax * s->esz);
    s->alpha = (double*)c_alloc(s, 64);
    ok = s->ws.part && small && s->ws.p && s->alpha;
    if (ok) {
      s->ws.z = small;
      s->ws.w = small + P;
      s->ws.wout = small + 2 * P;
      s->ws.d = small + 3 * P;
      s->ws.s2 = small + 4 * P;
      s->ws.wg = small + 5 * P;
      s->ws.c = small + 6 * P;
      s->ws.h = small + 7 * P;
      ok = cudaMemset(small, 0, (size_t)8 * P * sizeof(Cd)) == cudaSuccess;
    }
    if (ok && ensemble == HD_GINIBRE && m == n) {
      s->tmp = c_alloc(s, (size_t)ldmax * s->esz);
      ok = s->tmp != nullptr;
    }
  }
  if (!ok) {
    c_free(s);
    delete s;
    return HD_ERR_OOM;
  }
  const int rc = c_clear(s);
  if (rc) {
    c_free(s);
    delete s;
    return rc;
  }
  *out = s;
  return HD_OK;
}

HD_API int hd_complex_set_options(hd_cstate* s, double sigma, uint32_t trial, void* stream) {
  if (!s) return HD_ERR_ARG;
  if (!(sigma > 0.0) || !std::isfinite(sigma)) return HD_ERR_ARG;
  if (s->t > 0 && (trial != s->trial || sigma != s->sigma)) return HD_ERR_ARG;
  s->trial = trial;
  s->sigma = sigma;
  s->stream = (cudaStream_t)stream;
  return HD_OK;
}

HD_API int hd_complex_apply(hd_cstate* s, const void* x, int adjoint, void* y) {
  if (!s || !x || !y || x == y) return HD_ERR_ARG;
  if (adjoint != 0 && adjoint != 1) return HD_ERR_ARG;
  if (((uintptr_t)x % s->esz) != 0 || ((uintptr_t)y % s->esz) != 0) return HD_ERR_ARG;
  if (s->poisoned) return s->poisoned;
  if (s->t >= s->Tm) return HD_ERR_TMAX;
  if (cudaSetDevice(s->device) != cudaSuccess) return c_fail(s, "cudaSetDevice", cudaErrorInvalidDevice);
  return c_product(s, x, adjoint, y);
}

HD_API int hd_complex_gue_apply(hd_cstate* s, const void* x, void* y) {
  if (!s || !x || !y || x == y) return HD_ERR_ARG;
  if (s->ens != HD_GINIBRE || s->dim[0] != s->dim[1]) return HD_ERR_ARG;
  if (((uintptr_t)x % s->esz) != 0 || ((uintptr_t)y % s->esz) != 0) return HD_ERR_ARG;
  if (s->poisoned) return s->poisoned;
  if (s->t + 2 > s->Tm) return HD_ERR_TMAX;
  if (cudaSetDevice(s->device) != cudaSuccess) return c_fail(s, "cudaSetDevice", cudaErrorInvalidDevice);
  int rc = c_product(s, x, 0, y);
  if (!rc) rc = c_product(s, x, 1, s->tmp);
  if (rc) return rc;
  const int64_t n = s->dim[0];
  const unsigned blocks = (unsigned)std::min<int64_t>((n + 255) / 256, 4096);
  if (s->dtype == HD_F64)
    k_c_gue_combine<double><<<blocks, 256, 0, s->stream>>>((Cx<double>*)y, (const Cx<double>*)s->tmp, n);
  else
    k_c_gue_combine<float><<<blocks, 256, 0, s->stream>>>((Cx<float>*)y, (const Cx<float>*)s->tmp, n);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? HD_OK : c_fail(s, "hd_complex_gue_apply launch", e);
}

HD_API int hd_complex_reset(hd_cstate* s, uint64_t seed) {
  if (!s) return HD_ERR_ARG;
  if (cudaSetDevice(s->device) != cudaSuccess) return c_fail(s, "cudaSetDevice", cudaErrorInvalidDevice);
  s->seed = seed;
  s->poisoned = 0;
  return c_clear(s);
}

HD_API int hd_complex_get_counts(const hd_cstate* s, int32_t* t) {
  if (!s || !t) return HD_ERR_ARG;
  *t = s->t;
  return HD_OK;
}

HD_API void hd_complex_destroy(hd_cstate* s) {
  if (!s) return;
  cudaSetDevice(s->device);
  if (s->stream) cudaStreamSynchronize(s->stream); else cudaDeviceSynchronize();
  c_free(s);
  delete s;
}

}  // extern "C"
