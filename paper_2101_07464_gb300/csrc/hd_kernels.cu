// Streaming kernels of one Householder Dice step (Algorithms 1 and 2) for sm_103a.
//
// One step with data-side stack D (R for M_t = Q, L for M_t = Q^T), k_D reflectors, and the
// other stack N, k_N reflectors, is three sweeps over HBM-resident stacks:
//
//   K1 dots    z = V_D^T x (and, for Ginibre, x . basis columns of the data space)
//              last CTA: w = S_D^T z, G_D w                           [pass 1 over V_D]
//   K2 update  p = Delta_D (x - V_D w)   (= R_{r-1}...R_1 x, eq. pt / Algorithm 1);
//              writes p[k:] as the new reflector vector of H_k(p) (eq. Householder_e),
//              draws g_{t+1} and its dots with V_D for the next step;
//              last CTA: ||p[k:]||, the sign, tau, the new S and Gram columns, and the
//              coefficients of the output sweep                      [pass 2 over V_D]
//   K3 output  Haar: y = L_1...L_{t-1} (L_t R_t p) with L_t R_t p = [p_head; alpha g/||g||]
//              (eq. Qtxt and eq. Householder_property), appends L_t = H_t(g_t) (eq.
//              Householder_e), dots of g_{t+1} with V_N.
//              Ginibre: u_t = L_1...L_l Z_{1:l} g_t and y = sum_i (v_i^T x) u_i
//              (Algorithm 1; the coefficients of earlier same-direction basis vectors are
//              entries of R_r...R_1 x, the others' are x . stored basis)  [pass over V_N]
//
// Every cross-CTA sum is formed in FP64 without waiting: each CTA writes its partial sums,
// the last CTA of each group of ~sqrt(#CTAs) sums its group, and the last group-finisher
// sums the groups and runs the O(k^2) FP64 finalisation.  The order of summation is fixed,
// so results are bitwise reproducible.
#include <cmath>

#include "hd_kernels.cuh"

namespace hd {

// ------------------------------------------------------------------------------------
// Block sums written to global memory: out[q] = sum over the CTA of a[q], q < nvalid.
template <int NV, typename T>
__device__ __forceinline__ void block_sum_to(const T (&a)[NV], double* red, double* out,
                                             int nvalid) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NV; q++) {
    T s = warp_sum(a[q]);
    if (lane == 0) red[warp * NV + q] = (double)s;
  }
  __syncthreads();
  if (threadIdx.x < nvalid) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < kWarps; w++) s += red[w * NV + threadIdx.x];
    out[threadIdx.x] = s;
  }
  __syncthreads();
}

__device__ __forceinline__ bool elect_last(unsigned int* counter, int expected) {
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned int prev = atomicAdd(counter, 1u);
    last = (prev == (unsigned int)(expected - 1));
  }
  __syncthreads();
  if (last) {
    __threadfence();
    if (threadIdx.x == 0) *counter = 0u;
  }
  return last;
}

// Two-level reduction of P partial sums per CTA (part[b * P + j]).  Returns true in the one
// CTA that finishes last; there out[j] holds the grand totals (FP64, fixed order).
__device__ bool reduce_partials(const Ws& ws, int set, int P, const Grid& g, double* out) {
  unsigned int* cnt = ws.cnt + set * (kMaxGroups + 1);
  const int b = blockIdx.x;
  const int grp = b / g.gsize;
  const int gfirst = grp * g.gsize;
  const int gcount = min(g.gsize, g.ctas - gfirst);
  if (!elect_last(&cnt[grp], gcount)) return false;
  for (int j = threadIdx.x; j < P; j += blockDim.x) {
    double s = 0.0;
    for (int c = 0; c < gcount; c++) s += ld_cg(&ws.part[(int64_t)(gfirst + c) * P + j]);
    ws.gpart[(int64_t)grp * P + j] = s;
  }
  if (!elect_last(&cnt[kMaxGroups], g.ngroups)) return false;
  for (int j = threadIdx.x; j < P; j += blockDim.x) {
    double s = 0.0;
    for (int q = 0; q < g.ngroups; q++) s += ld_cg(&ws.gpart[(int64_t)q * P + j]);
    out[j] = s;
  }
  __syncthreads();
  return true;
}

// Rows of this thread: vectors v0 + tid + c * kThreads, c < kChunkMax, inside [v0, v1).
struct Rows {
  int64_t v0, v1;
  __device__ Rows(const Grid& g, int64_t dim, int n) {
    const int64_t nvec = (dim + n - 1) / n;
    v0 = (int64_t)blockIdx.x * g.vpc;
    v1 = min(nvec, v0 + g.vpc);
  }
  __device__ __forceinline__ int64_t vec(int c) const { return v0 + threadIdx.x + (int64_t)c * kThreads; }
  __device__ __forceinline__ bool active(int c) const { return vec(c) < v1; }
};

template <typename T>
__device__ __forceinline__ T dot_vec(const Vec<T>& a, const Vec<T>& b, T acc) {
#pragma unroll
  for (int e = 0; e < Vec<T>::N; e++) acc = fma(a.e[e], b.e[e], acc);
  return acc;
}

// ------------------------------------------------------------------------------------
// First draw g_1 of a stack's space (rows >= count), its squared norm over rows > count.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_first_draw(StackDev X, int64_t count, DrawKey key,
                                                         T sigma, Ws ws, int set, Grid g) {
  constexpr int N = Vec<T>::N;
  __shared__ double red[kWarps];
  Rows rw(g, X.dim, N);
  T* gb = (T*)X.gbuf;
  T a[1] = {T(0)};
#pragma unroll
  for (int c = 0; c < kChunkMax; c++) {
    if (!rw.active(c)) continue;
    const int64_t row = rw.vec(c) * N;
    Vec<T> v;
    draw_vec(key, row, count, X.dim, sigma, v);
    st_vec(gb + row, v);
#pragma unroll
    for (int e = 0; e < N; e++)
      if (row + e > count) a[0] = fma(v.e[e], v.e[e], a[0]);
  }
  block_sum_to<1>(a, red, ws.part + blockIdx.x, 1);
  double* out = ws.scr(0);
  if (!reduce_partials(ws, set, 1, g, out)) return;
  if (threadIdx.x == 0) X.gg[0] = out[0];
}

// ------------------------------------------------------------------------------------
// K1: z = V_D^T x over k_D columns, then (Ginibre) the data-space basis columns.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_dots(StepPlan<T> p) {
  constexpr int N = Vec<T>::N;
  __shared__ double red[kWarps * kColBlock];
  const int64_t dim = p.D.dim;
  const int na = p.kD, nb = (p.ens == 0) ? p.kN : 0, nc = na + nb;
  const T* A = (const T*)p.D.V;
  const T* B = (const T*)p.Bd;
  Rows rw(p.g1, dim, N);
  Vec<T> xr[kChunkMax];
#pragma unroll
  for (int c = 0; c < kChunkMax; c++) {
    if (rw.active(c)) {
      ld_caller(p.x, rw.vec(c) * N, dim, p.xal != 0, xr[c]);
    } else {
#pragma unroll
      for (int e = 0; e < N; e++) xr[c].e[e] = T(0);
    }
  }
  double* part = p.ws.part + (int64_t)blockIdx.x * nc;
  for (int jb = 0; jb < nc; jb += kColBlock) {
    T acc[kColBlock];
#pragma unroll
    for (int q = 0; q < kColBlock; q++) acc[q] = T(0);
#pragma unroll
    for (int c = 0; c < kChunkMax; c++) {
      if (!rw.active(c)) continue;
      const int64_t row = rw.vec(c) * N;
#pragma unroll
      for (int q = 0; q < kColBlock; q++) {
        const int j = jb + q;
        if (j < nc) {
          const T* col = (j < na) ? A + (int64_t)j * p.D.ld : B + (int64_t)(j - na) * p.ldBd;
          Vec<T> v;
          ld_stream(col + row, v);
          acc[q] = dot_vec(v, xr[c], acc[q]);
        }
      }
    }
    block_sum_to<kColBlock>(acc, red, part + jb, min(kColBlock, nc - jb));
  }
  if (!reduce_partials(p.ws, 0, nc, p.g1, p.ws.z)) return;
  // w = S_D^T z (S upper triangular).
  const int Tm = p.Tm;
  for (int j = threadIdx.x; j < na; j += blockDim.x) {
    double s = 0.0;
    for (int i = 0; i <= j; i++) s = fma(p.D.S[i + (int64_t)j * Tm], p.ws.z[i], s);
    p.ws.w[j] = s;
  }
}

// ------------------------------------------------------------------------------------
// Finalisation after K2 (one CTA).  r[0..k) = dots of the next draw with the old columns of
// V_D, r[k] = with the new column, r[k+1] = ||p[k+1:]||^2, r[k+2] = ||g_{t+1}[k+2:]||^2,
// r[k+3+j] = V_D[k:, j] . p[k:] for the old columns j < k.
template <typename T>
__device__ void fin_update(const StepPlan<T>& p, const double* r) {
  const int k = p.kD, Tm = p.Tm;
  const int tid = threadIdx.x, nt = blockDim.x;
  __shared__ double sh[16];
  T* VD = (T*)p.D.V;
  const int64_t ldD = p.D.ld;
  double* vtu = p.ws.scr(0);
  double* vtg = p.ws.scr(1);
  double* zt = p.ws.scr(2);

  for (int j = tid; j <= k; j += nt) p.D.gdot[j] = r[j];
  if (tid == 0) {
    p.D.gg[0] = r[k + 2];
    const double ppiv = ld_cg(&p.ws.scal[kPpiv]);
    const double tail2 = r[k + 1];
    const double alpha = sqrt(tail2 + ppiv * ppiv);
    const double sp = (ppiv >= 0.0) ? 1.0 : -1.0;
    sh[0] = alpha;
    if (alpha == 0.0) {  // H_k(p) = I when p[k:] = 0 (eq. Householder_e)
      sh[1] = 0.0; sh[2] = 0.0; sh[3] = 1.0; sh[4] = 0.0;
    } else {
      const double us = (double)(T)(ppiv + sp * alpha);  // stored pivot of u
      const double uu = tail2 + us * us;                 // u^T u of the stored vector
      sh[1] = 2.0 / uu; sh[2] = us; sh[3] = -sp; sh[4] = uu;
    }
    sh[5] = ppiv;
    p.ws.scal[kAlpha] = alpha;
  }
  __syncthreads();
  const double alpha = sh[0], tau = sh[1], us = sh[2], dsign = sh[3], ppiv = sh[5];
  // V_D^T u with u = p[k:] + (u_k - p_k) e_k, from the exact dots of the sweep.
  for (int j = tid; j < k; j += nt)
    vtu[j] = r[k + 3 + j] + (us - ppiv) * (double)VD[k + (int64_t)j * ldD];
  __syncthreads();
  for (int j = tid; j < k; j += nt) {
    double s = 0.0;
    if (alpha != 0.0)
      for (int i = j; i < k; i++) s = fma(p.D.S[j + (int64_t)i * Tm], vtu[i], s);
    p.D.S[j + (int64_t)k * Tm] = -tau * s;
  }
  if (tid == 0) {
    p.D.S[k + (int64_t)k * Tm] = tau;
    p.D.dpre[k + 1] = p.D.dpre[k] * dsign;
    VD[k + (int64_t)k * ldD] = (T)us;
  }

  const T* VN = (const T*)p.N.V;
  const int64_t ldN = p.N.ld;
  if (p.ens == 1) {
    // Haar: L_t = H_t(g_t) from the stored draw, and the output coefficients
    // c = L_t R_t p = [p_head; alpha g[k:]/||g[k:]||]  (H(v) e_1 = v/||v||).
    if (tid == 0) {
      const double gpiv = (double)((const T*)p.N.gbuf)[k];
      const double gg = p.N.gg[0];
      const double ag = sqrt(gg + gpiv * gpiv);
      const double sg = (gpiv >= 0.0) ? 1.0 : -1.0;
      if (ag == 0.0) {
        sh[8] = 0.0; sh[9] = 0.0; sh[10] = 1.0; sh[11] = 0.0; sh[12] = 0.0; sh[13] = 1.0;
      } else {
        const double usg = (double)(T)(gpiv + sg * ag);
        const double uug = gg + usg * usg;
        sh[8] = 2.0 / uug; sh[9] = usg; sh[10] = -sg; sh[11] = uug; sh[12] = alpha / ag; sh[13] = 0.0;
      }
      sh[14] = gpiv;
      p.ws.scal[kCoef] = sh[12];
      p.ws.scal[kUpivG] = sh[9];
      p.ws.scal[kGFlag] = sh[13];
    }
    __syncthreads();
    const double taug = sh[8], usg = sh[9], dg = sh[10], coef = sh[12];
    const bool flag = sh[13] != 0.0;
    const double gpiv = sh[14];
    const double deltaN = p.N.dpre[k];
    for (int j = tid; j < k; j += nt) {
      const double vk = (double)VN[k + (int64_t)j * ldN];
      vtg[j] = flag ? 0.0 : p.N.gdot[j] + (usg - gpiv) * vk;
      double tz = 0.0;
      for (int i = j; i < k; i++)
        tz = fma((double)VN[i + (int64_t)j * ldN], p.N.dpre[i + 1] * ld_cg(&p.ws.phead[i]), tz);
      zt[j] = tz + deltaN * (flag ? alpha * vk : coef * p.N.gdot[j]);
    }
    __syncthreads();
    for (int j = tid; j < k; j += nt) {
      double sw = 0.0, sc = 0.0;
      for (int i = j; i < k; i++) {
        const double sji = p.N.S[j + (int64_t)i * Tm];
        sw = fma(sji, zt[i], sw);
        sc = fma(sji, vtg[i], sc);
      }
      p.ws.wout[j] = sw;
      p.N.S[j + (int64_t)k * Tm] = -taug * sc;
    }
    if (tid == 0) {
      p.N.S[k + (int64_t)k * Tm] = taug;
      p.N.dpre[k + 1] = p.N.dpre[k] * dg;
    }
  } else {
    // Ginibre: h = x . (data-space basis), w_h = S_N V_N^T Delta_N h (top block),
    // w_2 = S_N V_N^T Delta_N g (g on rows >= k_N where Delta_N is constant).
    const int kN = p.kN;
    const double* h = p.ws.z + p.kD;
    const double deltaN = p.N.dpre[kN];
    for (int j = tid; j < kN; j += nt) {
      double tz = 0.0;
      for (int i = j; i < kN; i++)
        tz = fma((double)VN[i + (int64_t)j * ldN], p.N.dpre[i + 1] * h[i], tz);
      zt[j] = tz;
    }
    __syncthreads();
    for (int j = tid; j < kN; j += nt) {
      double sw = 0.0, s2 = 0.0;
      for (int i = j; i < kN; i++) {
        const double sji = p.N.S[j + (int64_t)i * Tm];
        sw = fma(sji, zt[i], sw);
        s2 = fma(sji, p.N.gdot[i], s2);
      }
      p.ws.wout[j] = sw;
      p.ws.wout2[j] = deltaN * s2;
    }
  }
}

// K2: p = Delta_D (x - V_D w); new column k of V_D; next draw; exact dots of p[k:] and of
// the next draw with the old columns of V_D.
//
// The dots of p need p final, i.e. after all k columns of a row were applied, so the sweep
// stages a tile of R rows x k columns of V_D in shared memory (one HBM read):
//   loop 1, row owners:    p_i = Delta_i (x_i - sum_j V_ij w_j)  (256/R threads per row);
//   loop 2, column owners: thread j accumulates sum_i V_ij p_i and sum_i V_ij g_i.
// The tile has row stride R + 1 so that both loops are free of bank conflicts.
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}
__device__ __forceinline__ void cp_async_elem(float* s, const float* g) { cp_async4(s, g); }
__device__ __forceinline__ void cp_async_elem(double* s, const double* g) { cp_async8(s, g); }

template <typename T>
__global__ void __launch_bounds__(kThreads) k_update(StepPlan<T> p) {
  extern __shared__ __align__(16) unsigned char dsm_raw[];
  __shared__ double red[kWarps * 4];
  const int k = p.kD, R = p.R2, Rs = R + 1;
  const int G1 = kThreads / R;               // threads per row in loop 1
  T* Vt = reinterpret_cast<T*>(dsm_raw);     // k x Rs
  T* pv = Vt + (size_t)k * Rs;               // R: p[k:] (zero above row k)
  T* gv = pv + R;                            // R: next draw
  T* ps = gv + R;                            // kThreads: loop-1 partial sums
  T* wsm = ps + kThreads;                    // k: w
  const int tid = threadIdx.x;
  const int64_t dim = p.D.dim;
  for (int j = tid; j < k; j += kThreads) wsm[j] = (T)p.ws.w[j];
  T* V = (T*)p.D.V;
  const int64_t ld = p.D.ld;
  T* gb = (T*)p.D.gbuf;
  T* col = V + (int64_t)k * ld;
  const T dconst = (T)p.D.dpre[k];
  const int ri = tid % R, rq = tid / R;
  double accp[kColsPerThread], accg[kColsPerThread];  // columns tid + c*kThreads
#pragma unroll
  for (int c = 0; c < kColsPerThread; c++) accp[c] = accg[c] = 0.0;
  T ex[3] = {T(0), T(0), T(0)};              // p . g_next, ||p[k+1:]||^2, ||g_next[k+2:]||^2
  for (int64_t tile = blockIdx.x; tile < p.ntiles2; tile += gridDim.x) {
    const int64_t r0 = tile * R;
    for (int idx = tid; idx < k * R; idx += kThreads) {
      const int j = idx / R, i = idx - j * R;
      if (r0 + i < ld) cp_async_elem(&Vt[j * Rs + i], V + (int64_t)j * ld + r0 + i);
      else Vt[j * Rs + i] = T(0);
    }
    if (tid < R / 2) {
      T a, b;
      const int64_t row = r0 + 2 * tid;
      if (row + 1 >= (int64_t)k + 1 && row < dim) {
        normal_pair(p.key_next, (uint64_t)(row >> 1), a, b);
        a = (row >= (int64_t)k + 1 && row < dim) ? p.sigma * a : T(0);
        b = (row + 1 >= (int64_t)k + 1 && row + 1 < dim) ? p.sigma * b : T(0);
      } else {
        a = b = T(0);
      }
      gv[2 * tid] = a;
      gv[2 * tid + 1] = b;
    }
    cp_async_wait_all();
    __syncthreads();
    {
      T s = T(0);
      for (int j = rq; j < k; j += G1) s = fma(Vt[j * Rs + ri], wsm[j], s);
      ps[rq * R + ri] = s;
    }
    __syncthreads();
    if (tid < R) {
      const int64_t i = r0 + tid;
      T xi = T(0);
      if (i < dim) xi = p.x[i];
      T acc = xi;
      for (int q = 0; q < G1; q++) acc -= ps[q * R + tid];
      const T d = (i < k) ? (T)p.D.dpre[i + 1] : dconst;
      const T pvv = acc * d;
      const T g = gv[tid];
      if (i < dim) {
        if (i < k) p.ws.phead[i] = (double)pvv;
        else {
          col[i] = pvv;
          if (i == k) p.ws.scal[kPpiv] = (double)pvv;
          else ex[1] = fma(pvv, pvv, ex[1]);
          ex[0] = fma(pvv, g, ex[0]);
        }
        if (i >= (int64_t)k + 2) ex[2] = fma(g, g, ex[2]);
      }
      if (i < ld) gb[i] = g;
      pv[tid] = (i >= k && i < dim) ? pvv : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < kColsPerThread; c++) {
      const int j = tid + c * kThreads;
      if (j < k) {
        T sp = T(0), sg = T(0);
        const T* vc = Vt + j * Rs;
        for (int i = 0; i < R; i++) {
          const T v = vc[i];
          sp = fma(v, pv[i], sp);
          sg = fma(v, gv[i], sg);
        }
        accp[c] += (double)sp;
        accg[c] += (double)sg;
      }
    }
    __syncthreads();
  }
  const int P = 2 * k + 3;
  double* part = p.ws.part + (int64_t)blockIdx.x * P;
#pragma unroll
  for (int c = 0; c < kColsPerThread; c++) {
    const int j = tid + c * kThreads;
    if (j < k) {
      part[j] = accg[c];
      part[k + 3 + j] = accp[c];
    }
  }
  block_sum_to<3>(ex, red, part + k, 3);
  double* r = p.ws.scr(3);
  if (!reduce_partials(p.ws, 1, P, p.g2, r)) return;
  fin_update<T>(p, r);
}

// ------------------------------------------------------------------------------------
// K3 (Haar): y = Delta_N c - V_N w', appends the random reflector column, and dots of the
// next draw (copied from the data stack's buffer) with V_N.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_out_haar(StepPlan<T> p) {
  constexpr int N = Vec<T>::N;
  extern __shared__ unsigned char dsm_raw[];
  T* wsm = reinterpret_cast<T*>(dsm_raw);
  __shared__ double red[kWarps * kColBlock];
  const int k = p.kN;
  const int64_t dim = p.N.dim;
  for (int j = threadIdx.x; j < k; j += kThreads) wsm[j] = (T)p.ws.wout[j];
  __syncthreads();
  T* V = (T*)p.N.V;
  const int64_t ld = p.N.ld;
  T* gcur = (T*)p.N.gbuf;
  const T* gnext = (const T*)p.D.gbuf;
  const T coef = (T)p.ws.scal[kCoef];
  const T alpha = (T)p.ws.scal[kAlpha];
  const T usg = (T)p.ws.scal[kUpivG];
  const bool flag = p.ws.scal[kGFlag] != 0.0;
  const T dconst = (T)p.N.dpre[k];
  Rows rw(p.g3, dim, N);
  Vec<T> yr[kChunkMax], gn[kChunkMax];
  T ex[1] = {T(0)};
#pragma unroll
  for (int c = 0; c < kChunkMax; c++) {
    if (!rw.active(c)) {
#pragma unroll
      for (int e = 0; e < N; e++) yr[c].e[e] = gn[c].e[e] = T(0);
      continue;
    }
    const int64_t row = rw.vec(c) * N;
    Vec<T> g, ncol;
    ld_stream(gcur + row, g);
    ld_stream(gnext + row, gn[c]);
#pragma unroll
    for (int e = 0; e < N; e++) {
      const int64_t i = row + e;
      T ci;
      if (i < k) ci = (T)p.ws.phead[i];
      else if (flag) ci = (i == k) ? alpha : T(0);
      else ci = coef * g.e[e];
      const T d = (i < k) ? (T)p.N.dpre[i + 1] : dconst;
      yr[c].e[e] = d * ci;
      ncol.e[e] = (i > k) ? g.e[e] : ((i == k) ? usg : T(0));
      ex[0] = fma(ncol.e[e], gn[c].e[e], ex[0]);
    }
    T* col = V + (int64_t)k * ld;
    if (row >= k && row + N <= dim) {
      st_vec(col + row, ncol);
    } else {
#pragma unroll
      for (int e = 0; e < N; e++)
        if (row + e >= k && row + e < dim) col[row + e] = ncol.e[e];
    }
    st_vec(gcur + row, gn[c]);
  }
  const int P = k + 1;
  double* part = p.ws.part + (int64_t)blockIdx.x * P;
  for (int jb = 0; jb < k; jb += kColBlock) {
    T acc[kColBlock];
#pragma unroll
    for (int q = 0; q < kColBlock; q++) acc[q] = T(0);
#pragma unroll
    for (int c = 0; c < kChunkMax; c++) {
      if (!rw.active(c)) continue;
      const int64_t row = rw.vec(c) * N;
#pragma unroll
      for (int q = 0; q < kColBlock; q++) {
        const int j = jb + q;
        if (j < k) {
          Vec<T> v;
          ld_stream(V + (int64_t)j * ld + row, v);
          const T wj = wsm[j];
#pragma unroll
          for (int e = 0; e < N; e++) yr[c].e[e] = fma(-v.e[e], wj, yr[c].e[e]);
          acc[q] = dot_vec(v, gn[c], acc[q]);
        }
      }
    }
    block_sum_to<kColBlock>(acc, red, part + jb, min(kColBlock, k - jb));
  }
#pragma unroll
  for (int c = 0; c < kChunkMax; c++)
    if (rw.active(c)) st_caller(p.y, rw.vec(c) * N, dim, p.yal != 0, yr[c]);
  block_sum_to<1>(ex, red, part + k, 1);
  double* r = p.ws.scr(3);
  if (!reduce_partials(p.ws, 2, P, p.g3, r)) return;
  for (int j = threadIdx.x; j <= k; j += blockDim.x) p.N.gdot[j] = r[j];
  if (threadIdx.x == 0) p.N.gg[0] = p.D.gg[0];
}

// K3 (Ginibre): u = Delta_N g - V_N w_2 (= L_1..L_l Z g), y = alpha u + Delta_N h - V_N w_h
// + B_n c, appends u to the other-space basis, draws g_{t+1} and its dots with V_N.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_out_gin(StepPlan<T> p) {
  constexpr int N = Vec<T>::N;
  extern __shared__ unsigned char dsm_raw[];
  const int kN = p.kN, kD = p.kD;
  T* w2 = reinterpret_cast<T*>(dsm_raw);
  T* wh = w2 + kN;
  T* cb = wh + kN;
  __shared__ double red[kWarps * kColBlock];
  const int64_t dim = p.N.dim;
  for (int j = threadIdx.x; j < kN; j += kThreads) {
    w2[j] = (T)p.ws.wout2[j];
    wh[j] = (T)p.ws.wout[j];
  }
  for (int j = threadIdx.x; j < kD; j += kThreads) cb[j] = (T)p.ws.phead[j];
  __syncthreads();
  const T* V = (const T*)p.N.V;
  const int64_t ld = p.N.ld;
  T* Bn = (T*)p.Bn;
  T* gcur = (T*)p.N.gbuf;
  const double* h = p.ws.z + kD;
  const T alpha = (T)p.ws.scal[kAlpha];
  const T dconst = (T)p.N.dpre[kN];
  Rows rw(p.g3, dim, N);
  Vec<T> ur[kChunkMax], yr[kChunkMax], gn[kChunkMax];
#pragma unroll
  for (int c = 0; c < kChunkMax; c++) {
    if (!rw.active(c)) {
#pragma unroll
      for (int e = 0; e < N; e++) ur[c].e[e] = yr[c].e[e] = gn[c].e[e] = T(0);
      continue;
    }
    const int64_t row = rw.vec(c) * N;
    Vec<T> g;
    ld_stream(gcur + row, g);
    draw_vec(p.key_next, row, (int64_t)kN, dim, p.sigma, gn[c]);
#pragma unroll
    for (int e = 0; e < N; e++) {
      const int64_t i = row + e;
      const T d = (i < kN) ? (T)p.N.dpre[i + 1] : dconst;
      ur[c].e[e] = d * g.e[e];
      yr[c].e[e] = (i < kN) ? d * (T)h[i] : T(0);
    }
    st_vec(gcur + row, gn[c]);
  }
  const int P = kN;
  double* part = p.ws.part + (int64_t)blockIdx.x * P;
  for (int jb = 0; jb < kN; jb += kColBlock) {
    T acc[kColBlock];
#pragma unroll
    for (int q = 0; q < kColBlock; q++) acc[q] = T(0);
#pragma unroll
    for (int c = 0; c < kChunkMax; c++) {
      if (!rw.active(c)) continue;
      const int64_t row = rw.vec(c) * N;
#pragma unroll
      for (int q = 0; q < kColBlock; q++) {
        const int j = jb + q;
        if (j < kN) {
          Vec<T> v;
          ld_stream(V + (int64_t)j * ld + row, v);
          const T a2 = w2[j], ah = wh[j];
#pragma unroll
          for (int e = 0; e < N; e++) {
            ur[c].e[e] = fma(-v.e[e], a2, ur[c].e[e]);
            yr[c].e[e] = fma(-v.e[e], ah, yr[c].e[e]);
          }
          acc[q] = dot_vec(v, gn[c], acc[q]);
        }
      }
    }
    block_sum_to<kColBlock>(acc, red, part + jb, min(kColBlock, kN - jb));
  }
  for (int jb = 0; jb < kD; jb += kColBlock) {
#pragma unroll
    for (int c = 0; c < kChunkMax; c++) {
      if (!rw.active(c)) continue;
      const int64_t row = rw.vec(c) * N;
#pragma unroll
      for (int q = 0; q < kColBlock; q++) {
        const int j = jb + q;
        if (j < kD) {
          Vec<T> v;
          ld_stream(Bn + (int64_t)j * p.ldBn + row, v);
          const T cj = cb[j];
#pragma unroll
          for (int e = 0; e < N; e++) yr[c].e[e] = fma(v.e[e], cj, yr[c].e[e]);
        }
      }
    }
  }
  T* ucol = Bn + (int64_t)kD * p.ldBn;
#pragma unroll
  for (int c = 0; c < kChunkMax; c++) {
    if (!rw.active(c)) continue;
    const int64_t row = rw.vec(c) * N;
    Vec<T> yv;
#pragma unroll
    for (int e = 0; e < N; e++) {
      yv.e[e] = fma(alpha, ur[c].e[e], yr[c].e[e]);
      if (row + e >= dim) ur[c].e[e] = T(0);
    }
    st_vec(ucol + row, ur[c]);
    st_caller(p.y, row, dim, p.yal != 0, yv);
  }
  if (kN == 0) {
    // no partial sums: still elect nothing; the next draw needs no dots
    return;
  }
  double* r = p.ws.scr(3);
  if (!reduce_partials(p.ws, 2, P, p.g3, r)) return;
  for (int j = threadIdx.x; j < kN; j += blockDim.x) p.N.gdot[j] = r[j];
}

// ------------------------------------------------------------------------------------
template <typename T>
cudaError_t launch_first_draw(StackDev X, int64_t count, DrawKey key, T sigma, Ws ws, int set,
                              Grid g, cudaStream_t s) {
  k_first_draw<T><<<g.ctas, kThreads, 0, s>>>(X, count, key, sigma, ws, set, g);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_step(const StepPlan<T>& p, cudaStream_t s) {
  const int nc1 = p.kD + ((p.ens == 0) ? p.kN : 0);
  if (nc1 > 0) k_dots<T><<<p.g1.ctas, kThreads, 0, s>>>(p);
  k_update<T><<<p.g2.ctas, kThreads, update_smem_bytes<T>(p.kD, p.R2), s>>>(p);
  if (p.ens == 1)
    k_out_haar<T><<<p.g3.ctas, kThreads, (size_t)p.kN * sizeof(T), s>>>(p);
  else
    k_out_gin<T><<<p.g3.ctas, kThreads, (size_t)(2 * p.kN + p.kD) * sizeof(T), s>>>(p);
  return cudaGetLastError();
}

template <typename T>
cudaError_t set_update_smem_limit(int bytes) {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, k_update<T>);
  if (e != cudaSuccess) return e;
  const int dyn = bytes - (int)fa.sharedSizeBytes;
  return cudaFuncSetAttribute(k_update<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
}
template cudaError_t set_update_smem_limit<float>(int);
template cudaError_t set_update_smem_limit<double>(int);

template <typename T>
int kernel_occupancy(int which, size_t dynsmem) {
  int nb = 0;
  cudaError_t e = cudaSuccess;
  switch (which) {
    case 0: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_dots<T>, kThreads, dynsmem); break;
    case 1: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_update<T>, kThreads, dynsmem); break;
    case 2: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_out_haar<T>, kThreads, dynsmem); break;
    default: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_out_gin<T>, kThreads, dynsmem); break;
  }
  return (e == cudaSuccess && nb > 0) ? nb : 1;
}
template int kernel_occupancy<float>(int, size_t);
template int kernel_occupancy<double>(int, size_t);

template cudaError_t launch_first_draw<float>(StackDev, int64_t, DrawKey, float, Ws, int, Grid, cudaStream_t);
template cudaError_t launch_first_draw<double>(StackDev, int64_t, DrawKey, double, Ws, int, Grid, cudaStream_t);
template cudaError_t launch_step<float>(const StepPlan<float>&, cudaStream_t);
template cudaError_t launch_step<double>(const StepPlan<double>&, cudaStream_t);

// ------------------------------------------------------------------------------------
// Consistency probe (not on the hot path): y = Q^(t) x from the revealed part only.
//   q = H_{k_D-1}...H_0 x = Delta_D (x - V_D w)  (w = S_D^T V_D^T x from k_dots);
//   unrevealed = ||q[k_D:]||;
//   Haar:    y = B_N [q[:t]; 0]              (eq. H_t: the hidden block never sees q[:t])
//   Ginibre: y = B_N [h; 0] + B_n q[:k_D]    (h = x . data-space basis), eq. Gaussian_t.
template <typename T>
__global__ void k_probe_q(StepPlan<T> p, double* q, double* unrev) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int k = p.kD;
  double u2 = 0.0;
  if (i < p.D.dim) {
    const T* V = (const T*)p.D.V;
    double acc = (double)p.x[i];
    for (int j = 0; j < k; j++) acc -= (double)V[i + (int64_t)j * p.D.ld] * p.ws.w[j];
    const double d = (k == 0) ? 1.0 : ((i < k) ? p.D.dpre[i + 1] : p.D.dpre[k]);
    q[i] = d * acc;
    if (i >= k) u2 = q[i] * q[i];
  }
  u2 = warp_sum(u2);
  if ((threadIdx.x & 31) == 0) atomicAdd(unrev, u2);
}

template <typename T>
__global__ void k_probe_coef(StepPlan<T> p, const double* q) {
  // one CTA: zt = V_N[top]^T Delta_N c_top, w' = S_N zt  (c_top = q[:t] for Haar, h for Ginibre)
  const int kN = p.kN, Tm = p.Tm;
  const T* VN = (const T*)p.N.V;
  double* zt = p.ws.scr(0);
  const double* c = (p.ens == 1) ? q : p.ws.z + p.kD;
  for (int j = threadIdx.x; j < kN; j += blockDim.x) {
    double s = 0.0;
    for (int i = j; i < kN; i++) s += (double)VN[i + (int64_t)j * p.N.ld] * p.N.dpre[i + 1] * c[i];
    zt[j] = s;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < kN; j += blockDim.x) {
    double s = 0.0;
    for (int i = j; i < kN; i++) s += p.N.S[j + (int64_t)i * Tm] * zt[i];
    p.ws.wout[j] = s;
  }
}

template <typename T>
__global__ void k_probe_out(StepPlan<T> p, const double* q) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= p.N.dim) return;
  const int kN = p.kN;
  const T* VN = (const T*)p.N.V;
  const double* c = (p.ens == 1) ? q : p.ws.z + p.kD;
  const double d = (kN == 0) ? 1.0 : ((i < kN) ? p.N.dpre[i + 1] : p.N.dpre[kN]);
  double acc = (i < kN) ? d * c[i] : 0.0;
  for (int j = 0; j < kN; j++) acc -= (double)VN[i + (int64_t)j * p.N.ld] * p.ws.wout[j];
  if (p.ens == 0) {
    const T* Bn = (const T*)p.Bn;
    for (int j = 0; j < p.kD; j++) acc += (double)Bn[i + (int64_t)j * p.ldBn] * q[j];
  }
  p.y[i] = (T)acc;
}

template <typename T>
cudaError_t launch_probe(const StepPlan<T>& p, double* q, double* unrev, cudaStream_t s) {
  const int nc1 = p.kD + ((p.ens == 0) ? p.kN : 0);
  if (nc1 > 0) k_dots<T><<<p.g1.ctas, kThreads, 0, s>>>(p);
  const int thr = 256;
  k_probe_q<T><<<(unsigned)((p.D.dim + thr - 1) / thr), thr, 0, s>>>(p, q, unrev);
  k_probe_coef<T><<<1, thr, 0, s>>>(p, q);
  k_probe_out<T><<<(unsigned)((p.N.dim + thr - 1) / thr), thr, 0, s>>>(p, q);
  return cudaGetLastError();
}
template cudaError_t launch_probe<float>(const StepPlan<float>&, double*, double*, cudaStream_t);
template cudaError_t launch_probe<double>(const StepPlan<double>&, double*, double*, cudaStream_t);

// ------------------------------------------------------------------------------------
// Generator checks.
template <typename T>
__global__ void k_philox_normals(DrawKey key, int64_t start, int64_t count, T* out) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x + (start >> 1);
  const int64_t i0 = 2 * j;
  if (i0 >= start + count) return;
  T a, b;
  normal_pair(key, (uint64_t)j, a, b);
  if (i0 >= start) out[i0 - start] = a;
  if (i0 + 1 >= start && i0 + 1 < start + count) out[i0 + 1 - start] = b;
}

__global__ void k_philox_words(uint32_t k0, uint32_t k1, const uint32_t* ctr, int64_t nblocks,
                               uint32_t* out) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nblocks) return;
  PhiloxOut o = philox4x32_10(ctr[4 * b], ctr[4 * b + 1], ctr[4 * b + 2], ctr[4 * b + 3], k0, k1);
  for (int q = 0; q < 4; q++) out[4 * b + q] = o.w[q];
}

cudaError_t launch_philox_normals(DrawKey key, int64_t start, int64_t count, int dtype, void* out,
                                  cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  const int64_t pairs = ((start + count + 1) >> 1) - (start >> 1);
  const int thr = 256;
  const int64_t blocks = (pairs + thr - 1) / thr;
  if (dtype == 0)
    k_philox_normals<double><<<(unsigned)blocks, thr, 0, s>>>(key, start, count, (double*)out);
  else
    k_philox_normals<float><<<(unsigned)blocks, thr, 0, s>>>(key, start, count, (float*)out);
  return cudaGetLastError();
}

cudaError_t launch_philox_words(uint32_t k0, uint32_t k1, const uint32_t* ctr, int64_t nblocks,
                                uint32_t* out, cudaStream_t s) {
  if (nblocks <= 0) return cudaSuccess;
  const int thr = 256;
  k_philox_words<<<(unsigned)((nblocks + thr - 1) / thr), thr, 0, s>>>(k0, k1, ctr, nblocks, out);
  return cudaGetLastError();
}

}  // namespace hd
