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
    const int nw = blockDim.x >> 5;
    for (int w = 0; w < nw; w++) s += red[w * NV + threadIdx.x];
    out[threadIdx.x] = s;
  }
  __syncthreads();
}

// d * v for a prefix sign d, which is exactly +1 or -1 (a product of the reflectors' signs):
// the sign bit of d is moved onto v with integer operations (on this GPU an FP64 multiply
// takes a slot of the FP64 pipe, which bounds the FP64 sweeps).
__device__ __forceinline__ double sign_mul(double d, double v) {
  return __longlong_as_double(__double_as_longlong(v) ^ (__double_as_longlong(d) & (long long)0x8000000000000000ull));
}
__device__ __forceinline__ float sign_mul(float d, float v) {
  return __int_as_float(__float_as_int(v) ^ (__float_as_int(d) & (int)0x80000000u));
}
// sign(y) in {-1, 0, 1} (0 for +-0 and NaN) from the bits of y.
__device__ __forceinline__ double sign_of(double y) {
  const long long b = __double_as_longlong(y);
  const long long a = b & 0x7FFFFFFFFFFFFFFFll;
  return (a == 0 || a > 0x7FF0000000000000ll) ? 0.0 : ((b < 0) ? -1.0 : 1.0);
}
__device__ __forceinline__ float sign_of(float y) {
  const int b = __float_as_int(y);
  const int a = b & 0x7FFFFFFF;
  return (a == 0 || a > 0x7F800000) ? 0.0f : ((b < 0) ? -1.0f : 1.0f);
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

// Two-level reduction of P partial sums per CTA of one trial (part[local * P + j]): the last
// CTA of each group of ~sqrt(ncta) CTAs sums its group, the last group-finisher sums the
// groups.  Returns true in that one CTA; there out[j] holds the totals (FP64, fixed order).
__device__ __forceinline__ int group_size(int ncta) {
  int g = (int)sqrtf((float)ncta);
  while (g * g < ncta) g++;
  return g < 1 ? 1 : g;
}
__device__ bool reduce_partials(const Ws& ws, int set, int P, int local, int ncta, double* out) {
  unsigned int* cnt = ws.cnt + set * (kMaxGroups + 1);
  const int gsize = group_size(ncta);
  const int ngroups = (ncta + gsize - 1) / gsize;
  const int grp = local / gsize;
  const int gfirst = grp * gsize;
  const int gcount = min(gsize, ncta - gfirst);
  // (two interleaved FP64 sums per value: dependent FP64 adds are slow on this GPU)
  if (!elect_last(&cnt[grp], gcount)) return false;
  for (int j = threadIdx.x; j < P; j += blockDim.x) {
    double s0 = 0.0, s1 = 0.0;
    int c = 0;
#pragma unroll 4
    for (; c + 1 < gcount; c += 2) {
      s0 += ld_cg(&ws.part[(int64_t)(gfirst + c) * P + j]);
      s1 += ld_cg(&ws.part[(int64_t)(gfirst + c + 1) * P + j]);
    }
    if (c < gcount) s0 += ld_cg(&ws.part[(int64_t)(gfirst + c) * P + j]);
    ws.gpart[(int64_t)grp * P + j] = s0 + s1;
  }
  if (!elect_last(&cnt[kMaxGroups], ngroups)) return false;
  for (int j = threadIdx.x; j < P; j += blockDim.x) {
    double s0 = 0.0, s1 = 0.0;
    int q = 0;
#pragma unroll 4
    for (; q + 1 < ngroups; q += 2) {
      s0 += ld_cg(&ws.gpart[(int64_t)q * P + j]);
      s1 += ld_cg(&ws.gpart[(int64_t)(q + 1) * P + j]);
    }
    if (q < ngroups) s0 += ld_cg(&ws.gpart[(int64_t)q * P + j]);
    out[j] = s0 + s1;
  }
  __syncthreads();
  return true;
}

// The CTA's trial and place within it, and the trial's view of a batched step.
struct CtaCtx {
  int trial, local, ncta, spc;
};
// vb: the CTA's index in the space's CTA map (blockIdx.x, or a virtual CTA of the step kernel).
template <typename T>
__device__ __forceinline__ StepPlan<T> make_plan(const BatchStep<T>& b, int space, int vb, CtaCtx& c) {
  const CtaMap& m = b.map[space];
  c.trial = m.cta_trial[vb];
  const int c0 = m.cta0[c.trial];
  c.ncta = m.nct[c.trial];
  c.local = vb - c0;
  c.spc = m.spc[c.trial];
  const TrialDesc& td = b.desc[c.trial];
  const int d = b.d;
  StepPlan<T> p = b.base;
  p.D = td.st[d];
  p.N = td.st[1 - d];
  p.Bd = td.basis[d];
  p.ldBd = td.ldb[d];
  p.Bn = td.basis[1 - d];
  p.ldBn = td.ldb[1 - d];
  p.sigma = (T)td.sigma;
  p.ws = td.ws;
  p.key_next.trial = td.trial;
  p.x = b.base.x ? b.base.x + td.off[d] : nullptr;
  p.y = b.base.y ? b.base.y + td.off[1 - d] : nullptr;
  p.xnext = b.base.xnext ? b.base.xnext + td.off[1 - d] : nullptr;
  p.xprev = b.base.xprev ? b.base.xprev + td.off[1 - d] : nullptr;
  p.amp_v = b.base.amp_v ? b.base.amp_v + td.off[1 - d] : nullptr;
  p.amp_y = b.base.amp_y ? b.base.amp_y + td.off[1 - d] : nullptr;
  p.amp_w = b.base.amp_w ? b.base.amp_w + td.off[1 - d] : nullptr;
  p.yrec = b.base.yrec ? b.base.yrec + td.off[1 - d] : nullptr;
  p.xrec = b.base.xrec ? b.base.xrec + td.off[1 - d] : nullptr;
  p.xgiven = b.base.xgiven ? b.base.xgiven + td.off[1 - d] : nullptr;
  return p;
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
// First draw g_1 of a space (rows >= 0) into the buffer of the stack acting on that space,
// for every trial, with its squared norm over rows > 0.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_first_draw(BatchStep<T> b, int space, DrawKey key) {
  __shared__ double red[kWarps];
  CtaCtx c;
  const CtaMap& m = b.map[space];
  c.trial = m.cta_trial[blockIdx.x];
  const int c0 = m.cta0[c.trial];
  c.ncta = m.nct[c.trial];
  c.local = (int)blockIdx.x - c0;
  c.spc = m.spc[c.trial];
  const TrialDesc& td = b.desc[c.trial];
  const StackDev X = td.st[space];
  key.trial = td.trial;
  const T sigma = (T)td.sigma;
  const int64_t nsub = (X.dim + 31) / 32;
  const int64_t s0 = (int64_t)c.local * c.spc, s1 = min(nsub, s0 + c.spc);
  T* gb = (T*)X.gbuf;
  const int lane = threadIdx.x & 31, W = blockDim.x >> 5;
  T a[1] = {T(0)};
  for (int64_t s = s0 + (threadIdx.x >> 5); s < s1; s += W) {
    const int64_t r = s * 32 + lane;
    T g = T(0), h = T(0);
    const int64_t r2 = r & ~(int64_t)1;
    if (!(lane & 1) && r2 < X.dim) normal_pair(key, (uint64_t)(r2 >> 1), g, h);
    const T other = __shfl_up_sync(0xffffffffu, h, 1);
    T v = (lane & 1) ? other : g;
    v = (r < X.dim) ? sigma * v : T(0);
    gb[r] = v;
    if (r > 0) a[0] = fma(v, v, a[0]);
  }
  block_sum_to<1>(a, red, td.ws.part + c.local, 1);
  double* out = td.ws.scr(0);
  if (!reduce_partials(td.ws, 0, 1, c.local, c.ncta, out)) return;
  if (threadIdx.x == 0) X.gg[0] = out[0];
}

// ------------------------------------------------------------------------------------
// CTA-wide helpers of the finalisations (every thread of the CTA calls them).  The small
// matrices they read (S, the head block of V) are in L2 or DRAM.  They are copied into shared
// memory with one bulk copy per column, all in flight at once on one mbarrier (a single
// memory round trip); when a matrix does not fit in the free shared memory the product reads
// it from global memory instead.

__device__ __forceinline__ uint32_t smem_u32(const void* ptr) {
  return (uint32_t)__cvta_generic_to_shared(ptr);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
// A finalisation can run several times in one CTA of the step kernel (one trial after
// another), so it invalidates its barrier when done: an mbarrier is initialised only when
// the location holds no valid barrier object.
__device__ __forceinline__ void mbar_inval(uint64_t* bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t* bar, unsigned parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

// One staging round: the CTA's threads issue bulk copies (issue(tid) returns nothing), thread 0
// posts the byte count and waits, at most kStageSpins polls, for the copies; the outcome is
// one decision for the whole CTA.  On a timeout the error word is set, thread 0 gives the
// copies still in flight a second bounded wait (a CTA must not exit with bulk copies into its
// shared memory outstanding), and false is returned: the caller skips the product, and the
// state is poisoned (its outputs are undefined) until hd_reset.
constexpr unsigned kStageSpins = 1u << 22;
struct Stager {
  uint64_t* bar;
  unsigned parity;
  unsigned* err;
  unsigned limit = kStageSpins;   // polls before the wait gives up
  // begin(): issue the copies (every thread calls it); finish(): wait for them (bounded).
  template <typename Issue>
  __device__ void begin(unsigned bytes, Issue issue) {
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0) mbar_arrive_tx(bar, bytes);
    issue();
  }
  __device__ bool finish() {
    __shared__ int s_ok;
    if (threadIdx.x == 0) {
      unsigned spins = 0;
      bool ok = true;
      while (!mbar_test(bar, parity)) {
        if (++spins > limit) {
          ok = false;
          break;
        }
      }
      if (!ok) {
        if (err) atomicOr(err, 1u);
        unsigned drain = 0;
        while (!mbar_test(bar, parity) && ++drain <= limit) {
        }
      }
      s_ok = ok ? 1 : 0;
    }
    __syncthreads();
    const bool ok = s_ok != 0;
    parity ^= 1u;
    __syncthreads();   // s_ok is reused by the next round
    return ok;
  }
  template <typename Issue>
  __device__ bool run(unsigned bytes, Issue issue) {
    begin(bytes, issue);
    return finish();
  }
};

// Packed upper triangle: column c holds rows 0..c, padded to an even count (16-byte copies).
__device__ __forceinline__ int64_t up_off(int c) {
  return (c & 1) ? (int64_t)(c + 1) * (c + 1) / 2 : (int64_t)c * c / 2 + c;
}
__device__ __forceinline__ bool stage_upper(Stager& sg, const double* S, int Sld, int k, double* dst) {
  return sg.run((unsigned)(up_off(k) * 8), [&]() {
    for (int c = threadIdx.x; c < k; c += blockDim.x)
      bulk_g2s(dst + up_off(c), S + (int64_t)c * Sld, (unsigned)(((c + 2) & ~1) * 8), sg.bar);
  });
}
// Columns 0..ncol-1, rows 0..rows-1 of a stack, padded to 16 bytes: column j at j * Lv.
template <typename T>
__device__ __forceinline__ int stage_lv(int rows) {
  return (rows * (int)sizeof(T) + 15) / 16 * (16 / (int)sizeof(T));
}
template <typename T>
__device__ __forceinline__ bool stage_cols(Stager& sg, const T* V, int64_t ld, int rows, int ncol, T* dst) {
  const int Lv = stage_lv<T>(rows);
  return sg.run((unsigned)((int64_t)Lv * ncol * sizeof(T)), [&]() {
    for (int j = threadIdx.x; j < ncol; j += blockDim.x)
      bulk_g2s(dst + (int64_t)j * Lv, V + (int64_t)j * ld, (unsigned)(Lv * sizeof(T)), sg.bar);
  });
}

// FP64 on this GPU has a long dependent latency (about 65 cycles per FMA), so the products below
// split every row or column sum over a group of G lanes (G a power of two, G * rows <= CTA
// threads), each lane with two interleaved accumulators, and add the group's lanes with
// shuffles in a fixed order (deterministic).
__device__ __forceinline__ int lanes_per_item(int items) {
  int G = 32;
  while (G > 1 && G * items > (int)blockDim.x) G >>= 1;
  return G;
}
__device__ __forceinline__ double group_sum(double s, int G) {
  for (int o = G >> 1; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

// o_r[j] = sc_r sum_{i >= j} S[j, i] f_r[i] (j < k) from the packed upper triangle Su (or, when
// Su is null, from S in global memory).
template <int NR>
__device__ void upper_mv(const double* Su, const double* S, int Sld, int k, const double* f1, const double* f2,
                         double* o1, double sc1, double* o2, double sc2) {
  const int G = lanes_per_item(k);
  const int groups = blockDim.x / G, g = threadIdx.x % G;
  const int iters = (k + groups - 1) / groups;
  for (int it = 0; it < iters; it++) {
    const int j = it * groups + (int)threadIdx.x / G;
    double a0 = 0.0, a1 = 0.0, b0 = 0.0, b1 = 0.0;
    if (j < k) {
      int i = j + g;
      for (; i + G < k; i += 2 * G) {
        const double s0 = Su ? Su[up_off(i) + j] : S[j + (int64_t)i * Sld];
        const double s1 = Su ? Su[up_off(i + G) + j] : S[j + (int64_t)(i + G) * Sld];
        a0 = fma(s0, f1[i], a0);
        a1 = fma(s1, f1[i + G], a1);
        if (NR > 1) {
          b0 = fma(s0, f2[i], b0);
          b1 = fma(s1, f2[i + G], b1);
        }
      }
      if (i < k) {
        const double s0 = Su ? Su[up_off(i) + j] : S[j + (int64_t)i * Sld];
        a0 = fma(s0, f1[i], a0);
        if (NR > 1) b0 = fma(s0, f2[i], b0);
      }
    }
    const double r1 = group_sum(a0 + a1, G);
    const double r2 = (NR > 1) ? group_sum(b0 + b1, G) : 0.0;
    if (j < k && g == 0) {
      o1[j] = sc1 * r1;
      if (NR > 1) o2[j] = sc2 * r2;
    }
  }
  __syncthreads();
}

// out[j] = sum_{lo_j <= i <= hi_j} A[i, j] v[i] (j < ncol), A with leading dim lda (staged or
// global).
template <typename TA, typename LoHi>
__device__ void col_dots(const TA* A, int64_t lda, int ncol, const double* v, LoHi lohi, double* out) {
  const int G = lanes_per_item(ncol);
  const int groups = blockDim.x / G, g = threadIdx.x % G;
  const int iters = (ncol + groups - 1) / groups;
  for (int it = 0; it < iters; it++) {
    const int j = it * groups + (int)threadIdx.x / G;
    double a0 = 0.0, a1 = 0.0;
    if (j < ncol) {
      int lo, hi;
      lohi(j, lo, hi);
      const TA* Aj = A + (int64_t)j * lda;
      int i = lo + g;
      for (; i + G <= hi; i += 2 * G) {
        a0 = fma((double)Aj[i], v[i], a0);
        a1 = fma((double)Aj[i + G], v[i + G], a1);
      }
      if (i <= hi) a0 = fma((double)Aj[i], v[i], a0);
    }
    const double r = group_sum(a0 + a1, G);
    if (j < ncol && g == 0) out[j] = r;
  }
  __syncthreads();
}


// Finalisation of the dot sweep (one CTA): w = S^T z over n columns (w_j = S[0:j+1, j] . z),
// S staged as a packed upper triangle when it fits in the free shared memory.
__device__ void fin_dots(const double* S, int Sld, int na, const double* zs, double* w, double* scr, int64_t capb,
                         unsigned* err) {
  __shared__ uint64_t dbar;
  if (threadIdx.x == 0) mbar_init(&dbar);
  Stager sg{&dbar, 0u, err};
  const bool st = na > 0 && up_off(na) * 8 <= capb && stage_upper(sg, S, Sld, na, scr);
  if (st) {
    const int G = lanes_per_item(na);
    const int groups = blockDim.x / G, g = threadIdx.x % G;
    const int iters = (na + groups - 1) / groups;
    for (int it = 0; it < iters; it++) {
      const int j = it * groups + (int)threadIdx.x / G;
      double a0 = 0.0, a1 = 0.0;
      if (j < na) {
        const double* Sj = scr + up_off(j);
        int i = g;
        for (; i + G <= j; i += 2 * G) {
          a0 = fma(Sj[i], zs[i], a0);
          a1 = fma(Sj[i + G], zs[i + G], a1);
        }
        if (i <= j) a0 = fma(Sj[i], zs[i], a0);
      }
      const double r = group_sum(a0 + a1, G);
      if (j < na && g == 0) w[j] = r;
    }
  } else {
    col_dots(S, (int64_t)Sld, na, zs, [](int j, int& lo, int& hi) { lo = 0; hi = j; }, w);
  }
  __syncthreads();
  if (threadIdx.x == 0) mbar_inval(&dbar);
}

// Finalisation after K2 (one CTA).  r[0..k) = dots of the next draw with the old columns of
// V_D, r[k] = with the new column, r[k+1] = ||p[k+1:]||^2, r[k+2] = ||g_{t+1}[k+2:]||^2,
// r[k+3+j] = V_D[k:, j] . p[k:] for the old columns j < k.  Small vectors are staged in
// shared memory; the O(k^2) products read S and V columns coalesced, spread over the CTA's
// warps (scr: the sweep's dynamic shared memory, free at this point).
template <typename T>
__device__ void fin_update(const StepPlan<T>& p, const double* r, double* scr, int cap) {
  const int k = p.kD, Tm = p.Tm;
  const int tid = threadIdx.x, nt = blockDim.x;
  __shared__ double sh[16];
  __shared__ double f_a[kTmaxLimit + 1];
  __shared__ double f_b[kTmaxLimit + 1];
  __shared__ double f_c[kTmaxLimit + 1];
  __shared__ uint64_t fbar;
  T* VD = (T*)p.D.V;
  const int64_t ldD = p.D.ld;
  const T* VN = (const T*)p.N.V;
  const int64_t ldN = p.N.ld;
  if (tid == 0) mbar_init(&fbar);
  Stager sg{&fbar, 0u, p.ws.err};
  const int64_t capb = (int64_t)cap * 8;   // free shared memory in bytes

  // The three small matrices of this finalisation (S_D, the head block of V_N, S_N), staged in
  // one round while the scalars are formed, when they fit together.
  const int kNs = (p.ens == 1) ? k : p.kN;
  const int Lv = stage_lv<T>(kNs);
  const int64_t bSD = (k > 0) ? up_off(k) * 8 : 0;
  const int64_t bVN = (int64_t)Lv * kNs * (int64_t)sizeof(T);
  const int64_t bSN = (kNs > 0) ? up_off(kNs) * 8 : 0;
  const bool all = bSD + bVN + bSN > 0 && bSD + bVN + bSN <= capb;
  double* sSD = scr;
  T* sVN = (T*)((char*)scr + bSD);
  double* sSN = (double*)((char*)scr + bSD + bVN);
  if (all)
    sg.begin((unsigned)(bSD + bVN + bSN), [&]() {
      for (int c = tid; c < k; c += nt)
        bulk_g2s(sSD + up_off(c), p.D.S + (int64_t)c * Tm, (unsigned)(((c + 2) & ~1) * 8), sg.bar);
      for (int j = tid; j < kNs; j += nt)
        bulk_g2s(sVN + (int64_t)j * Lv, VN + (int64_t)j * ldN, (unsigned)(Lv * sizeof(T)), sg.bar);
      for (int c = tid; c < kNs; c += nt)
        bulk_g2s(sSN + up_off(c), p.N.S + (int64_t)c * Tm, (unsigned)(((c + 2) & ~1) * 8), sg.bar);
    });

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
  if (p.ens == 1 && tid == (nt > 32 ? 32 : 0)) {
    // Haar: L_t = H_t(g_t) from the stored draw (formed beside the data-side scalars)
    const double gpiv = (double)((const T*)p.N.gbuf)[k];
    const double gg = p.N.gg[0];
    const double ag = sqrt(gg + gpiv * gpiv);
    const double sg2 = (gpiv >= 0.0) ? 1.0 : -1.0;
    if (ag == 0.0) {
      sh[8] = 0.0; sh[9] = 0.0; sh[10] = 1.0; sh[11] = 0.0; sh[13] = 1.0;
    } else {
      const double usg = (double)(T)(gpiv + sg2 * ag);
      const double uug = gg + usg * usg;
      sh[8] = 2.0 / uug; sh[9] = usg; sh[10] = -sg2; sh[11] = ag; sh[13] = 0.0;
    }
    sh[14] = gpiv;
  }
  __syncthreads();
  const double alpha = sh[0], tau = sh[1], us = sh[2], dsign = sh[3], ppiv = sh[5];
  // V_D^T u with u = p[k:] + (u_k - p_k) e_k, from the exact dots of the sweep; then the new
  // column of S: S[:k, k] = -tau S V_D^T u
  double* ua_out = p.ws.scr(1);   // V_D^T u, kept for the reverse mode
  for (int j = tid; j < k; j += nt) {
    f_a[j] = r[k + 3 + j] + (us - ppiv) * (double)VD[k + (int64_t)j * ldD];
    ua_out[j] = f_a[j];
  }
  __syncthreads();
  const bool staged = all && sg.finish();
  {
    const bool st = staged || (k > 0 && !all && up_off(k) * 8 <= capb && stage_upper(sg, p.D.S, Tm, k, scr));
    upper_mv<1>(st ? sSD : nullptr, p.D.S, Tm, k, f_a, nullptr, p.D.S + (int64_t)k * Tm,
                (alpha != 0.0) ? -tau : 0.0, nullptr, 0.0);
  }
  if (tid == 0) {
    p.D.S[k + (int64_t)k * Tm] = tau;
    p.D.dpre[k + 1] = p.D.dpre[k] * dsign;
    VD[k + (int64_t)k * ldD] = (T)us;
  }

  if (p.ens == 1) {
    // Haar: the output coefficients c = L_t R_t p = [p_head; alpha g[k:]/||g[k:]||]
    // (H(v) e_1 = v/||v||)
    if (tid == 0) {
      sh[12] = (sh[13] != 0.0) ? 0.0 : alpha / sh[11];
      p.ws.scal[kCoef] = sh[12];
      p.ws.scal[kUpivG] = sh[9];
      p.ws.scal[kGFlag] = sh[13];
    }
    for (int i = tid; i < k; i += nt) f_b[i] = p.N.dpre[i + 1] * ld_cg(&p.ws.phead[i]);
    __syncthreads();
    const double taug = sh[8], usg = sh[9], dg = sh[10], coef = sh[12];
    const bool flag = sh[13] != 0.0;
    const double gpiv = sh[14];
    const double deltaN = p.N.dpre[k];
    // tz_j = V_N[j:k, j] . (Delta_N p_head)[j:k]
    {
      const bool st = staged || (k > 0 && !all && (int64_t)Lv * k * (int64_t)sizeof(T) <= capb &&
                                 stage_cols(sg, VN, ldN, k, k, (T*)scr));
      const T* vsrc = staged ? sVN : (st ? (const T*)scr : VN);
      col_dots(vsrc, st ? (int64_t)Lv : ldN, k, f_b, [k](int j, int& lo, int& hi) { lo = j; hi = k - 1; }, f_a);
    }
    __syncthreads();
    double* ug_out = p.ws.scr(2);   // V_N^T u_g, kept for the reverse mode
    for (int j = tid; j < k; j += nt) {
      const double vk = (double)VN[k + (int64_t)j * ldN];
      const double gd = p.N.gdot[j];
      f_c[j] = flag ? 0.0 : gd + (usg - gpiv) * vk;
      ug_out[j] = f_c[j];
      f_a[j] += deltaN * (flag ? alpha * vk : coef * gd);
    }
    __syncthreads();
    {
      const bool st = staged || (k > 0 && !all && up_off(k) * 8 <= capb && stage_upper(sg, p.N.S, Tm, k, scr));
      upper_mv<2>(st ? (staged ? sSN : scr) : nullptr, p.N.S, Tm, k, f_a, f_c, p.ws.wout, 1.0,
                  p.N.S + (int64_t)k * Tm, -taug);
    }
    if (tid == 0) {
      p.N.S[k + (int64_t)k * Tm] = taug;
      p.N.dpre[k + 1] = p.N.dpre[k] * dg;
    }
  } else {
    // Ginibre: h = x . (data-space basis), w_h = S_N V_N^T Delta_N h (top block),
    // w_2 = S_N V_N^T Delta_N g (g on rows >= k_N where Delta_N is constant).
    const int kN = p.kN;
    const double deltaN = p.N.dpre[kN];
    for (int i = tid; i < kN; i += nt) {
      f_b[i] = p.N.dpre[i + 1] * p.ws.z[p.kD + i];
      f_c[i] = p.N.gdot[i];
    }
    __syncthreads();
    {
      const bool st = staged || (kN > 0 && !all && (int64_t)Lv * kN * (int64_t)sizeof(T) <= capb &&
                                 stage_cols(sg, VN, ldN, kN, kN, (T*)scr));
      const T* vsrc = staged ? sVN : (st ? (const T*)scr : VN);
      col_dots(vsrc, st ? (int64_t)Lv : ldN, kN, f_b, [kN](int j, int& lo, int& hi) { lo = j; hi = kN - 1; },
               f_a);
    }
    {
      const bool st = staged || (kN > 0 && !all && up_off(kN) * 8 <= capb && stage_upper(sg, p.N.S, Tm, kN, scr));
      upper_mv<2>(st ? (staged ? sSN : scr) : nullptr, p.N.S, Tm, kN, f_a, f_c, p.ws.wout, 1.0, p.ws.wout2,
                  deltaN);
    }
  }
  __syncthreads();
  if (tid == 0) mbar_inval(&fbar);
}

// The finalisations out of line.  In a batch every trial has its own finaliser, so most CTAs
// of a launch run one (in a single-trial launch only the last CTA does, on the critical
// path); kept out of the sweep kernels' bodies, their code no longer shares the register
// allocation of the streaming loops, which then run faster, while each call pays for copying
// its arguments.  The batched sweeps call these (FIN_OUT), single-trial launches the inlined
// forms.
template <typename T>
__device__ __noinline__ void fin_update_out(const StepPlan<T>& p, const double* r, double* scr, int cap) {
  fin_update<T>(p, r, scr, cap);
}
__device__ __noinline__ void fin_dots_out(const double* S, int Sld, int na, const double* zs, double* w, double* scr,
                                          int64_t capb, unsigned* err) {
  fin_dots(S, Sld, na, zs, w, scr, capb, err);
}

// ------------------------------------------------------------------------------------
// Warp sub-tile engine shared by the three sweeps.
//
// Every warp walks its own 32-row sub-tiles (lane = row) of the stack, grid-strided over
// all warps of the launch, with no CTA-wide synchronisation inside the walk.  A sub-tile
// (32 rows x ncol columns) is copied by 16-byte cp.async into the warp's shared-memory
// slice, column-major with the 16-byte chunk q of column j stored at slot (q + j) mod NCH.
// On it two access patterns run without bank conflicts:
//   row owner:    lane i computes out[i] = sum_j V[i, j] coef[j]   (4-byte reads, one row
//                 per lane, coefficients read 16 bytes at a time);
//   column owner: lane l owns columns l, l + 32, ... (or, for up to 16 columns, a group of
//                 lanes shares a column) and adds sum_i V[i, j] rhs[i] (16-byte reads of its
//                 column's rotated chunks, the rhs chunk is a broadcast) to running sums in
//                 the storage type, which go into per-warp FP64 sums every kColFlush
//                 sub-tiles.
// At the end the warps of a CTA add their column sums in shared memory and the CTA joins
// the two-level last-block reduction.

template <typename T>
struct ColSrc {
  const T* A;
  int64_t ldA;
  int nA;
  const T* B;
  int64_t ldB;
  __device__ __forceinline__ const T* col(int j) const {
    return (j < nA) ? A + (int64_t)j * ldA : B + (int64_t)(j - nA) * ldB;
  }
};

template <typename T>
struct WT {
  static constexpr int ROWS = 32;
  static constexpr int VEC = 16 / (int)sizeof(T);  // elements per 16-byte chunk
  static constexpr int NCH = ROWS / VEC;           // chunks per column: 8 (FP32), 16 (FP64)
};

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(smem)), "l"(gmem) : "memory");
}
// L2 policy for the stack columns the sweeps stream once per launch: evict first, so that the
// small per-step data (S, coefficients, partial sums, vectors) stays resident in L2.
__device__ __forceinline__ uint64_t l2_evict_first() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;\n" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ void cp_async16_stream(void* smem, const void* gmem, uint64_t pol) {
  asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;\n" ::"r"(smem_u32(smem)), "l"(gmem),
               "l"(pol) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Copy rows [r0, r0 + 32) of ncol columns into a warp stage (no commit).  Lane l always
// copies chunk q = l mod NCH of the columns l / NCH, l / NCH + 32 / NCH, ...  Staged layout:
// column j at 32 j.  In FP64 chunk c of column j sits at slot (c + j) mod NCH (rotated); in
// FP32 at slot c (plain), and the column owners visit the chunks in rotated order instead
// (wt_col_pair), which keeps the same bank pattern and lets the row owners read at constant
// offsets (wt_rows).
template <typename T>
__device__ __forceinline__ int wt_slot(int c, int j) {
  return sizeof(T) == 4 ? c : ((c + j) & (WT<T>::NCH - 1));
}
template <typename T>
__device__ __forceinline__ void wt_load_cols(T* buf, const ColSrc<T>& src, int ncol, int64_t r0) {
  constexpr int NCH = WT<T>::NCH, VEC = WT<T>::VEC, CPI = 32 / NCH;
  const int lane = threadIdx.x & 31;
  const int q = lane & (NCH - 1);
  int j = lane / NCH;
  const int nA = min(ncol, src.nA);
  const uint64_t pol = l2_evict_first();
  {
    const T* g = src.A + (int64_t)j * src.ldA + r0 + q * VEC;
    const int64_t gstep = (int64_t)CPI * src.ldA;
    for (; j < nA; j += CPI, g += gstep) cp_async16_stream(buf + j * 32 + wt_slot<T>(q, j) * VEC, g, pol);
  }
  if (j < ncol) {
    const T* g = src.B + (int64_t)(j - src.nA) * src.ldB + r0 + q * VEC;
    const int64_t gstep = (int64_t)CPI * src.ldB;
    for (; j < ncol; j += CPI, g += gstep) cp_async16_stream(buf + j * 32 + wt_slot<T>(q, j) * VEC, g, pol);
  }
}
__device__ __forceinline__ void cp_async16_zfill(void* smem, const void* gmem, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(smem)), "l"(gmem),
               "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async4_zfill(void* smem, const void* gmem, int src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(smem_u32(smem)), "l"(gmem),
               "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async8_zfill(void* smem, const void* gmem, int src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(smem_u32(smem)), "l"(gmem),
               "r"(src_bytes) : "memory");
}
// Copy rows [r0, r0 + 32) of a vector of length dim into dst (32 elements), zero beyond
// dim; 16-byte copies when the vector is 16-byte aligned, element copies otherwise.
template <typename T>
__device__ __forceinline__ void wt_load_vec(T* dst, const T* v, int64_t r0, int64_t dim, bool al) {
  constexpr int VEC = WT<T>::VEC, NCH = WT<T>::NCH;
  const int lane = threadIdx.x & 31;
  if (al) {
    if (lane < NCH) {
      const int64_t row = r0 + lane * VEC;
      const int64_t avail = dim - row;
      const int bytes = (avail <= 0) ? 0 : (avail >= VEC ? 16 : (int)(avail * sizeof(T)));
      cp_async16_zfill(dst + lane * VEC, bytes > 0 ? (const void*)(v + row) : (const void*)v, bytes);
    }
  } else {
    const int64_t row = r0 + lane;
    const int bytes = (row < dim) ? (int)sizeof(T) : 0;
    if (sizeof(T) == 4) cp_async4_zfill(dst + lane, bytes ? (const void*)(v + row) : (const void*)v, bytes);
    else cp_async8_zfill(dst + lane, bytes ? (const void*)(v + row) : (const void*)v, bytes);
  }
}
// cp.async.wait_group with a run-time count of groups allowed to stay pending (0..7).
__device__ __forceinline__ void cp_async_wait_dyn(int pending) {
  switch (pending) {
    case 0: cp_async_wait<0>(); break;
    case 1: cp_async_wait<1>(); break;
    case 2: cp_async_wait<2>(); break;
    case 3: cp_async_wait<3>(); break;
    case 4: cp_async_wait<4>(); break;
    case 5: cp_async_wait<5>(); break;
    case 6: cp_async_wait<6>(); break;
    default: cp_async_wait<7>(); break;
  }
}

// FP32 dot-product steps as packed FMAs (two FP32 FMAs per instruction, sm_100 and later):
// acc.x collects the even terms, acc.y the odd ones, added once at the end of a sub-tile.
__device__ __forceinline__ float2 ffma2(float a0, float a1, float b0, float b1, float2 acc) {
  return __ffma2_rn(make_float2(a0, a1), make_float2(b0, b1), acc);
}

// Row owner: out[o] = sum_j V[lane, j] coef_o[j], o < NO (coef arrays padded to NCH).
// FP32 (plain layout): row lane of column j sits at 32 j + lane.  FP64 (rotated): column
// j = NCH g + u of the lane's row sits at NCH * 32 * g + off[u]; the NCH offsets of one
// rotation period depend only on the lane.
template <typename T, int NO>
__device__ __forceinline__ void wt_rows(const T* buf, int ncol, const T* coef0, const T* coef1,
                                        T (&out)[NO]) {
  constexpr int NCH = WT<T>::NCH, VEC = WT<T>::VEC;
  const int lane = threadIdx.x & 31;
  const int qi = lane / VEC, ri = lane & (VEC - 1);
  int off[NCH];
#pragma unroll
  for (int u = 0; u < NCH; u++) off[u] = u * 32 + ((qi + u) & (NCH - 1)) * VEC + ri;
#pragma unroll
  for (int o = 0; o < NO; o++) out[o] = T(0);
  const int ng = ncol / NCH;
  const T* base = buf;
  if constexpr (sizeof(T) == 4) {   // plain layout: row lane of column u at 32 u + lane
    float2 p[NO];   // packed FMAs over pairs of columns
#pragma unroll
    for (int o = 0; o < NO; o++) p[o] = make_float2(0.f, 0.f);
    const T* bl = buf + lane;
    for (int g = 0; g < ng; g++, bl += NCH * 32) {
      const T* c0 = coef0 + g * NCH;
      const T* c1 = coef1 + g * NCH;
#pragma unroll
      for (int u0 = 0; u0 < NCH; u0 += VEC) {
        const Vec<T> a0 = *reinterpret_cast<const Vec<T>*>(c0 + u0);
        Vec<T> a1;
        if (NO > 1) a1 = *reinterpret_cast<const Vec<T>*>(c1 + u0);
#pragma unroll
        for (int e = 0; e < VEC; e += 2) {
          const T v0 = bl[(u0 + e) * 32], v1 = bl[(u0 + e + 1) * 32];
          p[0] = ffma2(v0, v1, a0.e[e], a0.e[e + 1], p[0]);
          if (NO > 1) p[NO - 1] = ffma2(v0, v1, a1.e[e], a1.e[e + 1], p[NO - 1]);
        }
      }
    }
#pragma unroll
    for (int o = 0; o < NO; o++) out[o] = p[o].x + p[o].y;
  } else {
    for (int g = 0; g < ng; g++, base += NCH * 32) {
      const T* c0 = coef0 + g * NCH;
      const T* c1 = coef1 + g * NCH;
#pragma unroll
      for (int u0 = 0; u0 < NCH; u0 += VEC) {
        const Vec<T> a0 = *reinterpret_cast<const Vec<T>*>(c0 + u0);
        Vec<T> a1;
        if (NO > 1) a1 = *reinterpret_cast<const Vec<T>*>(c1 + u0);
#pragma unroll
        for (int e = 0; e < VEC; e++) {
          const T v = base[off[u0 + e]];
          out[0] = fma(v, a0.e[e], out[0]);
          if (NO > 1) out[NO - 1] = fma(v, a1.e[e], out[NO - 1]);
        }
      }
    }
  }
  const int rem = ncol - ng * NCH;
  if (rem > 0) {
    const T* c0 = coef0 + ng * NCH;
    const T* c1 = coef1 + ng * NCH;
#pragma unroll
    for (int u = 0; u < NCH; u++) {
      if (u < rem) {
        const T v = (sizeof(T) == 4) ? buf[(ng * NCH + u) * 32 + lane] : base[off[u]];
        out[0] = fma(v, c0[u], out[0]);
        if (NO > 1) out[NO - 1] = fma(v, c1[u], out[NO - 1]);
      }
    }
  }
}

constexpr int kColsPerLane = 8;   // column owner: up to 8 * 32 = 256 columns

// Column owner: acc[r][m] += sum_i V[i, lane + 32 m] rhs_r[i] over the 32 rows, m < 8.
// Step c reads slot coff[c] = (c + lane) mod NCH of the lane's columns (j mod NCH = lane mod
// NCH for every m), so the 8 lanes of a quarter warp read 8 distinct 16-byte bank groups.  In
// FP64 (rotated layout) that slot holds logical chunk c; in FP32 (plain layout) it holds chunk
// coff[c], and the same slot of the right-hand sides is read with it.  acc is in the storage
// type and covers at most kColFlush sub-tiles (wt_flush_cols).
// Columns j0 = lane + 32 m and (TWO) j1 = j0 + 32 of the sub-tile against the right-hand sides.
template <typename T, int NR, bool TWO>
__device__ __forceinline__ void wt_col_pair(const T* buf, int ncol, int m, const int (&coff)[WT<T>::NCH],
                                            const T* rhs0, const T* rhs1, T (&acc)[NR][kColsPerLane]) {
  constexpr int NCH = WT<T>::NCH, VEC = WT<T>::VEC;
  const int lane = threadIdx.x & 31;
  const int j0 = lane + 32 * m, j1 = j0 + 32;
  const bool h1 = TWO && j1 < ncol;
  if (j0 >= ncol) return;
  const T* col0 = buf + j0 * 32;
  const T* col1 = buf + (h1 ? j1 : j0) * 32;
  if constexpr (sizeof(T) == 4) {   // packed FMAs over pairs of rows
    float2 q0[NR], q1[NR];
#pragma unroll
    for (int r = 0; r < NR; r++) {
      q0[r] = make_float2(acc[r][m], 0.f);
      q1[r] = make_float2((TWO && h1) ? acc[r][m + 1] : 0.f, 0.f);
    }
#pragma unroll
    for (int c = 0; c < NCH; c++) {
      const Vec<T> v0 = *reinterpret_cast<const Vec<T>*>(col0 + coff[c]);
      Vec<T> v1;
      if (TWO) v1 = *reinterpret_cast<const Vec<T>*>(col1 + coff[c]);
      const Vec<T> b0 = *reinterpret_cast<const Vec<T>*>(rhs0 + coff[c]);
#pragma unroll
      for (int e = 0; e < VEC; e += 2) {
        q0[0] = ffma2(v0.e[e], v0.e[e + 1], b0.e[e], b0.e[e + 1], q0[0]);
        if (TWO) q1[0] = ffma2(v1.e[e], v1.e[e + 1], b0.e[e], b0.e[e + 1], q1[0]);
      }
      if (NR > 1) {
        const Vec<T> b1 = *reinterpret_cast<const Vec<T>*>(rhs1 + coff[c]);
#pragma unroll
        for (int e = 0; e < VEC; e += 2) {
          q0[NR - 1] = ffma2(v0.e[e], v0.e[e + 1], b1.e[e], b1.e[e + 1], q0[NR - 1]);
          if (TWO) q1[NR - 1] = ffma2(v1.e[e], v1.e[e + 1], b1.e[e], b1.e[e + 1], q1[NR - 1]);
        }
      }
    }
#pragma unroll
    for (int r = 0; r < NR; r++) {
      acc[r][m] = q0[r].x + q0[r].y;
      if (TWO && h1) acc[r][m + 1] = q1[r].x + q1[r].y;
    }
  } else {
    T s0[NR], s1[NR];   // the running sums themselves (no separate add per sub-tile)
#pragma unroll
    for (int r = 0; r < NR; r++) {
      s0[r] = acc[r][m];
      s1[r] = (TWO && h1) ? acc[r][m + 1] : T(0);
    }
#pragma unroll
    for (int c = 0; c < NCH; c++) {
      const Vec<T> v0 = *reinterpret_cast<const Vec<T>*>(col0 + coff[c]);
      Vec<T> v1;
      if (TWO) v1 = *reinterpret_cast<const Vec<T>*>(col1 + coff[c]);
      const Vec<T> b0 = *reinterpret_cast<const Vec<T>*>(rhs0 + c * VEC);
#pragma unroll
      for (int e = 0; e < VEC; e++) {
        s0[0] = fma(v0.e[e], b0.e[e], s0[0]);
        if (TWO) s1[0] = fma(v1.e[e], b0.e[e], s1[0]);
      }
      if (NR > 1) {
        const Vec<T> b1 = *reinterpret_cast<const Vec<T>*>(rhs1 + c * VEC);
#pragma unroll
        for (int e = 0; e < VEC; e++) {
          s0[NR - 1] = fma(v0.e[e], b1.e[e], s0[NR - 1]);
          if (TWO) s1[NR - 1] = fma(v1.e[e], b1.e[e], s1[NR - 1]);
        }
      }
    }
#pragma unroll
    for (int r = 0; r < NR; r++) {
      acc[r][m] = s0[r];
      if (TWO && h1) acc[r][m + 1] = s1[r];
    }
  }
}

// The FP32 column pass (wt_cols in FP32).  Few columns (ncol <= 16): Q = 32 / C lanes per
// column (C = 4, 8 or 16 column slots), lane = j Q + q.  Lane (j, q) takes NCH / Q chunks of
// column j, slot (c + j) mod NCH with c = q D + (i mod D) + 8 (i div D) at step i (D = 8 / Q),
// so that the 8 lanes of every quarter warp read 8 distinct 16-byte bank groups; in the plain
// FP32 layout the slot is the chunk, and the same chunk of the right-hand sides is read with
// it.  Its running sums stay in acc[r][0];
// wt_flush_cols_f32 adds the Q lanes of a column.  (The same scheme as wt_cols_seg, kept apart:
// the FP32 sweeps, bound by instruction issue with 128 registers, lose a few per cent to the
// register allocation that the shared form leads to.)
__device__ __forceinline__ int wt_col_slots_f32(int ncol) {
  return ncol <= 4 ? 4 : (ncol <= 8 ? 8 : (ncol <= 16 ? 16 : 0));
}
template <typename T, int NR, int Q>
__device__ __forceinline__ void wt_cols_grouped_f32(const T* buf, int ncol, const T* rhs0, const T* rhs1,
                                                T (&acc)[NR][kColsPerLane]) {
  constexpr int NCH = WT<T>::NCH, VEC = WT<T>::VEC, S = NCH / Q, D = 8 / Q;
  const int lane = threadIdx.x & 31, j = lane / Q, q = lane % Q;
  if (j >= ncol) return;
  const T* col = buf + j * 32;
  float2 s[NR];   // packed FMAs over pairs of rows
#pragma unroll
  for (int r = 0; r < NR; r++) s[r] = make_float2(acc[r][0], 0.f);
#pragma unroll
  for (int i = 0; i < S; i++) {
    const int c = q * D + (i % D) + 8 * (i / D);
    const int sl = ((c + j) & (NCH - 1)) * VEC;   // plain layout: chunk (c + j) mod NCH
    const Vec<T> v = *reinterpret_cast<const Vec<T>*>(col + sl);
    const Vec<T> b0 = *reinterpret_cast<const Vec<T>*>(rhs0 + sl);
#pragma unroll
    for (int e = 0; e < VEC; e += 2) s[0] = ffma2(v.e[e], v.e[e + 1], b0.e[e], b0.e[e + 1], s[0]);
    if (NR > 1) {
      const Vec<T> b1 = *reinterpret_cast<const Vec<T>*>(rhs1 + sl);
#pragma unroll
      for (int e = 0; e < VEC; e += 2) s[NR - 1] = ffma2(v.e[e], v.e[e + 1], b1.e[e], b1.e[e + 1], s[NR - 1]);
    }
  }
#pragma unroll
  for (int r = 0; r < NR; r++) acc[r][0] = s[r].x + s[r].y;
}

// More than 16 columns: column lane + 32 m in slot m, two per lane while a second one exists
// anywhere in the warp, then one (a partial last group shares the right-hand-side loads of
// the group before it, which issues fewer instructions than tail segments would).
template <typename T, int NR>
__device__ __forceinline__ void wt_cols_f32(const T* buf, int ncol, const T* rhs0, const T* rhs1,
                                        T (&acc)[NR][kColsPerLane]) {
  constexpr int NCH = WT<T>::NCH, VEC = WT<T>::VEC;
  switch (wt_col_slots_f32(ncol)) {   // uniform over the launch
    case 4: wt_cols_grouped_f32<T, NR, 8>(buf, ncol, rhs0, rhs1, acc); return;
    case 8: wt_cols_grouped_f32<T, NR, 4>(buf, ncol, rhs0, rhs1, acc); return;
    case 16: wt_cols_grouped_f32<T, NR, 2>(buf, ncol, rhs0, rhs1, acc); return;
    default: break;
  }
  const int lane = threadIdx.x & 31;
  int coff[NCH];
#pragma unroll
  for (int c = 0; c < NCH; c++) coff[c] = ((c + lane) & (NCH - 1)) * VEC;
#pragma unroll
  for (int m = 0; m < kColsPerLane; m += 2) {
    if (32 * m >= ncol) break;
    if (32 * (m + 1) < ncol)   // warp-uniform
      wt_col_pair<T, NR, true>(buf, ncol, m, coff, rhs0, rhs1, acc);
    else
      wt_col_pair<T, NR, false>(buf, ncol, m, coff, rhs0, rhs1, acc);
  }
}

// The FP64 column pass.  Its layout over ncol columns (uniform over the launch): groups of 32
// columns go one column per lane, column lane + 32 m in acc slot m < mfull.  Up to 16 columns,
// and the ncol mod 32 columns after the whole groups, form instead at most two tail segments of
// C = 4, 8 or 16 column slots each, with Q = 32 / C lanes per column: segment A (columns
// 32 mfull .. + min(rem, 16)) in slot kColsPerLane - 1, segment B (the columns past 16 of a
// longer tail) in slot kColsPerLane - 2.  A tail segment costs C FMA instructions per
// right-hand side and sub-tile, where a partial group of 32 costs 32: the FP64 sweeps are bound
// by the FP64 pipe, which takes a warp's FMA instruction whole however few of its lanes are
// active.  With mfull = 7 and more than 16 tail columns there is no second free slot: the tail
// is then a partial eighth group (its lanes past ncol idle).
struct ColLayout {
  int mfull, ca, cb;
};
__device__ __forceinline__ int wt_col_slots(int ncol) {
  return ncol <= 4 ? 4 : (ncol <= 8 ? 8 : 16);
}
__device__ __forceinline__ ColLayout wt_col_layout(int ncol) {
  const int rem = ncol & 31;
  if (ncol <= 16) return ColLayout{0, ncol > 0 ? wt_col_slots(ncol) : 0, 0};
  if (rem == 0) return ColLayout{ncol >> 5, 0, 0};
  if (rem <= 16) return ColLayout{ncol >> 5, wt_col_slots(rem), 0};
  if ((ncol >> 5) + 2 <= kColsPerLane) return ColLayout{ncol >> 5, 16, wt_col_slots(rem - 16)};
  return ColLayout{(ncol + 31) >> 5, 0, 0};
}

// A tail segment: columns j0 + j, j < nseg <= C = 32 / Q, lane = j Q + q.  Lane (j, q) takes
// NCH / Q chunks of column j, chunk q D + (i mod D) + 8 (i div D) at step i (D = 8 / Q), so
// that the 8 lanes of every quarter warp read 8 distinct 16-byte bank groups (j0 is a multiple
// of 16, so the rotation of column j0 + j is that of column j).  Its running sums stay in
// acc[r][M]; wt_flush_cols adds the Q lanes of a column.
template <typename T, int NR, int Q, int M>
__device__ __forceinline__ void wt_cols_seg(const T* buf, int j0, int nseg, const T* rhs0, const T* rhs1,
                                            T (&acc)[NR][kColsPerLane]) {
  constexpr int NCH = WT<T>::NCH, VEC = WT<T>::VEC, S = NCH / Q, D = 8 / Q;
  const int lane = threadIdx.x & 31, j = lane / Q, q = lane % Q;
  if (j >= nseg) return;
  const T* col = buf + (j0 + j) * 32;
  T s[NR];
#pragma unroll
  for (int r = 0; r < NR; r++) s[r] = acc[r][M];
#pragma unroll
  for (int i = 0; i < S; i++) {
    const int c = q * D + (i % D) + 8 * (i / D);
    const Vec<T> v = *reinterpret_cast<const Vec<T>*>(col + ((c + j) & (NCH - 1)) * VEC);
    const Vec<T> b0 = *reinterpret_cast<const Vec<T>*>(rhs0 + c * VEC);
#pragma unroll
    for (int e = 0; e < VEC; e++) s[0] = fma(v.e[e], b0.e[e], s[0]);
    if (NR > 1) {
      const Vec<T> b1 = *reinterpret_cast<const Vec<T>*>(rhs1 + c * VEC);
#pragma unroll
      for (int e = 0; e < VEC; e++) s[NR - 1] = fma(v.e[e], b1.e[e], s[NR - 1]);
    }
  }
#pragma unroll
  for (int r = 0; r < NR; r++) acc[r][M] = s[r];
}
template <typename T, int NR, int M>
__device__ __forceinline__ void wt_cols_tail(const T* buf, int C, int j0, int nseg, const T* rhs0, const T* rhs1,
                                             T (&acc)[NR][kColsPerLane]) {
  switch (C) {   // uniform over the launch
    case 4: wt_cols_seg<T, NR, 8, M>(buf, j0, nseg, rhs0, rhs1, acc); return;
    case 8: wt_cols_seg<T, NR, 4, M>(buf, j0, nseg, rhs0, rhs1, acc); return;
    default: wt_cols_seg<T, NR, 2, M>(buf, j0, nseg, rhs0, rhs1, acc); return;
  }
}

// Column owner: acc[r][m] += sum_i V[i, lane + 32 m] rhs_r[i] over the 32 rows.  FP32 goes to
// wt_cols_f32; FP64 takes the groups of 32 columns (two per lane while a second group exists),
// then the tail segments of its layout.  Logical chunk c of column j sits at slot (c + j) mod
// NCH, and j mod NCH = lane mod NCH for every m, so the NCH chunk offsets are per-lane
// constants.  acc is in the storage type and covers at most kColFlush sub-tiles
// (wt_flush_cols).
template <typename T, int NR>
__device__ __forceinline__ void wt_cols(const T* buf, int ncol, const T* rhs0, const T* rhs1,
                                        T (&acc)[NR][kColsPerLane]) {
  if constexpr (sizeof(T) == 4) {
    wt_cols_f32<T, NR>(buf, ncol, rhs0, rhs1, acc);
    return;
  }
  constexpr int NCH = WT<T>::NCH, VEC = WT<T>::VEC;
  const ColLayout L = wt_col_layout(ncol);
  const int lane = threadIdx.x & 31;
  if (L.mfull > 0) {
    int coff[NCH];
#pragma unroll
    for (int c = 0; c < NCH; c++) coff[c] = ((c + lane) & (NCH - 1)) * VEC;
#pragma unroll
    for (int m = 0; m < kColsPerLane; m += 2) {
      if (m >= L.mfull) break;
      if (m + 1 < L.mfull)   // warp-uniform
        wt_col_pair<T, NR, true>(buf, ncol, m, coff, rhs0, rhs1, acc);
      else
        wt_col_pair<T, NR, false>(buf, ncol, m, coff, rhs0, rhs1, acc);
    }
  }
  const int rem = ncol - 32 * L.mfull, j0 = 32 * L.mfull;
  if (L.ca) wt_cols_tail<T, NR, kColsPerLane - 1>(buf, L.ca, j0, min(rem, 16), rhs0, rhs1, acc);
  if (L.cb) wt_cols_tail<T, NR, kColsPerLane - 2>(buf, L.cb, j0 + 16, rem - 16, rhs0, rhs1, acc);
}

// The column owners' running sums in the storage type cover at most kColFlush sub-tiles
// (32 kColFlush products, FP32 in the mixed mode); wt_flush_cols then adds them into the
// warp's FP64 sums in shared memory (comb[warp][r][j], zeroed by wt_zero_cols) and clears
// them.  (FP64 adds are scarce on this GPU: one per column and right-hand side every
// kColFlush sub-tiles instead of every sub-tile.)  In the FP64 mode the running sums are
// already FP64 and are flushed once, after the warp's last sub-tile.
constexpr int kColFlush = 4;
template <int NR>
__device__ __forceinline__ void wt_zero_cols(double* comb, int ncolC) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int q = lane; q < NR * ncolC; q += 32) comb[(size_t)warp * NR * ncolC + q] = 0.0;
  __syncwarp();
}
template <typename T>
__device__ __forceinline__ bool wt_flush_due(int it, int count) {
  if (sizeof(T) == 8) return it + 1 == count;
  return (it + 1) % kColFlush == 0 || it + 1 == count;
}
template <typename T, int NR>
__device__ __forceinline__ void wt_flush_cols_f32(T (&acc)[NR][kColsPerLane], double* comb, int ncolC) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int C = wt_col_slots_f32(ncolC);
  if (C) {   // wt_cols_grouped: add the Q = 32 / C lanes of each column (fixed order)
    const int Q = 32 / C, j = lane / Q;
#pragma unroll
    for (int r = 0; r < NR; r++) {
      T v = acc[r][0];
      for (int o = Q >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane % Q == 0 && j < ncolC) comb[((size_t)warp * NR + r) * ncolC + j] += (double)v;
      acc[r][0] = T(0);
    }
    return;
  }
#pragma unroll
  for (int m = 0; m < kColsPerLane; m++) {
    if (32 * m >= ncolC) break;
    const int j = lane + 32 * m;
#pragma unroll
    for (int r = 0; r < NR; r++) {
      if (j < ncolC) comb[((size_t)warp * NR + r) * ncolC + j] += (double)acc[r][m];
      acc[r][m] = T(0);
    }
  }
}

// A tail segment's running sums: add the Q lanes of each column (fixed order), then into comb.
template <typename T, int NR, int M>
__device__ __forceinline__ void wt_flush_seg(T (&acc)[NR][kColsPerLane], double* comb, int ncolC, int C, int j0,
                                             int nseg) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int Q = 32 / C, j = lane / Q;
#pragma unroll
  for (int r = 0; r < NR; r++) {
    T v = acc[r][M];
    for (int o = Q >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane % Q == 0 && j < nseg) comb[((size_t)warp * NR + r) * ncolC + j0 + j] += (double)v;
    acc[r][M] = T(0);
  }
}
template <typename T, int NR>
__device__ __forceinline__ void wt_flush_cols(T (&acc)[NR][kColsPerLane], double* comb, int ncolC) {
  if constexpr (sizeof(T) == 4) {
    wt_flush_cols_f32<T, NR>(acc, comb, ncolC);
    return;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const ColLayout L = wt_col_layout(ncolC);
#pragma unroll
  for (int m = 0; m < kColsPerLane; m++) {
    if (m >= L.mfull) break;
    const int j = lane + 32 * m;
#pragma unroll
    for (int r = 0; r < NR; r++) {
      if (j < ncolC) comb[((size_t)warp * NR + r) * ncolC + j] += (double)acc[r][m];
      acc[r][m] = T(0);
    }
  }
  const int rem = ncolC - 32 * L.mfull, j0 = 32 * L.mfull;
  if (L.ca) wt_flush_seg<T, NR, kColsPerLane - 1>(acc, comb, ncolC, L.ca, j0, min(rem, 16));
  if (L.cb) wt_flush_seg<T, NR, kColsPerLane - 2>(acc, comb, ncolC, L.cb, j0 + 16, rem - 16);
}

// Shared-memory layout of a sweep launch with W warps, each with nb pipeline stages of ncolT
// staged columns and NRV staged row vectors (32 elements each), plus two scratch row vectors
// per warp, two coefficient arrays (padded to 16 bytes) and the W x NR x ncolC FP64 column
// sums.
template <typename T>
struct WtSmem {
  T* stages;         // W * nb * sstride
  T* scratch;        // W * 2 * 32
  T* coef;           // 2 * cpad
  double* comb;      // W * NR * ncolC
  int sstride;       // elements per stage: (ncolT + NRV) * 32
  int ncolT;
  int nb;
  int cpad;
  size_t total;      // bytes of the layout (the launch's dynamic shared memory)
  __device__ size_t bytes() const { return total; }
  __device__ WtSmem(unsigned char* base, int W, int nbuf, int ncolT_, int NRV, int ncolC, int NR) {
    constexpr int VEC = WT<T>::VEC;
    size_t off = 0;
    auto take = [&](size_t bytes) {
      unsigned char* p = base + off;
      off += (bytes + 15) & ~(size_t)15;
      return p;
    };
    ncolT = ncolT_;
    nb = nbuf;
    sstride = (ncolT + NRV) * 32;
    stages = (T*)take((size_t)W * nb * sstride * sizeof(T));
    scratch = (T*)take((size_t)W * 2 * 32 * sizeof(T));
    constexpr int NCH = WT<T>::NCH;
    (void)VEC;
    cpad = (ncolT + NCH - 1) / NCH * NCH;
    coef = (T*)take((size_t)2 * cpad * sizeof(T));
    comb = (double*)take((size_t)W * NR * (ncolC > 0 ? ncolC : 1) * sizeof(double));
    total = off;
  }
  __device__ __forceinline__ T* stage(int warp, int b) const {
    return stages + ((size_t)warp * nb + b) * sstride;
  }
  // staged row vector q of a stage (after the ncolT columns)
  __device__ __forceinline__ T* srow(T* st, int q) const { return st + (size_t)(ncolT + q) * 32; }
  __device__ __forceinline__ T* scr(int warp, int q) const { return scratch + ((size_t)warp * 2 + q) * 32; }
};

// Sum the warps' FP64 column sums (comb, after their last wt_flush_cols) and store this
// CTA's partials part[off_r + j].
template <int NR>
__device__ __forceinline__ void wt_store_cols(double* comb, int ncolC, double* part, const int (&off)[NR]) {
  const int W = blockDim.x >> 5;
  __syncthreads();
  for (int j = threadIdx.x; j < ncolC; j += blockDim.x) {
#pragma unroll
    for (int r = 0; r < NR; r++) {
      double s = 0.0;
      for (int w = 0; w < W; w++) s += comb[((size_t)w * NR + r) * ncolC + j];
      part[off[r] + j] = s;
    }
  }
}

// Draws for a warp's walk, two sub-tiles per Philox round: at even local iterations lane l
// forms the normal pair (2j, 2j+1) of sub-tile it (l < 16) or of sub-tile it + 1 (l >= 16);
// each iteration then hands every lane its row's normal by shuffle.  Rows outside
// [first, dim) get 0; scaled by sigma.
template <typename T>
struct PairDraws {
  T a = T(0), b = T(0);
  // cur0: first row of this iteration's sub-tile; nxt0: first row of the next one (used at
  // even iterations when has_next).
  __device__ __forceinline__ T next(const DrawKey& key, int it, int64_t cur0, int64_t nxt0, bool has_next,
                                    int64_t first, int64_t dim, T sigma) {
    const int lane = threadIdx.x & 31;
    if (!(it & 1)) {
      const int64_t row = ((lane < 16) ? cur0 : nxt0) + 2 * (lane & 15);
      a = b = T(0);
      if ((lane < 16 || has_next) && row + 1 >= first && row < dim) normal_pair(key, (uint64_t)(row >> 1), a, b);
    }
    const int src = ((it & 1) ? 16 : 0) + (lane >> 1);
    const T va = __shfl_sync(0xffffffffu, a, src);
    const T vb = __shfl_sync(0xffffffffu, b, src);
    const T g = (lane & 1) ? vb : va;
    const int64_t r = cur0 + lane;
    return (r >= first && r < dim) ? sigma * g : T(0);
  }
};

// Walk of a warp over its sub-tiles: first sub-tile gw, stride GW.
struct WarpWalk {
  int64_t first, stride, nsub;   // nsub: end of the CTA's sub-tile range
  __device__ WarpWalk(int64_t dim, const CtaCtx& c) {
    const int W = blockDim.x >> 5;
    const int64_t total = (dim + 31) / 32;
    const int64_t s0 = (int64_t)c.local * c.spc;
    first = s0 + (threadIdx.x >> 5);
    stride = W;
    nsub = min(total, s0 + c.spc);
  }
  __device__ __forceinline__ int64_t sub(int it) const { return first + (int64_t)it * stride; }
  __device__ __forceinline__ int count() const {
    return (first < nsub) ? (int)((nsub - 1 - first) / stride + 1) : 0;
  }
};

// Programmatic dependent launch: wait until the preceding kernel of the stream has completed
// and its writes are visible (no-op when launched without the attribute); then allow the next
// kernel to be scheduled.  A kernel triggers only after its own wait, so every kernel that
// starts early knows that everything before its predecessor has completed.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}

// Hand-over between the two phases of the step kernel (k_step), per trial.  The finaliser of
// the trial's update sweep publishes its results with a release store of 1 into the trial's
// step flag; every output-sweep CTA of that trial polls it with acquire loads, at most `limit`
// polls with a short sleep between them (about a second in all).  On expiry the error word
// gets bit 1 and false is returned: the CTA leaves the kernel and the state is poisoned until
// hd_reset, which clears the flags with the election counters.  The output sweep's own
// finaliser clears the flag (every CTA that waits on it has passed by then).
constexpr unsigned kFlagSpins = 1u << 21;
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;\n" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned* step_flag(const Ws& ws) { return ws.cnt + kStepFlagSlot; }
__device__ bool flag_wait(const unsigned* flag, unsigned* err, unsigned limit) {
  __shared__ int s_go;
  if (threadIdx.x == 0) {
    unsigned spins = 0;
    int ok = 1;
    while (ld_acquire_u32(flag) == 0u) {
      if (++spins > limit) {
        ok = 0;
        if (err) atomicOr(err, 2u);
        break;
      }
      __nanosleep(64);
    }
    s_go = ok;
  }
  __syncthreads();
  const bool ok = s_go != 0;
  asm volatile("fence.acq_rel.gpu;\n" ::: "memory");
  __syncthreads();   // s_go is reused by the next wait
  return ok;
}
// Called by every thread of the finalising CTA once its results are written.
__device__ __forceinline__ void flag_release(const Ws& ws) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    st_release_u32(step_flag(ws), 1u);
  }
}

// Gates of the sweeps (wt_pipeline): a stand-alone kernel waits for its predecessor under
// programmatic dependent launch; the step kernel's update phase needs no wait (the launch
// starts after the preceding one has completed) and its output phase waits for the trial's
// flag.
enum GateKind { kGatePdl = 0, kGateNone = 1, kGateFlag = 2 };
template <int G>
__device__ __forceinline__ bool gate_pass(const Ws& ws) {
  if (G == kGatePdl) {
    pdl_wait();
    pdl_trigger();
    return true;
  }
  if (G == kGateNone) return true;
  return flag_wait(step_flag(ws), ws.err, kFlagSpins);
}

// The walk of one warp as an nb-stage cp.async pipeline.  pre(it, stage) issues the copies of
// local sub-tile it that do not depend on the preceding phase (stack columns written by
// earlier launches), post(it, stage) the rest.  The prologue issues pre for the first nb - 1
// stages, then passes the gate (the wait for the preceding phase: the preceding kernel under
// programmatic dependent launch, or the trial's flag inside the step kernel), then issues their
// post part.  setup() runs in every thread of the CTA right after the gate (then one CTA
// barrier): it stages what the preceding phase produced (coefficients).  body(it, stage) runs
// once the stage is complete.  When the gate gives up (false), the copies in flight are
// drained and false is returned without running the walk.
template <typename Gate, typename Pre, typename Setup, typename Post, typename Body>
__device__ __forceinline__ bool wt_pipeline(int count, int nb, Gate&& gate, Pre&& pre, Setup&& setup, Post&& post,
                                            Body&& body) {
  for (int q = 0; q < nb - 1; q++) {
    if (q < count) pre(q, q);
    cp_async_commit();
  }
  if (!gate()) {
    cp_async_wait<0>();
    return false;
  }
  setup();
  __syncthreads();
  for (int q = 0; q < nb - 1; q++)
    if (q < count) post(q, q);
  cp_async_commit();
  for (int it = 0; it < count; it++) {
    const int nxt = it + nb - 1;
    if (nxt < count) {
      pre(nxt, nxt % nb);
      post(nxt, nxt % nb);
    }
    cp_async_commit();
    cp_async_wait_dyn(it + 1 < nb - 1 ? it + 1 : nb - 1);
    __syncwarp();
    body(it, it % nb);
    __syncwarp();
  }
  return true;
}

// ------------------------------------------------------------------------------------
// K1: z = V_D^T x over k_D columns (and, for Ginibre, x . the k_N data-space basis
// columns); last CTA: w = S_D^T z.
template <typename T>
__global__ void __launch_bounds__(kThreads, kSweepCtasPerSm) k_dots(BatchStep<T> bs) {
  CtaCtx cc;
  const int vb = blockIdx.x;
  const StepPlan<T> p = make_plan(bs, bs.d, vb, cc);
  extern __shared__ __align__(16) unsigned char dsm_raw[];
  const int na = p.kD, nb = (p.ens == 0) ? p.kN : 0, nc = na + nb;
  const SweepCfg& cfg = p.c1;
  const int warp = threadIdx.x >> 5;
  WtSmem<T> sm(dsm_raw, blockDim.x >> 5, cfg.nbuf, nc, 1, nc, 1);
  const ColSrc<T> src{(const T*)p.D.V, p.D.ld, na, (const T*)p.Bd, p.ldBd};
  const int64_t dim = p.D.dim;
  T acc[1][kColsPerLane];
#pragma unroll
  for (int m = 0; m < kColsPerLane; m++) acc[0][m] = T(0);
  const WarpWalk ww(dim, cc);
  const int cnt = ww.count();
  const bool xal = ((uintptr_t)p.x & 15u) == 0;   // per-trial offsets may break alignment
  wt_zero_cols<1>(sm.comb, nc);
  wt_pipeline(cnt, cfg.nbuf, [&]() { return gate_pass<kGatePdl>(p.ws); },
      [&](int it, int b) { wt_load_cols(sm.stage(warp, b), src, nc, ww.sub(it) * 32); },
      [&]() {},
      [&](int it, int b) { wt_load_vec(sm.srow(sm.stage(warp, b), 0), p.x, ww.sub(it) * 32, dim, xal); },
      [&](int it, int b) {
        T* st = sm.stage(warp, b);
        wt_cols<T, 1>(st, nc, sm.srow(st, 0), nullptr, acc);
        if (wt_flush_due<T>(it, cnt)) wt_flush_cols<T, 1>(acc, sm.comb, nc);
      });
  const int off[1] = {0};
  wt_store_cols<1>(sm.comb, nc, p.ws.part + (int64_t)cc.local * nc, off);
  if (!reduce_partials(p.ws, 0, nc, cc.local, cc.ncta, p.ws.z)) return;
  __shared__ double zs[kTmaxLimit];
  for (int i = threadIdx.x; i < na; i += blockDim.x) zs[i] = p.ws.z[i];
  __syncthreads();
  // w = S_D^T z: w_j = S[0:j+1, j] . z[0:j+1]
  fin_dots(p.D.S, p.Tm, na, zs, p.ws.w, (double*)dsm_raw, (int64_t)sm.bytes(), p.ws.err);
}

// K2: p = Delta_D (x - V_D w); writes p[k:] as the new column k of V_D; draws g_{t+1}
// (rows > k) into the data stack's buffer; exact V_D^T p[k:] and V_D^T g_{t+1}.
// The sweep of CTA vb of the data space's map.  G: its gate; STEP (inside k_step): the
// finalising CTA releases the trial's step flag once its results are written.
template <typename T, int G, bool STEP, bool FIN_OUT = false>
__device__ __forceinline__ void update_sweep(const BatchStep<T>& bs, int vb, unsigned char* dsm_raw) {
  CtaCtx cc;
  const StepPlan<T> p = make_plan(bs, bs.d, vb, cc);
  __shared__ double red[kWarps * 4];
  const int k = p.kD;
  const SweepCfg& cfg = p.c2;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  WtSmem<T> sm(dsm_raw, blockDim.x >> 5, cfg.nbuf, k, 1, k, 2);
  const ColSrc<T> src{(const T*)p.D.V, p.D.ld, k, nullptr, 0};
  const int64_t dim = p.D.dim;
  T* col = (T*)p.D.V + (int64_t)k * p.D.ld;
  T* gb = (T*)p.D.gbuf;
  const T dconst = (T)p.D.dpre[k];
  T acc[2][kColsPerLane];
#pragma unroll
  for (int m = 0; m < kColsPerLane; m++) acc[0][m] = acc[1][m] = T(0);
  T ex[3] = {T(0), T(0), T(0)};   // p . g_next, ||p[k+1:]||^2, ||g_next[k+2:]||^2
  T* pv = sm.scr(warp, 0);
  T* gv = sm.scr(warp, 1);
  PairDraws<T> draws;
  const WarpWalk ww(dim, cc);
  const int cnt = ww.count();
  const bool xal = ((uintptr_t)p.x & 15u) == 0;   // per-trial offsets may break alignment
  wt_zero_cols<2>(sm.comb, k);
  wt_pipeline(cnt, cfg.nbuf, [&]() { return gate_pass<G>(p.ws); },
      [&](int it, int b) {
        T* st = sm.stage(warp, b);
        const int64_t r0 = ww.sub(it) * 32;
        wt_load_cols(st, src, k, r0);
        wt_load_vec(sm.srow(st, 0), p.x, r0, dim, xal);
      },
      [&]() {   // w comes from the preceding kernel
        for (int j = threadIdx.x; j < sm.cpad; j += blockDim.x) sm.coef[j] = (j < k) ? (T)p.ws.w[j] : T(0);
      },
      [&](int, int) {},
      [&](int it, int b) {
        T* st = sm.stage(warp, b);
        const int64_t r = ww.sub(it) * 32 + lane;
        const bool has_next = it + 1 < cnt;
        const T g = draws.next(p.key_next, it, ww.sub(it) * 32, has_next ? ww.sub(it + 1) * 32 : 0, has_next,
                               (int64_t)k + 1, dim, p.sigma);
        T out[1];
        wt_rows<T, 1>(st, k, sm.coef, nullptr, out);
        const T d = (r < k) ? (T)p.D.dpre[r + 1] : dconst;
        const T pvv = sign_mul(d, sm.srow(st, 0)[lane] - out[0]);
        if (r < dim) {
          if (r < k) {
            p.ws.phead[r] = (double)pvv;
          } else {
            col[r] = pvv;
            if (r == k) p.ws.scal[kPpiv] = (double)pvv;
            else ex[1] = fma(pvv, pvv, ex[1]);
            ex[0] = fma(pvv, g, ex[0]);
          }
          if (r >= (int64_t)k + 2) ex[2] = fma(g, g, ex[2]);
        }
        gb[r] = g;   // the buffer has ld >= 32 * nsub entries
        pv[lane] = (r >= k && r < dim) ? pvv : T(0);
        gv[lane] = g;
        __syncwarp();
        wt_cols<T, 2>(st, k, pv, gv, acc);
        if (wt_flush_due<T>(it, cnt)) wt_flush_cols<T, 2>(acc, sm.comb, k);
      });
  const int P = 2 * k + 3;
  double* part = p.ws.part + (int64_t)cc.local * P;
  const int off[2] = {k + 3, 0};   // p-dots after the three extras, draw dots first
  wt_store_cols<2>(sm.comb, k, part, off);
  block_sum_to<3>(ex, red, part + k, 3);
  double* rr = p.ws.scr(3);
  if (!reduce_partials(p.ws, 1, P, cc.local, cc.ncta, rr)) return;
  if constexpr (FIN_OUT) fin_update_out<T>(p, rr, (double*)dsm_raw, (int)(sm.bytes() / sizeof(double)));
  else fin_update<T>(p, rr, (double*)dsm_raw, (int)(sm.bytes() / sizeof(double)));
  if (STEP) flag_release(p.ws);
}
template <typename T, bool FIN_OUT>
__global__ void __launch_bounds__(kThreads, kSweepCtasPerSm) k_update(BatchStep<T> bs) {
  extern __shared__ __align__(16) unsigned char dsm_raw[];
  update_sweep<T, kGatePdl, false, FIN_OUT>(bs, blockIdx.x, dsm_raw);
}

// Elementwise dynamics of the fused K3 (the same arithmetic as the stand-alone kernel).
template <typename T>
__device__ __forceinline__ T fused_dyn(int kind, T a, T y, T xprev) {
  if (kind == 1) return tanh(y);
  return fma(a, xprev, sign_of(y));
}

// K3 (Haar): y = Delta_N c - V_N w' with c = [p_head; coef g_t[k:]]; appends the random
// reflector column (g_t[k:] with the pivot entry replaced); the next draw (read from the
// data stack's buffer) replaces g_t in this stack's buffer; dots of it with V_N.
// FUSE: instead of storing y, applies the dynamics x_{t+1} = f(y, x_{t-1}) and adds the dots
// of x_{t+1} with V_N and the new column, i.e. the next step's K1 (this stack is the next
// step's data stack), finished by w = S_N^T z in the last CTA.
// The sweep of CTA vb of the output space's map.  G: its gate; STEP (inside k_step, FUSE):
// the finaliser clears the trial's step flag.
template <typename T, bool FUSE, int G, bool STEP, bool FIN_OUT = false>
__device__ __forceinline__ bool out_haar_sweep(const BatchStep<T>& bs, int vb, unsigned char* dsm_raw) {
  CtaCtx cc;
  const StepPlan<T> p = make_plan(bs, 1 - bs.d, vb, cc);
  __shared__ double red[kWarps * 4];
  const int k = p.kN;
  const SweepCfg& cfg = p.c3;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // FUSE (the next step is the other product): the next draw's dots with this stack and its
  // copy into this stack's buffer are not needed (the next step's kernels redo or overwrite
  // them); the column pass forms the dots of x_{t+1} instead
  WtSmem<T> sm(dsm_raw, blockDim.x >> 5, cfg.nbuf, k, 2, k, 1);
  const ColSrc<T> src{(const T*)p.N.V, p.N.ld, k, nullptr, 0};
  const int64_t dim = p.N.dim;
  T* col = (T*)p.N.V + (int64_t)k * p.N.ld;
  T* gcur = (T*)p.N.gbuf;
  const T* gnext = (const T*)p.D.gbuf;
  T coef = T(0), alpha = T(0), usg = T(0), dconst = T(0);
  bool flag = false;
  T acc[1][kColsPerLane];
#pragma unroll
  for (int m = 0; m < kColsPerLane; m++) acc[0][m] = T(0);
  T ex[1] = {T(0)};   // new column . g_{t+1}, or (FUSE) new column . x_{t+1}
  T* xv = sm.scr(warp, 0);
  const bool need_prev = FUSE && p.dyn != 1;
  const WarpWalk ww(dim, cc);
  const int cnt = ww.count();
  const int64_t ld = p.N.ld;
  wt_zero_cols<1>(sm.comb, k);
  const bool gate_ok = wt_pipeline(cnt, cfg.nbuf, [&]() { return gate_pass<G>(p.ws); },
      [&](int it, int b) {
        T* st = sm.stage(warp, b);
        const int64_t r0 = ww.sub(it) * 32;
        wt_load_cols(st, src, k, r0);
        wt_load_vec(sm.srow(st, 0), (const T*)gcur, r0, ld, true);
        if (need_prev) wt_load_vec(sm.srow(st, 1), p.xprev, r0, dim, ((uintptr_t)p.xprev & 15u) == 0);
      },
      [&]() {   // outputs of the preceding kernel's finalisation
        for (int j = threadIdx.x; j < sm.cpad; j += blockDim.x) sm.coef[j] = (j < k) ? (T)p.ws.wout[j] : T(0);
        coef = (T)p.ws.scal[kCoef];
        alpha = (T)p.ws.scal[kAlpha];
        usg = (T)p.ws.scal[kUpivG];
        flag = p.ws.scal[kGFlag] != 0.0;
        dconst = (T)p.N.dpre[k];
      },
      [&](int it, int b) {
        if (!FUSE) wt_load_vec(sm.srow(sm.stage(warp, b), 1), gnext, ww.sub(it) * 32, ld, true);
      },
      [&](int it, int b) {
        T* st = sm.stage(warp, b);
        const int64_t r = ww.sub(it) * 32 + lane;
        const T g = sm.srow(st, 0)[lane];
        T out[1];
        wt_rows<T, 1>(st, k, sm.coef, nullptr, out);
        T ci;
        if (r < k) ci = (T)p.ws.phead[r];
        else if (flag) ci = (r == k) ? alpha : T(0);
        else ci = coef * g;
        const T d = (r < k) ? (T)p.N.dpre[r + 1] : dconst;
        const T yi = sign_mul(d, ci) - out[0];
        const T nc = (r > k) ? g : ((r == k) ? usg : T(0));
        if (r < dim) {
          if (!FUSE) p.y[r] = yi;
          if (r >= k) col[r] = nc;
        }
        if (FUSE) {
          T xn = T(0);
          if (r < dim) {
            xn = fused_dyn<T>(p.dyn, p.dyn_a, yi, need_prev ? sm.srow(st, 1)[lane] : T(0));
            if (p.yrec) p.yrec[r] = yi;
            if (p.xrec) p.xrec[r] = xn;
            if (p.xgiven) xn = p.xgiven[r];
            p.xnext[r] = xn;
          }
          xv[lane] = xn;
          ex[0] = fma(nc, xn, ex[0]);
          __syncwarp();
          wt_cols<T, 1>(st, k, xv, nullptr, acc);
          __syncwarp();
        } else {
          const T gn = sm.srow(st, 1)[lane];
          ex[0] = fma(nc, gn, ex[0]);
          gcur[r] = gn;
          wt_cols<T, 1>(st, k, sm.srow(st, 1), nullptr, acc);
        }
        if (wt_flush_due<T>(it, cnt)) wt_flush_cols<T, 1>(acc, sm.comb, k);
      });
  if (!gate_ok) return false;
  // partial sums: [0, k) V_N . r, [k] new column . r, r = g_{t+1} or (FUSE) x_{t+1}
  const int P = k + 1;
  double* part = p.ws.part + (int64_t)cc.local * P;
  const int off[1] = {0};
  wt_store_cols<1>(sm.comb, k, part, off);
  block_sum_to<1>(ex, red, part + k, 1);
  double* rr = p.ws.scr(3);
  if (!reduce_partials(p.ws, 2, P, cc.local, cc.ncta, rr)) return true;
  if (STEP && threadIdx.x == 0) *step_flag(p.ws) = 0u;   // every waiter of the trial has passed
  if (!FUSE) {
    for (int j = threadIdx.x; j <= k; j += blockDim.x) p.N.gdot[j] = rr[j];
    if (threadIdx.x == 0) p.N.gg[0] = p.D.gg[0];
  } else {
    // the next step's K1: z = V_N^T x_{t+1} over the k + 1 columns, w = S_N^T z
    __shared__ double zs[kTmaxLimit + 1];
    for (int j = threadIdx.x; j <= k; j += blockDim.x) {
      zs[j] = rr[j];
      p.ws.z[j] = rr[j];
    }
    __syncthreads();
    if constexpr (FIN_OUT) fin_dots_out(p.N.S, p.Tm, k + 1, zs, p.ws.w, (double*)dsm_raw, (int64_t)sm.bytes(), p.ws.err);
    else fin_dots(p.N.S, p.Tm, k + 1, zs, p.ws.w, (double*)dsm_raw, (int64_t)sm.bytes(), p.ws.err);
  }
  return true;
}
template <typename T, bool FUSE, bool FIN_OUT = false>
__global__ void __launch_bounds__(kThreads, kSweepCtasPerSm) k_out_haar(BatchStep<T> bs) {
  extern __shared__ __align__(16) unsigned char dsm_raw[];
  out_haar_sweep<T, FUSE, kGatePdl, false, FIN_OUT>(bs, blockIdx.x, dsm_raw);
}

// K3 (Ginibre): u = Delta_N g - V_N w_2 (= L_1..L_l Z_{1:l} g), y = alpha u + Delta_N h
// - V_N w_h + B_n c; u becomes the new basis column; the next draw (rows >= k_N) replaces g
// in this stack's buffer, with its dots with V_N.
// FUSE: applies the dynamics instead of storing y and adds the next step's K1: the dots of
// x_{t+1} with V_N (the next data stack) and with B_n including u (the next step's data-space
// basis), then w = S_N^T z in the last CTA.
// The sweep of CTA vb of the output space's map (G, STEP as for out_haar_sweep).
template <typename T, bool FUSE, int G, bool STEP, bool FIN_OUT = false>
__device__ __forceinline__ bool out_gin_sweep(const BatchStep<T>& bs, int vb, unsigned char* dsm_raw) {
  CtaCtx cc;
  const StepPlan<T> p = make_plan(bs, 1 - bs.d, vb, cc);
  __shared__ double red[kWarps * 4];
  const int kN = p.kN, kD = p.kD, nc = kN + kD;
  const SweepCfg& cfg = p.c3;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // FUSE (the next step is the other product): the next draw in this space and its dots are
  // not needed; the column pass forms the dots of x_{t+1} with V_N and B_n instead
  const int ncc = FUSE ? nc : kN;   // column-owner columns
  WtSmem<T> sm(dsm_raw, blockDim.x >> 5, cfg.nbuf, nc, FUSE ? 3 : 1, ncc, 1);
  const bool ista = FUSE && p.dyn == 5;
  const bool amp = FUSE && (p.dyn == 4 || ista);
  const int amode = amp ? p.amp_mode : 0;
  const ColSrc<T> src{(const T*)p.N.V, p.N.ld, kN, (const T*)p.Bn, p.ldBn};
  const int64_t dim = p.N.dim;
  T* ucol = (T*)p.Bn + (int64_t)kD * p.ldBn;
  T* gcur = (T*)p.N.gbuf;
  const double* h = p.ws.z + kD;
  T alpha = T(0), dconst = T(0);
  T acc[1][kColsPerLane];
#pragma unroll
  for (int m = 0; m < kColsPerLane; m++) acc[0][m] = T(0);
  T ex[2] = {T(0), T(0)};   // (FUSE) u . x_{t+1}; (AMP) ||z||^2 or ||x||_0 of this CTA's rows
  T* rv = sm.scr(warp, 0);
  const bool need_prev = FUSE && !amp && p.dyn != 1;
  T amp_s = T(0);   // (AMP) threshold (mode 2) or Onsager factor (mode 3) of this trial
  PairDraws<T> draws;
  const WarpWalk ww(dim, cc);
  const int cnt = ww.count();
  const int64_t ld = p.N.ld;
  wt_zero_cols<1>(sm.comb, ncc);
  const bool gate_ok = wt_pipeline(cnt, cfg.nbuf, [&]() { return gate_pass<G>(p.ws); },
      [&](int it, int b) {
        T* st = sm.stage(warp, b);
        const int64_t r0 = ww.sub(it) * 32;
        wt_load_cols(st, src, nc, r0);
        wt_load_vec(sm.srow(st, 0), (const T*)gcur, r0, ld, true);
        if (need_prev) wt_load_vec(sm.srow(st, 1), p.xprev, r0, dim, ((uintptr_t)p.xprev & 15u) == 0);
        if (amode == 1) wt_load_vec(sm.srow(st, 1), p.amp_w, r0, dim, ((uintptr_t)p.amp_w & 15u) == 0);
        if (amode == 2 || amode == 3)
          wt_load_vec(sm.srow(st, 1), (const T*)p.amp_v, r0, dim, ((uintptr_t)p.amp_v & 15u) == 0);
        if (amode == 3) wt_load_vec(sm.srow(st, 2), (const T*)p.amp_y, r0, dim, ((uintptr_t)p.amp_y & 15u) == 0);
      },
      [&]() {   // outputs of the preceding kernel's finalisation
        if (amode == 2 || amode == 3) {
          const double mi = (double)bs.desc[cc.trial].st[1].dim;
          if (ista) amp_s = (amode == 2) ? p.dyn_a : T(0);
          else amp_s = (amode == 2) ? (T)(p.dyn_a * sqrt(p.amp_zsq[cc.trial] / mi)) : (T)((double)p.amp_nnz[cc.trial] / mi);
        }
        for (int j = threadIdx.x; j < sm.cpad; j += blockDim.x) {
          T c0 = T(0), c1 = T(0);
          if (j < kN) {
            c0 = (T)p.ws.wout2[j];
            c1 = (T)p.ws.wout[j];
          } else if (j < nc) {
            c1 = -(T)p.ws.phead[j - kN];
          }
          sm.coef[j] = c0;
          sm.coef[sm.cpad + j] = c1;
        }
        alpha = (T)p.ws.scal[kAlpha];
        dconst = (T)p.N.dpre[kN];
      },
      [&](int, int) {},
      [&](int it, int b) {
        T* st = sm.stage(warp, b);
        const int64_t r = ww.sub(it) * 32 + lane;
        const T g = sm.srow(st, 0)[lane];
        const T hi = (r < kN) ? (T)h[r] : T(0);
        T out[2];
        wt_rows<T, 2>(st, nc, sm.coef, sm.coef + sm.cpad, out);
        const T d = (r < kN) ? (T)p.N.dpre[r + 1] : dconst;
        const T u = sign_mul(d, g) - out[0];
        const T yi = fma(alpha, u, sign_mul(d, hi)) - out[1];
        if (r < dim) {
          ucol[r] = u;
          if (!FUSE) p.y[r] = yi;
        }
        if (FUSE) {
          T xn = T(0);
          if (r < dim) {
            if (amode == 1) {          // y = Q beta + w; z = y
              xn = yi + sm.srow(st, 1)[lane];
              p.amp_y[r] = xn;
            } else if (amode == 2) {   // x = eta(x + tau Q^T z; theta), tau = 1 for AMP
              const T v = fma(p.amp_tau, yi, sm.srow(st, 1)[lane]);
              const T m = fabs(v) - amp_s;
              xn = (m > T(0)) ? copysign(m, v) : T(0);
            } else if (amode == 3) {   // z = y - Q x + z ||x||_0 / m (AMP; the factor is 0 for ISTA)
              xn = fma(sm.srow(st, 1)[lane], amp_s, sm.srow(st, 2)[lane] - yi);
            } else {
              xn = fused_dyn<T>(p.dyn, p.dyn_a, yi, need_prev ? sm.srow(st, 1)[lane] : T(0));
            }
            if (p.yrec) p.yrec[r] = yi;
            if (p.xrec) p.xrec[r] = xn;
            if (p.xgiven) xn = p.xgiven[r];
            if (amp) {
              p.amp_v[r] = xn;
              ex[1] = (amode == 2) ? ex[1] + ((xn != T(0)) ? T(1) : T(0)) : fma(xn, xn, ex[1]);
            } else {
              p.xnext[r] = xn;
            }
          }
          rv[lane] = xn;
          ex[0] = fma(u, xn, ex[0]);
        } else {
          const bool has_next = it + 1 < cnt;
          const T gn = draws.next(p.key_next, it, ww.sub(it) * 32, has_next ? ww.sub(it + 1) * 32 : 0, has_next,
                                  (int64_t)kN, dim, p.sigma);
          gcur[r] = gn;
          rv[lane] = gn;
        }
        __syncwarp();
        wt_cols<T, 1>(st, ncc, rv, nullptr, acc);
        __syncwarp();
        if (wt_flush_due<T>(it, cnt)) wt_flush_cols<T, 1>(acc, sm.comb, ncc);
      });
  if (!gate_ok) return false;
  if (!FUSE && kN == 0) return true;   // no dots to form
  // partial sums: [0, ncc) columns . r (r = g_{t+1}, or (FUSE) x_{t+1}), (FUSE) [nc] u . x_{t+1}
  const int P = FUSE ? nc + 1 + (amp ? 1 : 0) : kN;
  double* part = p.ws.part + (int64_t)cc.local * P;
  const int off[1] = {0};
  wt_store_cols<1>(sm.comb, ncc, part, off);
  if (FUSE) block_sum_to<2>(ex, red, part + nc, amp ? 2 : 1);
  double* rr = p.ws.scr(3);
  if (!reduce_partials(p.ws, 2, P, cc.local, cc.ncta, rr)) return true;
  if (STEP && threadIdx.x == 0) *step_flag(p.ws) = 0u;   // every waiter of the trial has passed
  if (!FUSE) {
    for (int j = threadIdx.x; j < kN; j += blockDim.x) p.N.gdot[j] = rr[j];
  } else {
    // the next step's K1 (its data stack is V_N, k_D' = kN; its data-space basis is B_n with
    // kD + 1 columns): z = V_N^T x_{t+1}, h = B_n^T x_{t+1}, w = S_N^T z
    __shared__ double zs[kTmaxLimit + 1];
    for (int j = threadIdx.x; j < kN; j += blockDim.x) {
      zs[j] = rr[j];
      p.ws.z[j] = rr[j];
    }
    for (int i = threadIdx.x; i <= kD; i += blockDim.x) p.ws.z[kN + i] = (i < kD) ? rr[kN + i] : rr[nc];
    if (amp && threadIdx.x == 0) {   // the trial's AMP scalar for the following steps
      if (amode == 2) p.amp_nnz[cc.trial] = (int)(rr[nc + 1] + 0.5);
      else p.amp_zsq[cc.trial] = rr[nc + 1];
    }
    __syncthreads();
    if constexpr (FIN_OUT) fin_dots_out(p.N.S, p.Tm, kN, zs, p.ws.w, (double*)dsm_raw, (int64_t)sm.bytes(), p.ws.err);
    else fin_dots(p.N.S, p.Tm, kN, zs, p.ws.w, (double*)dsm_raw, (int64_t)sm.bytes(), p.ws.err);
  }
  return true;
}
template <typename T, bool FUSE, bool FIN_OUT = false>
__global__ void __launch_bounds__(kThreads, kSweepCtasPerSm) k_out_gin(BatchStep<T> bs) {
  extern __shared__ __align__(16) unsigned char dsm_raw[];
  out_gin_sweep<T, FUSE, kGatePdl, false, FIN_OUT>(bs, blockIdx.x, dsm_raw);
}

// ------------------------------------------------------------------------------------
// The step kernel: one launch per step of a fused trajectory (K2, then the fused K3).  It
// runs as a cooperative launch, so all its CTAs are resident at once.  Each CTA takes virtual
// CTAs of the data space's map through the update sweep, then virtual CTAs of the output
// space's map through the fused output sweep: first its own index, then (when a map has more
// CTAs than the launch) the next free index from a queue, as the hardware scheduler hands out
// the CTAs of a multi-wave launch; the fetch of the next index is issued before the current
// one's work, so its latency is hidden.  The update phase never waits.  A trial's output CTAs
// wait only for that trial's update finaliser (its step flag), after prefetching their first
// stages; that finaliser is the trial's last update CTA to arrive, so every flag is released
// once the update phase has run everywhere, and the per-trial flags let a trial's output
// sweep start while other trials still update.  Queues are taken in trial order, so the
// trials finalised first are the ones the output phase asks for first.  The last CTA to finish
// clears the queues for the next launch.
template <typename T, bool HAAR>
__global__ void __launch_bounds__(kThreads, kSweepCtasPerSm) k_step(BatchStep<T> bs) {
  extern __shared__ __align__(16) unsigned char dsm_raw[];
  __shared__ int s_next;
  const int n2 = bs.map[bs.d].ctas, n3 = bs.map[1 - bs.d].ctas;
  const int G = (int)gridDim.x;
  unsigned* q = bs.desc[0].ws.cnt + kStepQueueSlot;   // [0]: update queue, [1]: output queue, [2]: CTAs done
  const bool queued = n2 > G || n3 > G;
  int v = blockIdx.x;
  while (v < n2) {
    int nxt = n2;
    if (threadIdx.x == 0 && n2 > G) nxt = G + (int)atomicAdd(&q[0], 1u);
    update_sweep<T, kGateNone, true>(bs, v, dsm_raw);
    if (n2 <= G) break;
    if (threadIdx.x == 0) s_next = nxt;
    __syncthreads();   // also: the next virtual CTA reuses the shared memory
    v = s_next;
    __syncthreads();
  }
  __syncthreads();
  bool ok = true;
  v = blockIdx.x;
  while (v < n3) {
    int nxt = n3;
    if (threadIdx.x == 0 && n3 > G) nxt = G + (int)atomicAdd(&q[1], 1u);
    if constexpr (HAAR) ok = out_haar_sweep<T, true, kGateFlag, true>(bs, v, dsm_raw);
    else ok = out_gin_sweep<T, true, kGateFlag, true>(bs, v, dsm_raw);
    if (!ok || n3 <= G) break;   // (!ok: the flag wait expired, error word set)
    if (threadIdx.x == 0) s_next = nxt;
    __syncthreads();
    v = s_next;
    __syncthreads();
  }
  if (queued && threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&q[2], 1u) == (unsigned)G - 1u) {   // every CTA has left both queues
      q[0] = 0u;
      q[1] = 0u;
      q[2] = 0u;
    }
  }
}

// ------------------------------------------------------------------------------------
template <typename T>
cudaError_t launch_first_draw(const BatchStep<T>& b, int space, DrawKey key, cudaStream_t s) {
  k_first_draw<T><<<b.map[space].ctas, kThreads, 0, s>>>(b, space, key);
  return cudaGetLastError();
}

// Launch with programmatic stream serialisation (the kernel may start while its predecessor
// drains; it synchronises through griddepcontrol.wait) when pdl is set.
template <typename T>
cudaError_t launch_sweep(void (*kern)(BatchStep<T>), const SweepCfg& c, int ctas, size_t smem,
                         cudaStream_t s, bool pdl, const BatchStep<T>& b) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)ctas);
  cfg.blockDim = dim3((unsigned)(32 * c.W));
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = pdl ? attr : nullptr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, b);
}

template <typename T>
cudaError_t launch_step(const BatchStep<T>& b, cudaStream_t s, cudaEvent_t* ev, int* launched) {
  auto rec = [&](int i) {
    if (!ev || !ev[i]) return;
    // inside a stream capture the record becomes an event-record node of the graph (the
    // External flag); outside a capture that flag is not allowed
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) cs = cudaStreamCaptureStatusNone;
    if (cs == cudaStreamCaptureStatusActive)
      cudaEventRecordWithFlags(ev[i], s, cudaEventRecordExternal);
    else
      cudaEventRecord(ev[i], s);
  };
  const StepPlan<T>& p = b.base;
  const bool pdl = p.pdl != 0;
  const int dspace = b.d, ospace = 1 - b.d;
  cudaError_t e = cudaSuccess;
  const int nc1 = p.kD + ((p.ens == 0) ? p.kN : 0);
  if (nc1 > 0 && !p.skip_dots) {
    rec(0);
    // no early launch: its prologue copies the newest stack and basis columns, which the
    // previous step's output sweep may still be writing when the two steps follow each
    // other directly on the stream
    e = launch_sweep<T>(k_dots<T>, p.c1, b.map[dspace].ctas,
                        sweep_smem_bytes<T>(p.c1.W, p.c1.nbuf, nc1, 1, nc1, 1), s, false, b);
    if (e != cudaSuccess) return e;
    rec(1);
    if (launched) launched[0] = 1;
  }
  if (p.step_ctas > 0) {   // K2 and the fused K3 in one cooperative launch
    rec(2);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)p.step_ctas);
    cfg.blockDim = dim3((unsigned)(32 * p.c2.W));
    cfg.dynamicSmemBytes = (size_t)p.step_smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = (p.ens == 1) ? cudaLaunchKernelEx(&cfg, k_step<T, true>, b) : cudaLaunchKernelEx(&cfg, k_step<T, false>, b);
    if (e != cudaSuccess) return e;
    rec(3);
    if (launched) launched[1] = 2;
    return cudaGetLastError();
  }
  rec(2);
  // K2 prefetches x and its stack columns before waiting for the preceding kernel.  That
  // kernel is K1 or, at step 1, the first-draw kernel: both start only after everything
  // before them on the stream has completed, so x and the older columns are final.  After a
  // fused K3 (which writes x and the newest column) K2 is launched without the early start
  e = launch_sweep<T>(p.fin_out ? k_update<T, true> : k_update<T, false>, p.c2, b.map[dspace].ctas,
                      sweep_smem_bytes<T>(p.c2.W, p.c2.nbuf, p.kD, 1, p.kD, 2), s, pdl && !p.skip_dots, b);
  if (e != cudaSuccess) return e;
  rec(3);
  if (launched) launched[1] = 1;
  rec(4);
  const int ncg = p.kN + p.kD;
  if (p.ens == 1 && p.fuse)
    e = launch_sweep<T>(p.fin_out ? k_out_haar<T, true, true> : k_out_haar<T, true>, p.c3, b.map[ospace].ctas,
                        sweep_smem_bytes<T>(p.c3.W, p.c3.nbuf, p.kN, 2, p.kN, 1), s, pdl, b);
  else if (p.ens == 1)
    e = launch_sweep<T>(k_out_haar<T, false>, p.c3, b.map[ospace].ctas,
                        sweep_smem_bytes<T>(p.c3.W, p.c3.nbuf, p.kN, 2, p.kN, 1), s, pdl, b);
  else if (p.fuse)
    e = launch_sweep<T>(p.fin_out ? k_out_gin<T, true, true> : k_out_gin<T, true>, p.c3, b.map[ospace].ctas,
                        sweep_smem_bytes<T>(p.c3.W, p.c3.nbuf, ncg, 3, ncg, 1), s, pdl, b);
  else
    e = launch_sweep<T>(k_out_gin<T, false>, p.c3, b.map[ospace].ctas,
                        sweep_smem_bytes<T>(p.c3.W, p.c3.nbuf, ncg, 1, p.kN, 1), s, pdl, b);
  if (e != cudaSuccess) return e;
  rec(5);
  if (launched) launched[2] = 1;
  return cudaGetLastError();
}

template <typename T>
cudaError_t set_sweep_smem_limit(int bytes) {
  cudaError_t e = cudaSuccess;
  auto one = [&](const void* fn) {
    cudaFuncAttributes fa;
    cudaError_t r = cudaFuncGetAttributes(&fa, fn);
    if (r == cudaSuccess)
      r = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               bytes - (int)fa.sharedSizeBytes);
    if (r != cudaSuccess) e = r;
  };
  one((const void*)k_dots<T>);
  one((const void*)k_update<T, false>);
  one((const void*)k_update<T, true>);
  one((const void*)k_out_haar<T, false>);
  one((const void*)k_out_gin<T, false>);
  one((const void*)k_out_haar<T, true>);
  one((const void*)k_out_gin<T, true>);
  one((const void*)k_out_haar<T, true, true>);
  one((const void*)k_out_gin<T, true, true>);
  one((const void*)k_step<T, true>);
  one((const void*)k_step<T, false>);
  return e;
}
template cudaError_t set_sweep_smem_limit<float>(int);
template cudaError_t set_sweep_smem_limit<double>(int);

template <typename T>
int kernel_static_smem(int which) {
  cudaFuncAttributes fa;
  cudaError_t e = cudaErrorInvalidValue;
  switch (which) {
    case 0: e = cudaFuncGetAttributes(&fa, k_dots<T>); break;
    case 1: e = cudaFuncGetAttributes(&fa, k_update<T, false>); break;
    case 2: e = cudaFuncGetAttributes(&fa, k_out_haar<T, false>); break;
    case 3: e = cudaFuncGetAttributes(&fa, k_out_gin<T, false>); break;
    case 4: e = cudaFuncGetAttributes(&fa, k_out_haar<T, true>); break;
    default: e = cudaFuncGetAttributes(&fa, k_out_gin<T, true>); break;
  }
  return (e == cudaSuccess) ? (int)fa.sharedSizeBytes : 8192;
}
template int kernel_static_smem<float>(int);
template int kernel_static_smem<double>(int);

template <typename T>
int kernel_occupancy(int which, size_t dynsmem) {
  int nb = 0;
  cudaError_t e = cudaSuccess;
  switch (which) {
    case 0: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_dots<T>, kThreads, dynsmem); break;
    case 1: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_update<T, false>, kThreads, dynsmem); break;
    case 2: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_out_haar<T, false>, kThreads, dynsmem); break;
    case 3: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_out_gin<T, false>, kThreads, dynsmem); break;
    case 4: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_out_haar<T, true>, kThreads, dynsmem); break;
    default: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_out_gin<T, true>, kThreads, dynsmem); break;
  }
  return (e == cudaSuccess && nb > 0) ? nb : 1;
}
template int kernel_occupancy<float>(int, size_t);
template int kernel_occupancy<double>(int, size_t);

template <typename T>
int step_kernel_occupancy(bool haar, int threads, size_t dynsmem) {
  int nb = 0;
  const cudaError_t e = haar ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_step<T, true>, threads, dynsmem)
                             : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_step<T, false>, threads, dynsmem);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return nb;
}
template int step_kernel_occupancy<float>(bool, int, size_t);
template int step_kernel_occupancy<double>(bool, int, size_t);

template cudaError_t launch_first_draw<float>(const BatchStep<float>&, int, DrawKey, cudaStream_t);
template cudaError_t launch_first_draw<double>(const BatchStep<double>&, int, DrawKey, cudaStream_t);
template cudaError_t launch_step<float>(const BatchStep<float>&, cudaStream_t, cudaEvent_t*, int*);
template cudaError_t launch_step<double>(const BatchStep<double>&, cudaStream_t, cudaEvent_t*, int*);

// ------------------------------------------------------------------------------------
// Consistency probe (not on the hot path): y = Q^(t) x from the revealed part only.
//   q = H_{k_D-1}...H_0 x = Delta_D (x - V_D w)  (w = S_D^T V_D^T x from k_dots);
//   unrevealed = ||q[k_D:]||;
//   Haar:    y = B_N [q[:t]; 0]              (eq. H_t: the hidden block never sees q[:t])
//   Ginibre: y = B_N [h; 0] + B_n q[:k_D]    (h = x . data-space basis), eq. Gaussian_t.
template <typename T>
__device__ __forceinline__ StepPlan<T> trial0_plan(const BatchStep<T>& b) {
  const TrialDesc& td = b.desc[0];
  StepPlan<T> p = b.base;
  p.D = td.st[b.d];
  p.N = td.st[1 - b.d];
  p.Bd = td.basis[b.d];
  p.ldBd = td.ldb[b.d];
  p.Bn = td.basis[1 - b.d];
  p.ldBn = td.ldb[1 - b.d];
  p.ws = td.ws;
  return p;
}

template <typename T>
__global__ void __launch_bounds__(256) k_probe_q(BatchStep<T> b, double* q, double* unrev) {
  const StepPlan<T> p = trial0_plan(b);
  // row pass in the storage type, as the sweeps' row passes; four independent chains
  __shared__ T wsh[kTmaxLimit];
  const int k = p.kD;
  for (int j = threadIdx.x; j < k; j += blockDim.x) wsh[j] = (T)p.ws.w[j];
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double u2 = 0.0;
  if (i < p.D.dim) {
    const T* V = (const T*)p.D.V + i;
    const int64_t ld = p.D.ld;
    T a0 = p.x[i], a1 = T(0), a2 = T(0), a3 = T(0);
    int j = 0;
    for (; j + 4 <= k; j += 4) {
      a0 = fma(-V[(int64_t)j * ld], wsh[j], a0);
      a1 = fma(-V[(int64_t)(j + 1) * ld], wsh[j + 1], a1);
      a2 = fma(-V[(int64_t)(j + 2) * ld], wsh[j + 2], a2);
      a3 = fma(-V[(int64_t)(j + 3) * ld], wsh[j + 3], a3);
    }
    for (; j < k; j++) a0 = fma(-V[(int64_t)j * ld], wsh[j], a0);
    const double acc = (double)((a0 + a1) + (a2 + a3));
    const double d = (k == 0) ? 1.0 : ((i < k) ? p.D.dpre[i + 1] : p.D.dpre[k]);
    q[i] = d * acc;
    if (i >= k) u2 = q[i] * q[i];
  }
  u2 = warp_sum(u2);
  if ((threadIdx.x & 31) == 0) atomicAdd(unrev, u2);
}

template <typename T>
__global__ void k_probe_coef(BatchStep<T> b, const double* q) {
  const StepPlan<T> p = trial0_plan(b);
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
__global__ void __launch_bounds__(256) k_probe_out(BatchStep<T> b, const double* q) {
  const StepPlan<T> p = trial0_plan(b);
  // row passes in the storage type, as the sweeps' row passes; independent chains per column block
  __shared__ T wsh[kTmaxLimit], qsh[kTmaxLimit];
  const int kN = p.kN;
  const int kB = (p.ens == 0) ? p.kD : 0;
  for (int j = threadIdx.x; j < kN; j += blockDim.x) wsh[j] = (T)p.ws.wout[j];
  for (int j = threadIdx.x; j < kB; j += blockDim.x) qsh[j] = (T)q[j];
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= p.N.dim) return;
  const T* VN = (const T*)p.N.V + i;
  const int64_t ld = p.N.ld;
  const double* c = (p.ens == 1) ? q : p.ws.z + p.kD;
  const double d = (kN == 0) ? 1.0 : ((i < kN) ? p.N.dpre[i + 1] : p.N.dpre[kN]);
  T a0 = (i < kN) ? (T)(d * c[i]) : T(0), a1 = T(0), a2 = T(0), a3 = T(0);
  int j = 0;
  for (; j + 4 <= kN; j += 4) {
    a0 = fma(-VN[(int64_t)j * ld], wsh[j], a0);
    a1 = fma(-VN[(int64_t)(j + 1) * ld], wsh[j + 1], a1);
    a2 = fma(-VN[(int64_t)(j + 2) * ld], wsh[j + 2], a2);
    a3 = fma(-VN[(int64_t)(j + 3) * ld], wsh[j + 3], a3);
  }
  for (; j < kN; j++) a0 = fma(-VN[(int64_t)j * ld], wsh[j], a0);
  if (kB > 0) {
    const T* Bn = (const T*)p.Bn + i;
    for (j = 0; j < kB; j++) a1 = fma(Bn[(int64_t)j * p.ldBn], qsh[j], a1);
  }
  p.y[i] = (a0 + a1) + (a2 + a3);
}

template <typename T>
cudaError_t launch_probe(const BatchStep<T>& b, double* q, double* unrev, cudaStream_t s) {
  const StepPlan<T>& p = b.base;
  const int nc1 = p.kD + ((p.ens == 0) ? p.kN : 0);
  cudaError_t e = cudaSuccess;
  if (nc1 > 0)
    e = launch_sweep<T>(k_dots<T>, p.c1, b.map[b.d].ctas,
                        sweep_smem_bytes<T>(p.c1.W, p.c1.nbuf, nc1, 1, nc1, 1), s, false, b);
  if (e != cudaSuccess) return e;
  const int thr = 256;
  const int64_t dD = b.map[b.d].ctas > 0 ? p.D.dim : 0, dN = p.N.dim;
  k_probe_q<T><<<(unsigned)((dD + thr - 1) / thr), thr, 0, s>>>(b, q, unrev);
  k_probe_coef<T><<<1, thr, 0, s>>>(b, q);
  k_probe_out<T><<<(unsigned)((dN + thr - 1) / thr), thr, 0, s>>>(b, q);
  return cudaGetLastError();
}
template cudaError_t launch_probe<float>(const BatchStep<float>&, double*, double*, cudaStream_t);
template cudaError_t launch_probe<double>(const BatchStep<double>&, double*, double*, cudaStream_t);

// ------------------------------------------------------------------------------------
// Check of the bounded-wait path: one staging round that posts 16 expected bytes and issues
// no copy, so the wait runs out after `limit` polls, sets the error word and returns (no copy
// is ever in flight on the abandoned barrier).
// Both bounded waits, made to expire: a staging barrier whose copies are never issued, then
// a step flag that nothing releases (err[2], a word of the error block that stays zero).
__global__ void k_wait_selftest(unsigned* err, unsigned limit) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) mbar_init(&bar);
  Stager sg{&bar, 0u, err, limit};
  sg.run(16u, []() {});
  flag_wait(err + 2, err, limit);
}

cudaError_t launch_wait_selftest(unsigned* err, unsigned limit, cudaStream_t s) {
  k_wait_selftest<<<1, 64, 0, s>>>(err, limit);
  return cudaGetLastError();
}

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
