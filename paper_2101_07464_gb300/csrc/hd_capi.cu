// Host side of libhd.so: the hd_state, its device memory, launch shapes, and the C ABI
// declared in include/hd.h.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/hd.h"
#include "hd_dynamics.cuh"
#include "hd_kernels.cuh"

using namespace hd;

struct hd_state {
  int ens = 0, dtype = 0;
  int64_t m = 0, n = 0;
  int Tm = 0;
  uint64_t seed = 0;
  uint32_t trial = 0;
  double sigma = 1.0;
  cudaStream_t stream = nullptr;
  int device = 0;
  int t = 0, r = 0, l = 0;
  int drawn = 0;         // first draws made since create/reset
  int poisoned = 0;      // sticky error code
  size_t esz = 8;        // element size of vectors and stacks
  StackDev st[2];        // 0: R (acts on R^n), 1: L (acts on R^m)
  void* basis[2] = {nullptr, nullptr};  // Ginibre: 0 = Q^T-step v_i (n-space), 1 = Q-step u_i (m-space)
  int64_t ldb[2] = {0, 0};
  Ws ws;
  Grid grid[2];          // launch shape for each space (0: n, 1: m)
  int nsm = 1;
  int pdl = 1;           // programmatic dependent launch of the sweeps (HD_DISABLE_PDL=1: off)
  int occ_regs[4] = {1, 1, 1, 1};  // CTAs per SM allowed by registers: K1, K2, K3 Haar, K3 Gin
  int static_smem[4] = {0, 0, 0, 0};  // static shared memory of each sweep kernel
  int smem_sm = 0;       // shared memory per SM usable by CTAs
  int smem_blk_max = 0;  // opt-in dynamic shared memory per CTA
  int64_t bytes = 0;
  void* allocs[40];
  int nalloc = 0;
  // hd_run: work vectors and the cached trajectory graph
  void* xw[2] = {nullptr, nullptr};
  void* yw = nullptr;
  double* sumsq = nullptr;
  int run_final = 0;
  cudaStream_t own_stream = nullptr;
  cudaGraphExec_t gexec = nullptr;
  std::vector<uint8_t> g_flags;
  int g_T = 0, g_dyn = 0;
  double g_a = 0.0, g_sigma = 0.0;
  uint64_t g_seed = 0;
  uint32_t g_trial = 0;
  cudaStream_t g_stream = nullptr;
  int g_final = 0;
  int g_launches = 0;
  int g_prof = 0;
  // kernel launches issued (graph replays count the captured launches)
  int64_t launches = 0;
  // profiling: event pairs around each sweep, algorithmic bytes of each recorded launch
  int prof_on = 0;
  int prof_cap = 0;
  int prof_used = 0;
  std::vector<cudaEvent_t> prof_ev;   // 2 per slot
  std::vector<int> prof_kind;
  std::vector<double> prof_bytes;
  double prof_ms[3] = {0, 0, 0};
  int64_t prof_n[3] = {0, 0, 0};
  double prof_b[3] = {0, 0, 0};
};

namespace {

thread_local char g_last_error[256] = "";

void set_error(const char* where, cudaError_t e) {
  snprintf(g_last_error, sizeof(g_last_error), "%s: %s", where, cudaGetErrorString(e));
}

int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

int cuda_fail(hd_state* st, cudaError_t e) {
  set_error("kernel launch", e);
  if (st) st->poisoned = HD_ERR_CUDA;
  return HD_ERR_CUDA;
}

void* dalloc(hd_state* st, size_t bytes) {
  void* p = nullptr;
  if (bytes == 0) bytes = 16;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  st->allocs[st->nalloc++] = p;
  st->bytes += (int64_t)bytes;
  return p;
}

void free_all(hd_state* st) {
  for (int i = 0; i < st->nalloc; i++) cudaFree(st->allocs[i]);
  st->nalloc = 0;
}

Grid make_grid(int64_t dim, int vec, int occ, int nsm) {
  Grid g;
  const int64_t nvec = (dim + vec - 1) / vec;
  const int64_t cap = (int64_t)kThreads * kChunkMax;
  int64_t ctas = std::max<int64_t>((nvec + cap - 1) / cap,
                                   std::min<int64_t>((int64_t)occ * nsm, (nvec + kThreads - 1) / kThreads));
  if (ctas < 1) ctas = 1;
  g.vpc = (nvec + ctas - 1) / ctas;
  ctas = (nvec + g.vpc - 1) / g.vpc;
  g.ctas = (int)ctas;
  int gs = (int)std::ceil(std::sqrt((double)ctas));
  if (gs < 1) gs = 1;
  g.gsize = gs;
  g.ngroups = (int)((ctas + gs - 1) / gs);
  return g;
}

DrawKey key_for(const hd_state* st, int step) {
  DrawKey k;
  k.k0 = (uint32_t)(st->seed & 0xFFFFFFFFu);
  k.k1 = (uint32_t)(st->seed >> 32);
  k.step = (uint32_t)step;
  k.trial = st->trial;
  k.stream = 0;
  return k;
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

template <typename T>
int first_draws(hd_state* st) {
  const T sigma = (st->ens == HD_GINIBRE) ? (T)st->sigma : T(1);
  for (int s = 0; s < 2; s++) {
    cudaError_t e = launch_first_draw<T>(st->st[s], 0, key_for(st, 1), sigma, st->ws, 0,
                                         st->grid[s], st->stream);
    if (e != cudaSuccess) return cuda_fail(st, e);
  }
  st->drawn = 1;
  return HD_OK;
}

// Launch shape of a tiled sweep over ncol columns of a dim-row stack: the largest tile
// height R in {256, 128, 64, 32} whose two-stage footprint leaves room for two CTAs per
// SM; else one CTA per SM with two stages; else one stage.  Persistent grid of
// min(tiles, resident CTAs).
// Launch shape of a sweep over ncolT staged columns and NRV staged row vectors (ncolC
// column-owner columns, NR right-hand sides) of a dim-row stack: the (warps per CTA, pipeline
// stages per warp) pair that puts the most bytes in flight per SM (capped at 128 KB; then
// more resident warps, then fewer stages), and a persistent grid of min(sub-tile groups,
// resident CTAs).
template <typename T>
SweepCfg make_sweep(const hd_state* st, int which, int ncolT, int NRV, int ncolC, int NR, int64_t dim) {
  SweepCfg c;
  c.W = 8;
  c.nbuf = 1;
  const int stat = st->static_smem[which] + 1024;   // static + per-CTA reserve
  const int blk = st->smem_blk_max - stat;
  const double stage = (double)(ncolT + NRV) * 32.0 * sizeof(T);
  double best = -1.0;
  for (int W = 8; W >= 1; W /= 2) {
    for (int nb = 1; nb <= 8; nb *= 2) {
      const size_t b = sweep_smem_bytes<T>(W, nb, ncolT, NRV, ncolC, NR);
      if ((int)b > blk) continue;
      const int by_regs = std::max(1, st->occ_regs[which] * 8 / W);
      const int ctas = std::min(by_regs, (int)(st->smem_sm / (b + stat)));
      if (ctas < 1) continue;
      const int warps = std::min(64, ctas * W);
      const double inflight = std::min(warps * nb * stage, 131072.0);
      const double score = inflight * 1e4 + warps * 10.0 - nb;
      if (score > best) {
        best = score;
        c.W = W;
        c.nbuf = nb;
      }
    }
  }
  const size_t bytes = sweep_smem_bytes<T>(c.W, c.nbuf, ncolT, NRV, ncolC, NR);
  const int by_regs = std::max(1, st->occ_regs[which] * 8 / c.W);
  const int occ = std::max(1, std::min(by_regs, (int)(st->smem_sm / (bytes + stat))));
  const int64_t nsub = (dim + 31) / 32;
  int64_t ctas = std::min<int64_t>((nsub + c.W - 1) / c.W, (int64_t)occ * st->nsm);
  if (ctas < 1) ctas = 1;
  c.g.ctas = (int)ctas;
  c.g.vpc = 0;
  c.g.gsize = std::max(1, (int)std::ceil(std::sqrt((double)ctas)));
  c.g.ngroups = (int)((ctas + c.g.gsize - 1) / c.g.gsize);
  return c;
}

template <typename T>
void set_sweeps(const hd_state* st, StepPlan<T>* p) {
  const int nc1 = p->kD + ((p->ens == 0) ? p->kN : 0);
  p->c1 = make_sweep<T>(st, 0, nc1, 1, nc1, 1, p->D.dim);
  p->c2 = make_sweep<T>(st, 1, p->kD, 1, p->kD, 2, p->D.dim);
  if (p->ens == 1)
    p->c3 = make_sweep<T>(st, 2, p->kN, 2, p->kN, 1, p->N.dim);
  else
    p->c3 = make_sweep<T>(st, 3, p->kN + p->kD, 1, p->kN, 1, p->N.dim);
}

template <typename T>
int do_step(hd_state* st, const void* x, int transpose, void* y) {
  if (!st->drawn) {
    int rc = first_draws<T>(st);
    if (rc) return rc;
  }
  const int d = transpose ? 1 : 0;  // data-side stack: R for Q, L for Q^T
  StepPlan<T> p;
  p.ens = st->ens;
  p.Tm = st->Tm;
  const int cnt[2] = {st->r, st->l};
  if (st->ens == HD_HAAR) {
    p.kD = p.kN = st->t;
  } else {
    p.kD = cnt[d];
    p.kN = cnt[1 - d];
  }
  p.D = st->st[d];
  p.N = st->st[1 - d];
  p.Bd = st->basis[d];
  p.ldBd = st->ldb[d];
  p.Bn = st->basis[1 - d];
  p.ldBn = st->ldb[1 - d];
  p.x = (const T*)x;
  p.xal = aligned16(x);
  p.y = (T*)y;
  p.yal = aligned16(y);
  p.ws = st->ws;
  p.key_next = key_for(st, st->t + 2);
  p.sigma = (st->ens == HD_GINIBRE) ? (T)st->sigma : T(1);
  set_sweeps<T>(st, &p);
  p.pdl = st->pdl;
  cudaEvent_t ev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  int slot0 = -1;
  if (st->prof_on && st->prof_used + 3 <= st->prof_cap) {
    slot0 = st->prof_used;
    for (int q = 0; q < 3; q++) {
      ev[2 * q] = st->prof_ev[2 * (slot0 + q)];
      ev[2 * q + 1] = st->prof_ev[2 * (slot0 + q) + 1];
    }
  }
  int launched[3] = {0, 0, 0};
  cudaError_t e = launch_step<T>(p, st->stream, ev, launched);
  if (e != cudaSuccess) return cuda_fail(st, e);
  st->launches += launched[0] + launched[1] + launched[2];
  if (slot0 >= 0) {
    // algorithmic bytes: each sweep reads its stack once plus its vectors
    const double es = (double)sizeof(T);
    const double nD = (double)p.D.dim, nN = (double)p.N.dim;
    const double bd = (st->ens == HD_GINIBRE) ? (double)p.kN * nD : 0.0;  // data-space basis
    const double bn = (st->ens == HD_GINIBRE) ? (double)(p.kD + 1) * nN : 0.0;
    const double b[3] = {es * (nD * p.kD + bd + nD),
                         es * (nD * p.kD + 3.0 * nD),
                         es * (nN * p.kN + bn + 4.0 * nN)};
    for (int q = 0; q < 3; q++) {
      st->prof_kind[slot0 + q] = launched[q] ? q : -1;
      st->prof_bytes[slot0 + q] = b[q];
    }
    st->prof_used += 3;
  }
  st->t += 1;
  if (transpose) st->l += 1; else st->r += 1;
  return HD_OK;
}

template <typename T>
int do_probe(hd_state* st, const void* x, int transpose, void* y, double* unrevealed_host) {
  const int d = transpose ? 1 : 0;
  StepPlan<T> p;
  p.ens = st->ens;
  p.Tm = st->Tm;
  const int cnt[2] = {st->r, st->l};
  if (st->ens == HD_HAAR) {
    p.kD = p.kN = st->t;
  } else {
    p.kD = cnt[d];
    p.kN = cnt[1 - d];
  }
  p.D = st->st[d];
  p.N = st->st[1 - d];
  p.Bd = st->basis[d];
  p.ldBd = st->ldb[d];
  p.Bn = st->basis[1 - d];
  p.ldBn = st->ldb[1 - d];
  p.x = (const T*)x;
  p.xal = aligned16(x);
  p.y = (T*)y;
  p.yal = aligned16(y);
  p.ws = st->ws;
  p.sigma = T(1);
  set_sweeps<T>(st, &p);
  p.pdl = 0;
  double* q = nullptr;
  if (cudaMalloc(&q, (size_t)(p.D.dim + 1) * 8) != cudaSuccess) {
    set_error("hd_probe cudaMalloc", cudaGetLastError());
    return HD_ERR_OOM;
  }
  double* unrev = q + p.D.dim;
  cudaError_t e = cudaMemsetAsync(unrev, 0, 8, st->stream);
  if (e == cudaSuccess) e = launch_probe<T>(p, q, unrev, st->stream);
  double u2 = 0.0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&u2, unrev, 8, cudaMemcpyDeviceToHost, st->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st->stream);
  cudaFree(q);
  if (e != cudaSuccess) return cuda_fail(st, e);
  *unrevealed_host = std::sqrt(u2);
  return HD_OK;
}

template <typename T>
int run_steps(hd_state* st, const hd_run_spec* sp) {
  if (st->prof_on) st->prof_used = 0;
  st->t = st->r = st->l = 0;
  st->drawn = 0;
  int cur = 0;
  for (int t = 0; t < sp->T; t++) {
    const int tr = sp->transpose[t] ? 1 : 0;
    int rc = do_step<T>(st, st->xw[cur], tr, st->yw);
    if (rc) return rc;
    const int64_t nout = tr ? st->n : st->m;
    cudaError_t e = launch_dynamics<T>(sp->dynamics, sp->a, (const T*)st->yw, (const T*)st->xw[cur],
                                       (const T*)st->xw[1 - cur], (T*)st->xw[1 - cur], nout,
                                       st->sumsq, st->stream, st->pdl != 0);
    if (e != cudaSuccess) return cuda_fail(st, e);
    st->launches += (sp->dynamics == HD_DYN_NORM_TANH) ? 2 : 1;
    cur = 1 - cur;
  }
  st->run_final = cur;
  return HD_OK;
}

bool graph_matches(const hd_state* st, const hd_run_spec* sp) {
  if (!st->gexec || st->g_T != sp->T || st->g_dyn != sp->dynamics || st->g_a != sp->a) return false;
  if (st->g_seed != st->seed || st->g_trial != st->trial || st->g_sigma != st->sigma) return false;
  if (st->g_stream != st->stream || st->g_prof != st->prof_on) return false;
  for (int t = 0; t < sp->T; t++)
    if (st->g_flags[t] != (sp->transpose[t] ? 1 : 0)) return false;
  return true;
}

}  // namespace

extern "C" {

HD_API int hd_run(hd_state* st, const hd_run_spec* sp, const void* x1, void* x_out) {
  if (!st || !sp || !sp->transpose || !x1 || !x_out) return HD_ERR_ARG;
  if (st->poisoned) return st->poisoned;
  if (sp->T < 1 || sp->T > st->Tm) return HD_ERR_TMAX;
  if (sp->dynamics != HD_DYN_TANH && sp->dynamics != HD_DYN_SIGN_MEM && sp->dynamics != HD_DYN_NORM_TANH)
    return HD_ERR_ARG;
  if (!std::isfinite(sp->a)) return HD_ERR_ARG;
  // dimensions: input of step t+1 = output of step t; x_{t-1} (sign_mem) matches y_t
  for (int t = 0; t + 1 < sp->T; t++) {
    const int64_t out_t = sp->transpose[t] ? st->n : st->m;
    const int64_t in_next = sp->transpose[t + 1] ? st->m : st->n;
    if (out_t != in_next) return HD_ERR_DIM;
  }
  if (cudaSetDevice(st->device) != cudaSuccess) return cuda_fail(st, cudaErrorInvalidDevice);
  const int64_t dmax = std::max(st->m, st->n);
  if (!st->yw) {
    const int64_t ld = round_up(dmax, 64);
    st->xw[0] = dalloc(st, (size_t)ld * st->esz);
    st->xw[1] = dalloc(st, (size_t)ld * st->esz);
    st->yw = dalloc(st, (size_t)ld * st->esz);
    st->sumsq = (double*)dalloc(st, 64);
    if (!st->xw[0] || !st->xw[1] || !st->yw || !st->sumsq) return HD_ERR_OOM;
  }
  const int64_t nin = sp->transpose[0] ? st->m : st->n;
  const int64_t nfin = sp->transpose[sp->T - 1] ? st->n : st->m;
  cudaError_t e = cudaMemcpyAsync(st->xw[0], x1, (size_t)nin * st->esz, cudaMemcpyDefault, st->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(st->xw[1], 0, (size_t)dmax * st->esz, st->stream);
  if (e != cudaSuccess) {
    set_error("hd_run input copy", e);
    return cuda_fail(st, e);
  }
  int rc = HD_OK;
  if (sp->use_graph) {
    if (!graph_matches(st, sp)) {
      if (st->gexec) {
        cudaGraphExecDestroy(st->gexec);
        st->gexec = nullptr;
      }
      cudaStream_t user = st->stream;
      cudaStream_t cap = user;
      if (!cap) {
        if (!st->own_stream && cudaStreamCreateWithFlags(&st->own_stream, cudaStreamNonBlocking) != cudaSuccess)
          return cuda_fail(st, cudaGetLastError());
        cap = st->own_stream;
        // order the capture stream after the input copies on the legacy stream
        if (cudaStreamSynchronize(user) != cudaSuccess) return cuda_fail(st, cudaGetLastError());
      }
      cudaGraph_t graph = nullptr;
      e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) {
        set_error("cudaStreamBeginCapture", e);
        return cuda_fail(st, e);
      }
      st->stream = cap;
      const int64_t l0 = st->launches;
      rc = (st->dtype == HD_F64) ? run_steps<double>(st, sp) : run_steps<float>(st, sp);
      st->g_launches = (int)(st->launches - l0);
      st->launches = l0;
      st->stream = user;
      e = cudaStreamEndCapture(cap, &graph);
      if (rc) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
      }
      if (e == cudaSuccess) e = cudaGraphInstantiate(&st->gexec, graph, 0);
      if (graph) cudaGraphDestroy(graph);
      if (e != cudaSuccess) {
        set_error("graph capture", e);
        st->gexec = nullptr;
        return cuda_fail(st, e);
      }
      st->g_T = sp->T;
      st->g_dyn = sp->dynamics;
      st->g_a = sp->a;
      st->g_seed = st->seed;
      st->g_trial = st->trial;
      st->g_sigma = st->sigma;
      st->g_stream = st->stream;
      st->g_flags.assign(sp->transpose, sp->transpose + sp->T);
      for (auto& f : st->g_flags) f = f ? 1 : 0;
      st->g_final = st->run_final;
      st->g_prof = st->prof_on;
    }
    e = cudaGraphLaunch(st->gexec, st->stream);
    if (e != cudaSuccess) {
      set_error("cudaGraphLaunch", e);
      return cuda_fail(st, e);
    }
    st->launches += st->g_launches;
    st->t = sp->T;
    st->r = st->l = 0;
    for (int t = 0; t < sp->T; t++) (sp->transpose[t] ? st->l : st->r) += 1;
    st->drawn = 1;
    st->run_final = st->g_final;
  } else {
    rc = (st->dtype == HD_F64) ? run_steps<double>(st, sp) : run_steps<float>(st, sp);
    if (rc) return rc;
  }
  e = cudaMemcpyAsync(x_out, st->xw[st->run_final], (size_t)nfin * st->esz, cudaMemcpyDefault, st->stream);
  if (e != cudaSuccess) {
    set_error("hd_run output copy", e);
    return cuda_fail(st, e);
  }
  return HD_OK;
}


HD_API const char* hd_last_error(void) { return g_last_error; }

HD_API const char* hd_status_string(int status) {
  switch (status) {
    case HD_OK: return "HD_OK";
    case HD_ERR_ARG: return "HD_ERR_ARG: invalid argument";
    case HD_ERR_DIM: return "HD_ERR_DIM: invalid dimensions";
    case HD_ERR_TMAX: return "HD_ERR_TMAX: step limit exceeded";
    case HD_ERR_OOM: return "HD_ERR_OOM: device allocation failed";
    case HD_ERR_CUDA: return "HD_ERR_CUDA: CUDA error";
    case HD_ERR_TIMEOUT: return "HD_ERR_TIMEOUT: device wait expired";
    case HD_ERR_STATE: return "HD_ERR_STATE: state poisoned by an earlier error";
    default: return "unknown status";
  }
}

HD_API int hd_create(int ensemble, int64_t m, int64_t n, int32_t T_max, uint64_t seed, int dtype,
                     hd_state** out) {
  if (!out) return HD_ERR_ARG;
  *out = nullptr;
  if (ensemble != HD_GINIBRE && ensemble != HD_HAAR) return HD_ERR_ARG;
  if (dtype != HD_F64 && dtype != HD_F32) return HD_ERR_ARG;
  if (m <= 0 || n <= 0) return HD_ERR_DIM;
  if (ensemble == HD_HAAR && m != n) return HD_ERR_DIM;
  if (m > ((int64_t)1 << 40) || n > ((int64_t)1 << 40)) return HD_ERR_DIM;
  if (T_max <= 0) return HD_ERR_TMAX;
  if (ensemble == HD_GINIBRE && T_max > std::min(m, n)) return HD_ERR_TMAX;
  if (ensemble == HD_HAAR && T_max > n) return HD_ERR_TMAX;
  if (T_max > kTmaxLimit) return HD_ERR_TMAX;

  hd_state* st = new (std::nothrow) hd_state();
  if (!st) return HD_ERR_OOM;
  st->ens = ensemble;
  st->dtype = dtype;
  st->m = m;
  st->n = n;
  st->Tm = T_max;
  st->seed = seed;
  st->esz = (dtype == HD_F64) ? 8 : 4;
  if (cudaGetDevice(&st->device) != cudaSuccess) {
    set_error("cudaGetDevice", cudaGetLastError());
    delete st;
    return HD_ERR_CUDA;
  }
  int nsm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, st->device);
  if (nsm <= 0) nsm = 1;
  st->nsm = nsm;
  {
    const char* env = getenv("HD_DISABLE_PDL");
    st->pdl = (env && env[0] == '1') ? 0 : 1;
  }
  int smem_sm = 0, smem_blk = 0;
  cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, st->device);
  cudaDeviceGetAttribute(&smem_blk, cudaDevAttrMaxSharedMemoryPerBlockOptin, st->device);
  st->smem_sm = smem_sm;
  st->smem_blk_max = smem_blk;
  {
    const size_t need = (dtype == HD_F64) ? sweep_smem_bytes<double>(1, 1, T_max, 2, T_max, 2)
                                          : sweep_smem_bytes<float>(1, 1, T_max, 2, T_max, 2);
    if ((int)need > smem_blk - 1024) {
      delete st;
      return HD_ERR_TMAX;
    }
    cudaError_t e = (dtype == HD_F64) ? set_sweep_smem_limit<double>(smem_blk - 1024)
                                      : set_sweep_smem_limit<float>(smem_blk - 1024);
    if (e != cudaSuccess) {
      set_error("cudaFuncSetAttribute", e);
      cudaGetLastError();
      delete st;
      return HD_ERR_CUDA;
    }
  }
  const int vec = (dtype == HD_F64) ? 2 : 4;
  int occ;
  const size_t dsm = (size_t)3 * T_max * st->esz;
  (void)dsm;
  for (int q = 0; q < 4; q++) {
    st->occ_regs[q] = (dtype == HD_F64) ? kernel_occupancy<double>(q, 0) : kernel_occupancy<float>(q, 0);
    st->static_smem[q] = (dtype == HD_F64) ? kernel_static_smem<double>(q) : kernel_static_smem<float>(q);
  }
  occ = 4;
  const int64_t dims[2] = {n, m};
  int64_t maxctas = (int64_t)nsm * 8;
  for (int s = 0; s < 2; s++) {
    st->grid[s] = make_grid(dims[s], vec, occ, nsm);
    maxctas = std::max<int64_t>(maxctas, st->grid[s].ctas);
    if (st->grid[s].ngroups > kMaxGroups) {
      delete st;
      return HD_ERR_DIM;
    }
  }
  const int64_t Tm = T_max;
  bool ok = true;
  for (int s = 0; s < 2 && ok; s++) {
    StackDev& X = st->st[s];
    X.dim = dims[s];
    X.ld = round_up(dims[s], 256);
    X.V = dalloc(st, (size_t)X.ld * Tm * st->esz);
    X.S = (double*)dalloc(st, (size_t)Tm * Tm * 8);
    X.dpre = (double*)dalloc(st, (size_t)(Tm + 1) * 8);
    X.gbuf = dalloc(st, (size_t)X.ld * st->esz);
    X.gdot = (double*)dalloc(st, (size_t)(Tm + 1) * 8);
    X.gg = (double*)dalloc(st, 8);
    ok = X.V && X.S && X.dpre && X.gbuf && X.gdot && X.gg;
    if (ok && ensemble == HD_GINIBRE) {
      st->ldb[s] = X.ld;
      st->basis[s] = dalloc(st, (size_t)X.ld * Tm * st->esz);
      ok = st->basis[s] != nullptr;
    }
  }
  const int64_t stride = Tm + 8;
  if (ok) {
    Ws& w = st->ws;
    w.z = (double*)dalloc(st, (size_t)(2 * Tm + 8) * 8);
    w.w = (double*)dalloc(st, (size_t)stride * 8);
    w.phead = (double*)dalloc(st, (size_t)stride * 8);
    w.wout = (double*)dalloc(st, (size_t)stride * 8);
    w.wout2 = (double*)dalloc(st, (size_t)stride * 8);
    w.scr_stride = 2 * Tm + 8;
    w.scrb = (double*)dalloc(st, (size_t)4 * w.scr_stride * 8);
    w.scal = (double*)dalloc(st, (size_t)kNumScal * 8);
    w.part = (double*)dalloc(st, (size_t)maxctas * (2 * Tm + 8) * 8);
    w.gpart = (double*)dalloc(st, (size_t)kMaxGroups * (2 * Tm + 8) * 8);
    w.cnt = (unsigned int*)dalloc(st, (size_t)3 * (kMaxGroups + 1) * sizeof(unsigned int));
    w.err = (unsigned int*)dalloc(st, 16);
    ok = w.z && w.w && w.phead && w.wout && w.wout2 && w.scrb && w.scal && w.part &&
         w.gpart && w.cnt && w.err;
  }
  if (!ok) {
    free_all(st);
    delete st;
    return HD_ERR_OOM;
  }
  // Zero everything (reflector columns must be zero above their pivot; padding rows zero).
  bool zok = true;
  for (int s = 0; s < 2 && zok; s++) {
    StackDev& X = st->st[s];
    zok = cudaMemset(X.V, 0, (size_t)X.ld * Tm * st->esz) == cudaSuccess &&
          cudaMemset(X.gbuf, 0, (size_t)X.ld * st->esz) == cudaSuccess &&
          cudaMemset(X.S, 0, (size_t)Tm * Tm * 8) == cudaSuccess &&
          cudaMemset(X.gdot, 0, (size_t)(Tm + 1) * 8) == cudaSuccess;
    if (zok && st->basis[s]) zok = cudaMemset(st->basis[s], 0, (size_t)st->ldb[s] * Tm * st->esz) == cudaSuccess;
    const double one = 1.0;
    if (zok) zok = cudaMemcpy(X.dpre, &one, 8, cudaMemcpyHostToDevice) == cudaSuccess;
  }
  if (zok) zok = cudaMemset(st->ws.cnt, 0, (size_t)3 * (kMaxGroups + 1) * sizeof(unsigned int)) == cudaSuccess;
  if (zok) zok = cudaMemset(st->ws.err, 0, 16) == cudaSuccess;
  if (zok) zok = cudaMemset(st->ws.scal, 0, kNumScal * 8) == cudaSuccess;
  if (zok) zok = cudaDeviceSynchronize() == cudaSuccess;
  if (!zok) {
    set_error("hd_create initialisation", cudaGetLastError());
    free_all(st);
    delete st;
    return HD_ERR_CUDA;
  }
  *out = st;
  return HD_OK;
}

HD_API int hd_set_options(hd_state* st, double sigma, uint32_t trial, void* stream) {
  if (!st) return HD_ERR_ARG;
  if (!(sigma > 0.0) || !std::isfinite(sigma)) return HD_ERR_ARG;
  if (st->t > 0 && (sigma != st->sigma || trial != st->trial)) return HD_ERR_ARG;
  st->sigma = sigma;
  st->trial = trial;
  st->stream = (cudaStream_t)stream;
  return HD_OK;
}

HD_API int hd_apply(hd_state* st, const void* x, int transpose, void* y) {
  if (!st || !x || !y) return HD_ERR_ARG;
  if (transpose != 0 && transpose != 1) return HD_ERR_ARG;
  if (st->poisoned) return st->poisoned;
  if (st->t >= st->Tm) return HD_ERR_TMAX;
  if (cudaSetDevice(st->device) != cudaSuccess) return cuda_fail(st, cudaErrorInvalidDevice);
  return (st->dtype == HD_F64) ? do_step<double>(st, x, transpose, y)
                               : do_step<float>(st, x, transpose, y);
}

HD_API int hd_probe(hd_state* st, const void* x, int transpose, void* y, double* unrevealed_host) {
  if (!st || !x || !y || !unrevealed_host) return HD_ERR_ARG;
  if (transpose != 0 && transpose != 1) return HD_ERR_ARG;
  if (st->poisoned) return st->poisoned;
  if (cudaSetDevice(st->device) != cudaSuccess) return cuda_fail(st, cudaErrorInvalidDevice);
  return (st->dtype == HD_F64) ? do_probe<double>(st, x, transpose, y, unrevealed_host)
                               : do_probe<float>(st, x, transpose, y, unrevealed_host);
}

HD_API int hd_profile_enable(hd_state* st, int on) {
  if (!st) return HD_ERR_ARG;
  if (on && st->prof_cap == 0) {
    const int slots = 3 * st->Tm;
    st->prof_ev.assign(2 * slots, nullptr);
    for (auto& ev : st->prof_ev)
      if (cudaEventCreate(&ev) != cudaSuccess) {
        set_error("cudaEventCreate", cudaGetLastError());
        return HD_ERR_CUDA;
      }
    st->prof_kind.assign(slots, -1);
    st->prof_bytes.assign(slots, 0.0);
    st->prof_cap = slots;
  }
  st->prof_on = on ? 1 : 0;
  st->prof_used = 0;
  return HD_OK;
}

HD_API int hd_profile_read(hd_state* st, double* ms3, int64_t* launches3, double* bytes3, int clear) {
  if (!st) return HD_ERR_ARG;
  if (st->prof_used > 0) {
    if (cudaStreamSynchronize(st->stream) != cudaSuccess) return cuda_fail(st, cudaGetLastError());
    for (int s = 0; s < st->prof_used; s++) {
      const int q = st->prof_kind[s];
      if (q < 0) continue;
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, st->prof_ev[2 * s], st->prof_ev[2 * s + 1]) != cudaSuccess) {
        set_error("cudaEventElapsedTime", cudaGetLastError());
        return HD_ERR_CUDA;
      }
      st->prof_ms[q] += ms;
      st->prof_n[q] += 1;
      st->prof_b[q] += st->prof_bytes[s];
    }
    // graph replays re-record the same events: keep the slots, read them again next time
    if (!st->gexec || !st->prof_on) st->prof_used = 0;
  }
  for (int q = 0; q < 3; q++) {
    if (ms3) ms3[q] = st->prof_ms[q];
    if (launches3) launches3[q] = st->prof_n[q];
    if (bytes3) bytes3[q] = st->prof_b[q];
  }
  if (clear)
    for (int q = 0; q < 3; q++) st->prof_ms[q] = st->prof_n[q] = 0, st->prof_b[q] = 0.0;
  return HD_OK;
}

HD_API int hd_get_launches(const hd_state* st, int64_t* launches) {
  if (!st || !launches) return HD_ERR_ARG;
  *launches = st->launches;
  return HD_OK;
}

HD_API int hd_sync(hd_state* st) {
  if (!st) return HD_ERR_ARG;
  if (cudaSetDevice(st->device) != cudaSuccess) return cuda_fail(st, cudaErrorInvalidDevice);
  unsigned int err = 0;
  cudaError_t e = cudaMemcpyAsync(&err, st->ws.err, sizeof(err), cudaMemcpyDeviceToHost, st->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st->stream);
  if (e != cudaSuccess) {
    set_error("hd_sync", e);
    return cuda_fail(st, e);
  }
  if (err) {
    snprintf(g_last_error, sizeof(g_last_error), "device error word 0x%x (bounded wait expired)", err);
    st->poisoned = HD_ERR_TIMEOUT;
    return HD_ERR_TIMEOUT;
  }
  return st->poisoned;
}

HD_API int hd_reset(hd_state* st, uint64_t seed) {
  if (!st) return HD_ERR_ARG;
  if (cudaSetDevice(st->device) == cudaSuccess) {
    // clear election counters and the error word left by an aborted step
    cudaMemsetAsync(st->ws.cnt, 0, (size_t)3 * (kMaxGroups + 1) * sizeof(unsigned int), st->stream);
    cudaMemsetAsync(st->ws.err, 0, 16, st->stream);
  }
  st->seed = seed;
  st->t = st->r = st->l = 0;
  st->drawn = 0;
  st->poisoned = 0;
  return HD_OK;
}

HD_API void hd_destroy(hd_state* st) {
  if (!st) return;
  cudaSetDevice(st->device);
  if (st->stream) cudaStreamSynchronize(st->stream); else cudaDeviceSynchronize();
  if (st->gexec) cudaGraphExecDestroy(st->gexec);
  if (st->own_stream) cudaStreamDestroy(st->own_stream);
  for (auto& ev : st->prof_ev)
    if (ev) cudaEventDestroy(ev);
  free_all(st);
  delete st;
}

HD_API int hd_get_counts(const hd_state* st, int32_t* t, int32_t* r, int32_t* l) {
  if (!st) return HD_ERR_ARG;
  if (t) *t = st->t;
  if (r) *r = st->r;
  if (l) *l = st->l;
  return HD_OK;
}

HD_API int hd_get_device_bytes(const hd_state* st, int64_t* bytes) {
  if (!st || !bytes) return HD_ERR_ARG;
  *bytes = st->bytes;
  return HD_OK;
}

HD_API int hd_philox_normals(uint64_t seed, uint32_t trial, uint32_t step, uint32_t stream_id,
                             int64_t start, int64_t count, int dtype, void* out, void* stream) {
  if (!out || start < 0 || count < 0) return HD_ERR_ARG;
  if (dtype != HD_F64 && dtype != HD_F32) return HD_ERR_ARG;
  DrawKey k;
  k.k0 = (uint32_t)(seed & 0xFFFFFFFFu);
  k.k1 = (uint32_t)(seed >> 32);
  k.step = step;
  k.trial = trial;
  k.stream = stream_id;
  return launch_philox_normals(k, start, count, dtype, out, (cudaStream_t)stream) == cudaSuccess
             ? HD_OK : HD_ERR_CUDA;
}

HD_API int hd_philox_words(uint64_t seed, const uint32_t* counters, int64_t nblocks, uint32_t* out,
                           void* stream) {
  if (!counters || !out || nblocks < 0) return HD_ERR_ARG;
  return launch_philox_words((uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32), counters,
                             nblocks, out, (cudaStream_t)stream) == cudaSuccess
             ? HD_OK : HD_ERR_CUDA;
}

}  // extern "C"
