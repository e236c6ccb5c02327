// Host side of libhd.so: the hd_state, its device memory, launch shapes, and the C ABI
// declared in include/hd.h.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <new>

#include <cuda_runtime.h>

#include "../../include/hd.h"
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
  int occ_upd_regs = 1;  // K2 CTAs per SM allowed by registers
  int smem_sm = 0;       // shared memory per SM usable by CTAs
  int smem_blk_max = 0;  // opt-in dynamic shared memory per CTA
  int64_t bytes = 0;
  void* allocs[32];
  int nalloc = 0;
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

// K2 tile: the largest R in {256, 128, 64, 32} whose shared-memory footprint leaves room for
// two or more CTAs per SM (else the largest that fits one), grid = min(tiles, CTAs resident).
template <typename T>
void choose_update_tiles(const hd_state* st, int k, int64_t dim, StepPlan<T>* p) {
  int R = 32;
  for (int cand = 256; cand >= 32; cand /= 2) {
    const size_t b = update_smem_bytes<T>(k, cand);
    if ((int)(2 * (b + 1024)) <= st->smem_sm || cand == 32) {
      R = cand;
      break;
    }
  }
  const size_t bytes = update_smem_bytes<T>(k, R);
  int occ = std::max(1, std::min(st->occ_upd_regs, (int)(st->smem_sm / (bytes + 1024))));
  const int64_t ntiles = (dim + R - 1) / R;
  int64_t ctas = std::min<int64_t>(ntiles, (int64_t)occ * st->nsm);
  if (ctas < 1) ctas = 1;
  p->R2 = R;
  p->ntiles2 = ntiles;
  Grid g;
  g.ctas = (int)ctas;
  g.vpc = 0;
  g.gsize = std::max(1, (int)std::ceil(std::sqrt((double)ctas)));
  g.ngroups = (int)((ctas + g.gsize - 1) / g.gsize);
  p->g2 = g;
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
  p.g1 = st->grid[d];
  p.g3 = st->grid[1 - d];
  choose_update_tiles<T>(st, p.kD, p.D.dim, &p);
  cudaError_t e = launch_step<T>(p, st->stream);
  if (e != cudaSuccess) return cuda_fail(st, e);
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
  p.g1 = st->grid[d];
  p.g3 = st->grid[1 - d];
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

}  // namespace

extern "C" {

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
  int smem_sm = 0, smem_blk = 0;
  cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, st->device);
  cudaDeviceGetAttribute(&smem_blk, cudaDevAttrMaxSharedMemoryPerBlockOptin, st->device);
  st->smem_sm = smem_sm;
  st->smem_blk_max = smem_blk;
  {
    const size_t need = (dtype == HD_F64) ? update_smem_bytes<double>(T_max, 32)
                                          : update_smem_bytes<float>(T_max, 32);
    if ((int)need > smem_blk) {
      delete st;
      return HD_ERR_TMAX;
    }
    cudaError_t e = (dtype == HD_F64) ? set_update_smem_limit<double>(smem_blk - 1024)
                                      : set_update_smem_limit<float>(smem_blk - 1024);
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
  if (dtype == HD_F64) {
    occ = std::min(kernel_occupancy<double>(0, 0),
                   kernel_occupancy<double>(ensemble == HD_HAAR ? 2 : 3, dsm));
    st->occ_upd_regs = kernel_occupancy<double>(1, 0);
  } else {
    occ = std::min(kernel_occupancy<float>(0, 0),
                   kernel_occupancy<float>(ensemble == HD_HAAR ? 2 : 3, dsm));
    st->occ_upd_regs = kernel_occupancy<float>(1, 0);
  }
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
    X.ld = round_up(dims[s], 64);
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
    ok = w.z && w.w && w.phead && w.wout && w.wout2 && w.scrb && w.scal && w.part &&
         w.gpart && w.cnt;
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

HD_API int hd_reset(hd_state* st, uint64_t seed) {
  if (!st) return HD_ERR_ARG;
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
