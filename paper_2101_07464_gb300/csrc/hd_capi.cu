// Host side of libhd.so: the hd_state (a batch of independent trials; one for the
// single-trial API), its device memory, launch shapes, and the C ABI declared in
// include/hd.h.
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
#include "hd_state.cuh"

using namespace hd;

namespace {

thread_local char g_last_error[256] = "";


// Shape of a sweep over ncolT staged columns and NRV staged row vectors (ncolC column-owner
// columns, NR right-hand sides): the (warps per CTA, pipeline stages per warp) pair that puts
// the most bytes in flight per SM (capped at 128 KB; then more resident warps, then fewer
// stages), unless the state carries a measured shape for this kernel and column range
// (hd_autotune, hd_set_tuning).  The CTA count comes from the space's CTA map.  fixW > 0
// restricts the choice to that many warps per CTA (the step kernel runs both of its sweeps
// with the update sweep's warps).
template <typename T>
SweepCfg make_sweep(const hd_state* st, int which, int ncolT, int NRV, int ncolC, int NR, int fixW = 0) {
  SweepCfg c;
  c.W = (fixW > 0) ? fixW : 8;
  c.nbuf = 1;
  const int stat = st->static_smem[which] + 1024;
  const int blk = st->smem_blk_max - stat;
  const double stage = (double)(ncolT + NRV) * 32.0 * sizeof(T);
  auto ctas_of = [&](int W, int nb) {
    const size_t b = sweep_smem_bytes<T>(W, nb, ncolT, NRV, ncolC, NR);
    if ((int)b > blk) return 0;
    const int by_regs = std::max(1, st->occ_regs[which] * 8 / W);
    // the CTA maps give each SM at most kSweepCtasPerSm CTAs
    return std::min(std::min(by_regs, (int)(st->smem_sm / (b + stat))), kSweepCtasPerSm);
  };
  double best = -1.0;
  for (int W = 8; W >= 1; W /= 2) {
    if (fixW > 0 && W != fixW) continue;
    for (int nb = 1; nb <= 8; nb *= 2) {
      const int ctas = ctas_of(W, nb);
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
  // a shape forced by the autotuner, else the tuned one of this column range, when it fits
  const int bucket = hd::tune_bucket(ncolT);
  int tW = st->force_W, tnb = st->force_nb;
  if (!tW) {
    tW = st->tuneW[which][bucket];
    tnb = st->tuneNb[which][bucket];
  }
  if (tW > 0 && tnb > 0 && (fixW == 0 || tW == fixW) && ctas_of(tW, tnb) >= 1) {
    c.W = tW;
    c.nbuf = tnb;
  }
  c.per_sm = ctas_of(c.W, c.nbuf);
  c.tag = which | (bucket << 4);
  c.g.ctas = 0;
  c.g.vpc = 0;
  c.g.gsize = 1;
  c.g.ngroups = 1;
  return c;
}

template <typename T>
void pick_maps(const hd_state* st, BatchStep<T>& b);

template <typename T>
BatchStep<T> make_batch(const hd_state* st, int d, int kD, int kN, const void* x, void* y) {
  BatchStep<T> b;
  memset(&b, 0, sizeof(b));
  StepPlan<T>& p = b.base;
  p.ens = st->ens;
  p.Tm = st->Sld;   // leading dimension of S
  p.kD = kD;
  p.kN = kN;
  p.x = (const T*)x;
  p.y = (T*)y;
  p.sigma = (st->ens == HD_GINIBRE) ? (T)st->sigma : T(1);
  const int nc1 = kD + ((st->ens == 0) ? kN : 0);
  p.c1 = make_sweep<T>(st, 0, nc1, 1, nc1, 1);
  p.c2 = make_sweep<T>(st, 1, kD, 1, kD, 2);
  if (st->ens == HD_HAAR)
    p.c3 = make_sweep<T>(st, 2, kN, 2, kN, 1);
  else
    p.c3 = make_sweep<T>(st, 3, kN + kD, 1, kN, 1);
  p.pdl = st->pdl;
  p.fin_out = st->count > 1 ? 1 : 0;
  // trial 0's stacks give the host-side launch code its dimensions (probe)
  p.D = st->hdesc[0].st[d];
  p.N = st->hdesc[0].st[1 - d];
  b.d = d;
  b.desc = st->ddesc;
  b.map[0] = st->map[0];
  b.map[1] = st->map[1];
  return b;
}

// CTAs of the step kernel resident per SM for a block size and dynamic shared memory, cached
// per state (the occupancy query is a host call; trajectories ask once per step).
template <typename T>
int step_occupancy(hd_state* st, bool haar, int threads, size_t smem) {
  const int64_t key = ((int64_t)(haar ? 1 : 0) << 48) | ((int64_t)threads << 32) | (int64_t)smem;
  for (const auto& kv : st->step_occ)
    if (kv.first == key) return kv.second;
  const int occ = step_kernel_occupancy<T>(haar, threads, smem);
  st->step_occ.emplace_back(key, occ);
  return occ;
}

// The step kernel's shape: the update sweep's warps for both sweeps (the output sweep's stages
// re-chosen for them), the larger of the two shared-memory carves, and as many CTAs as are
// resident at once, at most the larger of the two CTA maps (the CTAs walk the maps' virtual
// CTAs).  Leaves step_ctas = 0, i.e. two launches, when no CTA of that shape fits an SM.
template <typename T>
void plan_step_kernel(hd_state* st, BatchStep<T>& b) {
  StepPlan<T>& p = b.base;
  const int kD = p.kD, kN = p.kN;
  const bool haar = st->ens == HD_HAAR;
  const int W = p.c2.W;
  if (p.c3.W != W)
    p.c3 = haar ? make_sweep<T>(st, 4, kN, 2, kN, 1, W) : make_sweep<T>(st, 5, kN + kD, 3, kN + kD, 1, W);
  const size_t s2 = sweep_smem_bytes<T>(W, p.c2.nbuf, kD, 1, kD, 2);
  const size_t s3 = haar ? sweep_smem_bytes<T>(W, p.c3.nbuf, kN, 2, kN, 1)
                         : sweep_smem_bytes<T>(W, p.c3.nbuf, kN + kD, 3, kN + kD, 1);
  const size_t smem = std::max(s2, s3);
  const int occ = step_occupancy<T>(st, haar, 32 * W, smem);
  if (occ < 1) return;
  const int want = std::max(b.map[b.d].ctas, b.map[1 - b.d].ctas);
  p.step_ctas = std::min(want, occ * st->nsm);
  p.step_smem = (int)smem;
}

// Row t (0-based) of one of hd_run's optional trajectory buffers (null when not given).
void* run_row(const hd_state* st, void* base, const hd_run_spec* sp, int t) {
  if (!base) return nullptr;
  return (char*)base + (size_t)t * (size_t)sp->ld_rows * st->esz;
}

template <typename T>
int first_draws(hd_state* st) {
  BatchStep<T> b = make_batch<T>(st, 0, 0, 0, nullptr, nullptr);
  for (int s = 0; s < 2; s++) {
    cudaError_t e = launch_first_draw<T>(b, s, key_for(st, 1), st->stream);
    if (e != cudaSuccess) return cuda_fail(st, e);
  }
  st->drawn = 1;
  st->launches += 2;
  return HD_OK;
}

// A step of a fused trajectory (hd_run): K3 applies the dynamics and forms the next step's
// K1 results (fuse), and/or this step's K1 was formed by the previous step (skip_dots).
struct FuseSpec {
  int fuse = 0;
  int skip_dots = 0;
  int dyn = 0;
  double a = 0.0;
  void* xnext = nullptr;
  const void* xprev = nullptr;
  int amp_mode = 0;          // HD_DYN_AMP / HD_DYN_ISTA: 1 after Q beta, 2 after Q^T z, 3 after Q x
  double amp_tau = 1.0;      // step size of the x update (1 for AMP)
  void* amp_v = nullptr;
  void* amp_y = nullptr;
  const void* amp_w = nullptr;
  void* yrec = nullptr;        // trajectory records of this step's row (hd_run_spec)
  void* xrec = nullptr;
  const void* xgiven = nullptr;
};

template <typename T>
int do_step(hd_state* st, const void* x, int transpose, void* y, const FuseSpec* fs = nullptr) {
  if (!st->drawn) {
    int rc = first_draws<T>(st);
    if (rc) return rc;
  }
  const int d = transpose ? 1 : 0;  // data-side stack: R for Q, L for Q^T
  const int cnt[2] = {st->r, st->l};
  const int kD = (st->ens == HD_HAAR) ? st->t : cnt[d];
  const int kN = (st->ens == HD_HAAR) ? st->t : cnt[1 - d];
  if (st->adj && st->adj->on) {
    const int rc = adj_record_step(st, x, transpose, kD, kN);
    if (rc) return rc;
  }
  BatchStep<T> b = make_batch<T>(st, d, kD, kN, x, y);
  b.base.key_next = key_for(st, st->t + 2);
  bool step_fallback = false;   // a fused step that the step kernel could not take
  if (fs) {
    b.base.skip_dots = fs->skip_dots;
    if (fs->fuse) {
      b.base.fuse = 1;
      b.base.dyn = fs->dyn;
      b.base.dyn_a = (T)fs->a;
      b.base.xnext = (T*)fs->xnext;
      b.base.xprev = (const T*)fs->xprev;
      b.base.amp_mode = fs->amp_mode;
      b.base.amp_tau = (T)fs->amp_tau;
      b.base.amp_v = (T*)fs->amp_v;
      b.base.amp_y = (T*)fs->amp_y;
      b.base.amp_w = (const T*)fs->amp_w;
      b.base.amp_zsq = st->amp_zsq;
      b.base.amp_nnz = st->amp_nnz;
      b.base.yrec = (T*)fs->yrec;
      b.base.xrec = (T*)fs->xrec;
      b.base.xgiven = (const T*)fs->xgiven;
      b.base.y = nullptr;
      if (st->ens == HD_HAAR)
        b.base.c3 = make_sweep<T>(st, 4, kN, 2, kN, 1);
      else
        b.base.c3 = make_sweep<T>(st, 5, kN + kD, 3, kN + kD, 1);
    }
  }
  pick_maps<T>(st, b);
  if (fs && fs->fuse && st->step_kernel) {
    plan_step_kernel<T>(st, b);
    step_fallback = b.base.step_ctas == 0;
  }
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
  cudaError_t e = launch_step<T>(b, st->stream, ev, launched);
  if (e != cudaSuccess) return cuda_fail(st, e);
  if (st->adj && st->adj->on) {
    const int rc = adj_record_after(st, kD, kN);
    if (rc) return rc;
  }
  st->launches += launched[0] + (launched[1] ? 1 : 0) + launched[2];
  if (slot0 >= 0) {
    // algorithmic bytes: each sweep reads its stack once plus the vectors it reads/writes
    const double es = (double)sizeof(T);
    const double nD = (double)(st->off[d][st->count]), nN = (double)(st->off[1 - d][st->count]);
    const double bd = (st->ens == HD_GINIBRE) ? (double)kN * nD : 0.0;
    const double bn = (st->ens == HD_GINIBRE) ? (double)(kD + 1) * nN : 0.0;
    const bool fz = fs && fs->fuse;
    double bb[3] = {es * (nD * kD + bd + nD), es * (nD * kD + 3.0 * nD),
                    es * (nN * kN + bn + (fz ? 5.0 : 4.0) * nN)};
    const SweepCfg* cs[3] = {&b.base.c1, &b.base.c2, &b.base.c3};
    int kind[3] = {launched[0] ? 0 : -1, launched[1] ? 1 : -1, launched[2] ? 2 : -1};
    if (launched[1] == 2) {   // the step kernel: K2 and K3 in the K2 slot, profiled as kind 3
      kind[1] = 3;
      bb[1] += bb[2];
    }
    for (int q = 0; q < 3; q++) {
      st->prof_kind[slot0 + q] = kind[q];
      st->prof_bytes[slot0 + q] = bb[q];
      st->prof_tag[slot0 + q] = cs[q]->tag | (cs[q]->W << 8) | (cs[q]->nbuf << 12);
      // a forced shape that left the step kernel is no shape for it: the autotuner drops it
      if (step_fallback && q >= 1) st->prof_tag[slot0 + q] &= ~(0xf << 8);
    }
    st->prof_used += 3;
  }
  st->t += 1;
  if (transpose) st->l += 1; else st->r += 1;
  st->hist.push_back((uint8_t)(transpose ? 1 : 0));
  return HD_OK;
}

// Probe with the representation as it stood after step `step` (1..t): the leading columns of
// the stacks, S and the prefix signs are exactly those of that step.
template <typename T>
int do_probe(hd_state* st, const void* x, int transpose, void* y, double* unrevealed_host, int step) {
  const int d = transpose ? 1 : 0;
  int cnt[2] = {0, 0};
  for (int q = 0; q < step; q++) cnt[st->hist[q] ? 1 : 0] += 1;
  const int kD = (st->ens == HD_HAAR) ? step : cnt[d];
  const int kN = (st->ens == HD_HAAR) ? step : cnt[1 - d];
  BatchStep<T> b = make_batch<T>(st, d, kD, kN, x, y);
  b.base.pdl = 0;
  // workspace of max(m, n) + 1 doubles, allocated by the first probe and kept by the state
  if (!st->probe_ws) {
    const int64_t dmax = std::max(st->dims[0][0], st->dims[1][0]);
    st->probe_ws = (double*)dalloc(st, (size_t)(dmax + 1) * 8);
    if (!st->probe_ws) {
      set_error("hd_probe workspace", cudaErrorMemoryAllocation);
      return HD_ERR_OOM;
    }
  }
  const int64_t dimD = st->dims[d][0];
  double* q = st->probe_ws;
  double* unrev = q + dimD;
  cudaError_t e = cudaMemsetAsync(unrev, 0, 8, st->stream);
  if (e == cudaSuccess) e = launch_probe<T>(b, q, unrev, st->stream);
  double u2 = 0.0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&u2, unrev, 8, cudaMemcpyDeviceToHost, st->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st->stream);
  if (e != cudaSuccess) return cuda_fail(st, e);
  *unrevealed_host = std::sqrt(u2);
  return HD_OK;
}

template <typename T>
int run_steps(hd_state* st, const hd_run_spec* sp) {
  if (st->prof_on) st->prof_used = 0;
  st->t = st->r = st->l = 0;
  st->hist.clear();
  st->drawn = 0;
  if (int rc = adj_on_reset(st)) return rc;
  int cur = 0;
  // elementwise dynamics of a Q / Q^T alternating schedule: the output sweep of step t applies
  // f_t and forms step t+1's dot sweep (HD_ENGINE_NO_FUSE turns this off)
  // (a state recording for reverse mode keeps the unfused steps: their workspace holds each
  // step's own dots when the step is recorded)
  const bool fusable = (sp->dynamics == HD_DYN_TANH || sp->dynamics == HD_DYN_SIGN_MEM) && st->fuse &&
                       !(st->adj && st->adj->on);
  int prev_fused = 0;
  for (int t = 0; t < sp->T; t++) {
    const int tr = sp->transpose[t] ? 1 : 0;
    FuseSpec fs;
    fs.skip_dots = prev_fused;
    fs.fuse = fusable && t + 1 < sp->T && ((sp->transpose[t + 1] ? 1 : 0) != tr);
    fs.dyn = sp->dynamics;
    fs.a = sp->a;
    fs.xnext = st->xw[1 - cur];
    fs.xprev = st->xw[1 - cur];
    fs.yrec = run_row(st, sp->y_record, sp, t);
    fs.xrec = run_row(st, sp->x_record, sp, t);
    fs.xgiven = (t + 1 < sp->T) ? run_row(st, const_cast<void*>(sp->x_given), sp, t) : nullptr;
    int rc = do_step<T>(st, st->xw[cur], tr, st->yw, &fs);
    if (rc) return rc;
    prev_fused = fs.fuse;
    if (fs.fuse) {
      cur = 1 - cur;
      continue;
    }
    const int64_t nout = st->off[tr ? 0 : 1][st->count];   // packed length of the output space
    cudaError_t e = launch_dynamics<T>(sp->dynamics, sp->a, (const T*)st->yw, (const T*)st->xw[cur],
                                       (const T*)st->xw[1 - cur], (T*)st->xw[1 - cur], nout,
                                       st->sumsq, st->stream, st->pdl != 0);
    if (e != cudaSuccess) return cuda_fail(st, e);
    st->launches += (sp->dynamics == HD_DYN_NORM_TANH) ? 2 : 1;
    // records and teacher forcing of an unfused step: plain stream-ordered copies
    const size_t bytes = (size_t)nout * st->esz;
    if (fs.yrec) e = cudaMemcpyAsync(fs.yrec, st->yw, bytes, cudaMemcpyDeviceToDevice, st->stream);
    if (e == cudaSuccess && fs.xrec)
      e = cudaMemcpyAsync(fs.xrec, st->xw[1 - cur], bytes, cudaMemcpyDeviceToDevice, st->stream);
    if (e == cudaSuccess && fs.xgiven)
      e = cudaMemcpyAsync(st->xw[1 - cur], fs.xgiven, bytes, cudaMemcpyDeviceToDevice, st->stream);
    if (e != cudaSuccess) return cuda_fail(st, e);
    cur = 1 - cur;
  }
  st->run_final = cur;
  return HD_OK;
}

// HD_DYN_AMP: product 1 is Q beta, then Q^T z^k and Q x^{k+1} alternate (flags checked by
// hd_run); the AMP updates run per trial between the products.
template <typename T>
int run_amp(hd_state* st, const hd_run_spec* sp) {
  if (st->prof_on) st->prof_used = 0;
  st->t = st->r = st->l = 0;
  st->hist.clear();
  st->drawn = 0;
  if (int rc = adj_on_reset(st)) return rc;
  const int cnt = st->count;
  const int64_t ntot = st->off[0][cnt];
  cudaError_t e = cudaMemsetAsync(st->amp_x, 0, (size_t)ntot * st->esz, st->stream);
  if (e != cudaSuccess) return cuda_fail(st, e);
  // every step but the last runs its AMP update inside the fused output sweep, which also forms
  // the next step's dot sweep; the last step uses the stand-alone AMP kernel
  int prev_fused = 0;
  for (int t = 1; t <= sp->T; t++) {
    const int mode = (t == 1) ? 1 : ((t % 2 == 0) ? 2 : 3);
    FuseSpec fs;
    fs.skip_dots = prev_fused;
    fs.fuse = st->fuse && t < sp->T && !(st->adj && st->adj->on);
    const int ista = sp->dynamics == HD_DYN_ISTA;
    fs.dyn = sp->dynamics;
    fs.a = sp->a;
    fs.amp_tau = ista ? sp->b : 1.0;
    fs.amp_mode = mode;
    fs.amp_v = (mode == 2) ? st->amp_x : st->amp_z;
    fs.amp_y = st->amp_y;
    fs.amp_w = st->amp_w;
    fs.yrec = run_row(st, sp->y_record, sp, t - 1);
    fs.xrec = run_row(st, sp->x_record, sp, t - 1);
    fs.xgiven = (t < sp->T) ? run_row(st, const_cast<void*>(sp->x_given), sp, t - 1) : nullptr;
    // teacher forcing replaces the AMP vector inside the fused sweep, which also forms the
    // per-trial norm or count of the replacement; the stand-alone AMP kernels do not
    if (fs.xgiven && !fs.fuse) return HD_ERR_STATE;
    const void* xin = (mode == 1) ? st->xw[0] : ((mode == 2) ? st->amp_z : st->amp_x);
    int rc = do_step<T>(st, xin, mode == 2 ? 1 : 0, st->yw, &fs);
    if (rc) return rc;
    prev_fused = fs.fuse;
    if (fs.fuse) continue;
    const int64_t nout = st->off[mode == 2 ? 0 : 1][cnt];
    if (fs.yrec) {
      e = cudaMemcpyAsync(fs.yrec, st->yw, (size_t)nout * st->esz, cudaMemcpyDeviceToDevice, st->stream);
      if (e != cudaSuccess) return cuda_fail(st, e);
    }
    if (mode == 1)
      e = launch_amp_init<T>(cnt, st->d_off[1], (const T*)st->yw, (const T*)st->amp_w, (T*)st->amp_y,
                             (T*)st->amp_z, st->amp_zsq, st->stream);
    else if (mode == 2)
      e = launch_amp_x<T>(cnt, st->d_off[0], st->d_off[1], (const T*)st->yw, (T*)st->amp_x, st->amp_zsq, sp->a,
                          fs.amp_tau, ista, st->amp_nnz, st->stream);
    else
      e = launch_amp_z<T>(cnt, st->d_off[1], (const T*)st->amp_y, (const T*)st->yw, (T*)st->amp_z, st->amp_nnz,
                          ista, st->amp_zsq, st->stream);
    if (e != cudaSuccess) return cuda_fail(st, e);
    st->launches += 1;
    if (fs.xrec) {
      e = cudaMemcpyAsync(fs.xrec, mode == 2 ? st->amp_x : st->amp_z, (size_t)nout * st->esz,
                          cudaMemcpyDeviceToDevice, st->stream);
      if (e != cudaSuccess) return cuda_fail(st, e);
    }
  }
  return HD_OK;
}

int amp_buffers(hd_state* st) {
  if (st->amp_y) return HD_OK;
  const int cnt = st->count;
  const size_t bm = (size_t)round_up(st->off[1][cnt], 64) * st->esz;
  const size_t bn = (size_t)round_up(st->off[0][cnt], 64) * st->esz;
  st->amp_y = dalloc(st, bm);
  st->amp_z = dalloc(st, bm);
  st->amp_w = dalloc(st, bm);
  st->amp_x = dalloc(st, bn);
  st->amp_zsq = (double*)dalloc(st, (size_t)cnt * sizeof(double));
  st->amp_nnz = (int*)dalloc(st, (size_t)cnt * sizeof(int));
  for (int s = 0; s < 2; s++) {
    st->d_off[s] = (int64_t*)dalloc(st, (size_t)(cnt + 1) * sizeof(int64_t));
    if (!st->d_off[s]) return HD_ERR_OOM;
    if (cudaMemcpy(st->d_off[s], st->off[s].data(), (size_t)(cnt + 1) * sizeof(int64_t),
                   cudaMemcpyHostToDevice) != cudaSuccess)
      return cuda_fail(st, cudaGetLastError());
  }
  if (!st->amp_y || !st->amp_z || !st->amp_w || !st->amp_x || !st->amp_zsq || !st->amp_nnz) return HD_ERR_OOM;
  return HD_OK;
}

int run_any(hd_state* st, const hd_run_spec* sp) {
  if (sp->dynamics == HD_DYN_AMP || sp->dynamics == HD_DYN_ISTA)
    return (st->dtype == HD_F64) ? run_amp<double>(st, sp) : run_amp<float>(st, sp);
  return (st->dtype == HD_F64) ? run_steps<double>(st, sp) : run_steps<float>(st, sp);
}

bool graph_matches(const hd_state* st, const hd_run_spec* sp) {
  if (!st->gexec || st->g_T != sp->T || st->g_dyn != sp->dynamics || st->g_a != sp->a || st->g_b != sp->b)
    return false;
  if (st->g_seed != st->seed || st->g_trial != st->trial || st->g_sigma != st->sigma) return false;
  if (st->g_sigma_gen != st->sigma_gen) return false;
  if (st->g_tune_gen != st->tune_gen) return false;
  if (st->g_stream != st->stream || st->g_prof != st->prof_on) return false;
  if (st->g_rows[0] != sp->y_record || st->g_rows[1] != sp->x_record || st->g_rows[2] != sp->x_given ||
      st->g_ld_rows != sp->ld_rows)
    return false;
  for (int t = 0; t < sp->T; t++)
    if (st->g_flags[t] != (sp->transpose[t] ? 1 : 0)) return false;
  return true;
}

// CTA map of one space: every trial gets ceil(nsub_i / spc) CTAs of spc 32-row sub-tiles.
// The trials' CTA ranges are laid out largest trial first.  The GPU hands out the CTAs of a
// launch roughly in index order, so the longest CTAs start first and the short ones fill in
// behind them (the longest-processing-time-first rule), instead of a large trial at the end
// of the batch running alone.  cta0[i] is trial i's first CTA and nct[i] its number of CTAs
// (contiguous: a CTA's local index is blockIdx - cta0[trial]); cta0[count] is the total.
bool build_map(hd_state* st, int s, int64_t spc, CtaMap* out) {
  const int count = st->count;
  std::vector<int> cta0(count + 1), spcv(count), nct(count), order(count);
  std::vector<int> ct;
  for (int i = 0; i < count; i++) {
    const int64_t nsub = (st->dims[s][i] + 31) / 32;
    nct[i] = (int)((nsub + spc - 1) / spc);
    spcv[i] = (int)spc;
    order[i] = i;
    st->maxncta = std::max(st->maxncta, nct[i]);
  }
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return st->dims[s][a] > st->dims[s][b]; });
  int next = 0;
  for (int q = 0; q < count; q++) {
    const int i = order[q];
    cta0[i] = next;
    for (int c = 0; c < nct[i]; c++) ct.push_back(i);
    next += nct[i];
  }
  cta0[count] = next;
  int* d_ct = (int*)dalloc(st, ct.size() * sizeof(int));
  int* d_c0 = (int*)dalloc(st, cta0.size() * sizeof(int));
  int* d_nc = (int*)dalloc(st, nct.size() * sizeof(int));
  int* d_sp = (int*)dalloc(st, spcv.size() * sizeof(int));
  if (!d_ct || !d_c0 || !d_nc || !d_sp) return false;
  if (cudaMemcpy(d_ct, ct.data(), ct.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(d_c0, cta0.data(), cta0.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(d_nc, nct.data(), nct.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(d_sp, spcv.data(), spcv.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess)
    return false;
  out->cta_trial = d_ct;
  out->cta0 = d_c0;
  out->nct = d_nc;
  out->spc = d_sp;
  out->ctas = cta0[count];
  return true;
}

// The candidate CTA splits.  Option 0 (the built-in rule): spc chosen so that the whole batch
// fills kSweepCtasPerSm CTAs per SM (one wave; at least 16 sub-tiles per CTA).  Options 1.. halve
// the sub-tiles per CTA from min(that, the largest trial's sub-tiles), which splits the largest
// trials over more CTAs (load balance of unequal trials, more waves); at least 16 sub-tiles.
bool build_maps(hd_state* st) {
  int64_t spc0[2], base[2];
  for (int s = 0; s < 2; s++) {
    int64_t total = 0, maxsub = 1;
    for (int i = 0; i < st->count; i++) {
      const int64_t nsub = (st->dims[s][i] + 31) / 32;
      total += nsub;
      maxsub = std::max(maxsub, nsub);
    }
    const int64_t per = (int64_t)kSweepCtasPerSm * st->nsm;
    spc0[s] = std::max<int64_t>(16, (total + per - 1) / per);
    base[s] = std::min(spc0[s], maxsub);
  }
  st->nmaps = 0;
  for (int j = 0; j < kMapOpts; j++) {
    int64_t spc[2];
    for (int s = 0; s < 2; s++)
      spc[s] = (j == 0) ? spc0[s] : std::max<int64_t>(16, (base[s] + (1 << j) - 1) >> j);
    if (j > 0 && spc[0] >= std::min(spc0[0], base[0]) && spc[1] >= std::min(spc0[1], base[1])) continue;
    bool dup = false;
    for (int o = 0; o < st->nmaps; o++)
      dup = dup || (st->map_spc[o][0] == spc[0] && st->map_spc[o][1] == spc[1]);
    if (dup) continue;
    const int o = st->nmaps;
    for (int s = 0; s < 2; s++) {
      st->map_spc[o][s] = (int)spc[s];
      if (!build_map(st, s, spc[s], &st->maps[o][s])) return false;
    }
    st->nmaps++;
  }
  st->map_opt = 0;
  st->map[0] = st->maps[0][0];
  st->map[1] = st->maps[0][1];
  // the built-in rule for one CTA per SM
  st->has_map_one = 0;
  int64_t spc1[2];
  for (int s = 0; s < 2; s++) {
    int64_t total = 0;
    for (int i = 0; i < st->count; i++) total += (st->dims[s][i] + 31) / 32;
    spc1[s] = std::max<int64_t>(16, (total + st->nsm - 1) / st->nsm);
  }
  if (spc1[0] != spc0[0] || spc1[1] != spc0[1]) {
    for (int s = 0; s < 2; s++)
      if (!build_map(st, s, spc1[s], &st->map_one[s])) return false;
    st->has_map_one = 1;
  }
  return true;
}

// With the built-in split, a sweep whose launch shape leaves room for one CTA per SM takes
// the split with one CTA per SM, one wave of CTAs instead of two (the second wave's
// stragglers would otherwise leave SMs idle at the end of the sweep).  K1 and K2 share the
// data space's split, K3 has the output space's.  Every split of a space gives the same
// results up to the order of the FP64 sums over CTAs.
template <typename T>
void pick_maps(const hd_state* st, BatchStep<T>& b) {
  if (st->map_opt != 0 || !st->has_map_one) return;
  const StepPlan<T>& p = b.base;
  if (p.c2.per_sm == 1) b.map[b.d] = st->map_one[b.d];
  if (p.c3.per_sm == 1) b.map[1 - b.d] = st->map_one[1 - b.d];
}

int create_common(int ensemble, int count, const int64_t* m, const int64_t* n, int32_t T_max,
                  uint64_t seed, int dtype, hd_state** out) {
  if (!out || !m || !n) return HD_ERR_ARG;
  *out = nullptr;
  if (count < 1) return HD_ERR_DIM;
  if (ensemble != HD_GINIBRE && ensemble != HD_HAAR) return HD_ERR_ARG;
  if (dtype != HD_F64 && dtype != HD_F32) return HD_ERR_ARG;
  if (T_max <= 0 || T_max > kTmaxLimit) return HD_ERR_TMAX;
  for (int i = 0; i < count; i++) {
    if (m[i] <= 0 || n[i] <= 0) return HD_ERR_DIM;
    if (ensemble == HD_HAAR && m[i] != n[i]) return HD_ERR_DIM;
    if (m[i] > ((int64_t)1 << 40) || n[i] > ((int64_t)1 << 40)) return HD_ERR_DIM;
    if (ensemble == HD_GINIBRE && T_max > std::min(m[i], n[i])) return HD_ERR_TMAX;
    if (ensemble == HD_HAAR && T_max > n[i]) return HD_ERR_TMAX;
  }
  hd_state* st = new (std::nothrow) hd_state();
  if (!st) return HD_ERR_OOM;
  auto fail = [&](int code) {
    free_all(st);
    delete st;
    return code;
  };
  st->ens = ensemble;
  st->dtype = dtype;
  st->count = count;
  st->Tm = T_max;
  st->seed = seed;
  st->esz = (dtype == HD_F64) ? 8 : 4;
  for (int i = 0; i < count; i++) {
    st->dims[0].push_back(n[i]);
    st->dims[1].push_back(m[i]);
  }
  for (int s = 0; s < 2; s++) {
    st->off[s].assign(count + 1, 0);
    for (int i = 0; i < count; i++) st->off[s][i + 1] = st->off[s][i] + st->dims[s][i];
  }
  if (cudaGetDevice(&st->device) != cudaSuccess) {
    set_error("cudaGetDevice", cudaGetLastError());
    return fail(HD_ERR_CUDA);
  }
  cudaDeviceGetAttribute(&st->nsm, cudaDevAttrMultiProcessorCount, st->device);
  if (st->nsm <= 0) st->nsm = 1;
  cudaDeviceGetAttribute(&st->smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, st->device);
  cudaDeviceGetAttribute(&st->smem_blk_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, st->device);
  {
    const size_t need = (dtype == HD_F64) ? sweep_smem_bytes<double>(1, 1, T_max, 2, T_max, 2)
                                          : sweep_smem_bytes<float>(1, 1, T_max, 2, T_max, 2);
    if ((int)need > st->smem_blk_max - 8192) return fail(HD_ERR_TMAX);
    cudaError_t e = (dtype == HD_F64) ? set_sweep_smem_limit<double>(st->smem_blk_max - 1024)
                                      : set_sweep_smem_limit<float>(st->smem_blk_max - 1024);
    if (e != cudaSuccess) {
      set_error("cudaFuncSetAttribute", e);
      cudaGetLastError();
      return fail(HD_ERR_CUDA);
    }
  }
  for (int q = 0; q < 6; q++) {
    st->occ_regs[q] = (dtype == HD_F64) ? kernel_occupancy<double>(q, 0) : kernel_occupancy<float>(q, 0);
    st->static_smem[q] = (dtype == HD_F64) ? kernel_static_smem<double>(q) : kernel_static_smem<float>(q);
  }
  if (!build_maps(st)) return fail(HD_ERR_OOM);
  const int64_t Tm = T_max;
  const int64_t Sld = (T_max + 1) / 2 * 2;   // even: every column of S starts 16-byte aligned
  st->Sld = (int)Sld;
  const size_t es = st->esz;
  // per-space packed stacks: trial i at element offset voff[s][i] (ld_i = round_up(dim, 256))
  std::vector<int64_t> ld[2], voff[2], goff[2];
  int64_t vtot[2] = {0, 0}, gtot[2] = {0, 0};
  for (int s = 0; s < 2; s++) {
    for (int i = 0; i < count; i++) {
      const int64_t L = round_up(st->dims[s][i], 256);
      ld[s].push_back(L);
      voff[s].push_back(vtot[s]);
      goff[s].push_back(gtot[s]);
      vtot[s] += L * Tm;
      gtot[s] += L;
    }
  }
  void* V[2];
  void* G[2];
  void* B[2] = {nullptr, nullptr};
  double* S[2];
  double* DP[2];
  double* GD[2];
  double* GG[2];
  for (int s = 0; s < 2; s++) {
    V[s] = dalloc(st, (size_t)vtot[s] * es);
    G[s] = dalloc(st, (size_t)gtot[s] * es);
    S[s] = (double*)dalloc(st, (size_t)count * Sld * Sld * 8);
    DP[s] = (double*)dalloc(st, (size_t)count * (Tm + 1) * 8);
    GD[s] = (double*)dalloc(st, (size_t)count * (Tm + 1) * 8);
    GG[s] = (double*)dalloc(st, (size_t)count * 8);
    if (!V[s] || !G[s] || !S[s] || !DP[s] || !GD[s] || !GG[s]) return fail(HD_ERR_OOM);
    if (ensemble == HD_GINIBRE) {
      B[s] = dalloc(st, (size_t)vtot[s] * es);
      if (!B[s]) return fail(HD_ERR_OOM);
    }
  }
  // per-trial FP64 workspace (vectors, scratch, partial sums) and election counters
  const int64_t vs = 2 * Tm + 8;                 // length of the longest small vector
  const int64_t gmax = (int64_t)std::ceil(std::sqrt((double)st->maxncta)) + 1;
  const int64_t per_trial = vs /*z*/ + 4 * vs /*w phead wout wout2*/ + 4 * vs /*scr*/ + kNumScal +
                            (int64_t)st->maxncta * vs /*part*/ + gmax * vs /*gpart*/;
  double* wsb = (double*)dalloc(st, (size_t)count * per_trial * 8);
  st->cnt_bytes = (size_t)count * kCntSets * (kMaxGroups + 1) * sizeof(unsigned int);
  st->cnt = (unsigned int*)dalloc(st, st->cnt_bytes);
  st->err = (unsigned int*)dalloc(st, 16);
  if (!wsb || !st->cnt || !st->err) return fail(HD_ERR_OOM);
  st->hdesc.resize(count);
  for (int i = 0; i < count; i++) {
    TrialDesc& td = st->hdesc[i];
    memset(&td, 0, sizeof(td));
    for (int s = 0; s < 2; s++) {
      StackDev& X = td.st[s];
      X.V = (char*)V[s] + (size_t)voff[s][i] * es;
      X.ld = ld[s][i];
      X.dim = st->dims[s][i];
      X.S = S[s] + (size_t)i * Sld * Sld;
      X.dpre = DP[s] + (size_t)i * (Tm + 1);
      X.gbuf = (char*)G[s] + (size_t)goff[s][i] * es;
      X.gdot = GD[s] + (size_t)i * (Tm + 1);
      X.gg = GG[s] + i;
      td.basis[s] = B[s] ? (char*)B[s] + (size_t)voff[s][i] * es : nullptr;
      td.ldb[s] = ld[s][i];
      td.off[s] = st->off[s][i];
    }
    double* w = wsb + (size_t)i * per_trial;
    Ws& ws = td.ws;
    ws.z = w; w += vs;
    ws.w = w; w += vs;
    ws.phead = w; w += vs;
    ws.wout = w; w += vs;
    ws.wout2 = w; w += vs;
    ws.scrb = w; w += 4 * vs;
    ws.scr_stride = vs;
    ws.scal = w; w += kNumScal;
    ws.part = w; w += (int64_t)st->maxncta * vs;
    ws.gpart = w; w += gmax * vs;
    ws.cnt = st->cnt + (size_t)i * kCntSets * (kMaxGroups + 1);
    ws.err = st->err;
    td.trial = (uint32_t)i;
    td.sigma = 1.0;
  }
  st->ddesc = (TrialDesc*)dalloc(st, (size_t)count * sizeof(TrialDesc));
  if (!st->ddesc) return fail(HD_ERR_OOM);
  // zero everything: reflector columns must be zero above their pivot, padding rows zero
  bool ok = true;
  for (int s = 0; s < 2 && ok; s++) {
    ok = cudaMemset(V[s], 0, (size_t)vtot[s] * es) == cudaSuccess &&
         cudaMemset(G[s], 0, (size_t)gtot[s] * es) == cudaSuccess &&
         cudaMemset(S[s], 0, (size_t)count * Sld * Sld * 8) == cudaSuccess &&
         cudaMemset(GD[s], 0, (size_t)count * (Tm + 1) * 8) == cudaSuccess &&
         cudaMemset(GG[s], 0, (size_t)count * 8) == cudaSuccess;
    if (ok && B[s]) ok = cudaMemset(B[s], 0, (size_t)vtot[s] * es) == cudaSuccess;
    if (ok) {
      std::vector<double> dp((size_t)count * (Tm + 1), 0.0);
      for (int i = 0; i < count; i++) dp[(size_t)i * (Tm + 1)] = 1.0;   // dpre[0] = 1
      ok = cudaMemcpy(DP[s], dp.data(), dp.size() * 8, cudaMemcpyHostToDevice) == cudaSuccess;
    }
  }
  if (ok) ok = cudaMemset(wsb, 0, (size_t)count * per_trial * 8) == cudaSuccess;
  if (ok) ok = cudaMemset(st->cnt, 0, st->cnt_bytes) == cudaSuccess;
  if (ok) ok = cudaMemset(st->err, 0, 16) == cudaSuccess;
  if (ok) ok = cudaMemcpy(st->ddesc, st->hdesc.data(), (size_t)count * sizeof(TrialDesc),
                          cudaMemcpyHostToDevice) == cudaSuccess;
  if (ok) ok = cudaDeviceSynchronize() == cudaSuccess;
  if (!ok) {
    set_error("hd_create initialisation", cudaGetLastError());
    return fail(HD_ERR_CUDA);
  }
  tune_load_cached(st);
  *out = st;
  return HD_OK;
}

// Philox trial words of the trials: base + i.
int upload_trials(hd_state* st) {
  for (int i = 0; i < st->count; i++) {
    st->hdesc[i].trial = st->trial + (uint32_t)i;
    st->hdesc[i].sigma = (st->ens == HD_HAAR) ? 1.0 : (st->sigmas.empty() ? st->sigma : st->sigmas[i]);
  }
  if (cudaMemcpy(st->ddesc, st->hdesc.data(), (size_t)st->count * sizeof(TrialDesc),
                 cudaMemcpyHostToDevice) != cudaSuccess) {
    set_error("trial upload", cudaGetLastError());
    return HD_ERR_CUDA;
  }
  return HD_OK;
}

}  // namespace

namespace hd {

void set_error(const char* where, cudaError_t e) {
  snprintf(g_last_error, sizeof(g_last_error), "%s: %s", where, cudaGetErrorString(e));
}

int cuda_fail(hd_state* st, cudaError_t e) {
  set_error("kernel launch", e);
  if (st) st->poisoned = HD_ERR_CUDA;
  return HD_ERR_CUDA;
}

int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

void* dalloc(hd_state* st, size_t bytes) {
  void* p = nullptr;
  if (bytes == 0) bytes = 16;
  bytes = (bytes + 255) & ~(size_t)255;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  st->allocs.push_back(p);
  st->bytes += (int64_t)bytes;
  return p;
}

void free_all(hd_state* st) {
  for (void* p : st->allocs) cudaFree(p);
  st->allocs.clear();
}

DrawKey key_for(const hd_state* st, int step) {
  DrawKey k;
  k.k0 = (uint32_t)(st->seed & 0xFFFFFFFFu);
  k.k1 = (uint32_t)(st->seed >> 32);
  k.step = (uint32_t)step;
  k.trial = st->trial;   // replaced per trial by the kernels (desc.trial)
  k.stream = 0;
  return k;
}

// Lets other translation units of the library set hd_last_error's text.
void record_error_text(const char* msg) { snprintf(g_last_error, sizeof(g_last_error), "%s", msg); }
}  // namespace hd

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
    case HD_ERR_STATE: return "HD_ERR_STATE: call not valid in the state's current phase";
    default: return "unknown status";
  }
}

HD_API int hd_create(int ensemble, int64_t m, int64_t n, int32_t T_max, uint64_t seed, int dtype,
                     hd_state** out) {
  return create_common(ensemble, 1, &m, &n, T_max, seed, dtype, out);
}

HD_API int hd_create_batched(int ensemble, int32_t count, const int64_t* m, const int64_t* n,
                             int32_t T_max, uint64_t seed, int dtype, hd_state** out) {
  return create_common(ensemble, count, m, n, T_max, seed, dtype, out);
}

HD_API int hd_get_batch_layout(const hd_state* st, int32_t* count, int64_t* off_n, int64_t* off_m) {
  if (!st) return HD_ERR_ARG;
  if (count) *count = st->count;
  for (int i = 0; i <= st->count; i++) {
    if (off_n) off_n[i] = st->off[0][i];
    if (off_m) off_m[i] = st->off[1][i];
  }
  return HD_OK;
}

HD_API int hd_set_options(hd_state* st, double sigma, uint32_t trial, void* stream) {
  if (!st) return HD_ERR_ARG;
  if (!(sigma > 0.0) || !std::isfinite(sigma)) return HD_ERR_ARG;
  if (st->t > 0 && (sigma != st->sigma || trial != st->trial)) return HD_ERR_ARG;
  const bool changed = trial != st->hdesc[0].trial || sigma != st->sigma || !st->sigmas.empty();
  st->sigma = sigma;
  st->sigmas.clear();
  st->stream = (cudaStream_t)stream;
  st->trial = trial;
  if (changed) {
    st->sigma_gen += 1;
    if (cudaSetDevice(st->device) != cudaSuccess) return cuda_fail(st, cudaErrorInvalidDevice);
    return upload_trials(st);
  }
  return HD_OK;
}

HD_API int hd_set_engine(hd_state* st, int flags) {
  if (!st) return HD_ERR_ARG;
  if (flags & ~(HD_ENGINE_NO_FUSE | HD_ENGINE_NO_PDL | HD_ENGINE_STEP_KERNEL)) return HD_ERR_ARG;
  st->fuse = (flags & HD_ENGINE_NO_FUSE) ? 0 : 1;
  st->pdl = (flags & HD_ENGINE_NO_PDL) ? 0 : 1;
  st->step_kernel = (flags & HD_ENGINE_STEP_KERNEL) ? 1 : 0;
  st->tune_gen += 1;   // a cached trajectory graph was captured with the old launches
  return HD_OK;
}

HD_API int hd_set_trial_sigmas(hd_state* st, const double* sigma) {
  if (!st || !sigma) return HD_ERR_ARG;
  if (st->t > 0) return HD_ERR_STATE;
  for (int i = 0; i < st->count; i++)
    if (!(sigma[i] > 0.0) || !std::isfinite(sigma[i])) return HD_ERR_ARG;
  st->sigmas.assign(sigma, sigma + st->count);
  st->sigma_gen += 1;
  if (cudaSetDevice(st->device) != cudaSuccess) return cuda_fail(st, cudaErrorInvalidDevice);
  return upload_trials(st);
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

HD_API int hd_run(hd_state* st, const hd_run_spec* sp, const void* x1, void* x_out) {
  if (!st || !sp || !sp->transpose || !x1 || !x_out) return HD_ERR_ARG;
  if (st->poisoned) return st->poisoned;
  if (sp->T < 1 || sp->T > st->Tm) return HD_ERR_TMAX;
  if (sp->dynamics != HD_DYN_TANH && sp->dynamics != HD_DYN_SIGN_MEM && sp->dynamics != HD_DYN_NORM_TANH &&
      sp->dynamics != HD_DYN_AMP && sp->dynamics != HD_DYN_ISTA)
    return HD_ERR_ARG;
  if (sp->dynamics == HD_DYN_NORM_TANH && st->count != 1) return HD_ERR_ARG;
  const bool amp = sp->dynamics == HD_DYN_AMP || sp->dynamics == HD_DYN_ISTA;
  if (sp->dynamics == HD_DYN_ISTA && !std::isfinite(sp->b)) return HD_ERR_ARG;
  if (amp) {
    if (!sp->aux || st->ens != HD_GINIBRE) return HD_ERR_ARG;
    for (int t = 0; t < sp->T; t++)
      if ((sp->transpose[t] ? 1 : 0) != (t % 2)) return HD_ERR_ARG;   // Q, Q^T, Q, ...
  }
  if (!std::isfinite(sp->a)) return HD_ERR_ARG;
  if (sp->y_record || sp->x_record || sp->x_given) {
    const int64_t need = std::max(st->off[0][st->count], st->off[1][st->count]);
    if (sp->ld_rows < need) return HD_ERR_ARG;
    const void* rows[3] = {sp->y_record, sp->x_record, sp->x_given};
    for (int i = 0; i < 3; i++)
      if (rows[i] && ((uintptr_t)rows[i] % st->esz) != 0) return HD_ERR_ARG;
  }
  // dimensions: input of step t+1 = output of step t for every trial
  for (int t = 0; t + 1 < sp->T; t++) {
    const int so = sp->transpose[t] ? 0 : 1, si = sp->transpose[t + 1] ? 1 : 0;
    for (int i = 0; i < st->count; i++)
      if (st->dims[so][i] != st->dims[si][i]) return HD_ERR_DIM;
  }
  if (cudaSetDevice(st->device) != cudaSuccess) return cuda_fail(st, cudaErrorInvalidDevice);
  const int64_t dmax = std::max(st->off[0][st->count], st->off[1][st->count]);
  if (!st->yw) {
    const int64_t L = round_up(dmax, 64);
    st->xw[0] = dalloc(st, (size_t)L * st->esz);
    st->xw[1] = dalloc(st, (size_t)L * st->esz);
    st->yw = dalloc(st, (size_t)L * st->esz);
    st->sumsq = (double*)dalloc(st, 64);
    if (!st->xw[0] || !st->xw[1] || !st->yw || !st->sumsq) return HD_ERR_OOM;
  }
  const int64_t nin = st->off[sp->transpose[0] ? 1 : 0][st->count];
  const int64_t nfin = amp ? st->off[0][st->count] : st->off[sp->transpose[sp->T - 1] ? 0 : 1][st->count];
  if (amp) {
    if (int rc0 = amp_buffers(st)) return rc0;
  }
  cudaError_t e = cudaMemcpyAsync(st->xw[0], x1, (size_t)nin * st->esz, cudaMemcpyDefault, st->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(st->xw[1], 0, (size_t)dmax * st->esz, st->stream);
  if (e == cudaSuccess && amp)
    e = cudaMemcpyAsync(st->amp_w, sp->aux, (size_t)st->off[1][st->count] * st->esz, cudaMemcpyDefault,
                        st->stream);
  if (e != cudaSuccess) {
    set_error("hd_run input copy", e);
    return cuda_fail(st, e);
  }
  int rc = HD_OK;
  // reverse mode records every step on the host, so a recording state runs without the graph
  if (sp->use_graph && !(st->adj && st->adj->on)) {
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
      rc = run_any(st, sp);
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
      st->g_b = sp->b;
      st->g_seed = st->seed;
      st->g_trial = st->trial;
      st->g_sigma = st->sigma;
      st->g_sigma_gen = st->sigma_gen;
      st->g_tune_gen = st->tune_gen;
      st->g_stream = st->stream;
      st->g_flags.assign(sp->transpose, sp->transpose + sp->T);
      for (auto& f : st->g_flags) f = f ? 1 : 0;
      st->g_final = st->run_final;
      st->g_prof = st->prof_on;
      st->g_rows[0] = sp->y_record;
      st->g_rows[1] = sp->x_record;
      st->g_rows[2] = sp->x_given;
      st->g_ld_rows = sp->ld_rows;
    }
    e = cudaGraphLaunch(st->gexec, st->stream);
    if (e != cudaSuccess) {
      set_error("cudaGraphLaunch", e);
      return cuda_fail(st, e);
    }
    st->launches += st->g_launches;
    st->t = sp->T;
    st->r = st->l = 0;
    st->hist.assign(sp->transpose, sp->transpose + sp->T);
    for (auto& f : st->hist) f = f ? 1 : 0;
    for (int t = 0; t < sp->T; t++) (sp->transpose[t] ? st->l : st->r) += 1;
    st->drawn = 1;
    st->run_final = st->g_final;
  } else {
    rc = run_any(st, sp);
    if (rc) return rc;
  }
  e = cudaMemcpyAsync(x_out, amp ? st->amp_x : st->xw[st->run_final], (size_t)nfin * st->esz, cudaMemcpyDefault,
                      st->stream);
  if (e != cudaSuccess) {
    set_error("hd_run output copy", e);
    return cuda_fail(st, e);
  }
  return HD_OK;
}

HD_API int hd_probe(hd_state* st, const void* x, int transpose, void* y, double* unrevealed_host) {
  if (!st || !x || !y || !unrevealed_host) return HD_ERR_ARG;
  if (transpose != 0 && transpose != 1) return HD_ERR_ARG;
  if (st->count != 1) return HD_ERR_ARG;
  if (st->poisoned) return st->poisoned;
  if (cudaSetDevice(st->device) != cudaSuccess) return cuda_fail(st, cudaErrorInvalidDevice);
  return (st->dtype == HD_F64) ? do_probe<double>(st, x, transpose, y, unrevealed_host, st->t)
                               : do_probe<float>(st, x, transpose, y, unrevealed_host, st->t);
}

HD_API int hd_probe_at(hd_state* st, int32_t step, const void* x, int transpose, void* y, double* unrevealed_host) {
  if (!st || !x || !y || !unrevealed_host) return HD_ERR_ARG;
  if (transpose != 0 && transpose != 1) return HD_ERR_ARG;
  if (st->count != 1) return HD_ERR_ARG;
  if (step < 0 || step > st->t || (size_t)st->t != st->hist.size()) return HD_ERR_ARG;
  if (st->poisoned) return st->poisoned;
  if (cudaSetDevice(st->device) != cudaSuccess) return cuda_fail(st, cudaErrorInvalidDevice);
  return (st->dtype == HD_F64) ? do_probe<double>(st, x, transpose, y, unrevealed_host, step)
                               : do_probe<float>(st, x, transpose, y, unrevealed_host, step);
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
    st->prof_tag.assign(slots, 0);
    st->prof_cap = slots;
  }
  st->prof_on = on ? 1 : 0;
  st->prof_used = 0;
  return HD_OK;
}

HD_API int hd_profile_read(hd_state* st, double* ms4, int64_t* launches4, double* bytes4, int clear) {
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
  for (int q = 0; q < 4; q++) {
    if (ms4) ms4[q] = st->prof_ms[q];
    if (launches4) launches4[q] = st->prof_n[q];
    if (bytes4) bytes4[q] = st->prof_b[q];
  }
  if (clear)
    for (int q = 0; q < 4; q++) st->prof_ms[q] = st->prof_n[q] = 0, st->prof_b[q] = 0.0;
  return HD_OK;
}

HD_API int hd_get_launches(const hd_state* st, int64_t* launches) {
  if (!st || !launches) return HD_ERR_ARG;
  *launches = st->launches;
  return HD_OK;
}

HD_API int hd_check_bounded_wait(hd_state* st, uint32_t polls) {
  if (!st || polls < 1 || polls > (1u << 24)) return HD_ERR_ARG;
  if (st->poisoned) return st->poisoned;
  if (cudaSetDevice(st->device) != cudaSuccess) return cuda_fail(st, cudaErrorInvalidDevice);
  const cudaError_t e = launch_wait_selftest(st->err, polls, st->stream);
  if (e != cudaSuccess) return cuda_fail(st, e);
  st->launches += 1;
  return HD_OK;
}

HD_API int hd_sync(hd_state* st) {
  if (!st) return HD_ERR_ARG;
  if (cudaSetDevice(st->device) != cudaSuccess) return cuda_fail(st, cudaErrorInvalidDevice);
  unsigned int err = 0;
  cudaError_t e = cudaMemcpyAsync(&err, st->err, sizeof(err), cudaMemcpyDeviceToHost, st->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st->stream);
  if (e != cudaSuccess) {
    set_error("hd_sync", e);
    return cuda_fail(st, e);
  }
  if (err) {
    snprintf(g_last_error, sizeof(g_last_error), "device error word 0x%x (bounded wait expired: bit 0 a "
             "staging barrier, bit 1 a step kernel flag)", err);
    st->poisoned = HD_ERR_TIMEOUT;
    return HD_ERR_TIMEOUT;
  }
  return st->poisoned;
}

HD_API int hd_reset(hd_state* st, uint64_t seed) {
  if (!st) return HD_ERR_ARG;
  if (cudaSetDevice(st->device) == cudaSuccess) {
    // clear election counters and the error word left by an aborted step
    cudaMemsetAsync(st->cnt, 0, st->cnt_bytes, st->stream);
    cudaMemsetAsync(st->err, 0, 16, st->stream);
  }
  st->seed = seed;
  st->t = st->r = st->l = 0;
  st->hist.clear();
  st->drawn = 0;
  st->poisoned = 0;
  return adj_on_reset(st);
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
  delete st->adj;
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
