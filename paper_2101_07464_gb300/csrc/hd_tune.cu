// Measured launch shapes of the sweeps: hd_autotune, hd_get_tuning, hd_set_tuning.
//
// Each sweep kernel streams its stack in 32-row sub-tiles.  Two choices set its speed and have
// no closed-form optimum on a given GPU: the shape of a CTA (warps, and pipeline stages per
// warp, which together fix the bytes in flight) and the split of each trial's rows over CTAs
// (sub-tiles per CTA: one wave of large CTAs, or more, smaller CTAs that balance trials of
// unequal size).  The built-in rule (make_sweep, the CTA maps' option 0) is a model of the
// first and a one-wave default for the second; the autotuner measures instead.  It runs the
// caller's own trajectory once per candidate: first every (warps, stages) pair forced on all
// sweeps, with CUDA events around each launch, keeping per kernel and per column range the
// pair with the least device time; then each CTA split with the tuned shapes, keeping the one
// with the least trajectory time.  Results are cached for the process under the state's shape.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "hd.h"
#include "hd_state.cuh"

using namespace hd;

namespace {

std::mutex g_tune_mu;
std::map<std::string, std::vector<int32_t>>& tune_cache() {
  static std::map<std::string, std::vector<int32_t>> cache;
  return cache;
}

// Cache key: ensemble, dtype, trials, T_max, device (name, SMs), fusion, and a hash of every
// trial's dimensions (FNV-1a over their bytes).
// Device names, looked up once per device (cudaGetDeviceProperties is slow).
std::string device_name(int dev) {
  static std::mutex mu;
  static std::map<int, std::string> names;
  std::lock_guard<std::mutex> lk(mu);
  auto it = names.find(dev);
  if (it != names.end()) return it->second;
  cudaDeviceProp prop;
  memset(&prop, 0, sizeof(prop));
  if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) cudaGetLastError();
  prop.name[sizeof(prop.name) - 1] = 0;
  return names[dev] = std::string(prop.name);
}

std::string shape_key(const hd_state* st) {
  const std::string name = device_name(st->device);
  uint64_t h = 1469598103934665603ull;
  for (int s = 0; s < 2; s++)
    for (int64_t d : st->dims[s])
      for (int b = 0; b < 8; b++) {
        h ^= (uint64_t)((d >> (8 * b)) & 0xff);
        h *= 1099511628211ull;
      }
  char buf[384];
  snprintf(buf, sizeof(buf), "%d/%d/%d/%d/%d/%.200s/%d/%016llx", st->ens, st->dtype, st->count, st->Tm,
           st->nsm, name.c_str(), st->fuse, (unsigned long long)h);
  return std::string(buf);
}

void words_of(const hd_state* st, int32_t* w) {
  w[0] = 1;
  w[1] = st->map_opt;
  for (int q = 0; q < kSweepKinds; q++)
    for (int b = 0; b < kTuneBuckets; b++) {
      w[2 + 2 * (q * kTuneBuckets + b)] = st->tuneW[q][b];
      w[3 + 2 * (q * kTuneBuckets + b)] = st->tuneNb[q][b];
    }
}

bool valid_shape(int v) { return v == 0 || v == 1 || v == 2 || v == 4 || v == 8; }

struct Acc {
  double ms = 0.0;
  int n = 0;
};
// kernel | bucket << 4  ->  W | stages << 4  ->  summed device time
using Table = std::map<int, std::map<int, Acc>>;

// Reads the recorded launches of the last run.  Launches whose shape is not `only` (a forced
// shape that did not fit there) are left out; only < 0 takes every launch and counts them.
int drain(hd_state* st, Table* acc, int only, std::map<int, int>* counts) {
  if (st->prof_used == 0) return HD_OK;
  if (cudaStreamSynchronize(st->stream) != cudaSuccess) return cuda_fail(st, cudaGetLastError());
  for (int s = 0; s < st->prof_used; s++) {
    if (st->prof_kind[s] < 0) continue;
    const int tag = st->prof_tag[s];
    const int key = tag & 0xff, shape = ((tag >> 8) & 0xf) | (((tag >> 12) & 0xf) << 4);
    if (counts) (*counts)[key] += 1;
    if (!acc || (only >= 0 && shape != only)) continue;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, st->prof_ev[2 * s], st->prof_ev[2 * s + 1]) != cudaSuccess) {
      set_error("cudaEventElapsedTime", cudaGetLastError());
      st->prof_used = 0;
      return HD_ERR_CUDA;
    }
    Acc& a = (*acc)[key][shape];
    a.ms += ms;
    a.n += 1;
  }
  st->prof_used = 0;
  return HD_OK;
}

}  // namespace

namespace hd {

void set_map_option(hd_state* st, int opt) {
  st->map_opt = opt;
  st->map[0] = st->maps[opt][0];
  st->map[1] = st->maps[opt][1];
  st->tune_gen++;
}

int tune_apply_words(hd_state* st, const int32_t* w) {
  if (w[0] != 1) return HD_ERR_ARG;
  if (w[1] < 0 || w[1] >= st->nmaps) return HD_ERR_ARG;
  for (int q = 0; q < kSweepKinds * kTuneBuckets; q++) {
    const int W = w[2 + 2 * q], nb = w[3 + 2 * q];
    if (!valid_shape(W) || !valid_shape(nb) || ((W == 0) != (nb == 0))) return HD_ERR_ARG;
  }
  for (int q = 0; q < kSweepKinds; q++)
    for (int b = 0; b < kTuneBuckets; b++) {
      st->tuneW[q][b] = (int8_t)w[2 + 2 * (q * kTuneBuckets + b)];
      st->tuneNb[q][b] = (int8_t)w[3 + 2 * (q * kTuneBuckets + b)];
    }
  set_map_option(st, w[1]);
  return HD_OK;
}

void tune_load_cached(hd_state* st) {
  st->tune_key = shape_key(st);
  std::vector<int32_t> w;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = tune_cache().find(st->tune_key);
    if (it == tune_cache().end()) return;
    w = it->second;
  }
  tune_apply_words(st, w.data());
}

}  // namespace hd

HD_API int hd_get_tuning(const hd_state* st, int32_t* words, int32_t nwords) {
  if (!st || !words || nwords < kTuneWords) return HD_ERR_ARG;
  words_of(st, words);
  return HD_OK;
}

HD_API int hd_set_tuning(hd_state* st, const int32_t* words, int32_t nwords) {
  if (!st || nwords < 0 || (nwords > 0 && !words)) return HD_ERR_ARG;
  if (nwords == 0) {   // back to the built-in rule
    memset(st->tuneW, 0, sizeof(st->tuneW));
    memset(st->tuneNb, 0, sizeof(st->tuneNb));
    set_map_option(st, 0);
    return HD_OK;
  }
  if (nwords < kTuneWords) return HD_ERR_ARG;
  return tune_apply_words(st, words);
}

HD_API int hd_get_map_options(const hd_state* st, int32_t* count, int32_t* spc) {
  if (!st || !count) return HD_ERR_ARG;
  *count = st->nmaps;
  if (spc)
    for (int o = 0; o < st->nmaps; o++) {
      spc[2 * o] = st->map_spc[o][0];
      spc[2 * o + 1] = st->map_spc[o][1];
    }
  return HD_OK;
}

HD_API int hd_autotune(hd_state* st, const hd_run_spec* sp, const void* x1, void* x_out, int32_t reps) {
  if (!st || !sp) return HD_ERR_ARG;
  if (reps < 1 || reps > 64) return HD_ERR_ARG;
  if (st->poisoned) return st->poisoned;
  if (st->adj && st->adj->on) return HD_ERR_STATE;
  if (cudaSetDevice(st->device) != cudaSuccess) return cuda_fail(st, cudaErrorInvalidDevice);
  hd_run_spec rs = *sp;
  rs.use_graph = 0;
  const int prof_was = st->prof_on;
  int rc = hd_profile_enable(st, 1);
  if (rc) return rc;
  memset(st->tuneW, 0, sizeof(st->tuneW));
  memset(st->tuneNb, 0, sizeof(st->tuneNb));
  set_map_option(st, 0);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  auto finish = [&](int code) {
    st->force_W = st->force_nb = 0;
    st->tune_gen++;
    st->prof_used = 0;
    hd_profile_enable(st, prof_was);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return code;
  };
  // warm-up with the built-in shapes; counts the launches per kernel and column range
  std::map<int, int> per_run;
  rc = hd_run(st, &rs, x1, x_out);
  if (!rc) rc = drain(st, nullptr, -1, &per_run);
  if (rc) return finish(rc);
  // stage 1: every (warps, stages) pair on every sweep
  Table acc;
  for (int W = 8; W >= 1; W /= 2)
    for (int nb = 1; nb <= 8; nb *= 2) {
      st->force_W = W;
      st->force_nb = nb;
      for (int r = 0; r < reps; r++) {
        rc = hd_run(st, &rs, x1, x_out);
        if (!rc) rc = drain(st, &acc, W | (nb << 4), nullptr);
        if (rc) return finish(rc);
      }
    }
  st->force_W = st->force_nb = 0;
  for (const auto& kv : acc) {
    const int q = kv.first & 0xf, b = kv.first >> 4;
    const int want = per_run[kv.first] * reps;
    double best = 0.0;
    int pick = -1;
    for (const auto& sv : kv.second) {
      if (sv.second.n != want) continue;   // the shape did not fit every launch of the range
      if (pick < 0 || sv.second.ms < best) {
        best = sv.second.ms;
        pick = sv.first;
      }
    }
    if (pick >= 0 && q < kSweepKinds && b < kTuneBuckets) {
      st->tuneW[q][b] = (int8_t)(pick & 0xf);
      st->tuneNb[q][b] = (int8_t)(pick >> 4);
    }
  }
  st->tune_gen++;
  // stage 2: the CTA splits, timed over whole trajectories (no per-launch events)
  hd_profile_enable(st, 0);
  if (st->nmaps > 1) {
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
      set_error("cudaEventCreate", cudaGetLastError());
      return finish(HD_ERR_CUDA);
    }
    int best_o = 0;
    float best_ms = 0.f;
    for (int o = 0; o < st->nmaps; o++) {
      set_map_option(st, o);
      rc = hd_run(st, &rs, x1, x_out);   // warm-up of this split
      if (rc) return finish(rc);
      cudaEventRecord(e0, st->stream);
      for (int r = 0; r < reps && !rc; r++) rc = hd_run(st, &rs, x1, x_out);
      if (rc) return finish(rc);
      cudaEventRecord(e1, st->stream);
      float ms = 0.f;
      cudaError_t e = cudaEventSynchronize(e1);
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e != cudaSuccess) {
        cuda_fail(st, e);
        set_error("autotune timing", e);
        return finish(HD_ERR_CUDA);
      }
      if (o == 0 || ms < best_ms) {
        best_ms = ms;
        best_o = o;
      }
    }
    set_map_option(st, best_o);
  }
  {
    std::vector<int32_t> w(kTuneWords);
    words_of(st, w.data());
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tune_cache()[st->tune_key] = w;
  }
  rc = hd_reset(st, st->seed);
  return finish(rc);
}
