// The library's state object (host side) and the helpers shared by its translation units.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "hd_kernels.cuh"

namespace hd {

// Launch-shape tuning: per sweep kernel (dots, update, out Haar, out Gin, fused out Haar,
// fused out Gin) and per range of column counts (bucket b holds counts c with bit width b:
// 0, 1, 2-3, 4-7, ...), the tuned (warps per CTA, stages per warp); 0 = the built-in rule.
constexpr int kSweepKinds = 6;
constexpr int kTuneBuckets = 11;
constexpr int kMapOpts = 5;            // CTA splits (sub-tiles per CTA) tried by the autotuner
constexpr int kTuneWords = 2 + 2 * kSweepKinds * kTuneBuckets;
inline int tune_bucket(int cols) {
  int b = 0;
  while (cols > 0 && b < kTuneBuckets - 1) {
    cols >>= 1;
    b++;
  }
  return b;
}

// Reverse-mode record and accumulators of a single-trial state (hd_adjoint_*).
struct AdjState {
  int on = 0;
  int record_x = 0;
  std::vector<int8_t> flag;      // per forward step: transpose flag
  std::vector<int> kD, kN;       // per forward step: reflectors in the data / other stack before it
                                 // (every trial of a batched state has the same dimensions)
  int rev = 0;                   // forward steps not yet reversed
  void* Vbar[2] = {nullptr, nullptr};     // d loss / d V per stack (state dtype, dim x T_max, ld of the stack)
  void* Bbar[2] = {nullptr, nullptr};     // d loss / d basis store per space (Ginibre; state dtype)
  double* Sbar[2] = {nullptr, nullptr};   // d loss / d S per stack (T_max x T_max)
  void* X = nullptr;             // recorded step inputs x_t (state dtype), column t-1
  int64_t ldx = 0;
  int64_t dmax = 0;              // longest vector (rounded)
  void* vec = nullptr;           // work vectors (state dtype), kAdjVecs x dmax
  double* small = nullptr;       // FP64 small arena, kAdjSmall x (T_max + 8)
  int64_t small_ld = 0;
  double* part = nullptr;        // column-pass partial sums
  int nblk = 1;
  // distances between consecutive trials of the reverse mode's own arrays (batched states)
  int64_t part_stride = 0, vec_stride = 0, small_stride = 0, rec_stride = 0, sbar_stride = 0;
  int64_t vbar_stride[2] = {0, 0}, bbar_stride[2] = {0, 0};
  // per forward step: z (k_D + k_N: data-stack dots, then Gin basis dots), w (k_D), p_head
  // (k_D), then p's pivot entry and alpha, copied from the workspace after the step
  double* rec = nullptr;
  int64_t rec_ld = 0;
  // A data-side update Vbar += sum_q v_q (s_q c_q)^T of one reverse step, held back so that
  // the next reverse step adds it in the same pass over that stack as its own output-side
  // update (Haar, Q and Q^T alternating: both cover the same columns).
  struct Pending {
    int on = 0;
    int s = 0;                   // stack
    int K = 0;                   // columns 0..K-1
    int n = 0;                   // terms
    const void* v[3] = {nullptr, nullptr, nullptr};
    const double* c[3] = {nullptr, nullptr, nullptr};
    double sc[3] = {0.0, 0.0, 0.0};
    int Kq[3] = {0, 0, 0};       // columns each term covers
    int64_t sv[3] = {0, 0, 0};   // trial strides of v and c
    int64_t scs[3] = {0, 0, 0};
  } pend;
  // Haar: the data side of a reverse step runs on a second stream beside the output side
  // (fork at the start, cbar hand-over in the middle, join at the end)
  cudaStream_t aux = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_mid = nullptr, ev_join = nullptr;
  ~AdjState() {
    if (ev_fork) cudaEventDestroy(ev_fork);
    if (ev_mid) cudaEventDestroy(ev_mid);
    if (ev_join) cudaEventDestroy(ev_join);
    if (aux) cudaStreamDestroy(aux);
  }
};

}  // namespace hd

using hd::TrialDesc;
using hd::CtaMap;

struct hd_state {
  int ens = 0, dtype = 0;
  int count = 1;                 // trials
  std::vector<int64_t> dims[2];  // per trial: dims[0] = n_i (space of R), dims[1] = m_i (space of L)
  std::vector<int64_t> off[2];   // packed vector offsets per space (count + 1)
  int Tm = 0;
  int Sld = 0;                   // leading dimension of the S matrices (T_max rounded up to even)
  uint64_t seed = 0;
  uint32_t trial = 0;            // Philox trial word of trial 0 (trial i uses trial + i)
  double sigma = 1.0;
  std::vector<double> sigmas;    // per-trial entry scales (hd_set_trial_sigmas); empty: all sigma
  int64_t sigma_gen = 0;         // bumped whenever the draw scales change
  cudaStream_t stream = nullptr;
  int device = 0;
  int t = 0, r = 0, l = 0;
  std::vector<uint8_t> hist;     // transpose flag of every step since create/reset
  int drawn = 0;                 // first draws made since create/reset
  int poisoned = 0;              // sticky error code
  size_t esz = 8;                // element size of vectors and stacks
  std::vector<TrialDesc> hdesc;  // host copy of the per-trial descriptors
  TrialDesc* ddesc = nullptr;
  CtaMap map[2];                 // the CTA split in use (maps[map_opt])
  CtaMap maps[hd::kMapOpts][2];  // candidate splits per space (option 0: the built-in rule)
  int map_spc[hd::kMapOpts][2] = {};
  int nmaps = 1;
  int map_opt = 0;
  // the built-in split with one CTA per SM instead of kSweepCtasPerSm (one wave for sweeps whose
  // shape leaves room for one CTA per SM); has_map_one = 0 when it equals the built-in split
  CtaMap map_one[2];
  int has_map_one = 0;
  int maxncta = 1;
  // launch shapes: tuned table, autotuner override, cache key of the state's shape
  int8_t tuneW[hd::kSweepKinds][hd::kTuneBuckets] = {};
  int8_t tuneNb[hd::kSweepKinds][hd::kTuneBuckets] = {};
  int force_W = 0, force_nb = 0;
  int64_t tune_gen = 0;
  std::string tune_key;
  unsigned int* err = nullptr;
  unsigned int* cnt = nullptr;
  size_t cnt_bytes = 0;
  int nsm = 1;
  int pdl = 1;                   // programmatic dependent launch of the sweeps (hd_set_engine)
  int fuse = 1;                  // fused output + dynamics + dot sweeps in hd_run (hd_set_engine)
  int step_kernel = 0;           // update + fused output sweep as one launch (hd_set_engine)
  std::vector<std::pair<int64_t, int>> step_occ;   // step kernel occupancy per launch shape
  int occ_regs[6] = {1, 1, 1, 1, 1, 1};  // CTAs of 256 threads per SM allowed by registers, per sweep kernel
  int static_smem[6] = {0, 0, 0, 0, 0, 0};   // (dots, update, out Haar, out Gin, fused out Haar, fused out Gin)
  int smem_sm = 0;
  int smem_blk_max = 0;
  int64_t bytes = 0;
  std::vector<void*> allocs;
  // hd_run: work vectors and the cached trajectory graph
  void* xw[2] = {nullptr, nullptr};
  void* yw = nullptr;
  void* ens_tmp[2] = {nullptr, nullptr};   // hd_goe_apply / hd_usv_apply intermediates
  double* sumsq = nullptr;
  double* probe_ws = nullptr;    // hd_probe: max(m, n) + 1 doubles (allocated by the first probe)
  int run_final = 0;
  cudaStream_t own_stream = nullptr;
  cudaGraphExec_t gexec = nullptr;
  std::vector<uint8_t> g_flags;
  int g_T = 0, g_dyn = 0;
  double g_a = 0.0, g_b = 0.0, g_sigma = 0.0;
  int64_t g_sigma_gen = -1;
  uint64_t g_seed = 0;
  uint32_t g_trial = 0;
  cudaStream_t g_stream = nullptr;
  int g_final = 0;
  int g_launches = 0;
  int g_prof = 0;
  int64_t g_tune_gen = -1;
  const void* g_rows[3] = {nullptr, nullptr, nullptr};   // hd_run_spec record / teacher buffers
  int64_t g_ld_rows = 0;
  int64_t launches = 0;          // kernel launches issued (graph replays count their kernels)
  // profiling: event pairs around each sweep, algorithmic bytes of each recorded launch
  int prof_on = 0;
  int prof_cap = 0;
  int prof_used = 0;
  std::vector<cudaEvent_t> prof_ev;
  std::vector<int> prof_kind;
  std::vector<double> prof_bytes;
  std::vector<int> prof_tag;     // per slot: kernel | bucket << 4 | W << 8 | stages << 12
  double prof_ms[4] = {0, 0, 0, 0};   // per kind: dots, update, output, step kernel
  int64_t prof_n[4] = {0, 0, 0, 0};
  double prof_b[4] = {0, 0, 0, 0};
  hd::AdjState* adj = nullptr;   // reverse mode (hd_adjoint_enable)
  // hd_run with HD_DYN_AMP: packed per-trial vectors and scalars (allocated on first use)
  void* amp_y = nullptr;         // y = Q beta + w (m-space)
  void* amp_z = nullptr;         // z^k (m-space)
  void* amp_x = nullptr;         // x^k (n-space)
  void* amp_w = nullptr;         // the caller's w, copied (m-space)
  double* amp_zsq = nullptr;     // ||z^k||^2 per trial
  int* amp_nnz = nullptr;        // ||x^k||_0 per trial
  int64_t* d_off[2] = {nullptr, nullptr};   // packed offsets per space on the device
};

namespace hd {
void set_error(const char* where, cudaError_t e);
int cuda_fail(hd_state* st, cudaError_t e);
int64_t round_up(int64_t a, int64_t b);
void* dalloc(hd_state* st, size_t bytes);
void free_all(hd_state* st);
DrawKey key_for(const hd_state* st, int step);
void record_error_text(const char* msg);
// reverse mode hooks of the forward path (hd_adjoint.cu)
int adj_record_step(hd_state* st, const void* x, int transpose, int kD, int kN);
int adj_record_after(hd_state* st, int kD, int kN);
int adj_on_reset(hd_state* st);
// launch-shape tuning (hd_tune.cu)
void tune_load_cached(hd_state* st);
int tune_apply_words(hd_state* st, const int32_t* words);
void set_map_option(hd_state* st, int opt);
}  // namespace hd
