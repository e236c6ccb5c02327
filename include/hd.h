/*
 * hd.h -- C ABI of the GB300 Householder Dice library (libhd.so).
 *
 * Householder Dice (Y. M. Lu, arXiv 2101.07464) simulates the dynamics of eq. (dynamics),
 *     x_{t+1} = f_t(M_t x_t, x_t, ..., x_{t-d}),   M_t in {Q, Q^T},
 * for a random Q from the Ginibre ensemble Gin(m, n) (Algorithm 1, Section 3.2) or the
 * Haar ensemble on O(n) (Algorithm 2, Section 3.3) without ever forming Q: each call
 * reveals only the randomness the current product needs, applies the stored Householder
 * reflectors and appends new ones, for O((m+n)T) memory and O((m+n)T^2) work.
 * The caller owns the dynamics f_t and chooses M_t at every step.
 *
 * Conventions of every entry point:
 *   - Return value: an hd_status (0 = HD_OK).  Functions never abort the process.
 *   - Pointers named x, y, out are DEVICE pointers (cudaMalloc / torch CUDA tensors) on
 *     the current CUDA device, unless the name ends in _host.  They are caller-owned;
 *     the library keeps no reference after the call returns.
 *   - Work is enqueued on the state's CUDA stream (hd_set_options; default stream 0) and
 *     is asynchronous: results are ready when that stream is synchronised.  Calls on one
 *     state must be ordered on one stream; distinct states are independent.
 *   - Layout: vectors are dense, contiguous, 8-byte (HD_F64) or 4-byte (HD_F32) elements.
 *     Buffers aligned to 16 bytes take the vectorised path; others are accepted and take
 *     a scalar path.
 *   - After an error inside a step (HD_ERR_CUDA, HD_ERR_TIMEOUT) the state is poisoned:
 *     every later hd_apply returns the same code until hd_reset.
 */
#ifndef HD_H
#define HD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define HD_API __attribute__((visibility("default")))
#else
#define HD_API
#endif

typedef struct hd_state hd_state;

typedef enum {
  HD_OK = 0,
  HD_ERR_ARG = 1,      /* null or invalid argument (bad enum, non-finite sigma, ...)      */
  HD_ERR_DIM = 2,      /* non-positive sizes, or m != n for the Haar ensemble            */
  HD_ERR_TMAX = 3,     /* the step would exceed T_max, or T_max > min(m, n) (Alg. 1) /
                          T_max > n (Alg. 2)                                              */
  HD_ERR_OOM = 4,      /* device allocation failed                                        */
  HD_ERR_CUDA = 5,     /* a CUDA call or kernel launch failed                             */
  HD_ERR_TIMEOUT = 6,  /* a bounded device-side wait expired                              */
  HD_ERR_STATE = 7     /* the call is not valid in the state's current phase (e.g. after
                          the first step, or with reverse mode on or not enabled)         */
} hd_status;

typedef enum { HD_GINIBRE = 0, HD_HAAR = 1 } hd_ensemble;
/* HD_F64: vectors, reflector stacks and all arithmetic in FP64.
 * HD_F32: vectors and reflector stacks stored and streamed in FP32 with FP32 math; the
 *         cross-warp/cross-block sums of every dot product and norm, the Householder
 *         coefficients and the compact-WY triangular factor S stay in FP64.            */
typedef enum { HD_F64 = 0, HD_F32 = 1 } hd_dtype;

/* Create a state for y = M_t x with Q ~ Gin(m, n) (entries sigma * N(0,1), sigma = 1 by
 * default: Section 3 notation) or Q ~ Haar(n) (requires m == n).  T_max bounds the number
 * of products: T_max <= min(m, n) for Gin (Algorithm 1 requires T <= min(m, n)), T_max <= n
 * for Haar (Algorithm 2 requires T <= n); this library also caps T_max at 256.  Allocates all device memory up front:
 * two reflector stacks (n x T_max and m x T_max elements), for Gin two basis stores of the
 * same sizes, and O(T_max^2) FP64 coefficients.  seed keys the Philox4x32-10 generator
 * that draws the Gaussian vectors g_t (key = seed, counter = (index/2, t, trial, 0)).
 * *out receives the state (owned by the caller; release with hd_destroy). */
HD_API int hd_create(int ensemble, int64_t m, int64_t n, int32_t T_max, uint64_t seed,
                     int dtype, hd_state** out);

/* A batch of `count` independent trials in one state (the paper's Monte-Carlo use: many
 * trajectories of the same dynamics): trial i is Q_i ~ Gin(m[i], n[i]) or Haar(n[i])
 * (m[i] == n[i]), with its own draws (Philox trial word = the state's trial option + i) and
 * its own reflector stacks; every step of the batch is one launch per sweep for all trials.
 * Vectors passed to hd_apply / hd_run are packed: trial i's entries of an n-space vector
 * occupy [off_n[i], off_n[i+1]) and of an m-space vector [off_m[i], off_m[i+1]) (no padding;
 * hd_get_batch_layout).  All trials share T_max (bounded by every trial's dimensions, as in
 * hd_create), the schedule of Q / Q^T and the options.
 * hd_probe is for single-trial states only. */
HD_API int hd_create_batched(int ensemble, int32_t count, const int64_t* m, const int64_t* n,
                             int32_t T_max, uint64_t seed, int dtype, hd_state** out);

/* Engine switches of a state (all off by default), for measurement and for checking one
 * code path against another; results differ only in the order of floating-point sums.
 *   HD_ENGINE_NO_FUSE  hd_run keeps the three separate sweeps of every step instead of
 *                      folding f_t and the next step's dot sweep into the output sweep
 *   HD_ENGINE_NO_PDL   launch the sweeps without programmatic dependent launch (no early
 *                      start of a sweep's prologue while its predecessor drains)
 *   HD_ENGINE_STEP_KERNEL  run the update sweep and the fused output sweep of a step of hd_run
 *                      as one launch, the step kernel, instead of two.  The step kernel is a
 *                      cooperative launch over all trials of the batch: its CTAs take the
 *                      update sweep's CTAs, then the output sweep's, from work queues, and a
 *                      trial's output CTAs start as soon as that trial's update finaliser has
 *                      released them (a bounded wait: on expiry the step fails with
 *                      HD_ERR_TIMEOUT at hd_sync).  Used for every fused step except the last
 *                      of a trajectory, when its launch shape fits at least one CTA per SM.
 *                      Off by default: on GB300 the merged kernel executes about 11 % more
 *                      instructions per sub-tile than the two sweeps apart (register allocation
 *                      over both sweep bodies), which costs more than the launch it saves.
 * Take effect from the next step; a cached hd_run graph is recaptured.  HD_ERR_ARG for an
 * unknown bit. */
#define HD_ENGINE_NO_FUSE 1
#define HD_ENGINE_NO_PDL 2
#define HD_ENGINE_STEP_KERNEL 4
HD_API int hd_set_engine(hd_state* st, int flags);

/* Per-trial entry scales of a Gin batch (count values, each finite and > 0): trial i's draws
 * are sigma[i] N(0, 1), i.e. Q_i has entry variance sigma[i]^2 (e.g. 1/m_i for the AMP
 * workload).  Before the first step only (HD_ERR_STATE otherwise); hd_set_options sets every
 * trial back to its single sigma.  Haar states ignore the scales. */
HD_API int hd_set_trial_sigmas(hd_state* st, const double* sigma);

/* Packed layout of a state's vectors: *count trials; off_n and off_m (either may be NULL)
 * receive count + 1 offsets each (prefix sums of n[i] and m[i]). */
HD_API int hd_get_batch_layout(const hd_state* st, int32_t* count, int64_t* off_n, int64_t* off_m);

/* Options; take effect from the next step.  sigma: entry standard deviation of the
 * Ginibre ensemble (> 0, finite; ignored for Haar, whose reflector H(g) does not depend on
 * the scale of g).  trial: the Philox counter word that separates independent trials
 * sharing one seed.  stream: a cudaStream_t (NULL = legacy default stream).
 * Changing sigma or trial after the first step returns HD_ERR_ARG (the draws of one
 * matrix must come from one stream of randomness); call hd_reset first. */
HD_API int hd_set_options(hd_state* st, double sigma, uint32_t trial, void* stream);

/* One product of eq. (dynamics): y = M_t x with M_t = Q (transpose = 0; x in R^n,
 * y in R^m) or M_t = Q^T (transpose = 1; x in R^m, y in R^n), for the t-th call since
 * create/reset (Algorithm 1 lines for M_t = Q / Q^T; Algorithm 2).  Draws g_t, extends the
 * reflector stacks by the new reflector(s) and writes y.  x and y must not overlap.
 * Errors: HD_ERR_TMAX when t would exceed T_max (state unchanged), HD_ERR_ARG for null
 * pointers or a bad transpose flag. */
HD_API int hd_apply(hd_state* st, const void* x, int transpose, void* y);

/* Consistency probe (does not add a step): y = Q^(t) x (or its transpose) using only the
 * revealed part of the current representation (eq. Gaussian_t for Gin, eq. H_t for Haar),
 * and *unrevealed_host = the norm of the component of x that the hidden block would see
 * (||Z_{1:r} R_r...R_1 x|| for Q); y equals M x exactly when it is zero, e.g. for any
 * earlier input x_s of the same direction, or Q^T applied to an earlier output.
 * Synchronises the state's stream (the norm is returned on the host).  The first probe of a
 * state allocates a workspace of max(m, n) + 1 doubles that the state keeps (HD_ERR_OOM if
 * that fails); later probes allocate nothing. */
HD_API int hd_probe(hd_state* st, const void* x, int transpose, void* y,
                    double* unrevealed_host);

/* hd_probe with the representation as it stood after product `step` (0 <= step <= t; the
 * leading columns of the reflector stacks, S and the signs are exactly that step's, since
 * later steps only append): y = Q^(step) x on the part revealed by then.  For an earlier input
 * x_s this reproduces y_s = M_s x_s with the reflectors that step used, at the cost of s
 * rather than t columns (the checkpointed reverse mode recomputes segments with it).
 * Errors: those of hd_probe; HD_ERR_ARG for a step out of range. */
HD_API int hd_probe_at(hd_state* st, int32_t step, const void* x, int transpose, void* y,
                       double* unrevealed_host);

/* Built-in dynamics f_t for hd_run (run in the library's kernels):
 *   HD_DYN_TANH       x_{t+1} = tanh(y_t)
 *   HD_DYN_SIGN_MEM   x_{t+1} = sign(y_t) + a x_{t-1}   (sign(0) = 0; x_0 = 0)
 *   HD_DYN_NORM_TANH  x_{t+1} = v/||v||, v = tanh(y_t) + a x_t      (single-trial states)
 *   HD_DYN_AMP        approximate message passing for y = Q beta + w, per trial (one of the
 *                     iterative algorithms eq. dynamics covers, Section 1).  Product 1 is
 *                     Q beta (x1 = beta, n-space); then y = Q beta + w, z^0 = y, x^0 = 0, and
 *                     the products alternate Q^T z^k (even t) and Q x^{k+1} (odd t):
 *                       x^{k+1} = eta(x^k + Q^T z^k; a ||z^k|| / sqrt(m)),
 *                       z^{k+1} = y - Q x^{k+1} + z^k ||x^{k+1}||_0 / m,
 *                     eta the soft threshold, a the threshold multiplier (1.1 in the batched
 *                     AMP workload), norms and counts per trial.  spec.aux = w (m-space);
 *                     x_out receives the last x^k (n-space).  The schedule must be Q, Q^T,
 *                     Q, ... (HD_ERR_ARG otherwise).
 *   HD_DYN_ISTA       ISTA for the lasso (Section 2.1), the same products and buffers as
 *                     HD_DYN_AMP with a fixed threshold and step size and no Onsager term:
 *                       x^{k+1} = eta(x^k + b Q^T z^k; a),   z^{k+1} = y - Q x^{k+1},
 *                     a = the threshold (lambda tau in Section 2.1), b = the step size tau;
 *                     z^0 = y is y - Q x^0 with x^0 = 0, so that product is not made.      */
typedef enum { HD_DYN_TANH = 1, HD_DYN_SIGN_MEM = 2, HD_DYN_NORM_TANH = 3, HD_DYN_AMP = 4, HD_DYN_ISTA = 5 } hd_dynamics;

typedef struct {
  int32_t T;                 /* number of products, 1 <= T <= T_max                      */
  const uint8_t* transpose;  /* host array of T flags: M_t = Q^T where nonzero           */
  int32_t dynamics;          /* an hd_dynamics value                                     */
  double a;                  /* coefficient of the dynamics                              */
  int32_t use_graph;         /* nonzero: capture the trajectory once in a CUDA graph and
                                replay it on later calls with the same (T, flags,
                                dynamics, a); the first call with use_graph must not
                                happen while the state's stream is being captured       */
  const void* aux;           /* HD_DYN_AMP / HD_DYN_ISTA: the noise w (packed m-space vector, device or
                                page-locked host, copied at the start of every call);
                                ignored otherwise                                       */
  /* Trajectory records, all optional (NULL = off).  Each is a device buffer of the state's
   * dtype holding T rows of ld_rows elements; row t-1 belongs to step t and holds a packed
   * vector of step t's output space (rows are not padded or cleared beyond that length).
   * They exist to check the trajectory path step by step: the fused sweeps that hd_run uses
   * for Q / Q^T alternating schedules never store y_t otherwise.                          */
  void* y_record;            /* receives y_t = M_t x_t                                   */
  void* x_record;            /* receives f_t's result as the library computed it: x_{t+1}
                                (HD_DYN_AMP: z^0, x^1, z^1, ... as each step updates them) */
  const void* x_given;       /* teacher forcing: row t-1 (t < T) replaces f_t's result as
                                the input of product t+1 and as the value later steps of
                                f read (x_{t-1} of sign_mem, x^k / z^k of AMP, whose norm
                                or nonzero count is then taken of the given vector); row
                                T-1 is not read, so x_out is f_T's own result.  With
                                HD_DYN_AMP it needs the fused sweeps (HD_ERR_STATE under
                                HD_ENGINE_NO_FUSE or reverse-mode recording)            */
  int64_t ld_rows;           /* elements between rows; >= the longest packed vector of the
                                state when any record is given (HD_ERR_ARG otherwise)     */
  double b;                  /* second coefficient of the dynamics (HD_DYN_ISTA: the step
                                size); ignored otherwise                                  */
} hd_run_spec;

/* A whole trajectory of eq. (dynamics): resets the state (same seed, trial and sigma),
 * then for t = 1..T computes y_t = M_t x_t (hd_apply) and x_{t+1} = f_t(y_t, x_t, x_{t-1})
 * with the built-in dynamics, all on the state's stream.  x1 (input, length n if M_1 = Q,
 * else m) and x_out (output x_{T+1}) may be device or page-locked host pointers (copied
 * with cudaMemcpyAsync, cudaMemcpyDefault); they are read/written on the stream.  Every
 * step's input dimension must match the previous output (HD_ERR_DIM otherwise: for a
 * rectangular Gin, Q and Q^T must alternate).  Work vectors are allocated by the state
 * on the first call (3 x max(m, n) elements; HD_DYN_AMP adds 3 x m + 2 x n).  Batched
 * states: every vector is packed (hd_get_batch_layout). */
HD_API int hd_run(hd_state* st, const hd_run_spec* spec, const void* x1, void* x_out);

/* Synchronise the state's stream and check the device error word: returns HD_ERR_TIMEOUT
 * (and poisons the state) if a bounded device-side wait expired in an earlier step, else the
 * state's sticky status (HD_OK when healthy). */
HD_API int hd_sync(hd_state* st);

/* Check of the failure path of the kernels' bounded waits (no fault involved): launches one
 * CTA that waits on a shared-memory barrier nothing will complete, then on a step-kernel flag
 * nothing will release; each wait gives up after `polls` polls (1..2^24; the flag wait sleeps
 * about 64 ns between polls) and sets its bit of the state's device error word (bit 0, bit 1).
 * The next hd_sync then returns HD_ERR_TIMEOUT and poisons the state, as after a real
 * expired wait; hd_reset clears it.  Errors: HD_ERR_ARG (polls out of range), the state's
 * sticky status, HD_ERR_CUDA. */
HD_API int hd_check_bounded_wait(hd_state* st, uint32_t polls);

/* Forget all steps (t = r = l = 0) and re-key the generator with seed; keeps the
 * allocations and options.  Clears a poisoned state. */
HD_API int hd_reset(hd_state* st, uint64_t seed);

/* Release the state and its device memory (synchronises its stream).  NULL is allowed. */
HD_API void hd_destroy(hd_state* st);

/* Step counters: *t = products so far, *r = number of Q products, *l = number of Q^T
 * products (r + l = t; for Haar both stacks hold t reflectors). */
HD_API int hd_get_counts(const hd_state* st, int32_t* t, int32_t* r, int32_t* l);

/* Device bytes allocated by the state. */
HD_API int hd_get_device_bytes(const hd_state* st, int64_t* bytes);

/* Text of the last CUDA failure seen by a call of this library in the calling thread
 * (empty if none); valid until the next failing call in that thread. */
HD_API const char* hd_last_error(void);

/* Profiling of the sweeps of every step (kind 0 = dots K1, 1 = update K2, 2 = output K3,
 * 3 = the step kernel, K2 and the fused K3 in one launch): when enabled, CUDA events are
 * recorded on the state's stream around each sweep launch (also inside a graph captured by
 * hd_run, which then re-records the same events on
 * every replay).  hd_profile_read synchronises the stream, adds the elapsed times of the
 * recorded launches to running totals and returns, per kind, the total milliseconds, the
 * number of launches and their algorithmic bytes (each stack read once plus the vectors
 * the sweep reads and writes); clear != 0 zeroes the totals after reading. */
HD_API int hd_profile_enable(hd_state* st, int on);
HD_API int hd_profile_read(hd_state* st, double* ms4, int64_t* launches4, double* bytes4,
                           int clear);

/* Launch shapes of the sweeps (the paper fixes none: these are the engine's own choices for
 * streaming the reflector stacks of Algorithms 1 and 2; results depend on them only through
 * the order of floating-point sums).  Two choices are tunable:
 *   - per sweep kernel (dots, update, output Haar, output Ginibre, and the fused output
 *     sweeps of both) and per range of column counts (bit width of the count: 0, 1, 2-3,
 *     4-7, ..., >= 512), the pair (warps per CTA, pipeline stages per warp), each 1, 2, 4
 *     or 8; 0 means the built-in rule (the pair with the most bytes in flight per SM);
 *   - the CTA split, one of hd_get_map_options' candidates: sub-tiles of 32 rows per CTA in
 *     the n-space and in the m-space (option 0, the built-in rule: one wave of CTAs over the
 *     whole batch; later options split large trials over more CTAs).
 * A shape that does not fit the shared memory at some column count falls back to the rule.
 *
 * hd_autotune measures them on the caller's trajectory: it runs `spec` as hd_run (without a
 * graph, from x1, writing x_out; reps >= 1 timed runs per candidate, at most 64) under every
 * (warps, stages) pair with CUDA events around each sweep, keeps per kernel and column range
 * the pair of least device time, then times each CTA split over whole trajectories and keeps
 * the fastest.  About 16 * reps + nmaps * (reps + 1) + 1 trajectories.  The result applies to
 * this state and is cached for the process under the state's shape (ensemble, dtype, trials
 * and their dimensions, T_max, device); hd_create / hd_create_batched of the same shape
 * start from it.  The state is left reset (hd_reset with its seed); profiling totals are
 * kept, unread profiling records dropped.  Errors: those of hd_run; HD_ERR_ARG (reps out of
 * range), HD_ERR_STATE (reverse mode on).
 *
 * hd_get_tuning writes the state's choices as HD_TUNE_WORDS int32 words (nwords >= that):
 * [1, split option, then for kernel q = 0..5 and range b = 0..10: warps, stages]; the words
 * can be stored and handed to hd_set_tuning on a state of the same shape (HD_ERR_ARG for a
 * bad version, split option or value).  hd_set_tuning with nwords = 0 restores the rules.
 * hd_get_map_options returns the number of candidate splits and, when spc is non-null,
 * their sub-tiles per CTA (2 x count int32: n-space, m-space). */
#define HD_TUNE_WORDS 134
HD_API int hd_autotune(hd_state* st, const hd_run_spec* spec, const void* x1, void* x_out, int32_t reps);
HD_API int hd_get_tuning(const hd_state* st, int32_t* words, int32_t nwords);
HD_API int hd_set_tuning(hd_state* st, const int32_t* words, int32_t nwords);
HD_API int hd_get_map_options(const hd_state* st, int32_t* count, int32_t* spc);

/* Other ensembles from the Gaussian and Haar ones (paper, section "Other Random Matrix
 * Ensembles").
 *
 * hd_goe_apply: y = W x for W = (Q + Q^T)/sqrt(2) ~ GOE(n), Q the square Ginibre matrix of
 * `st` (entries N(0, sigma^2); sigma = 1 gives GOE(n) with W_ii ~ N(0, 2), W_ij ~ N(0, 1)).
 * Two products of the state, Q x then Q^T x, and their scaled sum, on the state's stream;
 * T_max counts both.  Batched states: every trial square, vectors packed.  x, y: distinct
 * device vectors of n (packed) elements in the state's dtype.  Errors: HD_ERR_ARG (not
 * Ginibre, null or aliased vectors), HD_ERR_DIM (a trial with m != n), HD_ERR_TMAX (fewer than
 * two products left), HD_ERR_OOM (the intermediate vector, allocated on first use), and those
 * of hd_apply.
 *
 * hd_usv_apply: the product with Q = U Sigma V (eq. inv): U = the Haar(m) state `U`, V = the
 * Haar(n) state `V`, Sigma the m x n rectangular diagonal matrix with s[0..min(m,n)) (device
 * FP64 array) on its diagonal.  transpose = 0: y = U (Sigma (V x)), x of length n, y of m;
 * transpose = 1: y = V^T (Sigma^T (U^T x)), x of length m, y of n.  One product of each state
 * per call; both single-trial, same dtype, device and stream.  Intermediates live in U (two
 * vectors of max(m, n), allocated on first use).  Errors: HD_ERR_ARG (wrong ensembles,
 * batched, mismatched dtype / stream, null pointers, U == V), HD_ERR_TMAX, HD_ERR_OOM, and
 * those of hd_apply. */
HD_API int hd_goe_apply(hd_state* st, const void* x, void* y);
HD_API int hd_usv_apply(hd_state* U, hd_state* V, const double* s, const void* x, int transpose, void* y);

/* Measured rate of the FP64 fused multiply-add pipe of the current device, in TFLOP/s (2 flops
 * per FMA): the roofline of the FP64 form, whose streaming passes are bound by this pipe rather
 * than by HBM on this GPU.  A measurement helper with no counterpart in the paper.  Runs
 * reps + 1 launches (the first untimed) of a kernel in which every thread advances 8
 * independent FMA chains for `iters` iterations over 8 CTAs of 256 threads per SM, timed with
 * CUDA events on `stream` (NULL = legacy default stream); *tflops_host receives the best
 * timed launch.  Synchronises the stream; allocates no device memory.  Errors: HD_ERR_ARG
 * (iters or reps < 1, null output), HD_ERR_CUDA. */
HD_API int hd_fp64_fma_rate(int32_t iters, int32_t reps, double* tflops_host, void* stream);

/* ---- Complex ensembles ---------------------------------------------------------------
 * The paper's section "Other Random Matrix Ensembles" carries Householder Dice over to
 * complex matrices, with M^T replaced by M^H and the complex reflector of eq.
 * Householder_c, H(v) = -e^{-i theta}[I - w w^H / (1 + r)], w = v/||v|| + e^{i theta} e_1,
 * v_1/||v|| = r e^{i theta} (theta = 0 when v_1 = 0), which maps v to ||v|| e_1.  The
 * reflectors enter as adjoints where they act on the left of the revealed block:
 *   Q ~ Haar(U(n)) (Algorithm 2):
 *     M_t = Q:    p = R_{t-1}...R_1 x, R_t = H_t(p), L_t = H_t(g_t), y = L_1^H...L_t^H R_t p;
 *     M_t = Q^H:  the mirror image with L and R exchanged;
 *   Q ~ CGin(m, n), entries sigma CN(0, 1) (Algorithm 1):
 *     M_t = Q:    R_r = H_r(R_{r-1}...R_1 x), u_t = L_1^H...L_l^H (Z g_t), v_t = R_1^H...R_r^H e_r,
 *                 y = sum_{i <= t} (v_i^H x) u_i;
 *     M_t = Q^H:  the mirror image (L_l = H_l(L_{l-1}...L_1 x), u_t = L_1^H...L_l^H e_l,
 *                 v_t = R_1^H...R_r^H (Z g_t), y = sum_i (u_i^H x) v_i).
 * Draws: entry i of g_t is (N_{2i} + i N_{2i+1}) / sqrt(2), N the standard normals of step
 * t's Philox stream (key = seed, counter = (i, t, trial, 0): one Box-Muller pair per entry);
 * Ginibre draws are scaled by sigma and masked to the unrevealed rows.
 *
 * hd_complex_create: a single-trial state for ensemble HD_HAAR (Q ~ Haar(U(n)), m == n, else
 * HD_ERR_DIM) or HD_GINIBRE (Q ~ CGin(m, n)); 1 <= T_max <= min(m, n, 256) (HD_ERR_TMAX
 * otherwise).  dtype HD_F64 stores vectors, stacks and (Ginibre) basis stores as interleaved
 * complex FP64 pairs (re, im); HD_F32 as complex FP32 pairs with FP32 streaming arithmetic,
 * and FP64 for every cross-thread sum, the reflector coefficients, the phases and the
 * compact-WY factor S.  Allocates everything up front (two stacks of n x T_max and m x T_max
 * complex elements, for Ginibre two basis stores of the same sizes, two T_max x T_max FP64
 * complex factors, work vectors); *out is owned by the caller (hd_complex_destroy).
 * hd_complex_set_options: the Ginibre entry scale sigma (> 0, finite; ignored for Haar), the
 * Philox trial word (changing either after the first step gives HD_ERR_ARG; reset first)
 * and the CUDA stream the work goes on (NULL = legacy stream).
 * hd_complex_apply: y = Q x (adjoint = 0; x of n entries, y of m) or y = Q^H x (adjoint = 1;
 * x of m, y of n), x and y distinct device vectors of complex elements aligned to one element
 * (16 bytes for HD_F64, 8 for HD_F32; HD_ERR_ARG otherwise); enqueued on the stream.
 * HD_ERR_TMAX after T_max products (state unchanged); after a launch failure (HD_ERR_CUDA)
 * the state stays poisoned until reset.
 * hd_complex_gue_apply: y = W x for W = (Q + Q^H)/sqrt(2) ~ GUE(n) (sigma = 1: W_ii ~ N(0, 1),
 * W_ij ~ CN(0, 1)), Q the square complex Ginibre matrix of the state (HD_ERR_ARG for Haar or
 * m != n): a Q and a Q^H product (T_max counts both; HD_ERR_TMAX when fewer than two are left)
 * and their scaled sum, with the intermediate in a state-owned vector.
 * hd_complex_reset: forget all steps and re-key with seed (synchronises the stream).
 * hd_complex_get_counts: products so far. */
typedef struct hd_cstate hd_cstate;
HD_API int hd_complex_create(int ensemble, int64_t m, int64_t n, int32_t T_max, uint64_t seed, int dtype,
                             hd_cstate** out);
HD_API int hd_complex_set_options(hd_cstate* st, double sigma, uint32_t trial, void* stream);
HD_API int hd_complex_apply(hd_cstate* st, const void* x, int adjoint, void* y);
HD_API int hd_complex_gue_apply(hd_cstate* st, const void* x, void* y);
HD_API int hd_complex_reset(hd_cstate* st, uint64_t seed);
HD_API int hd_complex_get_counts(const hd_cstate* st, int32_t* t);
HD_API void hd_complex_destroy(hd_cstate* st);

/* Number of kernels this state has launched (graph replays count their kernels). */
HD_API int hd_get_launches(const hd_state* st, int64_t* launches);

/* Human-readable name of a status code (static string). */
HD_API const char* hd_status_string(int status);

/* The library's Gaussian draws, exposed for checking the generator:
 * out[k] = the normal of absolute index start+k of (seed, trial, step, stream), as
 * defined for hd_create (Box-Muller on 53-bit uniforms in FP64 for HD_F64; the same
 * Philox words through a 32-bit Box-Muller for HD_F32).  out is a device buffer of count
 * elements of the dtype.  Enqueued on `stream`. */
HD_API int hd_philox_normals(uint64_t seed, uint32_t trial, uint32_t step, uint32_t stream_id,
                             int64_t start, int64_t count, int dtype, void* out, void* stream);

/* Raw Philox4x32-10 words: for block b < nblocks, counter = counters[4b .. 4b+3] and key =
 * seed; out[4b .. 4b+3] = the four output words.  Both are device buffers. */
HD_API int hd_philox_words(uint64_t seed, const uint32_t* counters, int64_t nblocks,
                           uint32_t* out, void* stream);

/* ---- Reverse mode (adjoint) ---------------------------------------------------------
 * With the Gaussian draws held fixed, y_1..y_T of Algorithms 1 and 2 are a deterministic,
 * almost everywhere differentiable function of the step inputs x_1..x_T.  y_t depends on x_t
 * directly and on earlier inputs through the data-side reflectors they built (R_s = H_s(p_s),
 * eq. Householder_e) and, for Gin, through the basis vectors built with them (Alg. 1).  The
 * paper has no gradients; this is the pathwise derivative of the sampler, so it is an
 * unbiased estimator of the derivative of an expectation, not the derivative for a fixed
 * dense Q.  The sign choices of the reflectors are piecewise constant and pass no
 * derivative; an identity reflector (zero tail) passes none either.  A batched state whose
 * trials all have the same dimensions reverses all its trials at once (packed vectors, one
 * set of launches per reverse step); batches of unequal trials give HD_ERR_ARG.
 *
 * hd_adjoint_enable(st, flags): call on a fresh or just-reset state (no step taken).  From
 * then on every forward step is recorded; with HD_ADJ_RECORD_X the library also keeps a copy
 * of each x_t (T_max vectors of the longer dimension, state dtype), otherwise the caller
 * passes x_t back to hd_adjoint_step (recomputing them, e.g. from checkpoints with hd_probe_at).
 * Allocates the accumulators once, per trial: per stack dim x T_max elements of the state dtype
 * (dV) and T_max^2 FP64 (dS), per Gin basis store dim x T_max of the state dtype, plus 4 work
 * vectors; with HD_ADJ_RECORD_X one packed input vector per step.
 * The streaming passes compute in the state's precision with FP64 cross-thread sums, as the
 * forward sweeps do.  hd_run on a recording state
 * runs without its CUDA graph.  Errors: HD_ERR_ARG (batch of unequal trials, unknown flag),
 * HD_ERR_STATE (steps already taken), HD_ERR_OOM, HD_ERR_CUDA. */
#define HD_ADJ_RECORD_X 1
HD_API int hd_adjoint_enable(hd_state* st, int flags);

/* Reverse the latest forward step not yet reversed (step t, counting down from the last).
 * ybar: dLoss/dy_t, a device buffer of y_t's length (state dtype; packed for a batch).  x_t:
 * the step's input (device, x_t's length) or NULL to use the recorded copy.  xbar (device, x_t's length)
 * receives dLoss/dx_t through y_t and through every later product that used a reflector or
 * basis vector built from x_t (their contributions were accumulated when those later steps
 * were reversed).  It does not include the caller's own f_t: the caller adds
 * d x_{t+1} / d x_t terms itself.  Enqueued on the state's stream.  Once a reverse pass has
 * started, hd_apply returns HD_ERR_STATE until hd_reset or hd_adjoint_restart.
 * Errors: HD_ERR_STATE (not enabled, or every step reversed), HD_ERR_ARG, HD_ERR_CUDA. */
HD_API int hd_adjoint_step(hd_state* st, const void* ybar, const void* x_t, void* xbar);

/* Zero the accumulators and set the reverse pass back to the last forward step, so that
 * another loss can be differentiated through the same forward trajectory. */
HD_API int hd_adjoint_restart(hd_state* st);

/* Number of forward steps not yet reversed. */
HD_API int hd_adjoint_position(const hd_state* st, int32_t* remaining);

/* Allocation-free first product of a fresh matrix.  The paper has no counterpart of this
 * entry point: it is a library convenience for callers that must not allocate device
 * memory, such as code whose framework already holds the device memory in its own pool
 * (a cudaMalloc outside that pool can fail or fragment it) or code on a latency-critical
 * stream (cudaMalloc / cudaFree may synchronise the whole device).
 *
 * Computes y = Q x (transpose == 0: x has n entries, y has m) or y = Q^T x (transpose != 0:
 * x has m, y has n) for the matrix that hd_create(ensemble, m, n, T_max, seed, dtype) with
 * options (sigma, trial) would sample, at its step 1: the result equals that state's first
 * hd_apply up to rounding, namely y = ||x|| g / ||g|| for Haar(n) and y = ||x|| g for
 * Gin(m, n), g the step-1 Philox draw of the output space (entry scale sigma for Gin; sigma
 * is ignored for Haar).  x and y are device buffers of dtype on the calling thread's current
 * device, not overlapping; work is enqueued on `stream` (NULL = the legacy default stream).
 *
 * Scratch: one file-scope device array of 66,048 bytes per device holds the per-tile partial
 * sums, a tile counter and the coefficient, which bounds max(m, n) at 16,777,216 entries.
 * The counter must be zero when the norm kernel starts: every call clears it on `stream`
 * first.  Calls that overlap on one device (on different streams, or from different host
 * threads without ordering) share that array and race on it, giving wrong results: order
 * them on one stream.  Every call looks up the array's device address on the current device
 * (cudaGetSymbolAddress); the first lookup on a device can load the library's device code,
 * so a caller that captures the call into a CUDA graph should make one call before beginning
 * the capture.  The call allocates no device memory.
 *
 * Errors: HD_ERR_ARG (bad ensemble or dtype, NULL x or y, m or n <= 0, Gin sigma not finite
 * and positive), HD_ERR_DIM (Haar with m != n; max(m, n) above 16,777,216, with the limit in
 * hd_last_error), HD_ERR_CUDA (set-up or launch failure, text in hd_last_error). */
HD_API int hd_first_product_noalloc(int ensemble, int dtype, int64_t m, int64_t n, int transpose,
                                    uint64_t seed, uint32_t trial, double sigma, const void* x,
                                    void* y, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* HD_H */
