// Kernel argument blocks and launchers of the Householder Dice step (sm_103a).
//
// Representation (Remark after Algorithm 1: products of reflectors in compact storage,
// Schreiber & Van Loan).  A stack of k generalised reflectors H_j(a_j) = D_j P_j, j = 0..k-1
// (0-based pivot j), with P_j = I - tau_j u_j u_j^T, u_j = a_j[j:] + s_j ||a_j[j:]|| e_j and
// D_j = diag(I_j, -s_j I) (the scalar -sign of eq. Householder), is kept as
//   V = [u_0 .. u_{k-1}]           column-major, dim x T_max, column j zero above row j,
//   S   (k x k, upper triangular)  P_0 P_1 ... P_{k-1} = I - V S V^T,
//   G = V^T V                      (k x k, FP64),
//   dpre[q] = prod_{j<q} (-s_j)    (D_j commutes with P_i for i >= j, so the signs collect
//                                   into the diagonal Delta_k[i] = dpre[min(i, k-1) + 1]).
// Then   H_{k-1}...H_0 = Delta_k (I - V S^T V^T)      ("forward" product, first acts first)
//        H_0...H_{k-1} = (I - V S V^T) Delta_k        ("backward" product).
// A step needs two streaming passes over the data-side stack (z = V^T x, then
// p = Delta (x - V S^T z)) and one over the other stack (the output), see hd_kernels.cu.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "hd_common.cuh"

namespace hd {

// Offsets of the FP64 scalar slots in Ws::scal.
enum ScalSlot {
  kPpiv = 0,     // data-side p at the pivot row
  kAlpha = 1,    // ||p[k:]||
  kCoef = 2,     // Haar: alpha / ||g[k:]||
  kUpivG = 3,    // Haar: pivot entry of the new random-side reflector vector
  kGFlag = 4,    // Haar: 1 when g[k:] = 0 (the random reflector is the identity)
  kErr = 5,      // device error word (0 = fine)
  kNumScal = 8
};

struct StackDev {
  void* V;        // T*, column-major, dim x Tm with leading dimension ld
  int64_t ld;
  int64_t dim;
  double* S;      // Tm x Tm, S[i + j*Tm], upper triangular
  double* dpre;   // Tm + 1 prefix signs, dpre[0] = 1
  void* gbuf;     // T*, dim: the next Gaussian draw in this stack's space (rows >= count)
  double* gdot;   // Tm + 1: dots of gbuf with the stack's columns (rows >= count)
  double* gg;     // 1: squared norm of gbuf over rows >= count + 1 (pivot excluded)
};

struct Ws {
  double* z;      // 2 Tm: x . data-stack columns, then x . data-space basis columns (Ginibre)
  double* w;      // Tm: S^T z
  double* phead;  // Tm + 1: p rows < k
  double* wout;   // Tm: output coefficients (Haar w'; Ginibre w_h)
  double* wout2;  // Tm: Ginibre w_2
  double* scrb;   // 4 scratch vectors of scr_stride doubles (V^T u, top-block products, sums)
  int64_t scr_stride;
  double* scal;   // kNumScal
  double* part;   // per-CTA partial sums
  double* gpart;  // per-group partial sums
  unsigned int* cnt;  // election counters: [kCntSets][kMaxGroups + 1]; set 3, slot 0: step flag
  unsigned int* err;  // device error word: bit 0 = a bounded mbarrier wait expired
  __device__ __forceinline__ double* scr(int i) const { return scrb + i * scr_stride; }
};
constexpr int kMaxGroups = 512;
// Counter sets of a trial's workspace: the elections of K1, K2 and K3, then the flag that
// hands the update sweep's results to the output sweep inside the step kernel (and, in trial
// 0's set only, the step kernel's two work queues and its count of finished CTAs).
constexpr int kCntSets = 4;
constexpr int kStepFlagSlot = 3 * (kMaxGroups + 1);
constexpr int kStepQueueSlot = kStepFlagSlot + 1;

struct Grid {
  int ctas;         // CTAs of the sweep
  int64_t vpc;      // 16-byte vectors per CTA
  int gsize;        // CTAs per election group
  int ngroups;
};

// Launch shape of one sweep: W warps per CTA (each walking 32-row sub-tiles), nbuf
// sub-tile buffers per warp, persistent grid.
struct SweepCfg {
  int W;
  int nbuf;
  int per_sm;       // CTAs of this shape resident per SM (host bookkeeping)
  Grid g;
  int tag;          // host bookkeeping (profiling): kernel | column bucket << 4
};

// Dynamic shared memory of a sweep (the carve of WtSmem: W * nbuf stages of ncolT columns and
// NRV row vectors of 32 elements, W * 2 scratch row vectors, two coefficient arrays padded to
// 16 bytes, and the W * NR * ncolC FP64 column sums; every section rounded up to 16 bytes).
template <typename T>
inline size_t sweep_smem_bytes(int W, int nbuf, int ncolT, int NRV, int ncolC, int NR) {
  constexpr int NCH = 32 * (int)sizeof(T) / 16;   // 16-byte chunks per 32-row column
  auto r16 = [](size_t b) { return (b + 15) & ~(size_t)15; };
  const size_t cpad = (size_t)(ncolT + NCH - 1) / NCH * NCH;
  return r16((size_t)W * nbuf * (ncolT + NRV) * 32 * sizeof(T)) + r16((size_t)W * 2 * 32 * sizeof(T)) +
         r16(2 * cpad * sizeof(T)) + r16((size_t)W * NR * (ncolC > 0 ? ncolC : 1) * sizeof(double));
}

// The three sweeps of one step plus the first draw; T = float or double.
template <typename T>
struct StepPlan {
  int ens;              // 0 Ginibre, 1 Haar
  int Tm;
  int kD, kN;           // reflectors in the data / other stack before the step
  StackDev D, N;        // data-side and other stack
  void* Bd;             // Ginibre: basis columns living in the data space (kN of them)
  int64_t ldBd;
  void* Bn;             // Ginibre: basis columns living in the other space (kD + 1 after)
  int64_t ldBn;
  const T* x;
  T* y;
  Ws ws;
  DrawKey key_next;     // the next step's draw (t + 1)
  T sigma;              // entry scale of the draws (Ginibre), 1 for Haar
  SweepCfg c1, c2, c3;  // launch shapes of the three sweeps
  int pdl;              // launch with programmatic dependent launch
  int fin_out;          // the update and fused output sweeps call their finalisations out of line
                        // (batches: every trial has a finaliser)
  int step_ctas;        // > 0: K2 and the fused K3 run as one step kernel (k_step) of this many
                        // CTAs (cooperative launch; c2.W == c3.W) with step_smem bytes of
  int step_smem;        // dynamic shared memory
  // Fused trajectories (hd_run, Q / Q^T alternating, elementwise f_t): K3 also applies the
  // dynamics x_{t+1} = f(y_t, x_{t-1}) and forms the next step's K1 results (z, h, w), so the
  // next step skips K1.
  int fuse;             // this step's K3 is the fused one
  int skip_dots;        // this step's K1 was done by the previous step's fused K3
  int dyn;              // kDynTanh or kDynSignMem
  T dyn_a;
  T* xnext;             // x_{t+1} (output space, packed base); written by the fused K3
  const T* xprev;       // x_{t-1} (output space, packed base); may alias xnext
  // AMP in the fused Ginibre K3 (dyn == kDynAmp), per trial: amp_mode 1 = after Q beta
  // (y = Q beta + w, z = y), 2 = after Q^T z (x = eta(x + s; a ||z|| / sqrt(m))), 3 = after Q x
  // (z = y - q + z ||x||_0 / m).  Vectors in the output space (packed bases).
  int amp_mode;
  T* amp_v;             // updated in place: z (modes 1, 3) or x (mode 2)
  T* amp_y;             // y = Q beta + w: written in mode 1, read in mode 3
  const T* amp_w;       // the noise w (mode 1)
  double* amp_zsq;      // per trial ||z||^2: written in modes 1 and 3, read in mode 2
  int* amp_nnz;         // per trial ||x||_0: written in mode 2, read in mode 3
  // ISTA in the same sweep (dyn == kDynIsta): mode 2 is x = eta(x + amp_tau Q^T z; dyn_a) with
  // the fixed threshold dyn_a, mode 3 is z = y - Q x (no Onsager term)
  T amp_tau;
  // Trajectory records of the fused K3 (hd_run's y_record / x_record / x_given; null = off),
  // output-space packed bases of this step's rows: y_t, the library's own f_t result, and
  // the caller's replacement of that result (teacher forcing).
  T* yrec;
  T* xrec;
  const T* xgiven;
};

// ------------------------------------------------------------------------------------
// Batches.  A state holds `count` independent trials (one for the single-trial API); every
// trial has its own stacks, basis stores and workspace, packed in shared allocations.  A
// launch covers all trials: the CTA map of a space (0: the n-dimensional space of R, 1: the
// m-dimensional space of L) gives each CTA its trial and a contiguous range of 32-row
// sub-tiles; elections and finalisations are per trial.
struct TrialDesc {
  StackDev st[2];
  void* basis[2];
  int64_t ldb[2];
  Ws ws;
  uint32_t trial;       // Philox trial word
  int64_t off[2];       // offset of the trial's vector in packed n-space / m-space buffers
  double sigma;         // entry scale of the trial's draws (Ginibre), 1 for Haar
};

struct CtaMap {
  const int* cta_trial; // [ctas]: trial of each CTA
  const int* cta0;      // [count]: first CTA of each trial (trials laid out largest first)
  const int* nct;       // [count]: CTAs of each trial (contiguous from cta0)
  const int* spc;       // [count]: sub-tiles per CTA of each trial
  int ctas;             // CTAs of a launch over this space
};

template <typename T>
struct BatchStep {
  StepPlan<T> base;     // fields shared by all trials (pointers filled per trial)
  int d;                // data-side stack index (0 for M_t = Q, 1 for Q^T)
  const TrialDesc* desc;
  CtaMap map[2];
};

template <typename T>
cudaError_t launch_first_draw(const BatchStep<T>& b, int space, DrawKey key,
                              cudaStream_t s);
// ev (optional): start/stop event pairs recorded around K1, K2, K3 (ev[2*kind], ev[2*kind+1]);
// a null entry skips the record.  launched[kind] is set to 1 for each sweep launched;
// launched[1] = 2 (and the K2 events) when the step kernel ran K2 and K3 as one launch.
template <typename T>
cudaError_t launch_step(const BatchStep<T>& b, cudaStream_t s, cudaEvent_t* ev = nullptr,
                        int* launched = nullptr);
template <typename T>
cudaError_t launch_probe(const BatchStep<T>& b, double* q, double* unrevealed, cudaStream_t s);

template <typename T>
int kernel_occupancy(int which, size_t dynsmem);
// CTAs of the step kernel (Haar or Ginibre) resident per SM with `threads` threads and dynsmem
// bytes of dynamic shared memory (0 when it does not fit).
template <typename T>
int step_kernel_occupancy(bool haar, int threads, size_t dynsmem);
template <typename T>
int kernel_static_smem(int which);
template <typename T>
cudaError_t set_sweep_smem_limit(int bytes);

cudaError_t launch_philox_normals(DrawKey key, int64_t start, int64_t count, int dtype, void* out,
                                  cudaStream_t s);
cudaError_t launch_wait_selftest(unsigned* err, unsigned limit, cudaStream_t s);
cudaError_t launch_philox_words(uint32_t k0, uint32_t k1, const uint32_t* ctr, int64_t nblocks,
                                uint32_t* out, cudaStream_t s);

}  // namespace hd
