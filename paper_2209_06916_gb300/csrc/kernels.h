// Launch interface of the MGRIT device kernels (internal to the library).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

namespace mg {

// Kernel attributes (dynamic shared memory limits, non-portable cluster
// sizes) are set per device: `f` runs the first time a call site sees the
// current device, under the site's mutex, so a process driving several GPUs
// configures each of them and concurrent first launches wait for it.
template <typename F>
inline void once_per_device(std::mutex& mu, uint64_t& done, F f) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    dev = 0;
  }
  const uint64_t bit = 1ull << (dev & 63);
  std::lock_guard<std::mutex> lk(mu);
  if (!(done & bit)) {
    f();
    done |= bit;
  }
}

constexpr int kMaxTaps = 1024;   // composite level-0 stencil taps (folded mod nx)
constexpr int kMaxRounds = 5;    // in-warp chunk-scan rounds (distances 1..16)
constexpr int kPMax = 64;        // chunk length of the in-block banded solves

// ---------------------------------------------------------------------------
// Level-0 composite stencil: out[r] = sum_t a_t in[r][i+t] (+ rhs[r]) (- sub[r])
// for rows r = 0..rows-1 (pointers are pre-offset by the caller).  With
// `partial`, each CTA also writes sum(out^2) of its tile (FP64).
// ---------------------------------------------------------------------------
template <typename T>
struct StencilParams {
  const T* in;
  T* out;
  const T* rhs;
  const T* sub;
  double* partial;
  int64_t nx;
  int64_t rows;
  int64_t ld;          // row stride of in / out / rhs / sub in elements (0: nx)
  int lo;
  int ntaps;
  int tile_r;          // outputs per thread (tile = 256 * tile_r points); 0 = by n_x
  int persistent;      // 1: one wave of CTAs looping over the tiles, the next tile's
                       // window fetched (cp.async) while the current one computes
  T taps[kMaxTaps];
};

int stencil_tiles(int64_t nx, int tile_r = 0);
// Launch; returns the number of CTAs (= partial slots written).
int64_t launch_stencil_rows(const StencilParams<double>& p, cudaStream_t st);
int64_t launch_stencil_rows(const StencilParams<float>& p, cudaStream_t st);

// ---------------------------------------------------------------------------
// Periodic banded solve tables (one recurrence direction).  A vector of n
// points is split over C CTAs of a thread-block cluster, each CTA over NT
// chunks of P points (one chunk per thread).  The carry between chunks is
// found by an intra-CTA Hillis-Steele scan (transfer powers Mpow), then a
// cluster-level sum over the previous `jterms` CTAs' aggregates (McPow, the
// closure Clc when the sum wraps the whole ring), then the per-chunk term
// M^t X (device table Mt, t < tcut; beyond tcut it is below 1e-18).
// ---------------------------------------------------------------------------
template <typename T>
struct SolveDir {
  int h;
  int rounds;
  int tcut;
  int jterms;
  int closure;
  int wterms;          // cross-warp terms (warp totals combined per chunk)
  int dcut;            // lanes with distance d <= dcut from the warp edge need M^d
  T ncoef[3];          // negated recurrence coefficients
  T Mpow[kMaxRounds][9];
  T Mlane[32][9];      // M^d, d = 1..32 (index d - 1)
  T M32pow[8][9];      // (M^32)^j, j = 0..wterms-1
  T McPow[16][9];
  T Clc[9];
  T G[kPMax * 3];      // impulse responses G[j*3+q]
  const T* Mt;         // tcut x 9 (device)
};

// Coarse-level step Phi_l v + g: SL gather (weights pre-scaled by 1/kappa),
// then the factored periodic solve (causal then anticausal recurrences).
enum CoarseMode { kModeCF = 0, kModeFRES = 1, kModeFOUT = 2, kModeSEQ = 3, kModeAPPLY = 4 };

// largest GMRES iteration cap of the coarse kernel's correction solves
constexpr int kGmMax = 32;

// TS: storage / SL-gather precision; TC: precision of the banded correction
// solve (and of its tables).
template <typename TS, typename TC = TS>
struct CoarseParams {
  typedef TS T;
  int n, P, nthr;
  int csize;           // CTAs per vector (thread-block cluster size)
  int npc;             // points per CTA = nthr * P
  int p1;              // p + 1 SL weights
  int jlo;             // node offset of weight 0: -(p+1)/2
  int kshift;          // SL shift k_l mod n
  int shift;           // y_i = v_{i+shift}
  T w[8];
  SolveDir<TC> c, a;
  int mode;
  int zero_start;
  int nsteps;
  int m;
  int nosolve;         // 1: Psi = S (direct SL coarse operator, no correction solve)
  int64_t K;
  const T* start;
  T* g;                // RHS rows; FOUT / SEQ overwrite the rows they consumed with the
                       // level's values there (C-points and F-relaxed points), which the
                       // host then adds into the parent level
  T* out;
  const T* sub;
  T* parent;           // unused by the kernel (kept for the host's bookkeeping)
  double* partial;     // FRES: one slot per CTA (K * csize)
  // GMRES correction solves (Sec. 6.1, Sec. 6.3), used when gm_max > 0: the
  // SL weights w are then unscaled and the system is (I - sum phi D) x = S v
  int gm_max;                    // iteration cap (<= kGmMax); 0: exact banded solve
  double gm_rtol;                // stop at ||b - A x_k|| <= gm_rtol ||b||
  TC gm_taps[7];                 // the matrix's taps at offsets -3..3
  TC* gm_V;                      // Krylov basis scratch: K x (gm_max + 1) x n values
  unsigned long long* gm_stats;  // [0] += GMRES iterations, [1] += solves (may be null)
};

// bytes of dynamic shared memory of the coarse kernel; gm_elem = sizeof of
// the GMRES vector type (0: no GMRES)
size_t coarse_smem_bytes(int npc, int P, int nthr, int elem, int gm_elem = 0);

// ---------------------------------------------------------------------------
// Level-0 SDIRK step kernel: m (or nsteps) steps of Phi = R_q(-c L_p) for an
// SDIRK method, one CF-interval per thread-block cluster.  A step is a small
// program over shared-memory vector slots (slot 0 holds the state):
//   COPY  dst = src          ZERO  dst = 0          AXPY  dst += c src
//   AXPYL dst += c L_p src   SOLVE dst = kappa (I + gamma c L_p)^{-1} src
//   AXPBY dst = c2 dst + c src
// (the solve leaves out the 1/kappa of its factorisation; the host keeps a
// scale per slot, folds it into the coefficients and undoes it once per
// step with rscale)
// built on the host from the tableau (stiffly accurate stages) or from the
// factored stability function (SDIRK5).
// ---------------------------------------------------------------------------
enum SdirkOpKind { kOpCopy = 0, kOpZero = 1, kOpAxpy = 2, kOpAxpyL = 3, kOpSolve = 4, kOpAxpby = 5 };
constexpr int kSdirkMaxOps = 40;
constexpr int kSdirkMaxSlots = 6;

template <typename T>
struct SdirkParams {
  int n, P, nthr, csize, npc;
  int p1, llo;         // L_p taps at offsets llo = -p1/2 .. llo + p1 - 1
  T ltaps[8];
  SolveDir<T> c, a;    // factored stage matrix (I + gamma c L_p)
  T sscale;            // 1/kappa of the factorisation (folded into the op coefficients)
  T rscale;            // end of step: slot 0 = rscale * slot `result` (undoes the folded scales)
  int nops, nslots, result;
  int opk[kSdirkMaxOps], opd[kSdirkMaxOps], ops[kSdirkMaxOps];
  int opg[kSdirkMaxOps];   // AXPYL group head: number of consecutive AXPYL ops on the same src (else 1)
  int opb[kSdirkMaxOps];   // 1: barrier over the vector's threads before the op (halo hazards)
  int resb;                // barrier before the end-of-step copy result -> slot 0
  T opc[kSdirkMaxOps];
  T opc2[kSdirkMaxOps];  // AXPBY: dst = opc2 * dst + opc * src
  int mode;            // kModeCF, kModeFRES, kModeFOUT, kModeAPPLY, kModeSEQ
  int zero_start, nsteps;
  int m;               // coarsening factor (RHS row of step s of interval k: k m + s)
  int64_t K;
  const T* start;      // rows k
  const T* rhs;        // optional C-point RHS, rows k+1 (CF / FRES on level 0)
  T* g;                // optional RHS at every step (a rediscretised coarse level, as in
                       // CoarseParams): v <- Phi v + g_{k m + s}; FOUT / SEQ store each step's
                       // value into the row it consumed
  T* out;              // CF / FRES: rows k+1; APPLY: rows k; SEQ: row 0
  const T* sub;        // FRES: rows k+1
  double* partial;     // FRES: one slot per CTA
  T* traj;             // SEQ: state after every `every` steps, rows 0, 1, ...
  int every;
};
size_t sdirk_smem_bytes(int npc, int P, int nthr, int nslots, int elem);

// ---------------------------------------------------------------------------
// Level-0 SDIRK steps for many CF-intervals in FP64 (sdirk_seg.cuh): one CTA
// per interval, one segment of kSegLen points per thread in shared memory,
// the stage solves' recurrences entered through a warm-up over the
// neighbouring segment (where the neglected start state has decayed below
// 2^-56).  Stiffly accurate SDIRK with 1..3 stages, right-hand
// sides from the solves; modes CF, FRES (no C-point RHS) and APPLY.
// ---------------------------------------------------------------------------
constexpr int kSegPoints = 128;
struct SdirkSegParams {
  int n, T;              // points per vector, threads per CTA (n / kSegPoints)
  int rc1, rc2;          // causal warm-up: first section over rc1 points, second over the last
                         // rc2 of them (multiples of 8, rc2 <= rc1 <= kSegPoints)
  int ra1, ra2;          // the same for the anticausal recurrence
  int stages;            // 1..3
  // each recurrence direction as two cascaded sections (two independent
  // multiply-add chains): a first-order section y_i = b_i + r y_{i-1} (order
  // c1 / a1 = 0 or 1) feeding a section of order c2 / a2 <= 2,
  // x_i = y_i + d[0] x_{i-1} + d[1] x_{i-2} (anticausal: indices i+1, i+2)
  int c1, c2, a1, a2;    // section orders (the kernel's template)
  double cr, cd[2];      // causal sections
  double ar, ad[2];      // anticausal sections
  // unscaled solve U(b) = kappa (I + gamma c L)^{-1} b; stage 1: R2' = e1u2 u
  // + e1y2 U(u), aux = e1u3 u + e1y3 U(u); stage 2: aux += e2y3 Y2; the last
  // stage's output is scaled by `last`
  double e1u2, e1y2, e1u3, e1y3, e2y3, last;
  int mode, zero_start, nsteps;
  int64_t K;
  const double* start;   // rows k
  double* out;           // CF / FRES: rows k+1; APPLY: rows k (also the per-interval scratch)
  const double* sub;     // FRES: rows k+1
  double* partial;       // FRES: one slot per interval
};
size_t sdirk_seg_smem_bytes(int n);

// The FP32 stage kernel of MIXED inner cycles (sdirk_seg32.cuh): one CTA per
// interval, the three stage slots in shared memory, kSeg32Points per thread,
// the mat-vec form of the stages (R_j += g L Y_i), warm-ups cut at 2^-27;
// modes CF and FRES with the optional C-point rhs / sub of the FP32 paths.
constexpr int kSeg32Points = 64;
struct SdirkSeg32Params {
  int n, T;
  int rc1, rc2, ra1, ra2;
  int c1, c2, a1, a2;    // section orders (the kernel's template)
  int p1;                // L_p taps (the kernel's template: l(p) west, r(p) east)
  int stages;            // 1 or 3
  float cr, cd[2], ar, ad[2];
  float ik;              // 1/kappa of the factorisation (applied after each solve)
  float ltaps[8];
  float g[3];            // -c a_10, -c a_20, -c a_21
  int mode, zero_start, nsteps;
  int64_t K;
  const float* start;
  const float* rhs;      // optional, rows k+1
  float* out;            // CF / FRES: rows k+1
  const float* sub;      // optional, rows k+1
  double* partial;       // FRES: one slot per interval
};
size_t sdirk_seg32_smem_bytes(int n);
int launch_sdirk_seg32(const SdirkSeg32Params& p, cudaStream_t st);
// 1 on success, -1 on a launch error or an order the kernel lacks
int launch_sdirk_seg(const SdirkSegParams& p, cudaStream_t st);
// Chunk lengths the step kernels are compiled for (one chunk per thread).
constexpr int kChunkLens[4] = {4, 8, 16, 32};
// Largest co-schedulable cluster size <= want (power of two) for a CTA of
// nthr threads and smem bytes of dynamic shared memory.
int sdirk_max_cluster(int want, size_t smem, int nthr);
int launch_sdirk(const SdirkParams<double>& p, cudaStream_t st);
int launch_sdirk(const SdirkParams<float>& p, cudaStream_t st);
int launch_coarse(const CoarseParams<double>& p, cudaStream_t st);
int launch_coarse(const CoarseParams<float>& p, cudaStream_t st);
int launch_coarse(const CoarseParams<float, double>& p, cudaStream_t st);
int coarse_max_cluster(int want, size_t smem, int nthr);

// ---------------------------------------------------------------------------
// Utilities
// ---------------------------------------------------------------------------
// elementwise precision conversions over n values:
//   kCvtD2F: f[i] = (float) d[i]     kCvtF2D: d[i] = f[i]
//   kAddF2D: d[i] += f[i]            kAddD2F: f[i] += (float) d[i]
enum CvtOp { kCvtD2F = 0, kCvtF2D = 1, kAddF2D = 2, kAddD2F = 3, kAddD2D = 4, kAddF2F = 5 };
//   kAddD2D: d[i] += d2[i]          kAddF2F: f[i] += f2[i]   (d2 / f2: src)
void launch_convert(int op, double* d, float* f, int64_t n, cudaStream_t st, const double* d2 = nullptr,
                    const float* f2 = nullptr);
// Device-side state of a graph-resident MGRIT solve (stop test on the GPU).
struct DevSolveState {
  double r0, rnorm, tol;
  int it, max_iter, converged, status, hist_len, pad;
  // MIXED adaptive inner solve: FP32 V-cycles of one refinement step repeat
  // while the FP32 residual of the error equation is above the step's
  // target (inner_target) times the FP64 residual it corrects and still
  // falls by 0.8 per cycle, at most in_max cycles
  double in_rho0, in_prev, in_tol, in_base;
  int in_count, in_max, in_total, in_pad;
  double hist[128];
};
constexpr int kInnerMax = 16;
constexpr double kInnerTol = 1e-2;
constexpr double kInnerStall = 0.8;
// Target of one inner solve, relative to the FP64 residual it corrects:
// `base` (the handle's inner tolerance), or what the refinement still needs
// to end two orders under its stop level (0.01 tol r0 / current residual),
// whichever is larger.  One refinement step cuts the error by at most about
// kappa eps_FP32; an inner solve driven further leaves the error behind the
// residual, so the target never goes below `base`.
__host__ __device__ inline double inner_target(double tol, double r0, double rho0, double base) {
  const double need = rho0 > 0.0 ? 0.01 * tol * r0 / rho0 : base;
  return need > base ? (need < 0.1 ? need : 0.1) : base;
}
// First residual: r0, history[0]; sets the loop condition (0 when already
// converged).  Check: after each iteration, appends the norm and sets the
// condition to continue, or records converged / diverged / not converged.
void* solve_init_kernel_fn();
void* solve_check_kernel_fn();
void launch_solve_check(DevSolveState* s, const double* dnorm_sq, cudaGraphConditionalHandle hnd,
                        cudaStream_t st);
// Adaptive inner solve: init after the first (zero-guess) FP32 cycle from the
// FP64 residual norm; check after every further cycle from the FP32 one.
void launch_inner_init(DevSolveState* s, const double* dnorm64_sq, cudaGraphConditionalHandle hnd, cudaStream_t st);
void launch_inner_check(DevSolveState* s, const double* dnormf_sq, cudaGraphConditionalHandle hnd, cudaStream_t st);
// the continuation rule shared by the device check and the eager host loop
__host__ __device__ inline bool inner_continue(double rho, double prev, double rho0, int count, int max_count,
                                               double tol) {
  return rho == rho && rho <= 1e300 && rho > tol * rho0 && rho < kInnerStall * prev && count < max_count;
}
// sum of partial[0..n) in a fixed order, written to out[0] (FP64)
void launch_reduce_sum(const double* partial, int64_t n, double* out, cudaStream_t st);
// C-point iterate: row 0 = u0, rows k >= 1 uniform [0,1) at time index k*m
void launch_random_cpoints(double* uC, const double* u0, int64_t rows, int64_t nx, int m,
                           uint64_t seed, cudaStream_t st);

}  // namespace mg

namespace mg {
// ---------------------------------------------------------------------------
// GPU sequential time-stepping u_{n+1} = Phi u_n: one thread-block cluster
// per vector, the vector split over the cluster's CTAs in shared memory,
// halos exchanged through distributed shared memory once per pass of the
// composite stencil Phi^B.
// ---------------------------------------------------------------------------
constexpr int kSeqMaxTaps = 1024;
struct SeqParams {
  const double* u0;   // nx
  double* u_out;      // nx
  double* traj;       // optional rows written after every `every_passes` passes
  int64_t nx;
  int csize;          // CTAs per cluster
  int npc;            // points per CTA
  int halo_l, halo_r; // -lo, hi of the composite stencil
  int64_t passes;     // passes of the main stencil
  int every_passes;   // trajectory stride in passes (0: none)
  int lo, ntaps;
  double taps[kSeqMaxTaps];
  // tail: `tail_steps` single steps with the one-step stencil afterwards
  int tail_passes, tail_lo, tail_ntaps;
  double tail_taps[64];
};
int launch_seq(const SeqParams& p, cudaStream_t st);
int seq_max_cluster(int want, size_t smem);
}  // namespace mg
