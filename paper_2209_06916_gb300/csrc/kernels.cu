// MGRIT device kernels for sm_103a (GB300).
//
//  stencil_rows_kernel  level-0 relaxation: the fine map of one CF-interval,
//                       Phi^m = R_q(-c L_p)^m (Eq. MOL_M_def), applied as one
//                       composite periodic stencil to C-point rows (the m
//                       fine steps collapse into one wide stencil; the vector
//                       is read from HBM once per interval); optional RHS,
//                       subtraction (C-point residual, Sec. 2.2) and per-CTA
//                       sum of squares for the residual norm.
//  coarse_kernel        coarse-level steps v <- Phi_l v + g_n with
//                       Phi_l = (I - phi_l D)^{-1} S_p^{(m^l dt)} (Eq.
//                       MOL-SL-corrected and its multilevel form): SL
//                       Lagrange gather (Sec. 3) and the periodic banded
//                       solve as causal + anticausal linear recurrences
//                       over per-thread chunks, joined by a circular
//                       Hillis-Steele scan of the chunk carries.  Modes:
//                       C-relaxation after F (CF), F-relaxation + C-point
//                       residual (FRES), post F-relaxation added to the
//                       parent level (FOUT: the coarse-grid correction),
//                       sequential coarsest solve (SEQ), plain apply.
//  reduce_sum_kernel    fixed-order sum of per-CTA partials (deterministic).
//  random_cpoints_kernel  SplitMix64 random initial C-point iterate.
#include <cuda_runtime.h>
#include <stdint.h>

#include "kernels.h"

namespace mg {

// ---------------------------------------------------------------------------
// block reductions (fixed order)
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Sum over the block; result valid in thread 0.  `red` holds >= 32 doubles.
__device__ __forceinline__ double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < nw; ++w) s += red[w];
  return s;
}

// ---------------------------------------------------------------------------
// Level-0 composite stencil
// ---------------------------------------------------------------------------
constexpr int kStencilThreads = 256;

template <typename T, int R>
__global__ void __launch_bounds__(kStencilThreads)
    stencil_rows_kernel(const __grid_constant__ StencilParams<T> p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* s = reinterpret_cast<T*>(smem_raw);
  __shared__ double red[32];
  const int B = kStencilThreads;
  const int W = B * R;
  const int64_t row = blockIdx.x;
  const int64_t nx = p.nx;
  const int64_t x0 = (int64_t)blockIdx.y * W;
  const int nload = W + p.ntaps - 1;
  const T* in = p.in + row * nx;
  for (int j = threadIdx.x; j < nload; j += B) {
    int64_t gi = (x0 + p.lo + j) % nx;
    if (gi < 0) gi += nx;
    s[j] = in[gi];
  }
  __syncthreads();
  T acc[R];
#pragma unroll
  for (int r = 0; r < R; ++r) acc[r] = T(0);
  const T* sp = s + threadIdx.x;
  for (int t = 0; t < p.ntaps; ++t) {
    const T a = p.taps[t];
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] = fma(a, sp[B * r + t], acc[r]);
  }
  double sq = 0.0;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int64_t i = x0 + threadIdx.x + (int64_t)B * r;
    if (i < nx) {
      T v = acc[r];
      if (p.rhs) v += p.rhs[row * nx + i];
      if (p.sub) v -= p.sub[row * nx + i];
      p.out[row * nx + i] = v;
      sq += (double)v * (double)v;
    }
  }
  if (p.partial) {
    double tot = block_sum(sq, red);
    if (threadIdx.x == 0) p.partial[row * gridDim.y + blockIdx.y] = tot;
  }
}

static int stencil_r(int64_t nx) {
  if (nx >= 4 * kStencilThreads) return 4;
  if (nx >= 2 * kStencilThreads) return 2;
  return 1;
}

int stencil_tiles(int64_t nx) {
  int R = stencil_r(nx);
  return (int)((nx + (int64_t)kStencilThreads * R - 1) / ((int64_t)kStencilThreads * R));
}

template <typename T, int R>
static int64_t launch_stencil_r(const StencilParams<T>& p, cudaStream_t st) {
  const int W = kStencilThreads * R;
  size_t smem = (size_t)(W + p.ntaps - 1) * sizeof(T);
  static bool configured = false;
  if (!configured) {
    cudaFuncSetAttribute(stencil_rows_kernel<T, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         64 * 1024);
    configured = true;
  }
  dim3 grid((unsigned)p.rows, (unsigned)stencil_tiles(p.nx));
  stencil_rows_kernel<T, R><<<grid, kStencilThreads, smem, st>>>(p);
  return (int64_t)grid.x * grid.y;
}

template <typename T>
static int64_t launch_stencil_any(const StencilParams<T>& p, cudaStream_t st) {
  if (p.rows <= 0) return 0;
  switch (stencil_r(p.nx)) {
    case 4:
      return launch_stencil_r<T, 4>(p, st);
    case 2:
      return launch_stencil_r<T, 2>(p, st);
    default:
      return launch_stencil_r<T, 1>(p, st);
  }
}

int64_t launch_stencil_rows(const StencilParams<double>& p, cudaStream_t st) {
  return launch_stencil_any(p, st);
}
int64_t launch_stencil_rows(const StencilParams<float>& p, cudaStream_t st) {
  return launch_stencil_any(p, st);
}

// ---------------------------------------------------------------------------
// Coarse-level step kernel
// ---------------------------------------------------------------------------

// Circular Hillis-Steele scan of chunk carries: on return S holds the true
// recurrence state entering this thread's chunk (from chunk t-1 when
// dir = -1, from chunk t+1 when dir = +1).
template <int H, typename T>
__device__ __forceinline__ void chunk_scan(const T (&e)[H], T (&S)[H], const SolveDir<T>& D, T* sq,
                                           int t, int NT, int dir) {
  T Q[H];
#pragma unroll
  for (int a = 0; a < H; ++a) Q[a] = e[a];
  int buf = 0;
  for (int r = 0; r < D.rounds; ++r) {
#pragma unroll
    for (int a = 0; a < H; ++a) sq[(buf * 3 + a) * NT + t] = Q[a];
    __syncthreads();
    const int src = (t + dir * (1 << r)) & (NT - 1);
    T Qo[H];
#pragma unroll
    for (int a = 0; a < H; ++a) Qo[a] = sq[(buf * 3 + a) * NT + src];
#pragma unroll
    for (int a = 0; a < H; ++a)
#pragma unroll
      for (int q = 0; q < H; ++q) Q[a] = fma(D.Mpow[r][a * 3 + q], Qo[q], Q[a]);
    buf ^= 1;
  }
#pragma unroll
  for (int a = 0; a < H; ++a) sq[(buf * 3 + a) * NT + t] = Q[a];
  __syncthreads();
  const int src = (t + dir) & (NT - 1);
  T Rv[H];
#pragma unroll
  for (int a = 0; a < H; ++a) Rv[a] = sq[(buf * 3 + a) * NT + src];
  if (D.closure) {
#pragma unroll
    for (int a = 0; a < H; ++a) {
      T v = T(0);
#pragma unroll
      for (int q = 0; q < H; ++q) v = fma(D.Cl[a * 3 + q], Rv[q], v);
      S[a] = v;
    }
  } else {
#pragma unroll
    for (int a = 0; a < H; ++a) S[a] = Rv[a];
  }
}

// Periodic banded solve of the chunk x (in registers) in place:
// causal recurrence, carry scan, fixup fused with the anticausal local pass,
// carry scan, fixup.  Every thread of the block must call it.
template <int H, typename T, int PM>
__device__ __forceinline__ void banded_solve(T (&x)[PM], const CoarseParams<T>& A, T* sqc, T* sqa,
                                             int t) {
  const int P = A.P, NT = A.nthr;
  T e[H];
#pragma unroll
  for (int a = 0; a < H; ++a) e[a] = T(0);
#pragma unroll
  for (int j = 0; j < PM; ++j) {
    if (j < P) {
      T v = x[j];
#pragma unroll
      for (int q = 1; q <= H; ++q)
        if (j - q >= 0) v = fma(A.c.ncoef[q - 1], x[j - q], v);
      x[j] = v;
#pragma unroll
      for (int a = 0; a < H; ++a)
        if (j == P - 1 - a) e[a] = v;
    }
  }
  T S[H];
  chunk_scan<H>(e, S, A.c, sqc, t, NT, -1);
#pragma unroll
  for (int j = PM - 1; j >= 0; --j) {
    if (j < P) {
      T v = x[j];
#pragma unroll
      for (int q = 0; q < H; ++q) v = fma(A.c.G[j * 3 + q], S[q], v);
#pragma unroll
      for (int q = 1; q <= H; ++q)
        if (j + q < PM) {
          if (j + q < P) v = fma(A.a.ncoef[q - 1], x[j + q], v);
        }
      x[j] = v;
    }
  }
  T ea[H];
#pragma unroll
  for (int a = 0; a < H; ++a) ea[a] = x[a];
  T Sa[H];
  chunk_scan<H>(ea, Sa, A.a, sqa, t, NT, +1);
#pragma unroll
  for (int j = 0; j < PM; ++j) {
    if (j < P) {
      const int d = P - 1 - j;
      T v = x[j];
#pragma unroll
      for (int q = 0; q < H; ++q) v = fma(A.a.G[d * 3 + q], Sa[q], v);
      x[j] = v;
    }
  }
}

template <typename T, int PM, int P1>
__global__ void __launch_bounds__(256) coarse_kernel(const __grid_constant__ CoarseParams<T> A) {
  constexpr int H = P1 / 2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n = A.n, P = A.P, NT = A.nthr, t = threadIdx.x;
  const int npad = n + (n + P - 1) / P;
  T* sv = reinterpret_cast<T*>(smem_raw);
  T* sg = sv + npad;
  T* sqc = sg + npad;
  T* sqa = sqc + 6 * NT;
  double* red = reinterpret_cast<double*>(sqa + 6 * NT);
  const int64_t k = blockIdx.x;
  const int64_t nn = n;

  // initial state
  if (A.zero_start) {
    for (int i = t; i < n; i += NT) sv[i + i / P] = T(0);
  } else {
    const T* src = A.start + k * nn;
    for (int i = t; i < n; i += NT) sv[i + i / P] = src[i];
  }
  if (A.mode == kModeFOUT) {
    // the C-points themselves: parent row k m gets start[k]; the last CTA
    // also adds start[K] to parent row K m
    const T* src = A.start + k * nn;
    T* par = A.parent + k * A.m * nn;
    for (int i = t; i < n; i += NT) par[i] += src[i];
    if (k == A.K - 1) {
      const T* s2 = A.start + A.K * nn;
      T* p2 = A.parent + A.K * A.m * nn;
      for (int i = t; i < n; i += NT) p2[i] += s2[i];
    }
  }
  __syncthreads();

  const int64_t gbase = (A.mode == kModeSEQ) ? 0 : k * A.m;
  for (int s = 1; s <= A.nsteps; ++s) {
    if (A.g) {
      const T* gr = A.g + (gbase + s) * nn;
      for (int i = t; i < n; i += NT) sg[i + i / P] = gr[i];
    }
    T x[PM];
    if (s == 1 && A.zero_start) {
#pragma unroll
      for (int j = 0; j < PM; ++j) x[j] = T(0);
      __syncthreads();
    } else {
      // SL gather over the own chunk with a sliding window of P1 values:
      // (S v)_i = sum_a w_a v_{i - k + jlo + a}
      int idx = (t * P - A.kshift + A.jlo) % n;
      if (idx < 0) idx += n;
      T win[P1];
#pragma unroll
      for (int a = 0; a < P1 - 1; ++a) {
        int ii = idx + a;
        if (ii >= n) ii -= n;
        if (ii >= n) ii -= n;
        win[a] = sv[ii + ii / P];
      }
#pragma unroll
      for (int j = 0; j < PM; ++j) {
        if (j < P) {
          int ii = idx + j + P1 - 1;
          if (ii >= n) ii -= n;
          if (ii >= n) ii -= n;
          win[P1 - 1] = sv[ii + ii / P];
          T acc = T(0);
#pragma unroll
          for (int a = 0; a < P1; ++a) acc = fma(A.w[a], win[a], acc);
          x[j] = acc;
#pragma unroll
          for (int a = 0; a < P1 - 1; ++a) win[a] = win[a + 1];
        }
      }
      __syncthreads();
      banded_solve<H, T, PM>(x, A, sqc, sqa, t);
    }
    // new state v_{i - shift} = x_i + g
#pragma unroll
    for (int j = 0; j < PM; ++j) {
      if (j < P) {
        int i2 = t * P + j - A.shift;
        if (i2 < 0) i2 += n;
        if (i2 >= n) i2 -= n;
        T v = x[j];
        if (A.g) v += sg[i2 + i2 / P];
        sv[i2 + i2 / P] = v;
      }
    }
    __syncthreads();
    if (A.mode == kModeFOUT || A.mode == kModeSEQ) {
      T* par = A.parent + (gbase + s) * nn;
      for (int i = t; i < n; i += NT) par[i] += sv[i + i / P];
    }
  }

  if (A.mode == kModeCF) {
    T* o = A.out + (k + 1) * nn;
    for (int i = t; i < n; i += NT) o[i] = sv[i + i / P];
  } else if (A.mode == kModeAPPLY) {
    T* o = A.out + k * nn;
    for (int i = t; i < n; i += NT) o[i] = sv[i + i / P];
  } else if (A.mode == kModeFRES) {
    T* o = A.out + (k + 1) * nn;
    const T* sb = A.sub ? A.sub + (k + 1) * nn : nullptr;
    double sq = 0.0;
    for (int i = t; i < n; i += NT) {
      T r = sv[i + i / P];
      if (sb) r -= sb[i];
      o[i] = r;
      sq += (double)r * (double)r;
    }
    if (A.partial) {
      double tot = block_sum(sq, red);
      if (t == 0) A.partial[k] = tot;
    }
  }
}

size_t coarse_smem_bytes(int n, int P, int nthr, int elem) {
  size_t npad = (size_t)n + (size_t)((n + P - 1) / P);
  return (2 * npad + 12 * (size_t)nthr) * (size_t)elem + 32 * sizeof(double) + 16;
}

template <typename T, int PM, int P1>
static int launch_coarse_t(const CoarseParams<T>& A, cudaStream_t st) {
  size_t smem = coarse_smem_bytes(A.n, A.P, A.nthr, (int)sizeof(T));
  static bool configured = false;
  if (!configured) {
    cudaFuncSetAttribute(coarse_kernel<T, PM, P1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         227 * 1024);
    configured = true;
  }
  if (A.K <= 0) return 0;
  coarse_kernel<T, PM, P1><<<(unsigned)A.K, A.nthr, smem, st>>>(A);
  return 1;
}

template <typename T>
static int launch_coarse_any(const CoarseParams<T>& A, cudaStream_t st) {
  const bool big = A.P > 32;
  switch (A.p1) {
    case 2:
      return big ? launch_coarse_t<T, 64, 2>(A, st) : launch_coarse_t<T, 32, 2>(A, st);
    case 4:
      return big ? launch_coarse_t<T, 64, 4>(A, st) : launch_coarse_t<T, 32, 4>(A, st);
    case 6:
      return big ? launch_coarse_t<T, 64, 6>(A, st) : launch_coarse_t<T, 32, 6>(A, st);
    default:
      return -1;
  }
}

int launch_coarse(const CoarseParams<double>& p, cudaStream_t st) { return launch_coarse_any(p, st); }
int launch_coarse(const CoarseParams<float>& p, cudaStream_t st) { return launch_coarse_any(p, st); }

// ---------------------------------------------------------------------------
// utilities
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) reduce_sum_kernel(const double* __restrict__ a, int64_t n,
                                                          double* out) {
  __shared__ double red[32];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += a[i];
  double tot = block_sum(s, red);
  if (threadIdx.x == 0) out[0] = tot;
}

void launch_reduce_sum(const double* partial, int64_t n, double* out, cudaStream_t st) {
  reduce_sum_kernel<<<1, 1024, 0, st>>>(partial, n, out);
}

// SplitMix64 output function (Steele, Lea, Flood 2014; constants of Vigna's
// public-domain splitmix64.c), applied to seed + ctr * golden gamma.
__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t ctr) {
  uint64_t z = seed + ctr * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void random_cpoints_kernel(double* uC, const double* u0, int64_t rows, int64_t nx, int m,
                                      uint64_t seed) {
  const int64_t total = rows * nx;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = e / nx, i = e - k * nx;
    if (k == 0) {
      uC[e] = u0[i];
    } else {
      const uint64_t ctr = (uint64_t)(k * m) * (uint64_t)nx + (uint64_t)i + 1ull;
      uC[e] = (double)(splitmix64_at(seed, ctr) >> 11) * 0x1.0p-53;
    }
  }
}

void launch_random_cpoints(double* uC, const double* u0, int64_t rows, int64_t nx, int m,
                           uint64_t seed, cudaStream_t st) {
  int64_t total = rows * nx;
  int blocks = (int)((total + 255) / 256);
  if (blocks > 152 * 16) blocks = 152 * 16;
  random_cpoints_kernel<<<blocks, 256, 0, st>>>(uC, u0, rows, nx, m, seed);
}

}  // namespace mg

// ---------------------------------------------------------------------------
// GPU sequential stepping (baseline): persistent cluster kernel
// ---------------------------------------------------------------------------
#include <cooperative_groups.h>
namespace cg = cooperative_groups;

namespace mg {

constexpr int kSeqThreads = 256;

__device__ __forceinline__ void seq_pass(double* src, double* dst, int HL, int npc, int lo, int ntaps,
                                         const double* taps) {
  // dst[HL + i] = sum_t taps[t] src[HL + i + lo + t], i in [0, npc)
  for (int i = threadIdx.x; i < npc; i += blockDim.x) {
    const double* sp = src + HL + i + lo;
    double acc = 0.0;
    for (int t = 0; t < ntaps; ++t) acc = fma(taps[t], sp[t], acc);
    dst[HL + i] = acc;
  }
}

__device__ __forceinline__ void seq_halo(cg::cluster_group& cl, double* buf, int HL, int HR, int npc) {
  const int r = (int)cl.block_rank();
  const int C = (int)cl.num_blocks();
  const int left = (r + C - 1) % C, right = (r + 1) % C;
  const double* lb = cl.map_shared_rank(buf, left);
  const double* rb = cl.map_shared_rank(buf, right);
  for (int j = threadIdx.x; j < HL; j += blockDim.x) buf[j] = lb[HL + npc - HL + j];
  for (int j = threadIdx.x; j < HR; j += blockDim.x) buf[HL + npc + j] = rb[HL + j];
}

__global__ void __launch_bounds__(kSeqThreads) seq_kernel(const __grid_constant__ SeqParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cg::cluster_group cl = cg::this_cluster();
  const int HL = p.halo_l, HR = p.halo_r, npc = p.npc;
  const int W = HL + npc + HR;
  double* A = reinterpret_cast<double*>(smem_raw);
  double* B = A + W;
  const int r = (int)cl.block_rank();
  const int64_t base = (int64_t)r * npc;
  for (int i = threadIdx.x; i < npc; i += blockDim.x) A[HL + i] = p.u0[base + i];
  cl.sync();
  seq_halo(cl, A, HL, HR, npc);
  __syncthreads();
  for (int64_t s = 0; s < p.passes; ++s) {
    seq_pass(A, B, HL, npc, p.lo, p.ntaps, p.taps);
    cl.sync();
    seq_halo(cl, B, HL, HR, npc);
    __syncthreads();
    double* t = A;
    A = B;
    B = t;
    if (p.traj && p.every_passes > 0 && (s + 1) % p.every_passes == 0) {
      double* row = p.traj + ((s + 1) / p.every_passes - 1) * p.nx + base;
      for (int i = threadIdx.x; i < npc; i += blockDim.x) row[i] = A[HL + i];
    }
  }
  for (int s = 0; s < p.tail_passes; ++s) {
    seq_pass(A, B, HL, npc, p.tail_lo, p.tail_ntaps, p.tail_taps);
    cl.sync();
    seq_halo(cl, B, HL, HR, npc);
    __syncthreads();
    double* t = A;
    A = B;
    B = t;
  }
  for (int i = threadIdx.x; i < npc; i += blockDim.x) p.u_out[base + i] = A[HL + i];
  // keep this CTA's shared memory alive until every neighbour finished its
  // last halo read
  cl.sync();
}

int launch_seq(const SeqParams& p, cudaStream_t st) {
  static bool configured = false;
  if (!configured) {
    cudaFuncSetAttribute(seq_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaFuncSetAttribute(seq_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    configured = true;
  }
  size_t smem = 2 * sizeof(double) * (size_t)(p.halo_l + p.npc + p.halo_r);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)p.csize);
  cfg.blockDim = dim3(kSeqThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)p.csize;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e = cudaLaunchKernelEx(&cfg, seq_kernel, p);
  return e == cudaSuccess ? 0 : -1;
}

// Largest cluster size <= want that the device can co-schedule for seq_kernel.
int seq_max_cluster(int want, size_t smem) {
  cudaFuncSetAttribute(seq_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  cudaFuncSetAttribute(seq_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  for (int c = want; c >= 1; c >>= 1) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)c);
    cfg.blockDim = dim3(kSeqThreads);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)c;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, seq_kernel, &cfg) == cudaSuccess && n > 0) return c;
    cudaGetLastError();
  }
  return 1;
}

}  // namespace mg
