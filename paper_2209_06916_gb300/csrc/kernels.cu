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
// Coarse-level step kernel (vector distributed over a thread-block cluster)
// ---------------------------------------------------------------------------
}  // namespace mg
#include <cooperative_groups.h>
namespace mg {
namespace cgc = cooperative_groups;

// Non-circular inclusive Hillis-Steele scan of chunk states inside the CTA in
// direction dir (-1: from lower chunks, +1: from higher chunks).  On return
// the final states are in sq (buffer index returned) and Q holds this
// chunk's prefix.
template <int H, typename T>
__device__ __forceinline__ int hs_scan(T (&Q)[H], const SolveDir<T>& D, T* sq, int t, int NT, int dir) {
  int buf = 0;
  for (int r = 0; r < D.rounds; ++r) {
#pragma unroll
    for (int a = 0; a < H; ++a) sq[(buf * 3 + a) * NT + t] = Q[a];
    __syncthreads();
    const int src = t + dir * (1 << r);
    if (src >= 0 && src < NT) {
      T Qo[H];
#pragma unroll
      for (int a = 0; a < H; ++a) Qo[a] = sq[(buf * 3 + a) * NT + src];
#pragma unroll
      for (int a = 0; a < H; ++a)
#pragma unroll
        for (int q = 0; q < H; ++q) Q[a] = fma(D.Mpow[r][a * 3 + q], Qo[q], Q[a]);
    }
    buf ^= 1;
  }
#pragma unroll
  for (int a = 0; a < H; ++a) sq[(buf * 3 + a) * NT + t] = Q[a];
  return buf;
}

// Carry S entering this thread's chunk in direction dir, from the final
// intra-CTA prefixes (sq[buf]) and the cluster-level carry.  `agg` is this
// CTA's cluster-visible aggregate slot (H values), already published and
// synchronised across the cluster by the caller.
template <int H, typename T>
__device__ __forceinline__ void chunk_carry(T (&S)[H], const SolveDir<T>& D, const T* sq, int buf, T* agg,
                                            int t, int NT, int dir, int rank, int C) {
  cgc::cluster_group cl = cgc::this_cluster();
  T X[H];
#pragma unroll
  for (int a = 0; a < H; ++a) X[a] = T(0);
  for (int j = 0; j < D.jterms; ++j) {
    int src = rank + dir * (1 + j);
    src %= C;
    if (src < 0) src += C;
    const T* Ap = (C == 1) ? agg : cl.map_shared_rank(agg, src);
    T Aj[H];
#pragma unroll
    for (int a = 0; a < H; ++a) Aj[a] = Ap[a];
#pragma unroll
    for (int a = 0; a < H; ++a)
#pragma unroll
      for (int q = 0; q < H; ++q) X[a] = fma(D.McPow[j][a * 3 + q], Aj[q], X[a]);
  }
  if (D.closure) {
    T Y[H];
#pragma unroll
    for (int a = 0; a < H; ++a) {
      T v = T(0);
#pragma unroll
      for (int q = 0; q < H; ++q) v = fma(D.Clc[a * 3 + q], X[q], v);
      Y[a] = v;
    }
#pragma unroll
    for (int a = 0; a < H; ++a) X[a] = Y[a];
  }
  // distance (in chunks) from the CTA edge the carry enters through
  const int tdist = (dir < 0) ? t : (NT - 1 - t);
#pragma unroll
  for (int a = 0; a < H; ++a) S[a] = T(0);
  if (tdist > 0) {
    const int src = t + dir;
#pragma unroll
    for (int a = 0; a < H; ++a) S[a] = sq[(buf * 3 + a) * NT + src];
  }
  if (tdist < D.tcut) {
    const T* Mt = D.Mt + (size_t)tdist * 9;
#pragma unroll
    for (int a = 0; a < H; ++a)
#pragma unroll
      for (int q = 0; q < H; ++q) S[a] = fma(__ldg(Mt + a * 3 + q), X[q], S[a]);
  }
}

// Periodic banded solve of the thread's chunk x (registers) in place: causal
// recurrence, carry, fixup fused with the anticausal local pass, carry,
// fixup.  Every thread of every CTA of the cluster must call it.
template <int HC, int HA, typename T, int PM>
__device__ __forceinline__ void banded_solve(T (&x)[PM], const CoarseParams<T>& A, T* sqc, T* sqa,
                                             T* aggc, T* agga, int t, int rank) {
  cgc::cluster_group cl = cgc::this_cluster();
  const int P = A.P, NT = A.nthr, C = A.csize;
  if (HC > 0) {
    T Q[HC > 0 ? HC : 1];
#pragma unroll
    for (int a = 0; a < HC; ++a) Q[a] = T(0);
#pragma unroll
    for (int j = 0; j < PM; ++j) {
      if (j < P) {
        T v = x[j];
#pragma unroll
        for (int q = 1; q <= HC; ++q)
          if (j - q >= 0) v = fma(A.c.ncoef[q - 1], x[j - q], v);
        x[j] = v;
#pragma unroll
        for (int a = 0; a < HC; ++a)
          if (j == P - 1 - a) Q[a] = v;
      }
    }
    int buf = hs_scan<HC>(Q, A.c, sqc, t, NT, -1);
    if (t == NT - 1) {
#pragma unroll
      for (int a = 0; a < HC; ++a) aggc[a] = Q[a];
    }
    cl.sync();
    T S[HC > 0 ? HC : 1];
    chunk_carry<HC>(S, A.c, sqc, buf, aggc, t, NT, -1, rank, C);
#pragma unroll
    for (int j = 0; j < PM; ++j) {
      if (j < P) {
        T v = x[j];
#pragma unroll
        for (int q = 0; q < HC; ++q) v = fma(A.c.G[j * 3 + q], S[q], v);
        x[j] = v;
      }
    }
  }
  if (HA > 0) {
    T Q[HA > 0 ? HA : 1];
#pragma unroll
    for (int a = 0; a < HA; ++a) Q[a] = T(0);
#pragma unroll
    for (int j = PM - 1; j >= 0; --j) {
      if (j < P) {
        T v = x[j];
#pragma unroll
        for (int q = 1; q <= HA; ++q)
          if (j + q < PM) {
            if (j + q < P) v = fma(A.a.ncoef[q - 1], x[j + q], v);
          }
        x[j] = v;
      }
    }
#pragma unroll
    for (int a = 0; a < HA; ++a) Q[a] = x[a];
    int buf = hs_scan<HA>(Q, A.a, sqa, t, NT, +1);
    if (t == 0) {
#pragma unroll
      for (int a = 0; a < HA; ++a) agga[a] = Q[a];
    }
    cl.sync();
    T S[HA > 0 ? HA : 1];
    chunk_carry<HA>(S, A.a, sqa, buf, agga, t, NT, +1, rank, C);
#pragma unroll
    for (int j = 0; j < PM; ++j) {
      if (j < P) {
        const int d = P - 1 - j;
        T v = x[j];
#pragma unroll
        for (int q = 0; q < HA; ++q) v = fma(A.a.G[d * 3 + q], S[q], v);
        x[j] = v;
      }
    }
  }
}

template <typename T, int PM, int P1>
__global__ void __launch_bounds__(256) coarse_kernel(const __grid_constant__ CoarseParams<T> A) {
  constexpr int H = P1 / 2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cgc::cluster_group cl = cgc::this_cluster();
  const int n = A.n, P = A.P, NT = A.nthr, C = A.csize, npc = A.npc, t = threadIdx.x;
  const int rank = (int)cl.block_rank();
  const int npad = npc + (npc + P - 1) / P;
  T* sv0 = reinterpret_cast<T*>(smem_raw);
  T* sv1 = sv0 + npad;
  T* sg = sv1 + npad;
  T* sqc = sg + npad;
  T* sqa = sqc + 6 * NT;
  T* aggc = sqa + 6 * NT;
  T* agga = aggc + 4;
  double* red = reinterpret_cast<double*>(agga + 4);
  const int64_t k = blockIdx.x / C;
  const int64_t nn = n;
  const int64_t off = (int64_t)rank * npc;  // first global point of this CTA
  T* cur = sv0;
  T* nxt = sv1;

  if (A.zero_start) {
    for (int i = t; i < npc; i += NT) cur[i + i / P] = T(0);
  } else {
    const T* src = A.start + k * nn + off;
    for (int i = t; i < npc; i += NT) cur[i + i / P] = src[i];
  }
  if (A.mode == kModeFOUT) {
    const T* src = A.start + k * nn + off;
    T* par = A.parent + k * A.m * nn + off;
    for (int i = t; i < npc; i += NT) par[i] += src[i];
    if (k == A.K - 1) {
      const T* s2 = A.start + A.K * nn + off;
      T* p2 = A.parent + A.K * A.m * nn + off;
      for (int i = t; i < npc; i += NT) p2[i] += s2[i];
    }
  }
  cl.sync();

  // SL gather window of this thread: global indices gw0 + w, w < P + P1 - 1
  int gw0 = (int)((off + (int64_t)t * P - A.kshift + A.jlo) % nn);
  if (gw0 < 0) gw0 += n;

  const int64_t gbase = (A.mode == kModeSEQ) ? 0 : k * A.m;
  for (int s = 1; s <= A.nsteps; ++s) {
    if (A.g) {
      const T* gr = A.g + (gbase + s) * nn + off;
      for (int i = t; i < npc; i += NT) sg[i + i / P] = gr[i];
    }
    T x[PM];
    if (s == 1 && A.zero_start) {
#pragma unroll
      for (int j = 0; j < PM; ++j) x[j] = T(0);
      __syncthreads();
    } else {
      T win[P1];
      auto fetch = [&](int w) -> T {
        int gi = gw0 + w;
        if (gi >= n) gi -= n;
        if (gi >= n) gi -= n;
        if (C == 1) return cur[gi + gi / P];
        const int owner = gi / npc;
        const int li = gi - owner * npc;
        const T* base = cl.map_shared_rank(cur, owner);
        return base[li + li / P];
      };
#pragma unroll
      for (int a = 0; a < P1 - 1; ++a) win[a] = fetch(a);
#pragma unroll
      for (int j = 0; j < PM; ++j) {
        if (j < P) {
          win[P1 - 1] = fetch(j + P1 - 1);
          T acc = T(0);
#pragma unroll
          for (int a = 0; a < P1; ++a) acc = fma(A.w[a], win[a], acc);
          x[j] = acc;
#pragma unroll
          for (int a = 0; a < P1 - 1; ++a) win[a] = win[a + 1];
        }
      }
      __syncthreads();
      banded_solve<H, H, T, PM>(x, A, sqc, sqa, aggc, agga, t, rank);
    }
    // new state v_{i - shift} = x_i + g (the shift stays inside this CTA's
    // range for the symmetric factorisation: shift = 0)
#pragma unroll
    for (int j = 0; j < PM; ++j) {
      if (j < P) {
        int i2 = t * P + j - A.shift;
        if (i2 < 0) i2 += npc;
        T v = x[j];
        if (A.g) v += sg[i2 + i2 / P];
        nxt[i2 + i2 / P] = v;
      }
    }
    cl.sync();
    T* tmp = cur;
    cur = nxt;
    nxt = tmp;
    if (A.mode == kModeFOUT || A.mode == kModeSEQ) {
      T* par = A.parent + (gbase + s) * nn + off;
      for (int i = t; i < npc; i += NT) par[i] += cur[i + i / P];
    }
  }

  if (A.mode == kModeCF) {
    T* o = A.out + (k + 1) * nn + off;
    for (int i = t; i < npc; i += NT) o[i] = cur[i + i / P];
  } else if (A.mode == kModeAPPLY) {
    T* o = A.out + k * nn + off;
    for (int i = t; i < npc; i += NT) o[i] = cur[i + i / P];
  } else if (A.mode == kModeFRES) {
    T* o = A.out + (k + 1) * nn + off;
    const T* sb = A.sub ? A.sub + (k + 1) * nn + off : nullptr;
    double sq = 0.0;
    for (int i = t; i < npc; i += NT) {
      T r = cur[i + i / P];
      if (sb) r -= sb[i];
      o[i] = r;
      sq += (double)r * (double)r;
    }
    if (A.partial) {
      double tot = block_sum(sq, red);
      if (t == 0) A.partial[blockIdx.x] = tot;
    }
  }
  // keep this CTA's shared memory alive until the cluster has finished its
  // remote reads of it
  cl.sync();
}

size_t coarse_smem_bytes(int npc, int P, int nthr, int elem) {
  size_t npad = (size_t)npc + (size_t)((npc + P - 1) / P);
  return (3 * npad + 12 * (size_t)nthr + 8) * (size_t)elem + 32 * sizeof(double) + 16;
}

template <typename T, int PM, int P1>
static void configure_coarse() {
  static bool configured = false;
  if (!configured) {
    cudaFuncSetAttribute(coarse_kernel<T, PM, P1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    cudaFuncSetAttribute(coarse_kernel<T, PM, P1>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    configured = true;
  }
}

template <typename T, int PM, int P1>
static int launch_coarse_t(const CoarseParams<T>& A, cudaStream_t st) {
  configure_coarse<T, PM, P1>();
  if (A.K <= 0) return 0;
  size_t smem = coarse_smem_bytes(A.npc, A.P, A.nthr, (int)sizeof(T));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(A.K * A.csize));
  cfg.blockDim = dim3((unsigned)A.nthr);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)A.csize;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, coarse_kernel<T, PM, P1>, A) == cudaSuccess ? 1 : -1;
}

template <typename T, int P1>
static int launch_coarse_p(const CoarseParams<T>& A, cudaStream_t st) {
  if (A.P <= 16) return launch_coarse_t<T, 16, P1>(A, st);
  if (A.P <= 32) return launch_coarse_t<T, 32, P1>(A, st);
  return launch_coarse_t<T, 64, P1>(A, st);
}

template <typename T>
static int launch_coarse_any(const CoarseParams<T>& A, cudaStream_t st) {
  switch (A.p1) {
    case 2:
      return launch_coarse_p<T, 2>(A, st);
    case 4:
      return launch_coarse_p<T, 4>(A, st);
    case 6:
      return launch_coarse_p<T, 6>(A, st);
    default:
      return -1;
  }
}

int launch_coarse(const CoarseParams<double>& p, cudaStream_t st) { return launch_coarse_any(p, st); }
int launch_coarse(const CoarseParams<float>& p, cudaStream_t st) { return launch_coarse_any(p, st); }

// Largest cluster size <= want (power of two) that can be co-scheduled.
int coarse_max_cluster(int want, size_t smem, int nthr) {
  configure_coarse<double, 32, 4>();
  for (int c = want; c >= 1; c >>= 1) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)c);
    cfg.blockDim = dim3((unsigned)nthr);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)c;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nc = 0;
    if (cudaOccupancyMaxActiveClusters(&nc, coarse_kernel<double, 32, 4>, &cfg) == cudaSuccess && nc > 0)
      return c;
    cudaGetLastError();
  }
  return 1;
}

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
