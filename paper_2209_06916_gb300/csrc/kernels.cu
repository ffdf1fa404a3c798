// MGRIT device kernels for sm_103a (GB300).
//
//  stencil_rows_kernel  level-0 relaxation: the fine map of one CF-interval,
//                       Phi^m = R_q(-c L_p)^m (Eq. MOL_M_def), applied as one
//                       composite periodic stencil to C-point rows (the m
//                       fine steps collapse into one wide stencil; the vector
//                       is read from HBM once per interval); optional RHS,
//                       subtraction (C-point residual, Sec. 2.2) and per-CTA
//                       sum of squares for the residual norm.
//  (the coarse-level kernel is in kernels_coarse.cu, the SDIRK step kernel
//   in kernels_sdirk.cu)
//  reduce_sum_kernel    fixed-order sum of per-CTA partials (deterministic).
//  random_cpoints_kernel  SplitMix64 random initial C-point iterate.
#include <cuda_pipeline.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "kernels.h"
#include "dsolve.cuh"

namespace mg {

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
  const int64_t ld = p.ld ? p.ld : nx;
  const T* in = p.in + row * ld;
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
      if (p.rhs) v += p.rhs[row * ld + i];
      if (p.sub) v -= p.sub[row * ld + i];
      p.out[row * ld + i] = v;
      sq += (double)v * (double)v;
    }
  }
  if (p.partial) {
    double tot = block_sum(sq, red);
    if (threadIdx.x == 0) p.partial[row * gridDim.y + blockIdx.y] = tot;
  }
}

// Persistent form: gridDim.x CTAs (one wave) walk the rows x tiles in a
// strided order; the input window of a CTA's next tile streams into the
// second shared-memory buffer (cp.async) while the current tile computes, so
// no wave starts with every CTA waiting on its loads.
template <typename T, int R>
__global__ void __launch_bounds__(kStencilThreads)
    stencil_rows_persistent(const __grid_constant__ StencilParams<T> p, int ntx) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[32];
  const int B = kStencilThreads;
  const int W = B * R;
  const int64_t nx = p.nx;
  const int nload = W + p.ntaps - 1;
  const int stride = (nload + 1) & ~1;
  T* const buf0 = reinterpret_cast<T*>(smem_raw);
  T* const buf1 = buf0 + stride;
  const int64_t ntiles = p.rows * (int64_t)ntx;
  const int64_t ld = p.ld ? p.ld : nx;
  auto fetch = [&](int64_t tl, T* dst) {
    const int64_t row = tl / ntx;
    const int64_t x0 = (tl - row * ntx) * W;
    const T* in = p.in + row * ld;
    int64_t g0 = (x0 + p.lo) % nx;
    if (g0 < 0) g0 += nx;
    for (int j = threadIdx.x; j < nload; j += B) {
      int64_t gi = g0 + j;
      while (gi >= nx) gi -= nx;
      __pipeline_memcpy_async(&dst[j], &in[gi], sizeof(T));
    }
    __pipeline_commit();
  };
  int64_t tile = blockIdx.x;
  if (tile < ntiles) fetch(tile, buf0);
  int cur = 0;
  for (; tile < ntiles; tile += gridDim.x) {
    const int64_t next = tile + gridDim.x;
    if (next < ntiles)
      fetch(next, cur ? buf0 : buf1);
    else
      __pipeline_commit();  // an empty group keeps the wait below uniform
    __pipeline_wait_prior(1);  // this tile's window has landed
    __syncthreads();
    const int64_t row = tile / ntx;
    const int64_t tx = tile - row * ntx;
    const int64_t x0 = tx * W;
    const T* sp = (cur ? buf1 : buf0) + threadIdx.x;
    T acc[R];
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] = T(0);
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
        if (p.rhs) v += p.rhs[row * ld + i];
        if (p.sub) v -= p.sub[row * ld + i];
        p.out[row * ld + i] = v;
        sq += (double)v * (double)v;
      }
    }
    if (p.partial) {
      double tot = block_sum(sq, red);
      if (threadIdx.x == 0) p.partial[row * ntx + tx] = tot;
    }
    __syncthreads();  // the window is read before the next fetch refills it
    cur ^= 1;
  }
  __pipeline_wait_prior(0);
}

static int stencil_r(int64_t nx) {
  if (nx >= 4 * kStencilThreads) return 4;
  if (nx >= 2 * kStencilThreads) return 2;
  return 1;
}

int stencil_tiles(int64_t nx, int tile_r) {
  int R = tile_r > 0 ? tile_r : stencil_r(nx);
  return (int)((nx + (int64_t)kStencilThreads * R - 1) / ((int64_t)kStencilThreads * R));
}

template <typename T, int R>
static int64_t launch_stencil_r(const StencilParams<T>& p, cudaStream_t st) {
  const int W = kStencilThreads * R;
  static std::mutex mu;
  static uint64_t done = 0;
  once_per_device(mu, done, [] {
    cudaFuncSetAttribute(stencil_rows_kernel<T, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
    cudaFuncSetAttribute(stencil_rows_persistent<T, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, 128 * 1024);
  });
  const int ntx = stencil_tiles(p.nx, R);
  if (p.persistent) {
    const int nload = W + p.ntaps - 1;
    const size_t smem = (size_t)2 * ((nload + 1) & ~1) * sizeof(T);
    int nsm = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, stencil_rows_persistent<T, R>, kStencilThreads,
                                                      smem) != cudaSuccess || per_sm < 1)
      per_sm = 1;
    const int64_t ntiles = p.rows * (int64_t)ntx;
    const int64_t grid = std::min<int64_t>(ntiles, (int64_t)nsm * per_sm);
    stencil_rows_persistent<T, R><<<(unsigned)grid, kStencilThreads, smem, st>>>(p, ntx);
    return ntiles;
  }
  size_t smem = (size_t)(W + p.ntaps - 1) * sizeof(T);
  dim3 grid((unsigned)p.rows, (unsigned)ntx);
  stencil_rows_kernel<T, R><<<grid, kStencilThreads, smem, st>>>(p);
  return (int64_t)grid.x * grid.y;
}

template <typename T>
static int64_t launch_stencil_any(const StencilParams<T>& p, cudaStream_t st) {
  if (p.rows <= 0) return 0;
  switch (p.tile_r > 0 ? p.tile_r : stencil_r(p.nx)) {
    case 8:
      return launch_stencil_r<T, 8>(p, st);
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

__global__ void convert_kernel(int op, double* __restrict__ d, float* __restrict__ f, int64_t n,
                               const double* __restrict__ d2, const float* __restrict__ f2) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    switch (op) {
      case kAddD2D:
        d[i] += d2[i];
        break;
      case kAddF2F:
        f[i] += f2[i];
        break;
      case kCvtD2F:
        f[i] = (float)d[i];
        break;
      case kCvtF2D:
        d[i] = (double)f[i];
        break;
      case kAddF2D:
        d[i] += (double)f[i];
        break;
      default:
        f[i] += (float)d[i];
        break;
    }
  }
}

void launch_convert(int op, double* d, float* f, int64_t n, cudaStream_t st, const double* d2, const float* f2) {
  if (n <= 0) return;
  int blocks = (int)std::min<int64_t>((n + 255) / 256, 152 * 8);
  convert_kernel<<<blocks, 256, 0, st>>>(op, d, f, n, d2, f2);
}

// sqrt of a sum of squares with NaN kept: a NaN residual must stop the solve
// as diverged, not read as zero (fmax would drop it)
__device__ __forceinline__ double dev_norm_of_sq(double x) { return x == x ? sqrt(x > 0.0 ? x : 0.0) : x; }

__global__ void solve_init_kernel(DevSolveState* s, const double* dnorm_sq, cudaGraphConditionalHandle hnd) {
  const double nrm = dev_norm_of_sq(dnorm_sq[0]);
  s->r0 = nrm;
  s->rnorm = nrm;
  s->it = 0;
  s->hist[0] = nrm;
  s->hist_len = 1;
  s->status = 0;
  s->converged = (nrm <= s->tol * nrm) ? 1 : 0;
  int go = 1;
  if (!isfinite(nrm)) {
    s->status = -4;
    go = 0;
  } else if (s->converged) {
    go = 0;
  } else if (s->max_iter <= 0) {
    s->status = -3;
    go = 0;
  }
  cudaGraphSetConditional(hnd, go);
}

__global__ void solve_check_kernel(DevSolveState* s, const double* dnorm_sq, cudaGraphConditionalHandle hnd) {
  const double nrm = dev_norm_of_sq(dnorm_sq[0]);
  s->it += 1;
  s->rnorm = nrm;
  if (s->hist_len < 128) s->hist[s->hist_len++] = nrm;
  int go = 1;
  if (!isfinite(nrm) || nrm > 1e3 * s->r0) {
    s->status = -4;
    go = 0;
  } else if (nrm <= s->tol * s->r0) {
    s->converged = 1;
    go = 0;
  } else if (s->it >= s->max_iter) {
    s->status = -3;
    go = 0;
  }
  cudaGraphSetConditional(hnd, go);
}

__global__ void inner_init_kernel(DevSolveState* s, const double* dnorm64_sq, cudaGraphConditionalHandle hnd) {
  const double rho0 = dev_norm_of_sq(dnorm64_sq[0]);
  s->in_rho0 = rho0;
  s->in_prev = rho0;
  s->in_tol = inner_target(s->tol, s->r0, rho0, s->in_base);
  s->in_count = 1;
  s->in_total += 1;
  cudaGraphSetConditional(hnd, s->in_count < s->in_max ? 1 : 0);
}

__global__ void inner_check_kernel(DevSolveState* s, const double* dnormf_sq, cudaGraphConditionalHandle hnd) {
  const double rho = dev_norm_of_sq(dnormf_sq[0]);
  s->in_count += 1;
  s->in_total += 1;
  const bool go = inner_continue(rho, s->in_prev, s->in_rho0, s->in_count, s->in_max, s->in_tol);
  s->in_prev = rho;
  cudaGraphSetConditional(hnd, go ? 1 : 0);
}

void launch_inner_init(DevSolveState* s, const double* dnorm64_sq, cudaGraphConditionalHandle hnd, cudaStream_t st) {
  inner_init_kernel<<<1, 1, 0, st>>>(s, dnorm64_sq, hnd);
}

void launch_inner_check(DevSolveState* s, const double* dnormf_sq, cudaGraphConditionalHandle hnd, cudaStream_t st) {
  inner_check_kernel<<<1, 1, 0, st>>>(s, dnormf_sq, hnd);
}

void* solve_init_kernel_fn() { return (void*)solve_init_kernel; }
void* solve_check_kernel_fn() { return (void*)solve_check_kernel; }

void launch_solve_check(DevSolveState* s, const double* dnorm_sq, cudaGraphConditionalHandle hnd,
                        cudaStream_t st) {
  solve_check_kernel<<<1, 1, 0, st>>>(s, dnorm_sq, hnd);
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
  static std::mutex mu;
  static uint64_t done = 0;
  once_per_device(mu, done, [] {
    cudaFuncSetAttribute(seq_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaFuncSetAttribute(seq_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  });
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
