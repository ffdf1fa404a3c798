// Coarse-level MGRIT step kernel (Sec. 6.1-6.2): v <- Phi_l v + g_n with
// Phi_l = (I - phi_l D^{(p+1)}_2)^{-1} S_p^{(m^l dt)}, one CF-interval per
// thread-block cluster (the vector split over its CTAs), in the modes
// C-relaxation after F (CF), F-relaxation + C-point residual (FRES), F
// post-relaxation added into the parent level (FOUT, the coarse-grid
// correction), sequential coarsest solve (SEQ) and plain apply (APPLY).
#include <cooperative_groups.h>
#include <cuda_pipeline.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "dsolve.cuh"
#include "kernels.h"

namespace mg {

template <typename T, typename TC, int PM, int P1>
__global__ void __launch_bounds__(256) coarse_kernel(const __grid_constant__ CoarseParams<T, TC> A) {
  constexpr int H = P1 / 2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cgc::cluster_group cl = cgc::this_cluster();
  const int n = A.n, P = A.P, NT = A.nthr, C = A.csize, npc = A.npc, t = threadIdx.x;
  const int rank = (int)cl.block_rank();
  const int npad = npc + (npc + P - 1) / P;
  T* sv0 = reinterpret_cast<T*>(smem_raw);
  T* sv1 = sv0 + npad;
  // RHS row: row s+1 is fetched (cp.async) into it as soon as the cluster
  // barrier after step s has retired its last reader, and lands while step
  // s+1 gathers and solves
  T* sg = sv1 + npad;
  // scan buffers of the solve precision, 16-byte aligned after the slots
  size_t slot_bytes = (((size_t)3 * npad * sizeof(T)) + 15) & ~(size_t)15;
  const int SQ = max(6 * NT, 48);
  TC* sqc = reinterpret_cast<TC*>(smem_raw + slot_bytes);
  TC* sqa = sqc + SQ;
  TC* aggc = sqa + SQ;
  TC* agga = aggc + 4;
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
    // the C-points themselves go to RHS row k m (and the last CTA's
    // start[K] to row K m): rows the F post-relaxation does not read
    const T* src = A.start + k * nn + off;
    T* gr = A.g + k * A.m * nn + off;
    for (int i = t; i < npc; i += NT) gr[i] = src[i];
    if (k == A.K - 1) {
      const T* s2 = A.start + A.K * nn + off;
      T* g2 = A.g + A.K * A.m * nn + off;
      for (int i = t; i < npc; i += NT) g2[i] = s2[i];
    }
  }
  const int64_t gbase = (A.mode == kModeSEQ) ? 0 : k * A.m;
  auto prefetch = [&](int s, T* dst) {
    const T* gr = A.g + (gbase + s) * nn + off;
    for (int i = t; i < npc; i += NT) __pipeline_memcpy_async(&dst[i + i / P], &gr[i], sizeof(T));
    __pipeline_commit();
  };
  if (A.g && A.nsteps >= 1) prefetch(1, sg);
  cl.sync();

  TC mtc[9], mta[9];
  load_carry_power(mtc, A.c, t, NT, -1);
  load_carry_power(mta, A.a, t, NT, +1);
  // SL gather window of this thread: global indices gw0 + w, w < P + P1 - 1
  int gw0 = (int)((off + (int64_t)t * P - A.kshift + A.jlo) % nn);
  if (gw0 < 0) gw0 += n;

  for (int s = 1; s <= A.nsteps; ++s) {
    TC x[PM];
    if (s == 1 && A.zero_start) {
#pragma unroll
      for (int j = 0; j < PM; ++j) x[j] = TC(0);
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
          x[j] = (TC)acc;
#pragma unroll
          for (int a = 0; a < P1 - 1; ++a) win[a] = win[a + 1];
        }
      }
      __syncthreads();
      banded_solve<H, H, TC, PM>(x, A, sqc, sqa, aggc, agga, mtc, mta, t, rank);
    }
    if (A.g) {  // this step's RHS row has landed (for every thread)
      __pipeline_wait_prior(0);
      __syncthreads();
    }
    // new state v_{i - shift} = x_i + g (the shift stays inside this CTA's
    // range for the symmetric factorisation: shift = 0)
#pragma unroll
    for (int j = 0; j < PM; ++j) {
      if (j < P) {
        int i2 = t * P + j - A.shift;
        if (i2 < 0) i2 += npc;
        T v = (T)x[j];
        if (A.g) v += sg[i2 + i2 / P];
        nxt[i2 + i2 / P] = v;
      }
    }
    cl.sync();
    if (A.g && s + 1 <= A.nsteps) prefetch(s + 1, sg);
    T* tmp = cur;
    cur = nxt;
    nxt = tmp;
    if (A.mode == kModeFOUT || A.mode == kModeSEQ) {  // store only: no read on the critical path
      T* gr = A.g + (gbase + s) * nn + off;
      for (int i = t; i < npc; i += NT) gr[i] = cur[i + i / P];
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
  // slots of `elem` bytes; scan buffers budgeted at 8 bytes (FP64 solve)
  size_t npad = (size_t)npc + (size_t)((npc + P - 1) / P);
  const size_t sq = std::max<size_t>(6 * (size_t)nthr, 48);
  return ((3 * npad * (size_t)elem + 15) & ~(size_t)15) + (2 * sq + 8) * 8 + 32 * sizeof(double) + 16;
}

template <typename T, typename TC, int PM, int P1>
static void configure_coarse() {
  static bool configured = false;
  if (!configured) {
    cudaFuncSetAttribute(coarse_kernel<T, TC, PM, P1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    cudaFuncSetAttribute(coarse_kernel<T, TC, PM, P1>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    configured = true;
  }
}

template <typename T, typename TC, int PM, int P1>
static int launch_coarse_t(const CoarseParams<T, TC>& A, cudaStream_t st) {
  configure_coarse<T, TC, PM, P1>();
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
  return cudaLaunchKernelEx(&cfg, coarse_kernel<T, TC, PM, P1>, A) == cudaSuccess ? 1 : -1;
}

template <typename T, typename TC, int P1>
static int launch_coarse_p(const CoarseParams<T, TC>& A, cudaStream_t st) {
  if (A.P <= 16) return launch_coarse_t<T, TC, 16, P1>(A, st);
  if (A.P <= 32) return launch_coarse_t<T, TC, 32, P1>(A, st);
  return launch_coarse_t<T, TC, 64, P1>(A, st);
}

template <typename T, typename TC>
static int launch_coarse_any(const CoarseParams<T, TC>& A, cudaStream_t st) {
  switch (A.p1) {
    case 2:
      return launch_coarse_p<T, TC, 2>(A, st);
    case 4:
      return launch_coarse_p<T, TC, 4>(A, st);
    case 6:
      return launch_coarse_p<T, TC, 6>(A, st);
    default:
      return -1;
  }
}

int launch_coarse(const CoarseParams<double>& p, cudaStream_t st) { return launch_coarse_any(p, st); }
int launch_coarse(const CoarseParams<float>& p, cudaStream_t st) { return launch_coarse_any(p, st); }
int launch_coarse(const CoarseParams<float, double>& p, cudaStream_t st) { return launch_coarse_any(p, st); }

// Largest cluster size <= want (power of two) that can be co-scheduled.
int coarse_max_cluster(int want, size_t smem, int nthr) {
  configure_coarse<double, double, 32, 4>();
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
    if (cudaOccupancyMaxActiveClusters(&nc, coarse_kernel<double, double, 32, 4>, &cfg) == cudaSuccess && nc > 0)
      return c;
    cudaGetLastError();
  }
  return 1;
}

}  // namespace mg
