#pragma once
// Coarse-level MGRIT step kernel (Sec. 6.1-6.2): v <- Phi_l v + g_n with
// Phi_l = (I - phi_l D^{(p+1)}_2)^{-1} S_p^{(m^l dt)}, one CF-interval per
// thread-block cluster (the vector split over its CTAs), in the modes
// C-relaxation after F (CF), F-relaxation + C-point residual (FRES), F
// post-relaxation added into the parent level (FOUT, the coarse-grid
// correction), sequential coarsest solve (SEQ) and plain apply (APPLY).
// GM = true replaces the exact banded correction solve by GMRES (Sec. 6.1,
// Sec. 6.3; gmres.cuh).
#include <cooperative_groups.h>
#include <cuda_pipeline.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "dsolve.cuh"
#include "gmres.cuh"
#include "kernels.h"

namespace mg {

template <int P>
struct Log2c {
  static constexpr int v = (P <= 1) ? 0 : 1 + Log2c<P / 2>::v;
};
template <>
struct Log2c<1> {
  static constexpr int v = 0;
};

// One step's SL gather for the thread's chunk: x_j = sum_a w_a v(g0 + j + a),
// the window g0 .. g0 + P + P1 - 2 starting at local index l0 of CTA `b0`
// and running into CTA `b1` past npc (b0 == b1 and a wrap for one CTA).
template <typename T, typename TC, int P, int P1, int LP>
__device__ __forceinline__ void sl_gather(TC (&x)[P], const T* b0, const T* b1, int l0, int npc, const T* w) {
  auto val = [&](int l) -> T {
    if (l < npc) return b0[l + (l >> LP)];
    l -= npc;
    return b1[l + (l >> LP)];
  };
  T win[P1];
#pragma unroll
  for (int a = 0; a < P1 - 1; ++a) win[a] = val(l0 + a);
#pragma unroll
  for (int j = 0; j < P; ++j) {
    win[P1 - 1] = val(l0 + j + P1 - 1);
    T acc = T(0);
#pragma unroll
    for (int a = 0; a < P1; ++a) acc = fma(w[a], win[a], acc);
    x[j] = (TC)acc;
#pragma unroll
    for (int a = 0; a < P1 - 1; ++a) win[a] = win[a + 1];
  }
}

template <typename T, typename TC, int P, int P1, bool GM>
__global__ void __launch_bounds__(256) coarse_kernel(const __grid_constant__ CoarseParams<T, TC> A) {
  // recurrence orders of the correction solve: (p+1)/2 both ways for the
  // centred D of odd p (P1 even); (p+2)/2 causal and p/2 anticausal for the
  // left-biased D of even p (P1 odd).  The GMRES mat-vec reads HCm points on
  // either side.
  constexpr int HCm = (P1 % 2 == 0) ? P1 / 2 : (P1 + 1) / 2;
  constexpr int HAm = (P1 % 2 == 0) ? P1 / 2 : (P1 - 1) / 2;
  constexpr int LP = Log2c<P>::v;
  static_assert((1 << LP) == P, "chunk length must be a power of two");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cgc::cluster_group cl = cgc::this_cluster();
  const int n = A.n, NT = A.nthr, C = A.csize, npc = A.npc, t = threadIdx.x;
  const int rank = (int)cl.block_rank();
  const int npad = NT * (P + 1);  // one padded chunk of P + 1 per thread
  T* const sv0 = reinterpret_cast<T*>(smem_raw);
  T* const sv1 = sv0 + npad;
  // RHS row: row s+1 is fetched (cp.async) into it as soon as the cluster
  // barrier after step s has retired its last reader, and lands while step
  // s+1 gathers and solves
  T* const sg = sv1 + npad;
  const size_t slot_bytes = (((size_t)3 * npad * sizeof(T)) + 15) & ~(size_t)15;
  TC* sqc = reinterpret_cast<TC*>(smem_raw + slot_bytes);
  TC* sqa = sqc + 48;
  TC* aggc = sqa + 48;
  TC* agga = aggc + 4;
  double* red = reinterpret_cast<double*>(smem_raw + slot_bytes + ((104 * sizeof(TC) + 15) & ~(size_t)15));
  // GMRES: the Krylov vector's halo buffer and the reduction / Hessenberg area
  const size_t gm_off = slot_bytes + ((104 * 8 + 15) & ~(size_t)15) + 32 * sizeof(double);
  TC* const gmv = reinterpret_cast<TC*>(smem_raw + gm_off);
  double* const gms =
      reinterpret_cast<double*>(smem_raw + gm_off + (((size_t)npad * sizeof(TC) + 15) & ~(size_t)15));
  const int64_t k = blockIdx.x / C;
  const int64_t nn = n;
  const int64_t off = (int64_t)rank * npc;  // first global point of this CTA
  const int base = t * (P + 1);
  auto pos = [](int i) { return i + (i >> LP); };
  int cur = 0;

  if (A.zero_start) {
    for (int i = t; i < npc; i += NT) sv0[pos(i)] = T(0);
  } else {
    const T* src = A.start + k * nn + off;
    for (int i = t; i < npc; i += NT) sv0[pos(i)] = src[i];
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
  // each thread fetches its own chunk of the row (P consecutive values), so
  // its wait covers everything it reads: no CTA barrier per step
  auto prefetch = [&](int s) {
    const T* gr = A.g + (gbase + s) * nn + off + t * P;
#pragma unroll
    for (int j = 0; j < P; ++j) __pipeline_memcpy_async(&sg[base + j], &gr[j], sizeof(T));
    __pipeline_commit();
  };
  if (A.g && A.nsteps >= 1) prefetch(1);
  // departure window of this thread: global points gw0 .. gw0 + P + P1 - 2
  int gw0 = (int)((off + (int64_t)t * P - A.kshift + A.jlo) % nn);
  if (gw0 < 0) gw0 += n;
  const int r0 = gw0 / npc, l0 = gw0 - r0 * npc, r1 = (r0 + 1) % C;
  // the window's two CTAs, for either state slot (generic addresses)
  const T* const w00 = cl.map_shared_rank(sv0, r0);
  const T* const w01 = cl.map_shared_rank(sv1, r0);
  const T* const w10 = cl.map_shared_rank(sv0, r1);
  const T* const w11 = cl.map_shared_rank(sv1, r1);
  vec_sync(C);

  for (int s = 1; s <= A.nsteps; ++s) {
    TC x[P];
    if (s == 1 && A.zero_start) {
#pragma unroll
      for (int j = 0; j < P; ++j) x[j] = TC(0);
    } else {
      if (C == 1) {
        const T* v = cur ? sv1 : sv0;
        sl_gather<T, TC, P, P1, LP>(x, v, v, l0, npc, A.w);
      } else {
        sl_gather<T, TC, P, P1, LP>(x, cur ? w01 : w00, cur ? w11 : w10, l0, npc, A.w);
      }
      if constexpr (GM) {
        gmres_solve<TC, P, HCm>(x, A, gmv, gms, t, rank, C, k);
      } else {
        if (!A.nosolve) banded_solve<HCm, HAm, TC, P>(x, A, sqc, sqa, aggc, agga, t, rank, C);
      }
    }
    if (A.g) __pipeline_wait_prior(0);  // this thread's chunk of the RHS row has landed
    T* nxt = (cur ? sv0 : sv1) + base;
#pragma unroll
    for (int j = 0; j < P; ++j) {
      T v = (T)x[j];
      if (A.g) v += sg[base + j];
      nxt[j] = v;
    }
    vec_sync(C);
    if (A.g && s + 1 <= A.nsteps) prefetch(s + 1);
    cur ^= 1;
    if (A.mode == kModeFOUT || A.mode == kModeSEQ) {  // store only: no read on the critical path
      T* gr = A.g + (gbase + s) * nn + off;
      const T* v = cur ? sv1 : sv0;
      for (int i = t; i < npc; i += NT) gr[i] = v[pos(i)];
    }
  }

  const T* fin = cur ? sv1 : sv0;
  if (A.mode == kModeCF) {
    T* o = A.out + (k + 1) * nn + off;
    for (int i = t; i < npc; i += NT) o[i] = fin[pos(i)];
  } else if (A.mode == kModeAPPLY) {
    T* o = A.out + k * nn + off;
    for (int i = t; i < npc; i += NT) o[i] = fin[pos(i)];
  } else if (A.mode == kModeFRES) {
    T* o = A.out + (k + 1) * nn + off;
    const T* sb = A.sub ? A.sub + (k + 1) * nn + off : nullptr;
    double sq = 0.0;
    for (int i = t; i < npc; i += NT) {
      T r = fin[pos(i)];
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
  if (C > 1) cl.sync();
}

template <typename T, typename TC, int P, int P1, bool GM>
static void configure_coarse() {
  static std::mutex mu;
  static uint64_t done = 0;
  once_per_device(mu, done, [] {
    cudaFuncSetAttribute(coarse_kernel<T, TC, P, P1, GM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         227 * 1024);
    cudaFuncSetAttribute(coarse_kernel<T, TC, P, P1, GM>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  });
}

template <typename T, typename TC, int P, int P1, bool GM>
static int launch_coarse_t(const CoarseParams<T, TC>& A, cudaStream_t st) {
  configure_coarse<T, TC, P, P1, GM>();
  if (A.K <= 0) return 0;
  size_t smem = coarse_smem_bytes(A.npc, A.P, A.nthr, (int)sizeof(T), GM ? (int)sizeof(TC) : 0);
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
  return cudaLaunchKernelEx(&cfg, coarse_kernel<T, TC, P, P1, GM>, A) == cudaSuccess ? 1 : -1;
}

template <typename T, typename TC, int P1>
static int launch_coarse_p(const CoarseParams<T, TC>& A, cudaStream_t st) {
  if (A.gm_max > 0) {  // GMRES correction solves: chunks of 4 or 8 points
    if (A.gm_max > kGmMax || !A.gm_V) return -1;
    switch (A.P) {
      case 4:
        return launch_coarse_t<T, TC, 4, P1, true>(A, st);
      case 8:
        return launch_coarse_t<T, TC, 8, P1, true>(A, st);
      default:
        return -1;
    }
  }
  switch (A.P) {
    case 4:
      return launch_coarse_t<T, TC, 4, P1, false>(A, st);
    case 8:
      return launch_coarse_t<T, TC, 8, P1, false>(A, st);
    case 16:
      return launch_coarse_t<T, TC, 16, P1, false>(A, st);
    case 32:
      return launch_coarse_t<T, TC, 32, P1, false>(A, st);
    default:
      return -1;
  }
}

template <typename T, typename TC>
static int launch_coarse_any(const CoarseParams<T, TC>& A, cudaStream_t st) {
  switch (A.p1) {
    case 2:
      return launch_coarse_p<T, TC, 2>(A, st);
    case 3:
      return launch_coarse_p<T, TC, 3>(A, st);
    case 4:
      return launch_coarse_p<T, TC, 4>(A, st);
    case 5:
      return launch_coarse_p<T, TC, 5>(A, st);
    case 6:
      return launch_coarse_p<T, TC, 6>(A, st);
    default:
      return -1;
  }
}

}  // namespace mg
