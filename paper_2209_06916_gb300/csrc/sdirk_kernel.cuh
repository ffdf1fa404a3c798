#pragma once
// Level-0 SDIRK step kernel (Sec. 4.2-4.3): the fine one-step map
// Phi = R_q(-c L_p) of an SDIRK method applied through its stages, each a
// periodic banded solve with (I + gamma c L_p) and mat-vecs with L_p (the
// practical form of a step described in the footnote of Sec. 4.3).  One
// CF-interval per thread-block cluster; the vector is split over the
// cluster's CTAs and, inside a CTA, into one chunk of P points per thread
// (P a compile-time length, so every shared-memory index is an immediate
// offset from the thread's chunk).  L_p halos come from the neighbouring
// chunk (distributed shared memory only at CTA edges); the solve carries
// cross CTAs through distributed shared memory.
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "dsolve.cuh"
#include "kernels.h"

namespace mg {

template <int P>
struct Log2 {
  static constexpr int v = (P <= 1) ? 0 : 1 + Log2<P / 2>::v;
};
template <>
struct Log2<1> {
  static constexpr int v = 0;
};

template <typename T, int P, int P1>
__global__ void __launch_bounds__(256) sdirk_kernel(const __grid_constant__ SdirkParams<T> A) {
  // L_p taps at offsets LLO .. LLO + P1 - 1, LLO = -l(p) (Sec. 4.1 bias:
  // l = (p+1)/2 for odd p, p/2 + 1 for even p); the stage solves' recurrence
  // orders are l (causal) and r = P1 - 1 - l (anticausal)
  constexpr int LLO = (P1 % 2 == 0) ? -(P1 / 2) : -((P1 + 1) / 2);
  constexpr int HC = -LLO, HA = P1 - 1 + LLO;
  constexpr int HL = -LLO;           // left halo width
  constexpr int HR = P1 - 1 + LLO;   // right halo width
  constexpr int LP = Log2<P>::v;
  static_assert((1 << LP) == P, "chunk length must be a power of two");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cgc::cluster_group cl = cgc::this_cluster();
  const int NT = A.nthr, C = A.csize, npc = A.npc, t = threadIdx.x;
  const int rank = (int)cl.block_rank();
  const int npad = NT * (P + 1);     // one padded chunk of P + 1 per thread
  T* slots = reinterpret_cast<T*>(smem_raw);
  const size_t slot_bytes = ((size_t)A.nslots * npad * sizeof(T) + 15) & ~(size_t)15;
  T* sqc = reinterpret_cast<T*>(smem_raw + slot_bytes);
  T* sqa = sqc + 48;
  T* aggc = sqa + 48;
  T* agga = aggc + 4;
  double* red = reinterpret_cast<double*>(smem_raw + slot_bytes + ((104 * sizeof(T) + 15) & ~(size_t)15));
  const int64_t k = blockIdx.x / C;
  const int64_t nn = A.n;
  const int64_t off = (int64_t)rank * npc;
  const int base = t * (P + 1);      // this thread's chunk
  auto pos = [](int i) { return i + (i >> LP); };

  // state (slot 0), coalesced
  if (A.zero_start) {
    for (int i = t; i < npc; i += NT) slots[pos(i)] = T(0);
  } else {
    const T* src = A.start + k * nn + off;
    for (int i = t; i < npc; i += NT) slots[pos(i)] = src[i];
  }
  if (A.mode == kModeFOUT && A.g) {
    // the C-points themselves go to RHS row k m (and the last CTA's start[K]
    // to row K m): rows the F post-relaxation does not read
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
  // neighbouring chunks for the L_p halos (slot 0 of the owning CTA)
  const T* lnb = (t > 0) ? slots + base - (P + 1)
                         : cl.map_shared_rank(slots, (rank + C - 1) % C) + (NT - 1) * (P + 1);
  const T* rnb = (t < NT - 1) ? slots + base + (P + 1) : cl.map_shared_rank(slots, (rank + 1) % C);
  vec_sync(C);

  for (int s = 1; s <= A.nsteps; ++s) {
    for (int o = 0; o < A.nops; ++o) {
      const int kind = A.opk[o];
      if (A.opb[o]) vec_sync(C);
      T* dst = slots + (size_t)A.opd[o] * npad + base;
      const int so = A.ops[o] * npad;
      const T* src = slots + so + base;
      if (kind == kOpCopy) {
#pragma unroll
        for (int j = 0; j < P; ++j) dst[j] = src[j];
      } else if (kind == kOpZero) {
#pragma unroll
        for (int j = 0; j < P; ++j) dst[j] = T(0);
      } else if (kind == kOpAxpy) {
        const T cf = A.opc[o];
#pragma unroll
        for (int j = 0; j < P; ++j) dst[j] = fma(cf, src[j], dst[j]);
      } else if (kind == kOpAxpby) {
        const T cf = A.opc[o], cf2 = A.opc2[o];
#pragma unroll
        for (int j = 0; j < P; ++j) dst[j] = fma(cf, src[j], cf2 * dst[j]);
      } else if (kind == kOpAxpyL) {
        // acc = L_p src on this chunk (sliding window), then every op of
        // the group: dst_g += c_g acc
        T hl[HL], hr[HR > 0 ? HR : 1];
#pragma unroll
        for (int a = 0; a < HL; ++a) hl[a] = lnb[so + P - HL + a];
#pragma unroll
        for (int a = 0; a < HR; ++a) hr[a] = rnb[so + a];
        auto val = [&](int d) -> T {
          if (d < 0) return hl[d + HL];
          if (d >= P) return hr[d - P];
          return src[d];
        };
        T acc[P];
        T win[P1];
#pragma unroll
        for (int a = 0; a < P1 - 1; ++a) win[a] = val(LLO + a);
#pragma unroll
        for (int j = 0; j < P; ++j) {
          win[P1 - 1] = val(j + LLO + P1 - 1);
          T v = T(0);
#pragma unroll
          for (int a = 0; a < P1; ++a) v = fma(A.ltaps[a], win[a], v);
          acc[j] = v;
#pragma unroll
          for (int a = 0; a < P1 - 1; ++a) win[a] = win[a + 1];
        }
        const int g = A.opg[o];
        for (int e = 0; e < g; ++e) {
          T* dg = slots + (size_t)A.opd[o + e] * npad + base;
          const T cf = A.opc[o + e];
#pragma unroll
          for (int j = 0; j < P; ++j) dg[j] = fma(cf, acc[j], dg[j]);
        }
        o += g - 1;
      } else {  // kOpSolve
        T x[P];
#pragma unroll
        for (int j = 0; j < P; ++j) x[j] = src[j];
        banded_solve<HC, HA, T, P>(x, A, sqc, sqa, aggc, agga, t, rank, C);
#pragma unroll
        for (int j = 0; j < P; ++j) dst[j] = x[j];
      }
    }
    const bool endcopy = A.result != 0 || A.rscale != T(1);
    if ((endcopy || A.g) && A.resb) vec_sync(C);
    if (endcopy) {
      const T* r = slots + (size_t)A.result * npad + base;
#pragma unroll
      for (int j = 0; j < P; ++j) slots[base + j] = A.rscale * r[j];
    }
    if (A.g) {  // + g_{k m + s} on this thread's chunk; FOUT / SEQ keep the value in that row
      T* gr = A.g + (gbase + s) * nn + off + t * P;
      const bool keep = A.mode == kModeFOUT || A.mode == kModeSEQ;
#pragma unroll
      for (int j = 0; j < P; ++j) {
        const T v = slots[base + j] + gr[j];
        slots[base + j] = v;
        if (keep) gr[j] = v;
      }
    }
    if (A.mode == kModeSEQ && A.traj && A.every > 0 && s % A.every == 0) {
      __syncthreads();
      T* row = A.traj + (int64_t)(s / A.every - 1) * nn + off;
      for (int i = t; i < npc; i += NT) row[i] = slots[pos(i)];
      __syncthreads();
    }
  }
  __syncthreads();
  if (A.mode == kModeCF || A.mode == kModeFRES) {
    T* o = A.out + (k + 1) * nn + off;
    const T* rh = A.rhs ? A.rhs + (k + 1) * nn + off : nullptr;
    const T* sb = A.sub ? A.sub + (k + 1) * nn + off : nullptr;
    double sq = 0.0;
    for (int i = t; i < npc; i += NT) {
      T v = slots[pos(i)];
      if (rh) v += rh[i];
      if (sb) v -= sb[i];
      o[i] = v;
      sq += (double)v * (double)v;
    }
    if (A.mode == kModeFRES && A.partial) {
      double tot = block_sum(sq, red);
      if (t == 0) A.partial[blockIdx.x] = tot;
    }
  } else if (A.out) {  // APPLY: rows k; SEQ: row 0 (FOUT and a coarsest SEQ keep g instead)
    T* o = A.out + (A.mode == kModeAPPLY ? k * nn : 0) + off;
    for (int i = t; i < npc; i += NT) o[i] = slots[pos(i)];
  }
  // remote readers of this CTA's shared memory are done before it exits
  if (C > 1) cl.sync();
}

template <typename T, int P, int P1>
static void configure_sdirk() {
  static std::mutex mu;
  static uint64_t done = 0;
  once_per_device(mu, done, [] {
    cudaFuncSetAttribute(sdirk_kernel<T, P, P1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    cudaFuncSetAttribute(sdirk_kernel<T, P, P1>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  });
}

template <typename T, int P, int P1>
static int launch_sdirk_t(const SdirkParams<T>& A, cudaStream_t st) {
  configure_sdirk<T, P, P1>();
  if (A.K <= 0) return 0;
  size_t smem = sdirk_smem_bytes(A.npc, A.P, A.nthr, A.nslots, (int)sizeof(T));
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
  return cudaLaunchKernelEx(&cfg, sdirk_kernel<T, P, P1>, A) == cudaSuccess ? 1 : -1;
}

template <typename T, int P1>
static int launch_sdirk_p(const SdirkParams<T>& A, cudaStream_t st) {
  switch (A.P) {
    case 4:
      return launch_sdirk_t<T, 4, P1>(A, st);
    case 8:
      return launch_sdirk_t<T, 8, P1>(A, st);
    case 16:
      return launch_sdirk_t<T, 16, P1>(A, st);
    case 32:
      return launch_sdirk_t<T, 32, P1>(A, st);
    default:
      return -1;
  }
}

template <typename T>
static int launch_sdirk_any(const SdirkParams<T>& A, cudaStream_t st) {
  switch (A.p1) {
    case 2:
      return launch_sdirk_p<T, 2>(A, st);
    case 3:
      return launch_sdirk_p<T, 3>(A, st);
    case 4:
      return launch_sdirk_p<T, 4>(A, st);
    case 5:
      return launch_sdirk_p<T, 5>(A, st);
    case 6:
      return launch_sdirk_p<T, 6>(A, st);
    default:
      return -1;
  }
}

}  // namespace mg
