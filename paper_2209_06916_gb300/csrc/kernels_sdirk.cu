// Level-0 SDIRK step kernel (Sec. 4.2-4.3): the fine one-step map
// Phi = R_q(-c L_p) of an SDIRK method applied through its stages, each a
// periodic banded solve with (I + gamma c L_p) and mat-vecs with L_p (the
// practical form of a step described in the footnote of Sec. 4.3).  One
// CF-interval per thread-block cluster; the vector is split over the
// cluster's CTAs, L_p halos and the solve carries cross CTAs through
// distributed shared memory.
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "dsolve.cuh"
#include "kernels.h"

namespace mg {

template <typename T, int PM, int P1>
__global__ void __launch_bounds__(256) sdirk_kernel(const __grid_constant__ SdirkParams<T> A) {
  constexpr int HC = P1 / 2, HA = P1 / 2 - 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cgc::cluster_group cl = cgc::this_cluster();
  const int n = A.n, P = A.P, NT = A.nthr, C = A.csize, npc = A.npc, t = threadIdx.x;
  const int rank = (int)cl.block_rank();
  const int npad = npc + (npc + P - 1) / P;
  T* slots = reinterpret_cast<T*>(smem_raw);
  const int SQ = max(6 * NT, 48);
  T* sqc = slots + (size_t)A.nslots * npad;
  T* sqa = sqc + SQ;
  T* aggc = sqa + SQ;
  T* agga = aggc + 4;
  // 16-byte aligned FP64 reduction scratch after the (possibly FP32) slots
  double* red = reinterpret_cast<double*>((reinterpret_cast<uintptr_t>(agga + 4) + 15) & ~(uintptr_t)15);
  const int64_t k = blockIdx.x / C;
  const int64_t nn = n;
  const int64_t off = (int64_t)rank * npc;
  const int c0 = t * P;  // first local point of this thread's chunk

  if (A.zero_start) {
    for (int j = 0; j < P; ++j) slots[c0 + j + (c0 + j) / P] = T(0);
  } else {
    const T* src = A.start + k * nn + off;
    for (int j = 0; j < P; ++j) slots[c0 + j + (c0 + j) / P] = src[c0 + j];
  }
  T mtc[9], mta[9];
  load_carry_power(mtc, A.c, t, NT, -1);
  load_carry_power(mta, A.a, t, NT, +1);
  // L_p window of this thread: global points gw0 + w, w < P + P1 - 1
  int gw0 = (int)((off + c0 + A.llo) % nn);
  if (gw0 < 0) gw0 += n;

  for (int s = 1; s <= A.nsteps; ++s) {
    for (int o = 0; o < A.nops; ++o) {
      const int kind = A.opk[o];
      T* dst = slots + (size_t)A.opd[o] * npad;
      T* src = slots + (size_t)A.ops[o] * npad;
      const T cf = A.opc[o];
      if (kind == kOpCopy) {
        for (int j = 0; j < P; ++j) {
          const int i = c0 + j + (c0 + j) / P;
          dst[i] = src[i];
        }
      } else if (kind == kOpZero) {
        for (int j = 0; j < P; ++j) dst[c0 + j + (c0 + j) / P] = T(0);
      } else if (kind == kOpAxpy) {
        for (int j = 0; j < P; ++j) {
          const int i = c0 + j + (c0 + j) / P;
          dst[i] = fma(cf, src[i], dst[i]);
        }
      } else if (kind == kOpAxpyL) {
        cl.sync();  // every CTA's src is final
        auto fetch = [&](int w) -> T {
          int gi = gw0 + w;
          if (gi >= n) gi -= n;
          if (gi >= n) gi -= n;
          if (C == 1) return src[gi + gi / P];
          const int owner = gi / npc;
          const int li = gi - owner * npc;
          const T* base = cl.map_shared_rank(src, owner);
          return base[li + li / P];
        };
        T win[P1];
#pragma unroll
        for (int a = 0; a < P1 - 1; ++a) win[a] = fetch(a);
        T acc[PM];
#pragma unroll
        for (int j = 0; j < PM; ++j) {
          if (j < P) {
            win[P1 - 1] = fetch(j + P1 - 1);
            T v = T(0);
#pragma unroll
            for (int a = 0; a < P1; ++a) v = fma(A.ltaps[a], win[a], v);
            acc[j] = v;
#pragma unroll
            for (int a = 0; a < P1 - 1; ++a) win[a] = win[a + 1];
          }
        }
        cl.sync();  // remote reads of src done before anyone overwrites it
#pragma unroll
        for (int j = 0; j < PM; ++j) {
          if (j < P) {
            const int i = c0 + j + (c0 + j) / P;
            dst[i] = fma(cf, acc[j], dst[i]);
          }
        }
      } else {  // kOpSolve
        T x[PM];
#pragma unroll
        for (int j = 0; j < PM; ++j)
          if (j < P) x[j] = A.sscale * src[c0 + j + (c0 + j) / P];
        banded_solve<HC, HA, T, PM>(x, A, sqc, sqa, aggc, agga, mtc, mta, t, rank);
#pragma unroll
        for (int j = 0; j < PM; ++j)
          if (j < P) dst[c0 + j + (c0 + j) / P] = x[j];
      }
    }
    if (A.result != 0) {
      const T* r = slots + (size_t)A.result * npad;
      for (int j = 0; j < P; ++j) {
        const int i = c0 + j + (c0 + j) / P;
        slots[i] = r[i];
      }
    }
    if (A.mode == kModeSEQ && A.traj && A.every > 0 && s % A.every == 0) {
      T* row = A.traj + (int64_t)(s / A.every - 1) * nn + off;
      for (int j = 0; j < P; ++j) row[c0 + j] = slots[c0 + j + (c0 + j) / P];
    }
  }
  __syncthreads();
  if (A.mode == kModeCF || A.mode == kModeFRES) {
    T* o = A.out + (k + 1) * nn + off;
    const T* rh = A.rhs ? A.rhs + (k + 1) * nn + off : nullptr;
    const T* sb = A.sub ? A.sub + (k + 1) * nn + off : nullptr;
    double sq = 0.0;
    for (int i = t; i < npc; i += NT) {
      T v = slots[i + i / P];
      if (rh) v += rh[i];
      if (sb) v -= sb[i];
      o[i] = v;
      sq += (double)v * (double)v;
    }
    if (A.mode == kModeFRES && A.partial) {
      double tot = block_sum(sq, red);
      if (t == 0) A.partial[blockIdx.x] = tot;
    }
  } else {
    T* o = A.out + (A.mode == kModeAPPLY ? k * nn : 0) + off;
    for (int i = t; i < npc; i += NT) o[i] = slots[i + i / P];
  }
  cl.sync();
}

size_t sdirk_smem_bytes(int npc, int P, int nthr, int nslots, int elem) {
  size_t npad = (size_t)npc + (size_t)((npc + P - 1) / P);
  const size_t sq = std::max<size_t>(6 * (size_t)nthr, 48);
  return ((size_t)nslots * npad + 2 * sq + 8) * (size_t)elem + 32 * sizeof(double) + 16;
}

template <typename T, int PM, int P1>
static int launch_sdirk_t(const SdirkParams<T>& A, cudaStream_t st) {
  static bool configured = false;
  if (!configured) {
    cudaFuncSetAttribute(sdirk_kernel<T, PM, P1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    cudaFuncSetAttribute(sdirk_kernel<T, PM, P1>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    configured = true;
  }
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
  return cudaLaunchKernelEx(&cfg, sdirk_kernel<T, PM, P1>, A) == cudaSuccess ? 1 : -1;
}

template <typename T, int P1>
static int launch_sdirk_p(const SdirkParams<T>& A, cudaStream_t st) {
  if (A.P <= 16) return launch_sdirk_t<T, 16, P1>(A, st);
  if (A.P <= 32) return launch_sdirk_t<T, 32, P1>(A, st);
  return launch_sdirk_t<T, 64, P1>(A, st);
}

template <typename T>
static int launch_sdirk_any(const SdirkParams<T>& A, cudaStream_t st) {
  switch (A.p1) {
    case 2:
      return launch_sdirk_p<T, 2>(A, st);
    case 4:
      return launch_sdirk_p<T, 4>(A, st);
    case 6:
      return launch_sdirk_p<T, 6>(A, st);
    default:
      return -1;
  }
}

int launch_sdirk(const SdirkParams<double>& p, cudaStream_t st) { return launch_sdirk_any(p, st); }
int launch_sdirk(const SdirkParams<float>& p, cudaStream_t st) { return launch_sdirk_any(p, st); }

}  // namespace mg
