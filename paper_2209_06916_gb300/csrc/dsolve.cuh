// Device helpers shared by the MGRIT kernels: fixed-order block sums and the
// periodic banded solve over a vector split into per-thread chunks and,
// optionally, over the CTAs of a thread-block cluster (carries between
// chunks by an intra-CTA Hillis-Steele scan and a cluster-level sum of CTA
// aggregates through distributed shared memory).
#pragma once
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "kernels.h"

namespace mg {
namespace cgc = cooperative_groups;

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
template <int HC, int HA, typename T, int PM, typename Prm>
__device__ __forceinline__ void banded_solve(T (&x)[PM], const Prm& A, T* sqc, T* sqa, T* aggc, T* agga,
                                             int t, int rank) {
  cgc::cluster_group cl = cgc::this_cluster();
  const int P = A.P, NT = A.nthr, C = A.csize;
  if constexpr (HC > 0) {
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
  if constexpr (HA > 0) {
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


}  // namespace mg
