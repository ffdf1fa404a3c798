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


// Barrier over every thread that shares the vector: the CTA, or the whole
// thread-block cluster when the vector is split over C > 1 CTAs (also makes
// the shared-memory writes before it visible to the cluster).
__device__ __forceinline__ void vec_sync(int C) {
  if (C == 1)
    __syncthreads();
  else
    cgc::this_cluster().sync();
}

// Inclusive prefix of chunk states inside the CTA in direction dir (-1: from
// lower chunks, +1: from higher chunks).  Rounds at distances < 32 run on
// warp shuffles; the carry from other warps comes from one exchange of warp
// totals through shared memory (sw), combined with the host tables
// (M^32)^j and M^d.  On return Q is this chunk's prefix and the CTA-end lane
// of every warp has written its prefix to sq[w*3 + a] (read by chunk_carry
// after the caller's barrier).
template <int H, typename T>
__device__ __forceinline__ void hs_scan(T (&Q)[H], const SolveDir<T>& D, T* sq, T* sw, int t, int NT, int dir) {
  const int lane = t & 31, w = t >> 5, nw = (NT + 31) >> 5;
  const int wlen = min(32, NT - (w << 5));
  const unsigned mask = (wlen == 32) ? 0xffffffffu : ((1u << wlen) - 1u);
#pragma unroll
  for (int r = 0; r < 5; ++r) {
    if (r < D.rounds) {
      const int d = 1 << r;
      T Qo[H];
#pragma unroll
      for (int a = 0; a < H; ++a)
        Qo[a] = dir < 0 ? __shfl_up_sync(mask, Q[a], d) : __shfl_down_sync(mask, Q[a], d);
      const bool ok = dir < 0 ? (lane >= d) : (lane + d < wlen);
      if (ok) {
#pragma unroll
        for (int a = 0; a < H; ++a)
#pragma unroll
          for (int q = 0; q < H; ++q) Q[a] = fma(D.Mpow[r][a * 3 + q], Qo[q], Q[a]);
      }
    }
  }
  const int end_lane = dir < 0 ? wlen - 1 : 0;
  if (nw > 1 && D.rounds > 0 && D.dcut > 0) {
    if (lane == end_lane) {
#pragma unroll
      for (int a = 0; a < H; ++a) sw[w * 3 + a] = Q[a];
    }
    __syncthreads();
    const int dd = dir < 0 ? lane + 1 : wlen - lane;  // chunks from the warp edge, 1..32
    if (dd <= D.dcut) {
      T X[H];
#pragma unroll
      for (int a = 0; a < H; ++a) X[a] = T(0);
      for (int j = 1; j <= D.wterms; ++j) {
        const int v = w + dir * j;
        if (v < 0 || v >= nw) break;
#pragma unroll
        for (int a = 0; a < H; ++a)
#pragma unroll
          for (int q = 0; q < H; ++q) X[a] = fma(D.M32pow[j - 1][a * 3 + q], sw[v * 3 + q], X[a]);
      }
#pragma unroll
      for (int a = 0; a < H; ++a)
#pragma unroll
        for (int q = 0; q < H; ++q) Q[a] = fma(D.Mlane[dd - 1][a * 3 + q], X[q], Q[a]);
    }
  }
  if (lane == end_lane) {
#pragma unroll
    for (int a = 0; a < H; ++a) sq[w * 3 + a] = Q[a];
  }
}

// Carry S entering this thread's chunk in direction dir: the neighbouring
// chunk's prefix (a shuffle inside the warp, sq across warps) plus
// M^{tdist} X, X the cluster-level carry into the CTA.  `agg` is this CTA's
// cluster-visible aggregate slot (H values), published and synchronised by
// the caller; M^{tdist} comes from the device table D.Mt (zero beyond tcut).
template <int H, typename T>
__device__ __forceinline__ void chunk_carry(T (&S)[H], const T (&Q)[H], const SolveDir<T>& D, const T* sq,
                                            T* agg, int t, int NT, int dir, int rank, int C) {
  const int lane = t & 31, w = t >> 5;
  const int wlen = min(32, NT - (w << 5));
  const unsigned mask = (wlen == 32) ? 0xffffffffu : ((1u << wlen) - 1u);
  T Qs[H];
#pragma unroll
  for (int a = 0; a < H; ++a) Qs[a] = dir < 0 ? __shfl_up_sync(mask, Q[a], 1) : __shfl_down_sync(mask, Q[a], 1);
  const bool edge = dir < 0 ? (lane == 0) : (lane == wlen - 1);
  const int tdist = (dir < 0) ? t : (NT - 1 - t);
#pragma unroll
  for (int a = 0; a < H; ++a) S[a] = T(0);
  if (tdist > 0) {
    if (edge) {
      const int v = w + dir;
#pragma unroll
      for (int a = 0; a < H; ++a) S[a] = sq[v * 3 + a];
    } else {
#pragma unroll
      for (int a = 0; a < H; ++a) S[a] = Qs[a];
    }
  }
  if (tdist >= D.tcut) return;  // the cluster-level carry has decayed below 1e-18 here
  T X[H];
#pragma unroll
  for (int a = 0; a < H; ++a) X[a] = T(0);
  cgc::cluster_group cl = cgc::this_cluster();
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
  const T* Mt = D.Mt + (size_t)tdist * 9;
#pragma unroll
  for (int a = 0; a < H; ++a)
#pragma unroll
    for (int q = 0; q < H; ++q) S[a] = fma(__ldg(Mt + a * 3 + q), X[q], S[a]);
}

// Periodic banded solve of the thread's chunk x (P values in registers, P a
// compile-time chunk length) in place: causal local recurrence, carry,
// fix-up; anticausal local recurrence, carry, fix-up.  Every thread of every
// CTA sharing the vector must call it (C = CTAs per vector).
template <int HC, int HA, typename T, int P, typename Prm>
__device__ __forceinline__ void banded_solve(T (&x)[P], const Prm& A, T* sqc, T* sqa, T* aggc, T* agga, int t,
                                             int rank, int C) {
  const int NT = A.nthr;
  if constexpr (HC > 0) {
    // x_j -= sum_q c_q x_{j-q}, oldest term first: the newest value enters
    // through the last FMA only
#pragma unroll
    for (int j = 0; j < P; ++j) {
      T v = x[j];
#pragma unroll
      for (int q = HC; q >= 1; --q)
        if (j - q >= 0) v = fma(A.c.ncoef[q - 1], x[j - q], v);
      x[j] = v;
    }
    T Q[HC];
#pragma unroll
    for (int a = 0; a < HC; ++a) Q[a] = x[P - 1 - a];
    hs_scan<HC>(Q, A.c, sqc, sqc + 24, t, NT, -1);
    if (t == NT - 1) {
#pragma unroll
      for (int a = 0; a < HC; ++a) aggc[a] = Q[a];
    }
    vec_sync(C);
    T S[HC];
    chunk_carry<HC>(S, Q, A.c, sqc, aggc, t, NT, -1, rank, C);
#pragma unroll
    for (int j = 0; j < P; ++j) {
      T v = x[j];
#pragma unroll
      for (int q = 0; q < HC; ++q) v = fma(A.c.G[j * 3 + q], S[q], v);
      x[j] = v;
    }
  }
  if constexpr (HA > 0) {
#pragma unroll
    for (int j = P - 1; j >= 0; --j) {
      T v = x[j];
#pragma unroll
      for (int q = HA; q >= 1; --q)
        if (j + q < P) v = fma(A.a.ncoef[q - 1], x[j + q], v);
      x[j] = v;
    }
    T Q[HA];
#pragma unroll
    for (int a = 0; a < HA; ++a) Q[a] = x[a];
    hs_scan<HA>(Q, A.a, sqa, sqa + 24, t, NT, +1);
    if (t == 0) {
#pragma unroll
      for (int a = 0; a < HA; ++a) agga[a] = Q[a];
    }
    vec_sync(C);
    T S[HA];
    chunk_carry<HA>(S, Q, A.a, sqa, agga, t, NT, +1, rank, C);
#pragma unroll
    for (int j = 0; j < P; ++j) {
      T v = x[j];
#pragma unroll
      for (int q = 0; q < HA; ++q) v = fma(A.a.G[(P - 1 - j) * 3 + q], S[q], v);
      x[j] = v;
    }
  }
}

}  // namespace mg
