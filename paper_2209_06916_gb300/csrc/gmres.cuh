#pragma once
// GMRES for the correction system (I - sum_t phi_t D_t) x = b of a coarse
// level, b the SL-gathered vector (Sec. 6.1: the exact solve may be replaced
// by a few GMRES iterations; Sec. 6.3: stop once the l2 residual has fallen
// by a factor rtol = 1e-2 from a zero guess, or at the iteration cap).
//
// The vector is split over the CTAs of a thread-block cluster and over their
// threads in chunks of P points held in registers.  The Krylov basis lives
// in global scratch (one region per CF-interval), each thread reading back
// only the points it wrote, in a layout where a warp's loads of one point
// index are contiguous.  Orthogonalisation is classical Gram-Schmidt with
// one re-orthogonalisation; the new vector's norm comes from the second
// pass's sums (||w2||^2 = ||w1||^2 - ||h2||^2), so an iteration costs one
// mat-vec halo exchange and two cluster-wide reductions.  Every CTA's thread
// 0 applies the Givens rotations to the Hessenberg column from the same
// fixed-order sums, so all CTAs of the cluster agree bit for bit.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "dsolve.cuh"
#include "kernels.h"

namespace mg {

// shared work area of one CTA, in doubles: per-warp partials [8][KS], CTA
// sums [2][KS] (read by the cluster, double-buffered), cluster sums [KS],
// Hessenberg columns [kGmMax][kGmMax + 1], rotations cs, sn [kGmMax], the
// rotated right-hand side g [kGmMax + 1], y [kGmMax], flags [2]
constexpr int kGmKS = kGmMax + 2;
constexpr int kGmSharedDoubles = 8 * kGmKS + 2 * kGmKS + kGmKS + kGmMax * (kGmMax + 1) + 2 * kGmMax +
                                 (kGmMax + 1) + kGmMax + 2;

// w = (I - sum phi D) v on the thread's chunk; the H points on either side
// come from the neighbouring chunks in `gv` (this CTA) or in the previous /
// next CTA's buffer (gl / gr; the same buffer when the vector has one CTA).
template <typename TC, int P, int H>
__device__ __forceinline__ void gm_matvec(TC (&w)[P], const TC (&v)[P], const TC* gv, const TC* gl, const TC* gr,
                                          const TC* taps, int t, int NT) {
  TC win[P + 2 * H];
  const TC* lsrc = (t > 0) ? gv + (t - 1) * (P + 1) + P - H : gl + (NT - 1) * (P + 1) + P - H;
  const TC* rsrc = (t + 1 < NT) ? gv + (t + 1) * (P + 1) : gr;
#pragma unroll
  for (int a = 0; a < H; ++a) win[a] = lsrc[a];
#pragma unroll
  for (int i = 0; i < P; ++i) win[H + i] = v[i];
#pragma unroll
  for (int a = 0; a < H; ++a) win[H + P + a] = rsrc[a];
#pragma unroll
  for (int i = 0; i < P; ++i) {
    TC acc = TC(0);
#pragma unroll
    for (int d = 0; d <= 2 * H; ++d) acc = fma(taps[3 - H + d], win[i + d], acc);
    w[i] = acc;
  }
}

// In place: x holds b on entry and the GMRES iterate on return.  Every
// thread of every CTA of the cluster calls it.  gv: TC[NT * (P + 1)] shared
// buffer; gs: kGmSharedDoubles shared doubles; k: the cluster's interval.
template <typename TC, int P, int H, typename Prm>
__device__ __forceinline__ void gmres_solve(TC (&x)[P], const Prm& A, TC* gv, double* gs, int t, int rank, int C,
                                            int64_t k) {
  const int NT = A.nthr, lane = t & 31, wid = t >> 5, nw = (NT + 31) >> 5;
  const int wlen = min(32, NT - (wid << 5));
  const unsigned mask = (wlen == 32) ? 0xffffffffu : ((1u << wlen) - 1u);
  double* red = gs;
  double* part = red + 8 * kGmKS;
  double* tot = part + 2 * kGmKS;
  double* Hc = tot + kGmKS;
  double* cs = Hc + kGmMax * (kGmMax + 1);
  double* sn = cs + kGmMax;
  double* gg = sn + kGmMax;
  double* y = gg + kGmMax + 1;
  double* flag = y + kGmMax;
  const int M = A.gm_max;
  const size_t cstride = (size_t)NT * P;  // one CTA's share of one basis vector
  TC* const V0 = A.gm_V + ((size_t)k * (size_t)(M + 1) * (size_t)C + (size_t)rank) * cstride + t;
  auto Vj = [&](int j) -> TC* { return V0 + (size_t)j * (size_t)C * cstride; };
  cgc::cluster_group cl = cgc::this_cluster();
  const TC* gl = (C == 1) ? gv : cl.map_shared_rank(gv, (rank + C - 1) % C);
  const TC* gr = (C == 1) ? gv : cl.map_shared_rank(gv, (rank + 1) % C);

  // warp sum of d (lanes in order) into red[warp][i]
  auto warp_put = [&](double d, int i) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double u = __shfl_down_sync(mask, d, o);
      if (lane + o < wlen) d += u;
    }
    if (lane == 0) red[wid * kGmKS + i] = d;
  };
  // cluster sums tot[0..nv) of the values put since the last call: warps in
  // order, then CTAs in rank order
  auto reduce = [&](int nv, int buf) {
    __syncthreads();
    for (int i = t; i < nv; i += NT) {
      double s = 0.0;
      for (int q = 0; q < nw; ++q) s += red[q * kGmKS + i];
      part[buf * kGmKS + i] = s;
    }
    vec_sync(C);
    for (int i = t; i < nv; i += NT) {
      double s = 0.0;
      for (int r = 0; r < C; ++r) {
        const double* pr = (C == 1) ? part : cl.map_shared_rank(part, r);
        s += pr[buf * kGmKS + i];
      }
      tot[i] = s;
    }
    __syncthreads();
  };
  auto dot_put = [&](const TC (&w)[P], int i) {
    const TC* Vi = Vj(i);
    TC s = TC(0);
#pragma unroll
    for (int p = 0; p < P; ++p) s = fma(w[p], Vi[(size_t)p * NT], s);
    warp_put((double)s, i);
  };
  auto axpy_basis = [&](TC (&w)[P], int i, TC c) {
    const TC* Vi = Vj(i);
#pragma unroll
    for (int p = 0; p < P; ++p) w[p] = fma(c, Vi[(size_t)p * NT], w[p]);
  };
  auto store_basis = [&](const TC (&v)[P], int j) {
    TC* Vd = Vj(j);
#pragma unroll
    for (int p = 0; p < P; ++p) Vd[(size_t)p * NT] = v[p];
  };

  // beta = ||b||
  {
    TC s = TC(0);
#pragma unroll
    for (int p = 0; p < P; ++p) s = fma(x[p], x[p], s);
    warp_put((double)s, 0);
    reduce(1, 1);
  }
  const double beta = sqrt(tot[0]);
  if (beta == 0.0) {
#pragma unroll
    for (int p = 0; p < P; ++p) x[p] = TC(0);
    return;
  }
  if (!isfinite(beta)) return;  // a non-finite RHS stays non-finite
  TC v[P];
  {
    const double ib = 1.0 / beta;
#pragma unroll
    for (int p = 0; p < P; ++p) v[p] = (TC)((double)x[p] * ib);
  }
  store_basis(v, 0);
  if (t == 0) gg[0] = beta;
  int kk = 0;
  for (int j = 0; j < M; ++j) {
    // w = A v_j
#pragma unroll
    for (int p = 0; p < P; ++p) gv[t * (P + 1) + p] = v[p];
    vec_sync(C);
    TC w[P];
    gm_matvec<TC, P, H>(w, v, gv, gl, gr, A.gm_taps, t, NT);
    // first Gram-Schmidt pass
    for (int i = 0; i <= j; ++i) dot_put(w, i);
    reduce(j + 1, 0);
    for (int i = 0; i <= j; ++i) axpy_basis(w, i, (TC)(-tot[i]));
    if (t == 0)
      for (int i = 0; i <= j; ++i) Hc[j * (kGmMax + 1) + i] = tot[i];
    // second pass, with ||w||^2 of the vector it starts from
    for (int i = 0; i <= j; ++i) dot_put(w, i);
    {
      TC s = TC(0);
#pragma unroll
      for (int p = 0; p < P; ++p) s = fma(w[p], w[p], s);
      warp_put((double)s, j + 1);
    }
    reduce(j + 2, 1);
    for (int i = 0; i <= j; ++i) axpy_basis(w, i, (TC)(-tot[i]));
    if (t == 0) {
      double* hc = Hc + j * (kGmMax + 1);
      double s2 = 0.0;
      for (int i = 0; i <= j; ++i) {
        hc[i] += tot[i];
        s2 += tot[i] * tot[i];
      }
      const double hn = sqrt(fmax(tot[j + 1] - s2, 0.0));
      for (int i = 0; i < j; ++i) {
        const double a = hc[i], b = hc[i + 1];
        hc[i] = cs[i] * a + sn[i] * b;
        hc[i + 1] = -sn[i] * a + cs[i] * b;
      }
      const double a = hc[j];
      const double den = hypot(a, hn);
      const double c = den > 0.0 ? a / den : 1.0, s = den > 0.0 ? hn / den : 0.0;
      cs[j] = c;
      sn[j] = s;
      hc[j] = den;
      gg[j + 1] = -s * gg[j];
      gg[j] = c * gg[j];
      const bool stop = fabs(gg[j + 1]) <= A.gm_rtol * beta || hn == 0.0 || j + 1 == M;
      flag[0] = stop ? 1.0 : 0.0;
      flag[1] = hn;
    }
    __syncthreads();
    kk = j + 1;
    if (flag[0] != 0.0) break;
    const double ih = 1.0 / flag[1];
#pragma unroll
    for (int p = 0; p < P; ++p) v[p] = (TC)((double)w[p] * ih);
    store_basis(v, j + 1);
  }
  // y = R^{-1} g, x = V y
  if (t == 0) {
    for (int i = kk - 1; i >= 0; --i) {
      double s = gg[i];
      for (int l = i + 1; l < kk; ++l) s -= Hc[l * (kGmMax + 1) + i] * y[l];
      y[i] = s / Hc[i * (kGmMax + 1) + i];
    }
    if (rank == 0 && A.gm_stats) {
      atomicAdd(A.gm_stats, (unsigned long long)kk);
      atomicAdd(A.gm_stats + 1, 1ull);
    }
  }
  __syncthreads();
#pragma unroll
  for (int p = 0; p < P; ++p) x[p] = TC(0);
  for (int i = 0; i < kk; ++i) axpy_basis(x, i, (TC)y[i]);
}

}  // namespace mg
