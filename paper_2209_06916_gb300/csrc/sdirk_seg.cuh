#pragma once
// Level-0 SDIRK step kernel for many CF-intervals, FP64, one CTA per
// interval (Sec. 4.2-4.3: Phi = R_q(-c L_p) through the stages of a stiffly
// accurate SDIRK method with q <= 3 stages, each stage a periodic banded
// solve with (I + gamma c L_p)).
//
// The interval's vector lives in shared memory, one segment of S points per
// thread.  A stage solve runs the two recurrences of the factored stage
// matrix (causal, then anticausal) sequentially over the thread's segment,
// each as two cascaded sections (a real root split off as a first-order
// recurrence).  The state entering a segment is not exchanged or fixed up
// afterwards: the thread first runs the same recurrence over the last
// points of its left neighbour's segment (first points of its right
// neighbour's) from a zero state.  The recurrences are stable with roots
// inside the unit circle, so the neglected start state decays below 2^-58
// of the data within the warm-up, and the thread enters its own segment
// with the carry to that accuracy.  The first section runs over w1 points,
// the second over the last w2 of them (w2 <= w1, multiples of 8, chosen on
// the host to cost the fewest multiply-adds).
//
// Stage right-hand sides come from the solves (c L_p Y_i = (R_i - Y_i) /
// gamma), so no L_p mat-vec is needed.  For three stages, with U(b) the
// unscaled solve kappa (I + gamma c L_p)^{-1} b:
//   stage 1: U(u); R2' = e1u2 u + e1y2 U(u) (in shared memory),
//            A = e1u3 u + e1y3 U(u)       (global scratch)
//   stage 2: Y2 = U(R2');  A += e2y3 Y2
//   stage 3: u_new = U(A)
// with the 1/kappa scales folded into the coefficients.  The second vector
// (u during stage 1, A afterwards) is kept in global memory: the interval's
// own output row, written only at the end of the launch, serves as that
// scratch.
//
// Every FP64 multiply-add of a warp occupies its SM sub-partition's FP64
// pipe for 64 cycles, and the kernel runs one warp per sub-partition, so
// the other instructions must neither stall the next multiply-add nor be
// numerous: data moves in 16-byte pairs (shared memory segments padded to
// S + 2 values; the scratch row interleaved in pairs, element j of thread t
// at (j/2) 2T + 2t + j%2, so a warp's pair loads are one contiguous 512-byte
// access), and the pairs of the next block of 8 points are loaded while the
// current block computes.
#include <cuda_runtime.h>
#include <stdint.h>

#include "dsolve.cuh"
#include "kernels.h"

namespace mg {

// One pass over `count` points (a multiple of 8) in pass order i = 0, 1, ...
// ld(i), i even, loads the pair of inputs of points i and i+1 (an ascending
// pass: .x is point i; a descending one: .y is point i); f(i, x) maps an
// input to a result (a double2: one or two outputs); st(i, r_i, r_{i+1})
// stores the results of the pair.  Blocks of 8 points are double buffered:
// the next block's four pairs load while the current one computes.
template <bool DESC, typename LD, typename F, typename ST>
__device__ __forceinline__ void pair_pass(int count, LD ld, F f, ST st) {
  if (count <= 0) return;
  typedef decltype(ld(0)) V;
  V a[4], b[4];
  auto run = [&](int i0, const V (&v)[4]) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i = i0 + 2 * q;
      const auto r0 = f(i, v[q], DESC ? 1 : 0);
      const auto r1 = f(i + 1, v[q], DESC ? 0 : 1);
      st(i, r0, r1);
    }
  };
#pragma unroll
  for (int q = 0; q < 4; ++q) a[q] = ld(2 * q);
  int i0 = 0;
  for (; i0 + 16 <= count; i0 += 16) {
#pragma unroll
    for (int q = 0; q < 4; ++q) b[q] = ld(i0 + 8 + 2 * q);
    run(i0, a);
    if (i0 + 16 < count) {
#pragma unroll
      for (int q = 0; q < 4; ++q) a[q] = ld(i0 + 16 + 2 * q);
    }
    run(i0 + 8, b);
  }
  if (i0 < count) run(i0, a);
}

// two pairs loaded together (the shared-memory input and the scratch)
struct Pair2 {
  double2 w, z;
};
__device__ __forceinline__ double lane_of(const double2& v, int h) { return h ? v.y : v.x; }

template <int C1, int C2, int A1, int A2, int S>
__global__ void __launch_bounds__(128) sdirk_seg_kernel(const __grid_constant__ SdirkSegParams A) {
  extern __shared__ __align__(16) double smem[];
  constexpr int SP = S + 2;  // padded segment stride: 16-byte aligned, conflict-free pair columns
  const int T = A.T, t = threadIdx.x, n = A.n;
  double* w = smem;
  double* red = smem + (size_t)T * SP;
  const int64_t k = blockIdx.x;
  const int mode = A.mode;
  double* orow = A.out + (mode == kModeAPPLY ? k : k + 1) * (int64_t)n;
  double* aux = orow;  // scratch until the final write
  const int tl = (t == 0) ? T - 1 : t - 1;
  const int tr = (t == T - 1) ? 0 : t + 1;
  double* wo = w + t * SP;         // own segment
  const double* wl = w + tl * SP;  // left neighbour's segment
  const double* wr = w + tr * SP;  // right neighbour's segment
  const int stages = A.stages;
  const int rc1 = A.rc1, rc2 = A.rc2, ra1 = A.ra1, ra2 = A.ra2;
  const double cr = A.cr, cd0 = A.cd[0], cd1 = A.cd[1];
  const double ar = A.ar, ad0 = A.ad[0], ad1 = A.ad[1];

  if (A.zero_start) {
    for (int i = t; i < n; i += T) w[i + 2 * (i / S)] = 0.0;
  } else {
    const double* src = A.start + k * (int64_t)n;
    for (int i = t; i < n; i += T) w[i + 2 * (i / S)] = src[i];
  }

  // pair loads / stores: shared-memory segments, and the pair-interleaved
  // scratch of thread tt (the pair j, j+1 at (j/2) 2T + 2tt)
  auto lds2 = [](const double* p, int j) { return *reinterpret_cast<const double2*>(p + j); };
  auto sts2 = [&](int j, double a, double b) { *reinterpret_cast<double2*>(wo + j) = make_double2(a, b); };
  auto aux2 = [&](int tt, int j) -> double2* {
    return reinterpret_cast<double2*>(aux + (size_t)(j >> 1) * (2 * T) + 2 * tt);
  };
  auto nost = [](int, double, double) {};

  // causal recurrence, two cascaded sections: y_i = b_i + cr y_{i-1},
  // x_i = y_i + cd1 x_{i-2} + cd0 x_{i-1}
  double cy, cx1, cx2;
  auto csec1 = [&](double b) {
    if (!C1) return b;
    cy = fma(cr, cy, b);
    return cy;
  };
  auto csec2 = [&](double y) {
    double x = y;
    if (C2 >= 2) x = fma(cd1, cx2, x);
    if (C2 >= 1) {
      x = fma(cd0, cx1, x);
      cx2 = cx1;
      cx1 = x;
    }
    return x;
  };
  // anticausal recurrence, the same two sections towards decreasing i
  double au, av1, av2;
  auto asec1 = [&](double b) {
    if (!A1) return b;
    au = fma(ar, au, b);
    return au;
  };
  auto asec2 = [&](double u) {
    double v = u;
    if (A2 >= 2) v = fma(ad1, av2, v);
    if (A2 >= 1) {
      v = fma(ad0, av1, v);
      av2 = av1;
      av1 = v;
    }
    return v;
  };
  constexpr bool anti = (A1 + A2) > 0;
  // the pair element h of v through the sections
  auto c1only = [&](int, double2 v, int h) { return csec1(lane_of(v, h)); };
  auto cboth = [&](int, double2 v, int h) { return csec2(csec1(lane_of(v, h))); };
  auto a1only = [&](int, double2 v, int h) { return asec1(lane_of(v, h)); };
  auto aboth = [&](int, double2 v, int h) { return asec2(asec1(lane_of(v, h))); };
  auto yv = [&](double xv) { return anti ? asec2(asec1(xv)) : xv; };

  for (int s = 0; s < A.nsteps; ++s) {
    for (int st = 1; st <= stages; ++st) {
      const bool from_aux = (st == 3);
      // every write of the previous stage (shared memory and scratch) is
      // visible and every read of a neighbour's segment is done
      __syncthreads();
      // causal warm-up over the left neighbour's last rc1 points: the first
      // section alone, then both over the last rc2
      cy = cx1 = cx2 = 0.0;
      if (from_aux) {
        pair_pass<false>(rc1 - rc2, [&](int i) { return *aux2(tl, S - rc1 + i); }, c1only, nost);
        pair_pass<false>(rc2, [&](int i) { return *aux2(tl, S - rc2 + i); }, cboth, nost);
      } else {
        pair_pass<false>(rc1 - rc2, [&](int i) { return lds2(wl, S - rc1 + i); }, c1only, nost);
        pair_pass<false>(rc2, [&](int i) { return lds2(wl, S - rc2 + i); }, cboth, nost);
        __syncthreads();  // the neighbour's tail is read before it is overwritten
      }
      // causal pass over the own segment (stage 1 of several also keeps u
      // in the scratch for its epilogue)
      if (from_aux) {
        pair_pass<false>(S, [&](int j) { return *aux2(t, j); }, cboth, sts2);
      } else if (st == 1 && stages >= 2) {
        pair_pass<false>(S, [&](int j) {
          const double2 v = lds2(wo, j);
          *aux2(t, j) = v;
          return v;
        }, cboth, sts2);
      } else {
        pair_pass<false>(S, [&](int j) { return lds2(wo, j); }, cboth, sts2);
      }
      // anticausal warm-up over the right neighbour's first ra1 points,
      // descending: the first section alone, then both over the last ra2
      au = av1 = av2 = 0.0;
      if (anti) {
        __syncthreads();
        pair_pass<true>(ra1 - ra2, [&](int i) { return lds2(wr, ra1 - 2 - i); }, a1only, nost);
        pair_pass<true>(ra2, [&](int i) { return lds2(wr, ra2 - 2 - i); }, aboth, nost);
        __syncthreads();  // the neighbour's head is read before it is overwritten
      }
      // own segment, descending (pass index i: point S - 1 - i; the pair of
      // pass indices i, i+1 sits at S - 2 - i): anticausal pass and the
      // stage's epilogue
      //   last stage            w = last * y
      //   stage 1 (of 2 or 3)   w = e1u2 u + e1y2 y, and for 3 stages
      //                         aux = e1u3 u + e1y3 y (u read from aux)
      //   stage 2 of 3          aux += e2y3 y
      if (st == stages) {
        const double sc = A.last;
        pair_pass<true>(S, [&](int i) { return lds2(wo, S - 2 - i); },
                        [&](int, double2 v, int h) { return sc * yv(lane_of(v, h)); },
                        [&](int i, double r0, double r1) { sts2(S - 2 - i, r1, r0); });
      } else if (st == 1) {
        const double e1u2 = A.e1u2, e1y2 = A.e1y2, e1u3 = A.e1u3, e1y3 = A.e1y3;
        const bool three = (stages == 3);
        pair_pass<true>(S, [&](int i) { return Pair2{lds2(wo, S - 2 - i), *aux2(t, S - 2 - i)}; },
                        [&](int, Pair2 v, int h) {
                          const double y = yv(lane_of(v.w, h)), u = lane_of(v.z, h);
                          return make_double2(fma(e1y2, y, e1u2 * u), fma(e1y3, y, e1u3 * u));
                        },
                        [&](int i, double2 r0, double2 r1) {
                          sts2(S - 2 - i, r1.x, r0.x);
                          if (three) *aux2(t, S - 2 - i) = make_double2(r1.y, r0.y);
                        });
      } else {
        const double e2y3 = A.e2y3;
        pair_pass<true>(S, [&](int i) { return Pair2{lds2(wo, S - 2 - i), *aux2(t, S - 2 - i)}; },
                        [&](int, Pair2 v, int h) { return fma(e2y3, yv(lane_of(v.w, h)), lane_of(v.z, h)); },
                        [&](int i, double r0, double r1) { *aux2(t, S - 2 - i) = make_double2(r1, r0); });
      }
    }
  }
  __syncthreads();
  if (mode == kModeCF || mode == kModeFRES || mode == kModeAPPLY) {
    const double* sb = (mode == kModeFRES && A.sub) ? A.sub + (k + 1) * (int64_t)n : nullptr;
    double sq = 0.0;
    for (int i = t; i < n; i += T) {
      double v = w[i + 2 * (i / S)];
      if (sb) v -= sb[i];
      orow[i] = v;
      sq = fma(v, v, sq);
    }
    if (mode == kModeFRES && A.partial) {
      const double tot = block_sum(sq, red);
      if (t == 0) A.partial[k] = tot;
    }
  }
}

}  // namespace mg
