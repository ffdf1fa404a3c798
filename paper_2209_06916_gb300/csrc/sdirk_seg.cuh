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
// inside the unit circle, so the neglected start state decays below 2^-56
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

// A stream of value pairs: pair jj at p + jj * stride (in pairs; stride 1
// for a shared-memory segment, T for a thread's pairs in the interleaved
// scratch).  Block loads take a base pointer per block of 4 pairs and
// constant multiples of the stride, so the address arithmetic per access is
// one add.
struct PairStream {
  double2* p;
  int s1, s2, s3;  // stride, 2 stride, 3 stride
  __device__ __forceinline__ double2* at(int jj) const { return p + (size_t)jj * s1; }
  __device__ __forceinline__ void load4(const double2* b, double2 (&v)[4]) const {
    v[0] = b[0];
    v[1] = b[s1];
    v[2] = b[s2];
    v[3] = b[s3];
  }
};
__device__ __forceinline__ PairStream pair_stream(double* base, int stride) {
  return PairStream{reinterpret_cast<double2*>(base), stride, 2 * stride, 3 * stride};
}

// One pass over npairs pairs of a stream (a multiple of 4), ascending
// (pairs 0, 1, ...; element .x first) or descending (pairs from the last
// down; element .y first).  f(x) is called once per element in pass order;
// st(pair index, result of .x, result of .y) stores a pair.  The next block of 4 pairs loads while the current block
// computes (two register buffers, no copies).
template <bool DESC, typename F, typename ST>
__device__ __forceinline__ void stream_pass(const PairStream& in, int npairs, F f, ST st) {
  if (npairs <= 0) return;
  const int blocks = npairs >> 2;
  auto base = [&](int b) -> const double2* { return in.at(DESC ? npairs - 4 - 4 * b : 4 * b); };
  double2 va[4], vb[4];
  auto run = [&](int b, const double2 (&v)[4]) {
    const int jj0 = DESC ? npairs - 4 - 4 * b : 4 * b;
#pragma unroll
    for (int q0 = 0; q0 < 4; ++q0) {
      const int q = DESC ? 3 - q0 : q0;
      double r0, r1;
      if (DESC) {
        r1 = f(v[q].y);
        r0 = f(v[q].x);
      } else {
        r0 = f(v[q].x);
        r1 = f(v[q].y);
      }
      st(jj0 + q, r0, r1);
    }
  };
  in.load4(base(0), va);
  int b = 0;
  for (; b + 2 <= blocks; b += 2) {
    in.load4(base(b + 1), vb);
    run(b, va);
    if (b + 2 < blocks) in.load4(base(b + 2), va);
    run(b + 1, vb);
  }
  if (b < blocks) run(b, va);
}

// the same over two streams read together: f(x, z) per element
template <bool DESC, typename F, typename ST>
__device__ __forceinline__ void stream_pass2(const PairStream& in, const PairStream& in2, int npairs, F f, ST st) {
  if (npairs <= 0) return;
  const int blocks = npairs >> 2;
  auto jjb = [&](int b) { return DESC ? npairs - 4 - 4 * b : 4 * b; };
  double2 va[4], vb[4], za[4], zb[4];
  auto run = [&](int b, const double2 (&v)[4], const double2 (&z)[4]) {
    const int jj0 = jjb(b);
#pragma unroll
    for (int q0 = 0; q0 < 4; ++q0) {
      const int q = DESC ? 3 - q0 : q0;
      double r0, r1;
      if (DESC) {
        r1 = f(v[q].y, z[q].y);
        r0 = f(v[q].x, z[q].x);
      } else {
        r0 = f(v[q].x, z[q].x);
        r1 = f(v[q].y, z[q].y);
      }
      st(jj0 + q, r0, r1);
    }
  };
  in.load4(in.at(jjb(0)), va);
  in2.load4(in2.at(jjb(0)), za);
  int b = 0;
  for (; b + 2 <= blocks; b += 2) {
    in.load4(in.at(jjb(b + 1)), vb);
    in2.load4(in2.at(jjb(b + 1)), zb);
    run(b, va, za);
    if (b + 2 < blocks) {
      in.load4(in.at(jjb(b + 2)), va);
      in2.load4(in2.at(jjb(b + 2)), za);
    }
    run(b + 1, vb, zb);
  }
  if (b < blocks) run(b, va, za);
}

template <int STAGES, int C1, int C2, int A1, int A2, int S>
__global__ void __launch_bounds__(128) sdirk_seg_kernel(const __grid_constant__ SdirkSegParams A) {
  extern __shared__ __align__(16) double smem[];
  constexpr int SP = S + 2;  // padded segment stride: 16-byte aligned, conflict-free pair columns
  constexpr int NP = S / 2;  // pairs per segment
  const int T = A.T, t = threadIdx.x, n = A.n;
  double* w = smem;
  double* red = smem + (size_t)T * SP;
  const int64_t k = blockIdx.x;
  const int mode = A.mode;
  double* orow = A.out + (mode == kModeAPPLY ? k : k + 1) * (int64_t)n;
  double* aux = orow;  // scratch until the final write (the host launches this kernel on 16-byte aligned rows only)
  const int tl = (t == 0) ? T - 1 : t - 1;
  const int tr = (t == T - 1) ? 0 : t + 1;
  // streams: own / left / right segments, own / left scratch pairs
  const PairStream own = pair_stream(w + t * SP, 1);
  const PairStream left = pair_stream(w + tl * SP, 1);
  const PairStream right = pair_stream(w + tr * SP, 1);
  const PairStream xown = pair_stream(aux + 2 * t, T);
  const PairStream xleft = pair_stream(aux + 2 * tl, T);
  const int rc1 = A.rc1, rc2 = A.rc2, ra1 = A.ra1, ra2 = A.ra2;
  const double cr = A.cr, cd0 = A.cd[0], cd1 = A.cd[1];
  const double ar = A.ar, ad0 = A.ad[0], ad1 = A.ad[1];

  // rows of global memory move as 16-byte pairs when the pointers allow it
  // (a test uniform over the CTA), in batches of independent loads so that
  // their latencies overlap
  auto al16 = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
  auto sidx = [&](int i) { return i + 2 * (i / S); };  // vector element -> segment slot
  constexpr int NPR = S / 2;                              // pairs per thread (n = S T)
  constexpr int PB = 8;                                   // pairs per batch
  static_assert(NPR % PB == 0, "segment length");
  {
    const double* src = A.start + k * (int64_t)n;
    if (A.zero_start) {
      for (int i = t; i < n; i += T) w[sidx(i)] = 0.0;
    } else if (al16(src)) {
      const double2* s2 = reinterpret_cast<const double2*>(src);
      for (int j0 = 0; j0 < NPR; j0 += PB) {
        double2 v[PB];
#pragma unroll
        for (int u = 0; u < PB; ++u) v[u] = s2[t + (j0 + u) * T];
#pragma unroll
        for (int u = 0; u < PB; ++u) *reinterpret_cast<double2*>(w + sidx(2 * (t + (j0 + u) * T))) = v[u];
      }
    } else {
      for (int i = t; i < n; i += T) w[sidx(i)] = src[i];
    }
  }

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
  auto cboth = [&](double b) { return csec2(csec1(b)); };
  auto yv = [&](double xv) { return anti ? asec2(asec1(xv)) : xv; };
  auto nost = [](int, double, double) {};
  auto st_own = [&](int jj, double r0, double r1) { *own.at(jj) = make_double2(r0, r1); };

  for (int s = 0; s < A.nsteps; ++s) {
#pragma unroll 1
    for (int st = 1; st <= STAGES; ++st) {
      const bool from_aux = (st == 3);
      // every write of the previous stage (shared memory and scratch) is
      // visible and every read of a neighbour's segment is done
      __syncthreads();
      // causal warm-up over the left neighbour's last rc1 points: the first
      // section alone, then both over the last rc2
      cy = cx1 = cx2 = 0.0;
      {
        const PairStream& src = from_aux ? xleft : left;
        const PairStream w1 = PairStream{src.at(NP - rc1 / 2), src.s1, src.s2, src.s3};
        const PairStream w2 = PairStream{src.at(NP - rc2 / 2), src.s1, src.s2, src.s3};
        stream_pass<false>(w1, (rc1 - rc2) / 2, [&](double b) { return csec1(b); }, nost);
        stream_pass<false>(w2, rc2 / 2, cboth, nost);
      }
      if (!from_aux) __syncthreads();  // the neighbour's tail is read before it is overwritten
      // causal pass over the own segment (stage 1 of several also keeps u
      // in the scratch for its epilogue)
      if (from_aux) {
        stream_pass<false>(xown, NP, cboth, st_own);
      } else if (st == 1 && STAGES >= 2) {
        stream_pass2<false>(own, own, NP, [&](double b, double) { return cboth(b); },
                            [&](int jj, double r0, double r1) {
                              *xown.at(jj) = *own.at(jj);
                              *own.at(jj) = make_double2(r0, r1);
                            });
      } else {
        stream_pass<false>(own, NP, cboth, st_own);
      }
      // anticausal warm-up over the right neighbour's first ra1 points,
      // descending: the first section alone, then both over the last ra2
      au = av1 = av2 = 0.0;
      if (anti) {
        __syncthreads();
        const PairStream w1 = PairStream{right.at(ra2 / 2), 1, 2, 3};
        stream_pass<true>(w1, (ra1 - ra2) / 2, [&](double b) { return asec1(b); }, nost);
        stream_pass<true>(right, ra2 / 2, [&](double b) { return asec2(asec1(b)); }, nost);
        __syncthreads();  // the neighbour's head is read before it is overwritten
      }
      // own segment, descending: anticausal pass and the stage's epilogue
      //   last stage            w = last * y
      //   stage 1 (of 2 or 3)   w = e1u2 u + e1y2 y, and for 3 stages
      //                         aux = e1u3 u + e1y3 y (u read from aux)
      //   stage 2 of 3          aux += e2y3 y
      if (st == STAGES) {
        if (STAGES == 1) {  // one stage: Y = U(u) / kappa
          const double sc = A.last;
          stream_pass<true>(own, NP, [&](double xv) { return sc * yv(xv); }, st_own);
        } else {  // the scales are folded into the right-hand side
          stream_pass<true>(own, NP, [&](double xv) { return yv(xv); }, st_own);
        }
      } else if (st == 1) {
        const double e1u2 = A.e1u2, e1y2 = A.e1y2, e1u3 = A.e1u3, e1y3 = A.e1y3;
        double a3 = 0.0, a3p = 0.0;
        stream_pass2<true>(own, xown, NP,
                           [&](double xv, double u) {
                             const double y = yv(xv);
                             a3p = a3;
                             if (STAGES == 3) a3 = fma(e1y3, y, e1u3 * u);
                             return fma(e1y2, y, e1u2 * u);
                           },
                           [&](int jj, double r0, double r1) {
                             *own.at(jj) = make_double2(r0, r1);
                             // descending: r1 (point 2jj+1) was computed first, r0 last
                             if (STAGES == 3) *xown.at(jj) = make_double2(a3, a3p);
                           });
      } else {
        const double e2y3 = A.e2y3;
        stream_pass2<true>(own, xown, NP,
                           [&](double xv, double a) { return fma(e2y3, yv(xv), a); },
                           [&](int jj, double r0, double r1) { *xown.at(jj) = make_double2(r0, r1); });
      }
    }
  }
  __syncthreads();
  if (mode == kModeCF || mode == kModeFRES || mode == kModeAPPLY) {
    const double* sb = (mode == kModeFRES && A.sub) ? A.sub + (k + 1) * (int64_t)n : nullptr;
    double sq = 0.0;
    if (al16(orow) && (!sb || al16(sb))) {
      const double2* sb2 = reinterpret_cast<const double2*>(sb);
      double2* o2 = reinterpret_cast<double2*>(orow);
      for (int j0 = 0; j0 < NPR; j0 += PB) {
        double2 b[PB];
        if (sb) {
#pragma unroll
          for (int u = 0; u < PB; ++u) b[u] = sb2[t + (j0 + u) * T];
        }
#pragma unroll
        for (int u = 0; u < PB; ++u) {
          const int pr = t + (j0 + u) * T;
          double2 v = *reinterpret_cast<const double2*>(w + sidx(2 * pr));
          if (sb) {
            v.x -= b[u].x;
            v.y -= b[u].y;
          }
          o2[pr] = v;
          sq = fma(v.x, v.x, sq);
          sq = fma(v.y, v.y, sq);
        }
      }
    } else {
      for (int i = t; i < n; i += T) {
        double v = w[sidx(i)];
        if (sb) v -= sb[i];
        orow[i] = v;
        sq = fma(v, v, sq);
      }
    }
    if (mode == kModeFRES && A.partial) {
      const double tot = block_sum(sq, red);
      if (t == 0) A.partial[k] = tot;
    }
  }
}

}  // namespace mg
