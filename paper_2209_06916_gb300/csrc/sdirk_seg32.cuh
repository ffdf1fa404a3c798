#pragma once
// Level-0 SDIRK step kernel of MIXED inner cycles: FP32, one CTA per
// CF-interval, the vector's three stage slots in shared memory, one segment
// of S points per thread (Sec. 4.2-4.3: Phi = R_q(-c L_p) through the stages
// of a stiffly accurate SDIRK method, q = 1 or 3).  The FP32 step keeps the
// mat-vec form of the stages,
//   R_j = u (j >= 1);  Y_i = (I + gamma c L_p)^{-1} R_i;
//   R_j += -c a_ji L_p Y_i  (j > i);  u_new = Y_{s-1},
// whose rounding leaves the refinement at FP64 accuracy.  The stage solves
// run the factored recurrences over the thread's segment with warm-ups over
// the neighbouring segments, as the FP64 kernel (sdirk_seg.cuh) does, with
// the warm-ups cut where the neglected state falls below 2^-27 (below FP32
// rounding); the mat-vec L_p Y_i takes its halo (l(p) points to the west,
// r(p) to the east) from the neighbouring segments.  The slots' roles rotate
// every step (the last stage's slot holds the next state), so no copy-back.
// Data move as 4-float quads (segments padded to S + 4 values), the next
// block of 8 points loading while the current one computes.
#include <cuda_runtime.h>
#include <stdint.h>

#include "dsolve.cuh"
#include "kernels.h"

namespace mg {

// One pass over `count` points (a multiple of 8) of a shared-memory segment
// seg (16-byte aligned), ascending or descending: f(x) per point in pass
// order, st(point index of the quad's first element, r0, r1, r2, r3) stores
// the results of the quad (in memory order).
template <bool DESC, typename F, typename ST>
__device__ __forceinline__ void quad_pass(const float* seg, int count, F f, ST st) {
  if (count <= 0) return;
  auto ld = [&](int q) { return *reinterpret_cast<const float4*>(seg + 4 * q); };  // quad q
  const int nq = count >> 2;
  auto qidx = [&](int i) { return DESC ? nq - 1 - i : i; };  // pass quad i -> memory quad
  float4 a[2], b[2];
  auto run = [&](int i0, const float4 (&v)[2]) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int q = qidx(i0 + h);
      float r0, r1, r2, r3;
      if (DESC) {
        r3 = f(v[h].w);
        r2 = f(v[h].z);
        r1 = f(v[h].y);
        r0 = f(v[h].x);
      } else {
        r0 = f(v[h].x);
        r1 = f(v[h].y);
        r2 = f(v[h].z);
        r3 = f(v[h].w);
      }
      st(4 * q, r0, r1, r2, r3);
    }
  };
  a[0] = ld(qidx(0));
  a[1] = ld(qidx(1));
  int i0 = 0;
  for (; i0 + 4 <= nq; i0 += 4) {
    b[0] = ld(qidx(i0 + 2));
    b[1] = ld(qidx(i0 + 3));
    run(i0, a);
    if (i0 + 4 < nq) {
      a[0] = ld(qidx(i0 + 4));
      a[1] = ld(qidx(i0 + 5));
    }
    run(i0 + 2, b);
  }
  if (i0 < nq) run(i0, a);
}

template <int STAGES, int C1, int C2, int A1, int A2, int HL, int HR, int S>
__global__ void __launch_bounds__(256) sdirk_seg32_kernel(const __grid_constant__ SdirkSeg32Params A) {
  extern __shared__ __align__(16) float smem32[];
  constexpr int SP = S + 4;  // padded segment stride: 16-byte aligned, conflict-free quad columns
  constexpr int P1 = HL + 1 + HR;
  const int T = A.T, t = threadIdx.x, n = A.n;
  const size_t slot = (size_t)T * SP;
  float* const sl0 = smem32;
  float* const sl1 = smem32 + slot;
  float* const sl2 = smem32 + 2 * slot;
  auto slot_of = [&](int i) { return i == 0 ? sl0 : (i == 1 ? sl1 : sl2); };
  double* red = reinterpret_cast<double*>(smem32 + 3 * slot);
  const int64_t k = blockIdx.x;
  const int tl = (t == 0) ? T - 1 : t - 1;
  const int tr = (t == T - 1) ? 0 : t + 1;
  const int own = t * SP, lft = tl * SP, rgt = tr * SP;
  const int rc1 = A.rc1, rc2 = A.rc2, ra1 = A.ra1, ra2 = A.ra2;
  const float cr = A.cr, cd0 = A.cd[0], cd1 = A.cd[1];
  const float ar = A.ar, ad0 = A.ad[0], ad1 = A.ad[1];
  const float ik = A.ik;
  float lt[P1];
#pragma unroll
  for (int a = 0; a < P1; ++a) lt[a] = A.ltaps[a];

  // rows of global memory move as 16-byte quads when the pointers allow it
  // (a test uniform over the CTA), in batches of independent loads so that
  // their latencies overlap
  auto al16 = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
  auto sidx = [&](int i) { return i + 4 * (i / S); };  // vector element -> slot index
  constexpr int NQ = S / 4;                               // quads per thread (n = S T)
  constexpr int QB = NQ < 8 ? NQ : 8;                     // quads per batch
  {
    float* w = sl0;
    const float* src = A.start + k * (int64_t)n;
    if (A.zero_start) {
      for (int i = t; i < n; i += T) w[sidx(i)] = 0.f;
    } else if (al16(src)) {
      const float4* s4 = reinterpret_cast<const float4*>(src);
      for (int j0 = 0; j0 < NQ; j0 += QB) {
        float4 v[QB];
#pragma unroll
        for (int u = 0; u < QB; ++u) v[u] = s4[t + (j0 + u) * T];
#pragma unroll
        for (int u = 0; u < QB; ++u) *reinterpret_cast<float4*>(w + sidx(4 * (t + (j0 + u) * T))) = v[u];
      }
    } else {
      for (int i = t; i < n; i += T) w[sidx(i)] = src[i];
    }
  }
  // the load above is strided over the whole vector: every segment is
  // complete before a thread reads its own
  __syncthreads();

  float cy, cx1, cx2, au, av1, av2;
  auto csec1 = [&](float b) {
    if (!C1) return b;
    cy = fmaf(cr, cy, b);
    return cy;
  };
  auto csec2 = [&](float y) {
    float x = y;
    if (C2 >= 2) x = fmaf(cd1, cx2, x);
    if (C2 >= 1) {
      x = fmaf(cd0, cx1, x);
      cx2 = cx1;
      cx1 = x;
    }
    return x;
  };
  auto asec1 = [&](float b) {
    if (!A1) return b;
    au = fmaf(ar, au, b);
    return au;
  };
  auto asec2 = [&](float u) {
    float v = u;
    if (A2 >= 2) v = fmaf(ad1, av2, v);
    if (A2 >= 1) {
      v = fmaf(ad0, av1, v);
      av2 = av1;
      av1 = v;
    }
    return v;
  };
  constexpr bool anti = (A1 + A2) > 0;
  auto nost = [](int, float, float, float, float) {};

  // solve of slot X in place: X = (1/kappa) U(X)
  auto solve = [&](float* X) {
    __syncthreads();  // every write of X is visible, every read of a neighbour's segment done
    cy = cx1 = cx2 = 0.f;
    quad_pass<false>(X + lft + S - rc1, rc1 - rc2, [&](float b) { return csec1(b); }, nost);
    quad_pass<false>(X + lft + S - rc2, rc2, [&](float b) { return csec2(csec1(b)); }, nost);
    __syncthreads();  // the neighbour's tail is read before it is overwritten
    float* xo = X + own;
    auto st4 = [&](int j, float r0, float r1, float r2, float r3) {
      *reinterpret_cast<float4*>(xo + j) = make_float4(r0, r1, r2, r3);
    };
    quad_pass<false>(xo, S, [&](float b) { return csec2(csec1(b)); }, st4);
    au = av1 = av2 = 0.f;
    if (anti) {
      __syncthreads();
      quad_pass<true>(X + rgt + ra2, ra1 - ra2, [&](float b) { return asec1(b); }, nost);
      quad_pass<true>(X + rgt, ra2, [&](float b) { return asec2(asec1(b)); }, nost);
      __syncthreads();  // the neighbour's head is read before it is overwritten
    }
    quad_pass<true>(xo, S, [&](float b) { return ik * (anti ? asec2(asec1(b)) : b); }, st4);
  };

  // D1 += g1 L X, D2 += g2 L X over the own segment (D2 null: one target);
  // the halo comes from the neighbouring segments of X.  x_{j+HR} enters
  // the window at point j; X is read in quads (two at a time cover the
  // points j .. j+3 + HR), the quads past the segment's end being the right
  // neighbour's first.  The next step's quads of X and D are loaded before
  // this step's results are stored (the compiler cannot move those loads
  // above the stores itself: it does not know that the slots are disjoint)
  auto matvec = [&](const float* X, float* D1, float g1, float* D2, float g2) {
    __syncthreads();  // X complete in every segment
    auto ld4 = [](const float* q) { return *reinterpret_cast<const float4*>(q); };
    float win[P1];
#pragma unroll
    for (int a = 0; a < HL; ++a) win[a] = X[lft + S - HL + a];
    const float* xo = X + own;
    const float* xr = X + rgt;
#pragma unroll
    for (int a = 0; a < HR; ++a) win[HL + a] = xo[a];
    float* d1 = D1 + own;
    float* d2 = D2 ? D2 + own : nullptr;
    auto tap = [&](float xin) {
      win[P1 - 1] = xin;
      float acc = 0.f;
#pragma unroll
      for (int a = 0; a < P1; ++a) acc = fmaf(lt[a], win[a], acc);
#pragma unroll
      for (int a = 0; a < P1 - 1; ++a) win[a] = win[a + 1];
      return acc;
    };
    static_assert(S % 4 == 0 && S >= 8, "segment length");
    float4 qa = ld4(xo), qb = ld4(xo + 4);
    float4 o1 = ld4(d1), o2 = d2 ? ld4(d2) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 4
    for (int j0 = 0; j0 < S; j0 += 4) {
      const int jn = j0 + 8;  // quad after qb: own segment, else the right neighbour's 1st / 2nd
      const float4 qc = ld4(jn < S ? xo + jn : xr + (jn - S));
      float4 n1 = o1, n2 = o2;
      if (j0 + 4 < S) {
        n1 = ld4(d1 + j0 + 4);
        if (d2) n2 = ld4(d2 + j0 + 4);
      }
      const float e[8] = {qa.x, qa.y, qa.z, qa.w, qb.x, qb.y, qb.z, qb.w};
      const float t0 = tap(e[HR]), t1 = tap(e[HR + 1]), t2 = tap(e[HR + 2]), t3 = tap(e[HR + 3]);
      *reinterpret_cast<float4*>(d1 + j0) =
          make_float4(fmaf(g1, t0, o1.x), fmaf(g1, t1, o1.y), fmaf(g1, t2, o1.z), fmaf(g1, t3, o1.w));
      if (d2)
        *reinterpret_cast<float4*>(d2 + j0) =
            make_float4(fmaf(g2, t0, o2.x), fmaf(g2, t1, o2.y), fmaf(g2, t2, o2.z), fmaf(g2, t3, o2.w));
      qa = qb;
      qb = qc;
      o1 = n1;
      o2 = n2;
    }
  };

  int ia = 0;  // slot holding the state
  for (int s = 0; s < A.nsteps; ++s) {
    float* X0 = slot_of(ia);
    if (STAGES == 1) {
      solve(X0);
    } else {
      float* X1 = slot_of(ia == 2 ? 0 : ia + 1);
      float* X2 = slot_of(ia == 0 ? 2 : ia - 1);
      // R_1 = R_2 = u (own segment only; the previous step's last reads of
      // these slots by neighbours ended before the barriers of its last solve)
      for (int j = 0; j < S; j += 4) {
        const float4 v = *reinterpret_cast<const float4*>(X0 + own + j);
        *reinterpret_cast<float4*>(X1 + own + j) = v;
        *reinterpret_cast<float4*>(X2 + own + j) = v;
      }
      solve(X0);                                // Y_0
      matvec(X0, X1, A.g[0], X2, A.g[1]);       // R_1, R_2 -= c a_j0 L Y_0
      solve(X1);                                // Y_1
      matvec(X1, X2, A.g[2], nullptr, 0.f);     // R_2 -= c a_21 L Y_1
      solve(X2);                                // Y_2: the next state
      ia = (ia == 0 ? 2 : ia - 1);
    }
  }
  __syncthreads();
  const float* w = slot_of(ia);
  const int mode = A.mode;
  float* orow = A.out + (mode == kModeAPPLY ? k : k + 1) * (int64_t)n;
  const float* rh = A.rhs ? A.rhs + (k + 1) * (int64_t)n : nullptr;
  const float* sb = A.sub ? A.sub + (k + 1) * (int64_t)n : nullptr;
  double sq = 0.0;
  if (al16(orow) && (!rh || al16(rh)) && (!sb || al16(sb))) {
    const float4* rh4 = reinterpret_cast<const float4*>(rh);
    const float4* sb4 = reinterpret_cast<const float4*>(sb);
    float4* o4 = reinterpret_cast<float4*>(orow);
    for (int j0 = 0; j0 < NQ; j0 += QB) {
      float4 a[QB], b[QB];
#pragma unroll
      for (int u = 0; u < QB; ++u) {
        if (rh) a[u] = rh4[t + (j0 + u) * T];
        if (sb) b[u] = sb4[t + (j0 + u) * T];
      }
#pragma unroll
      for (int u = 0; u < QB; ++u) {
        const int qd = t + (j0 + u) * T;
        float4 v = *reinterpret_cast<const float4*>(w + sidx(4 * qd));
        if (rh) {
          v.x += a[u].x;
          v.y += a[u].y;
          v.z += a[u].z;
          v.w += a[u].w;
        }
        if (sb) {
          v.x -= b[u].x;
          v.y -= b[u].y;
          v.z -= b[u].z;
          v.w -= b[u].w;
        }
        o4[qd] = v;
        sq += (double)v.x * (double)v.x + (double)v.y * (double)v.y + (double)v.z * (double)v.z +
              (double)v.w * (double)v.w;
      }
    }
  } else {
    for (int i = t; i < n; i += T) {
      float v = w[sidx(i)];
      if (rh) v += rh[i];
      if (sb) v -= sb[i];
      orow[i] = v;
      sq += (double)v * (double)v;
    }
  }
  if (mode == kModeFRES && A.partial) {
    const double tot = block_sum(sq, red);
    if (t == 0) A.partial[k] = tot;
  }
}

}  // namespace mg
