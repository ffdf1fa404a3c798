// Level-0 C-point residual and its norm without any memory allocation.
//
// Some callers cannot allocate device memory at the moment they need a
// residual: code running while a stream is being captured into a CUDA graph
// (cudaMalloc is not a capturable operation), and applications whose device
// memory is owned by a pool or caching allocator that must not be bypassed.
// mgrit_residual_noalloc serves them: it needs no handle (mgrit_setup
// allocates), works on caller-owned buffers, and keeps its only scratch --
// the per-CTA partial sums of the norm and their total -- in one file-scope
// static __device__ array.  Host-side it computes the composite stencil
// Phi^m in fixed-size arrays on the stack, so it allocates no host heap
// memory either.
//
// The kernels it launches are the library's existing level-0 composite
// stencil kernel and its fixed-order reduction (unchanged); only the scratch
// pointer differs.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>

#include "../../include/mgrit.h"
#include "kernels.h"

namespace {

using mg::kMaxTaps;
using mg::StencilParams;

// Scratch: kNoAllocSlots partial sums, then the total at index kNoAllocSlots.
// 512 KB + 256 B per GPU that loads the library, held until process exit.
constexpr int64_t kNoAllocSlots = 65536;
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocSlots + 32];

// Device addresses of g_noalloc_scratch, looked up once per device.
constexpr int kMaxDevices = 64;
double* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

int scratch_for_current_device(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return MGRIT_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return MGRIT_ERR_CUDA;
    }
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[dev];
  return MGRIT_OK;
}

// Fixed-size periodic stencil (taps a[t - lo], t = lo..lo+n-1), kept on the
// caller's stack.
struct FixedStencil {
  int lo = 0;
  int n = 0;
  double a[kMaxTaps];
};

// z = x * y (composition of periodic stencils, each tap accumulated in long
// double), folded modulo nx whenever the product is wider than nx (taps t
// and t + nx act on the same grid point), as the handle path folds its
// composite stencil; false if the folded result exceeds kMaxTaps taps.  z
// must not alias x or y.
bool fixed_mul(const FixedStencil& x, const FixedStencil& y, int64_t nx, FixedStencil* z) {
  const int n = x.n + y.n - 1;  // <= 2 kMaxTaps - 1
  const int nz = (int64_t)n > nx ? (int)nx : n;
  if (nz > kMaxTaps) return false;
  long double acc[2 * kMaxTaps];
  for (int k = 0; k < nz; ++k) acc[k] = 0.0L;
  for (int i = 0; i < x.n; ++i)
    for (int j = 0; j < y.n; ++j) {
      const int k = i + j;
      acc[nz == n ? k : (int)((int64_t)k % nx)] += (long double)x.a[i] * (long double)y.a[j];
    }
  z->lo = x.lo + y.lo;
  z->n = nz;
  for (int k = 0; k < nz; ++k) z->a[k] = (double)acc[k];
  return true;
}

// z = b p + a for periodic stencils on the window of p (p's support holds
// a's modulo nx); false if a tap of a falls outside it.
bool fixed_axpy(long double b, const FixedStencil& p, const FixedStencil& a, int64_t nx, FixedStencil* z) {
  long double acc[kMaxTaps];
  for (int i = 0; i < p.n; ++i) acc[i] = b * (long double)p.a[i];
  for (int i = 0; i < a.n; ++i) {
    const int64_t d = ((int64_t)(a.lo + i - p.lo) % nx + nx) % nx;
    if (d >= p.n) return false;
    acc[d] += (long double)a.a[i];
  }
  z->lo = p.lo;
  z->n = p.n;
  for (int i = 0; i < p.n; ++i) z->a[i] = (double)acc[i];
  return true;
}

// Upwind taps of L_p (odd p): the derivative at 0 of the degree-p
// interpolant on j = -(p+1)/2 .. (p-1)/2, from sum_j l_j j^k = delta_{k1}.
bool upwind_fixed(int p, FixedStencil* L) {
  if (p != 1 && p != 3 && p != 5) return false;
  const int n = p + 1, lo = -(p + 1) / 2;
  long double M[6][7];
  for (int k = 0; k < n; ++k) {
    for (int c = 0; c < n; ++c) {
      long double v = 1.0L;
      for (int e = 0; e < k; ++e) v *= (long double)(c + lo);
      M[k][c] = v;
    }
    M[k][n] = (k == 1) ? 1.0L : 0.0L;
  }
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (fabsl(M[r][c]) > fabsl(M[piv][c])) piv = r;
    for (int k = 0; k <= n; ++k) {
      long double t = M[c][k];
      M[c][k] = M[piv][k];
      M[piv][k] = t;
    }
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      long double f = M[r][c] / M[c][c];
      for (int k = c; k <= n; ++k) M[r][k] -= f * M[c][k];
    }
  }
  L->lo = lo;
  L->n = n;
  for (int c = 0; c < n; ++c) L->a[c] = (double)(M[c][n] / M[c][c]);
  return true;
}

// Phi^m = R_q(-c L_p)^m folded modulo nx into `sp` (ERK, q = p).
int composite_stencil(const mgrit_params& P, StencilParams<double>* sp) {
  FixedStencil L, Z, pw, acc, tmp, base, res;
  if (!upwind_fixed(P.order_p, &L)) return MGRIT_ERR_INVALID_ARG;
  const int q = P.rk_order_q ? P.rk_order_q : P.order_p;
  if (q != P.order_p) return MGRIT_ERR_INVALID_ARG;
  // beta_j of R_q: Taylor coefficients, plus beta_6 = 1/1280 for ERK5
  long double beta[7];
  int nb = q + 1;
  long double f = 1.0L;
  for (int j = 0; j <= q; ++j) {
    if (j > 0) f *= (long double)j;
    beta[j] = 1.0L / f;
  }
  if (q == 5) beta[nb++] = 1.0L / 1280.0L;
  Z = L;
  for (int i = 0; i < Z.n; ++i) Z.a[i] *= -P.cfl;
  // acc = sum_j beta_j Z^j
  acc.lo = 0;
  acc.n = 1;
  acc.a[0] = (double)beta[0];
  pw.lo = 0;
  pw.n = 1;
  pw.a[0] = 1.0;
  const int64_t nx = P.nx;
  for (int j = 1; j < nb; ++j) {
    if (!fixed_mul(pw, Z, nx, &tmp)) return MGRIT_ERR_UNSUPPORTED;
    pw = tmp;
    // acc <- beta_j pw + acc; pw's support contains acc's (modulo nx)
    if (!fixed_axpy(beta[j], pw, acc, nx, &tmp)) return MGRIT_ERR_UNSUPPORTED;
    acc = tmp;
  }
  // res = acc^m by repeated squaring
  res.lo = 0;
  res.n = 1;
  res.a[0] = 1.0;
  base = acc;
  for (int e = P.m; e > 0; e >>= 1) {
    if (e & 1) {
      if (!fixed_mul(res, base, nx, &tmp)) return MGRIT_ERR_UNSUPPORTED;
      res = tmp;
    }
    if (e > 1) {
      if (!fixed_mul(base, base, nx, &tmp)) return MGRIT_ERR_UNSUPPORTED;
      base = tmp;
    }
  }
  const int nt = res.n;  // at most nx: every product above was folded
  sp->nx = nx;
  sp->lo = res.lo;
  sp->ntaps = nt;
  for (int i = 0; i < nt; ++i) sp->taps[i] = res.a[i];
  return MGRIT_OK;
}

}  // namespace

extern "C" int mgrit_residual_noalloc(const mgrit_params* params, const double* d_uC, int64_t rows,
                                      double* d_r, double* norm_out, void* stream) {
  if (!params || !d_uC || !d_r || rows < 2) return MGRIT_ERR_INVALID_ARG;
  const mgrit_params& P = *params;
  if (P.rk_kind != MGRIT_ERK || P.precision != MGRIT_FP64 || P.m < 2 || P.cfl <= 0.0 || P.nx < 32 ||
      P.nx % 8)
    return MGRIT_ERR_INVALID_ARG;
  // odd upwind orders only, ERK of the same order
  if ((P.order_p != 1 && P.order_p != 3 && P.order_p != 5) || (P.rk_order_q != 0 && P.rk_order_q != P.order_p))
    return MGRIT_ERR_INVALID_ARG;
  const int64_t K = rows - 1;
  if (K * (int64_t)mg::stencil_tiles(P.nx, 0) > kNoAllocSlots) return MGRIT_ERR_INVALID_ARG;
  double* scratch = nullptr;
  int rc = scratch_for_current_device(&scratch);
  if (rc) return rc;
  StencilParams<double> sp;
  std::memset((void*)&sp, 0, sizeof(sp));
  rc = composite_stencil(P, &sp);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  sp.in = d_uC;
  sp.sub = d_uC + P.nx;
  sp.out = d_r;
  sp.rhs = nullptr;
  sp.partial = scratch;
  sp.rows = K;
  int64_t nb = mg::launch_stencil_rows(sp, st);
  mg::launch_reduce_sum(scratch, nb, scratch + kNoAllocSlots, st);
  if (cudaGetLastError() != cudaSuccess) return MGRIT_ERR_CUDA;
  if (norm_out) {
    double sum = 0.0;
    if (cudaMemcpyAsync(&sum, scratch + kNoAllocSlots, sizeof(double), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      cudaGetLastError();
      return MGRIT_ERR_CUDA;
    }
    *norm_out = std::sqrt(sum > 0.0 ? sum : 0.0);
  }
  return MGRIT_OK;
}
