// Host driver and C ABI of the MGRIT library (see include/mgrit.h).
//
// Level data layout in HBM (FP64, row-major rows of nx):
//   level 0:  uC0[2] -- C-point iterate, nt/m + 1 rows, double buffered so a
//             C-relaxation reads one buffer and writes the other;
//   level l:  g_l    -- RHS, N_l + 1 rows (the injected C-point residual of
//                       level l-1, Sec. 2.2), row 0 is always 0;
//             uC_l[2] -- C-point unknowns, N_{l+1} + 1 rows (l < L-1).
// F-points are never stored: every kernel regenerates them from C-points.
// The post F-relaxation of level 0 is skipped inside the iteration because
// the next pre-relaxation recomputes every F-point from the C-points.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/mgrit.h"
#include "coeffs.h"
#include "graph_batch.h"
#include "kernels.h"

using namespace mg;

// sqrt of a sum of squares, NaN kept (a NaN residual must read as diverged,
// not as zero)
static inline double norm_of_sq(double s) { return s == s ? std::sqrt(s > 0.0 ? s : 0.0) : s; }

static inline bool is_mixed(int precision) { return precision == MGRIT_MIXED || precision == MGRIT_MIXED_FAST; }

namespace {

struct LevelData {
  int64_t N = 0;  // steps on the level
  int64_t K = 0;  // CF-intervals (N / m_l); 0 on the coarsest level
  int m = 0;              // m_l: steps of this level per step of the next (its interval length)
  long long tstep = 1;    // this level's time step in units of dt (m_0 m_1 .. m_{l-1})
  double* uC[2] = {nullptr, nullptr};
  int cur = 0;
  double* g = nullptr;
  // coarse operator (l >= 1)
  CoarseParams<double> cp;
  double* Mt_dev[2] = {nullptr, nullptr};  // per-chunk carry tables (causal, anticausal)
  // MIXED: FP32 inner-cycle data (level 0: uCf = error e, gf = its C-point
  // RHS r; level l: uCf, gf as in FP64), FP32-SL operators with an FP32 or
  // FP64 correction solve
  float* uCf[2] = {nullptr, nullptr};
  int curf = 0;
  float* gf = nullptr;
  CoarseParams<float, float> cpf;
  CoarseParams<float, double> cpfd;
  float* Mtf_dev[2] = {nullptr, nullptr};
  bool solve64 = false;
  // geometry-free coarse operator data: factorised correction, SL weights
  // (scaled by 1/kappa of the factorisation)
  BandFactor bf;
  double slw[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  double kappa = 1.0;
  // rediscretised coarse operator (SDIRK with step m^l dt): SDIRK step
  // parameters in FP64 and, in MIXED, FP32
  bool redisc = false;
  bool nosolve = false;  // direct SL coarse operator: no correction solve
  std::unique_ptr<SdirkParams<double>> rd;
  std::unique_ptr<SdirkParams<float>> rdf;
  double* rd_Mt[2] = {nullptr, nullptr};
  float* rdf_Mt[2] = {nullptr, nullptr};
  long long kshift = 0;
  double eps = 0.0, phi = 0.0, phi_q = 0.0;
  int jlo = 0;  // SL node offset of weight 0 (sl_lo: depends on eps for even p)
  // GMRES correction solves: unscaled SL weights, the taps of I - sum phi D
  // (offsets -3..3), the Krylov basis scratch for gm_cap intervals (sized
  // for doubles) and the device counters [iterations, solves]
  double slw_raw[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  double gm_taps[7] = {0, 0, 0, 0, 0, 0, 0};
  double* gm_V = nullptr;
  int64_t gm_cap = 0;
  unsigned long long* gm_stats = nullptr;
};

}  // namespace

// profiling categories: 0 level-0 stencil, 1 coarse kernel (all levels),
// 2 reductions, 3 sequential stepping, 4 + l coarse kernel on level l
constexpr int kProfCats = 20;
constexpr int kStencilThreadsHost = 256;  // threads of stencil_rows_kernel
constexpr int kProfL0F32 = 19;  // MIXED: level-0 FP32 inner-cycle kernels

struct mgrit_handle {
  mgrit_params prm;
  cudaStream_t st = nullptr;
  int L = 0;
  int64_t nx = 0;
  int m = 0;
  int device = 0;
  std::unique_ptr<StencilParams<double>> fineM;  // Phi^m composite (ERK)
  std::unique_ptr<StencilParams<double>> fine1;  // Phi (one step, ERK)
  std::unique_ptr<SdirkParams<double>> sd0;      // SDIRK step program (level 0)
  std::unique_ptr<StencilParams<float>> fineMf;  // MIXED: Phi^m in FP32 (ERK)
  std::unique_ptr<SdirkParams<float>> sd0f;      // MIXED: SDIRK programme in FP32
  float* sdf_Mt[2] = {nullptr, nullptr};
  std::unique_ptr<SdirkSeg32Params> seg0f;       // MIXED: the FP32 segmented stage kernel
  std::unique_ptr<SdirkSegParams> seg0;          // FP64 level-0 SDIRK with per-thread segments
                                                 // (used for CF / FRES / APPLY when set)
  std::unique_ptr<SdirkParams<double>> sdseq;    // SDIRK sequential stepping (one vector)
  double* sdseq_Mt[2] = {nullptr, nullptr};
  double* seq_tmp = nullptr;                     // MIXED: FP64 coarsest-level output
  bool mixed = false;
  // graph-resident solve: prologue (first relaxation and residual) and a
  // conditional while node whose body is one MGRIT iteration with the stop
  // test on the device
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  DevSolveState* dstate = nullptr;
  DevSolveState* hstate = nullptr;  // pinned
  cudaEvent_t done = nullptr;
  bool graph_pending = false;
  int graph_cur = 0;  // level-0 C-point buffer holding the result of a graph solve
  double* sd_Mt[2] = {nullptr, nullptr};
  bool sdirk = false;
  int fineM_taps_raw = 0;
  std::vector<LevelData> lev;
  double* partials = nullptr;
  int64_t npart = 0;
  double* dnorm = nullptr;
  double* dnorm_f = nullptr;  // MIXED: squared norm of the FP32 inner residual
  double inner_tol = kInnerTol;  // MIXED: target of one adaptive inner solve (MGRIT_INNER_TOL)
  double* hnorm = nullptr;  // pinned
  double* du0 = nullptr;
  int64_t launches = 0;
  bool have_initial = false;
  // optional per-category CUDA-event timing (0: level-0 stencil, 1: coarse
  // step kernel, 2: reductions / utilities, 3: sequential stepping)
  struct Prof {
    bool on = false;
    std::vector<cudaEvent_t> pool;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev[kProfCats];
    double flops[kProfCats] = {};
    int64_t count[kProfCats] = {};
  } prof;
};

static cudaEvent_t prof_event(mgrit_handle* h) {
  if (!h->prof.pool.empty()) {
    cudaEvent_t e = h->prof.pool.back();
    h->prof.pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  cudaEventCreate(&e);
  return e;
}

// Bracket one launch of category `cat` with events when profiling is on.
struct ProfScope {
  mgrit_handle* h;
  int cat;
  cudaEvent_t a = nullptr;
  ProfScope(mgrit_handle* hh, int c, double flops) : h(hh), cat(c) {
    if (!h->prof.on) return;
    a = prof_event(h);
    cudaEventRecord(a, h->st);
    h->prof.flops[cat] += flops;
    h->prof.count[cat] += 1;
  }
  ~ProfScope() {
    if (!a) return;
    cudaEvent_t b = prof_event(h);
    cudaEventRecord(b, h->st);
    h->prof.ev[cat].push_back({a, b});
  }
};

// Text of the last failing CUDA call on this host thread (mgrit_last_error).
static thread_local char g_last_error[256] = "";

static void note_cuda_error(const char* what, cudaError_t e) {
  std::snprintf(g_last_error, sizeof(g_last_error), "%s: %s", what, cudaGetErrorString(e));
}

#define CUDA_TRY(expr)                \
  do {                                \
    cudaError_t e_ = (expr);          \
    if (e_ != cudaSuccess) {          \
      note_cuda_error(#expr, e_);     \
      return MGRIT_ERR_CUDA;          \
    }                                 \
  } while (0)

static int check_launch() {
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) return MGRIT_OK;
  note_cuda_error("kernel launch", e);
  return MGRIT_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// setup helpers
// ---------------------------------------------------------------------------

// Host check that an n-point vector has a chunk geometry of the step
// kernels at all: C <= 16 CTAs of <= 256 threads with a chunk length P in
// {4, 8, 16, 32} (so n <= 131072).
static bool has_chunk_geometry(int64_t n) {
  for (int C = 1; C <= 16; C *= 2)
    for (int P : kChunkLens)
      if (n % ((int64_t)C * P) == 0 && n / ((int64_t)C * P) <= 256) return true;
  return false;
}


template <typename T>
static void fill_solve_dir(SolveDir<T>* d, const double* coef, int horder, int Hpad, int P, int nthr, int C,
                           std::vector<T>* mt_out) {
  std::memset((void*)d, 0, sizeof(*d));
  if (Hpad == 0) {  // no recurrence in this direction (the kernel skips it)
    mt_out->clear();
    return;
  }
  double c3[3] = {0, 0, 0};
  for (int q = 0; q < horder; ++q) c3[q] = coef[q];
  // carries below the kernel precision are dropped
  DistScanTables tb = dist_scan_tables(c3, Hpad, P, nthr, C, sizeof(T) == 4 ? 1e-10 : 1e-18);
  d->h = Hpad;
  d->rounds = std::min(tb.rounds, kMaxRounds);
  d->tcut = tb.tcut;
  d->jterms = std::min(tb.jterms, 16);
  d->closure = tb.closure;
  for (int q = 0; q < 3; ++q) d->ncoef[q] = (T)(-c3[q]);
  for (int r = 0; r < d->rounds; ++r)
    for (int i = 0; i < 9; ++i) d->Mpow[r][i] = (T)tb.Mpow[r * 9 + i];
  for (int j = 0; j < d->jterms; ++j)
    for (int i = 0; i < 9; ++i) d->McPow[j][i] = (T)tb.McPow[j * 9 + i];
  d->wterms = std::min(tb.wterms, 8);
  d->dcut = tb.dcut;
  for (int dd = 0; dd < 32; ++dd)
    for (int i = 0; i < 9; ++i) d->Mlane[dd][i] = (T)tb.Mlane[dd * 9 + i];
  for (int j = 0; j < d->wterms; ++j)
    for (int i = 0; i < 9; ++i) d->M32pow[j][i] = (T)tb.M32pow[j * 9 + i];
  for (int i = 0; i < 9; ++i) d->Clc[i] = (T)tb.Clc[i];
  for (int j = 0; j < P && j < kPMax; ++j)
    for (int q = 0; q < 3; ++q) d->G[j * 3 + q] = (T)tb.G[(size_t)j * 3 + q];
  mt_out->assign(tb.Mt.begin(), tb.Mt.end());
}

static Stencil fold_mod(const Stencil& s, int64_t nx) {
  if (s.width() <= nx) return s;
  Stencil f;
  f.lo = s.lo;
  f.hi = s.lo + (int)nx - 1;
  f.a.assign((size_t)nx, 0.0);
  for (int t = s.lo; t <= s.hi; ++t) {
    int64_t off = ((int64_t)(t - s.lo)) % nx;
    f.a[(size_t)off] += s.a[t - s.lo];
  }
  return f;
}

template <typename T>
static int set_stencil(StencilParams<T>* sp, const Stencil& s0, int64_t nx) {
  Stencil s = fold_mod(s0, nx);
  if (s.width() > kMaxTaps) return MGRIT_ERR_UNSUPPORTED;
  std::memset((void*)sp, 0, sizeof(*sp));
  sp->nx = nx;
  sp->lo = s.lo;
  sp->ntaps = s.width();
  for (int i = 0; i < s.width(); ++i) sp->taps[i] = (T)s.a[i];
  return MGRIT_OK;
}


// ---------------------------------------------------------------------------
// Memory of a handle.  Device buffers come from one stream-ordered pool per
// device (cudaMallocFromPoolAsync / cudaFreeAsync on the handle's stream):
// freeing never synchronises the device, so solves that finish while others
// run (batches, the server) do not stall them, and freed hierarchies stay
// reserved in the pool for the next setup instead of going back to the
// driver.  Small pinned host blocks (the device-state mirror, the norm) are
// recycled through a free list for the same reason (cudaFreeHost
// synchronises).
// ---------------------------------------------------------------------------
static std::mutex g_pool_mu;
static std::map<int, cudaMemPool_t> g_pools;

static cudaMemPool_t device_pool(int dev) {
  std::lock_guard<std::mutex> lk(g_pool_mu);
  auto it = g_pools.find(dev);
  if (it != g_pools.end()) return it->second;
  cudaMemPoolProps props;
  std::memset(&props, 0, sizeof(props));
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = dev;
  cudaMemPool_t pool = nullptr;
  if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  uint64_t keep = UINT64_MAX;  // keep freed memory reserved in the pool
  cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  g_pools[dev] = pool;
  return pool;
}

static int dev_alloc(mgrit_handle* h, void** p, size_t bytes) {
  *p = nullptr;
  cudaMemPool_t pool = device_pool(h->device);
  if (!pool || cudaMallocFromPoolAsync(p, std::max<size_t>(bytes, 16), pool, h->st) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return MGRIT_ERR_OOM;
  }
  return MGRIT_OK;
}

static void dev_free(mgrit_handle* h, void* p) {
  if (p) cudaFreeAsync(p, h->st);  // ordered after the handle's last work on its stream
}

static std::mutex g_pin_mu;
static std::vector<void*> g_pin_free;  // 4 KiB pinned host blocks
constexpr size_t kPinBlock = 4096;

static void* pinned_get() {
  {
    std::lock_guard<std::mutex> lk(g_pin_mu);
    if (!g_pin_free.empty()) {
      void* p = g_pin_free.back();
      g_pin_free.pop_back();
      return p;
    }
  }
  void* p = nullptr;
  if (cudaMallocHost(&p, kPinBlock) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

static void pinned_put(void* p) {
  if (!p) return;
  std::lock_guard<std::mutex> lk(g_pin_mu);
  g_pin_free.push_back(p);
}

template <typename T>
static int upload_table(mgrit_handle* h, const std::vector<T>& v, T** dev) {
  int rc = dev_alloc(h, (void**)dev, sizeof(T) * std::max<size_t>(9, v.size()));
  if (rc) return rc;
  // pageable source: staged before the call returns
  if (!v.empty() && cudaMemcpyAsync(*dev, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, h->st) !=
                        cudaSuccess)
    return MGRIT_ERR_CUDA;
  return MGRIT_OK;
}

// Condition number of a periodic banded (circulant, hence normal) matrix:
// the extreme moduli of its symbol sampled on the unit circle.
static double band_condition(const Stencil& A) {
  double amin = 1e300, amax = 0.0;
  const int ns = 4096;
  for (int i = 0; i < ns; ++i) {
    double th = 2.0 * M_PI * i / ns, re = 0.0, im = 0.0;
    for (int t = A.lo; t <= A.hi; ++t) {
      re += A.at(t) * std::cos(t * th);
      im += A.at(t) * std::sin(t * th);
    }
    const double v = std::hypot(re, im);
    amin = std::min(amin, v);
    amax = std::max(amax, v);
  }
  return amin > 0.0 ? amax / amin : 1e300;
}

// phi recursion (Lemma 6.1 / the multilevel recursion of Sec. 6.2) and the generalised two-term form
// for q != p.  Returns per-level (phi_p, phi_q), level index 1..L-1.
static void phi_recursion(const mgrit_params& P, int L, std::vector<double>* php,
                          std::vector<double>* phq, std::vector<long long>* ks,
                          std::vector<double>* es) {
  int p = P.order_p, q = P.rk_order_q;
  double c = P.cfl;
  double efd = e_fd(p), erk = e_rk(P.rk_kind == MGRIT_SDIRK ? 1 : 0, q);
  double sgn = ((p + 1) % 2) ? -1.0 : 1.0;
  php->assign(L, 0.0);
  phq->assign(L, 0.0);
  ks->assign(L, 0);
  es->assign(L, 0.0);
  // level l steps m_1 .. m_l dt (m_1 = m, m_l = m_coarse below); the
  // recursion of Sec. 6.2 with the factor m_l of the level in place of m
  double mpow = 1.0;
  for (int l = 1; l < L; ++l) {
    const double ml = (l == 1 || P.m_coarse <= 0) ? P.m : P.m_coarse;
    mpow *= ml;
    long long k;
    double eps;
    sl_shift(c * mpow, &k, &eps);
    (*ks)[l] = k;
    (*es)[l] = eps;
    double f = f_poly(p, eps);
    double cq = std::pow(-c, q + 1) * erk;
    if (l == 1) {
      (*php)[l] = ml * c * efd + sgn * f;
      (*phq)[l] = ml * cq;
    } else {
      double fprev = f_poly(p, (*es)[l - 1]);
      (*php)[l] = sgn * (-ml * fprev + f) + ml * (*php)[l - 1];
      (*phq)[l] = ml * (*phq)[l - 1];
    }
  }
  if (q == p) {  // single correction constant phi = phi_p + phi_q (Eq. varphi-constant-MOL-SL)
    for (int l = 1; l < L; ++l) {
      (*php)[l] += (*phq)[l];
      (*phq)[l] = 0.0;
    }
  }
}

// MGRIT_GEOM="C:P" restricts the step kernels' geometries to C CTAs per
// vector and chunk length P where that geometry fits (testing every
// geometry against the oracle); tuning and its cache are then bypassed.
static bool geom_forced(int* C, int* P) {
  const char* f = std::getenv("MGRIT_GEOM");
  return f && std::sscanf(f, "%d:%d", C, P) == 2;
}

// Coarse-level parameters of level l for geometry g: FP64, and in MIXED the
// FP32-storage forms with an FP32 or FP64 correction solve; chunk-scan
// tables built on the host, per-chunk carry tables uploaded.
struct GeomC {
  int C = 0, P = 0, nthr = 0;
};
static int coarse_with_geom(mgrit_handle* h, int l, const GeomC& g) {
  const mgrit_params& P = h->prm;
  LevelData& Lv = h->lev[l];
  const int p = P.order_p;
  // recurrence orders of the kernel (the template's): see build_coarse
  const int HC = (p % 2) ? (p + 1) / 2 : (p + 2) / 2, HA = (p % 2) ? (p + 1) / 2 : p / 2;
  const BandFactor& bf = Lv.bf;
  CoarseParams<double>& cp = Lv.cp;
  std::memset((void*)&cp, 0, sizeof(cp));
  cp.n = (int)h->nx;
  cp.P = g.P;
  cp.nthr = g.nthr;
  cp.csize = g.C;
  cp.npc = (int)(h->nx / g.C);
  cp.p1 = p + 1;
  cp.jlo = Lv.jlo;
  cp.kshift = (int)(((Lv.kshift % h->nx) + h->nx) % h->nx);
  cp.shift = 0;
  cp.nosolve = Lv.nosolve ? 1 : 0;
  for (int a = 0; a <= p; ++a) cp.w[a] = Lv.slw[a];
  if (P.coarse_solve == MGRIT_SOLVE_GMRES) {  // GMRES solves the unscaled system
    cp.gm_max = P.gmres_maxit;
    cp.gm_rtol = P.gmres_rtol;
    for (int a = 0; a <= p; ++a) cp.w[a] = Lv.slw_raw[a];
    for (int i = 0; i < 7; ++i) cp.gm_taps[i] = Lv.gm_taps[i];
  }
  for (int d = 0; d < 2; ++d) {
    dev_free(h, Lv.Mt_dev[d]);
    Lv.Mt_dev[d] = nullptr;
    dev_free(h, Lv.Mtf_dev[d]);
    Lv.Mtf_dev[d] = nullptr;
  }
  std::vector<double> mtc, mta;
  fill_solve_dir(&cp.c, bf.cc, bf.hc, HC, g.P, g.nthr, g.C, &mtc);
  fill_solve_dir(&cp.a, bf.ca, bf.ha, HA, g.P, g.nthr, g.C, &mta);
  for (int d = 0; d < 2; ++d) {
    int rc = upload_table(h, d ? mta : mtc, &Lv.Mt_dev[d]);
    if (rc) return rc;
  }
  cp.c.Mt = Lv.Mt_dev[0];
  cp.a.Mt = Lv.Mt_dev[1];
  cp.m = Lv.m;
  if (is_mixed(P.precision)) {
    auto geom = [&](auto& q) {
      std::memset((void*)&q, 0, sizeof(q));
      q.n = cp.n;
      q.P = cp.P;
      q.nthr = cp.nthr;
      q.csize = cp.csize;
      q.npc = cp.npc;
      q.p1 = cp.p1;
      q.jlo = cp.jlo;
      q.kshift = cp.kshift;
      q.shift = cp.shift;
      q.m = cp.m;
      q.nosolve = cp.nosolve;
      for (int a = 0; a <= p; ++a) q.w[a] = (float)cp.w[a];
      q.gm_max = cp.gm_max;
      q.gm_rtol = cp.gm_rtol;
      for (int i = 0; i < 7; ++i) q.gm_taps[i] = cp.gm_taps[i];
    };
    geom(Lv.cpfd);
    Lv.cpfd.c = cp.c;
    Lv.cpfd.a = cp.a;
    geom(Lv.cpf);
    std::vector<float> mtcf, mtaf;
    fill_solve_dir(&Lv.cpf.c, bf.cc, bf.hc, HC, g.P, g.nthr, g.C, &mtcf);
    fill_solve_dir(&Lv.cpf.a, bf.ca, bf.ha, HA, g.P, g.nthr, g.C, &mtaf);
    int rc = upload_table(h, mtcf, &Lv.Mtf_dev[0]);
    if (!rc) rc = upload_table(h, mtaf, &Lv.Mtf_dev[1]);
    if (rc) return rc;
    Lv.cpf.c.Mt = Lv.Mtf_dev[0];
    Lv.cpf.a.Mt = Lv.Mtf_dev[1];
  }
  return MGRIT_OK;
}

// Candidate geometries of the coarse kernel on this handle's vectors: the
// SL window (P + p + 1 points) must lie within two neighbouring CTAs.
static std::vector<GeomC> coarse_geometries(mgrit_handle* h, int max_out) {
  const int elem = is_mixed(h->prm.precision) ? 4 : 8;
  const bool gm = h->prm.coarse_solve == MGRIT_SOLVE_GMRES;  // GMRES kernels: P = 4 or 8
  std::vector<std::pair<double, GeomC>> all;
  for (int C = 1; C <= 16; C *= 2) {
    if (h->nx % C) continue;
    const int64_t npc = h->nx / C;
    for (int P : kChunkLens) {
      if (gm && P > 8) continue;
      if (npc % P || npc < P + h->prm.order_p + 2) continue;
      const int64_t nthr = npc / P;
      if (nthr < 1 || nthr > 256) continue;
      const size_t sm = coarse_smem_bytes((int)npc, P, (int)nthr, 8, gm ? 8 : 0);
      if (sm > 227 * 1024) continue;
      if (C > 1 && coarse_max_cluster(C, sm, (int)nthr) < C) continue;
      const int warps = ((int)nthr + 31) / 32;
      int regs = elem == 8 ? (P <= 8 ? 80 : P <= 16 ? 112 : 192) : (P <= 8 ? 64 : P <= 16 ? 96 : 160);
      if (gm) regs = 128;
      int cps = std::min<int>((int)(228 * 1024 / (sm + 1024)), 64 / warps);
      cps = std::min(cps, 65536 / (regs * warps * 32));
      cps = std::min(cps, 32);
      const double lanes = (double)nthr / (32.0 * warps);
      all.push_back({std::min(16.0, (double)(cps * warps)) * lanes - 0.01 * C, GeomC{C, P, (int)nthr}});
    }
  }
  std::stable_sort(all.begin(), all.end(),
                   [](const std::pair<double, GeomC>& a, const std::pair<double, GeomC>& b) { return a.first > b.first; });
  int fc, fp;
  if (geom_forced(&fc, &fp)) {
    std::vector<std::pair<double, GeomC>> keep;
    for (auto& x : all)
      if (x.second.C == fc && x.second.P == fp) keep.push_back(x);
    if (!keep.empty()) all.swap(keep);
  }
  std::vector<GeomC> out;
  for (auto& x : all)
    if ((int)out.size() < max_out) out.push_back(x.second);
  return out;
}

static int build_sdirk_params(mgrit_handle* h, int64_t K, std::unique_ptr<SdirkParams<double>>* out,
                              double** mt_dev, std::unique_ptr<SdirkParams<float>>* outf, float** mtf_dev,
                              std::string* why, bool buffers, double cfl);

// Rediscretised coarse operator of level l: the fine SDIRK method with the
// coarse step m^l dt (c_l = m^l c), as SDIRK step parameters for the level's
// intervals (the coarsest: one vector).
static int build_redisc(mgrit_handle* h, int l, bool buffers, std::string* why) {
  LevelData& Lv = h->lev[l];
  const bool coarsest = (l == h->L - 1);
  const double cl = h->prm.cfl * (double)Lv.tstep;
  for (int d = 0; d < 2; ++d) {
    dev_free(h, Lv.rd_Mt[d]);
    Lv.rd_Mt[d] = nullptr;
    dev_free(h, Lv.rdf_Mt[d]);
    Lv.rdf_Mt[d] = nullptr;
  }
  int rc = build_sdirk_params(h, coarsest ? 1 : Lv.K, &Lv.rd, Lv.rd_Mt,
                              (is_mixed(h->prm.precision) && !coarsest) ? &Lv.rdf : nullptr, Lv.rdf_Mt, why,
                              buffers, cl);
  if (rc) return rc;
  Lv.redisc = true;
  return MGRIT_OK;
}

static int build_coarse(mgrit_handle* h, int l, double phi_p, double phi_q, long long k, double eps,
                        std::string* why) {
  const mgrit_params& P = h->prm;
  LevelData& Lv = h->lev[l];
  int p = P.order_p, q = P.rk_order_q;
  Stencil A = stencil_identity();
  A = stencil_add(A, diff_stencil(p + 1), -phi_p);
  if (q != p && phi_q != 0.0) A = stencil_add(A, diff_stencil(q + 1), -phi_q);
  BandFactor bf;
  if (!band_factor(A, &bf, why)) return MGRIT_ERR_UNSTABLE;
  // the kernel's recurrence orders: (p+1)/2 both ways for the centred D of
  // odd p; (p+2)/2 causal and p/2 anticausal for the left-biased D of even p
  const int HCm = (p % 2) ? (p + 1) / 2 : (p + 2) / 2, HAm = (p % 2) ? (p + 1) / 2 : p / 2;
  if (bf.hc > HCm || bf.ha > HAm) {
    if (why) *why = "correction band wider than the SL stencil order supports";
    return MGRIT_ERR_UNSUPPORTED;
  }
  if (bf.shift != 0) {
    if (why) *why = "correction factorisation needs an index shift";
    return MGRIT_ERR_UNSUPPORTED;
  }
  Lv.bf = bf;
  std::vector<double> w = sl_weights(p, eps);
  for (int a = 0; a <= p; ++a) {
    Lv.slw[a] = w[a] * bf.inv_kappa;
    Lv.slw_raw[a] = w[a];
  }
  for (int t = -3; t <= 3; ++t) Lv.gm_taps[3 + t] = A.at(t);
  Lv.kappa = band_condition(A);
  // MIXED: FP32 storage and SL gather; the correction solve in FP64.
  // MIXED_FAST: the correction solve in FP32 too, except where the
  // condition number exceeds MGRIT_FAST_KAPPA (default 1e6, where an FP32
  // solve keeps about one of its seven digits).  The coarse operator of an
  // FP32 inner cycle only has to cut the error-equation residual by 1e-2
  // per refinement step; the FP64 residuals of the refinement correct its
  // rounding (16384 x 65536 U5+SDIRK3, condition numbers 1.8e3 to 4.5e5:
  // the same refinement steps and error as with FP64 correction solves)
  if (is_mixed(P.precision)) {
    double kmax = 1e6;
    if (const char* e = std::getenv("MGRIT_FAST_KAPPA")) {
      const double v = std::atof(e);
      if (v > 0.0) kmax = v;
    }
    Lv.solve64 = P.precision == MGRIT_MIXED || Lv.kappa > kmax;
  }
  Lv.kshift = k;
  Lv.eps = eps;
  Lv.jlo = sl_lo(p, eps);
  Lv.phi = phi_p;
  Lv.phi_q = phi_q;
  std::vector<GeomC> cand = coarse_geometries(h, 1);
  if (cand.empty()) {
    if (why) *why = "no coarse-kernel chunk geometry fits the vector";
    return MGRIT_ERR_INVALID_ARG;
  }
  return coarse_with_geom(h, l, cand[0]);
}

// Level-0 SDIRK step programme: stiffly accurate stages (q <= 4), with the
// stage derivative taken from the solve itself: (I + gamma c L) Y_i = R_i
// gives c L Y_i = (R_i - Y_i) / gamma, so
//   R_0 = u, R_i = u (i >= 1);  Y_i = (I + gamma c L)^{-1} R_i;
//   R_j += -(a_ji / gamma) (R_i - Y_i) for j > i  (local: no L_p halos);
// u_new = Y_s; or the factored SDIRK5 stability function
//   v <- (I + gamma c L)^{-1} f_k(-c L) v for each real factor f_k of P,
// then the remaining solves.
static bool sdirk_program(int q, double c, SdirkParams<double>* sp, double* gamma, std::string* why, bool deriv) {
  int n = 0;
  auto op = [&](int kind, int dst, int src, double cf) {
    if (n >= kSdirkMaxOps) return;
    sp->opk[n] = kind;
    sp->opd[n] = dst;
    sp->ops[n] = src;
    sp->opc[n] = cf;
    sp->opc2[n] = 0.0;
    ++n;
  };
  auto axpby = [&](int dst, int src, double cf2, double cf) {  // dst = cf2 dst + cf src
    if (n >= kSdirkMaxOps) return;
    op(kOpAxpby, dst, src, cf);
    sp->opc2[n - 1] = cf2;
  };
  if (q <= 4 && !deriv) {
    SdirkTableau tb;
    if (!sdirk_tableau(q, &tb)) return false;
    *gamma = tb.A[0][0];
    for (int i = 1; i < tb.s; ++i) op(kOpCopy, i, 0, 0.0);
    for (int i = 0; i < tb.s; ++i) {
      op(kOpSolve, i, i, 0.0);
      for (int j = i + 1; j < tb.s; ++j) op(kOpAxpyL, j, i, -c * tb.A[j][i]);
    }
    sp->nslots = tb.s;
    sp->result = tb.s - 1;
  } else if (q <= 4) {
    SdirkTableau tb;
    if (!sdirk_tableau(q, &tb)) return false;
    const double g = tb.A[0][0];
    *gamma = g;
    const int s = tb.s;
    if (s == 1) {
      op(kOpSolve, 0, 0, 0.0);
      sp->nslots = 1;
    } else {
      // the later stages' right-hand sides P_j accumulate in slots freed by
      // earlier stages: Y_0 = solve(u); P_j = (1 - al_j) u + al_j Y_0 with
      // al_j = a_j0 / gamma (P_1 in place of Y_0, formed last); then for
      // each stage i >= 1: Y_i = solve(P_i), P_j -= (a_ji/gamma)(P_i - Y_i);
      // the last stage solves into slot 0.  Peak s slots (3 for SDIRK3).
      std::vector<int> Pj(s, -1), freel;
      int nsl = 1;  // slot 0 holds u
      auto alloc = [&]() {
        if (!freel.empty()) {
          const int x = freel.back();
          freel.pop_back();
          return x;
        }
        return nsl++;
      };
      const int y0 = alloc();
      op(kOpSolve, y0, 0, 0.0);
      for (int j = s - 1; j >= 1; --j) {
        const double al = tb.A[j][0] / g;
        if (j == 1) {
          axpby(y0, 0, al, 1.0 - al);
          Pj[1] = y0;
        } else {
          Pj[j] = alloc();
          op(kOpCopy, Pj[j], 0, 0.0);
          if (al != 0.0) axpby(Pj[j], y0, 1.0 - al, al);
        }
      }
      freel.push_back(0);  // u is dead
      for (int i = 1; i < s - 1; ++i) {
        const int yi = alloc();
        op(kOpSolve, yi, Pj[i], 0.0);
        for (int j = i + 1; j < s; ++j) {
          const double a = tb.A[j][i] / g;
          if (a == 0.0) continue;
          op(kOpAxpy, Pj[j], Pj[i], -a);
          op(kOpAxpy, Pj[j], yi, a);
        }
        freel.push_back(Pj[i]);
        freel.push_back(yi);
      }
      op(kOpSolve, 0, Pj[s - 1], 0.0);
      sp->nslots = nsl;
    }
    sp->result = 0;
  } else {
    std::vector<std::vector<double>> f = sdirk5_factors(gamma);
    for (auto& fk : f) {
      op(kOpCopy, 1, 0, 0.0);
      op(kOpZero, 2, 0, 0.0);
      op(kOpAxpyL, 2, 0, 1.0);
      op(kOpAxpy, 1, 2, -c * fk[1]);
      if (fk.size() == 3) op(kOpAxpyL, 1, 2, c * c * fk[2]);
      op(kOpSolve, 0, 1, 0.0);
    }
    for (int r = (int)f.size(); r < 5; ++r) op(kOpSolve, 0, 0, 0.0);
    sp->nslots = 3;
    sp->result = 0;
  }
  if (n >= kSdirkMaxOps) {
    if (why) *why = "SDIRK programme too long";
    return false;
  }
  sp->nops = n;
  return true;
}

static std::mutex g_tune_mu;
static std::map<std::string, int> g_tune;
static bool g_tune_loaded = false;

static void tune_load() {
  if (g_tune_loaded) return;
  g_tune_loaded = true;
  const char* f = std::getenv("MGRIT_AUTOTUNE_CACHE");
  if (!f) return;
  FILE* fp = std::fopen(f, "r");
  if (!fp) return;
  char key[128];
  int r;
  while (std::fscanf(fp, "%127s %d", key, &r) == 2) g_tune[key] = r;
  std::fclose(fp);
}

static void tune_store(const std::string& key, int r) {
  g_tune[key] = r;
  const char* f = std::getenv("MGRIT_AUTOTUNE_CACHE");
  if (!f) return;
  FILE* fp = std::fopen(f, "a");
  if (!fp) return;
  std::fprintf(fp, "%s %d\n", key.c_str(), r);
  std::fclose(fp);
}

// Barrier schedule of an SDIRK step programme.  Every op reads and writes
// only its own thread's chunk, except that an AXPYL reads L_p halos from the
// neighbouring chunks; a SOLVE has barriers of its own between its read and
// its write.  A barrier is needed before an AXPYL group whose source was
// written since the last barrier (read after write), and before any write
// to a slot whose halos were read since the last barrier (write after read).
// Consecutive AXPYLs on one source form a group (one mat-vec).  The
// schedule is iterated over steps until it is stable.
static bool schedule_sdirk(SdirkParams<double>* sp, std::string* why, bool one_pass) {
  const int n = sp->nops;
  for (int o = 0; o < n; ++o) {
    sp->opg[o] = 1;
    sp->opb[o] = 0;
  }
  sp->resb = 0;
  for (int o = 0; o < n;) {
    if (sp->opk[o] != kOpAxpyL) {
      ++o;
      continue;
    }
    int g = 1;
    while (o + g < n && sp->opk[o + g] == kOpAxpyL && sp->ops[o + g] == sp->ops[o]) ++g;
    for (int e = 0; e < g; ++e)
      if (sp->opd[o + e] == sp->ops[o]) {
        if (why) *why = "SDIRK programme: a mat-vec writes its own source";
        return false;
      }
    sp->opg[o] = g;
    for (int e = 1; e < g; ++e) sp->opg[o + e] = 0;
    o += g;
  }
  // A solve with a single recurrence direction (one_pass: no anticausal
  // order) ends with remote reads of its cluster-visible carry aggregate and
  // of the CTA's warp carries; the next solve rewrites both, so a barrier
  // must separate two such solves (the anticausal pass's barrier does it
  // otherwise).  `S` tracks a one-pass solve since the last barrier.
  for (int pass = 0; pass < 16; ++pass) {
    bool changed = false;
    unsigned W = 0, R = 0;  // slots written / halo-read since the last barrier
    bool S = false;
    for (int step = 0; step < 4; ++step) {
      for (int o = 0; o < n;) {
        const int kind = sp->opk[o];
        if (kind == kOpAxpyL) {
          const int g = sp->opg[o];
          unsigned dsts = 0;
          for (int e = 0; e < g; ++e) dsts |= 1u << sp->opd[o + e];
          const bool need = ((W >> sp->ops[o]) & 1u) || (R & dsts);
          if (need && !sp->opb[o]) {
            sp->opb[o] = 1;
            changed = true;
          }
          if (sp->opb[o]) {
            W = R = 0;
            S = false;
          }
          R |= 1u << sp->ops[o];
          W |= dsts;
          o += g;
        } else if (kind == kOpSolve) {
          if (S && !sp->opb[o]) {
            sp->opb[o] = 1;
            changed = true;
          }
          W = R = 0;  // the solve's own barriers precede its write
          S = one_pass;
          W |= 1u << sp->opd[o];
          ++o;
        } else {
          const int dst = sp->opd[o];
          if (((R >> dst) & 1u) && !sp->opb[o]) {
            sp->opb[o] = 1;
            changed = true;
          }
          if (sp->opb[o]) {
            W = R = 0;
            S = false;
          }
          W |= 1u << dst;
          ++o;
        }
      }
      {  // end of step: the result copy and/or the RHS add write slot 0
        if ((R & 1u) && !sp->resb) {
          sp->resb = 1;
          changed = true;
        }
        if (sp->resb) {
          W = R = 0;
          S = false;
        }
        W |= 1u;
      }
    }
    if (!changed) return true;
  }
  if (why) *why = "SDIRK barrier schedule did not settle";
  return false;
}

// Geometry of a vector split for the step kernels: C CTAs (one thread-block
// cluster), nthr threads per CTA, a chunk of P points per thread.
struct Geom {
  int C = 0, P = 0, nthr = 0;
};

// Rough resident warps per SM of a geometry (shared memory, threads,
// registers), used to order candidates and as the untuned choice.
static double geom_score(const Geom& g, size_t smem, int elem) {
  const int warps = (g.nthr + 31) / 32;
  const int regs = elem == 8 ? (g.P <= 8 ? 96 : g.P <= 16 ? 128 : 224) : (g.P <= 8 ? 64 : g.P <= 16 ? 96 : 168);
  int cps = (int)(228 * 1024 / (smem + 1024));
  cps = std::min(cps, 64 / warps);
  cps = std::min(cps, 65536 / (regs * warps * 32));
  cps = std::min(cps, 32);
  const double lanes = (double)g.nthr / (32.0 * warps);
  return std::min(16.0, (double)(cps * warps)) * lanes - 0.01 * g.C;
}

// Candidate geometries of an n-point vector: P a compiled chunk length,
// 1..256 threads, at least `minpts` points per CTA, shared memory within the
// CTA limit and a co-schedulable cluster; best-scored first.
template <typename F>
static std::vector<Geom> chunk_geometries(int64_t n, int64_t minpts, int elem, F smem_of, int max_out) {
  std::vector<std::pair<double, Geom>> all;
  for (int C = 1; C <= 16; C *= 2) {
    if (n % C) continue;
    const int64_t npc = n / C;
    if (npc < minpts) continue;
    for (int P : kChunkLens) {
      if (npc % P) continue;
      const int64_t nthr = npc / P;
      if (nthr < 1 || nthr > 256) continue;
      Geom g{C, P, (int)nthr};
      const size_t sm = smem_of(g);
      if (sm > 227 * 1024) continue;
      if (C > 1 && sdirk_max_cluster(C, sm, g.nthr) < C) continue;
      all.push_back({geom_score(g, sm, elem), g});
    }
  }
  std::stable_sort(all.begin(), all.end(), [](const std::pair<double, Geom>& a, const std::pair<double, Geom>& b) {
    return a.first > b.first;
  });
  int fc, fp;
  if (geom_forced(&fc, &fp)) {
    std::vector<std::pair<double, Geom>> keep;
    for (auto& x : all)
      if (x.second.C == fc && x.second.P == fp) keep.push_back(x);
    if (!keep.empty()) all.swap(keep);
  }
  std::vector<Geom> out;
  for (auto& x : all)
    if ((int)out.size() < max_out) out.push_back(x.second);
  return out;
}

// Measured tuning is off inside a running server (no candidate is timed
// while other solves share the GPU; cached decisions still apply, else the
// best-scored candidate): set for the serving thread by mgrit_serve.
static thread_local bool g_no_measure = false;
void set_measured_tuning(bool on) { g_no_measure = !on; }
// Setup that does not wait for the device (calling thread): mgrit_setup and
// the solve-graph capture return once their device work is queued on the
// handle's stream, which orders it before anything launched there later.
static thread_local bool g_setup_nowait = false;
void set_setup_nowait(bool on) { g_setup_nowait = on; }

static bool tuning_on() {
  if (g_no_measure) return false;
  const char* on = std::getenv("MGRIT_AUTOTUNE");
  return !(on && on[0] == '0');
}

// Cached geometry decision for a tuning key (process-wide, optionally in
// the MGRIT_AUTOTUNE_CACHE file as C * 1000000 + P * 1000 + nthr).
static bool geom_cached(const std::string& key, Geom* g) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  tune_load();
  auto it = g_tune.find(key);
  if (it == g_tune.end()) return false;
  g->C = it->second / 1000000;
  g->P = (it->second / 1000) % 1000;
  g->nthr = it->second % 1000;
  return true;
}

static void geom_store(const std::string& key, const Geom& g) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  tune_store(key, g.C * 1000000 + g.P * 1000 + g.nthr);
}

// Time `launch` (one warm-up, two timed) on the handle's stream; ms per
// launch, or a negative value on a launch error.
template <typename F>
static float time_launches(mgrit_handle* h, F launch) {
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return -1.f;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return -1.f;
  }
  float ms = -1.f;
  if (launch() >= 0) {
    cudaEventRecord(e0, h->st);
    bool ok = launch() >= 0 && launch() >= 0;
    cudaEventRecord(e1, h->st);
    if (ok && cudaEventSynchronize(e1) == cudaSuccess) {
      cudaEventElapsedTime(&ms, e0, e1);
      ms *= 0.5f;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (cudaGetLastError() != cudaSuccess) return -1.f;
  return ms;
}

// The solves of a step programme leave out the 1/kappa of the stage-matrix
// factorisation: slot s then holds scale_s times its value (a solve
// multiplies the scale of its input by kappa), every AXPY / AXPYL
// coefficient is rescaled to the scales of its operands, and the end of the
// step maps the result back to scale 1 (rscale).  One multiply per point and
// step replaces one per solve.
static void fold_solve_scale(SdirkParams<double>* sp) {
  const double kappa = 1.0 / sp->sscale;
  double scale[kSdirkMaxSlots + 1];
  bool zero[kSdirkMaxSlots + 1];
  for (int s = 0; s <= kSdirkMaxSlots; ++s) {
    scale[s] = 1.0;
    zero[s] = false;
  }
  for (int o = 0; o < sp->nops; ++o) {
    const int dst = sp->opd[o], src = sp->ops[o];
    switch (sp->opk[o]) {
      case kOpCopy:
        scale[dst] = scale[src];
        zero[dst] = false;
        break;
      case kOpZero:
        zero[dst] = true;
        break;
      case kOpAxpy:
      case kOpAxpyL:
        if (zero[dst]) {  // dst starts at 0: take the source's scale
          scale[dst] = scale[src];
          zero[dst] = false;
        } else {
          sp->opc[o] *= scale[dst] / scale[src];
        }
        break;
      case kOpAxpby:  // dst keeps its scale; only the source term is rescaled
        sp->opc[o] *= scale[dst] / scale[src];
        break;
      default:  // kOpSolve
        scale[dst] = scale[src] * kappa;
        zero[dst] = false;
        break;
    }
  }
  sp->rscale = 1.0 / scale[sp->result];
}

// Geometry-free part of the level-0 SDIRK operator: the step programme with
// its barrier schedule, L_p taps, the factorised stage matrix.
static int sdirk_operator(mgrit_handle* h, SdirkParams<double>* sp, BandFactor* bf, std::string* why, double cfl,
                          bool deriv) {
  const mgrit_params& P = h->prm;
  const int p = P.order_p;
  std::memset((void*)sp, 0, sizeof(*sp));
  double gamma = 0.0;
  if (!sdirk_program(P.rk_order_q, cfl, sp, &gamma, why, deriv)) return MGRIT_ERR_UNSUPPORTED;
  Stencil L = upwind_taps(p);
  int ul, ur;
  upwind_bias(p, &ul, &ur);
  sp->p1 = L.width();
  sp->llo = L.lo;
  // the kernel's layout: taps at -l(p) .. r(p) (Sec. 4.1 bias)
  if (L.lo != -ul || L.hi != ur) {
    if (why) *why = "upwind stencil offsets outside the kernel's layout";
    return MGRIT_ERR_UNSUPPORTED;
  }
  for (int i = 0; i < L.width(); ++i) sp->ltaps[i] = L.a[i];
  Stencil A = stencil_add(stencil_identity(), L, gamma * cfl);
  if (!band_factor(A, bf, why)) return MGRIT_ERR_UNSTABLE;
  const int HC = ul, HA = ur;
  if (bf->hc > HC || bf->ha > HA || bf->shift != 0) {
    if (why) *why = "stage matrix factorisation outside the kernel's orders";
    return MGRIT_ERR_UNSUPPORTED;
  }
  sp->sscale = bf->inv_kappa;
  fold_solve_scale(sp);
  if (!schedule_sdirk(sp, why, bf->ha == 0)) return MGRIT_ERR_UNSUPPORTED;
  return MGRIT_OK;
}

// The SDIRK step parameters for geometry g (FP64, and FP32 when outf):
// chunk-scan tables on the host, per-chunk carry tables uploaded.
static int sdirk_with_geom(mgrit_handle* h, const SdirkParams<double>& op, const SdirkParams<double>& op32,
                           const BandFactor& bf, const Geom& g, std::unique_ptr<SdirkParams<double>>* out,
                           double** mt_dev, std::unique_ptr<SdirkParams<float>>* outf, float** mtf_dev) {
  int HC, HA;  // the kernel's recurrence orders: the upwind bias l(p), r(p)
  upwind_bias(h->prm.order_p, &HC, &HA);
  out->reset(new SdirkParams<double>(op));
  SdirkParams<double>& sp = **out;
  sp.n = (int)h->nx;
  sp.P = g.P;
  sp.nthr = g.nthr;
  sp.csize = g.C;
  sp.npc = (int)(h->nx / g.C);
  for (int d = 0; d < 2; ++d) {
    dev_free(h, mt_dev[d]);
    mt_dev[d] = nullptr;
  }
  std::vector<double> mtc, mta;
  fill_solve_dir(&sp.c, bf.cc, bf.hc, HC, g.P, g.nthr, g.C, &mtc);
  fill_solve_dir(&sp.a, bf.ca, bf.ha, HA, g.P, g.nthr, g.C, &mta);
  for (int dd = 0; dd < 2; ++dd) {
    int rc = upload_table(h, dd ? mta : mtc, &mt_dev[dd]);
    if (rc) return rc;
  }
  sp.c.Mt = mt_dev[0];
  sp.a.Mt = mt_dev[1];
  if (outf) {
    outf->reset(new SdirkParams<float>());
    SdirkParams<float>& f = **outf;
    std::memset((void*)&f, 0, sizeof(f));
    f.n = sp.n;
    f.P = sp.P;
    f.nthr = sp.nthr;
    f.csize = sp.csize;
    f.npc = sp.npc;
    f.p1 = sp.p1;
    f.llo = sp.llo;
    // the FP32 step runs its own programme (op32)
    for (int i = 0; i < 8; ++i) f.ltaps[i] = (float)op32.ltaps[i];
    f.sscale = (float)op32.sscale;
    f.rscale = (float)op32.rscale;
    f.nops = op32.nops;
    f.nslots = op32.nslots;
    f.result = op32.result;
    f.resb = op32.resb;
    for (int o = 0; o < kSdirkMaxOps; ++o) {
      f.opk[o] = op32.opk[o];
      f.opd[o] = op32.opd[o];
      f.ops[o] = op32.ops[o];
      f.opg[o] = op32.opg[o];
      f.opb[o] = op32.opb[o];
      f.opc[o] = (float)op32.opc[o];
      f.opc2[o] = (float)op32.opc2[o];
    }
    for (int d = 0; d < 2; ++d) {
      dev_free(h, mtf_dev[d]);
      mtf_dev[d] = nullptr;
    }
    std::vector<float> mtcf, mtaf;
    fill_solve_dir(&f.c, bf.cc, bf.hc, HC, g.P, g.nthr, g.C, &mtcf);
    fill_solve_dir(&f.a, bf.ca, bf.ha, HA, g.P, g.nthr, g.C, &mtaf);
    int rc = upload_table(h, mtcf, &mtf_dev[0]);
    if (!rc) rc = upload_table(h, mtaf, &mtf_dev[1]);
    if (rc) return rc;
    f.c.Mt = mtf_dev[0];
    f.a.Mt = mtf_dev[1];
  }
  return MGRIT_OK;
}

// Build the SDIRK step parameters for K vectors per launch (the level-0
// CF-intervals, or K = 1 for sequential stepping).  The geometry is the
// fastest candidate measured on this handle's buffers (a warm-up plus two
// timed launches of one step on up to 608 vectors; two steps of one vector
// for sequential stepping) when `buffers` is set and tuning is on, else the
// best-scored candidate; decisions are cached per (n_x, K, p, q, precision).
static int build_sdirk_params(mgrit_handle* h, int64_t K, std::unique_ptr<SdirkParams<double>>* out,
                              double** mt_dev, std::unique_ptr<SdirkParams<float>>* outf, float** mtf_dev,
                              std::string* why, bool buffers, double cfl) {
  // FP64 steps take the stage derivatives from the solves (no L_p
  // applications); FP32 steps keep the mat-vec form, whose rounding leaves
  // MIXED refinement at FP64 MGRIT's accuracy (the derivative form's FP32
  // rounding let the error at a 1e-10 residual grow ~15x on the 16384 x
  // 65536 SDIRK3+U5 workload)
  SdirkParams<double> op, op32;
  BandFactor bf, bf32;
  if (cfl <= 0.0) cfl = h->prm.cfl;
  int rc = sdirk_operator(h, &op, &bf, why, cfl, true);
  if (rc) return rc;
  if (outf && (rc = sdirk_operator(h, &op32, &bf32, why, cfl, false))) return rc;
  const int elem = outf ? 4 : 8;
  auto smem_of = [&](const Geom& g) {
    size_t b = sdirk_smem_bytes((int)(h->nx / g.C), g.P, g.nthr, op.nslots, 8);
    if (outf) b = std::max(b, sdirk_smem_bytes((int)(h->nx / g.C), g.P, g.nthr, op32.nslots, 4));
    return b;
  };
  std::vector<Geom> cand = chunk_geometries(h->nx, 1, elem, smem_of, 6);
  if (cand.empty()) {
    if (why) *why = "no SDIRK chunk geometry fits the vector";
    return MGRIT_ERR_UNSUPPORTED;
  }
  const bool seq = (K == 1);
  char keyb[160];
  // c enters the timing only through the scan lengths (carry decay): one
  // significant digit of log2 c is enough to reuse a decision
  std::snprintf(keyb, sizeof(keyb), "sdirk:n=%lld:K=%lld:p=%d:q=%d:b=%d:lc=%d", (long long)h->nx, (long long)K,
                h->prm.order_p, h->prm.rk_order_q, elem, (int)std::lround(std::log2(cfl)));
  const std::string key(keyb);
  Geom best = cand[0];
  Geom cached;
  int fc, fp;
  const bool forced = geom_forced(&fc, &fp);
  bool have = forced || geom_cached(key, &cached);
  if (forced) cached = best;
  if (have) {
    have = false;
    for (auto& g : cand)
      if (g.C == cached.C && g.P == cached.P && g.nthr == cached.nthr) have = true;
    if (have) best = cached;
  }
  if (!have && buffers && tuning_on() && cand.size() > 1) {
    LevelData& L0 = h->lev[0];
    const int64_t Kt = seq ? 1 : std::min<int64_t>(K, 608);
    float bms = 1e30f;
    for (auto& g : cand) {
      if ((rc = sdirk_with_geom(h, op, op32, bf, g, out, mt_dev, outf, mtf_dev))) return rc;
      float ms;
      if (outf) {
        SdirkParams<float> sp = **outf;
        sp.mode = seq ? kModeSEQ : kModeCF;
        sp.zero_start = 0;
        sp.start = L0.uCf[0];
        sp.out = L0.uCf[1];
        sp.rhs = nullptr;
        sp.sub = nullptr;
        sp.partial = nullptr;
        sp.traj = nullptr;
        sp.nsteps = seq ? 2 : 1;
        sp.K = Kt;
        ms = time_launches(h, [&]() { return launch_sdirk(sp, h->st); });
      } else {
        SdirkParams<double> sp = **out;
        sp.mode = seq ? kModeSEQ : kModeCF;
        sp.zero_start = 0;
        sp.start = seq ? h->du0 : L0.uC[0];
        sp.out = seq ? L0.uC[1 - L0.cur] : L0.uC[1];  // sequential: the scratch buffer
        sp.rhs = nullptr;
        sp.sub = nullptr;
        sp.partial = nullptr;
        sp.traj = nullptr;
        sp.nsteps = seq ? 2 : 1;
        sp.K = Kt;
        ms = time_launches(h, [&]() { return launch_sdirk(sp, h->st); });
      }
      if (ms < 0.f) return MGRIT_ERR_CUDA;
      if (ms < bms) {
        bms = ms;
        best = g;
      }
    }
    geom_store(key, best);
  }
  return sdirk_with_geom(h, op, op32, bf, best, out, mt_dev, outf, mtf_dev);
}

// Steps of a stable recurrence x_i = -sum_q coef[q-1] x_{i-q} (order hord)
// after which the response to any start state stays below `cut` of it: the
// warm-up length of the segmented SDIRK kernel (limit + 1 if it does not
// decay within `limit` steps).
static int recurrence_reach(const double* coef, int hord, double cut, int limit) {
  if (hord == 0) return 0;
  int last = -1;
  for (int b = 0; b < hord; ++b) {
    double x[3] = {0.0, 0.0, 0.0};  // x_{i-1}, x_{i-2}, x_{i-3}
    x[b] = 1.0;
    for (int i = 0; i < 4 * limit; ++i) {
      double v = 0.0;
      for (int q = 0; q < hord; ++q) v -= coef[q] * x[q];
      x[2] = x[1];
      x[1] = x[0];
      x[0] = v;
      if (!(std::fabs(v) < cut)) last = std::max(last, i);
    }
  }
  return std::min(last + 1, limit + 1);
}

// A stable recurrence x_i = b_i - sum_q coef[q-1] x_{i-q} of order h <= 3 as
// two cascaded sections: y_i = b_i + r y_{i-1} (order o1 = 0 or 1), then
// x_i = y_i + d[0] x_{i-1} + d[1] x_{i-2} (order o2 = h - o1).  A real root r
// of t^h + coef[0] t^{h-1} + ... is split off (order 3 always has one, in
// (-1, 1) since every root of a stable factor lies inside the unit circle;
// order 2 when its roots are real), the rest deflated.  False if the
// factors do not reproduce the coefficients.
static bool split_sections(const double* coef, int h, int* o1, int* o2, double* r, double d[2]) {
  *o1 = 0;
  *o2 = h;
  *r = 0.0;
  d[0] = d[1] = 0.0;
  if (h == 0) return true;
  if (h == 1) {
    *o1 = 1;
    *o2 = 0;
    *r = -coef[0];
    return true;
  }
  double rt;
  if (h == 3) {
    // bisection on [-1, 1]: f(-1) < 0 < f(1) for roots inside the unit circle
    auto f = [&](double t) { return ((t + coef[0]) * t + coef[1]) * t + coef[2]; };
    double lo = -1.0, hi = 1.0;
    if (!(f(lo) < 0.0 && f(hi) > 0.0)) return false;
    for (int it = 0; it < 200; ++it) {
      const double mid = 0.5 * (lo + hi);
      (f(mid) < 0.0 ? lo : hi) = mid;
    }
    rt = 0.5 * (lo + hi);
    // t^3 + c0 t^2 + c1 t + c2 = (t - rt)(t^2 + e1 t + e2)
    const double e1 = coef[0] + rt, e2 = coef[1] + rt * e1;
    if (std::fabs(-rt * e2 - coef[2]) > 1e-13 * (1.0 + std::fabs(coef[2]))) return false;
    *o1 = 1;
    *o2 = 2;
    *r = rt;
    d[0] = -e1;
    d[1] = -e2;
    return true;
  }
  // h == 2: t^2 + c0 t + c1
  const double disc = coef[0] * coef[0] - 4.0 * coef[1];
  if (disc < 0.0) {  // complex pair: one second-order section
    d[0] = -coef[0];
    d[1] = -coef[1];
    return true;
  }
  const double sq = std::sqrt(disc);
  const double t1 = coef[0] >= 0.0 ? 0.5 * (-coef[0] - sq) : 0.5 * (-coef[0] + sq);  // larger |root|
  const double t2 = coef[1] / t1;
  *o1 = 1;
  *o2 = 1;
  *r = t1;
  d[0] = t2;
  return true;
}

// Segmented FP64 level-0 SDIRK kernel for this handle, or nothing when the
// scheme or vector does not fit it: stiffly accurate SDIRK with at most 3
// stages (q <= 3) and odd p, n_x a multiple of kSegPoints with 32..128
// segments, both warm-up lengths (2^-56 decay of the factor recurrences)
// at most one segment.
static void build_sdirk_seg(mgrit_handle* h) {
  h->seg0.reset();
  const mgrit_params& P = h->prm;
  const int q = P.rk_order_q ? P.rk_order_q : P.order_p;
  if (P.rk_kind != MGRIT_SDIRK || (q != 1 && q != 3) || P.order_p % 2 == 0) return;
  if (h->nx % kSegPoints) return;
  const int64_t T = h->nx / kSegPoints;
  if (T < 32 || T > 128) return;
  SdirkTableau tb;
  if (!sdirk_tableau(q, &tb)) return;
  const double g = tb.A[0][0];
  Stencil L = upwind_taps(P.order_p);
  Stencil A = stencil_add(stencil_identity(), L, g * P.cfl);
  BandFactor bf;
  std::string why;
  if (!band_factor(A, &bf, &why) || bf.shift != 0) return;
  int HC, HA;
  upwind_bias(P.order_p, &HC, &HA);
  if (bf.hc != HC || bf.ha > HA) return;
  std::unique_ptr<SdirkSegParams> sp(new SdirkSegParams());
  std::memset((void*)sp.get(), 0, sizeof(SdirkSegParams));
  sp->n = (int)h->nx;
  sp->T = (int)T;
  sp->stages = tb.s;
  if (!split_sections(bf.cc, bf.hc, &sp->c1, &sp->c2, &sp->cr, sp->cd) ||
      !split_sections(bf.ca, bf.ha, &sp->a1, &sp->a2, &sp->ar, sp->ad))
    return;
  // warm-up lengths (multiples of 8, the kernel's load ring): both sections
  // over the reach of the whole recurrence, or the first section over its
  // own reach plus the second's and the second only over its own, whichever
  // costs fewer multiply-adds; every neglected start state decays below
  // 2^-56 of the data (a sixth of an FP64 rounding unit)
  const double cut = std::ldexp(1.0, -56);
  const int lim = 4 * kSegPoints;
  auto r8 = [](int v) { return (v + 7) & ~7; };
  auto lengths = [&](const double* coef, int hord, int o1, int o2, double r, const double* d, int* w1, int* w2) {
    const int rf = r8(recurrence_reach(coef, hord, cut, lim));
    *w1 = rf;
    *w2 = o2 > 0 ? rf : 0;
    if (o1 == 1 && o2 >= 1) {
      const double c1[1] = {-r};
      const double c2[2] = {-d[0], -d[1]};
      const int b = r8(recurrence_reach(c2, o2, cut, lim));
      const int a = b + r8(recurrence_reach(c1, 1, cut, lim));
      if (a <= kSegPoints && (rf > kSegPoints || a + o2 * b < (1 + o2) * rf)) {
        *w1 = a;
        *w2 = b;
      }
    }
    return *w1 <= kSegPoints;
  };
  if (!lengths(bf.cc, bf.hc, sp->c1, sp->c2, sp->cr, sp->cd, &sp->rc1, &sp->rc2) ||
      !lengths(bf.ca, bf.ha, sp->a1, sp->a2, sp->ar, sp->ad, &sp->ra1, &sp->ra2))
    return;
  // the section orders the kernel is instantiated for
  const int key = sp->c1 * 1000 + sp->c2 * 100 + sp->a1 * 10 + sp->a2;
  if (key != 1211 && key != 1202 && key != 1110 && key != 210 && key != 1000) return;
  // stage right-hand sides from the solves: K_j = (R_j - Y_j) / gamma,
  // R_2 = a2 u + b2 Y_1, R_3 = a3 u + b3 Y_1 + (a_32 / gamma) Y_2, with the
  // unscaled solve U = kappa (I + gamma c L)^{-1} (inv_kappa = 1 / kappa)
  const double ik = bf.inv_kappa;
  sp->last = 1.0;
  if (tb.s == 1) {
    sp->last = ik;
  } else {
    const double a2 = 1.0 - tb.A[1][0] / g, b2 = tb.A[1][0] / g;
    sp->e1u2 = a2 * ik;
    sp->e1y2 = b2 * ik * ik;
    if (tb.s == 3) {
      const double r32 = tb.A[2][1] / g;
      const double a3 = 1.0 - tb.A[2][0] / g - r32 * a2, b3 = tb.A[2][0] / g - r32 * b2;
      sp->e1u3 = a3 * ik;
      sp->e1y3 = b3 * ik * ik;
      sp->e2y3 = r32 * ik;
    }
  }
  h->seg0 = std::move(sp);
}

// FP32 segmented stage kernel of MIXED inner cycles, or nothing when the
// scheme or vector does not fit it: q = 1 or 3, odd p, n_x a multiple of
// kSeg32Points with 32..256 segments, warm-ups (2^-27 decay) within one
// segment.  The stages in mat-vec form: R_j += -c a_ji L_p Y_i.
static void build_sdirk_seg32(mgrit_handle* h) {
  h->seg0f.reset();
  const mgrit_params& P = h->prm;
  const int q = P.rk_order_q ? P.rk_order_q : P.order_p;
  if (!is_mixed(P.precision) || P.rk_kind != MGRIT_SDIRK || (q != 1 && q != 3) || P.order_p % 2 == 0) return;
  if (h->nx % kSeg32Points) return;
  const int64_t T = h->nx / kSeg32Points;
  if (T < 32 || T > 256) return;
  SdirkTableau tb;
  if (!sdirk_tableau(q, &tb)) return;
  const double g = tb.A[0][0];
  Stencil L = upwind_taps(P.order_p);
  int HC, HA;
  upwind_bias(P.order_p, &HC, &HA);
  if (L.lo != -HC || L.hi != HA || L.width() > 8) return;
  Stencil Am = stencil_add(stencil_identity(), L, g * P.cfl);
  BandFactor bf;
  std::string why;
  if (!band_factor(Am, &bf, &why) || bf.shift != 0 || bf.hc != HC || bf.ha > HA) return;
  int c1, c2, a1, a2;
  double cr, cd[2], ar, ad[2];
  if (!split_sections(bf.cc, bf.hc, &c1, &c2, &cr, cd) || !split_sections(bf.ca, bf.ha, &a1, &a2, &ar, ad)) return;
  const int key = c1 * 1000 + c2 * 100 + a1 * 10 + a2;
  if (key != 1211 && key != 1202 && key != 1110 && key != 210 && key != 1000) return;
  const double cut = std::ldexp(1.0, -27);
  const int lim = 4 * kSeg32Points;
  auto r8 = [](int v) { return (v + 7) & ~7; };
  auto lengths = [&](const double* coef, int hord, int o1, int o2, double r, const double* d, int* w1, int* w2) {
    const int rf = r8(recurrence_reach(coef, hord, cut, lim));
    *w1 = rf;
    *w2 = o2 > 0 ? rf : 0;
    if (o1 == 1 && o2 >= 1) {
      const double k1[1] = {-r};
      const double k2[2] = {-d[0], -d[1]};
      const int b = r8(recurrence_reach(k2, o2, cut, lim));
      const int a = b + r8(recurrence_reach(k1, 1, cut, lim));
      if (a <= kSeg32Points && (rf > kSeg32Points || a + o2 * b < (1 + o2) * rf)) {
        *w1 = a;
        *w2 = b;
      }
    }
    return *w1 <= kSeg32Points;
  };
  std::unique_ptr<SdirkSeg32Params> sp(new SdirkSeg32Params());
  std::memset((void*)sp.get(), 0, sizeof(SdirkSeg32Params));
  if (!lengths(bf.cc, bf.hc, c1, c2, cr, cd, &sp->rc1, &sp->rc2) ||
      !lengths(bf.ca, bf.ha, a1, a2, ar, ad, &sp->ra1, &sp->ra2))
    return;
  sp->n = (int)h->nx;
  sp->T = (int)T;
  sp->c1 = c1;
  sp->c2 = c2;
  sp->a1 = a1;
  sp->a2 = a2;
  sp->p1 = L.width();
  sp->stages = tb.s;
  sp->cr = (float)cr;
  sp->cd[0] = (float)cd[0];
  sp->cd[1] = (float)cd[1];
  sp->ar = (float)ar;
  sp->ad[0] = (float)ad[0];
  sp->ad[1] = (float)ad[1];
  sp->ik = (float)bf.inv_kappa;
  for (int i = 0; i < L.width(); ++i) sp->ltaps[i] = (float)L.a[i];
  if (tb.s == 3) {
    sp->g[0] = (float)(-P.cfl * tb.A[1][0]);
    sp->g[1] = (float)(-P.cfl * tb.A[2][0]);
    sp->g[2] = (float)(-P.cfl * tb.A[2][1]);
  }
  h->seg0f = std::move(sp);
}

// MGRIT_SDIRK_SEG=0 never uses the segmented kernel, =1 always where it fits;
// otherwise it runs when it measures faster than the chunked kernel.
static int seg_policy() {
  const char* e = std::getenv("MGRIT_SDIRK_SEG");
  if (!e || !*e) return -1;
  return std::atoi(e) ? 1 : 0;
}

static int build_sdirk(mgrit_handle* h, std::string* why, bool buffers = false) {
  int rc = build_sdirk_params(h, h->lev[0].K, &h->sd0, h->sd_Mt,
                              is_mixed(h->prm.precision) ? &h->sd0f : nullptr, h->sdf_Mt, why, buffers, -1.0);
  if (rc) return rc;
  h->sdirk = true;
  int fc, fp;
  const int pol = seg_policy();
  build_sdirk_seg(h);
  build_sdirk_seg32(h);
  if (pol == 0 || geom_forced(&fc, &fp) || h->lev[0].K < 1) {
    h->seg0.reset();
    h->seg0f.reset();
    return MGRIT_OK;
  }
  if (h->seg0f && pol != 1 && buffers) {
    // measured choice for the FP32 inner kernel, as for FP64 below
    char kb[160];
    std::snprintf(kb, sizeof(kb), "sdseg32:n=%lld:K=%lld:p=%d:q=%d:lc=%d", (long long)h->nx,
                  (long long)h->lev[0].K, h->prm.order_p, h->prm.rk_order_q, (int)std::lround(std::log2(h->prm.cfl)));
    const std::string key32(kb);
    int cached = -1;
    {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      tune_load();
      auto it = g_tune.find(key32);
      if (it != g_tune.end()) cached = it->second;
    }
    if (cached == 0) {
      h->seg0f.reset();
    } else if (cached < 0 && tuning_on()) {
      LevelData& L0 = h->lev[0];
      const int64_t Kt = std::min<int64_t>(L0.K, 608);
      SdirkParams<float> sp = *h->sd0f;
      sp.mode = kModeCF;
      sp.zero_start = 0;
      sp.start = L0.uCf[0];
      sp.out = L0.uCf[1];
      sp.rhs = nullptr;
      sp.sub = nullptr;
      sp.partial = nullptr;
      sp.traj = nullptr;
      sp.g = nullptr;
      sp.nsteps = 2;
      sp.K = Kt;
      const float ms_chunk = time_launches(h, [&]() { return launch_sdirk(sp, h->st); });
      SdirkSeg32Params gp = *h->seg0f;
      gp.mode = kModeCF;
      gp.zero_start = 0;
      gp.start = L0.uCf[0];
      gp.out = L0.uCf[1];
      gp.rhs = nullptr;
      gp.sub = nullptr;
      gp.partial = nullptr;
      gp.nsteps = 2;
      gp.K = Kt;
      const float ms_seg = time_launches(h, [&]() { return launch_sdirk_seg32(gp, h->st); });
      if (ms_chunk < 0.f || ms_seg < 0.f) return MGRIT_ERR_CUDA;
      const bool use = ms_seg < ms_chunk;
      {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        tune_store(key32, use ? 1 : 0);
      }
      if (!use) h->seg0f.reset();
    }
  }
  if (!h->seg0) return MGRIT_OK;
  if (pol == 1 || !buffers) return MGRIT_OK;
  // measured choice: two steps of a CF relaxation on up to 608 intervals,
  // chunked kernel against segmented kernel; cached per shape
  char keyb[160];
  std::snprintf(keyb, sizeof(keyb), "sdseg:n=%lld:K=%lld:p=%d:q=%d:lc=%d", (long long)h->nx,
                (long long)h->lev[0].K, h->prm.order_p, h->prm.rk_order_q, (int)std::lround(std::log2(h->prm.cfl)));
  const std::string key(keyb);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tune_load();
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
      if (!it->second) h->seg0.reset();
      return MGRIT_OK;
    }
  }
  if (!tuning_on()) return MGRIT_OK;
  LevelData& L0 = h->lev[0];
  const int64_t Kt = std::min<int64_t>(L0.K, 608);
  SdirkParams<double> sp = *h->sd0;
  sp.mode = kModeCF;
  sp.zero_start = 0;
  sp.start = L0.uC[0];
  sp.out = L0.uC[1];
  sp.rhs = nullptr;
  sp.sub = nullptr;
  sp.partial = nullptr;
  sp.traj = nullptr;
  sp.g = nullptr;
  sp.nsteps = 2;
  sp.K = Kt;
  const float ms_chunk = time_launches(h, [&]() { return launch_sdirk(sp, h->st); });
  SdirkSegParams gp = *h->seg0;
  gp.mode = kModeCF;
  gp.zero_start = 0;
  gp.start = L0.uC[0];
  gp.out = L0.uC[1];
  gp.sub = nullptr;
  gp.partial = nullptr;
  gp.nsteps = 2;
  gp.K = Kt;
  const float ms_seg = time_launches(h, [&]() { return launch_sdirk_seg(gp, h->st); });
  if (ms_chunk < 0.f || ms_seg < 0.f) return MGRIT_ERR_CUDA;
  const bool use = ms_seg < ms_chunk;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tune_store(key, use ? 1 : 0);
  }
  if (!use) h->seg0.reset();
  return MGRIT_OK;
}

// Measured geometry of level l (after the buffers exist): the candidate
// that runs the level's main launch fastest -- CF relaxation of up to 608
// intervals (m - 1 steps) on an intermediate level, sequential stepping
// (up to 8 steps) on the coarsest -- in the precision the solve runs it
// in; cached per (n_x, intervals, m, p, precision, solve precision).
static int tune_coarse(mgrit_handle* h, int l) {
  LevelData& Lv = h->lev[l];
  if (Lv.redisc) {
    std::string why;
    return build_redisc(h, l, true, &why);
  }
  const bool gm = h->prm.coarse_solve == MGRIT_SOLVE_GMRES;
  const bool coarsest = (l == h->L - 1);
  const bool f32 = h->mixed && !coarsest;
  std::vector<GeomC> cand = coarse_geometries(h, 10);
  int fc, fp;
  if (cand.size() <= 1 || geom_forced(&fc, &fp)) return MGRIT_OK;
  char keyb[160];
  std::snprintf(keyb, sizeof(keyb), "coarse:n=%lld:K=%lld:N=%lld:m=%d:p=%d:b=%d:s=%d:gm=%d", (long long)h->nx,
                (long long)Lv.K, (long long)(coarsest ? Lv.N : 0), Lv.m, h->prm.order_p, f32 ? 4 : 8,
                f32 ? (Lv.solve64 ? 8 : 4) : 8, gm ? h->prm.gmres_maxit : 0);
  const std::string key(keyb);
  Geom cg;
  GeomC best = cand[0];
  if (geom_cached(key, &cg)) {
    for (auto& g : cand)
      if (g.C == cg.C && g.P == cg.P && g.nthr == cg.nthr) return coarse_with_geom(h, l, g);
  }
  if (!tuning_on()) return MGRIT_OK;
  if (gm) {
    // a GMRES solve's time grows with its iteration count: every candidate
    // runs on random level data with the stop tolerance at zero (exactly
    // gmres_maxit iterations per solve); setup zeroes the buffers afterwards
    const uint64_t sd = h->prm.seed + 0x9e37u + (uint64_t)l;
    launch_random_cpoints(Lv.g, h->du0, Lv.N + 1, h->nx, 1, sd, h->st);
    if (Lv.uC[0]) launch_random_cpoints(Lv.uC[0], h->du0, Lv.K + 1, h->nx, 1, sd + 1, h->st);
    if (f32) {
      launch_convert(kCvtD2F, Lv.g, Lv.gf, (Lv.N + 1) * h->nx, h->st);
      launch_convert(kCvtD2F, Lv.uC[0], Lv.uCf[0], (Lv.K + 1) * h->nx, h->st);
    }
    CUDA_TRY(cudaGetLastError());
  }
  auto gm_timing = [&](auto& cp) {
    cp.gm_rtol = 0.0;
    cp.gm_V = reinterpret_cast<decltype(cp.gm_V)>(Lv.gm_V);
    cp.gm_stats = nullptr;
  };
  float bms = 1e30f;
  for (auto& g : cand) {
    int rc = coarse_with_geom(h, l, g);
    if (rc) return rc;
    float ms;
    if (coarsest) {
      CoarseParams<double> cp = Lv.cp;
      gm_timing(cp);
      cp.mode = kModeSEQ;
      cp.zero_start = 1;
      cp.start = nullptr;
      cp.out = nullptr;
      cp.sub = nullptr;
      cp.partial = nullptr;
      cp.g = Lv.g;
      cp.nsteps = (int)std::min<int64_t>(Lv.N, 8);
      cp.K = 1;
      ms = time_launches(h, [&]() { return launch_coarse(cp, h->st); });
    } else {
      const int64_t Kt = std::min<int64_t>(Lv.K, 608);
      auto fill = [&](auto& cp, auto* start, auto* out, auto* gg) {
        gm_timing(cp);
        cp.mode = kModeCF;
        cp.zero_start = 0;
        cp.start = start;
        cp.out = out;
        cp.sub = nullptr;
        cp.partial = nullptr;
        cp.g = gg;
        cp.nsteps = Lv.m - 1;
        cp.K = Kt;
      };
      if (!f32) {
        CoarseParams<double> cp = Lv.cp;
        fill(cp, Lv.uC[0], Lv.uC[1], Lv.g);
        ms = time_launches(h, [&]() { return launch_coarse(cp, h->st); });
      } else if (Lv.solve64) {
        CoarseParams<float, double> cp = Lv.cpfd;
        fill(cp, Lv.uCf[0], Lv.uCf[1], Lv.gf);
        ms = time_launches(h, [&]() { return launch_coarse(cp, h->st); });
      } else {
        CoarseParams<float, float> cp = Lv.cpf;
        fill(cp, Lv.uCf[0], Lv.uCf[1], Lv.gf);
        ms = time_launches(h, [&]() { return launch_coarse(cp, h->st); });
      }
    }
    if (ms < 0.f) return MGRIT_ERR_CUDA;
    if (ms < bms) {
      bms = ms;
      best = g;
    }
  }
  geom_store(key, Geom{best.C, best.P, best.nthr});
  return coarse_with_geom(h, l, best);
}




// Algorithmic flops of `steps` SDIRK steps on K vectors: 2 per multiply-add
// of the two recurrences of each solve, of each L_p mat-vec (plus its axpy)
// and of each axpy, 3 per axpby, and 1 for the step's 1/kappa scaling.
template <typename T>
static double sdirk_flops(const SdirkParams<T>& sp, int64_t nx, int64_t K, int64_t steps) {
  int nsolve = 0, naxl = 0, nax = 0, naxb = 0;
  for (int o = 0; o < sp.nops; ++o) {
    nsolve += sp.opk[o] == kOpSolve;
    naxl += sp.opk[o] == kOpAxpyL;
    nax += sp.opk[o] == kOpAxpy;
    naxb += sp.opk[o] == kOpAxpby;
  }
  const double per_pt = 2.0 * (nsolve * (sp.c.h + sp.a.h) + naxl * (sp.p1 + 1) + nax) + 3.0 * naxb + 1.0;
  return per_pt * (double)nx * (double)K * (double)steps;
}

static int sdirk_launch(mgrit_handle* h, int mode, int zero_start, const double* start, double* out,
                        const double* sub, int nsteps, int64_t K, double* traj, int every, int cat_flops,
                        const SdirkParams<double>* base = nullptr) {
  SdirkParams<double> sp = base ? *base : *h->sd0;
  sp.mode = mode;
  sp.zero_start = zero_start;
  sp.start = start;
  sp.out = out;
  sp.sub = sub;
  sp.rhs = nullptr;
  sp.nsteps = nsteps;
  sp.K = K;
  sp.traj = traj;
  sp.every = every;
  sp.partial = (mode == kModeFRES) ? h->partials : nullptr;
  ProfScope ps(h, cat_flops, sdirk_flops(sp, h->nx, K, nsteps));
  // the segmented kernel keeps a stage vector in each output row and moves
  // it in 16-byte pairs: it runs only on rows that start 16-byte aligned
  // (rows of n_x % 128 == 0 values keep the base pointer's alignment); a
  // caller's row views that do not go to the chunked kernel
  const bool rows16 = (((uintptr_t)start | (uintptr_t)out | (uintptr_t)sub) & 15) == 0;
  if (!base && h->seg0 && !traj && rows16 && (mode == kModeCF || mode == kModeFRES || mode == kModeAPPLY)) {
    SdirkSegParams gp = *h->seg0;
    gp.mode = mode;
    gp.zero_start = zero_start;
    gp.start = start;
    gp.out = out;
    gp.sub = sub;
    gp.nsteps = nsteps;
    gp.K = K;
    gp.partial = sp.partial;
    if (launch_sdirk_seg(gp, h->st) < 0) return MGRIT_ERR_UNSUPPORTED;
  } else if (launch_sdirk(sp, h->st) < 0) {
    return MGRIT_ERR_UNSUPPORTED;
  }
  ++h->launches;
  return check_launch();
}


// ---------------------------------------------------------------------------
// Autotuner of the level-0 stencil tile (outputs per thread R: a CTA covers
// 256 R points of one CF-interval).  Each candidate is timed with CUDA
// events on the handle's own buffers; decisions are cached per (n_x, taps,
// element size, rows) for the process and, if MGRIT_AUTOTUNE_CACHE names a
// file, across processes.  MGRIT_AUTOTUNE=0 keeps the n_x-based default.
// ---------------------------------------------------------------------------
template <typename T>
static int autotune_stencil(mgrit_handle* h, StencilParams<T>* sp, T* in, T* out, int64_t rows) {
  // MGRIT_STENCIL=R or R+16 forces the tile (and the persistent form)
  const char* force = std::getenv("MGRIT_STENCIL");
  if (force) {
    const int code = std::atoi(force);
    const int R = code & 15;
    if (R == 1 || R == 2 || R == 4 || R == 8) {
      sp->tile_r = R;
      sp->persistent = code >> 4 ? 1 : 0;
      return MGRIT_OK;
    }
  }
  const char* on = std::getenv("MGRIT_AUTOTUNE");
  if ((on && on[0] == '0') || rows <= 0) return MGRIT_OK;
  // rows enter only through the wave count: bucket them by powers of two
  int64_t rb = 1;
  while (rb < rows) rb <<= 1;
  char keyb[128];
  std::snprintf(keyb, sizeof(keyb), "stencil2:nx=%lld:taps=%d:b=%d:rows<=%lld", (long long)sp->nx, sp->ntaps,
                (int)sizeof(T), (long long)rb);
  const std::string key(keyb);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tune_load();
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
      sp->tile_r = it->second & 15;
      sp->persistent = it->second >> 4;
      return MGRIT_OK;
    }
  }
  cudaEvent_t e0, e1;
  CUDA_TRY(cudaEventCreate(&e0));
  CUDA_TRY(cudaEventCreate(&e1));
  StencilParams<T> p = *sp;
  p.in = in;
  p.out = out;
  p.rhs = nullptr;
  p.sub = nullptr;
  p.partial = nullptr;
  p.rows = rows;
  float best = 1e30f;
  int bestR = 0;
  for (int code : {1, 2, 4, 8, 17, 18, 20, 24}) {  // R, + 16 for the persistent form
    const int R = code & 15;
    if ((int64_t)kStencilThreadsHost * R > 2 * sp->nx && R > 1) continue;
    p.tile_r = R;
    p.persistent = code >> 4;
    launch_stencil_rows(p, h->st);  // warm-up
    cudaEventRecord(e0, h->st);
    for (int i = 0; i < 3; ++i) launch_stencil_rows(p, h->st);
    cudaEventRecord(e1, h->st);
    if (cudaEventSynchronize(e1) != cudaSuccess) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) {
      best = ms;
      bestR = code;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (check_launch()) return MGRIT_ERR_CUDA;
  if (bestR > 0) {
    sp->tile_r = bestR & 15;
    sp->persistent = bestR >> 4;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tune_store(key, bestR);
  }
  return MGRIT_OK;
}

// ---------------------------------------------------------------------------
// kernels on levels
// ---------------------------------------------------------------------------

// level 0: out rows 1..K = Phi^m in rows 0..K-1 (+ optional residual form)
static int l0_cf(mgrit_handle* h) {
  LevelData& L0 = h->lev[0];
  if (h->sdirk) {
    int rc = sdirk_launch(h, kModeCF, 0, L0.uC[L0.cur], L0.uC[1 - L0.cur], nullptr, h->m, L0.K, nullptr, 0, 0);
    L0.cur = 1 - L0.cur;
    return rc;
  }
  StencilParams<double>& sp = *h->fineM;
  sp.in = L0.uC[L0.cur];
  sp.out = L0.uC[1 - L0.cur] + h->nx;
  sp.rhs = nullptr;
  sp.sub = nullptr;
  sp.partial = nullptr;
  sp.rows = L0.K;
  {
    ProfScope ps(h, 0, 2.0 * sp.ntaps * (double)h->nx * (double)sp.rows);
    launch_stencil_rows(sp, h->st);
  }
  ++h->launches;
  L0.cur = 1 - L0.cur;
  return check_launch();
}

static int l0_fres(mgrit_handle* h) {
  LevelData& L0 = h->lev[0];
  if (h->sdirk) {
    int rc = sdirk_launch(h, kModeFRES, 0, L0.uC[L0.cur], h->lev[1].g, L0.uC[L0.cur], h->m, L0.K, nullptr, 0, 0);
    if (rc) return rc;
    {
      ProfScope ps(h, 2, 0.0);
      launch_reduce_sum(h->partials, L0.K * (h->seg0 ? 1 : h->sd0->csize), h->dnorm, h->st);
    }
    ++h->launches;
    return check_launch();
  }
  StencilParams<double>& sp = *h->fineM;
  sp.in = L0.uC[L0.cur];
  sp.sub = L0.uC[L0.cur] + h->nx;
  sp.out = h->lev[1].g + h->nx;
  sp.rhs = nullptr;
  sp.partial = h->partials;
  sp.rows = L0.K;
  int64_t nb;
  {
    ProfScope ps(h, 0, 2.0 * sp.ntaps * (double)h->nx * (double)sp.rows);
    nb = launch_stencil_rows(sp, h->st);
  }
  ++h->launches;
  {
    ProfScope ps(h, 2, 0.0);
    launch_reduce_sum(h->partials, nb, h->dnorm, h->st);
  }
  ++h->launches;
  return check_launch();
}

// A coarse-level launch with a rediscretised (SDIRK) operator: the SDIRK step
// kernel with the coarse kernel's RHS and output conventions.
template <typename T>
static int redisc_launch(mgrit_handle* h, int l, const SdirkParams<T>& base, int mode, int zero_start,
                         const T* start, T* out, const T* sub, int nsteps, int64_t K, T* g, double* partial) {
  SdirkParams<T> sp = base;
  sp.mode = mode;
  sp.zero_start = zero_start;
  sp.start = start;
  sp.out = out;
  sp.sub = sub;
  sp.rhs = nullptr;
  sp.g = g;
  sp.m = h->lev[l].m;
  sp.nsteps = nsteps;
  sp.K = K;
  sp.traj = nullptr;
  sp.every = 0;
  sp.partial = partial;
  const double fl = sdirk_flops(sp, h->nx, K, nsteps);
  ProfScope ps(h, 1, fl);
  ProfScope psl(h, 4 + std::min(l, kProfCats - 6), fl);
  if (launch_sdirk(sp, h->st) < 0) return MGRIT_ERR_UNSUPPORTED;
  ++h->launches;
  return check_launch();
}

static int coarse_launch(mgrit_handle* h, int l, int mode, int zero_start, const double* start,
                         double* out, const double* sub, double* parent, int nsteps, int64_t K, double* g) {
  if (h->lev[l].redisc)
    return redisc_launch(h, l, *h->lev[l].rd, mode, zero_start, start, out, sub, nsteps, K, g,
                         mode == kModeFRES ? h->partials : nullptr);
  CoarseParams<double> cp = h->lev[l].cp;
  cp.mode = mode;
  cp.zero_start = zero_start;
  cp.start = start;
  cp.out = out;
  cp.sub = sub;
  cp.parent = parent;
  cp.nsteps = nsteps;
  cp.K = K;
  cp.g = g;
  cp.partial = (mode == kModeFRES) ? h->partials : nullptr;
  cp.gm_V = h->lev[l].gm_V;
  cp.gm_stats = h->lev[l].gm_stats;
  const int H = cp.p1 / 2;
  double steps = (double)K * (double)(nsteps - (zero_start ? 1 : 0));
  const double fl = 2.0 * (double)h->nx * steps * (double)(cp.p1 + 2 * H);
  ProfScope ps(h, 1, fl);
  ProfScope psl(h, 4 + std::min(l, kProfCats - 6), fl);
  const int64_t cap = h->lev[l].gm_cap;
  if (cp.gm_max > 0 && K > cap) {
    // the GMRES scratch holds gm_cap intervals: plain applies to more
    // vectors run in pieces
    if (mode != kModeAPPLY || cap < 1) return MGRIT_ERR_UNSUPPORTED;
    for (int64_t k0 = 0; k0 < K; k0 += cap) {
      CoarseParams<double> c2 = cp;
      c2.K = std::min<int64_t>(cap, K - k0);
      c2.start = start + k0 * h->nx;
      c2.out = out + k0 * h->nx;
      if (launch_coarse(c2, h->st) < 0) return MGRIT_ERR_UNSUPPORTED;
      ++h->launches;
      int rc = check_launch();
      if (rc) return rc;
    }
    return MGRIT_OK;
  }
  if (launch_coarse(cp, h->st) < 0) return MGRIT_ERR_UNSUPPORTED;
  ++h->launches;
  return check_launch();
}

static int coarse_correct(mgrit_handle* h, int l);

static int level_pre_and_residual(mgrit_handle* h, int l, bool zero_guess) {
  LevelData& Lv = h->lev[l];
  const int nu = h->prm.nu;
  int rc;
  if (nu == 0) {
    if (zero_guess) {
      CUDA_TRY(cudaMemsetAsync(Lv.uC[Lv.cur], 0, sizeof(double) * (Lv.K + 1) * h->nx, h->st));
      rc = coarse_launch(h, l, kModeFRES, 1, nullptr, h->lev[l + 1].g, nullptr, nullptr, Lv.m, Lv.K, Lv.g);
    } else {
      rc = coarse_launch(h, l, kModeFRES, 0, Lv.uC[Lv.cur], h->lev[l + 1].g, Lv.uC[Lv.cur],
                         nullptr, Lv.m, Lv.K, Lv.g);
    }
    return rc;
  }
  for (int s = 0; s < nu; ++s) {
    bool zs = zero_guess && s == 0;
    rc = coarse_launch(h, l, kModeCF, zs ? 1 : 0, zs ? nullptr : Lv.uC[Lv.cur], Lv.uC[1 - Lv.cur],
                       nullptr, nullptr, Lv.m, Lv.K, Lv.g);
    if (rc) return rc;
    Lv.cur = 1 - Lv.cur;
  }
  rc = coarse_launch(h, l, kModeFRES, 0, Lv.uC[Lv.cur], h->lev[l + 1].g, Lv.uC[Lv.cur], nullptr,
                     Lv.m, Lv.K, Lv.g);
  return rc;
}

// Solve the level-l error equation (RHS lev[l].g, zero initial guess) with
// one cycle and add the result to the C-point unknowns of level l-1.
static int coarse_correct(mgrit_handle* h, int l) {
  LevelData& Lv = h->lev[l];
  LevelData& Par = h->lev[l - 1];
  double* parent = Par.uC[Par.cur];
  int rc;
  if (l == h->L - 1) {
    rc = coarse_launch(h, l, kModeSEQ, 1, nullptr, nullptr, nullptr, parent, (int)Lv.N, 1, Lv.g);
  } else {
    rc = level_pre_and_residual(h, l, true);
    if (rc) return rc;
    rc = coarse_correct(h, l + 1);
    if (rc) return rc;
    rc = coarse_launch(h, l, kModeFOUT, 0, Lv.uC[Lv.cur], nullptr, nullptr, parent, Lv.m - 1, Lv.K, Lv.g);
  }
  if (rc) return rc;
  // the kernel left this level's values at all its points in its RHS rows:
  // add them into the parent's C-points (rows 1..N; row 0 stays exact)
  {
    ProfScope ps(h, 2, 0.0);
    launch_convert(kAddD2D, parent + h->nx, nullptr, Lv.N * h->nx, h->st, Lv.g + h->nx);
  }
  ++h->launches;
  return check_launch();
}

static int level0_relax_residual(mgrit_handle* h, double* norm) {
  int rc;
  for (int s = 0; s < h->prm.nu; ++s) {
    rc = l0_cf(h);
    if (rc) return rc;
  }
  rc = l0_fres(h);
  if (rc) return rc;
  CUDA_TRY(cudaMemcpyAsync(h->hnorm, h->dnorm, sizeof(double), cudaMemcpyDeviceToHost, h->st));
  CUDA_TRY(cudaStreamSynchronize(h->st));
  *norm = norm_of_sq(*h->hnorm);
  return MGRIT_OK;
}


// ---------------------------------------------------------------------------
// MIXED precision: FP32 inner cycles on the error equation
//   e_{km} = Phi^m e_{(k-1)m} + r_k  (level 0, RHS r at C-points only)
// with FP32 relaxation sweeps, FP64 correction solves on ill-conditioned
// levels, and the coarsest level solved sequentially in FP64.
// ---------------------------------------------------------------------------
// One FP32 level-0 step launch of MIXED (CF / FRES): the segmented kernel
// when it runs, else the chunked one; < 0 on a launch error.
static int launch_l0_f32(mgrit_handle* h, const SdirkParams<float>& sp) {
  if (h->seg0f && !sp.traj && !sp.g && (sp.mode == kModeCF || sp.mode == kModeFRES)) {
    SdirkSeg32Params gp = *h->seg0f;
    gp.mode = sp.mode;
    gp.zero_start = sp.zero_start;
    gp.start = sp.start;
    gp.rhs = sp.rhs;
    gp.out = sp.out;
    gp.sub = sp.sub;
    gp.partial = sp.partial;
    gp.nsteps = sp.nsteps;
    gp.K = sp.K;
    return launch_sdirk_seg32(gp, h->st);
  }
  return launch_sdirk(sp, h->st);
}

static int l0f_cf(mgrit_handle* h, bool zero_start) {
  LevelData& L0 = h->lev[0];
  const size_t row = sizeof(float) * (size_t)h->nx;
  float* dst = L0.uCf[1 - L0.curf];
  if (zero_start) {
    // Phi^m 0 + r = r
    CUDA_TRY(cudaMemcpyAsync(dst, L0.gf, row * (L0.K + 1), cudaMemcpyDeviceToDevice, h->st));
    CUDA_TRY(cudaMemsetAsync(dst, 0, row, h->st));
    L0.curf = 1 - L0.curf;
    return MGRIT_OK;
  }
  if (h->sdirk) {
    SdirkParams<float> sp = *h->sd0f;
    sp.mode = kModeCF;
    sp.zero_start = 0;
    sp.start = L0.uCf[L0.curf];
    sp.out = dst;
    sp.rhs = L0.gf;
    sp.sub = nullptr;
    sp.partial = nullptr;
    sp.nsteps = h->m;
    sp.K = L0.K;
    sp.traj = nullptr;
    ProfScope ps(h, kProfL0F32, sdirk_flops(sp, h->nx, L0.K, h->m));
    if (launch_l0_f32(h, sp) < 0) return MGRIT_ERR_UNSUPPORTED;
  } else {
    StencilParams<float>& sp = *h->fineMf;
    sp.in = L0.uCf[L0.curf];
    sp.out = dst + h->nx;
    sp.rhs = L0.gf + h->nx;
    sp.sub = nullptr;
    sp.partial = nullptr;
    sp.rows = L0.K;
    ProfScope ps(h, kProfL0F32, 2.0 * sp.ntaps * (double)h->nx * (double)sp.rows);
    launch_stencil_rows(sp, h->st);
  }
  ++h->launches;
  L0.curf = 1 - L0.curf;
  return check_launch();
}

// rho_{k+1} = Phi^m e_k + r_{k+1} - e_{k+1}  ->  level-1 RHS (FP32)
static int l0f_fres(mgrit_handle* h, bool zero_guess, bool want_norm = false) {
  LevelData& L0 = h->lev[0];
  float* g1 = h->lev[1].gf;
  const size_t row = sizeof(float) * (size_t)h->nx;
  if (zero_guess) {  // e = 0: rho = r, and the coarse correction starts from e = 0
    CUDA_TRY(cudaMemcpyAsync(g1, L0.gf, row * (L0.K + 1), cudaMemcpyDeviceToDevice, h->st));
    CUDA_TRY(cudaMemsetAsync(L0.uCf[L0.curf], 0, row * (L0.K + 1), h->st));
    return MGRIT_OK;
  }
  if (h->sdirk) {
    SdirkParams<float> sp = *h->sd0f;
    sp.mode = kModeFRES;
    sp.zero_start = 0;
    sp.start = L0.uCf[L0.curf];
    sp.out = g1;
    sp.rhs = L0.gf;
    sp.sub = L0.uCf[L0.curf];
    sp.partial = h->partials;
    sp.nsteps = h->m;
    sp.K = L0.K;
    sp.traj = nullptr;
    ProfScope ps(h, kProfL0F32, sdirk_flops(sp, h->nx, L0.K, h->m));
    if (launch_l0_f32(h, sp) < 0) return MGRIT_ERR_UNSUPPORTED;
    if (want_norm) launch_reduce_sum(h->partials, L0.K * (h->seg0f ? 1 : sp.csize), h->dnorm_f, h->st);
  } else {
    StencilParams<float>& sp = *h->fineMf;
    sp.in = L0.uCf[L0.curf];
    sp.out = g1 + h->nx;
    sp.rhs = L0.gf + h->nx;
    sp.sub = L0.uCf[L0.curf] + h->nx;
    sp.partial = h->partials;
    sp.rows = L0.K;
    int64_t nb;
    {
      ProfScope ps(h, kProfL0F32, 2.0 * sp.ntaps * (double)h->nx * (double)sp.rows);
      nb = launch_stencil_rows(sp, h->st);
    }
    if (want_norm) launch_reduce_sum(h->partials, nb, h->dnorm_f, h->st);
  }
  ++h->launches;
  if (want_norm) ++h->launches;
  return check_launch();
}

static int coarse_launch_f(mgrit_handle* h, int l, int mode, int zero_start, const float* start, float* out,
                           const float* sub, float* parent, int nsteps, int64_t K, float* g) {
  LevelData& Lv = h->lev[l];
  if (Lv.redisc) return redisc_launch(h, l, *Lv.rdf, mode, zero_start, start, out, sub, nsteps, K, g, nullptr);
  auto fill = [&](auto& cp) {
    cp.mode = mode;
    cp.zero_start = zero_start;
    cp.start = start;
    cp.out = out;
    cp.sub = sub;
    cp.parent = parent;
    cp.nsteps = nsteps;
    cp.K = K;
    cp.g = g;
    cp.partial = nullptr;
  };
  const int H = Lv.cp.p1 / 2;
  double steps = (double)K * (double)(nsteps - (zero_start ? 1 : 0));
  const double fl = 2.0 * (double)h->nx * steps * (double)(Lv.cp.p1 + 2 * H);
  ProfScope ps(h, 1, fl);
  ProfScope psl(h, 4 + std::min(l, kProfCats - 6), fl);
  if (Lv.gm_V && K > Lv.gm_cap) return MGRIT_ERR_UNSUPPORTED;
  int r;
  if (Lv.solve64) {
    CoarseParams<float, double> cp = Lv.cpfd;
    fill(cp);
    cp.gm_V = Lv.gm_V;
    cp.gm_stats = Lv.gm_stats;
    r = launch_coarse(cp, h->st);
  } else {
    CoarseParams<float, float> cp = Lv.cpf;
    fill(cp);
    cp.gm_V = reinterpret_cast<float*>(Lv.gm_V);
    cp.gm_stats = Lv.gm_stats;
    r = launch_coarse(cp, h->st);
  }
  if (r < 0) return MGRIT_ERR_UNSUPPORTED;
  ++h->launches;
  return check_launch();
}

static int coarse_correct_f(mgrit_handle* h, int l) {
  LevelData& Lv = h->lev[l];
  LevelData& Par = h->lev[l - 1];
  float* parent = Par.uCf[Par.curf];
  int rc;
  const size_t rowd = sizeof(double) * (size_t)h->nx;
  if (l == h->L - 1) {
    // coarsest level in FP64: g (FP32) -> FP64, sequential solve (its
    // values replace the RHS rows), then added to the FP32 parent
    (void)rowd;
    launch_convert(kCvtF2D, Lv.g, Lv.gf, (Lv.N + 1) * h->nx, h->st);
    rc = coarse_launch(h, l, kModeSEQ, 1, nullptr, nullptr, nullptr, nullptr, (int)Lv.N, 1, Lv.g);
    if (rc) return rc;
    launch_convert(kAddD2F, Lv.g + h->nx, parent + h->nx, Lv.N * h->nx, h->st);
    h->launches += 2;
    return check_launch();
  }
  const int nu = h->prm.nu;
  const size_t rowf = sizeof(float) * (size_t)h->nx;
  if (nu == 0) {
    CUDA_TRY(cudaMemsetAsync(Lv.uCf[Lv.curf], 0, rowf * (Lv.K + 1), h->st));
    rc = coarse_launch_f(h, l, kModeFRES, 1, nullptr, h->lev[l + 1].gf, nullptr, nullptr, Lv.m, Lv.K, Lv.gf);
  } else {
    for (int s = 0; s < nu; ++s) {
      bool zs = s == 0;
      rc = coarse_launch_f(h, l, kModeCF, zs ? 1 : 0, zs ? nullptr : Lv.uCf[Lv.curf], Lv.uCf[1 - Lv.curf],
                           nullptr, nullptr, Lv.m, Lv.K, Lv.gf);
      if (rc) return rc;
      Lv.curf = 1 - Lv.curf;
    }
    rc = coarse_launch_f(h, l, kModeFRES, 0, Lv.uCf[Lv.curf], h->lev[l + 1].gf, Lv.uCf[Lv.curf], nullptr, Lv.m,
                         Lv.K, Lv.gf);
  }
  if (rc) return rc;
  rc = coarse_correct_f(h, l + 1);
  if (rc) return rc;
  rc = coarse_launch_f(h, l, kModeFOUT, 0, Lv.uCf[Lv.curf], nullptr, nullptr, parent, Lv.m - 1, Lv.K, Lv.gf);
  if (rc) return rc;
  launch_convert(kAddF2F, nullptr, parent + h->nx, Lv.N * h->nx, h->st, nullptr, Lv.gf + h->nx);
  ++h->launches;
  return check_launch();
}

// One FP32 inner cycle for the level-0 error equation with RHS lev[0].gf.
// One FP32 V-cycle on the error equation A e = r; with want_norm (not on
// the zero-guess cycle) the squared norm of its level-0 residual after the
// pre-relaxation goes to dnorm_f.
static int inner_cycle(mgrit_handle* h, bool zero_guess, bool want_norm = false) {
  const int nu = h->prm.nu;
  int rc;
  if (zero_guess && nu == 0) {
    rc = l0f_fres(h, true);
  } else {
    for (int s = 0; s < nu; ++s) {
      rc = l0f_cf(h, zero_guess && s == 0);
      if (rc) return rc;
    }
    rc = l0f_fres(h, false, want_norm && !zero_guess);
  }
  if (rc) return rc;
  return coarse_correct_f(h, 1);
}


// MIXED pre-relaxation sweep of the FP64 iterate in FP32: C-points rounded
// to FP32, one C-relaxation (zero RHS on level 0), rows 1..K widened back
// into the other FP64 buffer (row 0, the initial condition, stays exact).
// Its rounding is an error like any other that the refinement removes.
static int l0_cf_fp32(mgrit_handle* h) {
  LevelData& L0 = h->lev[0];
  const int64_t nx = h->nx, K = L0.K;
  float* src = L0.uCf[L0.curf];
  float* dst = L0.uCf[1 - L0.curf];
  launch_convert(kCvtD2F, L0.uC[L0.cur], src, (K + 1) * nx, h->st);
  ++h->launches;
  if (h->sdirk) {
    SdirkParams<float> sp = *h->sd0f;
    sp.mode = kModeCF;
    sp.zero_start = 0;
    sp.start = src;
    sp.out = dst;
    sp.rhs = nullptr;
    sp.sub = nullptr;
    sp.partial = nullptr;
    sp.nsteps = h->m;
    sp.K = K;
    sp.traj = nullptr;
    ProfScope ps(h, kProfL0F32, sdirk_flops(sp, nx, K, h->m));
    if (launch_l0_f32(h, sp) < 0) return MGRIT_ERR_UNSUPPORTED;
  } else {
    StencilParams<float> sp = *h->fineMf;
    sp.in = src;
    sp.out = dst + nx;
    sp.rhs = nullptr;
    sp.sub = nullptr;
    sp.partial = nullptr;
    sp.rows = K;
    ProfScope ps(h, kProfL0F32, 2.0 * sp.ntaps * (double)nx * (double)K);
    launch_stencil_rows(sp, h->st);
  }
  ++h->launches;
  if (int rc = check_launch()) return rc;
  launch_convert(kCvtF2D, L0.uC[1 - L0.cur] + nx, dst + nx, K * nx, h->st);
  ++h->launches;
  // the FP32 buffers hold the error iterate between refinement steps, whose
  // t = 0 row is zero: no C-relaxation rewrites it, so clear it here
  CUDA_TRY(cudaMemsetAsync(src, 0, sizeof(float) * (size_t)nx, h->st));
  L0.cur = 1 - L0.cur;
  return check_launch();
}

static int level0_relax_residual_async_mixed(mgrit_handle* h) {
  int rc;
  for (int s = 0; s < h->prm.nu; ++s)
    if ((rc = l0_cf_fp32(h))) return rc;
  return l0_fres(h);
}

// ---------------------------------------------------------------------------
// Graph-resident solve
// ---------------------------------------------------------------------------
// Level-0 pre-relaxation and residual, asynchronous, leaving the C-point
// iterate in buffer 0 so that a replayed graph finds it where it was
// captured (FP64 mode; MIXED keeps the FP64 iterate in place).
static int l0_relax_residual_async(mgrit_handle* h) {
  LevelData& L0 = h->lev[0];
  int rc;
  for (int s = 0; s < h->prm.nu; ++s)
    if ((rc = l0_cf(h))) return rc;
  if (L0.cur != 0) {
    CUDA_TRY(cudaMemcpyAsync(L0.uC[0], L0.uC[1], sizeof(double) * (size_t)h->nx * (L0.K + 1),
                             cudaMemcpyDeviceToDevice, h->st));
    L0.cur = 0;
  }
  return l0_fres(h);
}

// One refinement step captured into the graph: FP64 residual -> FP32 RHS,
// the inner FP32 V-cycles (a fixed count, or adaptive: the first cycle, then
// a nested conditional while node whose body is one cycle and its check),
// the FP32 correction added into the FP64 iterate, and the new FP64
// residual.  cap2 is a second stream for capturing the nested body.
static int mixed_outer_body(mgrit_handle* h, cudaStream_t cap2) {
  LevelData& L0 = h->lev[0];
  int rc;
  launch_convert(kCvtD2F, h->lev[1].g, L0.gf, (L0.K + 1) * h->nx, h->st);
  ++h->launches;
  if (h->prm.inner_cycles > 0) {
    for (int j = 0; j < h->prm.inner_cycles; ++j)
      if ((rc = inner_cycle(h, j == 0))) return rc;
  } else {
    if ((rc = inner_cycle(h, true))) return rc;
    cudaStreamCaptureStatus cs;
    cudaGraph_t cg = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    cudaGraphConditionalHandle hin;
    if (cudaStreamGetCaptureInfo(h->st, &cs, nullptr, &cg, &deps, nullptr, &nd) != cudaSuccess ||
        cs != cudaStreamCaptureStatusActive ||
        cudaGraphConditionalHandleCreate(&hin, cg, 0, cudaGraphCondAssignDefault) != cudaSuccess) {
      note_cuda_error("inner conditional handle", cudaGetLastError());
      return MGRIT_ERR_CUDA;
    }
    launch_inner_init(h->dstate, h->dnorm, hin, h->st);
    ++h->launches;
    if (cudaStreamGetCaptureInfo(h->st, &cs, nullptr, &cg, &deps, nullptr, &nd) != cudaSuccess) {
      note_cuda_error("cudaStreamGetCaptureInfo", cudaGetLastError());
      return MGRIT_ERR_CUDA;
    }
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = hin;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t ncond;
    if (cudaGraphAddNode(&ncond, cg, deps, nullptr, nd, &np) != cudaSuccess) {
      note_cuda_error("inner conditional node", cudaGetLastError());
      return MGRIT_ERR_CUDA;
    }
    cudaGraph_t ibody = np.conditional.phGraph_out[0];
    cudaStream_t outer = h->st;
    if (cudaStreamBeginCaptureToGraph(cap2, ibody, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) !=
        cudaSuccess) {
      note_cuda_error("inner body capture", cudaGetLastError());
      return MGRIT_ERR_CUDA;
    }
    h->st = cap2;
    // the body replays on the same buffers: it must leave the level-0 error
    // iterate where it found it (an odd number of C-relaxations moves it)
    const int curf0 = L0.curf;
    rc = inner_cycle(h, false, true);
    if (!rc && L0.curf != curf0) {
      if (cudaMemcpyAsync(L0.uCf[curf0], L0.uCf[L0.curf], sizeof(float) * (size_t)h->nx * (L0.K + 1),
                          cudaMemcpyDeviceToDevice, h->st) != cudaSuccess)
        rc = MGRIT_ERR_CUDA;
      L0.curf = curf0;
    }
    if (!rc) {
      launch_inner_check(h->dstate, h->dnorm_f, hin, h->st);
      ++h->launches;
    }
    cudaGraph_t ib = nullptr;
    cudaError_t ee = cudaStreamEndCapture(cap2, &ib);
    h->st = outer;
    if (rc) return rc;
    if (ee != cudaSuccess) {
      note_cuda_error("inner body capture end", ee);
      return MGRIT_ERR_CUDA;
    }
    if (cudaStreamUpdateCaptureDependencies(h->st, &ncond, nullptr, 1, cudaStreamSetCaptureDependencies) !=
        cudaSuccess) {
      note_cuda_error("cudaStreamUpdateCaptureDependencies", cudaGetLastError());
      return MGRIT_ERR_CUDA;
    }
  }
  launch_convert(kAddF2D, L0.uC[L0.cur] + h->nx, L0.uCf[L0.curf] + h->nx, L0.K * h->nx, h->st);
  ++h->launches;
  return l0_fres(h);
}

// Device state of a graph-resident solve (allocated once per handle).
static int ensure_solve_state(mgrit_handle* h) {
  if (h->dstate) return MGRIT_OK;
  static_assert(sizeof(DevSolveState) <= kPinBlock, "device state exceeds a pinned block");
  if (dev_alloc(h, (void**)&h->dstate, sizeof(DevSolveState)) || !(h->hstate = (DevSolveState*)pinned_get()))
    return MGRIT_ERR_OOM;
  if (cudaEventCreateWithFlags(&h->done, cudaEventDisableTiming) != cudaSuccess) {
    note_cuda_error("cudaEventCreate", cudaGetLastError());
    return MGRIT_ERR_CUDA;
  }
  return MGRIT_OK;
}

// Add one graph-resident solve of h to graph g as an independent branch:
// prologue (first pre-relaxation and residual, captured from buffer 0) ->
// stop-test init -> conditional while node whose body is one MGRIT
// iteration followed by the check kernel.  g may be the handle's own graph
// or a batch graph holding many solves.
static int capture_solve(mgrit_handle* h, cudaGraph_t g) {
  const bool prof = h->prof.on;
  h->prof.on = false;  // no event records inside the graph
  int rc = ensure_solve_state(h);
  if (rc) {
    h->prof.on = prof;
    return rc;
  }
  cudaGraph_t pro = nullptr;
  // capture on private streams (the legacy default stream cannot capture)
  cudaStream_t user = h->st, cap = nullptr, cap2 = nullptr;
  if ((!g_setup_nowait && cudaStreamSynchronize(user) != cudaSuccess) ||
      cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&cap2, cudaStreamNonBlocking) != cudaSuccess) {
    h->prof.on = prof;
    note_cuda_error("capture stream", cudaGetLastError());
    return MGRIT_ERR_CUDA;
  }
  h->st = cap;
  do {
    cudaGraphConditionalHandle hnd;
    if (cudaGraphConditionalHandleCreate(&hnd, g, 1, cudaGraphCondAssignDefault) != cudaSuccess) {
      note_cuda_error("cudaGraphConditionalHandleCreate", cudaGetLastError());
      rc = MGRIT_ERR_CUDA;
      break;
    }
    h->lev[0].cur = 0;
    if (cudaStreamBeginCapture(h->st, cudaStreamCaptureModeRelaxed) != cudaSuccess) { note_cuda_error("cudaStreamBeginCapture", cudaGetLastError()); rc = MGRIT_ERR_CUDA; break; }
    rc = h->mixed ? level0_relax_residual_async_mixed(h) : l0_relax_residual_async(h);
    if (cudaStreamEndCapture(h->st, &pro) != cudaSuccess && !rc) rc = MGRIT_ERR_CUDA;
    if (rc) break;
    cudaGraphNode_t npro, ninit, ncond;
    if (cudaGraphAddChildGraphNode(&npro, g, nullptr, 0, pro) != cudaSuccess) { note_cuda_error("cudaGraphAddChildGraphNode", cudaGetLastError()); rc = MGRIT_ERR_CUDA; break; }
    void* args[3] = {(void*)&h->dstate, (void*)&h->dnorm, (void*)&hnd};
    cudaKernelNodeParams kp = {};
    kp.func = solve_init_kernel_fn();
    kp.gridDim = dim3(1);
    kp.blockDim = dim3(1);
    kp.sharedMemBytes = 0;
    kp.kernelParams = args;
    if (cudaGraphAddKernelNode(&ninit, g, &npro, 1, &kp) != cudaSuccess) { note_cuda_error("cudaGraphAddKernelNode", cudaGetLastError()); rc = MGRIT_ERR_CUDA; break; }
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = hnd;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    if (cudaGraphAddNode(&ncond, g, &ninit, nullptr, 1, &cp) != cudaSuccess) { note_cuda_error("cudaGraphAddNode", cudaGetLastError()); rc = MGRIT_ERR_CUDA; break; }
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    if (cudaStreamBeginCaptureToGraph(h->st, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) !=
        cudaSuccess) {
      note_cuda_error("cudaStreamBeginCaptureToGraph", cudaGetLastError());
      rc = MGRIT_ERR_CUDA;
      break;
    }
    if (h->mixed) {
      rc = mixed_outer_body(h, cap2);
    } else {
      rc = coarse_correct(h, 1);
      if (!rc) rc = l0_relax_residual_async(h);
    }
    if (!rc) {
      launch_solve_check(h->dstate, h->dnorm, hnd, h->st);
      ++h->launches;
    }
    cudaGraph_t body_out = nullptr;
    if (cudaStreamEndCapture(h->st, &body_out) != cudaSuccess && !rc) rc = MGRIT_ERR_CUDA;
    if (rc) break;
    h->graph_cur = h->lev[0].cur;
  } while (0);
  if (pro) cudaGraphDestroy(pro);
  h->st = user;
  cudaStreamDestroy(cap);
  cudaStreamDestroy(cap2);
  h->prof.on = prof;
  if (rc) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) note_cuda_error("graph build", e);
  }
  return rc;
}

static int build_solve_graph(mgrit_handle* h) {
  if (h->gexec) return MGRIT_OK;
  if (cudaGraphCreate(&h->graph, 0) != cudaSuccess) {
    note_cuda_error("cudaGraphCreate", cudaGetLastError());
    return MGRIT_ERR_CUDA;
  }
  int rc = capture_solve(h, h->graph);
  if (!rc && cudaGraphInstantiate(&h->gexec, h->graph, 0) != cudaSuccess) {
    note_cuda_error("cudaGraphInstantiate", cudaGetLastError());
    rc = MGRIT_ERR_CUDA;
  }
  if (rc) {
    cudaGraphDestroy(h->graph);
    h->graph = nullptr;
    h->gexec = nullptr;
  }
  return rc;
}

// Capture and instantiate the handle's solve graph now (a later
// mgrit_solve_async only launches it): lets a server prepare solves off its
// serving thread.
int solve_graph_prepare(mgrit_handle* h) {
  if (!h) return MGRIT_ERR_INVALID_ARG;
  return build_solve_graph(h);
}

static bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

static int copy_any(void* dst, const void* src, size_t bytes, cudaStream_t st) {
  CUDA_TRY(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, st));
  return MGRIT_OK;
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

const char* mgrit_last_error(void) { return g_last_error; }

const char* mgrit_strerror(int code) {
  switch (code) {
    case MGRIT_OK:
      return "ok";
    case MGRIT_ERR_INVALID_ARG:
      return "invalid argument";
    case MGRIT_ERR_OOM:
      return "out of device memory";
    case MGRIT_ERR_NOT_CONVERGED:
      return "not converged within max_iter";
    case MGRIT_ERR_DIVERGED:
      return "diverged (non-finite or growing residual)";
    case MGRIT_ERR_TIMEOUT:
      return "bounded device wait timed out";
    case MGRIT_ERR_CUDA:
      return "CUDA runtime error";
    case MGRIT_ERR_UNSTABLE:
      return "singular or unstable coarse correction";
    case MGRIT_ERR_UNSUPPORTED:
      return "unsupported parameter combination";
    default:
      return "unknown error";
  }
}

int mgrit_destroy(mgrit_handle* h) {
  if (!h) return MGRIT_OK;
  // a solve still in flight writes the pinned state block: let it land
  // before the block is recycled
  if (h->done) cudaEventSynchronize(h->done);
  for (auto& Lv : h->lev) {
    dev_free(h, Lv.uC[0]);
    dev_free(h, Lv.uC[1]);
    dev_free(h, Lv.g);
    dev_free(h, Lv.Mt_dev[0]);
    dev_free(h, Lv.Mt_dev[1]);
  }
  for (int c = 0; c < kProfCats; ++c)
    for (auto& pr : h->prof.ev[c]) {
      cudaEventDestroy(pr.first);
      cudaEventDestroy(pr.second);
    }
  for (auto e : h->prof.pool) cudaEventDestroy(e);
  dev_free(h, h->sd_Mt[0]);
  dev_free(h, h->sd_Mt[1]);
  dev_free(h, h->sdf_Mt[0]);
  dev_free(h, h->sdf_Mt[1]);
  dev_free(h, h->sdseq_Mt[0]);
  dev_free(h, h->sdseq_Mt[1]);
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  if (h->graph) cudaGraphDestroy(h->graph);
  if (h->done) cudaEventDestroy(h->done);
  dev_free(h, h->dstate);
  pinned_put(h->hstate);
  dev_free(h, h->seq_tmp);
  for (auto& Lv : h->lev) {
    for (int d = 0; d < 2; ++d) {
      dev_free(h, Lv.rd_Mt[d]);
      dev_free(h, Lv.rdf_Mt[d]);
    }
    dev_free(h, Lv.uCf[0]);
    dev_free(h, Lv.uCf[1]);
    dev_free(h, Lv.gf);
    dev_free(h, Lv.Mtf_dev[0]);
    dev_free(h, Lv.Mtf_dev[1]);
    dev_free(h, Lv.gm_V);
    dev_free(h, Lv.gm_stats);
  }
  dev_free(h, h->partials);
  dev_free(h, h->dnorm);
  dev_free(h, h->dnorm_f);
  dev_free(h, h->du0);
  pinned_put(h->hnorm);
  delete h;
  return MGRIT_OK;
}

int mgrit_setup(const mgrit_params* params, void* stream, mgrit_handle** out) {
  if (!params || !out) return MGRIT_ERR_INVALID_ARG;
  *out = nullptr;
  mgrit_params P = *params;
  if (P.rk_order_q == 0) P.rk_order_q = P.order_p;
  if (P.tol <= 0.0) P.tol = 1e-10;
  if (P.max_iter <= 0) P.max_iter = 30;
  if (P.alpha <= 0.0) P.alpha = 1.0;
  if (P.nx < 32 || P.nx % 8 || P.nt < 2 || P.m < 2 || P.cfl <= 0.0 || P.nu < 0 || P.nu > 4)
    return MGRIT_ERR_INVALID_ARG;
  if (P.order_p < 1 || P.order_p > 5) return MGRIT_ERR_INVALID_ARG;
  if (P.rk_kind != MGRIT_ERK && P.rk_kind != MGRIT_SDIRK) return MGRIT_ERR_INVALID_ARG;
  if (P.rk_kind == MGRIT_ERK && P.rk_order_q != P.order_p) return MGRIT_ERR_INVALID_ARG;
  if (P.rk_order_q < 1 || P.rk_order_q > 5) return MGRIT_ERR_INVALID_ARG;
  if (P.precision != MGRIT_FP64 && !is_mixed(P.precision)) return MGRIT_ERR_INVALID_ARG;
  if (P.coarse_op < MGRIT_COARSE_SL_CORRECTED || P.coarse_op > MGRIT_COARSE_REDISC) return MGRIT_ERR_INVALID_ARG;
  if (P.coarse_solve != MGRIT_SOLVE_DIRECT && P.coarse_solve != MGRIT_SOLVE_GMRES) return MGRIT_ERR_INVALID_ARG;
  if (P.coarse_solve == MGRIT_SOLVE_GMRES) {
    // only the corrected operator has a correction system to solve
    if (P.coarse_op != MGRIT_COARSE_SL_CORRECTED) return MGRIT_ERR_INVALID_ARG;
    if (P.gmres_maxit == 0) P.gmres_maxit = P.order_p == 1 ? 10 : 20;  // Sec. 6.3
    if (P.gmres_rtol == 0.0) P.gmres_rtol = 1e-2;
    if (P.gmres_maxit < 1 || P.gmres_maxit > kGmMax || !(P.gmres_rtol > 0.0 && P.gmres_rtol < 1.0))
      return MGRIT_ERR_INVALID_ARG;
  }
  // rediscretising an explicit method at m^l dt is unstable for practical
  // m c (Sec. 5): offered for SDIRK only
  if (P.coarse_op == MGRIT_COARSE_REDISC && P.rk_kind != MGRIT_SDIRK) return MGRIT_ERR_UNSUPPORTED;
  // SDIRKq with q != p adds a phi_q D^{(q+1)}_2 correction term: q must be
  // odd (a symmetric even-order difference) and q <= p (inside the SL band);
  // even p (the dispersive schemes of Sec. 6.4) pairs q = p only
  if (P.rk_kind == MGRIT_SDIRK && P.rk_order_q != P.order_p &&
      (P.order_p % 2 == 0 || P.rk_order_q > P.order_p || P.rk_order_q % 2 == 0))
    return MGRIT_ERR_UNSUPPORTED;
  if (P.m_coarse == 0) P.m_coarse = P.m;
  if (P.m_coarse < 2) return MGRIT_ERR_INVALID_ARG;
  if (P.nt % P.m) return MGRIT_ERR_INVALID_ARG;
  // m from level 0 to 1, m_coarse below
  auto factor = [&](int l) { return l == 0 ? P.m : P.m_coarse; };
  int L = P.levels;
  if (L == 0) {  // coarsen until fewer than two time points would result
    L = 1;
    int64_t N = P.nt;
    while (N % factor(L - 1) == 0 && N / factor(L - 1) >= 2) {
      N /= factor(L - 1);
      ++L;
    }
    if (L < 2) L = 2;
  }
  if (L < 2 || L > MGRIT_MAX_LEVELS) return MGRIT_ERR_INVALID_ARG;
  {
    int64_t N = P.nt;
    for (int l = 1; l < L; ++l) {
      if (N % factor(l - 1)) return MGRIT_ERR_INVALID_ARG;
      N /= factor(l - 1);
    }
    if (N < 1) return MGRIT_ERR_INVALID_ARG;
  }
  if (!has_chunk_geometry(P.nx)) return MGRIT_ERR_INVALID_ARG;
  // stencil wider than the grid is rejected (wrap-around of one step)
  if ((int64_t)(P.order_p + 1) * P.rk_order_q + 1 > P.nx) return MGRIT_ERR_INVALID_ARG;

  struct Del {
    void operator()(mgrit_handle* x) const { mgrit_destroy(x); }
  };
  auto h = std::unique_ptr<mgrit_handle, Del>(new mgrit_handle());
  h->prm = P;
  h->prm.levels = L;
  h->st = (cudaStream_t)stream;
  h->L = L;
  h->nx = P.nx;
  h->m = P.m;
  if (const char* it = std::getenv("MGRIT_INNER_TOL")) {
    const double v = std::atof(it);
    if (v > 0.0 && v < 1.0) h->inner_tol = v;
  }
  cudaGetDevice(&h->device);
  h->lev.resize(L);
  int64_t N = P.nt;
  long long tstep = 1;
  for (int l = 0; l < L; ++l) {
    h->lev[l].N = N;
    h->lev[l].m = factor(l);
    h->lev[l].tstep = tstep;
    h->lev[l].K = (l < L - 1) ? N / factor(l) : 0;
    N /= factor(l);
    tstep *= factor(l);
  }
  // level-0 operators
  int rc = MGRIT_OK;
  h->fine1.reset(new StencilParams<double>());
  h->fineM.reset(new StencilParams<double>());
  if (P.rk_kind == MGRIT_ERK) {
    Stencil step = erk_step_stencil(P.order_p, P.rk_order_q, P.cfl);
    rc = set_stencil(h->fine1.get(), step, P.nx);
    if (rc) return rc;
    Stencil stepM = stencil_power(step, P.m);
    h->fineM_taps_raw = stepM.width();
    rc = set_stencil(h->fineM.get(), stepM, P.nx);
    if (rc) return rc;
    if (is_mixed(P.precision)) {
      h->fineMf.reset(new StencilParams<float>());
      rc = set_stencil(h->fineMf.get(), stepM, P.nx);
      if (rc) return rc;
    }
  } else {
    std::string why0;
    rc = build_sdirk(h.get(), &why0);
    if (rc) return rc;
  }
  // coarse operators
  std::vector<double> php, phq, es;
  std::vector<long long> ks;
  phi_recursion(P, L, &php, &phq, &ks, &es);
  std::string why;
  for (int l = 1; l < L; ++l) {
    if (P.coarse_op == MGRIT_COARSE_SL) {  // direct SL operator: phi = 0, no correction solve
      h->lev[l].nosolve = true;
      rc = build_coarse(h.get(), l, 0.0, 0.0, ks[l], es[l], &why);
    } else {
      rc = build_coarse(h.get(), l, php[l], phq[l], ks[l], es[l], &why);
    }
    if (rc) return rc;
    if (P.coarse_op == MGRIT_COARSE_REDISC && (rc = build_redisc(h.get(), l, false, &why))) return rc;
  }
  // buffers
  const size_t row = sizeof(double) * (size_t)P.nx;
  auto alloc = [&](double** p, size_t bytes) -> int { return dev_alloc(h.get(), (void**)p, bytes); };
  for (int l = 0; l < L; ++l) {
    LevelData& Lv = h->lev[l];
    if (l < L - 1) {
      for (int b = 0; b < 2; ++b) {
        if ((rc = alloc(&Lv.uC[b], row * (Lv.K + 1)))) return rc;
        CUDA_TRY(cudaMemsetAsync(Lv.uC[b], 0, row * (Lv.K + 1), h->st));
      }
    }
    if (l >= 1) {
      if ((rc = alloc(&Lv.g, row * (Lv.N + 1)))) return rc;
      CUDA_TRY(cudaMemsetAsync(Lv.g, 0, row * (Lv.N + 1), h->st));
    }
    if (l >= 1 && P.coarse_solve == MGRIT_SOLVE_GMRES) {
      Lv.gm_cap = std::max<int64_t>(Lv.K, 1);
      if ((rc = alloc(&Lv.gm_V, row * (size_t)Lv.gm_cap * (size_t)(P.gmres_maxit + 1)))) return rc;
      if ((rc = dev_alloc(h.get(), (void**)&Lv.gm_stats, 2 * sizeof(unsigned long long)))) return rc;
      CUDA_TRY(cudaMemsetAsync(Lv.gm_stats, 0, 2 * sizeof(unsigned long long), h->st));
    }
  }
  if (is_mixed(P.precision)) {
    h->mixed = true;
    const size_t rowf = sizeof(float) * (size_t)P.nx;
    auto allocf = [&](float** p, size_t bytes) -> int {
      if (dev_alloc(h.get(), (void**)p, bytes)) return MGRIT_ERR_OOM;
      return cudaMemsetAsync(*p, 0, bytes, h->st) == cudaSuccess ? MGRIT_OK : MGRIT_ERR_CUDA;
    };
    for (int l = 0; l < L; ++l) {
      LevelData& Lv = h->lev[l];
      if (l < L - 1) {
        for (int b = 0; b < 2; ++b)
          if ((rc = allocf(&Lv.uCf[b], rowf * (Lv.K + 1)))) return rc;
      }
      int64_t grow = (l == 0) ? Lv.K + 1 : Lv.N + 1;
      if ((rc = allocf(&Lv.gf, rowf * grow))) return rc;
    }
    if ((rc = alloc(&h->seq_tmp, row * (h->lev[L - 1].N + 1)))) return rc;
  }
  // partial sums: one per CTA of any launch (tile count of the stencil at
  // its smallest tile, clusters of up to 16 CTAs for the step kernels)
  h->npart = h->lev[0].K * std::max<int64_t>(stencil_tiles(P.nx, 1), 16) + 1;
  for (int l = 1; l < L; ++l) h->npart = std::max<int64_t>(h->npart, (h->lev[l].K + 1) * 16);
  if ((rc = alloc(&h->partials, sizeof(double) * h->npart))) return rc;
  if ((rc = alloc(&h->dnorm, sizeof(double)))) return rc;
  if ((rc = alloc(&h->dnorm_f, sizeof(double)))) return rc;
  if ((rc = alloc(&h->du0, row))) return rc;
  CUDA_TRY(cudaMemsetAsync(h->du0, 0, row, h->st));
  if (!(h->hnorm = (double*)pinned_get())) return MGRIT_ERR_OOM;
  // measured launch geometries on this handle's buffers (cached per shape):
  // the level-0 stencil tile or SDIRK chunk geometry, each coarse level's
  LevelData& L0 = h->lev[0];
  if (!h->sdirk) {
    if ((rc = autotune_stencil(h.get(), h->fineM.get(), L0.uC[0], L0.uC[1], L0.K))) return rc;
    if (h->mixed && (rc = autotune_stencil(h.get(), h->fineMf.get(), L0.uCf[0], L0.uCf[1], L0.K))) return rc;
  } else {
    std::string why0;
    if ((rc = build_sdirk(h.get(), &why0, true))) return rc;
  }
  for (int l = 1; l < L; ++l)
    if ((rc = tune_coarse(h.get(), l))) return rc;
  // the timing launches wrote into the level buffers: back to zero
  for (int l = 0; l < L; ++l) {
    LevelData& Lv = h->lev[l];
    for (int b = 0; b < 2; ++b) {
      if (Lv.uC[b]) CUDA_TRY(cudaMemsetAsync(Lv.uC[b], 0, row * (Lv.K + 1), h->st));
      if (Lv.uCf[b]) CUDA_TRY(cudaMemsetAsync(Lv.uCf[b], 0, sizeof(float) * P.nx * (Lv.K + 1), h->st));
    }
    if (Lv.g) CUDA_TRY(cudaMemsetAsync(Lv.g, 0, row * (Lv.N + 1), h->st));
    if (Lv.gf) CUDA_TRY(cudaMemsetAsync(Lv.gf, 0, sizeof(float) * P.nx * ((l == 0 ? Lv.K : Lv.N) + 1), h->st));
  }
  if (!g_setup_nowait) CUDA_TRY(cudaStreamSynchronize(h->st));
  *out = h.release();
  return MGRIT_OK;
}

int mgrit_set_initial(mgrit_handle* h, const double* u0, const double* init) {
  if (!h || !u0) return MGRIT_ERR_INVALID_ARG;
  LevelData& L0 = h->lev[0];
  const size_t row = sizeof(double) * (size_t)h->nx;
  int rc = copy_any(h->du0, u0, row, h->st);
  if (rc) return rc;
  if (init) {
    rc = copy_any(L0.uC[0], init, row * (L0.K + 1), h->st);
    if (rc) return rc;
    CUDA_TRY(cudaMemcpyAsync(L0.uC[0], h->du0, row, cudaMemcpyDeviceToDevice, h->st));
  } else {
    launch_random_cpoints(L0.uC[0], h->du0, L0.K + 1, h->nx, h->m, h->prm.seed, h->st);
    ++h->launches;
    if ((rc = check_launch())) return rc;
  }
  CUDA_TRY(cudaMemcpyAsync(L0.uC[1], h->du0, row, cudaMemcpyDeviceToDevice, h->st));
  L0.cur = 0;
  h->have_initial = true;
  CUDA_TRY(cudaStreamSynchronize(h->st));
  return MGRIT_OK;
}

int mgrit_relax(mgrit_handle* h, int level, int nu) {
  if (!h || level < 0 || level >= h->L - 1 || nu < 0) return MGRIT_ERR_INVALID_ARG;
  int rc;
  for (int s = 0; s < nu; ++s) {
    if (level == 0) {
      rc = l0_cf(h);
    } else {
      LevelData& Lv = h->lev[level];
      rc = coarse_launch(h, level, kModeCF, 0, Lv.uC[Lv.cur], Lv.uC[1 - Lv.cur], nullptr, nullptr, Lv.m,
                         Lv.K, Lv.g);
      Lv.cur = 1 - Lv.cur;
    }
    if (rc) return rc;
  }
  return MGRIT_OK;
}

int mgrit_residual(mgrit_handle* h, int level, double* norm_out) {
  if (!h || level < 0 || level >= h->L - 1) return MGRIT_ERR_INVALID_ARG;
  int rc;
  if (level == 0) {
    rc = l0_fres(h);
  } else {
    LevelData& Lv = h->lev[level];
    rc = coarse_launch(h, level, kModeFRES, 0, Lv.uC[Lv.cur], h->lev[level + 1].g, Lv.uC[Lv.cur],
                       nullptr, Lv.m, Lv.K, Lv.g);
    if (!rc) {
      launch_reduce_sum(h->partials, Lv.K * (Lv.redisc ? Lv.rd->csize : Lv.cp.csize), h->dnorm, h->st);
      ++h->launches;
      rc = check_launch();
    }
  }
  if (rc) return rc;
  if (norm_out) {
    CUDA_TRY(cudaMemcpyAsync(h->hnorm, h->dnorm, sizeof(double), cudaMemcpyDeviceToHost, h->st));
    CUDA_TRY(cudaStreamSynchronize(h->st));
    *norm_out = norm_of_sq(*h->hnorm);
  }
  return MGRIT_OK;
}

int mgrit_coarse_apply(mgrit_handle* h, int level, const double* d_in, double* d_out, int64_t nvec) {
  if (!h || level < 0 || level >= h->L || !d_in || !d_out || nvec < 0) return MGRIT_ERR_INVALID_ARG;
  if (nvec == 0) return MGRIT_OK;
  if (level == 0 && h->sdirk) return sdirk_launch(h, kModeAPPLY, 0, d_in, d_out, nullptr, 1, nvec, nullptr, 0, 0);
  if (level == 0) {
    StencilParams<double>& sp = *h->fine1;
    sp.in = d_in;
    sp.out = d_out;
    sp.rhs = nullptr;
    sp.sub = nullptr;
    sp.partial = nullptr;
    sp.rows = nvec;
    launch_stencil_rows(sp, h->st);
    ++h->launches;
    return check_launch();
  }
  return coarse_launch(h, level, kModeAPPLY, 0, d_in, d_out, nullptr, nullptr, 1, nvec, nullptr);
}

int mgrit_coarse_correct(mgrit_handle* h) {
  if (!h || h->L < 2) return MGRIT_ERR_INVALID_ARG;
  if (h->mixed) return MGRIT_ERR_UNSUPPORTED;
  return coarse_correct(h, 1);
}

int mgrit_level_rows(mgrit_handle* h, int level, int field, int64_t row0, int64_t nrows, double* ptr, int op) {
  if (!h || level < 0 || level >= h->L || !ptr || row0 < 0 || nrows < 0 || op < 0 || op > 2)
    return MGRIT_ERR_INVALID_ARG;
  LevelData& Lv = h->lev[level];
  double* buf = nullptr;
  int64_t rows = 0;
  if (field == 0) {
    if (level == h->L - 1) return MGRIT_ERR_INVALID_ARG;
    buf = Lv.uC[Lv.cur];
    rows = Lv.K + 1;
  } else if (field == 1) {
    if (level == 0) return MGRIT_ERR_INVALID_ARG;
    buf = Lv.g;
    rows = Lv.N + 1;
  } else {
    return MGRIT_ERR_INVALID_ARG;
  }
  if (row0 + nrows > rows) return MGRIT_ERR_INVALID_ARG;
  if (nrows == 0) return MGRIT_OK;
  double* at = buf + row0 * h->nx;
  const size_t bytes = sizeof(double) * (size_t)h->nx * (size_t)nrows;
  int rc = MGRIT_OK;
  if (op == 0) {
    rc = copy_any(ptr, at, bytes, h->st);
    if (!rc && !is_device_ptr(ptr)) CUDA_TRY(cudaStreamSynchronize(h->st));
  } else if (op == 1) {
    rc = copy_any(at, ptr, bytes, h->st);
    if (!rc && !is_device_ptr(ptr)) CUDA_TRY(cudaStreamSynchronize(h->st));
  } else {
    if (!is_device_ptr(ptr)) return MGRIT_ERR_INVALID_ARG;
    launch_convert(kAddD2D, at, nullptr, nrows * h->nx, h->st, ptr);
    ++h->launches;
    rc = check_launch();
  }
  if (!rc && level == 0 && field == 0 && op != 0) h->have_initial = true;
  return rc;
}

int mgrit_vcycle(mgrit_handle* h, double* norm_out) {
  if (!h) return MGRIT_ERR_INVALID_ARG;
  int rc = coarse_correct(h, 1);
  if (rc) return rc;
  double nrm = 0.0;
  rc = level0_relax_residual(h, &nrm);
  if (rc) return rc;
  if (norm_out) *norm_out = nrm;
  return MGRIT_OK;
}

int mgrit_solve(mgrit_handle* h, const double* u0, double* u_out, mgrit_stats* stats) {
  if (!h) return MGRIT_ERR_INVALID_ARG;
  auto t0 = std::chrono::steady_clock::now();
  int rc;
  if (u0) {
    rc = mgrit_set_initial(h, u0, nullptr);
    if (rc) return rc;
  } else if (!h->have_initial) {
    return MGRIT_ERR_INVALID_ARG;
  }
  mgrit_stats st;
  std::memset(&st, 0, sizeof(st));
  st.levels = h->L;
  double nrm = 0.0;
  int it = 0;
  int status = MGRIT_OK;
  if (h->mixed) {
    // FP64 iterative refinement around FP32 inner cycles: the first residual
    // follows the FP64 pre-relaxation; every later one is the FP64 C-point
    // residual of the corrected iterate (F-relaxation implied).
    LevelData& L0 = h->lev[0];
    const int inner = h->prm.inner_cycles;  // 0: adaptive
    for (int s = 0; s < h->prm.nu; ++s)
      if ((rc = l0_cf_fp32(h))) return rc;
    if ((rc = l0_fres(h))) return rc;
    CUDA_TRY(cudaMemcpyAsync(h->hnorm, h->dnorm, sizeof(double), cudaMemcpyDeviceToHost, h->st));
    CUDA_TRY(cudaStreamSynchronize(h->st));
    nrm = norm_of_sq(*h->hnorm);
    if (rc) return rc;
    while (true) {
      if (st.history_len < MGRIT_MAX_HISTORY) st.rnorm_history[st.history_len++] = nrm;
      if (it == 0) st.rnorm0 = nrm;
      st.rnorm = nrm;
      if (!std::isfinite(nrm) || (it > 0 && nrm > 1e3 * st.rnorm0)) {
        status = MGRIT_ERR_DIVERGED;
        break;
      }
      if (nrm <= h->prm.tol * st.rnorm0) {
        st.converged = 1;
        break;
      }
      if (it >= h->prm.max_iter) {
        status = MGRIT_ERR_NOT_CONVERGED;
        break;
      }
      // r (FP64, rows 0..K of the level-1 RHS) -> FP32 RHS of the inner solve
      launch_convert(kCvtD2F, h->lev[1].g, L0.gf, (L0.K + 1) * h->nx, h->st);
      ++h->launches;
      if (h->prm.inner_cycles > 0) {
        for (int j = 0; j < inner; ++j) {
          rc = inner_cycle(h, j == 0);
          if (rc) return rc;
          ++st.inner_cycles;
        }
      } else {  // adaptive: the rule of inner_check_kernel, on the host
        rc = inner_cycle(h, true);
        if (rc) return rc;
        ++st.inner_cycles;
        const double rho0 = nrm;
        const double target = inner_target(h->prm.tol, st.rnorm0, rho0, h->inner_tol);
        double prev = rho0;
        int count = 1;
        bool go = count < kInnerMax;
        while (go) {
          rc = inner_cycle(h, false, true);
          if (rc) return rc;
          ++st.inner_cycles;
          ++count;
          CUDA_TRY(cudaMemcpyAsync(h->hnorm, h->dnorm_f, sizeof(double), cudaMemcpyDeviceToHost, h->st));
          CUDA_TRY(cudaStreamSynchronize(h->st));
          const double rho = norm_of_sq(*h->hnorm);
          go = inner_continue(rho, prev, rho0, count, kInnerMax, target);
          prev = rho;
        }
      }
      // u += e at the C-points k = 1..K (FP64 master iterate)
      launch_convert(kAddF2D, L0.uC[L0.cur] + h->nx, L0.uCf[L0.curf] + h->nx, L0.K * h->nx, h->st);
      ++h->launches;
      rc = l0_fres(h);
      if (rc) return rc;
      CUDA_TRY(cudaMemcpyAsync(h->hnorm, h->dnorm, sizeof(double), cudaMemcpyDeviceToHost, h->st));
      CUDA_TRY(cudaStreamSynchronize(h->st));
      nrm = norm_of_sq(*h->hnorm);
      ++it;
      ++st.outer_iterations;
    }
  }
  while (!h->mixed) {
    rc = level0_relax_residual(h, &nrm);
    if (rc) return rc;
    if (st.history_len < MGRIT_MAX_HISTORY) st.rnorm_history[st.history_len++] = nrm;
    if (it == 0) st.rnorm0 = nrm;
    st.rnorm = nrm;
    if (!std::isfinite(nrm) || (it > 0 && nrm > 1e3 * st.rnorm0)) {
      status = MGRIT_ERR_DIVERGED;
      break;
    }
    if (nrm <= h->prm.tol * st.rnorm0) {
      st.converged = 1;
      break;
    }
    if (it >= h->prm.max_iter) {
      status = MGRIT_ERR_NOT_CONVERGED;
      break;
    }
    rc = coarse_correct(h, 1);
    if (rc) return rc;
    ++it;
  }
  st.iterations = it;
  if (st.history_len >= 2 && st.rnorm_history[st.history_len - 2] > 0)
    st.conv_factor = st.rnorm_history[st.history_len - 1] / st.rnorm_history[st.history_len - 2];
  if (u_out) {
    LevelData& L0 = h->lev[0];
    rc = copy_any(u_out, L0.uC[L0.cur], sizeof(double) * (size_t)h->nx * (L0.K + 1), h->st);
    if (rc) return rc;
  }
  CUDA_TRY(cudaStreamSynchronize(h->st));
  st.ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (stats) *stats = st;
  return status;
}

int mgrit_level_io(mgrit_handle* h, int level, int field, double* ptr, int to_device, int64_t* rows_out) {
  if (!h || level < 0 || level >= h->L || !ptr) return MGRIT_ERR_INVALID_ARG;
  LevelData& Lv = h->lev[level];
  double* buf = nullptr;
  int64_t rows = 0;
  if (field == 0) {
    if (level == h->L - 1) return MGRIT_ERR_INVALID_ARG;
    buf = Lv.uC[Lv.cur];
    rows = Lv.K + 1;
  } else if (field == 1) {
    if (level == 0) return MGRIT_ERR_INVALID_ARG;
    buf = Lv.g;
    rows = Lv.N + 1;
  } else {
    return MGRIT_ERR_INVALID_ARG;
  }
  size_t bytes = sizeof(double) * (size_t)h->nx * rows;
  int rc = to_device ? copy_any(buf, ptr, bytes, h->st) : copy_any(ptr, buf, bytes, h->st);
  if (rc) return rc;
  if (to_device && field == 0) {
    // keep both buffers' row 0 consistent (the t = 0 row never changes)
    size_t row = sizeof(double) * (size_t)h->nx;
    CUDA_TRY(cudaMemcpyAsync(Lv.uC[1 - Lv.cur], buf, row, cudaMemcpyDeviceToDevice, h->st));
    if (level == 0) CUDA_TRY(cudaMemcpyAsync(h->du0, buf, row, cudaMemcpyDeviceToDevice, h->st));
    if (level == 0) h->have_initial = true;
  }
  CUDA_TRY(cudaStreamSynchronize(h->st));
  if (rows_out) *rows_out = rows;
  return MGRIT_OK;
}

static int fine_propagate_impl(mgrit_handle* h, const double* u0, double* u_out, int64_t nsteps, int64_t every,
                               double* traj, bool sync);

int mgrit_fine_propagate(mgrit_handle* h, const double* u0, double* u_out, int64_t nsteps, int64_t every,
                         double* traj) {
  return fine_propagate_impl(h, u0, u_out, nsteps, every, traj, true);
}

int mgrit_fine_propagate_async(mgrit_handle* h, const double* d_u0, double* d_out, int64_t nsteps) {
  if (!h || !d_u0 || !d_out || !is_device_ptr(d_u0) || !is_device_ptr(d_out)) return MGRIT_ERR_INVALID_ARG;
  return fine_propagate_impl(h, d_u0, d_out, nsteps, 0, nullptr, false);
}

static int fine_propagate_impl(mgrit_handle* h, const double* u0, double* u_out, int64_t nsteps, int64_t every,
                               double* traj, bool sync) {
  if (!h || !u0 || !u_out || nsteps < 0 || every < 0) return MGRIT_ERR_INVALID_ARG;
  const int64_t nx = h->nx;
  if (h->sdirk) {
    const size_t row = sizeof(double) * (size_t)nx;
    int rc = copy_any(h->du0, u0, row, h->st);
    if (rc) return rc;
    bool out_dev = is_device_ptr(u_out);
    double* dout = out_dev ? u_out : h->lev[0].uC[1 - h->lev[0].cur];
    if (nsteps > INT32_MAX) return MGRIT_ERR_INVALID_ARG;
    if (!h->sdseq) {
      std::string why;
      rc = build_sdirk_params(h, 1, &h->sdseq, h->sdseq_Mt, nullptr, nullptr, &why, true, -1.0);
      if (rc) return rc;
    }
    rc = sdirk_launch(h, kModeSEQ, 0, h->du0, dout, nullptr, (int)nsteps, 1, every > 0 ? traj : nullptr,
                      (int)every, 3, h->sdseq.get());
    if (rc) return rc;
    if (!out_dev && (rc = copy_any(u_out, dout, row, h->st))) return rc;
    if (sync) CUDA_TRY(cudaStreamSynchronize(h->st));
    return MGRIT_OK;
  }
  Stencil step = erk_step_stencil(h->prm.order_p, h->prm.rk_order_q, h->prm.cfl);
  // cluster size: power of two <= 16 dividing nx with >= 256 points per CTA
  int C = 1;
  while (C < 16 && nx % (2 * C) == 0 && nx / (2 * C) >= 256) C *= 2;
  int64_t npc = nx / C;
  // passes of Phi^B: B <= 64, halo within one neighbour, taps <= kSeqMaxTaps,
  // and B | every when a trajectory is requested
  int B = 1;
  for (int b = 64; b >= 1; --b) {
    if (every > 0 && every % b) continue;
    if (nsteps > 0 && b > nsteps) continue;
    int64_t hl = (int64_t)b * (-step.lo), hr = (int64_t)b * step.hi;
    if (hl > npc || hr > npc || b * (step.width() - 1) + 1 > kSeqMaxTaps) continue;
    B = b;
    break;
  }
  std::unique_ptr<SeqParams> sp(new SeqParams());
  std::memset((void*)sp.get(), 0, sizeof(SeqParams));
  Stencil SB = stencil_power(step, B);
  sp->nx = nx;
  sp->npc = (int)npc;
  sp->halo_l = -SB.lo;
  sp->halo_r = SB.hi;
  sp->lo = SB.lo;
  sp->ntaps = SB.width();
  for (int i = 0; i < SB.width(); ++i) sp->taps[i] = SB.a[i];
  sp->passes = nsteps / B;
  sp->tail_passes = (int)(nsteps % B);
  sp->tail_lo = step.lo;
  sp->tail_ntaps = step.width();
  if (step.width() > 64) return MGRIT_ERR_UNSUPPORTED;
  for (int i = 0; i < step.width(); ++i) sp->tail_taps[i] = step.a[i];
  sp->every_passes = (every > 0 && traj) ? (int)(every / B) : 0;
  sp->traj = (every > 0) ? traj : nullptr;
  size_t smem = 2 * sizeof(double) * (size_t)(sp->halo_l + npc + sp->halo_r);
  if (smem > 227 * 1024) return MGRIT_ERR_UNSUPPORTED;
  int Cmax = seq_max_cluster(C, smem);
  while (C > Cmax) {
    C /= 2;
    npc = nx / C;
    sp->npc = (int)npc;
    smem = 2 * sizeof(double) * (size_t)(sp->halo_l + npc + sp->halo_r);
    if (smem > 227 * 1024) return MGRIT_ERR_UNSUPPORTED;
  }
  sp->csize = C;
  const size_t row = sizeof(double) * (size_t)nx;
  double* din = h->du0;
  int rc = copy_any(din, u0, row, h->st);
  if (rc) return rc;
  bool out_dev = is_device_ptr(u_out);
  double* dout = out_dev ? u_out : h->lev[0].uC[1 - h->lev[0].cur];  // scratch row when host
  sp->u0 = din;
  sp->u_out = dout;
  {
    ProfScope ps(h, 3, 2.0 * (double)nx * ((double)sp->passes * sp->ntaps + (double)sp->tail_passes * sp->tail_ntaps));
    if (launch_seq(*sp, h->st) != 0) return MGRIT_ERR_CUDA;
  }
  ++h->launches;
  if ((rc = check_launch())) return rc;
  if (!out_dev) {
    rc = copy_any(u_out, dout, row, h->st);
    if (rc) return rc;
  }
  if (sync) CUDA_TRY(cudaStreamSynchronize(h->st));
  return MGRIT_OK;
}

int mgrit_output_all(mgrit_handle* h, double* d_all) {
  if (!h || !d_all || !is_device_ptr(d_all)) return MGRIT_ERR_INVALID_ARG;
  if (!h->have_initial) return MGRIT_ERR_INVALID_ARG;
  LevelData& L0 = h->lev[0];
  const double* cpts = L0.uC[L0.cur];
  const int64_t nx = h->nx, K = L0.K, m = h->m;
  if (h->sdirk) {
    // F-relaxation in the step kernel's FOUT mode: C-point k into row k m,
    // the m - 1 steps after it into the following rows (RHS zero)
    CUDA_TRY(cudaMemsetAsync(d_all, 0, sizeof(double) * (size_t)nx * (size_t)(K * m + 1), h->st));
    SdirkParams<double> sp = *h->sd0;
    sp.mode = kModeFOUT;
    sp.zero_start = 0;
    sp.start = cpts;
    sp.out = nullptr;
    sp.sub = nullptr;
    sp.rhs = nullptr;
    sp.g = d_all;
    sp.m = (int)m;
    sp.nsteps = (int)(m - 1);
    sp.K = K;
    sp.partial = nullptr;
    sp.traj = nullptr;
    sp.every = 0;
    if (launch_sdirk(sp, h->st) < 0) return MGRIT_ERR_UNSUPPORTED;
    ++h->launches;
    if (int rc = check_launch()) return rc;
  } else {
    // C-points into rows k m, then F-point j of every interval at once: one
    // step of the fine stencil on the rows k m + j - 1 (row stride m n_x)
    CUDA_TRY(cudaMemcpy2DAsync(d_all, sizeof(double) * (size_t)(m * nx), cpts, sizeof(double) * (size_t)nx,
                               sizeof(double) * (size_t)nx, (size_t)(K + 1), cudaMemcpyDeviceToDevice, h->st));
    for (int64_t j = 1; j < m; ++j) {
      StencilParams<double> sp = *h->fine1;
      sp.in = d_all + (j - 1) * nx;
      sp.out = d_all + j * nx;
      sp.rhs = nullptr;
      sp.sub = nullptr;
      sp.partial = nullptr;
      sp.rows = K;
      sp.ld = m * nx;
      launch_stencil_rows(sp, h->st);
      ++h->launches;
      if (int rc = check_launch()) return rc;
    }
  }
  CUDA_TRY(cudaStreamSynchronize(h->st));
  return MGRIT_OK;
}

int mgrit_level_info(const mgrit_handle* h, int level, double out[8]) {
  if (!h || level < 0 || level >= h->L || !out) return MGRIT_ERR_INVALID_ARG;
  for (int i = 0; i < 8; ++i) out[i] = 0.0;
  const LevelData& Lv = h->lev[level];
  out[0] = (double)Lv.N;
  if (level == 0) {
    if (h->sdirk && h->seg0) {
      out[4] = 2.0;  // the segmented kernel runs CF / FRES / APPLY
      out[6] = (double)kSegPoints;
      out[7] = 1.0;
    } else if (h->sdirk) {
      out[6] = (double)h->sd0->P;
      out[7] = (double)h->sd0->csize;
    }
    if (h->sdirk) {
      out[5] = h->seg0f ? 1.0 : 0.0;  // MIXED: the FP32 segmented stage kernel runs
    } else {
      out[5] = (double)h->fineM->ntaps;
      out[4] = (double)h->fineM->persistent;
      const int64_t nx = h->nx;  // untuned: the kernel's own choice by n_x
      out[6] = (double)(h->fineM->tile_r > 0 ? h->fineM->tile_r : nx >= 1024 ? 4 : nx >= 512 ? 2 : 1);
    }
    return MGRIT_OK;
  }
  out[1] = (double)Lv.kshift;
  out[2] = Lv.eps;
  out[3] = Lv.phi;
  out[4] = Lv.phi_q;
  out[5] = (double)Lv.tstep;
  out[6] = (double)(Lv.redisc ? Lv.rd->P : Lv.cp.P);
  out[7] = (double)(Lv.redisc ? Lv.rd->csize : Lv.cp.csize);
  return MGRIT_OK;
}

int mgrit_gmres_stats(mgrit_handle* h, int level, int64_t out[2]) {
  if (!h || level < 1 || level >= h->L || !out) return MGRIT_ERR_INVALID_ARG;
  out[0] = out[1] = 0;
  const LevelData& Lv = h->lev[level];
  if (!Lv.gm_stats) return MGRIT_OK;
  unsigned long long v[2] = {0, 0};
  CUDA_TRY(cudaMemcpyAsync(v, Lv.gm_stats, sizeof(v), cudaMemcpyDeviceToHost, h->st));
  CUDA_TRY(cudaStreamSynchronize(h->st));
  out[0] = (int64_t)v[0];
  out[1] = (int64_t)v[1];
  return MGRIT_OK;
}


// Everything a graph-resident solve needs before its graph runs, enqueued
// on st: the initial iterate (u0 and the random C-points, or the one already
// set) and the device stop-test state.
// u0 (n_x values, host or device) and the random initial iterate into level
// 0, queued on st
static int stage_u0(mgrit_handle* h, const double* u0, cudaStream_t st) {
  LevelData& L0 = h->lev[0];
  const size_t row = sizeof(double) * (size_t)h->nx;
  int rc = copy_any(h->du0, u0, row, st);
  if (rc) return rc;
  launch_random_cpoints(L0.uC[0], h->du0, L0.K + 1, h->nx, h->m, h->prm.seed, st);
  ++h->launches;
  CUDA_TRY(cudaMemcpyAsync(L0.uC[1], h->du0, row, cudaMemcpyDeviceToDevice, st));
  L0.cur = 0;
  h->have_initial = true;
  return MGRIT_OK;
}

// The initial condition for the next mgrit_solve_async(h, NULL), queued on
// the handle's stream; from device or pinned host memory nothing waits.
int solve_stage_initial(mgrit_handle* h, const double* u0) {
  if (!h || !u0 || h->graph_pending) return MGRIT_ERR_INVALID_ARG;
  int rc = stage_u0(h, u0, h->st);
  if (rc) return rc;
  return check_launch();
}

static int solve_begin(mgrit_handle* h, const double* u0, cudaStream_t st) {
  int rc;
  if (u0) {
    if ((rc = stage_u0(h, u0, st))) return rc;
  } else if (!h->have_initial) {
    return MGRIT_ERR_INVALID_ARG;
  }
  DevSolveState init;
  std::memset(&init, 0, sizeof(init));
  init.tol = h->prm.tol;
  init.max_iter = h->prm.max_iter;
  init.in_base = h->inner_tol;
  init.in_max = kInnerMax;
  *h->hstate = init;
  CUDA_TRY(cudaMemcpyAsync(h->dstate, h->hstate, sizeof(DevSolveState), cudaMemcpyHostToDevice, st));
  return MGRIT_OK;
}

int mgrit_solve_async(mgrit_handle* h, const double* u0) {
  if (!h || h->graph_pending) return MGRIT_ERR_INVALID_ARG;
  int rc = build_solve_graph(h);
  if (rc) return rc;
  if ((rc = solve_begin(h, u0, h->st))) return rc;
  CUDA_TRY(cudaGraphLaunch(h->gexec, h->st));
  CUDA_TRY(cudaMemcpyAsync(h->hstate, h->dstate, sizeof(DevSolveState), cudaMemcpyDeviceToHost, h->st));
  CUDA_TRY(cudaEventRecord(h->done, h->st));
  h->graph_pending = true;
  h->lev[0].cur = h->graph_cur;
  return MGRIT_OK;
}

int mgrit_solve_query(mgrit_handle* h) {
  if (!h || !h->graph_pending) return MGRIT_ERR_INVALID_ARG;
  cudaError_t e = cudaEventQuery(h->done);
  if (e == cudaSuccess) return MGRIT_OK;
  if (e == cudaErrorNotReady) return 1;
  return MGRIT_ERR_CUDA;
}

static void fill_solve_stats(const mgrit_handle* h, const DevSolveState& s, mgrit_stats* stats);

int mgrit_solve_wait(mgrit_handle* h, double* u_out, mgrit_stats* stats) {
  if (!h || !h->graph_pending) return MGRIT_ERR_INVALID_ARG;
  CUDA_TRY(cudaEventSynchronize(h->done));
  h->graph_pending = false;
  const DevSolveState& s = *h->hstate;
  int rc;
  if (u_out) {
    LevelData& L0 = h->lev[0];
    if ((rc = copy_any(u_out, L0.uC[L0.cur], sizeof(double) * (size_t)h->nx * (L0.K + 1), h->st))) return rc;
    CUDA_TRY(cudaStreamSynchronize(h->st));
  }
  fill_solve_stats(h, s, stats);
  return s.status;
}

static void fill_solve_stats(const mgrit_handle* h, const DevSolveState& s, mgrit_stats* stats) {
  if (stats) {
    std::memset(stats, 0, sizeof(*stats));
    stats->iterations = s.it;
    stats->converged = s.converged;
    stats->levels = h->L;
    stats->history_len = std::min(s.hist_len, MGRIT_MAX_HISTORY);
    for (int i = 0; i < stats->history_len; ++i) stats->rnorm_history[i] = s.hist[i];
    stats->rnorm0 = s.r0;
    stats->rnorm = s.rnorm;
    if (stats->history_len >= 2 && s.hist[stats->history_len - 2] > 0)
      stats->conv_factor = s.hist[stats->history_len - 1] / s.hist[stats->history_len - 2];
    if (h->mixed) {
      stats->outer_iterations = s.it;
      stats->inner_cycles = h->prm.inner_cycles > 0 ? s.it * h->prm.inner_cycles : s.in_total;
    }
  }
}


int mgrit_solve_wait_for(mgrit_handle* h, double timeout_s, double* u_out, mgrit_stats* stats) {
  if (!h || !h->graph_pending || !(timeout_s >= 0.0)) return MGRIT_ERR_INVALID_ARG;
  const auto t0 = std::chrono::steady_clock::now();
  while (true) {
    const cudaError_t e = cudaEventQuery(h->done);
    if (e == cudaSuccess) break;
    if (e != cudaErrorNotReady) {
      note_cuda_error("cudaEventQuery", e);
      return MGRIT_ERR_CUDA;
    }
    if (std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() >= timeout_s)
      return MGRIT_ERR_TIMEOUT;  // still in flight: wait again later
    std::this_thread::sleep_for(std::chrono::microseconds(100));
  }
  return mgrit_solve_wait(h, u_out, stats);
}

int64_t mgrit_launch_count(const mgrit_handle* h) { return h ? h->launches : 0; }

int mgrit_profile(mgrit_handle* h, int enable) {
  if (!h) return MGRIT_ERR_INVALID_ARG;
  CUDA_TRY(cudaStreamSynchronize(h->st));
  for (int c = 0; c < kProfCats; ++c) {
    for (auto& pr : h->prof.ev[c]) {
      h->prof.pool.push_back(pr.first);
      h->prof.pool.push_back(pr.second);
    }
    h->prof.ev[c].clear();
    h->prof.flops[c] = 0.0;
    h->prof.count[c] = 0;
  }
  h->prof.on = enable != 0;
  return MGRIT_OK;
}

int mgrit_profile_read(mgrit_handle* h, double out[60]) {
  if (!h || !out) return MGRIT_ERR_INVALID_ARG;
  CUDA_TRY(cudaStreamSynchronize(h->st));
  for (int c = 0; c < kProfCats; ++c) {
    double ms = 0.0;
    for (auto& pr : h->prof.ev[c]) {
      float t = 0.f;
      CUDA_TRY(cudaEventElapsedTime(&t, pr.first, pr.second));
      ms += t;
    }
    out[c * 3 + 0] = (double)h->prof.count[c];
    out[c * 3 + 1] = ms;
    out[c * 3 + 2] = h->prof.flops[c];
  }
  return MGRIT_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// One CUDA graph for a batch of solves (graph_batch.h)
// ---------------------------------------------------------------------------
int batch_graph_build(mgrit_handle* const* hs, int64_t n, cudaGraphExec_t* out) {
  *out = nullptr;
  cudaGraph_t g = nullptr;
  if (cudaGraphCreate(&g, 0) != cudaSuccess) {
    note_cuda_error("cudaGraphCreate", cudaGetLastError());
    return MGRIT_ERR_CUDA;
  }
  int rc = MGRIT_OK;
  for (int64_t i = 0; i < n && !rc; ++i) rc = capture_solve(hs[i], g);
  if (!rc && cudaGraphInstantiate(out, g, 0) != cudaSuccess) {
    note_cuda_error("cudaGraphInstantiate", cudaGetLastError());
    rc = MGRIT_ERR_CUDA;
  }
  cudaGraphDestroy(g);
  return rc;
}

int batch_graph_run(mgrit_handle* const* hs, int64_t n, const double* const* u0s, cudaGraphExec_t ge,
                    cudaStream_t st) {
  int rc;
  for (int64_t i = 0; i < n; ++i)
    if ((rc = solve_begin(hs[i], u0s[i], st))) return rc;
  CUDA_TRY(cudaGraphLaunch(ge, st));
  for (int64_t i = 0; i < n; ++i) {
    mgrit_handle* h = hs[i];
    CUDA_TRY(cudaMemcpyAsync(h->hstate, h->dstate, sizeof(DevSolveState), cudaMemcpyDeviceToHost, st));
    h->lev[0].cur = h->graph_cur;
  }
  CUDA_TRY(cudaStreamSynchronize(st));
  return MGRIT_OK;
}

int batch_graph_stats(const mgrit_handle* h, mgrit_stats* stats) {
  fill_solve_stats(h, *h->hstate, stats);
  return h->hstate->status;
}
