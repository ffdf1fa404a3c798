// Batched and served MGRIT solves (host-side scheduling in C++).
//
// Every solve is a graph-resident MGRIT solve (iteration loop and stop test
// on the device).  A batch captures all its solves into one CUDA graph, one
// independent branch per solve, and runs them with one graph launch, so
// kernels of different solves share the GPU; the server admits requests of
// a Poisson stream as device memory (an HBM budget) and in-flight slots
// free up (one graph launch per request, mgrit_solve_async), and records
// arrival-to-completion latency per request.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include "../../include/mgrit.h"
#include "graph_batch.h"

namespace {

constexpr size_t kAdmitWindow = 64;  // pending requests considered per admission
constexpr double kMaxSkipS = 2.0;    // wait after which the oldest request is not overtaken

// coarsening factor from level l to level l+1
int factor_of(const mgrit_params& p, int64_t l) { return (l == 0 || p.m_coarse <= 0) ? p.m : p.m_coarse; }

int64_t levels_of(const mgrit_params& p) {
  if (p.levels > 0) return p.levels;
  int64_t L = 1, N = p.nt;
  while (N % factor_of(p, L - 1) == 0 && N / factor_of(p, L - 1) >= 2) {
    N /= factor_of(p, L - 1);
    ++L;
  }
  return std::max<int64_t>(L, 2);
}

}  // namespace

// Device bytes a solve with these parameters allocates (C-point and RHS
// buffers of every level, FP64 plus the FP32 copies of MIXED), used for
// admission against the HBM budget.
extern "C" int64_t mgrit_estimate_bytes(const mgrit_params* p) {
  if (!p || p->nx <= 0 || p->nt <= 0 || p->m < 2) return -1;
  const int64_t L = levels_of(*p);
  int64_t rows = 0, N = p->nt;
  const int64_t gm_it = p->coarse_solve == MGRIT_SOLVE_GMRES ? (p->gmres_maxit > 0 ? p->gmres_maxit : 20) : -1;
  for (int64_t l = 0; l < L; ++l) {
    const int64_t f = factor_of(*p, l);
    int64_t K = (l < L - 1) ? N / f : 0;
    if (l < L - 1) rows += 2 * (K + 1);  // C-point double buffer
    if (l >= 1) rows += N + 1;           // RHS
    if (l >= 1 && gm_it > 0) rows += std::max<int64_t>(K, 1) * (gm_it + 1);  // GMRES Krylov basis
    N /= f;
  }
  int64_t bytes = rows * p->nx * 8;
  if (p->precision == MGRIT_MIXED || p->precision == MGRIT_MIXED_FAST) bytes += rows * p->nx * 4 + (N + 2) * p->nx * 8;
  return bytes + (4 << 20);
}

struct mgrit_batch {
  std::vector<mgrit_handle*> hs;
  std::vector<cudaStream_t> streams;
  std::vector<mgrit_params> prm;
  cudaGraphExec_t ge = nullptr;  // every solve of the batch in one graph (built at the first solve)
};

extern "C" int mgrit_batch_destroy(mgrit_batch* b) {
  if (!b) return MGRIT_OK;
  if (b->ge) cudaGraphExecDestroy(b->ge);
  for (auto h : b->hs) mgrit_destroy(h);
  for (auto s : b->streams) cudaStreamDestroy(s);
  delete b;
  return MGRIT_OK;
}

extern "C" int mgrit_batch_create(const mgrit_params* params, int64_t count, int nstreams, mgrit_batch** out) {
  if (!params || count <= 0 || !out || nstreams <= 0) return MGRIT_ERR_INVALID_ARG;
  *out = nullptr;
  mgrit_batch* b = new mgrit_batch();
  for (int i = 0; i < nstreams; ++i) {
    cudaStream_t s;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
      mgrit_batch_destroy(b);
      return MGRIT_ERR_CUDA;
    }
    b->streams.push_back(s);
  }
  for (int64_t i = 0; i < count; ++i) {
    mgrit_handle* h = nullptr;
    int rc = mgrit_setup(&params[i], (void*)b->streams[i % nstreams], &h);
    if (rc) {
      mgrit_batch_destroy(b);
      return rc;
    }
    b->hs.push_back(h);
    b->prm.push_back(params[i]);
  }
  *out = b;
  return MGRIT_OK;
}

extern "C" int mgrit_batch_solve(mgrit_batch* b, const double* const* u0s, mgrit_stats* stats) {
  if (!b || !u0s) return MGRIT_ERR_INVALID_ARG;
  const int64_t n = (int64_t)b->hs.size();
  int rc;
  if (!b->ge && (rc = batch_graph_build(b->hs.data(), n, &b->ge))) return rc;
  if ((rc = batch_graph_run(b->hs.data(), n, u0s, b->ge, b->streams[0]))) return rc;
  int worst = MGRIT_OK;
  for (int64_t i = 0; i < n; ++i) {
    rc = batch_graph_stats(b->hs[i], stats ? &stats[i] : nullptr);
    if (rc && !worst) worst = rc;
  }
  return worst;
}

extern "C" int mgrit_batch_get(mgrit_batch* b, int64_t i, double* u_out) {
  if (!b || i < 0 || i >= (int64_t)b->hs.size() || !u_out) return MGRIT_ERR_INVALID_ARG;
  const mgrit_params& p = b->prm[i];
  // the C-point iterate of level 0
  return mgrit_level_io(b->hs[i], 0, 0, u_out, 0, nullptr);
}

extern "C" int mgrit_batch_sequential(mgrit_batch* b, const double* const* d_u0s, double* const* d_outs) {
  if (!b || !d_u0s || !d_outs) return MGRIT_ERR_INVALID_ARG;
  for (size_t i = 0; i < b->hs.size(); ++i) {
    int rc = mgrit_fine_propagate_async(b->hs[i], d_u0s[i], d_outs[i], b->prm[i].nt);
    if (rc) return rc;
  }
  for (auto s : b->streams)
    if (cudaStreamSynchronize(s) != cudaSuccess) return MGRIT_ERR_CUDA;
  return MGRIT_OK;
}

extern "C" int64_t mgrit_batch_dof(const mgrit_batch* b) {
  if (!b) return 0;
  int64_t s = 0;
  for (auto& p : b->prm) s += p.nx * p.nt;
  return s;
}

// ---------------------------------------------------------------------------
// server
//
// Two host threads.  The serving thread admits requests (slot and memory
// budget), launches prepared solves and collects finished ones; a setup
// worker builds each admitted request's hierarchy and solve graph
// (mgrit_setup, graph capture and instantiation), so no setup holds up a
// launch or the collection of a finished solve.  Neither thread times
// launch candidates.
// ---------------------------------------------------------------------------
namespace {

struct SetupJob {
  int slot;
  int64_t req;
};
struct SetupDone {
  int slot;
  int64_t req;
  mgrit_handle* h;
  int rc;
  double secs;
};

class SetupWorker {
 public:
  // stage: pinned host memory of stage_len doubles per slot, through which
  // an initial condition in pageable memory reaches the device
  SetupWorker(const mgrit_params* params, const double* const* u0s, const std::vector<cudaStream_t>* pool,
              double* stage, int64_t stage_len, int device)
      : params_(params), u0s_(u0s), pool_(pool), stage_(stage), stage_len_(stage_len), device_(device),
        th_([this] { run(); }) {}
  ~SetupWorker() {
    {
      std::lock_guard<std::mutex> lk(mu_);
      stop_ = true;
    }
    cv_.notify_all();
    th_.join();
  }
  void submit(int slot, int64_t req) {
    {
      std::lock_guard<std::mutex> lk(mu_);
      jobs_.push_back(SetupJob{slot, req});
    }
    cv_.notify_all();
  }
  // finished setups (moved out)
  std::vector<SetupDone> take() {
    std::lock_guard<std::mutex> lk(mu_);
    std::vector<SetupDone> out;
    out.swap(done_);
    return out;
  }
  bool idle() {
    std::lock_guard<std::mutex> lk(mu_);
    return jobs_.empty() && !busy_;
  }

 private:
  // u0 as it can be copied without waiting: device or pinned memory as
  // given, pageable memory through the slot's pinned stage
  const double* stage_u0(int slot, int64_t req) {
    const double* u0 = u0s_[req];
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, u0) == cudaSuccess && a.type != cudaMemoryTypeUnregistered) return u0;
    cudaGetLastError();
    double* dst = stage_ + (size_t)slot * (size_t)stage_len_;
    std::memcpy(dst, u0, sizeof(double) * (size_t)params_[req].nx);
    return dst;
  }
  void run() {
    cudaSetDevice(device_);
    set_measured_tuning(false);
    // setup, capture and the initial condition only queue device work on
    // the slot's stream: nothing here waits behind the running solves
    set_setup_nowait(true);
    for (;;) {
      SetupJob j;
      {
        std::unique_lock<std::mutex> lk(mu_);
        cv_.wait(lk, [this] { return stop_ || !jobs_.empty(); });
        if (jobs_.empty()) return;  // stop requested and nothing left
        j = jobs_.front();
        jobs_.pop_front();
        busy_ = true;
      }
      const auto t0 = std::chrono::steady_clock::now();
      mgrit_handle* h = nullptr;
      int rc = mgrit_setup(&params_[j.req], (void*)(*pool_)[j.slot], &h);
      if (rc == MGRIT_OK) rc = solve_graph_prepare(h);
      if (rc == MGRIT_OK) rc = solve_stage_initial(h, stage_u0(j.slot, j.req));
      const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
      std::lock_guard<std::mutex> lk(mu_);
      done_.push_back(SetupDone{j.slot, j.req, h, rc, secs});
      busy_ = false;
    }
  }
  const mgrit_params* params_;
  const double* const* u0s_;
  const std::vector<cudaStream_t>* pool_;
  double* stage_;
  int64_t stage_len_;
  int device_;
  std::mutex mu_;
  std::condition_variable cv_;
  std::deque<SetupJob> jobs_;
  std::vector<SetupDone> done_;
  bool busy_ = false;
  bool stop_ = false;
  std::thread th_;
};

}  // namespace

extern "C" int mgrit_serve(const mgrit_params* params, const double* const* u0s, double* const* u_outs,
                           const double* arrival_s, int64_t count, int64_t hbm_budget_bytes, int max_inflight,
                           double time_limit_s, mgrit_request_result* results, mgrit_serve_stats* st) {
  if (!params || !u0s || !arrival_s || count < 0 || max_inflight <= 0 || !results) return MGRIT_ERR_INVALID_ARG;
  for (int64_t i = 1; i < count; ++i)
    if (arrival_s[i] < arrival_s[i - 1]) return MGRIT_ERR_INVALID_ARG;
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess) return MGRIT_ERR_CUDA;
  int64_t max_nx = 1;
  for (int64_t i = 0; i < count; ++i) max_nx = std::max<int64_t>(max_nx, params[i].nx);
  double* stage = nullptr;
  if (cudaMallocHost((void**)&stage, sizeof(double) * (size_t)max_nx * (size_t)max_inflight) != cudaSuccess) {
    cudaGetLastError();
    return MGRIT_ERR_OOM;
  }
  std::vector<cudaStream_t> pool;
  for (int i = 0; i < max_inflight; ++i) {
    cudaStream_t s;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
      for (auto q : pool) cudaStreamDestroy(q);
      cudaFreeHost(stage);
      return MGRIT_ERR_CUDA;
    }
    pool.push_back(s);
  }
  // slot states: free, setting up (the worker holds it), running
  enum { kFree = 0, kSetup = 1, kRunning = 2 };
  struct Slot {
    int state = kFree;
    mgrit_handle* h = nullptr;
    int64_t req = -1;
    int64_t bytes = 0;
  };
  std::vector<Slot> slots(max_inflight);
  std::deque<int64_t> pending;
  for (int64_t i = 0; i < count; ++i) {
    std::memset(&results[i], 0, sizeof(results[i]));
    results[i].status = 1;  // not started
  }
  mgrit_serve_stats S;
  std::memset(&S, 0, sizeof(S));
  const auto t0 = std::chrono::steady_clock::now();
  auto now = [&]() { return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count(); };
  int64_t next = 0, finished = 0, mem = 0;
  int rc_fatal = MGRIT_OK;
  auto finish = [&](Slot& sl, int rc, const mgrit_stats* ms) {
    mgrit_request_result& r = results[sl.req];
    r.finish_s = now();
    r.latency_ms = (r.finish_s - arrival_s[sl.req]) * 1e3;
    r.iterations = ms ? ms->iterations : 0;
    r.status = rc;
    if (rc == MGRIT_OK) {
      ++S.completed;
      S.dof_completed += (double)params[sl.req].nx * (double)params[sl.req].nt;
    } else {
      ++S.failed;
    }
    if (sl.h) mgrit_destroy(sl.h);
    mem -= sl.bytes;
    sl = Slot();
    ++finished;
    if (rc == MGRIT_ERR_CUDA) rc_fatal = rc;
  };
  {
    SetupWorker worker(params, u0s, &pool, stage, max_nx, device);
    while (finished < count) {
      const double t = now();
      if (t > time_limit_s) break;
      while (next < count && arrival_s[next] <= t) pending.push_back(next++);
      S.max_backlog = std::max<int64_t>(S.max_backlog, (int64_t)pending.size());
      bool progress = false;
      // prepared solves: launch
      for (auto& d : worker.take()) {
        Slot& sl = slots[d.slot];
        sl.h = d.h;
        S.setup_s += d.secs;
        int rc = d.rc;
        if (rc == MGRIT_OK) rc = mgrit_solve_async(sl.h, nullptr);  // u0 staged by the worker
        if (rc) {
          finish(sl, rc, nullptr);
        } else {
          sl.state = kRunning;
          results[sl.req].start_s = now();
        }
        progress = true;
      }
      // completions
      for (auto& sl : slots) {
        if (sl.state != kRunning) continue;
        if (mgrit_solve_query(sl.h) == 1) continue;
        mgrit_stats ms;
        int rc = mgrit_solve_wait(sl.h, u_outs ? u_outs[sl.req] : nullptr, &ms);
        finish(sl, rc, &ms);
        progress = true;
      }
      if (rc_fatal) break;
      // admissions: first fit among the oldest kAdmitWindow pending requests
      // (a request that does not fit in the free budget does not block
      // smaller ones behind it), except that once the oldest has waited
      // kMaxSkipS seconds nothing overtakes it until it fits (no
      // starvation); a request larger than the whole budget is rejected
      while (!pending.empty()) {
        auto free_slot = std::find_if(slots.begin(), slots.end(), [](const Slot& s) { return s.state == kFree; });
        if (free_slot == slots.end()) break;
        const bool head_starving = (now() - arrival_s[pending.front()]) > kMaxSkipS;
        int64_t pick = -1;
        size_t pos = 0;
        for (size_t w = 0; w < pending.size() && w < kAdmitWindow; ++w) {
          const int64_t req = pending[w];
          const int64_t need = mgrit_estimate_bytes(&params[req]);
          if (need > hbm_budget_bytes) {
            results[req].status = MGRIT_ERR_OOM;
            ++S.rejected;
            ++finished;
            pending.erase(pending.begin() + (std::ptrdiff_t)w);
            pick = -2;
            break;
          }
          if (mem + need <= hbm_budget_bytes) {
            pick = req;
            pos = w;
            break;
          }
          if (head_starving) break;
        }
        if (pick == -2) continue;
        if (pick < 0) break;
        const int64_t need = mgrit_estimate_bytes(&params[pick]);
        Slot& sl = *free_slot;
        sl.state = kSetup;
        sl.req = pick;
        sl.bytes = need;
        mem += need;
        S.max_mem_bytes = std::max(S.max_mem_bytes, mem);
        ++S.admitted;
        pending.erase(pending.begin() + (std::ptrdiff_t)pos);
        worker.submit((int)(free_slot - slots.begin()), pick);
        progress = true;
      }
      int inflight = 0;
      for (auto& sl : slots) inflight += sl.state != kFree;
      S.max_inflight = std::max(S.max_inflight, inflight);
      // idle: wait a millisecond (solves take far longer; polling every
      // running solve in a tight loop would contend with the setup
      // worker's CUDA calls)
      if (!progress) std::this_thread::sleep_for(std::chrono::milliseconds(1));
    }
    // the worker's remaining setups finish (its destructor waits); their
    // solves are launched and drained below
    while (!worker.idle()) std::this_thread::sleep_for(std::chrono::microseconds(200));
    for (auto& d : worker.take()) {
      Slot& sl = slots[d.slot];
      sl.h = d.h;
      S.setup_s += d.secs;
      int rc = d.rc;
      if (rc == MGRIT_OK) rc = mgrit_solve_async(sl.h, nullptr);  // u0 staged by the worker
      if (rc) {
        finish(sl, rc, nullptr);
      } else {
        sl.state = kRunning;
        results[sl.req].start_s = now();
      }
    }
  }
  // drain whatever is still running at the time limit
  for (auto& sl : slots) {
    if (sl.state != kRunning) continue;
    mgrit_stats ms;
    int rc = mgrit_solve_wait(sl.h, u_outs ? u_outs[sl.req] : nullptr, &ms);
    finish(sl, rc, &ms);
  }
  S.arrived = next;
  S.backlog_end = (int64_t)pending.size() + (count - next);
  S.wall_s = now();
  for (auto q : pool) cudaStreamDestroy(q);
  cudaFreeHost(stage);  // after every queued copy from it (this synchronises)
  if (st) *st = S;
  return rc_fatal;
}
