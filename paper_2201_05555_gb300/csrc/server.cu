// Serving loop for parametric reduced solves, and checkpoint export/import.
//
// A query names a family of initial data, one parameter record per sample,
// the sizes (N, p, Nx, n_max), the time step, the number of steps and the
// arithmetic.  Queries wait in a FIFO; an admission thread admits them while
// both a slot and the HBM budget are free.  Every admitted query runs on its
// own context, CUDA stream and host thread, so steps of concurrent queries
// overlap on the device; a finished query frees its slot and its memory and
// the next waiting query is admitted.  A query's work on the device:
// particles (load.cu: quiet start or Philox-seeded), the truncated complex SVD start with n
// chosen from the singular values, then the partitioned RK2 steps (FP64,
// double-float or FP32 row work) in chunks, with the energy trace and the
// final coefficients copied to the caller's host buffers.  All kernels are
// deterministic, so a query's result does not depend on what runs beside it.
#include "vp_internal.cuh"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <memory>
#include <thread>
#include <unordered_map>
#include <vector>

namespace {

using Clock = std::chrono::steady_clock;

struct Job {
  vp_query q;
  std::vector<double> eta;
  size_t bytes = 0;    // own buffers
  size_t ws = 0;       // workspace arena it needs (with the arena's growth margin)
  size_t charged = 0;  // bytes added to the server's count at admission
  vp_result res{};
  bool done = false;
  bool cancel = false;
  std::thread th;
};

double family_k(int family) { return family == 1 ? 0.2 : 0.5; }

// Device bytes of a query's own buffers (particles, state, trace), with the
// pool's 2 MiB granularity per allocation.
size_t job_buffer_bytes(const vp_query& q) {
  const size_t N = (size_t)q.N, p = (size_t)q.p, n2 = 2 * (size_t)q.n_max;
  return 2 * p * N * 8 + N * n2 * 8 + 2 * n2 * p * 8 + (size_t)q.nsteps * p * 20 + p * 32 +
         9 * ((size_t)2 << 20);
}

}  // namespace

struct Slot {
  vp_ctx* ctx = nullptr;
  cudaStream_t st = nullptr;
  bool busy = false;
  size_t held = 0;  // workspace arena the slot's context keeps between queries
};

struct vp_server {
  int device = 0;
  size_t budget = 0;
  int max_slots = 1;
  cudaMemPool_t pool = nullptr;  // stream-ordered pool: no device-wide sync per query
  std::vector<Slot> slots;
  std::mutex mu;
  std::condition_variable cv_admit, cv_done;
  std::deque<uint64_t> pending;
  std::unordered_map<uint64_t, std::unique_ptr<Job>> jobs;
  size_t used = 0;  // arenas held by all slots + buffers and arena growth of running queries
  int active = 0;
  bool stopping = false;
  uint64_t next_ticket = 1;
  int64_t submitted = 0, completed = 0;
  bool wake = false;
  Clock::time_point t0 = Clock::now();
  std::thread admitter;

  double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
  void admit_loop();
  void run(Job* j, Slot* sl);
};

void vp_server::run(Job* j, Slot* sl) {
  const vp_query& q = j->q;
  vp_result& r = j->res;
  vp_status s = VP_OK;
  vp_ctx* ctx = sl->ctx;
  cudaStream_t st = sl->st;
  double *X = nullptr, *V = nullptr, *Q = nullptr, *Z = nullptr, *K = nullptr, *tr = nullptr,
         *eta = nullptr, *sig = nullptr;
  int32_t* its = nullptr;
  const int64_t N = q.N;
  const int p = q.p;
  int n = q.n_max;
  auto fail = [&](vp_status code) {
    if (s == VP_OK) s = code;
  };
  auto alloc = [&](auto** ptr, size_t bytes) {
    if (s == VP_OK && cudaMallocFromPoolAsync((void**)ptr, bytes, pool, st) != cudaSuccess) {
      *ptr = nullptr;
      fail(VP_ENOMEM);
    }
  };
  cudaSetDevice(device);
  const size_t n2 = 2 * (size_t)q.n_max;
  alloc(&X, sizeof(double) * p * N);
  alloc(&V, sizeof(double) * p * N);
  alloc(&Q, sizeof(double) * N * n2);
  alloc(&Z, sizeof(double) * n2 * p);
  alloc(&K, sizeof(double) * n2 * p);
  alloc(&tr, sizeof(double) * q.nsteps * p * 2);
  alloc(&eta, sizeof(double) * 3 * p);
  alloc(&sig, sizeof(double) * p);
  alloc(&its, sizeof(int32_t) * q.nsteps);
  // start: particles, complex SVD, rank from the singular values
  if (s == VP_OK) {
    cudaMemcpyAsync(eta, j->eta.data(), sizeof(double) * 3 * p, cudaMemcpyHostToDevice, st);
    vp_status s1 = vp_load_particles(ctx, q.family, q.loading, q.seed, N, p, eta, X, V, st);
    if (s1 != VP_OK) fail(s1);
    int32_t nsel = 0;
    vp_status s2 = s1 != VP_OK ? s1
                               : vp_init_csvd_rank(ctx, N, p, q.n_min, q.n_max, q.rank_tol, X, V, Q,
                                                   Z, sig, &nsel, st);
    if (s2 != VP_OK) fail(s2);
    n = nsel;
  }
  if (s == VP_OK) {
    if (cudaStreamSynchronize(st) != cudaSuccess) fail(VP_ECUDA);
    vp_status s2 = vp_ctx_sync_status(ctx, st);
    if (s2 != VP_OK) fail(s2);
  }
  if (X) cudaFreeAsync(X, st);
  if (V) cudaFreeAsync(V, st);
  X = V = nullptr;
  {
    std::lock_guard<std::mutex> lk(mu);
    r.t_start = now();
    r.n = n;
  }
  // steps in chunks, so that a cancelled query stops between chunks
  if (s == VP_OK) {
    cudaMemsetAsync(K, 0, sizeof(double) * n2 * p, st);
    const double L = 2.0 * 3.141592653589793 / family_k(q.family);
    vp_grid grid{q.Nx, L, -L / (double)N, L / (double)N, 1.0};
    vp_step_opts o{1e-9, 100, 0, 1e-3, 1e-2, q.arith, q.arith == 2 ? 1 : 0};
    const int chunk = 16;
    for (int s0 = 0; s0 < q.nsteps && s == VP_OK; s0 += chunk) {
      {
        std::lock_guard<std::mutex> lk(mu);
        if (j->cancel) {
          fail(VP_EAGAIN);
          break;
        }
      }
      int m = std::min(chunk, q.nsteps - s0);
      vp_status s2 = vp_basis_update(ctx, &grid, N, n, p, Q, Z, q.dt, m, &o, tr + (int64_t)s0 * p * 2,
                                     its + s0, K, st);
      if (s2 != VP_OK) fail(s2);
      std::lock_guard<std::mutex> lk(mu);
      r.steps_done = s0 + m;
    }
  }
  if (s == VP_OK) {
    if (q.trace_host)
      cudaMemcpyAsync(q.trace_host, tr, sizeof(double) * q.nsteps * p * 2, cudaMemcpyDeviceToHost, st);
    if (q.zeta_host) cudaMemcpyAsync(q.zeta_host, Z, sizeof(double) * 2 * n * p, cudaMemcpyDeviceToHost, st);
    std::vector<int32_t> ih(q.nsteps);
    cudaMemcpyAsync(ih.data(), its, sizeof(int32_t) * q.nsteps, cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) fail(VP_ECUDA);
    int mx = 0;
    for (int k = 0; k < q.nsteps; ++k) mx = std::max(mx, (int)ih[k]);
    r.max_iters = mx;
    vp_status s2 = vp_ctx_sync_status(ctx, st);
    if (s2 != VP_OK) fail(s2);
  }
  for (void* ptr : {(void*)Q, (void*)Z, (void*)K, (void*)tr, (void*)eta, (void*)sig, (void*)its})
    if (ptr) cudaFreeAsync(ptr, st);
  cudaStreamSynchronize(st);
  if (s != VP_OK) vp_ctx_sync_status(ctx, st);  // clear a stale device status word
  const size_t held_now = vp_ctx_workspace_bytes(ctx);
  std::lock_guard<std::mutex> lk(mu);
  r.status = s;
  r.t_done = now();
  j->done = true;
  used = used - j->charged - sl->held + held_now;
  sl->held = held_now;
  --active;
  sl->busy = false;
  ++completed;
  wake = true;
  cv_done.notify_all();
  cv_admit.notify_all();
}

// Admission: the queue head goes to the free slot holding the largest arena,
// if its buffers plus the arena growth it needs fit in what the budget has
// left.  When they do not, and freeing the idle slots' arenas would make room,
// those are freed (a device synchronisation, so only then); otherwise the head
// waits for a running query to end.  With nothing running every arena is
// idle, so a query that fits the budget alone is always admitted.
void vp_server::admit_loop() {
  std::unique_lock<std::mutex> lk(mu);
  for (;;) {
    cv_admit.wait(lk, [&] { return stopping || (!pending.empty() && active < max_slots); });
    if (stopping) return;
    uint64_t t = pending.front();
    auto it = jobs.find(t);
    if (it == jobs.end()) {
      pending.pop_front();
      continue;
    }
    Job* j = it->second.get();
    Slot* sl = nullptr;
    size_t idle_held = 0;
    for (auto& x : slots)
      if (!x.busy) {
        idle_held += x.held;
        if (!sl || x.held > sl->held) sl = &x;
      }
    const size_t grow = j->ws > sl->held ? j->ws - sl->held : 0;
    const size_t need = j->bytes + grow;
    if (used + need > budget) {
      if (idle_held > 0 && used - idle_held + j->bytes + j->ws <= budget) {
        std::vector<Slot*> rel;
        for (auto& x : slots)
          if (!x.busy && x.held > 0) {
            x.busy = true;
            rel.push_back(&x);
          }
        lk.unlock();
        for (Slot* x : rel) vp_workspace_release(x->ctx);
        lk.lock();
        for (Slot* x : rel) {
          used -= x->held;
          x->held = 0;
          x->busy = false;
        }
        continue;
      }
      // wait for a running query to finish or the head to be cancelled, then
      // decide again (alone, a query always fits: submit checks that)
      wake = false;
      cv_admit.wait(lk, [&] { return stopping || active == 0 || wake; });
      continue;
    }
    pending.pop_front();
    sl->busy = true;
    used += need;
    j->charged = need;
    ++active;
    j->res.t_admit = now();
    j->th = std::thread([this, j, sl] { run(j, sl); });
  }
}

extern "C" {

vp_status vp_server_create(vp_server** out, int device, size_t hbm_budget, int max_slots) {
  if (!out || max_slots < 1 || max_slots > 64 || hbm_budget == 0) return VP_EINVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return VP_ECUDA;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(device);
  vp_server* s = new vp_server();
  s->device = device;
  s->budget = hbm_budget;
  s->max_slots = max_slots;
  vp_status rc = VP_OK;
  cudaMemPoolProps props{};
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = device;
  if (cudaMemPoolCreate(&s->pool, &props) != cudaSuccess) rc = VP_ECUDA;
  if (rc == VP_OK) {
    uint64_t keep = hbm_budget;  // freed blocks stay cached up to the budget
    cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  s->slots.resize(max_slots);
  for (auto& sl : s->slots) {
    if (rc != VP_OK) break;
    if (vp_ctx_create(&sl.ctx, device, hbm_budget) != VP_OK) rc = VP_ENOMEM;
    else if (cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking) != cudaSuccess) rc = VP_ECUDA;
  }
  if (rc != VP_OK) {
    for (auto& sl : s->slots) {
      if (sl.st) cudaStreamDestroy(sl.st);
      if (sl.ctx) vp_ctx_destroy(sl.ctx);
    }
    if (s->pool) cudaMemPoolDestroy(s->pool);
    delete s;
    cudaSetDevice(prev);
    return rc;
  }
  s->admitter = std::thread([s] { s->admit_loop(); });
  *out = s;
  cudaSetDevice(prev);
  return VP_OK;
}

vp_status vp_serve_submit(vp_server* s, const vp_query* q, uint64_t* ticket) {
  if (!s || !q || !ticket) return VP_EINVAL;
  if (q->family < 0 || q->family > 2 || q->loading < 0 || q->loading > 1 || q->N < 2 || q->N >= (int64_t(1) << 31) || q->p < 1 ||
      q->p > 256 || q->n_max < 1 || q->n_max > 40 || q->n_max > q->p || q->n_min < 1 ||
      q->n_min > q->n_max || q->Nx < 3 ||
      q->Nx > VP_MAX_NX || !(q->dt > 0.0) || q->nsteps < 1 || q->arith < 0 || q->arith > 2 ||
      !(q->rank_tol >= 0.0) || !q->eta)
    return VP_EINVAL;
  if ((int64_t)4 * q->n_max * q->n_max + (int64_t)2 * q->n_max * q->p > 25600) return VP_EUNSUPPORTED;
  auto j = std::make_unique<Job>();
  j->q = *q;
  j->eta.assign(q->eta, q->eta + 3 * (size_t)q->p);
  j->bytes = job_buffer_bytes(*q);
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device);
  const size_t ws = vp_query_ws_bytes(sms, q->N, q->n_max, q->p, q->Nx, q->arith);
  j->ws = ws + ws / 4;
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stopping) return VP_EBUSY;
  if (j->bytes + j->ws > s->budget) return VP_ENOMEM;
  if (s->pending.size() >= 4096) return VP_EBUSY;
  j->res.t_submit = s->now();
  j->res.status = VP_EAGAIN;
  uint64_t t = s->next_ticket++;
  s->jobs[t] = std::move(j);
  s->pending.push_back(t);
  ++s->submitted;
  *ticket = t;
  s->cv_admit.notify_all();
  return VP_OK;
}

vp_status vp_serve_poll(vp_server* s, uint64_t ticket, vp_result* res, int timeout_ms) {
  if (!s) return VP_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->jobs.find(ticket);
  if (it == s->jobs.end()) return VP_EINVAL;
  Job* j = it->second.get();
  if (!j->done) {
    if (timeout_ms <= 0) return VP_EAGAIN;
    bool ok = s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return j->done; });
    if (!ok) return VP_ETIMEDOUT;
  }
  if (res) *res = j->res;
  std::thread th = std::move(j->th);
  s->jobs.erase(it);
  lk.unlock();
  if (th.joinable()) th.join();
  return VP_OK;
}

vp_status vp_serve_cancel(vp_server* s, uint64_t ticket) {
  if (!s) return VP_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->jobs.find(ticket);
  if (it == s->jobs.end()) return VP_EINVAL;
  Job* j = it->second.get();
  auto pit = std::find(s->pending.begin(), s->pending.end(), ticket);
  if (pit != s->pending.end()) {  // not admitted yet: finished at once
    s->pending.erase(pit);
    j->done = true;
    j->res.status = VP_EAGAIN;
    j->res.t_done = s->now();
    s->wake = true;
    s->cv_done.notify_all();
    s->cv_admit.notify_all();
    return VP_OK;
  }
  j->cancel = true;
  return VP_OK;
}

vp_status vp_server_stats(vp_server* s, int64_t* submitted, int64_t* completed, int32_t* active,
                          int32_t* pending, size_t* used_bytes) {
  if (!s) return VP_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  if (submitted) *submitted = s->submitted;
  if (completed) *completed = s->completed;
  if (active) *active = s->active;
  if (pending) *pending = (int32_t)s->pending.size();
  if (used_bytes) *used_bytes = s->used;
  return VP_OK;
}

vp_status vp_server_destroy(vp_server* s, int32_t drain_timeout_ms) {
  if (!s || drain_timeout_ms < 0) return VP_EINVAL;
  // let waiting and running queries finish for up to drain_timeout_ms
  bool drained = true;
  if (drain_timeout_ms > 0) {
    std::unique_lock<std::mutex> lk(s->mu);
    drained = s->cv_done.wait_for(lk, std::chrono::milliseconds(drain_timeout_ms),
                                  [&] { return s->pending.empty() && s->active == 0; });
  }
  std::vector<std::thread> ths;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stopping = true;
    s->pending.clear();
    for (auto& kv : s->jobs) {
      kv.second->cancel = true;
      if (kv.second->th.joinable()) ths.push_back(std::move(kv.second->th));
    }
    s->cv_admit.notify_all();
  }
  if (s->admitter.joinable()) s->admitter.join();
  for (auto& t : ths) t.join();
  for (auto& sl : s->slots) {
    if (sl.st) cudaStreamDestroy(sl.st);
    if (sl.ctx) vp_ctx_destroy(sl.ctx);
  }
  if (s->pool) cudaMemPoolDestroy(s->pool);
  delete s;
  return drained ? VP_OK : VP_ETIMEDOUT;
}

// ------------------------------------------------------------- checkpoint
// Layout: a header of 8 int64 {magic, version, N, n, p, step, has_k, 0}, then
// Q (N x 2n), Z (2n x p) and, if present, the fixed-point state k (2n x p).
static const int64_t kMagic = 0x5650535441544531ll;  // "VPSTATE1"

size_t vp_state_bytes(int64_t N, int32_t n, int32_t p, int32_t with_k) {
  return 8 * sizeof(int64_t) + sizeof(double) * ((size_t)N * 2 * n + (size_t)2 * n * p * (with_k ? 2 : 1));
}

vp_status vp_state_export(vp_ctx* ctx, int64_t N, int32_t n, int32_t p, const double* Q,
                          const double* Z, const double* K, int64_t step, void* host,
                          size_t host_bytes, void* stream) {
  if (!ctx || !Q || !Z || !host || N < 1 || n < 1 || p < 1) return VP_EINVAL;
  const size_t need = vp_state_bytes(N, n, p, K != nullptr);
  if (host_bytes < need) return vp_fail(ctx, VP_EINVAL, "host buffer of %zu bytes < %zu", host_bytes, need);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int64_t* h = static_cast<int64_t*>(host);
  h[0] = kMagic;
  h[1] = 1;
  h[2] = N;
  h[3] = n;
  h[4] = p;
  h[5] = step;
  h[6] = K != nullptr;
  h[7] = 0;
  char* b = static_cast<char*>(host) + 8 * sizeof(int64_t);
  const size_t qb = sizeof(double) * (size_t)N * 2 * n, zb = sizeof(double) * (size_t)2 * n * p;
  if (cudaMemcpyAsync(b, Q, qb, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaMemcpyAsync(b + qb, Z, zb, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      (K && cudaMemcpyAsync(b + qb + zb, K, zb, cudaMemcpyDeviceToHost, st) != cudaSuccess) ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return vp_cuda_check(ctx, cudaGetLastError(), "state export");
  return VP_OK;
}

vp_status vp_state_import(vp_ctx* ctx, const void* host, size_t host_bytes, int64_t N, int32_t n,
                          int32_t p, double* Q, double* Z, double* K, int64_t* step, void* stream) {
  if (!ctx || !Q || !Z || !host || host_bytes < 8 * sizeof(int64_t)) return VP_EINVAL;
  const int64_t* h = static_cast<const int64_t*>(host);
  if (h[0] != kMagic || h[1] != 1) return vp_fail(ctx, VP_EINVAL, "not a state checkpoint");
  if (h[2] != N || h[3] != n || h[4] != p)
    return vp_fail(ctx, VP_EINVAL, "checkpoint sizes (%lld, %lld, %lld) differ from (%lld, %d, %d)",
                   (long long)h[2], (long long)h[3], (long long)h[4], (long long)N, n, p);
  if (K && !h[6]) return vp_fail(ctx, VP_EINVAL, "checkpoint holds no fixed-point state");
  if (host_bytes < vp_state_bytes(N, n, p, h[6] != 0)) return vp_fail(ctx, VP_EINVAL, "truncated checkpoint");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const char* b = static_cast<const char*>(host) + 8 * sizeof(int64_t);
  const size_t qb = sizeof(double) * (size_t)N * 2 * n, zb = sizeof(double) * (size_t)2 * n * p;
  if (cudaMemcpyAsync(Q, b, qb, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(Z, b + qb, zb, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      (K && cudaMemcpyAsync(K, b + qb + zb, zb, cudaMemcpyHostToDevice, st) != cudaSuccess) ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return vp_cuda_check(ctx, cudaGetLastError(), "state import");
  if (step) *step = h[5];
  return VP_OK;
}

vp_status vp_load_particles(vp_ctx* ctx, int32_t family, int32_t mode, uint64_t seed, int64_t N,
                            int32_t p, const double* eta_dev, double* X_dev, double* V_dev,
                            void* stream) {
  if (!ctx || !eta_dev || !X_dev || !V_dev || family < 0 || family > 2 || mode < 0 || mode > 1 ||
      N < 1 || p < 1 || p > 65535)
    return VP_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  VP_K(VP_K_LOAD, vpk::load_particles(family, mode, seed, family_k(family), N, p, eta_dev, X_dev,
                                      V_dev, ctx->num_sms, st));
  VP_LAUNCHED();
  return VP_OK;
}

}  // extern "C"
