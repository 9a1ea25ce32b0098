// Serving loop: requests of different grids, frequencies and media are
// queued by hz_submit and admitted onto the GPU as slots and HBM budget free
// up; each admitted request runs its whole pipeline (medium set-up, plan,
// FGMRES solve, read-back) on its own non-blocking stream from its own
// worker thread, so the kernels of concurrent requests overlap on the device
// (for instance one request's FP64 Arnoldi with another's complex64
// transforms).  Memory comes from the stream-ordered pool, so a request
// starting or finishing does not synchronise the device.  Every reduction is
// fixed-order and per request, so a result does not depend on what else runs.
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "hz_internal.h"
#include "kernels.h"

using Clock = std::chrono::steady_clock;
using hz::cuda_error;
using hz::set_tls_stream;

namespace {

struct Req {
  uint64_t id = 0;
  hz_grid grid{};
  std::vector<double> c, zeta, a;
  double omega = 0;
  hz_interp interp{};
  hz_solver_opts opts{};
  int nrhs = 1;
  long n = 0;
  std::vector<double2> f, u;
  std::vector<hz_solve_stats> stats;
  hz_status status = HZ_OK;
  std::string error;
  size_t footprint = 0;
  Clock::time_point t_submit, t_start, t_done;
  int bypassed = 0;  // later arrivals admitted ahead of this request
  uint64_t key = 0;  // batch mode: hash of grid, medium, frequency and options
  bool batched = false;  // runs in (or joins) a batched solve
  bool done = false;
};

// 64-bit hash of a byte range (multiply-xorshift over 8-byte words)
uint64_t hash_bytes(const void* p, size_t nb, uint64_t h) {
  const unsigned char* c = static_cast<const unsigned char*>(p);
  size_t i = 0;
  for (; i + 8 <= nb; i += 8) {
    uint64_t w;
    memcpy(&w, c + i, 8);
    h = (h ^ w) * 0x9E3779B97F4A7C15ull;
    h ^= h >> 29;
  }
  for (; i < nb; ++i) h = (h ^ c[i]) * 0x100000001B3ull;
  return h;
}

// requests that may share one batched solve: the same grid, medium,
// frequency, interpolation and solver options (right-hand sides differ)
uint64_t batch_key(const Req& r) {
  uint64_t h = 0xcbf29ce484222325ull;
  h = hash_bytes(&r.grid.dim, sizeof(int), h);
  h = hash_bytes(r.grid.n, sizeof(r.grid.n), h);
  h = hash_bytes(&r.grid.L, sizeof(double), h);
  h = hash_bytes(&r.omega, sizeof(double), h);
  const int iv[5] = {r.interp.M, r.interp.Mt, r.interp.symbol_kind, r.interp.Ma, r.interp.basis};
  const double dv[4] = {r.interp.c_o, r.interp.zeta_max, r.interp.alpha, r.interp.a_node};
  const int ov[6] = {r.opts.precision, r.opts.restart, r.opts.maxit, r.opts.graphs,
                     r.opts.no_precond, r.opts.left};
  h = hash_bytes(iv, sizeof(iv), h);
  h = hash_bytes(dv, sizeof(dv), h);
  h = hash_bytes(ov, sizeof(ov), h);
  h = hash_bytes(&r.opts.tol, sizeof(double), h);
  h = hash_bytes(r.c.data(), r.c.size() * sizeof(double), h);
  h = hash_bytes(r.zeta.data(), r.zeta.size() * sizeof(double), h);
  h = hash_bytes(r.a.data(), r.a.size() * sizeof(double), h);
  return h;
}

bool same_problem(const Req& a, const Req& b) {
  return a.key == b.key && a.n == b.n && a.c == b.c && a.zeta == b.zeta && a.a == b.a &&
         a.omega == b.omega && memcmp(&a.grid, &b.grid, sizeof(hz_grid)) == 0 &&
         memcmp(&a.interp, &b.interp, sizeof(hz_interp)) == 0 &&
         memcmp(&a.opts, &b.opts, sizeof(hz_solver_opts)) == 0;
}

size_t fft_partial_bytes(long n, int B, int m) {
  const long nblk = std::max(1024L, (n + 255) / 256);
  return size_t(B) * (m + 2) * nblk * 2 * sizeof(double);
}

}  // namespace

// Device bytes one request holds while it runs: medium (gamma^2, records,
// damping, staging of c and zeta during set-up, masks) and plan (transformed
// input, K planes, Krylov basis, Z, staged f/u, partial sums).
extern "C" size_t hz_request_footprint(const hz_grid* g, const hz_interp* it,
                                       const hz_solver_opts* o, int nrhs, int has_a) {
  const long n = long(g->n[0]) * g->n[1] * (g->dim == 3 ? g->n[2] : 1);
  const int Ka = it->Ma > 1 ? it->Ma : 1;
  const int K = (it->M + it->Mt) * Ka + (it->basis == 2 ? it->M : 0);
  const bool generic = Ka > 1 || it->basis >= 1;  // per-point (node, weight) records
  const int m = o->restart;
  const size_t B = size_t(nrhs);
  const size_t es = o->precision == 0 ? 16 : 8;
  // (row masks, and at most K (row, node) items of 8 bytes per row)
  const size_t rows = size_t(n / g->n[0]);
  size_t med = size_t(n) * (16 + 8 + 4 + (has_a ? 8 : 0) + 16 + (generic ? 52 : 0)) +
               (rows + 1) * 16 * (generic ? 4 : 1) + rows * size_t(K) * 8 + (1 << 20);
  size_t plan = B * n * 16                      // tmp
                + B * K * n * es                // planes
                + size_t(m + 1) * B * n * 16    // V
                + (o->precision == 1 ? size_t(m) * B * n * 8 : B * n * 16)  // Z
                + 2 * B * n * 16                // staged u, f
                + fft_partial_bytes(n, int(B), m) + (1 << 20);
  return med + plan;
}

struct hz_server {
  hz_server_opts opts{};
  int device = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<Req>> queue;
  std::unordered_map<uint64_t, std::shared_ptr<Req>> table;
  size_t in_use = 0;
  int active = 0, max_active_seen = 0;
  bool stop = false;
  std::vector<std::thread> workers;
  uint64_t next_id = 1;
  long long submitted = 0, completed = 0, failed = 0, rejected = 0, rhs_done = 0, joins = 0;
  // batch mode: free slots of the running batches, by batch key
  std::unordered_map<uint64_t, int> batch_free;
  std::vector<double> lat_ms;
  Clock::time_point t0;
};

namespace {

void run_request(hz_server* s, Req& r, cudaStream_t st) {
  hz_medium* med = nullptr;
  hz_plan* plan = nullptr;
  r.u.assign(size_t(r.nrhs) * r.n, make_double2(0, 0));
  r.stats.assign(r.nrhs, hz_solve_stats{});
  hz_status rc = hz_create_medium(&r.grid, r.c.data(), r.zeta.empty() ? nullptr : r.zeta.data(),
                                  r.a.empty() ? nullptr : r.a.data(), r.omega, &r.interp, &med);
  if (rc == HZ_OK) rc = hz_plan_create(med, &r.opts, r.nrhs, &plan);
  // launch shapes: the autotuner's cached choice for this grid, K, restart
  // and precision (timing once per key on a miss when opts.autotune == 1)
  if (rc == HZ_OK && s->opts.autotune >= 0 && !hz::tune_from_cache(plan) && s->opts.autotune == 1)
    rc = hz_plan_autotune(plan, st, nullptr);
  if (rc == HZ_OK) {
    const size_t vb = size_t(r.nrhs) * r.n * sizeof(double2);
    cudaError_t ce = cudaMemcpyAsync(plan->f, r.f.data(), vb, cudaMemcpyHostToDevice, st);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(plan->u, 0, vb, st);
    if (ce != cudaSuccess) {
      rc = cuda_error(ce, "request upload");
    } else {
      rc = hz_gmres_solve(plan, plan->f, plan->u, r.nrhs, r.stats.data(), st);
      if (rc == HZ_OK || rc == HZ_ERR_NOT_CONVERGED || rc == HZ_ERR_BREAKDOWN) {
        ce = cudaMemcpyAsync(r.u.data(), plan->u, vb, cudaMemcpyDeviceToHost, st);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
        if (ce != cudaSuccess) rc = cuda_error(ce, "request read-back");
      }
    }
  }
  if (rc != HZ_OK) r.error = hz_last_error();
  if (plan) hz_destroy_plan(plan);
  if (med) hz_destroy_medium(med);
  cudaStreamSynchronize(st);
  r.status = rc;
}

// Under s->mu: the request has finished; book it and drop its inputs.
void finish_locked(hz_server* s, Req& r, bool holds_footprint) {
  if (holds_footprint) s->in_use -= r.footprint;
  r.t_done = Clock::now();
  r.done = true;
  if (r.status == HZ_OK) {
    ++s->completed;
    s->rhs_done += r.nrhs;
  } else {
    ++s->failed;
  }
  s->lat_ms.push_back(std::chrono::duration<double, std::milli>(r.t_done - r.t_submit).count());
  r.c.clear(); r.c.shrink_to_fit();
  r.zeta.clear(); r.zeta.shrink_to_fit();
  r.a.clear(); r.a.shrink_to_fit();
  r.f.clear(); r.f.shrink_to_fit();
}

// Batch mode: one medium and one plan of batch_slots right-hand-side slots
// for every request of the same problem (grid, medium, frequency, options).
// The first request and any queued ones of the same problem take slots; at
// every restart boundary, requests whose slots have all finished leave
// (solution and stats copied out) and queued requests of the same problem
// join the free slots, while the others keep iterating.
void run_batch(hz_server* s, std::shared_ptr<Req> first, cudaStream_t st) {
  const int B = s->opts.batch_slots;
  Req& r0 = *first;
  hz_medium* med = nullptr;
  hz_plan* plan = nullptr;
  hz_status rc = hz_create_medium(&r0.grid, r0.c.data(), r0.zeta.empty() ? nullptr : r0.zeta.data(),
                                  r0.a.empty() ? nullptr : r0.a.data(), r0.omega, &r0.interp, &med);
  if (rc == HZ_OK) rc = hz_plan_create(med, &r0.opts, B, &plan);
  if (rc == HZ_OK && s->opts.autotune >= 0 && !hz::tune_from_cache(plan) && s->opts.autotune == 1)
    rc = hz_plan_autotune(plan, st, nullptr);
  if (rc != HZ_OK) {
    r0.status = rc;
    r0.error = hz_last_error();
    {
      std::lock_guard<std::mutex> lk(s->mu);
      finish_locked(s, r0, false);
      auto it = s->batch_free.find(r0.key);
      if (it != s->batch_free.end() && (it->second -= B - r0.nrhs) <= 0) s->batch_free.erase(it);
    }
    s->cv_done.notify_all();
    if (plan) hz_destroy_plan(plan);
    if (med) hz_destroy_medium(med);
    return;
  }
  // the batch's own copy of the problem, to compare joining requests with
  Req proto;
  proto.key = r0.key;
  proto.n = r0.n;
  proto.grid = r0.grid;
  proto.omega = r0.omega;
  proto.interp = r0.interp;
  proto.opts = r0.opts;
  proto.c = r0.c;
  proto.zeta = r0.zeta;
  proto.a = r0.a;
  const long n = r0.n;
  std::vector<char> taken(B, 0);                  // slot assigned to a member
  std::vector<std::shared_ptr<Req>> members;
  std::vector<std::vector<int>> slots_of;         // per member: its slots
  std::vector<std::shared_ptr<Req>> pending{first};  // joining at the next boundary
  // this batch's share of s->batch_free[key] (registered by the worker when
  // it admitted the first request)
  int my_free = B - r0.nrhs;
  auto boundary = [&](hz::BatchCtl& ctl) -> int {
    // members whose slots have all finished leave
    for (size_t i = 0; i < members.size();) {
      Req& r = *members[i];
      bool fin = true;
      for (int b : slots_of[i]) fin = fin && ctl.done[b];
      if (!fin) {
        ++i;
        continue;
      }
      hz_status st_r = HZ_OK;
      const float ms = std::chrono::duration<float, std::milli>(Clock::now() - r.t_start).count();
      for (size_t k = 0; k < slots_of[i].size(); ++k) {
        const int b = slots_of[i][k];
        hz_solve_stats& x = r.stats[k];
        x.iters = ctl.iters[b];
        x.restarts = ctl.restarts[b];
        x.converged = ctl.conv[b];
        x.status = ctl.conv[b] ? HZ_OK : (ctl.status[b] == HZ_OK ? HZ_ERR_NOT_CONVERGED : ctl.status[b]);
        x.rel_true_resid = ctl.rel[b];
        x.rel_est_resid = ctl.est[b];
        x.ms_total = ms;
        if (x.status != HZ_OK && (st_r == HZ_OK || x.status == HZ_ERR_BREAKDOWN)) st_r = hz_status(x.status);
        if (cudaMemcpyAsync(r.u.data() + size_t(k) * n, ctl.u + long(b) * n, n * sizeof(double2),
                            cudaMemcpyDeviceToHost, st) != cudaSuccess)
          st_r = HZ_ERR_CUDA;
        ctl.release(b);
        taken[b] = 0;
      }
      if (cudaStreamSynchronize(st) != cudaSuccess) st_r = HZ_ERR_CUDA;
      r.status = st_r;
      if (st_r != HZ_OK) r.error = st_r == HZ_ERR_CUDA ? "read-back failed" : "not converged within maxit";
      {
        std::lock_guard<std::mutex> lk(s->mu);
        finish_locked(s, r, false);
        my_free += r.nrhs;
        s->batch_free[proto.key] += r.nrhs;
      }
      s->cv_done.notify_all();
      members.erase(members.begin() + long(i));
      slots_of.erase(slots_of.begin() + long(i));
    }
    // queued requests of the same problem join the free slots
    {
      std::lock_guard<std::mutex> lk(s->mu);
      for (auto it = s->queue.begin(); it != s->queue.end() && my_free > 0;) {
        Req& q = **it;
        if (q.batched && q.nrhs <= my_free && q.key == proto.key && same_problem(q, proto)) {
          q.t_start = Clock::now();
          pending.push_back(*it);
          my_free -= q.nrhs;
          s->batch_free[proto.key] -= q.nrhs;
          ++s->joins;
          it = s->queue.erase(it);
        } else {
          ++it;
        }
      }
    }
    if (pending.empty()) return 0;
    for (auto& q : pending) {
      std::vector<int> sl;
      for (int b = 0; b < B && int(sl.size()) < q->nrhs; ++b)
        if (!taken[b]) {
          taken[b] = 1;
          sl.push_back(b);
        }
      q->u.assign(size_t(q->nrhs) * n, make_double2(0, 0));
      q->stats.assign(q->nrhs, hz_solve_stats{});
      members.push_back(q);
      slots_of.push_back(sl);
      for (int k = 0; k < q->nrhs; ++k) {
        const int b = sl[k];
        if (cudaMemcpyAsync(ctl.f + long(b) * n, q->f.data() + size_t(k) * n, n * sizeof(double2),
                            cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaMemsetAsync(ctl.u + long(b) * n, 0, n * sizeof(double2), st) != cudaSuccess)
          return -int(HZ_ERR_CUDA);
        const hz_status a = ctl.admit(b);
        if (a != HZ_OK) return -int(a);
      }
    }
    pending.clear();
    return 1;
  };
  rc = hz::gmres_batch(plan, st, boundary);
  if (rc != HZ_OK) {
    // a failure ends every member still in the batch
    const std::string msg = hz_last_error();
    for (auto* v : {&members, &pending})
      for (auto& q : *v) {
        q->status = rc;
        q->error = msg;
        std::lock_guard<std::mutex> lk(s->mu);
        finish_locked(s, *q, false);
      }
    s->cv_done.notify_all();
  }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->batch_free.find(proto.key);
    if (it != s->batch_free.end()) {
      it->second -= my_free;
      if (it->second <= 0) s->batch_free.erase(it);
    }
  }
  hz_destroy_plan(plan);
  hz_destroy_medium(med);
  cudaStreamSynchronize(st);
}

void worker_main(hz_server* s) {
  cudaSetDevice(s->device);
  cudaStream_t st = nullptr;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    st = nullptr;
  }
  set_tls_stream(st, st != nullptr);
  for (;;) {
    std::shared_ptr<Req> r;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      for (;;) {
        if (s->stop) {
          set_tls_stream(nullptr, false);
          if (st) cudaStreamDestroy(st);
          return;
        }
        // Admission within the HBM budget, with aging: a request that later
        // arrivals have overtaken max_bypass times is not overtaken again
        // (admission waits until it fits).  order 0: the first request in
        // arrival order that fits; order 1: the one with the smallest
        // footprint (about the least work) that fits.
        size_t pick = s->queue.size();
        for (size_t i = 0; i < s->queue.size(); ++i) {
          const Req& q = *s->queue[i];
          // a running batch of the same problem with room takes it at its
          // next restart boundary
          if (q.batched) {
            auto bf = s->batch_free.find(q.key);
            if (bf != s->batch_free.end() && bf->second >= q.nrhs) continue;
          }
          const bool fits = s->in_use + q.footprint <= s->opts.hbm_budget || s->active == 0;
          if (fits && (pick == s->queue.size() || q.footprint < s->queue[pick]->footprint))
            pick = i;
          if (fits && s->opts.order == 0) break;
          // an aged request: nothing behind it may go first
          if (q.bypassed >= s->opts.max_bypass) {
            if (fits) pick = i;
            break;
          }
        }
        if (pick < s->queue.size()) {
          for (size_t i = 0; i < pick; ++i) ++s->queue[i]->bypassed;
          r = s->queue[pick];
          s->queue.erase(s->queue.begin() + long(pick));
          break;
        }
        s->cv_work.wait(lk);
      }
      s->in_use += r->footprint;
      ++s->active;
      // a new batch: its free slots take queued requests of the same problem
      if (r->batched) s->batch_free[r->key] += s->opts.batch_slots - r->nrhs;
      s->max_active_seen = std::max(s->max_active_seen, s->active);
      r->t_start = Clock::now();
    }
    if (r->batched) {
      // the batch holds the first request's footprint (a plan of
      // batch_slots right-hand sides) until its last member leaves
      run_batch(s, r, st);
      std::lock_guard<std::mutex> lk(s->mu);
      s->in_use -= r->footprint;
      --s->active;
    } else {
      run_request(s, *r, st);
      {
        std::lock_guard<std::mutex> lk(s->mu);
        finish_locked(s, *r, true);
        --s->active;
      }
    }
    s->cv_done.notify_all();
    s->cv_work.notify_all();
  }
}

double percentile(std::vector<double> v, double q) {
  if (v.empty()) return 0.0;
  std::sort(v.begin(), v.end());
  const double pos = q * double(v.size() - 1);
  const size_t i = size_t(pos);
  const double f = pos - double(i);
  return i + 1 < v.size() ? v[i] * (1 - f) + v[i + 1] * f : v[i];
}

}  // namespace

using namespace hz;

extern "C" hz_status hz_server_create(const hz_server_opts* opts, hz_server** out) {
  if (!opts || !out) return set_error(HZ_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  if (opts->max_slots < 1 || opts->max_slots > 64 || opts->max_queue < 1)
    return set_error(HZ_ERR_INVALID_ARG, "need 1 <= max_slots <= 64 and max_queue >= 1");
  if (opts->autotune < -1 || opts->autotune > 1 || opts->max_bypass < 0 || opts->batch_slots < 0 ||
      opts->batch_slots > 64 || opts->order < 0 || opts->order > 1)
    return set_error(HZ_ERR_INVALID_ARG,
                     "need autotune in {-1, 0, 1}, max_bypass >= 0, batch_slots in 0..64, "
                     "order 0 or 1");
  hz_server* s = new hz_server();
  s->opts = *opts;
  if (s->opts.max_bypass == 0) s->opts.max_bypass = 2 * s->opts.max_slots;
  s->device = opts->device;
  HZ_CUDA(cudaSetDevice(s->device));
  if (s->opts.hbm_budget == 0) {
    size_t fr = 0, tot = 0;
    HZ_CUDA(cudaMemGetInfo(&fr, &tot));
    s->opts.hbm_budget = fr / 10 * 8;
  }
  // keep freed blocks in the stream-ordered pool between requests
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, s->device) == cudaSuccess) {
    unsigned long long thr = ~0ull;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  cudaGetLastError();
  s->t0 = Clock::now();
  for (int i = 0; i < opts->max_slots; ++i) s->workers.emplace_back(worker_main, s);
  *out = s;
  return HZ_OK;
}

extern "C" hz_status hz_submit(hz_server* s, const hz_request* q, uint64_t* ticket) {
  if (!s || !q || !ticket || !q->c || !q->f) return set_error(HZ_ERR_INVALID_ARG, "null argument");
  if (q->nrhs < 1) return set_error(HZ_ERR_INVALID_ARG, "nrhs must be >= 1");
  if (q->grid.dim != 2 && q->grid.dim != 3) return set_error(HZ_ERR_INVALID_ARG, "dim must be 2 or 3");
  for (int d = 0; d < q->grid.dim; ++d)
    if (!fft_size_supported(q->grid.n[d]))
      return set_error(HZ_ERR_INVALID_ARG, "unsupported axis length %d", q->grid.n[d]);
  auto r = std::make_shared<Req>();
  r->grid = q->grid;
  if (r->grid.dim == 2) r->grid.n[2] = 1;
  r->n = long(r->grid.n[0]) * r->grid.n[1] * r->grid.n[2];
  r->omega = q->omega;
  r->interp = q->interp;
  r->opts = q->opts;
  r->nrhs = q->nrhs;
  r->batched = s->opts.batch_slots > 0 && r->nrhs <= s->opts.batch_slots && !r->opts.left;
  r->footprint = hz_request_footprint(&r->grid, &r->interp, &r->opts,
                                      r->batched ? s->opts.batch_slots : r->nrhs, q->a != nullptr);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (r->footprint > s->opts.hbm_budget) {
      ++s->rejected;
      return set_error(HZ_ERR_BUSY, "request needs %zu bytes, more than the server's budget %zu",
                       r->footprint, s->opts.hbm_budget);
    }
    if (int(s->queue.size()) >= s->opts.max_queue) {
      ++s->rejected;
      return set_error(HZ_ERR_BUSY, "queue full (%d requests)", s->opts.max_queue);
    }
  }
  r->c.assign(q->c, q->c + r->n);
  if (q->zeta) r->zeta.assign(q->zeta, q->zeta + r->n);
  if (q->a) r->a.assign(q->a, q->a + r->n);
  const double2* f = static_cast<const double2*>(q->f);
  r->f.assign(f, f + size_t(r->nrhs) * r->n);
  if (r->batched) r->key = batch_key(*r);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    r->id = s->next_id++;
    r->t_submit = Clock::now();
    s->table[r->id] = r;
    s->queue.push_back(r);
    ++s->submitted;
    *ticket = r->id;
  }
  s->cv_work.notify_one();
  return HZ_OK;
}

extern "C" hz_status hz_poll(hz_server* s, uint64_t ticket, int* done, void* u_out,
                             hz_solve_stats* stats) {
  if (!s || !done) return set_error(HZ_ERR_INVALID_ARG, "null argument");
  std::shared_ptr<Req> r;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->table.find(ticket);
    if (it == s->table.end()) return set_error(HZ_ERR_INVALID_ARG, "unknown ticket %llu", (unsigned long long)ticket);
    r = it->second;
    if (!r->done) {
      *done = 0;
      return HZ_OK;
    }
    s->table.erase(it);
  }
  *done = 1;
  if (u_out && !r->u.empty()) memcpy(u_out, r->u.data(), r->u.size() * sizeof(double2));
  if (stats && !r->stats.empty()) memcpy(stats, r->stats.data(), r->stats.size() * sizeof(hz_solve_stats));
  if (r->status != HZ_OK) return set_error(r->status, "%s", r->error.c_str());
  return HZ_OK;
}

extern "C" hz_status hz_server_wait(hz_server* s, uint64_t ticket, double timeout_s) {
  if (!s) return set_error(HZ_ERR_INVALID_ARG, "null argument");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->table.find(ticket);
  if (it == s->table.end()) return set_error(HZ_ERR_INVALID_ARG, "unknown ticket");
  auto r = it->second;
  const auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(
                                           std::chrono::duration<double>(timeout_s));
  while (!r->done) {
    if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && !r->done)
      return set_error(HZ_ERR_TIMEOUT, "request %llu not done within %.3f s",
                       (unsigned long long)ticket, timeout_s);
  }
  return HZ_OK;
}

extern "C" hz_status hz_server_get_stats(hz_server* s, hz_server_stats* out) {
  if (!s || !out) return set_error(HZ_ERR_INVALID_ARG, "null argument");
  std::lock_guard<std::mutex> lk(s->mu);
  out->submitted = s->submitted;
  out->completed = s->completed;
  out->failed = s->failed;
  out->rejected = s->rejected;
  out->active = s->active;
  out->queued = int(s->queue.size());
  out->max_active = s->max_active_seen;
  out->hbm_in_use = s->in_use;
  out->hbm_budget = s->opts.hbm_budget;
  out->p50_ms = percentile(s->lat_ms, 0.50);
  out->p99_ms = percentile(s->lat_ms, 0.99);
  double mean = 0;
  for (double v : s->lat_ms) mean += v;
  out->mean_ms = s->lat_ms.empty() ? 0 : mean / s->lat_ms.size();
  const double el = std::chrono::duration<double>(Clock::now() - s->t0).count();
  out->rhs_per_s = el > 0 ? double(s->rhs_done) / el : 0;
  out->batch_joins = s->joins;
  return HZ_OK;
}

extern "C" hz_status hz_server_destroy(hz_server* s) {
  if (!s) return HZ_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->queue.clear();
  }
  s->cv_work.notify_all();
  for (auto& t : s->workers) t.join();
  delete s;
  return HZ_OK;
}
