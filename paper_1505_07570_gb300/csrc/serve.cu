// Continuous-batching request server (host code).
//
// Requests queue in arrival order.  Each stream ("lane") has its own context, whose workspace is capped at
// the lane's share of the HBM budget, at most one launch in flight, and a host thread that issues the lane's
// launches (the kernel launches of a request cost host time; with one thread per lane the lanes' launches are
// issued in parallel, and the caller's thread only queues, admits and retires).  Whenever a lane is free the
// head of the queue is admitted: a request too large for the batched kernel runs alone through rmc_lsr_sketch or
// rmc_rsvd; otherwise every batchable request queued so far (in order, up to max_batch and the lane's memory)
// goes into one rmc_batch_run launch.  Requests that arrive while launches are in flight are admitted as soon
// as a lane frees up, so launches of different sizes overlap on the device.  Completion is seen by polling
// each lane's event; a request's latency runs from its submit call to the progress call that retires it.
//
// Results do not depend on the mix: a request always takes the same route (decided by its own size and
// precision, and by whether residency was on when it was submitted), and every route computes a problem with
// arithmetic that is independent of other problems.
//
// Residency (rmc_server_resident): least-squares requests take the resident route.  The server keeps, per
// (matrix, sketch kind, s, seed, precision), the sketch S^T A and the preconditioner M of its factor in device
// memory (a byte cap, least recently used entries evicted once no launch uses them).  A request whose entry is
// resident copies S^T A, sketches its own b with the same operator and refines against M; one whose entry is not
// resident first sketches A and factors (into a new entry, or into the lane's workspace when the cap leaves no
// room) and then does the same.  Both cases run the same kernels on the same values, so a result does not depend
// on what is resident.

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "rmc_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

// Resident state of one (matrix, sketch) pair: S^T A (s x n, row stride n), M (n x n) and the factor's failure
// flag, in one stream-ordered allocation.
struct ResKey {
  const float *A;
  int64_t m, n, lda, s;
  int sketch, prec;
  uint64_t seed;
  bool operator==(const ResKey &o) const {
    return A == o.A && m == o.m && n == o.n && lda == o.lda && s == o.s && sketch == o.sketch && prec == o.prec &&
           seed == o.seed;
  }
};

struct Resident {
  ResKey key;
  void *mem = nullptr;
  float *SA = nullptr, *M = nullptr;
  int *fail = nullptr;
  size_t bytes = 0;
  cudaEvent_t ready = nullptr;   // recorded once S^T A and M are complete
  uint64_t last_use = 0;
  int users = 0;                 // launches in flight that read it
  bool dead = false;             // released: freed once unused
  bool recorded = false;         // `ready` recorded: other lanes may read it
};

size_t resident_bytes(int64_t s, int64_t n) {
  WsCarve w;
  w.take<float>((size_t)s * n);
  w.take<float>((size_t)n * n);
  w.take<int>(4);
  return w.off;
}

struct Queued {
  rmc_serve_request r;
  uint64_t ticket;
  Clock::time_point t_submit;
  bool batch;
  bool resident = false;         // least squares through the resident route
  Resident *res = nullptr;       // the entry its launch reads
};

// Lane states: the main thread moves kIdle -> kPosted (work handed to the lane's thread), the lane's thread
// kPosted -> kEnqueued (launches issued, `done` recorded), the main thread kEnqueued -> kIdle once `done` has
// completed and the requests are retired.
enum LaneState { kIdle = 0, kPosted = 1, kEnqueued = 2 };

struct Lane {
  cudaStream_t stream = nullptr;
  rmc_ctx *ctx = nullptr;
  cudaEvent_t done = nullptr;
  int launch_status = RMC_OK;
  std::vector<Queued> work;        // the requests of the launch in flight
  std::vector<rmc_request> reqs;   // a batched launch's problems
  bool batch_job = false;
  std::atomic<int> state{kIdle};
  std::mutex mu;
  std::condition_variable cv;
  bool stop = false;
  std::thread thread;
};

struct Done {
  uint64_t ticket;
  int status;
  double latency_s;
};

bool valid_single(const rmc_serve_request &q) {
  const rmc_request &r = q.req;
  if (!r.A || r.m < 1 || r.n < 1 || r.lda < r.n || r.m > (int64_t(1) << 31)) return false;
  if (!rmc_prec_ok(q.prec)) return false;
  if (r.kind == RMC_REQ_LSR) {
    if (q.sketch != RMC_GAUSSIAN && q.sketch != RMC_SRHT && q.sketch != RMC_COUNTSKETCH) return false;
    if (q.sketch == RMC_GAUSSIAN && q.prec == RMC_TF32X3) return false;
    if (q.sketch == RMC_SRHT) {
      int64_t N = 1;
      while (N < r.m) N <<= 1;
      if (r.s > N) return false;
    }
    return r.b && r.x && r.s >= r.n && r.n <= 1024 && r.s <= (int64_t(1) << 31);
  }
  if (r.kind == RMC_REQ_RSVD) {
    const int64_t l = int64_t(r.k) + r.p;
    return r.U && r.sigma && r.V && r.k >= 1 && r.p >= 0 && r.q >= 0 && l <= r.m && l <= r.n && l <= 256;
  }
  return false;
}

bool batchable(const rmc_serve_request &q) {
  if (!rmc_batch_request_ok(q.req)) return false;
  if (q.req.kind == RMC_REQ_LSR) return q.sketch == RMC_COUNTSKETCH;
  // the batched kernel computes its products at FP32 accuracy (3xTF32 on mma.sync)
  return q.prec == RMC_FP32 || q.prec == RMC_TF32X3;
}

}  // namespace

struct rmc_server {
  size_t lane_budget = 0;
  int max_batch = 0;
  uint64_t next_ticket = 1;
  int device = 0;
  std::vector<std::unique_ptr<Lane>> lanes;
  std::deque<Queued> singles, batchables;   // the queue in arrival order, split by route (tickets increase)
  std::vector<Done> done;
  size_t res_cap = 0, res_used = 0;   // resident state: byte cap and bytes held
  uint64_t res_tick = 0;
  std::vector<Resident *> res;
  std::mutex res_mu;                  // the resident entries (lane threads make and read them)
};

namespace {

void retire(rmc_server *srv) {
  for (auto &Lp : srv->lanes) {
    Lane &L = *Lp;
    if (L.state.load(std::memory_order_acquire) != kEnqueued) continue;
    const cudaError_t e = cudaEventQuery(L.done);
    if (e == cudaErrorNotReady) continue;
    int st = e == cudaSuccess ? L.launch_status : RMC_ECUDA;
    if (e != cudaSuccess) (void)cudaGetLastError();
    if (st == RMC_OK && *L.ctx->h_status != RMC_OK) st = *L.ctx->h_status;
    const Clock::time_point now = Clock::now();
    {
      std::lock_guard<std::mutex> lk(srv->res_mu);
      for (const Queued &w : L.work) {
        srv->done.push_back({w.ticket, st, std::chrono::duration<double>(now - w.t_submit).count()});
        if (w.res) --w.res->users;
      }
    }
    L.work.clear();
    L.reqs.clear();
    L.state.store(kIdle, std::memory_order_release);
  }
}

// Free an unused entry (its last reader has retired, so any stream may order the free).
void res_free(rmc_server *srv, Resident *e, cudaStream_t st) {
  if (e->mem) (void)cudaFreeAsync(e->mem, st);
  if (e->ready) (void)cudaEventDestroy(e->ready);
  srv->res_used -= e->bytes;
  delete e;
}

// Drop released entries that no launch reads any more (caller holds res_mu).
void res_collect(rmc_server *srv) {
  cudaStream_t st = srv->lanes[0]->stream;
  for (size_t i = 0; i < srv->res.size();) {
    Resident *e = srv->res[i];
    if (e->dead && e->users == 0) {
      res_free(srv, e, st);
      srv->res.erase(srv->res.begin() + i);
    } else {
      ++i;
    }
  }
}

// A new entry for `key`, evicting unused entries (least recently used first) to stay within the cap; nullptr
// when it cannot be made (the request then uses the lane's workspace).
Resident *res_make(rmc_server *srv, const ResKey &key, cudaStream_t st) {
  const size_t bytes = resident_bytes(key.s, key.n);
  if (bytes > srv->res_cap) return nullptr;
  while (srv->res_used + bytes > srv->res_cap) {
    int victim = -1;
    for (int i = 0; i < (int)srv->res.size(); ++i)
      if (srv->res[i]->users == 0 && (victim < 0 || srv->res[i]->last_use < srv->res[victim]->last_use)) victim = i;
    if (victim < 0) return nullptr;
    res_free(srv, srv->res[victim], st);
    srv->res.erase(srv->res.begin() + victim);
  }
  Resident *e = new (std::nothrow) Resident();
  if (!e) return nullptr;
  e->key = key;
  e->bytes = bytes;
  if (cudaMallocAsync(&e->mem, bytes, st) != cudaSuccess ||
      cudaEventCreateWithFlags(&e->ready, cudaEventDisableTiming) != cudaSuccess) {
    (void)cudaGetLastError();
    if (e->mem) (void)cudaFreeAsync(e->mem, st);
    if (e->ready) (void)cudaEventDestroy(e->ready);
    delete e;
    return nullptr;
  }
  WsCarve w;
  w.base = static_cast<char *>(e->mem);
  e->SA = w.take<float>((size_t)key.s * key.n);
  e->M = w.take<float>((size_t)key.n * key.n);
  e->fail = w.take<int>(4);
  srv->res_used += bytes;
  srv->res.push_back(e);
  return e;
}

// Lane workspace of the resident route: [S^T A, S^T b] (s x (n+1)), S^T A, M and the failure flag when they are
// not resident, then the largest scratch of the sketches, the factor and the refinement.
size_t resident_plan(rmc_ctx *ctx, const rmc_request &r, int sketch, int prec, float **SAb, float **SA, float **M,
                     int **fail, void **rest, char *base) {
  size_t scratch = rmc_sketch_plan_bytes(ctx, r.m, r.n, r.s, sketch, prec);
  scratch = std::max(scratch, rmc_sketch_plan_bytes(ctx, r.m, 1, r.s, sketch, prec));
  scratch = std::max(scratch, rmc_lsr_factor_ws(r.s, r.n, ctx->num_sms));
  scratch = std::max(scratch, rmc_lsr_refine_ws(r.s, r.n, ctx->num_sms));
  WsCarve w;
  w.base = base;
  *SAb = w.take<float>((size_t)r.s * (r.n + 1));
  *SA = w.take<float>((size_t)r.s * r.n);
  *M = w.take<float>((size_t)r.n * r.n);
  *fail = w.take<int>(4);
  *rest = w.take<char>(scratch);
  return w.off;
}

// Least squares through the resident route on lane L (see the header comment).  Returns the entry read, if any.
int launch_resident(rmc_server *srv, Lane &L, const rmc_serve_request &q, Resident **used) {
  const rmc_request &r = q.req;
  rmc_ctx *ctx = L.ctx;
  cudaStream_t st = L.stream;
  *used = nullptr;
  float *SAb, *SA, *M;
  int *fail;
  void *rest;
  const size_t need = resident_plan(ctx, r, q.sketch, q.prec, &SAb, &SA, &M, &fail, &rest, nullptr);
  RMC_TRY(rmc_ws_reserve(ctx, need));
  resident_plan(ctx, r, q.sketch, q.prec, &SAb, &SA, &M, &fail, &rest, static_cast<char *>(ctx->ws));
  const ResKey key{r.A, r.m, r.n, r.lda, r.s, q.sketch, q.prec, r.seed};
  Resident *e = nullptr;
  bool fresh = false;
  {
    // an entry still being filled by another lane's thread (its ready event not yet recorded) is not used: this
    // request computes into its own workspace instead (the same values)
    std::lock_guard<std::mutex> lk(srv->res_mu);
    Resident *found = nullptr;
    for (Resident *c : srv->res)
      if (!c->dead && c->key == key) found = c;
    if (found && found->recorded) {
      e = found;
    } else if (!found) {
      e = res_make(srv, key, st);
      fresh = e != nullptr;
    }
    if (e) {
      e->last_use = ++srv->res_tick;
      ++e->users;
    }
  }
  if (e) {
    SA = e->SA;
    M = e->M;
    fail = e->fail;
    *used = e;
  }
  if (!e || fresh) {
    // S^T A (row stride n) and its factor; an entry whose filling could not be enqueued is never read
    int rc = rmc_run_sketch(ctx, r.A, r.m, r.n, r.lda, nullptr, r.s, q.sketch, r.seed, q.prec, SA, r.n, nullptr,
                            rest);
    if (rc == RMC_OK) rc = rmc_launch_lsr_factor(ctx, SA, r.s, r.n, r.n, M, fail, rest);
    if (rc == RMC_OK && e && cudaEventRecord(e->ready, st) != cudaSuccess) {
      (void)cudaGetLastError();
      rc = RMC_ECUDA;
    }
    if (e) {
      std::lock_guard<std::mutex> lk(srv->res_mu);
      if (rc == RMC_OK) e->recorded = true;
      else e->dead = true;
    }
    if (rc != RMC_OK) return rc;
  } else {
    RMC_TRY_CUDA(cudaStreamWaitEvent(st, e->ready, 0));
  }
  // [S^T A, S^T b]: the resident sketch, and this request's b through the same operator
  RMC_TRY_CUDA(cudaMemcpy2DAsync(SAb, sizeof(float) * (r.n + 1), SA, sizeof(float) * r.n, sizeof(float) * r.n,
                                 r.s, cudaMemcpyDeviceToDevice, st));
  RMC_TRY(rmc_run_sketch(ctx, r.b, r.m, 1, 1, nullptr, r.s, q.sketch, r.seed, q.prec, SAb + r.n, r.n + 1, nullptr,
                         rest));
  return rmc_launch_lsr_refine(ctx, SAb, r.s, r.n, r.n + 1, M, fail, r.x, rest);
}

// Close a launch: fetch the device status word behind it and mark its end with the lane's event.
void seal(Lane &L, int rc) {
  L.launch_status = rc;
  *L.ctx->h_status = RMC_OK;
  if (cudaMemcpyAsync(L.ctx->h_status, L.ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, L.stream) !=
          cudaSuccess ||
      cudaMemsetAsync(L.ctx->d_status, 0, sizeof(int), L.stream) != cudaSuccess ||
      cudaEventRecord(L.done, L.stream) != cudaSuccess) {
    (void)cudaGetLastError();
    L.launch_status = RMC_ECUDA;
    (void)cudaStreamSynchronize(L.stream);
    (void)cudaEventRecord(L.done, L.stream);
  }
}

// The lane's thread: issues the launches of the work posted to it, then marks the lane enqueued.
void lane_thread(rmc_server *srv, Lane *Lp) {
  Lane &L = *Lp;
  (void)cudaSetDevice(srv->device);
  for (;;) {
    {
      std::unique_lock<std::mutex> lk(L.mu);
      L.cv.wait(lk, [&] { return L.stop || L.state.load(std::memory_order_acquire) == kPosted; });
      if (L.stop) return;
    }
    int rc;
    if (L.batch_job) {
      rc = rmc_batch_run(L.ctx, L.reqs.data(), (int)L.reqs.size());
    } else {
      Queued &w = L.work.front();
      const rmc_request &r = w.r.req;
      if (w.resident)
        rc = launch_resident(srv, L, w.r, &w.res);
      else if (r.kind == RMC_REQ_LSR)
        rc = rmc_lsr_sketch(L.ctx, r.A, r.m, r.n, r.lda, r.b, r.s, w.r.sketch, r.seed, w.r.prec, r.x);
      else
        rc = rmc_rsvd(L.ctx, r.A, r.m, r.n, r.lda, r.k, r.p, r.q, r.seed, w.r.prec, r.U, r.k, r.sigma, r.V, r.k);
    }
    seal(L, rc);
    L.state.store(kEnqueued, std::memory_order_release);
  }
}

void post(Lane &L) {
  {
    std::lock_guard<std::mutex> lk(L.mu);
    L.state.store(kPosted, std::memory_order_release);
  }
  L.cv.notify_one();
}

void admit(rmc_server *srv) {
  for (auto &Lp : srv->lanes) {
    Lane &L = *Lp;
    if (L.state.load(std::memory_order_acquire) != kIdle) continue;
    if (srv->singles.empty() && srv->batchables.empty()) return;
    // the request that arrived first decides the launch
    if (!srv->singles.empty() &&
        (srv->batchables.empty() || srv->singles.front().ticket < srv->batchables.front().ticket)) {
      L.work.push_back(std::move(srv->singles.front()));
      srv->singles.pop_front();
      L.batch_job = false;
      post(L);
      continue;
    }
    // the batchable requests queued so far, in order, up to max_batch; halved until the launch fits the lane's
    // memory (one plan in the usual case)
    std::vector<rmc_request> &reqs = L.reqs;
    int take = (int)std::min<size_t>(srv->batchables.size(), (size_t)srv->max_batch);
    for (int i = 0; i < take; ++i) reqs.push_back(srv->batchables[i].r.req);
    while (take > 1 && rmc_batch_plan_bytes(reqs.data(), take) > srv->lane_budget) {
      take = (take + 1) / 2;
      reqs.resize(take);
    }
    for (int i = 0; i < take; ++i) {
      L.work.push_back(std::move(srv->batchables.front()));
      srv->batchables.pop_front();
    }
    L.batch_job = true;
    post(L);
  }
}

void stop_threads(rmc_server *srv) {
  for (auto &Lp : srv->lanes) {
    if (!Lp->thread.joinable()) continue;
    {
      std::lock_guard<std::mutex> lk(Lp->mu);
      Lp->stop = true;
    }
    Lp->cv.notify_one();
    Lp->thread.join();
  }
}

}  // namespace

extern "C" {

int rmc_server_create(rmc_server **out, size_t hbm_budget, int nstreams, int max_batch) {
  if (!out || nstreams < 1 || nstreams > 16 || max_batch < 1 || hbm_budget < size_t(nstreams) * (1u << 20))
    return RMC_EINVAL;
  *out = nullptr;
  rmc_server *srv = new (std::nothrow) rmc_server();
  if (!srv) return RMC_ENOMEM;
  srv->lane_budget = hbm_budget / nstreams;
  srv->max_batch = max_batch;
  if (cudaGetDevice(&srv->device) != cudaSuccess) {
    (void)cudaGetLastError();
    delete srv;
    return RMC_ECUDA;
  }
  for (int i = 0; i < nstreams; ++i) {
    srv->lanes.emplace_back(new (std::nothrow) Lane());
    if (!srv->lanes.back()) {
      srv->lanes.pop_back();
      rmc_server_destroy(srv);
      return RMC_ENOMEM;
    }
  }
  for (auto &Lp : srv->lanes) {
    Lane &L = *Lp;
    int rc = RMC_OK;
    if (cudaStreamCreateWithFlags(&L.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&L.done, cudaEventDisableTiming) != cudaSuccess) {
      (void)cudaGetLastError();
      rc = RMC_ECUDA;
    }
    if (rc == RMC_OK) rc = rmc_create(&L.ctx, L.stream, srv->lane_budget);
    if (rc != RMC_OK) {
      rmc_server_destroy(srv);
      return rc;
    }
  }
  try {
    for (auto &Lp : srv->lanes) Lp->thread = std::thread(lane_thread, srv, Lp.get());
  } catch (...) {
    rmc_server_destroy(srv);
    return RMC_ENOMEM;
  }
  *out = srv;
  return RMC_OK;
}

int rmc_server_destroy(rmc_server *srv) {
  if (!srv) return RMC_OK;
  int rc = RMC_OK;
  stop_threads(srv);   // a posted launch is issued before its thread stops
  for (auto &Lp : srv->lanes)
    if (Lp->stream && cudaStreamSynchronize(Lp->stream) != cudaSuccess) rc = RMC_ECUDA;
  if (!srv->lanes.empty() && srv->lanes[0]->stream) {
    for (Resident *e : srv->res) res_free(srv, e, srv->lanes[0]->stream);
    srv->res.clear();
    if (cudaStreamSynchronize(srv->lanes[0]->stream) != cudaSuccess) rc = RMC_ECUDA;
  }
  for (auto &Lp : srv->lanes) {
    Lane &L = *Lp;
    if (L.ctx) rmc_destroy(L.ctx);
    if (L.done) cudaEventDestroy(L.done);
    if (L.stream) cudaStreamDestroy(L.stream);
  }
  delete srv;
  return rc;
}

int rmc_server_submit(rmc_server *srv, const rmc_serve_request *req, uint64_t *ticket) {
  if (!srv || !req || !ticket) return RMC_EINVAL;
  Queued w;
  w.r = *req;
  const rmc_request &r = req->req;
  w.resident = srv->res_cap > 0 && r.kind == RMC_REQ_LSR;
  w.batch = !w.resident && batchable(*req);
  if (!w.batch && !valid_single(*req)) return RMC_EINVAL;
  rmc_ctx *ctx = srv->lanes[0]->ctx;   // plans read only the context's SM count
  float *p0, *p1, *p2;
  int *p3;
  void *p4;
  const size_t bytes = w.resident ? resident_plan(ctx, r, req->sketch, req->prec, &p0, &p1, &p2, &p3, &p4, nullptr)
                       : w.batch  ? rmc_batch_plan_bytes(&r, 1)
                       : r.kind == RMC_REQ_LSR
                           ? rmc_lsr_plan_bytes(ctx, r.m, r.n, r.s, req->sketch, req->prec)
                           : rmc_rsvd_plan_bytes(ctx, r.m, r.n, int64_t(r.k) + r.p, req->prec);
  if (bytes > srv->lane_budget) return RMC_ENOMEM;
  w.ticket = srv->next_ticket++;
  w.t_submit = Clock::now();
  *ticket = w.ticket;
  if (w.batch) srv->batchables.push_back(std::move(w));
  else srv->singles.push_back(std::move(w));
  return RMC_OK;
}

int rmc_server_progress(rmc_server *srv, int *inflight, int *queued) {
  if (!srv) return RMC_EINVAL;
  retire(srv);
  {
    std::lock_guard<std::mutex> lk(srv->res_mu);
    res_collect(srv);
  }
  admit(srv);
  if (inflight) {
    int n = 0;
    for (const auto &Lp : srv->lanes) n += (int)Lp->work.size();
    *inflight = n;
  }
  if (queued) *queued = (int)(srv->singles.size() + srv->batchables.size());
  return RMC_OK;
}

int rmc_server_poll(rmc_server *srv, uint64_t *tickets, int *status, double *latency_s, int max, int *count) {
  if (!srv || !count || max < 0 || (max > 0 && (!tickets || !status || !latency_s))) return RMC_EINVAL;
  const int n = (int)std::min<size_t>(size_t(max), srv->done.size());
  for (int i = 0; i < n; ++i) {
    tickets[i] = srv->done[i].ticket;
    status[i] = srv->done[i].status;
    latency_s[i] = srv->done[i].latency_s;
  }
  srv->done.erase(srv->done.begin(), srv->done.begin() + n);
  *count = n;
  return RMC_OK;
}

int rmc_server_resident(rmc_server *srv, size_t bytes) {
  if (!srv) return RMC_EINVAL;
  std::lock_guard<std::mutex> lk(srv->res_mu);
  srv->res_cap = bytes;
  // entries beyond the new cap (all of them for 0) are dropped as soon as no launch reads them
  size_t keep = 0;
  for (Resident *e : srv->res) {
    if (e->dead) continue;
    if (keep + e->bytes > bytes) e->dead = true;
    else keep += e->bytes;
  }
  res_collect(srv);
  return RMC_OK;
}

int rmc_server_release(rmc_server *srv, const float *A) {
  if (!srv || !A) return RMC_EINVAL;
  std::lock_guard<std::mutex> lk(srv->res_mu);
  for (Resident *e : srv->res)
    if (e->key.A == A) e->dead = true;
  res_collect(srv);
  return RMC_OK;
}

int rmc_server_drain(rmc_server *srv) {
  if (!srv) return RMC_EINVAL;
  for (;;) {
    int inflight = 0, queued = 0;
    RMC_TRY(rmc_server_progress(srv, &inflight, &queued));
    if (!inflight && !queued) return RMC_OK;
    std::this_thread::yield();
  }
}

}  // extern "C"
