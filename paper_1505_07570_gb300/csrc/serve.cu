// Continuous-batching request server (host code).
//
// Requests queue in arrival order.  Each stream ("lane") has its own context, whose workspace is capped at
// the lane's share of the HBM budget, and at most one launch in flight.  Whenever a lane is free the head of
// the queue is admitted: a request too large for the batched kernel runs alone through rmc_lsr_sketch or
// rmc_rsvd; otherwise every batchable request queued so far (in order, up to max_batch and the lane's memory)
// goes into one rmc_batch_run launch.  Requests that arrive while launches are in flight are admitted as soon
// as a lane frees up, so launches of different sizes overlap on the device.  Completion is seen by polling
// each lane's event; a request's latency runs from its submit call to the progress call that retires it.
//
// Results do not depend on the mix: a request always takes the same route (decided by its own size and
// precision), and both routes compute a problem with arithmetic that is independent of other problems.

#include <algorithm>
#include <chrono>
#include <deque>
#include <new>
#include <thread>
#include <vector>

#include "rmc_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct Queued {
  rmc_serve_request r;
  uint64_t ticket;
  Clock::time_point t_submit;
  bool batch;
};

struct Lane {
  cudaStream_t stream = nullptr;
  rmc_ctx *ctx = nullptr;
  cudaEvent_t done = nullptr;
  bool busy = false;
  int launch_status = RMC_OK;
  std::vector<Queued> work;  // the requests of the launch in flight
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
  std::vector<Lane> lanes;
  std::deque<Queued> queue;
  std::vector<Done> done;
};

namespace {

void retire(rmc_server *srv) {
  for (Lane &L : srv->lanes) {
    if (!L.busy) continue;
    const cudaError_t e = cudaEventQuery(L.done);
    if (e == cudaErrorNotReady) continue;
    int st = e == cudaSuccess ? L.launch_status : RMC_ECUDA;
    if (e != cudaSuccess) (void)cudaGetLastError();
    if (st == RMC_OK && *L.ctx->h_status != RMC_OK) st = *L.ctx->h_status;
    const Clock::time_point now = Clock::now();
    for (const Queued &w : L.work)
      srv->done.push_back({w.ticket, st, std::chrono::duration<double>(now - w.t_submit).count()});
    L.work.clear();
    L.busy = false;
  }
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
  L.busy = true;
}

void launch_single(Lane &L, Queued &&w) {
  const rmc_request &r = w.r.req;
  int rc;
  if (r.kind == RMC_REQ_LSR)
    rc = rmc_lsr_sketch(L.ctx, r.A, r.m, r.n, r.lda, r.b, r.s, w.r.sketch, r.seed, w.r.prec, r.x);
  else
    rc = rmc_rsvd(L.ctx, r.A, r.m, r.n, r.lda, r.k, r.p, r.q, r.seed, w.r.prec, r.U, r.k, r.sigma, r.V, r.k);
  L.work.push_back(std::move(w));
  seal(L, rc);
}

void admit(rmc_server *srv) {
  for (Lane &L : srv->lanes) {
    if (L.busy) continue;
    if (srv->queue.empty()) return;
    if (!srv->queue.front().batch) {
      Queued w = std::move(srv->queue.front());
      srv->queue.pop_front();
      launch_single(L, std::move(w));
      continue;
    }
    // every batchable request queued so far, in order, while the launch fits the lane's memory
    std::vector<rmc_request> reqs;
    for (auto it = srv->queue.begin(); it != srv->queue.end() && (int)reqs.size() < srv->max_batch;) {
      if (!it->batch) {
        ++it;
        continue;
      }
      reqs.push_back(it->r.req);
      if (reqs.size() > 1 && rmc_batch_plan_bytes(reqs.data(), (int)reqs.size()) > srv->lane_budget) {
        reqs.pop_back();
        break;
      }
      L.work.push_back(std::move(*it));
      it = srv->queue.erase(it);
    }
    seal(L, rmc_batch_run(L.ctx, reqs.data(), (int)reqs.size()));
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
  srv->lanes.resize(nstreams);
  for (Lane &L : srv->lanes) {
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
  *out = srv;
  return RMC_OK;
}

int rmc_server_destroy(rmc_server *srv) {
  if (!srv) return RMC_OK;
  int rc = RMC_OK;
  for (Lane &L : srv->lanes) {
    if (L.stream && cudaStreamSynchronize(L.stream) != cudaSuccess) rc = RMC_ECUDA;
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
  w.batch = batchable(*req);
  if (!w.batch && !valid_single(*req)) return RMC_EINVAL;
  const rmc_request &r = req->req;
  rmc_ctx *ctx = srv->lanes[0].ctx;
  const size_t bytes = w.batch ? rmc_batch_plan_bytes(&r, 1)
                       : r.kind == RMC_REQ_LSR
                           ? rmc_lsr_plan_bytes(ctx, r.m, r.n, r.s, req->sketch, req->prec)
                           : rmc_rsvd_plan_bytes(ctx, r.m, r.n, int64_t(r.k) + r.p, req->prec);
  if (bytes > srv->lane_budget) return RMC_ENOMEM;
  w.ticket = srv->next_ticket++;
  w.t_submit = Clock::now();
  *ticket = w.ticket;
  srv->queue.push_back(std::move(w));
  return RMC_OK;
}

int rmc_server_progress(rmc_server *srv, int *inflight, int *queued) {
  if (!srv) return RMC_EINVAL;
  retire(srv);
  admit(srv);
  if (inflight) {
    int n = 0;
    for (const Lane &L : srv->lanes) n += (int)L.work.size();
    *inflight = n;
  }
  if (queued) *queued = (int)srv->queue.size();
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
