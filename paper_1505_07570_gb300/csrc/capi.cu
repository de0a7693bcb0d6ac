// The C ABI: context, workspace, status word, argument checks and the sequence of kernels behind each call.
#include <cmath>
#include <cstdlib>
#include <new>

#include "rmc_internal.cuh"

namespace {

constexpr size_t kDefaultBudget = size_t(64) << 30;

bool bad_ld(int64_t ld, int64_t cols) { return ld < cols || ld < 1; }

int64_t next_pow2(int64_t m) {
  int64_t N = 1;
  while (N < m) N <<= 1;
  return N;
}

}  // namespace

int rmc_ws_reserve(rmc_ctx *ctx, size_t bytes) {
  if (bytes <= ctx->ws_bytes) return RMC_OK;
  if (bytes > ctx->budget) return RMC_ENOMEM;
  size_t want = bytes + bytes / 4;  // grow with headroom so a sequence of calls settles quickly
  if (want > ctx->budget) want = ctx->budget;
  if (ctx->ws) {
    RMC_TRY_CUDA(cudaFreeAsync(ctx->ws, ctx->stream));
    ctx->ws = nullptr;
    ctx->ws_bytes = 0;
  }
  void *p = nullptr;
  if (cudaMallocAsync(&p, want, ctx->stream) != cudaSuccess) {
    (void)cudaGetLastError();
    return RMC_ENOMEM;
  }
  ctx->ws = p;
  ctx->ws_bytes = want;
  return RMC_OK;
}

extern "C" {

int rmc_create(rmc_ctx **out, void *stream, size_t budget) {
  if (!out) return RMC_EINVAL;
  *out = nullptr;
  rmc_ctx *ctx = new (std::nothrow) rmc_ctx();
  if (!ctx) return RMC_ENOMEM;
  ctx->stream = static_cast<cudaStream_t>(stream);
  ctx->budget = budget ? budget : kDefaultBudget;
  if (cudaGetDevice(&ctx->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device) != cudaSuccess ||
      cudaMalloc(&ctx->d_status, sizeof(int)) != cudaSuccess ||
      cudaMallocHost(&ctx->h_status, sizeof(int)) != cudaSuccess ||
      cudaMemset(ctx->d_status, 0, sizeof(int)) != cudaSuccess) {
    (void)cudaGetLastError();
    if (ctx->d_status) cudaFree(ctx->d_status);
    if (ctx->h_status) cudaFreeHost(ctx->h_status);
    delete ctx;
    return RMC_ECUDA;
  }
  *out = ctx;
  return RMC_OK;
}

int rmc_destroy(rmc_ctx *ctx) {
  if (!ctx) return RMC_OK;
  int rc = RMC_OK;
  if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) rc = RMC_ECUDA;
  if (ctx->stage_ev) cudaEventDestroy(ctx->stage_ev);
  if (ctx->h_stage) cudaFreeHost(ctx->h_stage);
  if (ctx->prof_recs) {
    for (int r = 0; r < ctx->prof_cap; ++r) {
      cudaEventDestroy(ctx->prof_recs[r].start);
      cudaEventDestroy(ctx->prof_recs[r].stop);
    }
    delete[] ctx->prof_recs;
  }
  delete[] ctx->span_tag;
  delete[] ctx->span_start;
  delete[] ctx->span_stop;
  if (ctx->ws) cudaFree(ctx->ws);
  cudaFree(ctx->d_status);
  cudaFreeHost(ctx->h_status);
  (void)cudaGetLastError();
  delete ctx;
  return rc;
}

int rmc_set_stream(rmc_ctx *ctx, void *stream) {
  if (!ctx) return RMC_EINVAL;
  // Work already enqueued on the old stream may still use the workspace: order the new stream after it.
  cudaEvent_t ev;
  RMC_TRY_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  cudaError_t e = cudaEventRecord(ev, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(static_cast<cudaStream_t>(stream), ev, 0);
  cudaEventDestroy(ev);
  RMC_TRY_CUDA(e);
  ctx->stream = static_cast<cudaStream_t>(stream);
  return RMC_OK;
}

int rmc_sync(rmc_ctx *ctx) {
  if (!ctx) return RMC_EINVAL;
  RMC_TRY_CUDA(cudaMemcpyAsync(ctx->h_status, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  RMC_TRY_CUDA(cudaMemsetAsync(ctx->d_status, 0, sizeof(int), ctx->stream));
  RMC_TRY_CUDA(cudaStreamSynchronize(ctx->stream));
  return *ctx->h_status;
}

const char *rmc_status_string(int status) {
  switch (status) {
    case RMC_OK: return "ok";
    case RMC_EINVAL: return "invalid argument";
    case RMC_EALIGN: return "misaligned pointer or leading dimension for a TMA-fed path";
    case RMC_ENOMEM: return "workspace exceeds the HBM budget or allocation failed";
    case RMC_ENUMERIC: return "numerical breakdown (non-positive pivot or no Jacobi convergence)";
    case RMC_ETIMEOUT: return "a bounded device wait expired";
    case RMC_ECUDA: return "CUDA runtime error";
    case RMC_PENDING: return "pending";
    case RMC_ESCRATCH: return "needs more than the fixed scratch of the no-allocation entry point";
    default: return "unknown status";
  }
}

int rmc_set_option(rmc_ctx *ctx, int option, int value) {
  if (!ctx) return RMC_EINVAL;
  switch (option) {
    case RMC_OPT_SMALL_FP64:
      if (value != 0 && value != 1) return RMC_EINVAL;
      ctx->small_fp64 = value != 0;
      return RMC_OK;
    default:
      return RMC_EINVAL;
  }
}

int rmc_get_option(const rmc_ctx *ctx, int option, int *value) {
  if (!ctx || !value) return RMC_EINVAL;
  switch (option) {
    case RMC_OPT_SMALL_FP64: *value = ctx->small_fp64 ? 1 : 0; return RMC_OK;
    default: return RMC_EINVAL;
  }
}

int rmc_workspace_bytes(const rmc_ctx *ctx, size_t *bytes) {
  if (!ctx || !bytes) return RMC_EINVAL;
  *bytes = ctx->ws_bytes;
  return RMC_OK;
}

// ------------------------------------------------------------------------------------------------ sketch

int rmc_check_sketch_args(const float *A, int64_t m, int64_t n, int64_t lda, int64_t s, int kind, int prec) {
  if (!A || m < 1 || n < 1 || bad_ld(lda, n) || s < 1) return RMC_EINVAL;
  if (kind != RMC_GAUSSIAN && kind != RMC_SRHT && kind != RMC_COUNTSKETCH) return RMC_EINVAL;
  if (!rmc_prec_ok(prec)) return RMC_EINVAL;
  if (kind == RMC_GAUSSIAN && prec == RMC_TF32X3) return RMC_EINVAL;   // no split form of the drawn sketch
  if (kind == RMC_SRHT && s > next_pow2(m)) return RMC_EINVAL;
  if (m > (int64_t(1) << 31) || s > (int64_t(1) << 31)) return RMC_EINVAL;
  return RMC_OK;
}

size_t rmc_sketch_plan_bytes(rmc_ctx *ctx, int64_t m, int64_t ntot, int64_t s, int kind, int prec) {
  switch (kind) {
    case RMC_GAUSSIAN: return rmc_gauss_ws(m, ntot, s, prec, ctx->num_sms);
    case RMC_SRHT: return rmc_srht_ws(m, ntot, s, ctx->num_sms);
    default: return rmc_countsketch_ws(m, s);
  }
}

// Sketch A (and b, when given, as one more column of the same operator) into C (and Cb).
int rmc_run_sketch(rmc_ctx *ctx, const float *A, int64_t m, int64_t n, int64_t lda, const float *b, int64_t s,
                      int kind, uint64_t seed, int prec, float *C, int64_t ldc, float *Cb, void *ws) {
  switch (kind) {
    case RMC_GAUSSIAN:
      return rmc_launch_gauss_sketch(ctx, A, m, n, lda, b, s, seed, 0, prec, C, ldc, Cb, ws);
    case RMC_SRHT:
      return rmc_launch_srht(ctx, A, m, n, lda, b, s, seed, 0, C, ldc, Cb, ws);
    default:
      return rmc_launch_countsketch(ctx, A, m, n, lda, b, s, seed, 0, C, ldc, Cb, ws);
  }
}

int rmc_sketch(rmc_ctx *ctx, const float *A, int64_t m, int64_t n, int64_t lda, int64_t s, int kind, uint64_t seed,
               int prec, float *C, int64_t ldc) {
  if (!ctx || !C || bad_ld(ldc, n)) return RMC_EINVAL;
  RMC_TRY(rmc_check_sketch_args(A, m, n, lda, s, kind, prec));
  RMC_TRY(rmc_ws_reserve(ctx, rmc_sketch_plan_bytes(ctx, m, n, s, kind, prec)));
  return rmc_run_sketch(ctx, A, m, n, lda, nullptr, s, kind, seed, prec, C, ldc, nullptr, ctx->ws);
}

// Workspace plan of rmc_lsr_sketch: [S^T A, S^T b] (s x (n+1)), S^T b, then the larger of the sketch's and
// the solve's scratch.
static size_t lsr_rest_bytes(rmc_ctx *ctx, int64_t m, int64_t n, int64_t s, int kind, int prec) {
  size_t rest = rmc_sketch_plan_bytes(ctx, m, n + 1, s, kind, prec);
  const size_t solve = rmc_lsr_solve_ws(s, n, ctx->num_sms);
  return solve > rest ? solve : rest;
}

static void lsr_carve(WsCarve &w, int64_t n, int64_t s, size_t rest_bytes, float **SAb, float **Sb, void **rest) {
  *SAb = w.take<float>(size_t(s) * (n + 1));
  *Sb = w.take<float>(size_t(s));
  *rest = w.take<char>(rest_bytes);
}

size_t rmc_lsr_plan_bytes(rmc_ctx *ctx, int64_t m, int64_t n, int64_t s, int kind, int prec) {
  float *SAb, *Sb;
  void *rest;
  WsCarve plan;
  lsr_carve(plan, n, s, lsr_rest_bytes(ctx, m, n, s, kind, prec), &SAb, &Sb, &rest);
  return plan.off;
}

int rmc_lsr_sketch(rmc_ctx *ctx, const float *A, int64_t m, int64_t n, int64_t lda, const float *b, int64_t s,
                   int kind, uint64_t seed, int prec, double *x) {
  if (!ctx || !b || !x) return RMC_EINVAL;
  RMC_TRY(rmc_check_sketch_args(A, m, n, lda, s, kind, prec));
  if (s < n || n > 1024) return RMC_EINVAL;
  const size_t rest_bytes = lsr_rest_bytes(ctx, m, n, s, kind, prec);
  float *SAb, *Sb;
  void *rest;
  WsCarve plan;
  lsr_carve(plan, n, s, rest_bytes, &SAb, &Sb, &rest);
  RMC_TRY(rmc_ws_reserve(ctx, plan.off));
  WsCarve w;
  w.base = static_cast<char *>(ctx->ws);
  lsr_carve(w, n, s, rest_bytes, &SAb, &Sb, &rest);
  // [S^T A, S^T b] is kept as one s x (n+1) matrix; S^T b is sketched into its own vector first.
  RMC_TRY(rmc_run_sketch(ctx, A, m, n, lda, b, s, kind, seed, prec, SAb, n + 1, Sb, rest));
  return rmc_launch_lsr_solve(ctx, SAb, s, n, n + 1, Sb, x, rest);
}

// -------------------------------------------------------------------------------------------------- rsvd

// Workspace plan of rmc_rsvd: Omega (n x l), Y/Q (m x l), Z (n x l), B (l x n), Ub (l x l), sigma (l),
// Vb (n x l), then the largest scratch of its steps.
static size_t rsvd_scratch_bytes(rmc_ctx *ctx, int64_t m, int64_t n, int64_t l, int gp) {
  size_t scratch = rmc_cholqr2_ws(m > n ? m : n, l, ctx->num_sms);
  size_t t = rmc_matmul_ws(m, n, l, 0, gp, ctx->num_sms);
  if (t > scratch) scratch = t;
  t = rmc_matmul_ws(m, n, l, 1, gp, ctx->num_sms);
  if (t > scratch) scratch = t;
  t = rmc_svd_wide_ws(l, n, ctx->num_sms);
  return t > scratch ? t : scratch;
}

static void rsvd_carve(WsCarve &w, int64_t m, int64_t n, int64_t l, size_t scratch, float **Om, float **Y, float **Z,
                       float **B, float **Ub, float **sg, float **Vb, void **scr) {
  *Om = w.take<float>(size_t(n) * l);
  *Y = w.take<float>(size_t(m) * l);
  *Z = w.take<float>(size_t(n) * l);
  *B = w.take<float>(size_t(l) * n);
  *Ub = w.take<float>(size_t(l) * l);
  *sg = w.take<float>(size_t(l));
  *Vb = w.take<float>(size_t(n) * l);
  *scr = w.take<char>(scratch);
}

static int rsvd_gemm_prec(int prec) { return prec; }

size_t rmc_rsvd_plan_bytes(rmc_ctx *ctx, int64_t m, int64_t n, int64_t l, int prec) {
  float *Om, *Y, *Z, *B, *Ub, *sg, *Vb;
  void *scr;
  WsCarve plan;
  rsvd_carve(plan, m, n, l, rsvd_scratch_bytes(ctx, m, n, l, rsvd_gemm_prec(prec)), &Om, &Y, &Z, &B, &Ub, &sg, &Vb,
             &scr);
  return plan.off;
}

int rmc_rsvd(rmc_ctx *ctx, const float *A, int64_t m, int64_t n, int64_t lda, int k, int p, int q, uint64_t seed,
             int prec, float *U, int64_t ldu, float *sigma, float *V, int64_t ldv) {
  if (!ctx || !A || !U || !sigma || !V) return RMC_EINVAL;
  const int64_t l = int64_t(k) + p;
  if (k < 1 || p < 0 || q < 0 || m < 1 || n < 1 || bad_ld(lda, n) || l > m || l > n || l > 256) return RMC_EINVAL;
  if (bad_ld(ldu, k) || bad_ld(ldv, k)) return RMC_EINVAL;
  if (!rmc_prec_ok(prec)) return RMC_EINVAL;
  const int gp = rsvd_gemm_prec(prec);

  float *Om, *Y, *Z, *B, *Ub, *sg, *Vb;
  void *scr;
  const size_t scratch = rsvd_scratch_bytes(ctx, m, n, l, gp);
  WsCarve plan;
  rsvd_carve(plan, m, n, l, scratch, &Om, &Y, &Z, &B, &Ub, &sg, &Vb, &scr);
  RMC_TRY(rmc_ws_reserve(ctx, plan.off));
  WsCarve w;
  w.base = static_cast<char *>(ctx->ws);
  rsvd_carve(w, m, n, l, scratch, &Om, &Y, &Z, &B, &Ub, &sg, &Vb, &scr);

  cudaStream_t st = ctx->stream;
  RMC_TRY(rmc_launch_gaussian(st, seed, 0, n, l, Om, l, 1.0f));                  // Omega, n x l
  // Intermediate bases only need to be well conditioned (one CholeskyQR pass); the basis that B = Q^T A is
  // formed with is orthonormalised by CholeskyQR2.
  RMC_TRY(rmc_launch_matmul_an(ctx, A, m, n, lda, Om, l, l, gp, Y, l, scr));      // Y = A Omega
  RMC_TRY(rmc_launch_cholqr2(ctx, Y, m, l, l, nullptr, scr, q == 0 ? 2 : 1));    // Q = orth(Y)
  for (int it = 0; it < q; ++it) {
    RMC_TRY(rmc_launch_matmul_at(ctx, A, m, n, lda, Y, l, l, gp, B, n, scr));     // B = Q^T A  (l x n)
    RMC_TRY(rmc_launch_transpose(st, B, l, n, n, Z, l));                           // Z = B^T    (n x l)
    RMC_TRY(rmc_launch_cholqr2(ctx, Z, n, l, l, nullptr, scr, 1));                // Z = orth(A^T Q)
    RMC_TRY(rmc_launch_matmul_an(ctx, A, m, n, lda, Z, l, l, gp, Y, l, scr));     // Y = A Z
    RMC_TRY(rmc_launch_cholqr2(ctx, Y, m, l, l, nullptr, scr, it == q - 1 ? 2 : 1));  // Q = orth(Y)
  }
  RMC_TRY(rmc_launch_matmul_at(ctx, A, m, n, lda, Y, l, l, gp, B, n, scr));       // B = Q^T A
  RMC_TRY(rmc_launch_svd_wide(ctx, B, l, n, n, Ub, sg, Vb, l, scr));              // B = Ub S Vb^T
  return rmc_launch_rsvd_finish(ctx, Y, m, l, Ub, sg, Vb, n, k, U, ldu, sigma, V, ldv, scr);
}

// ------------------------------------------------------------------------------------------ step entries

int rmc_philox(rmc_ctx *ctx, uint64_t seed, uint32_t stream, uint32_t instance, uint64_t first, int64_t count,
               uint32_t *out) {
  if (!ctx || !out || count < 0) return RMC_EINVAL;
  return rmc_launch_philox(ctx->stream, seed, stream, instance, first, count, out);
}

int rmc_gaussian_matrix(rmc_ctx *ctx, uint64_t seed, uint32_t instance, int64_t rows, int64_t cols, float *out,
                        int64_t ld) {
  if (!ctx || !out || rows < 0 || cols < 0 || bad_ld(ld, cols)) return RMC_EINVAL;
  return rmc_launch_gaussian(ctx->stream, seed, instance, rows, cols, out, ld, 1.0f);
}

int rmc_countsketch_hash(rmc_ctx *ctx, uint64_t seed, uint32_t instance, int64_t m, int64_t s, int32_t *bucket,
                         float *sign) {
  if (!ctx || !bucket || !sign || m < 0 || s < 1 || s > (int64_t(1) << 31)) return RMC_EINVAL;
  return rmc_launch_cs_hash(ctx->stream, seed, instance, m, s, bucket, sign);
}

int rmc_srht_sample(rmc_ctx *ctx, uint64_t seed, uint32_t instance, int64_t N, int64_t s, int64_t *idx) {
  if (!ctx || !idx || N < 1 || s < 1 || s > N || N > (int64_t(1) << 31)) return RMC_EINVAL;
  RMC_TRY(rmc_ws_reserve(ctx, rmc_srht_sample_ws(N)));
  return rmc_launch_srht_sample(ctx, seed, instance, N, s, idx, ctx->ws);
}

int rmc_cholqr2(rmc_ctx *ctx, float *Y, int64_t m, int64_t l, int64_t ldy, double *R) {
  if (!ctx || !Y || l < 1 || l > 256 || m < l || bad_ld(ldy, l)) return RMC_EINVAL;
  RMC_TRY(rmc_ws_reserve(ctx, rmc_cholqr2_ws(m, l, ctx->num_sms)));
  return rmc_launch_cholqr2(ctx, Y, m, l, ldy, R, ctx->ws);
}

int rmc_svd_wide(rmc_ctx *ctx, const float *B, int64_t l, int64_t n, int64_t ldb, float *Ub, float *sigma,
                 float *Vb, int64_t ldv) {
  if (!ctx || !B || !Ub || !sigma || !Vb || l < 1 || l > 256 || n < l || bad_ld(ldb, n) || bad_ld(ldv, l))
    return RMC_EINVAL;
  RMC_TRY(rmc_ws_reserve(ctx, rmc_svd_wide_ws(l, n, ctx->num_sms)));
  return rmc_launch_svd_wide(ctx, B, l, n, ldb, Ub, sigma, Vb, ldv, ctx->ws);
}

int rmc_matmul_an(rmc_ctx *ctx, const float *A, int64_t m, int64_t n, int64_t lda, const float *X, int64_t l,
                  int64_t ldx, int prec, float *Y, int64_t ldy) {
  if (!ctx || !A || !X || !Y || m < 1 || n < 1 || l < 1 || l > 256 || bad_ld(lda, n) || bad_ld(ldx, l) ||
      bad_ld(ldy, l) || !rmc_prec_ok(prec))
    return RMC_EINVAL;
  RMC_TRY(rmc_ws_reserve(ctx, rmc_matmul_ws(m, n, l, 0, prec, ctx->num_sms)));
  return rmc_launch_matmul_an(ctx, A, m, n, lda, X, l, ldx, prec, Y, ldy, ctx->ws);
}

int rmc_matmul_at(rmc_ctx *ctx, const float *A, int64_t m, int64_t n, int64_t lda, const float *X, int64_t l,
                  int64_t ldx, int prec, float *W, int64_t ldw) {
  if (!ctx || !A || !X || !W || m < 1 || n < 1 || l < 1 || l > 256 || bad_ld(lda, n) || bad_ld(ldx, l) ||
      bad_ld(ldw, n) || !rmc_prec_ok(prec))
    return RMC_EINVAL;
  RMC_TRY(rmc_ws_reserve(ctx, rmc_matmul_ws(m, n, l, 1, prec, ctx->num_sms)));
  return rmc_launch_matmul_at(ctx, A, m, n, lda, X, l, ldx, prec, W, ldw, ctx->ws);
}

}  // extern "C"

// ------------------------------------------------------------------------------------ timeout delivery

namespace {

// One thread polls a flag that nothing sets, with the same kind of bound as every wait in the library (the
// global nanosecond timer), then reports RMC_ETIMEOUT and returns: no trap, the context stays usable.
__global__ void wait_never_set_kernel(const volatile int *flag, uint64_t limit_ns, int *status) {
  uint64_t t0;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  for (uint32_t i = 0;; ++i) {
    if (*flag) return;
    if ((i & 63) == 0) {
      uint64_t t;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
      if (t - t0 > limit_ns) {
        rmc_report(status, RMC_ETIMEOUT);
        return;
      }
    }
  }
}

}  // namespace

extern "C" int rmc_debug_wait_timeout(rmc_ctx *ctx, uint64_t limit_ns) {
  if (!ctx || limit_ns > 1000000000ull) return RMC_EINVAL;
  RMC_TRY(rmc_ws_reserve(ctx, 256));
  RMC_TRY_CUDA(cudaMemsetAsync(ctx->ws, 0, sizeof(int), ctx->stream));
  wait_never_set_kernel<<<1, 1, 0, ctx->stream>>>(static_cast<const int *>(ctx->ws), limit_ns, ctx->d_status);
  rmc_note_launch();
  RMC_LAUNCH_CHECK();
  return RMC_OK;
}

// ------------------------------------------------------------------------------------ measurement hooks

#include <atomic>

static std::atomic<uint64_t> g_launches{0};

void rmc_note_launch(int count) { g_launches.fetch_add((uint64_t)count, std::memory_order_relaxed); }

RmcProf::RmcProf(rmc_ctx *c, int tag) : ctx(c), rec(-1) {
  if (!ctx || !ctx->prof || ctx->prof_used >= ctx->prof_cap) return;
  rec = ctx->prof_used++;
  ctx->prof_recs[rec].tag = tag;
  cudaEventRecord(ctx->prof_recs[rec].start, ctx->stream);
}

RmcProf::~RmcProf() {
  if (rec >= 0) cudaEventRecord(ctx->prof_recs[rec].stop, ctx->stream);
}

// Process-wide reference event of the launch intervals (recorded by rmc_profile_reference).
static cudaEvent_t g_prof_ref = nullptr;
static bool g_prof_ref_recorded = false;

// Fold finished records into the per-tag totals (and, once a reference is recorded, the interval list) and
// recycle their events.
static int prof_drain(rmc_ctx *ctx) {
  RMC_TRY_CUDA(cudaStreamSynchronize(ctx->stream));
  for (int r = 0; r < ctx->prof_used; ++r) {
    float ms = 0.f;
    RMC_TRY_CUDA(cudaEventElapsedTime(&ms, ctx->prof_recs[r].start, ctx->prof_recs[r].stop));
    const int tag = ctx->prof_recs[r].tag;
    ctx->prof_launches[tag] += 1;
    ctx->prof_ms[tag] += ms;
    if (g_prof_ref_recorded && ctx->prof_nspans < ctx->prof_cap) {
      float t0 = 0.f, t1 = 0.f;
      // a launch recorded before the reference has no interval (the elapsed time would be negative)
      if (cudaEventElapsedTime(&t0, g_prof_ref, ctx->prof_recs[r].start) == cudaSuccess &&
          cudaEventElapsedTime(&t1, g_prof_ref, ctx->prof_recs[r].stop) == cudaSuccess && t0 >= 0.f) {
        ctx->span_tag[ctx->prof_nspans] = tag;
        ctx->span_start[ctx->prof_nspans] = t0;
        ctx->span_stop[ctx->prof_nspans] = t1;
        ++ctx->prof_nspans;
      } else {
        (void)cudaGetLastError();
      }
    }
  }
  ctx->prof_used = 0;
  return RMC_OK;
}

extern "C" {

int rmc_profile_begin(rmc_ctx *ctx) {
  if (!ctx) return RMC_EINVAL;
  if (!ctx->prof_recs) {
    const int cap = 4096;
    ctx->prof_recs = new (std::nothrow) RmcProfRec[cap];
    if (!ctx->prof_recs) return RMC_ENOMEM;
    ctx->span_tag = new (std::nothrow) int[cap];
    ctx->span_start = new (std::nothrow) double[cap];
    ctx->span_stop = new (std::nothrow) double[cap];
    if (!ctx->span_tag || !ctx->span_start || !ctx->span_stop) return RMC_ENOMEM;
    for (int r = 0; r < cap; ++r) {
      RMC_TRY_CUDA(cudaEventCreate(&ctx->prof_recs[r].start));
      RMC_TRY_CUDA(cudaEventCreate(&ctx->prof_recs[r].stop));
    }
    ctx->prof_cap = cap;
  }
  RMC_TRY_CUDA(cudaStreamSynchronize(ctx->stream));
  ctx->prof_used = 0;
  ctx->prof_nspans = 0;
  for (int t = 0; t < RMC_K_NTAGS; ++t) {
    ctx->prof_launches[t] = 0;
    ctx->prof_ms[t] = 0.0;
  }
  ctx->prof = true;
  return RMC_OK;
}

int rmc_profile_read(rmc_ctx *ctx, int tag, int64_t *launches, double *total_ms) {
  if (!ctx || tag < 0 || tag >= RMC_K_NTAGS || !launches || !total_ms) return RMC_EINVAL;
  RMC_TRY(prof_drain(ctx));
  *launches = ctx->prof_launches[tag];
  *total_ms = ctx->prof_ms[tag];
  return RMC_OK;
}

int rmc_profile_reference(rmc_ctx *ctx) {
  if (!ctx) return RMC_EINVAL;
  if (!g_prof_ref) RMC_TRY_CUDA(cudaEventCreate(&g_prof_ref));
  RMC_TRY_CUDA(cudaEventRecord(g_prof_ref, ctx->stream));
  g_prof_ref_recorded = true;
  return RMC_OK;
}

int rmc_profile_spans(rmc_ctx *ctx, int tag, double *start_ms, double *stop_ms, int max, int *count) {
  if (!ctx || tag < 0 || tag >= RMC_K_NTAGS || !count || max < 0 || (max > 0 && (!start_ms || !stop_ms)))
    return RMC_EINVAL;
  if (!g_prof_ref_recorded) return RMC_EINVAL;
  RMC_TRY(prof_drain(ctx));
  int n = 0;
  for (int i = 0; i < ctx->prof_nspans && n < max; ++i)
    if (ctx->span_tag[i] == tag) {
      start_ms[n] = ctx->span_start[i];
      stop_ms[n] = ctx->span_stop[i];
      ++n;
    }
  *count = n;
  return RMC_OK;
}

int rmc_profile_end(rmc_ctx *ctx) {
  if (!ctx) return RMC_EINVAL;
  RMC_TRY(prof_drain(ctx));
  ctx->prof = false;
  return RMC_OK;
}

int rmc_launch_counter(uint64_t *launches) {
  if (!launches) return RMC_EINVAL;
  *launches = g_launches.load(std::memory_order_relaxed);
  return RMC_OK;
}

}  // extern "C"
