// Internal declarations shared by the library's translation units: the context, workspace carving, the
// device status word, and the launchers each .cu file provides.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include "../../include/rmc.h"

constexpr int kBatchTileClasses = 16;   // k-SVD tuning classes of the batched kernel: 4 n classes x 4 l classes

struct RmcProfRec {
  int tag;
  cudaEvent_t start, stop;
};

struct rmc_ctx {
  cudaStream_t stream;
  size_t budget;        // cap on workspace bytes
  void *ws;             // device workspace (stream-ordered allocation)
  size_t ws_bytes;
  int *d_status;        // device status word: 0 or the first RMC_E* a kernel reported
  int *h_status;        // pinned host copy
  int device;
  int num_sms;
  bool small_fp64;      // RMC_OPT_SMALL_FP64: CholeskyQR2 Gram products, Cholesky and Jacobi SVD in FP64
  int batch_rtile[kBatchTileClasses];  // tuned row-tile height per k-SVD class of rmc_batch_run (0 = default)
  // measurement hooks
  bool prof;
  int prof_used, prof_cap;
  RmcProfRec *prof_recs;
  int64_t prof_launches[RMC_K_NTAGS];
  double prof_ms[RMC_K_NTAGS];
  int prof_nspans;      // drained launch intervals relative to the process-wide reference event
  int *span_tag;
  double *span_start, *span_stop;
  // pinned staging for host-built descriptors (batched launches); reused once stage_ev has completed
  void *h_stage;
  size_t h_stage_bytes;
  cudaEvent_t stage_ev;
};

// Count kernel launches (process-wide).
void rmc_note_launch(int count = 1);

// Bracket one launch with CUDA events when the context is profiling.
struct RmcProf {
  rmc_ctx *ctx;
  int rec;
  RmcProf(rmc_ctx *c, int tag);
  ~RmcProf();
};

// Operand precisions of the products with A (FP32 CUDA cores; TF32, 3xTF32 and BF16 tensor cores).
static inline bool rmc_prec_ok(int prec) {
  return prec == RMC_FP32 || prec == RMC_TF32 || prec == RMC_TF32X3 || prec == RMC_BF16;
}

#define RMC_TRY_CUDA(expr)                                   \
  do {                                                       \
    cudaError_t e_ = (expr);                                 \
    if (e_ != cudaSuccess) { (void)cudaGetLastError(); return RMC_ECUDA; } \
  } while (0)

#define RMC_TRY(expr)                                        \
  do { int r_ = (expr); if (r_ != RMC_OK) return r_; } while (0)

#define RMC_LAUNCH_CHECK() RMC_TRY_CUDA(cudaGetLastError())

// Make sure the context holds at least `bytes` of workspace (grows stream-ordered, never shrinks).
int rmc_ws_reserve(rmc_ctx *ctx, size_t bytes);

// Bump allocator over the workspace: carve once without a base to learn the total, reserve, then carve again
// with the real base in the same order.
struct WsCarve {
  size_t off = 0;
  char *base = nullptr;
  template <typename T> T *take(size_t count) {
    off = (off + 255) & ~size_t(255);
    T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
    off += count * sizeof(T);
    return p;
  }
};

// Device-side error report: the first error wins.
__device__ __forceinline__ void rmc_report(int *status, int code) {
  if (status) atomicCAS(status, 0, code);
}

// Allow `bytes` of dynamic shared memory for `kern`.  The cap is only ever raised, straight to the device's
// opt-in maximum: launches issued from several host threads at once (the request server's lanes, or callers'
// own threads) then never find it lowered below their own request by another thread's smaller problem.
template <typename K>
inline cudaError_t rmc_allow_smem(K kern, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  cudaFuncAttributes a;
  cudaError_t e = cudaFuncGetAttributes(&a, kern);
  if (e != cudaSuccess) return e;
  if ((size_t)a.maxDynamicSharedSizeBytes >= bytes) return cudaSuccess;
  int dev = 0, optin = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess) return e;
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)a.sharedSizeBytes);
}

static inline unsigned rmc_blocks(int64_t work, int per_block, int64_t cap = 1 << 30) {
  int64_t b = (work + per_block - 1) / per_block;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return (unsigned)b;
}

// ---------------------------------------------------------------------------------------- launchers
// rng.cu
int rmc_launch_philox(cudaStream_t st, uint64_t seed, uint32_t stream_id, uint32_t instance, uint64_t first,
                      int64_t count, uint32_t *out);
int rmc_launch_gaussian(cudaStream_t st, uint64_t seed, uint32_t instance, int64_t rows, int64_t cols,
                        float *out, int64_t ld, float scale);
int rmc_launch_gaussian_t(cudaStream_t st, uint64_t seed, uint32_t instance, int64_t rows, int64_t cols,
                          float *out_t, int64_t ld_t, float scale);
int rmc_launch_cs_hash(cudaStream_t st, uint64_t seed, uint32_t instance, int64_t m, int64_t s,
                       int32_t *bucket, float *sign);
size_t rmc_srht_sample_ws(int64_t N);
int rmc_launch_srht_sample(rmc_ctx *ctx, uint64_t seed, uint32_t instance, int64_t N, int64_t s, int64_t *idx,
                           void *ws);

// countsketch.cu
size_t rmc_countsketch_ws(int64_t m, int64_t s);
int rmc_launch_countsketch(rmc_ctx *ctx, const float *A, int64_t m, int64_t n, int64_t lda, const float *b,
                           int64_t s, uint64_t seed, uint32_t instance, float *C, int64_t ldc, float *Cb,
                           void *ws);

// srht.cu
size_t rmc_srht_ws(int64_t m, int64_t n_total, int64_t s, int num_sms);
// dense.cu: least squares against a resident sketch (the request server keeps S^T A and its factor)
size_t rmc_lsr_factor_ws(int64_t s, int64_t n, int num_sms);
int rmc_launch_lsr_factor(rmc_ctx *ctx, const float *SA, int64_t s, int64_t n, int64_t ldsa, float *M, int *fail,
                          void *ws);
size_t rmc_lsr_refine_ws(int64_t s, int64_t n, int num_sms);
int rmc_launch_lsr_refine(rmc_ctx *ctx, const float *SAb, int64_t s, int64_t n, int64_t ldsab, const float *M,
                          const int *fail, double *x, void *ws);
// tc_gemm.cu: a dense (unswizzled) 2-D TMA map of a row-major FP32 matrix
int rmc_make_tmap_dense(CUtensorMap *map, const float *base, int64_t rows, int64_t cols, int64_t ld, int box_cols,
                        int box_rows);
int rmc_launch_srht(rmc_ctx *ctx, const float *A, int64_t m, int64_t n, int64_t lda, const float *b,
                    int64_t s, uint64_t seed, uint32_t instance, float *C, int64_t ldc, float *Cb, void *ws);

// gaussian.cu
size_t rmc_gauss_ws(int64_t m, int64_t n_total, int64_t s, int prec, int num_sms);
int rmc_launch_gauss_sketch(rmc_ctx *ctx, const float *A, int64_t m, int64_t n, int64_t lda, const float *b,
                            int64_t s, uint64_t seed, uint32_t instance, int prec, float *C, int64_t ldc,
                            float *Cb, void *ws);

// dense.cu
size_t rmc_matmul_ws(int64_t m, int64_t n, int64_t l, int which, int prec, int num_sms);
int rmc_launch_matmul_an(rmc_ctx *ctx, const float *A, int64_t m, int64_t n, int64_t lda, const float *X,
                         int64_t l, int64_t ldx, int prec, float *Y, int64_t ldy, void *ws);
int rmc_launch_matmul_at(rmc_ctx *ctx, const float *A, int64_t m, int64_t n, int64_t lda, const float *X,
                         int64_t l, int64_t ldx, int prec, float *W, int64_t ldw, void *ws);
size_t rmc_cholqr2_ws(int64_t m, int64_t l, int num_sms);
// passes = 2: CholeskyQR2; passes = 1: one CholeskyQR pass (a well-conditioned, not orthonormal, basis).
// fp64_gram: FP64 products in the last pass's Gram matrix (else, and in earlier passes, FP32 products with FP64
// sums across 32-row slices); RMC_OPT_SMALL_FP64 makes every pass FP64.
int rmc_launch_cholqr2(rmc_ctx *ctx, float *Y, int64_t m, int64_t l, int64_t ldy, double *R, void *ws,
                       int passes = 2, bool fp64_gram = false);
size_t rmc_svd_wide_ws(int64_t l, int64_t n, int num_sms);
int rmc_launch_svd_wide(rmc_ctx *ctx, const float *B, int64_t l, int64_t n, int64_t ldb, float *Ub,
                        float *sigma, float *Vb, int64_t ldv, void *ws);
size_t rmc_lsr_solve_ws(int64_t s, int64_t n, int num_sms);
int rmc_launch_lsr_solve(rmc_ctx *ctx, const float *SA, int64_t s, int64_t n, int64_t ldsa, const float *Sb,
                         double *x, void *ws);

// out[r, 0:lo] = in[r, 0:li] M (or -= with subtract), rows independent; in and out may alias.
int rmc_launch_rowblock(cudaStream_t st, const float *in, int64_t m, int li, int64_t ldi, const float *M, int lo,
                        int64_t ldm, float *out, int64_t ldo, bool subtract = false);
size_t rmc_jacobi_square_ws(int64_t l);
int rmc_launch_jacobi_square(rmc_ctx *ctx, const double *Wrm, int l, float *Ml, float *sigma, float *Vr, void *ws);
int rmc_launch_transpose(cudaStream_t st, const float *in, int64_t rows, int64_t cols, int64_t ldi, float *out,
                         int64_t ldo);
int rmc_launch_rsvd_finish(rmc_ctx *ctx, const float *Q, int64_t m, int64_t l, const float *Ub, const float *sg,
                           const float *Vb, int64_t n, int k, float *U, int64_t ldu, float *sigma, float *V,
                           int64_t ldv, void *ws);

// capi.cu: argument checks, workspace and launch of one sketch of A (and of b as one more column, into Cb)
extern "C" int rmc_check_sketch_args(const float *A, int64_t m, int64_t n, int64_t lda, int64_t s, int kind,
                                     int prec);
extern "C" size_t rmc_sketch_plan_bytes(rmc_ctx *ctx, int64_t m, int64_t ntot, int64_t s, int kind, int prec);
extern "C" int rmc_run_sketch(rmc_ctx *ctx, const float *A, int64_t m, int64_t n, int64_t lda, const float *b, int64_t s,
                              int kind, uint64_t seed, int prec, float *C, int64_t ldc, float *Cb, void *ws);

// capi.cu / batch.cu: device workspace of one call (what rmc_ws_reserve will be asked for)
extern "C" size_t rmc_lsr_plan_bytes(rmc_ctx *ctx, int64_t m, int64_t n, int64_t s, int kind, int prec);
extern "C" size_t rmc_rsvd_plan_bytes(rmc_ctx *ctx, int64_t m, int64_t n, int64_t l, int prec);
size_t rmc_batch_plan_bytes(const rmc_request *reqs, int nreq);
// batch.cu: the limits of one batched problem (false when the problem must go to the single-problem path)
bool rmc_batch_request_ok(const rmc_request &r);

// nystrom.cu
int rmc_launch_rbf(rmc_ctx *ctx, const float *X, int64_t n1, int64_t ldx, const float *Y, int64_t n2, int64_t ldy,
                   int64_t d, double sigma, float *C, int64_t ldc);

// tc_gemm.cu (tcgen05 tensor-core kernels)
int rmc_tc_available(void);
