// Faster randomized k-SVD (Algorithm 5.3 and the listing of Sec. 5.3), built on the GaussianProjection +
// CountSketch composite of Sec. 3.2.4:
//
//   C = A S           S an n x s count sketch over the COLUMNS of A (Philox instance 1)      m x s
//   [L, D] = P^T [A, C] with P = P_cs P_gp: a count sketch of the rows to p_cs (instance 2) followed by a
//                     Gaussian projection to p rows (instance 3)                           p x n, p x s
//   D = Q_D R_D (CholeskyQR2, FP64 R);   Q_D^T L = U_bar diag(sigma_bar) V_bar^T (top k of an SVD);
//   C R_D^-1 U_bar diag(sigma_bar) = U_t diag(sigma_t) V_hat^T;   V_t = V_bar V_hat.
//
// Two passes over A (one for C, one for P_cs^T A), as the remarks after the listing count them; everything
// after the second pass works on sketches whose size does not depend on m or n beyond p x n and m x k.
//
// The column count sketch is a gather, not a scatter: the columns of each 1024-column chunk are sorted by
// bucket once (a stable counting sort, so each bucket keeps column order), then a CTA stages a 16-row x
// 1024-column tile of A in shared memory and thread b sums bucket b's columns of the chunk for its 16 rows.
// No atomics, and every C[i, b] is summed in column order (the order of Algorithm 3.1 over the columns).
#include "rmc_internal.cuh"
#include "philox.cuh"

using namespace rmc;

namespace {

constexpr int kColChunk = 1024;     // columns per chunk
constexpr int kRows = 16;           // rows of A per CTA
constexpr int kMaxBuckets = 256;    // s <= 256: one thread per bucket
constexpr int kInstS = 1, kInstPcs = 2, kInstPgp = 3;

// Per chunk: the chunk's columns sorted stably by bucket (perm: global column index, psign: the column's sign)
// and the bucket offsets off[chunk][0..s].
__global__ void __launch_bounds__(kMaxBuckets) cs_col_prep_kernel(uint64_t seed, uint32_t instance, int64_t n,
                                                                  int s, int *perm, float *psign, int *off) {
  __shared__ int bk[kColChunk];
  __shared__ float sg[kColChunk];
  __shared__ int cnt[kMaxBuckets + 1];
  const int64_t c0 = (int64_t)blockIdx.x * kColChunk;
  const int cols = (int)min((int64_t)kColChunk, n - c0);
  for (int t = threadIdx.x; t < cols; t += blockDim.x) {
    uint32_t b;
    float g;
    cs_hash(seed, instance, (uint64_t)(c0 + t), (uint32_t)s, &b, &g);
    bk[t] = (int)b;
    sg[t] = g;
  }
  __syncthreads();
  const int b = threadIdx.x;
  int mine = 0;
  if (b < s)
    for (int t = 0; t < cols; ++t) mine += (bk[t] == b);
  if (b < s) cnt[b] = mine;
  __syncthreads();
  if (threadIdx.x == 0) {
    int acc = 0;
    for (int q = 0; q < s; ++q) {
      const int c = cnt[q];
      cnt[q] = acc;
      acc += c;
    }
    cnt[s] = acc;
  }
  __syncthreads();
  int *o = off + (int64_t)blockIdx.x * (s + 1);
  for (int q = threadIdx.x; q <= s; q += blockDim.x) o[q] = cnt[q];
  if (b < s) {
    int pos = cnt[b];
    for (int t = 0; t < cols; ++t)
      if (bk[t] == b) {
        perm[c0 + pos] = (int)(c0 + t);
        psign[c0 + pos] = sg[t];
        ++pos;
      }
  }
}

// C[r, b] = sum over the columns j with h(j) = b, in column order, of g(j) A[r, j].
struct ColArgs {
  const float *A;
  int64_t m, n, lda;
  int s;
  const int *perm;
  const float *psign;
  const int *off;
  float *C;
  int64_t ldc;
};

template <bool VEC>
__global__ void __launch_bounds__(kMaxBuckets) cs_cols_kernel(ColArgs a) {
  extern __shared__ __align__(16) float smem[];
  float *tile = smem;                                            // kRows x kColChunk
  int *p = reinterpret_cast<int *>(tile + kRows * kColChunk);    // kColChunk
  float *g = reinterpret_cast<float *>(p + kColChunk);           // kColChunk
  int *o = reinterpret_cast<int *>(g + kColChunk);               // s + 1
  const int64_t r0 = (int64_t)blockIdx.x * kRows;
  const int rows = (int)min((int64_t)kRows, a.m - r0);
  const int b = threadIdx.x;
  float acc[kRows];
#pragma unroll
  for (int r = 0; r < kRows; ++r) acc[r] = 0.f;
  const int64_t nchunks = (a.n + kColChunk - 1) / kColChunk;
  for (int64_t ch = 0; ch < nchunks; ++ch) {
    const int64_t c0 = ch * kColChunk;
    const int cols = (int)min((int64_t)kColChunk, a.n - c0);
    if (VEC) {
      // cols % 4 == 0 on this path (n % 4 == 0, lda % 4 == 0, 16-byte aligned A)
      const int q4 = cols / 4;
      for (int e = threadIdx.x; e < kRows * q4; e += blockDim.x) {
        const int r = e / q4, c = 4 * (e % q4);
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (r < rows) v = __ldcs(reinterpret_cast<const float4 *>(a.A + (r0 + r) * a.lda + c0 + c));
        *reinterpret_cast<float4 *>(tile + r * kColChunk + c) = v;
      }
    } else {
      for (int e = threadIdx.x; e < kRows * cols; e += blockDim.x) {
        const int r = e / cols, c = e % cols;
        tile[r * kColChunk + c] = (r < rows) ? __ldcs(a.A + (r0 + r) * a.lda + c0 + c) : 0.f;
      }
    }
    for (int t = threadIdx.x; t < cols; t += blockDim.x) {
      p[t] = a.perm[c0 + t] - (int)c0;
      g[t] = a.psign[c0 + t];
    }
    for (int q = threadIdx.x; q <= a.s; q += blockDim.x) o[q] = a.off[ch * (a.s + 1) + q];
    __syncthreads();
    if (b < a.s) {
      const int t1 = o[b + 1];
      for (int t = o[b]; t < t1; ++t) {
        const int j = p[t];
        const float sgn = g[t];
#pragma unroll
        for (int r = 0; r < kRows; ++r) acc[r] = fmaf(sgn, tile[r * kColChunk + j], acc[r]);
      }
    }
    __syncthreads();
  }
  if (b < a.s)
#pragma unroll
    for (int r = 0; r < kRows; ++r)
      if (r < rows) a.C[(r0 + r) * a.ldc + b] = acc[r];
}

size_t cols_smem(int s) { return sizeof(float) * kRows * kColChunk + 8 * kColChunk + 4 * (size_t)(s + 1); }

// Z (s x k) = R^-1 Ubar diag(sbar) with R (s x s, FP64, upper) by back substitution per column (one warp per
// column of Z), in FP64; Ubar = Ub[:, :k] of the s x s left singular vectors (row-major, row stride s).
__global__ void fast_rinv_apply_kernel(const double *R, int s, const float *Ub, const float *sb, int k, float *Z,
                                       int *status) {
  const int j = blockIdx.x, lane = threadIdx.x;
  extern __shared__ double z[];
  for (int i = lane; i < s; i += 32) z[i] = 0.0;
  __syncwarp();
  const double sj = (double)sb[j];
  for (int i = s - 1; i >= 0; --i) {
    double acc = 0.0;
    for (int t = i + 1 + lane; t < s; t += 32) acc += R[(int64_t)i * s + t] * z[t];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) {
      const double d = R[(int64_t)i * s + i];
      if (!(d > 0.0)) rmc_report(status, RMC_ENUMERIC);
      z[i] = ((double)Ub[(int64_t)i * s + j] * sj - acc) / d;
    }
    __syncwarp();
  }
  for (int i = lane; i < s; i += 32) Z[(int64_t)i * k + j] = (float)z[i];
}

__global__ void f64_to_f32_kernel(const double *in, int64_t count, float *out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x)
    out[e] = (float)in[e];
}

struct FastBufs {
  int *perm, *off;
  float *psign, *C, *PA, *PC, *L, *D, *Mt, *Ub, *sb, *Vb, *Z, *N, *Ur, *sr, *Vr, *Vt;
  double *RD, *RN;
  void *scr;
};

FastBufs fast_carve(WsCarve &w, int64_t m, int64_t n, int s, int p_cs, int p, int k, size_t scratch) {
  FastBufs f;
  const int64_t nch = (n + kColChunk - 1) / kColChunk;
  f.perm = w.take<int>(n);
  f.psign = w.take<float>(n);
  f.off = w.take<int>((size_t)nch * (s + 1));
  f.C = w.take<float>((size_t)m * s);
  f.PA = w.take<float>((size_t)p_cs * n);
  f.PC = w.take<float>((size_t)p_cs * s);
  f.L = w.take<float>((size_t)p * n);
  f.D = w.take<float>((size_t)p * s);
  f.RD = w.take<double>((size_t)s * s);
  f.Mt = w.take<float>((size_t)s * n);
  f.Ub = w.take<float>((size_t)s * s);
  f.sb = w.take<float>(s);
  f.Vb = w.take<float>((size_t)n * s);
  f.Z = w.take<float>((size_t)s * k);
  f.N = w.take<float>((size_t)m * k);
  f.RN = w.take<double>((size_t)k * k);
  f.Ur = w.take<float>((size_t)k * k);
  f.sr = w.take<float>(k);
  f.Vr = w.take<float>((size_t)k * k);
  f.Vt = w.take<float>((size_t)n * k);
  f.scr = w.take<char>(scratch);
  return f;
}

size_t fast_scratch(rmc_ctx *ctx, int64_t m, int64_t n, int s, int p_cs, int p, int k, int prec) {
  if (prec == RMC_TF32X3) prec = RMC_FP32;
  const size_t c[] = {rmc_countsketch_ws(m, p_cs), rmc_gauss_ws(p_cs, n, p, prec, ctx->num_sms),
                      rmc_gauss_ws(p_cs, s, p, prec, ctx->num_sms), rmc_cholqr2_ws(p, s, ctx->num_sms),
                      rmc_matmul_ws(p, n, s, 1, RMC_FP32, ctx->num_sms), rmc_svd_wide_ws(s, n, ctx->num_sms),
                      rmc_cholqr2_ws(m, k, ctx->num_sms), rmc_svd_wide_ws(k, k, ctx->num_sms)};
  size_t t = 0;
  for (size_t v : c)
    if (v > t) t = v;
  return t;
}

}  // namespace

// The column count sketch C = A S (S n x s, Algorithm 3.1 over the columns) into C (m x s, ldc); workspace:
// perm, psign, off at the start of ws.
static int launch_cols(rmc_ctx *ctx, const float *A, int64_t m, int64_t n, int64_t lda, int s, uint64_t seed,
                       uint32_t instance, float *C, int64_t ldc, int *perm, float *psign, int *off) {
  cudaStream_t st = ctx->stream;
  const int64_t nch = (n + kColChunk - 1) / kColChunk;
  cs_col_prep_kernel<<<(unsigned)nch, kMaxBuckets, 0, st>>>(seed, instance, n, s, perm, psign, off);
  ColArgs a;
  a.A = A;
  a.m = m;
  a.n = n;
  a.lda = lda;
  a.s = s;
  a.perm = perm;
  a.psign = psign;
  a.off = off;
  a.C = C;
  a.ldc = ldc;
  const size_t smem = cols_smem(s);
  const bool vec = (n % 4 == 0) && (lda % 4 == 0) && (reinterpret_cast<uintptr_t>(A) % 16 == 0);
  const unsigned grid = (unsigned)((m + kRows - 1) / kRows);
  {
    RmcProf prof(ctx, RMC_K_COUNTSKETCH);
    if (vec) {
      RMC_TRY_CUDA(rmc_allow_smem(cs_cols_kernel<true>, smem));
      cs_cols_kernel<true><<<grid, kMaxBuckets, smem, st>>>(a);
    } else {
      RMC_TRY_CUDA(rmc_allow_smem(cs_cols_kernel<false>, smem));
      cs_cols_kernel<false><<<grid, kMaxBuckets, smem, st>>>(a);
    }
  }
  rmc_note_launch(2);
  RMC_LAUNCH_CHECK();
  return RMC_OK;
}

extern "C" int rmc_countsketch_columns(rmc_ctx *ctx, const float *A, int64_t m, int64_t n, int64_t lda, int64_t s,
                                       uint64_t seed, uint32_t instance, float *C, int64_t ldc) {
  if (!ctx || !A || !C || m < 1 || n < 1 || lda < n || s < 1 || s > kMaxBuckets || ldc < s) return RMC_EINVAL;
  if (n > (int64_t(1) << 31)) return RMC_EINVAL;
  const int64_t nch = (n + kColChunk - 1) / kColChunk;
  WsCarve plan;
  plan.take<int>(n);
  plan.take<float>(n);
  plan.take<int>((size_t)nch * (s + 1));
  RMC_TRY(rmc_ws_reserve(ctx, plan.off));
  WsCarve w;
  w.base = static_cast<char *>(ctx->ws);
  int *perm = w.take<int>(n);
  float *psign = w.take<float>(n);
  int *off = w.take<int>((size_t)nch * (s + 1));
  return launch_cols(ctx, A, m, n, lda, (int)s, seed, instance, C, ldc, perm, psign, off);
}

extern "C" int rmc_rsvd_fast(rmc_ctx *ctx, const float *A, int64_t m, int64_t n, int64_t lda, int k, int s, int p_cs,
                             int p, uint64_t seed, int prec, float *U, int64_t ldu, float *sigma, float *V,
                             int64_t ldv) {
  if (!ctx || !A || !U || !sigma || !V) return RMC_EINVAL;
  if (k < 1 || s < k || s > kMaxBuckets || p < s || p_cs < p || m < 1 || n < s || lda < n || ldu < k || ldv < k)
    return RMC_EINVAL;
  if (m < k || m > (int64_t(1) << 31) || n > (int64_t(1) << 31) || !rmc_prec_ok(prec)) return RMC_EINVAL;
  const size_t scratch = fast_scratch(ctx, m, n, s, p_cs, p, k, prec);
  WsCarve plan;
  fast_carve(plan, m, n, s, p_cs, p, k, scratch);
  RMC_TRY(rmc_ws_reserve(ctx, plan.off));
  WsCarve w;
  w.base = static_cast<char *>(ctx->ws);
  const FastBufs f = fast_carve(w, m, n, s, p_cs, p, k, scratch);
  cudaStream_t st = ctx->stream;

  // pass 1: C = A S (column count sketch)
  RMC_TRY(launch_cols(ctx, A, m, n, lda, s, seed, kInstS, f.C, s, f.perm, f.psign, f.off));
  // pass 2: P_cs^T A and P_cs^T C (one row hash for both), then the Gaussian projection of each to p rows
  RMC_TRY(rmc_launch_countsketch(ctx, A, m, n, lda, nullptr, p_cs, seed, kInstPcs, f.PA, n, nullptr, f.scr));
  RMC_TRY(rmc_launch_countsketch(ctx, f.C, m, s, s, nullptr, p_cs, seed, kInstPcs, f.PC, s, nullptr, f.scr));
  const int gp = prec == RMC_TF32X3 ? RMC_FP32 : prec;     // the drawn sketch has no split form
  RMC_TRY(rmc_launch_gauss_sketch(ctx, f.PA, p_cs, n, n, nullptr, p, seed, kInstPgp, gp, f.L, n, nullptr, f.scr));
  RMC_TRY(rmc_launch_gauss_sketch(ctx, f.PC, p_cs, s, s, nullptr, p, seed, kInstPgp, gp, f.D, s, nullptr, f.scr));
  // D = Q_D R_D;  Q_D^T L = Ub diag(sb) Vb^T
  RMC_TRY(rmc_launch_cholqr2(ctx, f.D, p, s, s, f.RD, f.scr, 2, true));
  RMC_TRY(rmc_launch_matmul_at(ctx, f.L, p, n, n, f.D, s, s, RMC_FP32, f.Mt, n, f.scr));
  RMC_TRY(rmc_launch_svd_wide(ctx, f.Mt, s, n, n, f.Ub, f.sb, f.Vb, s, f.scr));
  // Z = R_D^-1 Ubar diag(sbar) (s x k);  N = C Z (m x k)
  fast_rinv_apply_kernel<<<k, 32, sizeof(double) * s, st>>>(f.RD, s, f.Ub, f.sb, k, f.Z, ctx->d_status);
  rmc_note_launch();
  RMC_LAUNCH_CHECK();
  RMC_TRY(rmc_launch_rowblock(st, f.C, m, s, s, f.Z, k, k, f.N, k));
  // N = U_t diag(sigma_t) V_hat^T through N = Q_N R_N and the SVD of R_N;  V_t = V_bar V_hat
  RMC_TRY(rmc_launch_cholqr2(ctx, f.N, m, k, k, f.RN, f.scr, 2, true));
  {
    // R_N (FP64, k x k) -> FP32 for the small SVD
    float *Rn32 = f.Vt;   // borrowed: V_t is written only after the SVD below reads R_N
    f64_to_f32_kernel<<<rmc_blocks((int64_t)k * k, 256, 1024), 256, 0, st>>>(f.RN, (int64_t)k * k, Rn32);
    rmc_note_launch();
    RMC_LAUNCH_CHECK();
    RMC_TRY(rmc_launch_svd_wide(ctx, Rn32, k, k, k, f.Ur, f.sr, f.Vr, k, f.scr));
  }
  RMC_TRY(rmc_launch_rowblock(st, f.Vb, n, k, s, f.Vr, k, k, f.Vt, k));        // V_t = Vb[:, :k] V_hat
  return rmc_launch_rsvd_finish(ctx, f.N, m, k, f.Ur, f.sr, f.Vt, n, k, U, ldu, sigma, V, ldv, f.scr);
}
