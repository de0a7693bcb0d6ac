// k-SVD by the block Lanczos method (Algorithm 5.1 and the listing of Sec. 5.1):
//
//   C = A Omega (Omega n x s, iid N(0,1), the Philox stream of rmc_rsvd);
//   K = [C, (A A^T) C, ..., (A A^T)^(q-1) C];  Q = orth(K);  B = Q^T A;  B = U_B diag(sigma) V_B^T;
//   U = Q U_B[:, :k], sigma[:k], V = V_B[:, :k].
//
// The Krylov basis is built block by block as the listing does (the next block is A (A^T C) of the previous
// one, orthonormalised: the listing's "optional" qr), and each new block is also projected off the blocks
// before it, twice (classical Gram-Schmidt twice), before its CholeskyQR2.  Projection changes no span -- the
// part of A A^T C_i that lies in earlier blocks is removed, and A A^T maps the earlier blocks into the span of
// the blocks up to C_i -- so the columns of K stay an orthonormal basis of the same Krylov space, and the
// single QR of K that the listing takes at the end is already done.  Without the projection the blocks grow
// nearly dependent as they converge (the instability the footnote of Sec. 5.1 warns of) and a Cholesky-based
// QR of K would break down.  2q passes over A: one for C, two per further block, one for B.
#include "rmc_internal.cuh"

namespace {

struct LanczosBufs {
  float *Om, *K, *Z, *B, *P, *Ub, *sg, *Vb;
  void *scr;
};

LanczosBufs lanczos_carve(WsCarve &w, int64_t m, int64_t n, int64_t s, int64_t l, size_t scratch) {
  LanczosBufs b;
  b.Om = w.take<float>((size_t)n * s);
  b.K = w.take<float>((size_t)m * l);        // m x (s q), row stride l
  b.Z = w.take<float>((size_t)n * s);
  b.B = w.take<float>((size_t)l * n);
  b.P = w.take<float>((size_t)l * s);        // projection coefficients of a new block on the earlier ones
  b.Ub = w.take<float>((size_t)l * l);
  b.sg = w.take<float>((size_t)l);
  b.Vb = w.take<float>((size_t)n * l);
  b.scr = w.take<char>(scratch);
  return b;
}

size_t lanczos_scratch(rmc_ctx *ctx, int64_t m, int64_t n, int64_t s, int64_t l, int prec) {
  size_t t = rmc_cholqr2_ws(m, s, ctx->num_sms);
  const size_t c[] = {rmc_matmul_ws(m, n, s, 0, prec, ctx->num_sms), rmc_matmul_ws(m, n, s, 1, prec, ctx->num_sms),
                      rmc_matmul_ws(m, n, l, 1, prec, ctx->num_sms), rmc_matmul_ws(m, s, l, 1, RMC_FP32, ctx->num_sms),
                      rmc_svd_wide_ws(l, n, ctx->num_sms)};
  for (size_t v : c)
    if (v > t) t = v;
  return t;
}

}  // namespace

size_t rmc_lanczos_plan_bytes(rmc_ctx *ctx, int64_t m, int64_t n, int64_t s, int q, int prec) {
  WsCarve w;
  lanczos_carve(w, m, n, s, s * q, lanczos_scratch(ctx, m, n, s, s * q, prec));
  return w.off;
}

extern "C" int rmc_block_lanczos(rmc_ctx *ctx, const float *A, int64_t m, int64_t n, int64_t lda, int k, int s_,
                                 int q, uint64_t seed, int prec, float *U, int64_t ldu, float *sigma, float *V,
                                 int64_t ldv) {
  if (!ctx || !A || !U || !sigma || !V) return RMC_EINVAL;
  const int64_t s = s_, l = (int64_t)s_ * q;
  if (k < 1 || s < 1 || q < 1 || m < 1 || n < 1 || lda < n || ldu < k || ldv < k) return RMC_EINVAL;
  if (l > 256 || l > m || l > n || k > l) return RMC_EINVAL;
  if (!rmc_prec_ok(prec)) return RMC_EINVAL;
  const size_t scratch = lanczos_scratch(ctx, m, n, s, l, prec);
  WsCarve plan;
  lanczos_carve(plan, m, n, s, l, scratch);
  RMC_TRY(rmc_ws_reserve(ctx, plan.off));
  WsCarve w;
  w.base = static_cast<char *>(ctx->ws);
  const LanczosBufs b = lanczos_carve(w, m, n, s, l, scratch);
  cudaStream_t st = ctx->stream;

  RMC_TRY(rmc_launch_gaussian(st, seed, 0, n, s, b.Om, s, 1.0f));                        // Omega, n x s
  RMC_TRY(rmc_launch_matmul_an(ctx, A, m, n, lda, b.Om, s, s, prec, b.K, l, b.scr));     // K_0 = A Omega
  RMC_TRY(rmc_launch_cholqr2(ctx, b.K, m, s, l, nullptr, b.scr, 2));                     // orthonormal K_0
  for (int i = 1; i < q; ++i) {
    float *prev = b.K + (int64_t)(i - 1) * s, *cur = b.K + (int64_t)i * s;
    RMC_TRY(rmc_launch_matmul_at(ctx, A, m, n, lda, prev, s, l, prec, b.B, n, b.scr));   // A^T K_{i-1} (s x n)
    RMC_TRY(rmc_launch_transpose(st, b.B, s, n, n, b.Z, s));                              // Z = (A^T K_{i-1}), n x s
    RMC_TRY(rmc_launch_matmul_an(ctx, A, m, n, lda, b.Z, s, s, prec, cur, l, b.scr));    // K_i = A A^T K_{i-1}
    const int64_t done = (int64_t)i * s;                                                  // columns of K so far
    for (int rep = 0; rep < 2; ++rep) {
      // P = K_{<i}^T K_i (done x s), K_i -= K_{<i} P
      RMC_TRY(rmc_launch_matmul_at(ctx, cur, m, s, l, b.K, done, l, RMC_FP32, b.P, s, b.scr));
      RMC_TRY(rmc_launch_rowblock(st, b.K, m, (int)done, l, b.P, (int)s, s, cur, l, true));
    }
    RMC_TRY(rmc_launch_cholqr2(ctx, cur, m, s, l, nullptr, b.scr, 2));                   // orthonormal K_i
  }
  RMC_TRY(rmc_launch_matmul_at(ctx, A, m, n, lda, b.K, l, l, prec, b.B, n, b.scr));      // B = Q^T A (l x n)
  RMC_TRY(rmc_launch_svd_wide(ctx, b.B, l, n, n, b.Ub, b.sg, b.Vb, l, b.scr));           // B = Ub S Vb^T
  return rmc_launch_rsvd_finish(ctx, b.K, m, l, b.Ub, b.sg, b.Vb, n, k, U, ldu, sigma, V, ldv, b.scr);
}
