/*
 * rmc.h -- randomized matrix computations on one NVIDIA GB300 (sm_103a): sketching, randomized SVD and
 * sketch-and-solve least squares, after S. Wang, "A Practical Guide to Randomized Matrix Computations with
 * MATLAB Implementations" (arXiv:1505.07570).
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Matrices are FP32, row-major, with a leading dimension (elements between the starts of consecutive
 *    rows) >= the number of columns.  A is m x n.
 *  - Matrix and vector pointers are DEVICE pointers owned by the caller; the library never frees them and
 *    never keeps them after the call returns.  Outputs must not alias inputs.
 *  - Every call is asynchronous on the context's CUDA stream: it returns once the work is enqueued.
 *    Outputs are valid after rmc_sync(ctx) (or after the stream completes).
 *  - Argument errors are returned synchronously and nothing is enqueued.  Errors found on the device
 *    (a non-positive pivot, an iteration cap, a bounded wait that expired) are written to the context's
 *    device status word and returned by the next rmc_sync.  No kernel traps.
 *  - Workspace is owned by the context (stream-ordered device allocations, capped by the HBM budget given
 *    to rmc_create); a call whose workspace would exceed the budget returns RMC_ENOMEM.
 *  - The sketch acts on the ROW dimension: C = S^T A is s x n, the orientation of the sketched least
 *    squares problem of Sec. 4.2.  The column sketch C = A S of Ch. 3 is rmc_sketch applied to A^T.
 *
 * Randomness (one definition, shared with the oracle through this header and nothing else)
 * ------------------------------------------------------------------------------------------
 *  Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).  key = (seed mod 2^32, seed div 2^32);
 *  counter = (index mod 2^32, index div 2^32, stream, instance).  u(w) = ((w >> 9) + 1/2) * 2^-23.
 *   stream 0  Gaussian entries of the range finder's test matrices (rmc_rsvd, rmc_block_lanczos,
 *             rmc_gaussian_matrix).  Entry (i, j) of a rows x cols matrix uses block index
 *             i * ceil(cols/4) + j/4; words (0,1) -> columns 4t, 4t+1 and words (2,3) -> 4t+2, 4t+3 by
 *             Box-Muller: r = sqrt(-2 ln u(w_a)), (r cos 2 pi u(w_b), r sin 2 pi u(w_b)).
 *   stream 1  SRHT row sign of row i: -1 if bit 31 of word 0 of block i is set, else +1.
 *   stream 2  count-sketch row i: bucket h(i) = (word0 * s) >> 32, sign g(i) = -1 if bit 31 of word 1.
 *   stream 3  SRHT sample key of index j: (word0 << 32) | word1 of block j; the sample is the s indices
 *             with the smallest keys (ties to the smaller index), in ascending order.
 *   stream 4  Gaussian SKETCHING matrix G (m x s) of RMC_GAUSSIAN.  Entry (i, j) uses block index
 *             i * ceil(s/8) + j/8; the 16-bit halves of word w (low, high) are the pair of columns 8b + 2w,
 *             8b + 2w + 1: with u16(h) = (h + 1/2) * 2^-16, r = sqrt(-2 ln u16(low)),
 *             (r cos 2 pi u16(high), r sin 2 pi u16(high)).  Eight normals per block: half the Philox work of
 *             stream 0 per entry; the uniforms' 2^-16 steps are finer than TF32 operand rounding (2^-11).
 *  Hashes, signs and sample indices are bit-identical to the oracle's; Gaussian entries agree to FP32
 *  rounding of log/sqrt/sin/cos.
 */
#ifndef RMC_H
#define RMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------------------------------ status */
#define RMC_OK        0
#define RMC_EINVAL    1   /* bad argument: null pointer, ld < cols, s < 1, s > N (SRHT), k < 1, ...     */
#define RMC_EALIGN    2   /* a pointer or leading dimension breaks the 16-byte rule of a TMA-fed path    */
#define RMC_ENOMEM    3   /* workspace would exceed the context's HBM budget, or allocation failed       */
#define RMC_ENUMERIC  4   /* non-positive Cholesky pivot, or Jacobi SVD hit its sweep cap                */
#define RMC_ETIMEOUT  5   /* a bounded device-side wait expired                                          */
#define RMC_ECUDA     6   /* a CUDA runtime call or kernel launch failed                                 */
#define RMC_PENDING   7   /* request not finished yet                                                    */
#define RMC_ESCRATCH  8   /* the call needs more than the fixed scratch of rmc_countsketch_noalloc       */

/* ----------------------------------------------------------------------------------- sketch kinds */
#define RMC_GAUSSIAN     0   /* S = G / sqrt(s), G iid N(0,1)                                Sec. 3.2.1 */
#define RMC_SRHT         1   /* S^T = (1/sqrt(s)) P^T H_N D, rows zero-padded to N = 2^ceil(log2 m)
                                                                                             Sec. 3.2.2 */
#define RMC_COUNTSKETCH  2   /* one +-1 per row of S, in a uniformly hashed column   Sec. 3.2.3, Alg. 3.1 */

/* ------------------------------------------------------------- GEMM operand precision (accumulate FP32) */
#define RMC_FP32  0   /* FP32 operands on the CUDA cores (the plain form)                                 */
#define RMC_TF32  1   /* TF32 operands on the tensor cores (tcgen05.mma kind::tf32), FP32 accumulation    */
#define RMC_BF16  2   /* BF16 operands on the tensor cores (tcgen05.mma kind::f16), FP32 accumulation: A is read
                         in FP32 and rounded on chip, the other operand (Omega drawn, or X) rounded to BF16; about
                         2^-9 relative error per product (the Gaussian sketch: ~2e-3 relative Frobenius) */
#define RMC_TF32X3 3  /* 3xTF32 on the tensor cores: each FP32 operand split into a TF32 head and remainder,
                         three kind::tf32 MMAs per step (head*head + head*rest + rest*head), FP32 accumulation:
                         about 2^-21 relative error per product (FP32-level), for the products with A of
                         rmc_rsvd, rmc_block_lanczos, rmc_matmul_an/at (not the Gaussian sketch: RMC_EINVAL) */

typedef struct rmc_ctx rmc_ctx;

/* ------------------------------------------------------------------------------------------ context */

/* Create a context bound to the current CUDA device and to `cuda_stream` (a cudaStream_t; NULL = the legacy
 * default stream).  hbm_budget_bytes caps the context's workspace (0 = 64 GiB).  On success *ctx owns the
 * workspace and a device status word; release with rmc_destroy.  Errors: RMC_EINVAL (ctx NULL),
 * RMC_ECUDA. */
int rmc_create(rmc_ctx **ctx, void *cuda_stream, size_t hbm_budget_bytes);

/* Wait for the context's stream, free its workspace and the context.  NULL is accepted. */
int rmc_destroy(rmc_ctx *ctx);

/* Rebind the context to another stream (later calls are enqueued there). */
int rmc_set_stream(rmc_ctx *ctx, void *cuda_stream);

/* Wait for the context's stream, then return and clear the device status word: RMC_OK, or the first
 * device-detected error since the last rmc_sync (RMC_ENUMERIC, RMC_ETIMEOUT), or RMC_ECUDA. */
int rmc_sync(rmc_ctx *ctx);

/* A static description of a status code. */
const char *rmc_status_string(int status);

/* Context options (rmc_set_option / rmc_get_option):
 *   RMC_OPT_SMALL_FP64  0 (default): the small l x l factorizations run in FP32 where that meets the stated
 *                       tolerances -- CholeskyQR2's Cholesky in FP32 with an FP64 fallback on a non-positive
 *                       pivot, its Gram matrices with FP32 products summed in FP64, the one-sided Jacobi SVD in
 *                       FP32 above l = 32.  1: all of them in FP64 (Gram products, Cholesky, Jacobi rotations);
 *                       slower on this GPU, whose FP64 rate is a small fraction of its FP32 rate.
 * Errors: RMC_EINVAL for an unknown option or value. */
#define RMC_OPT_SMALL_FP64 1
int rmc_set_option(rmc_ctx *ctx, int option, int value);
int rmc_get_option(const rmc_ctx *ctx, int option, int *value);

/* Bytes of device workspace the context currently holds. */
int rmc_workspace_bytes(const rmc_ctx *ctx, size_t *bytes);

/* ---------------------------------------------------------------------------------- the three calls */

/* Sketch: C = S^T A, C is s x n with leading dimension ldc (Sec. 3.2; sketch C = A S, Ch. 3 opening, in the
 * row orientation of Sec. 4.2).
 *   kind  RMC_GAUSSIAN: S = G / sqrt(s), m x s (Sec. 3.2.1); any s >= 1.
 *         RMC_SRHT: rows sign-flipped (D), zero-padded to N = next power of two >= m, transformed by the
 *                   unnormalised Hadamard matrix H_N (Sylvester order), s sampled rows without replacement
 *                   kept in ascending index order, scaled by 1/sqrt(s) (Sec. 3.2.2); 1 <= s <= N.
 *         RMC_COUNTSKETCH: C[h(i), :] += g(i) A[i, :] for every row i (Algorithm 3.1); any s >= 1.
 *   prec  GEMM operand precision of the Gaussian kind (RMC_FP32, RMC_TF32 or RMC_BF16); ignored otherwise, but
 *         always checked (any other value is RMC_EINVAL).
 *         The tensor-core forms stream A with TMA and need 16-byte aligned rows (A and lda * 4 multiples of
 *         16 bytes); other layouts run the FP32 CUDA-core kernel.
 *   seed  64-bit Philox key; the same (seed, m, s, kind) always gives the same S.
 * Errors: RMC_EINVAL, RMC_ENOMEM, RMC_ECUDA. */
int rmc_sketch(rmc_ctx *ctx, const float *A, int64_t m, int64_t n, int64_t lda,
               int64_t s, int kind, uint64_t seed, int prec, float *C, int64_t ldc);

/* Sketch-and-solve least squares (Sec. 4.2): sketch the augmented matrix [A, b] with ONE operator S (as the
 * listing of Sec. 4.2 does), then x = argmin_x || (S^T A) x - S^T b ||_2 solved in FP64 by CholeskyQR2 of the
 * augmented s x (n+1) sketch (x = R11^-1 r12 from its R factor).  b has m entries; x (device, FP64) n.
 * Requires s >= n.  Errors: RMC_EINVAL, RMC_ENOMEM, RMC_ECUDA at the call; RMC_ENUMERIC at rmc_sync when the
 * sketch is numerically rank deficient (non-positive pivot). */
int rmc_lsr_sketch(rmc_ctx *ctx, const float *A, int64_t m, int64_t n, int64_t lda, const float *b,
                   int64_t s, int kind, uint64_t seed, int prec, double *x);

/* Randomized k-SVD with q power iterations (Algorithm 5.2 with the power step of the Sec. 5.1 listing),
 * l = k + p:
 *   Y = A Omega (Omega n x l iid N(0,1), stream 0), Q = orth(Y);
 *   q times: Z = orth(A^T Q), Q = orth(A Z)              (orth = CholeskyQR2, FP64 Gram and Cholesky);
 *   B = Q^T A (l x n); B = U_B diag(sigma) V_B^T (FP64 one-sided Jacobi on the R factor of B^T);
 *   U = Q U_B[:, :k] (m x k, ldu), sigma[k] descending, V = V_B[:, :k] (n x k, ldv).
 * Each column pair (u_i, v_i) is signed so the largest-magnitude entry of v_i is positive.
 * prec selects the operand precision of the products with A (RMC_FP32, RMC_TF32, RMC_TF32X3 or RMC_BF16).
 * Requires 1 <= k, l <= min(m, n), l <= 256,
 * q >= 0.  Errors: RMC_EINVAL, RMC_ENOMEM, RMC_ECUDA; RMC_ENUMERIC at rmc_sync (breakdown of CholeskyQR2
 * or no Jacobi convergence). */
int rmc_rsvd(rmc_ctx *ctx, const float *A, int64_t m, int64_t n, int64_t lda, int k, int p, int q,
             uint64_t seed, int prec, float *U, int64_t ldu, float *sigma, float *V, int64_t ldv);

/* ------------------------------------------------------------------------------- beyond the three calls */

/* Machine-precision least squares by sketch preconditioning (Algorithm 4.1, Sec. 4.3):
 *   Y = S^T A and S^T b from one sketch of [A, b] (kind, seed, prec as for rmc_lsr_sketch);
 *   Y = Q_Y R_Y (CholeskyQR2, FP64 Gram);  T = R_Y^-1 (FP64);  z = Q_Y^T S^T b;
 *   up to max_iters times:  r = b - A (T z);  z += theta T^T (A^T r);   x = T z (FP64, n entries).
 * A T is never formed: each step is ONE pass over A that forms r row by row with a compensated (Dot2) dot
 * product and accumulates A^T r from the same rows.  theta <= 0 selects 2 / ((1 - e)^-2 + (1 + e)^-2) with
 * e = min(0.9, sqrt(n / s)), the best fixed step for the singular values of A T that a Gaussian sketch of size s
 * gives.  The iteration stops early once a step changes z by at most tol * max|z| (max norms); *iters (device
 * int, optional: NULL) receives the number of steps taken.  Requires n <= s, n <= 256, n <= m.
 * Errors: RMC_EINVAL, RMC_ENOMEM, RMC_ECUDA; RMC_ENUMERIC at rmc_sync when S^T A is rank deficient. */
int rmc_lsr_precise(rmc_ctx *ctx, const float *A, int64_t m, int64_t n, int64_t lda, const float *b, int64_t s,
                    int kind, uint64_t seed, int prec, double theta, int max_iters, double tol, double *x,
                    int *iters);

/* k-SVD by block Lanczos (Algorithm 5.1 and the listing of Sec. 5.1): C = A Omega (Omega n x s, the Gaussian
 * stream of rmc_rsvd), K = [C, (A A^T) C, ..., (A A^T)^(q-1) C] (m x s q), Q = orth(K), B = Q^T A,
 * B = U_B diag(sigma) V_B^T; U = Q U_B[:, :k] (m x k, ldu), sigma[k] descending, V = V_B[:, :k] (n x k, ldv),
 * signed as rmc_rsvd signs them.  Each Krylov block is orthonormalised and projected off the earlier blocks
 * as it is formed (same span, stable basis).  2q passes over A.  prec: the operand precision of the products
 * with A, as for rmc_rsvd.  Requires 1 <= k <= s q, s q <= min(m, n), s q <= 256, q >= 1.  With q = 1 the result is rmc_rsvd's
 * with p = s - k and no power iteration.  Errors as rmc_rsvd. */
int rmc_block_lanczos(rmc_ctx *ctx, const float *A, int64_t m, int64_t n, int64_t lda, int k, int s, int q,
                      uint64_t seed, int prec, float *U, int64_t ldu, float *sigma, float *V, int64_t ldv);

/* Faster randomized k-SVD (Algorithm 5.3 and the listing of Sec. 5.3) on the GaussianProjection + CountSketch
 * composite of Sec. 3.2.4, two passes over A:
 *   C = A S (S an n x s count sketch over the columns, Philox instance 1);
 *   L = P^T A, D = P^T C with P = P_cs P_gp (a count sketch of the rows to p_cs, instance 2, then a Gaussian
 *   projection to p rows, instance 3; prec RMC_TF32 or RMC_BF16 runs it on the tensor cores, RMC_FP32 and
 *   RMC_TF32X3 in FP32);
 *   D = Q_D R_D;  Q_D^T L = U_bar diag(sigma_bar) V_bar^T (top k);  C R_D^-1 U_bar diag(sigma_bar) =
 *   U diag(sigma) V_hat^T;  V = V_bar V_hat.
 * Outputs as rmc_rsvd (U m x k, sigma[k] descending, V n x k, the same sign rule).  Requires
 * 1 <= k <= s <= 256, s <= p <= p_cs, s <= n, k <= m.  R_D is inverted (the listing's pinv(R_D) for a D of full
 * column rank, which needs rank(A) >= s); errors as rmc_rsvd, with RMC_ENUMERIC at rmc_sync when D is rank
 * deficient. */
int rmc_rsvd_fast(rmc_ctx *ctx, const float *A, int64_t m, int64_t n, int64_t lda, int k, int s, int p_cs, int p,
                  uint64_t seed, int prec, float *U, int64_t ldu, float *sigma, float *V, int64_t ldv);

/* The Nystrom method on the Gaussian RBF kernel (Sec. 6.4 and its listing; kernel of Sec. 6.1):
 *   S = the s landmarks, uniform without replacement in ascending order (the SRHT sample rule of stream 3,
 *       drawn over [0, n) with instance 0);
 *   C = K(:, S), K_ij = exp(-||x_i - x_j||^2 / (2 sigma^2)) (n x s; the n x n kernel matrix is never formed);
 *   W = C(S, :) = U_W diag(lam) U_W^T (one-sided Jacobi directly on W);
 *   L = C U_W[:, :k] diag(lam[:k])^-1/2 (n x k, ldl), so that K ~ L L^T.
 * X: n points of dimension d (row-major FP32, ldx).  k = 0 selects ceil(0.8 s), the listing's choice.  Each
 * column of U_W is signed so its largest-magnitude entry is positive.  lam (device, k floats) and landmarks
 * (device, s int64) are optional outputs (NULL to skip).  Requires 1 <= s <= min(n, 256), 1 <= k <= s.
 * RMC_ENUMERIC at rmc_sync when one of the k kept eigenvalues is not positive. */
int rmc_nystrom(rmc_ctx *ctx, const float *X, int64_t n, int64_t d, int64_t ldx, double sigma, int64_t s, int k,
                uint64_t seed, float *L, int64_t ldl, float *lam, int64_t *landmarks);

/* The RBF kernel block K (n1 x n2, ldk): K_ij = exp(-||x_i - y_j||^2 / (2 sigma^2)) for the rows x_i of X and
 * y_j of Y (dimension d), the rbf function of Sec. 6.1, with the squared distance summed coordinate by
 * coordinate.  n2 <= 4,194,240. */
int rmc_rbf(rmc_ctx *ctx, const float *X, int64_t n1, int64_t ldx, const float *Y, int64_t n2, int64_t ldy,
            int64_t d, double sigma, float *K, int64_t ldk);

/* ------------------------------------------------- steps of the path, exposed for step-level checks */

/* Philox4x32-10 words of one stream: out[4*t + w] = word w of block (first + t), t < count (device, u32). */
int rmc_philox(rmc_ctx *ctx, uint64_t seed, uint32_t stream, uint32_t instance, uint64_t first,
               int64_t count, uint32_t *out);

/* Count sketch of the COLUMNS (the C = A S of Ch. 3 with Algorithm 3.1 over the columns): C (m x s, ldc) gets
 * C[:, h(j)] += g(j) A[:, j] for every column j, with h, g the stream-2 hashes of the column indices under
 * `instance`; each C[i, b] is summed in column order (deterministic).  1 <= s <= 256. */
int rmc_countsketch_columns(rmc_ctx *ctx, const float *A, int64_t m, int64_t n, int64_t lda, int64_t s,
                            uint64_t seed, uint32_t instance, float *C, int64_t ldc);

/* The rows x cols standard-normal matrix of stream 0 (row-major, leading dimension ld), FP32. */
int rmc_gaussian_matrix(rmc_ctx *ctx, uint64_t seed, uint32_t instance, int64_t rows, int64_t cols,
                        float *out, int64_t ld);

/* Count-sketch hash of rows 0..m-1: bucket[i] = h(i) in [0, s), sign[i] = g(i) (Algorithm 3.1). */
int rmc_countsketch_hash(rmc_ctx *ctx, uint64_t seed, uint32_t instance, int64_t m, int64_t s,
                         int32_t *bucket, float *sign);

/* The SRHT sample (the randsample-then-sort step of the Sec. 3.2.2 listing): idx[0..s) = the s indices of
 * [0, N) with the smallest stream-3 keys, ascending.  1 <= s <= N <= 2^31. */
int rmc_srht_sample(rmc_ctx *ctx, uint64_t seed, uint32_t instance, int64_t N, int64_t s, int64_t *idx);

/* CholeskyQR2 in place (the qr(., 0) of Algorithm 5.2 and of the Sec. 5.1 listing): Y (m x l, ldy, FP32) is
 * overwritten by Q with orthonormal columns; R (l x l row-major FP64, upper triangular, optional: NULL) gets
 * the factor with Y_in = Q R.  Each pass forms the Gram matrix with FP32 products summed in FP64 across 32-row
 * slices and factors it in FP32, falling back to an FP64 Cholesky on a non-positive pivot; with
 * RMC_OPT_SMALL_FP64 the products and the Cholesky are FP64.  Requires 1 <= l <= 256, m >= l.  RMC_ENUMERIC at
 * rmc_sync when the FP64 factorization meets a non-positive pivot too. */
int rmc_cholqr2(rmc_ctx *ctx, float *Y, int64_t m, int64_t l, int64_t ldy, double *R);

/* SVD of a short, wide matrix B (l x n, ldb, l <= n, l <= 256) -- the svd(Q^T A, 'econ') step of Algorithm
 * 5.2: B = Ub diag(sigma) Vb^T with Ub l x l (row-major, FP32), sigma[l] descending (FP32) and Vb n x l
 * (ldv, FP32).  Computed as CholeskyQR2 of B^T (B^T = Q2 R, the last pass with FP64 Gram products) and a
 * one-sided Jacobi SVD of R = M diag(sigma) V^T (FP32 rotations, FP64 for l <= 32 or with RMC_OPT_SMALL_FP64):
 * Vb = Q2 M; Ub = V = R^T M diag(sigma)^-1 (FP64 products) for l up to 240 (120 in FP64), so column j of Ub is
 * accurate to about eps * sigma_1 / sigma_j (the leading columns, those a k-SVD keeps, to FP32 level); larger l
 * accumulates the rotations instead. */
int rmc_svd_wide(rmc_ctx *ctx, const float *B, int64_t l, int64_t n, int64_t ldb, float *Ub,
                 float *sigma, float *Vb, int64_t ldv);

/* The products with A of the range finder, power iterations and projection (Algorithm 5.2 steps 3 and 5,
 * and the C = A' * C; C = A * C power step of the Sec. 5.1 listing):
 *   rmc_matmul_an:  Y (m x l, ldy) = A (m x n) * X, with X n x l (ldx).
 *   rmc_matmul_at:  W (l x n, ldw) = X^T * A,       with X m x l (ldx).
 * prec: RMC_FP32 (CUDA cores), RMC_TF32, RMC_TF32X3 or RMC_BF16 (tensor cores); FP32 accumulation.
 * 1 <= l <= 256. */
int rmc_matmul_an(rmc_ctx *ctx, const float *A, int64_t m, int64_t n, int64_t lda, const float *X,
                  int64_t l, int64_t ldx, int prec, float *Y, int64_t ldy);
int rmc_matmul_at(rmc_ctx *ctx, const float *A, int64_t m, int64_t n, int64_t lda, const float *X,
                  int64_t l, int64_t ldx, int prec, float *W, int64_t ldw);

/* ------------------------------------------------------------------- batches of small, uneven problems */

#define RMC_REQ_LSR   0   /* count-sketch sketch-and-solve least squares (Sec. 4.2 with Alg. 3.1)          */
#define RMC_REQ_RSVD  1   /* randomized k-SVD with q power iterations (Alg. 5.2, power step of Sec. 5.1)   */

/* One problem of a batch.  All pointers are device pointers owned by the caller.
 *   LSR:  A (m x n, lda), b (m), sketch size s (n <= s <= 1024), output x (n, FP64).
 *   RSVD: A (m x n, lda), k, p, q with l = k + p <= 32, outputs U (m x k, row stride k), sigma (k),
 *         V (n x k, row stride k); the same algorithm and sign convention as rmc_rsvd.
 * Limits for both: 1 <= m <= 2^24, 1 <= n <= 256, l <= min(m, n) for RSVD. */
typedef struct rmc_request {
  int kind;
  int k, p, q;
  int64_t m, n, lda, s;
  uint64_t seed;
  const float *A;
  const float *b;
  double *x;
  float *U, *sigma, *V;
} rmc_request;

/* Run every request of the batch in ONE persistent kernel launch (the Ch. 4 and Ch. 5 problems, many at
 * once): the host orders the requests largest first and lays out their workspace; each CTA then pulls whole
 * problems from a device queue and runs all of a problem's passes itself, so uneven problems balance across
 * the SMs without a launch per problem.  Results match rmc_lsr_sketch / rmc_rsvd on the same problem within
 * the FP32 tolerances of those calls.  The descriptor array is read before the call returns.
 * Errors: RMC_EINVAL (a request breaks the limits; nothing is enqueued), RMC_ENOMEM, RMC_ECUDA; RMC_ENUMERIC
 * at rmc_sync when a problem's factorization broke down (its outputs are then NaN). */
int rmc_batch_run(rmc_ctx *ctx, const rmc_request *reqs, int nreq);

/* Autotuned schedule of rmc_batch_run.  The k-SVD problems of a batch fall into 16 tuning classes (n in 1-64,
 * 65-128, 129-192, 193-256, times l = k + p rounded up to 8, 16, 24, 32); each class has a row-tile height for
 * the passes over A (0 = as many rows as a ring stage holds, else 32, 64 or 128).  rmc_batch_autotune times
 * every candidate on up to 256 of the caller's own problems per class (reps timed launches each, after one
 * warm-up) and keeps the fastest in the context's table, which later rmc_batch_run calls on this context use.
 * It runs the problems (their outputs are overwritten) and synchronises the stream.  rmc_batch_get_tiles /
 * rmc_batch_set_tiles read and write the table (count >= 16 entries; entries multiples of 16 in [0, 256]) so it
 * can be kept between processes.  Different tables change the summation order, not the results beyond FP32
 * rounding; for a fixed table a problem's result is the same alone or in any mix.
 * Errors: RMC_EINVAL (bad arguments or requests), RMC_ENOMEM, RMC_ECUDA, and the status of the runs. */
#define RMC_BATCH_TILE_CLASSES 16
int rmc_batch_autotune(rmc_ctx *ctx, const rmc_request *reqs, int nreq, int reps);
int rmc_batch_get_tiles(const rmc_ctx *ctx, int *table, int count);
int rmc_batch_set_tiles(rmc_ctx *ctx, const int *table, int count);

/* ------------------------------------------------------------------ continuous-batching request server */

/* A served request: one problem of Ch. 4 (sketch-and-solve least squares) or Ch. 5 (randomized k-SVD) plus how to
 * run it.  `req` is as for rmc_batch_run, except that here LSR allows n <= 1024 with any sketch kind and RSVD
 * allows l = k + p <= 256; its inputs and outputs are device memory that the caller keeps resident and
 * untouched until the request completes. */
typedef struct rmc_serve_request {
  rmc_request req;
  int sketch;   /* LSR: RMC_GAUSSIAN, RMC_SRHT or RMC_COUNTSKETCH (RSVD: ignored)                        */
  int prec;     /* operand precision of the products with A (RMC_FP32, RMC_TF32, RMC_TF32X3, RMC_BF16)       */
} rmc_serve_request;

typedef struct rmc_server rmc_server;

/* A server on the current device with `nstreams` streams (1..16), each with its own workspace of at most
 * hbm_budget / nstreams bytes: the device memory the server holds never exceeds hbm_budget.  Small requests
 * (count-sketch LSR with n <= 256, s <= 1024; FP32 RSVD with l <= 32, n <= 256) are batched, up to
 * max_batch per launch, into rmc_batch_run launches; the others run one per launch through rmc_lsr_sketch /
 * rmc_rsvd.  Launches on different streams overlap on the device.  Single-threaded: one host thread drives
 * a server.  The paper has no counterpart (it treats one problem at a time). */
int rmc_server_create(rmc_server **out, size_t hbm_budget, int nstreams, int max_batch);
/* Waits for every launch in flight, then frees the server. */
int rmc_server_destroy(rmc_server *srv);
/* Queue a request; *ticket identifies it in rmc_server_poll.  Never blocks.  RMC_EINVAL for a malformed
 * request, RMC_ENOMEM when its workspace alone exceeds one stream's share of the budget. */
int rmc_server_submit(rmc_server *srv, const rmc_serve_request *req, uint64_t *ticket);
/* Retire finished launches, then admit queued requests onto free streams (continuous batching: a request
 * that arrives while others run is admitted as soon as a stream and its memory free up).  Never blocks.
 * Returns the number of requests in flight and still queued (either pointer may be NULL). */
int rmc_server_progress(rmc_server *srv, int *inflight, int *queued);
/* Completed requests since the last poll, in completion order: ticket, status (RMC_OK or the error its
 * launch reported) and latency in seconds from submit to the progress call that saw it finish. */
int rmc_server_poll(rmc_server *srv, uint64_t *tickets, int *status, double *latency_s, int max, int *count);
/* Progress until nothing is queued or in flight (blocks, yielding the CPU between checks). */
int rmc_server_drain(rmc_server *srv);
/* Residency of served least-squares state (the paper has no counterpart; a serving concern).  With a nonzero
 * byte cap, least-squares requests submitted afterwards take the resident route: for each (A, m, n, lda, sketch
 * kind, s, seed, precision) the server keeps the sketch S^T A and the preconditioner of its factor (the M of
 * rmc_lsr_sketch's refinement) in device memory, so a later request on the same matrix and sketch sketches only
 * its own b and refines against them.  Requests that find no resident state sketch and factor first (into a new
 * entry when the cap allows, evicting the least recently used entries that no launch reads, else into the
 * lane's workspace); the values are the same either way, so a result does not depend on what is resident.  The
 * route solves [S^T A, S^T b] with S^T b sketched on its own (not as one more column of A), so its x can differ
 * from rmc_lsr_sketch's in the last bits.  Resident memory is allocated stream-ordered and held in addition to
 * the lanes' workspaces.  A matrix with resident state must stay unchanged until rmc_server_release(A) (call it
 * before modifying or freeing A); bytes = 0 turns residency off and drops the state.  Errors: RMC_EINVAL. */
int rmc_server_resident(rmc_server *srv, size_t bytes);
int rmc_server_release(rmc_server *srv, const float *A);

/* ------------------------------------------------------------------------------- measurement hooks */

/* Kernel tags for rmc_profile_read. */
#define RMC_K_COUNTSKETCH  0   /* count-sketch gather-accumulate pass over A                         */
#define RMC_K_SRHT         1   /* SRHT stage 1: sign flip + FWHT of A's 4096-row blocks              */
#define RMC_K_SRHT_REDUCE  2   /* SRHT stage 2: combination of the row blocks for the sampled rows   */
#define RMC_K_GAUSSIAN     3   /* Gaussian sketch product with in-kernel Philox draws                */
#define RMC_K_MATMUL_AN    4   /* Y = A X                                                            */
#define RMC_K_MATMUL_AT    5   /* W = X^T A                                                          */
#define RMC_K_GRAM         6   /* FP64 Gram matrix of CholeskyQR2 / the least-squares solve          */
#define RMC_K_SMALL        7   /* Cholesky, triangular inverse, Jacobi SVD (single-block kernels)    */
#define RMC_K_BATCH        8   /* persistent batch kernel of rmc_batch_run                           */
#define RMC_K_LSR_PASS     9   /* residual + gradient pass over A of rmc_lsr_precise                 */
#define RMC_K_RBF         10   /* RBF kernel block of rmc_nystrom / rmc_rbf                          */
#define RMC_K_NTAGS       11

/* While profiling is on, the kernels above are bracketed by CUDA events recorded on the context's stream.
 * rmc_profile_begin clears the records; rmc_profile_read waits for the stream and returns, for one tag, the
 * number of launches and their summed device time in milliseconds (profiling stays on). */
int rmc_profile_begin(rmc_ctx *ctx);
int rmc_profile_read(rmc_ctx *ctx, int tag, int64_t *launches, double *total_ms);
int rmc_profile_end(rmc_ctx *ctx);

/* Launch intervals, for kernels that run concurrently on several streams (a launch's event pair then also
 * spans the time it waits for another stream's CTAs to leave the SMs).  rmc_profile_reference records one
 * process-wide reference event on the context's stream.  rmc_profile_spans waits for the stream and writes, for
 * each launch of `tag` recorded on this context since rmc_profile_begin and completed after the reference was
 * recorded, its start and stop times in milliseconds relative to that reference (host arrays of `max` entries;
 * *count = the number written; at most 4096 per context).  Errors: RMC_EINVAL (no reference recorded, bad
 * argument), RMC_ECUDA. */
int rmc_profile_reference(rmc_ctx *ctx);
int rmc_profile_spans(rmc_ctx *ctx, int tag, double *start_ms, double *stop_ms, int max, int *count);

/* Test hook for the delivery of device-side timeouts: enqueue one kernel whose bounded wait on a flag that
 * nothing sets runs out after limit_ns (at most 1 s), reports RMC_ETIMEOUT to the context's status word and
 * returns -- the same path every bounded wait of the library takes (mbarrier waits of the tensor-core kernels,
 * the batch ring).  The next rmc_sync returns RMC_ETIMEOUT and clears it; the context stays usable.
 * Errors: RMC_EINVAL (NULL context, limit above 1 s), RMC_ENOMEM, RMC_ECUDA. */
int rmc_debug_wait_timeout(rmc_ctx *ctx, uint64_t limit_ns);

/* Measurement hook for the drawing bound of the tensor-core Gaussian sketch: enqueue one kernel that draws the
 * m x s normals of the sketch's operator (Philox stream 4, the Box-Muller pairs of rmc_sketch's RMC_GAUSSIAN
 * tensor-core forms, rounded to TF32) with one CTA of 16 drawing warps per SM -- the sketch kernel's drawing
 * warps, with no product, staging or barrier -- and write their FP64 sum to *sum (device memory).  Its device
 * time is the time the sketch of an m-row matrix to s rows spends drawing at best.  Errors: RMC_EINVAL,
 * RMC_ECUDA. */
int rmc_gaussian_draw_floor(rmc_ctx *ctx, int64_t m, int64_t s, uint64_t seed, double *sum);

/* Number of kernels this library has launched in the process so far (all contexts). */
int rmc_launch_counter(uint64_t *launches);

/* ------------------------------------------------------------------ count sketch without allocation */

/* Bytes of the fixed device scratch array behind rmc_countsketch_noalloc. */
#define RMC_NOALLOC_SCRATCH_BYTES (32u << 20)

/* Count sketch C = S^T A (s x n, ldc), the same operator and result as rmc_sketch(..., RMC_COUNTSKETCH, ...),
 * for callers that must not allocate device memory at call time: a serving loop that reserves all of its
 * HBM up front and keeps allocation (which can synchronise the device) off its request path, or a host
 * framework whose device memory belongs to its own allocator.  Such a caller cannot use a context either,
 * since rmc_create allocates.  The paper has no counterpart.
 *
 * Nothing is allocated: no cudaMalloc, cudaFree or allocating library call.  The sorting scratch lives in
 * one file-scope __device__ array of RMC_NOALLOC_SCRATCH_BYTES (32 MiB), which every GPU that loads the
 * library holds until the process exits.  Every call looks up that array's device address on the current
 * device (cudaGetSymbolAddress); the first call on a device may load the module there, so make that first
 * call before any stream capture.  All calls share the one array and it keeps the previous call's contents
 * (the counters are cleared on the stream before use), so calls whose work overlaps on the GPU -- on
 * different streams, or from different host threads -- race on it and must be serialised by the caller.
 *   cuda_stream: the cudaStream_t to enqueue on (NULL = legacy default stream), on the current device.
 *   A, C: device pointers as for rmc_sketch (A m x n, lda >= n; C s x n, ldc >= n).
 * Returns RMC_OK once enqueued; RMC_EINVAL for bad arguments; RMC_ESCRATCH when the call would need more
 * than RMC_NOALLOC_SCRATCH_BYTES (about 8 m + 4 s ceil(m / 1024) bytes; e.g. m = 2^20 rows fit up to
 * s = 4096); RMC_ECUDA if the address lookup or a launch fails.  Nothing is enqueued on RMC_EINVAL or
 * RMC_ESCRATCH. */
int rmc_countsketch_noalloc(void *cuda_stream, const float *A, int64_t m, int64_t n, int64_t lda, int64_t s,
                            uint64_t seed, float *C, int64_t ldc);

#ifdef __cplusplus
}
#endif

#endif /* RMC_H */
