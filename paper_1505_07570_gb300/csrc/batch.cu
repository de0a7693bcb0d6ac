// Many small, uneven randomized least-squares and randomized-SVD problems in ONE persistent launch.
//
// Each CTA takes whole problems from a device queue (the host orders them largest first, so the long ones
// start early and the short ones fill the tail) and runs every step of a problem itself:
//   * count-sketch sketch-and-solve least squares (Sec. 4.2 with the count sketch of Algorithm 3.1):
//     hash the rows, counting-sort them by bucket, gather [S^T A, S^T b], Gram matrix, Cholesky, then
//     solves with two steps of iterative refinement against the sketched matrix;
//   * the randomized k-SVD with q power iterations (Algorithm 5.2 with the power step of Sec. 5.1):
//     Y = A Omega, one CholeskyQR pass for intermediate bases and CholeskyQR2 for the final one,
//     B = Q^T A, B^T = Q2 R by CholeskyQR2, one-sided Jacobi on R, U = Q Ub, V = Q2 Vr.
// A problem's A streams through shared memory in row tiles (cp.async, three stages).  Every product with
// A is an FP32 register-tiled SIMT product out of those tiles: with l <= 32 columns in Omega there is too
// little reuse per byte for tensor cores to matter, and the aggregate over the batch is bound by HBM.
// Factorizations are FP32 in shared memory (FP64 Gram sums, FP64 fallback for the small Cholesky).

#include <math.h>
#include <stdint.h>

#include <string.h>

#include <algorithm>
#include <vector>

#include "philox.cuh"
#include "rmc_internal.cuh"
#include "tc_common.cuh"

namespace {

constexpr int kThreads = 512;
constexpr int kWarps = kThreads / 32;
// Two large stages: the cost of a tile is dominated by its barriers and short dependent phases, not by load
// latency (one tile of ~73 KB in flight already streams at this SM's share of HBM), so fewer, larger tiles win.
constexpr int kStages = 2;
constexpr int kStageFloats = 18752;  // one stage of the row-tile ring (73.25 KB)
constexpr int kPartFloats = 8192;    // k-split partial products, the product tile, small-SVD matrices (32 KB)
constexpr int kZFloats = 256 * 32;   // Omega / Z / B^T / Q2, n x l (32 KB)
constexpr int kSmallFloats = 4096;   // T^-1 and R^-1 (FP32, 32 x 32) and the FP64 Gram matrix (32 x 32)
constexpr int kSmemFloats = kStages * kStageFloats + kPartFloats + kZFloats + kSmallFloats;
constexpr size_t kSmemBytes = sizeof(float) * kSmemFloats;
constexpr int kMaxN = 256, kMaxL = 32, kMaxS = 1024;
constexpr int64_t kMaxM = int64_t(1) << 24;

struct BatchItem {
  int kind, k, p, q;
  int m, n, s, vec;   // vec: rows of A start on 16-byte boundaries (16-byte cp.async)
  int rtile;          // rsvd: cap on the row-tile height (multiple of 16; 0 = as many rows as a stage holds)
  int64_t lda;
  uint64_t seed;
  const float *A, *b;
  double *x;
  float *U, *sigma, *V;
  float *ws0;         // rsvd: Y, then Q1 (m x LP); lsr: [S^T A, S^T b] (s x n8)
  uint32_t *ws1;      // lsr: bucket keys (m), then the row permutation (m)
  float *ws2;         // lsr: Gram block partials
};

// ------------------------------------------------------------------------------------- small helpers

__device__ __forceinline__ void cp16(float *dst, const float *src, int bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
               "l"(src), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void cp4(float *dst, const float *src, int bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
               "l"(src), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

template <int C>
__device__ __forceinline__ void ld_vec(const float *p, float (&v)[C]) {
  if constexpr (C % 4 == 0) {
#pragma unroll
    for (int i = 0; i < C; i += 4) {
      const float4 t = *reinterpret_cast<const float4 *>(p + i);
      v[i] = t.x; v[i + 1] = t.y; v[i + 2] = t.z; v[i + 3] = t.w;
    }
  } else {
#pragma unroll
    for (int i = 0; i < C; i += 2) {
      const float2 t = *reinterpret_cast<const float2 *>(p + i);
      v[i] = t.x; v[i + 1] = t.y;
    }
  }
}
template <int C>
__device__ __forceinline__ void st_vec(float *p, const float (&v)[C]) {
  if constexpr (C % 4 == 0) {
#pragma unroll
    for (int i = 0; i < C; i += 4) *reinterpret_cast<float4 *>(p + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
  } else {
#pragma unroll
    for (int i = 0; i < C; i += 2) *reinterpret_cast<float2 *>(p + i) = make_float2(v[i], v[i + 1]);
  }
}


// Rows [r0, r0 + R) of a row-major matrix (leading dimension ld) into shared memory with row stride S:
// columns [0, ncols), zeros in columns [ncols, npad) (npad a multiple of 4) and in rows at or past `rows`.
__device__ __forceinline__ void load_rows(float *dst, int S, const float *src, int64_t ld, int r0, int R, int rows,
                                          int ncols, int npad, bool vec) {
  const int nq = npad >> 2, total = R * nq;
  // element e = threadIdx.x + k kThreads is (row r, quad q) with e = r nq + q, stepped without a division per
  // element (a runtime division costs tens of instructions, more than the copy itself)
  const int dr = kThreads / nq, dq = kThreads - dr * nq;
  int r = threadIdx.x / nq, q = threadIdx.x - r * nq;
  for (int e = threadIdx.x; e < total; e += kThreads) {
    const int c = q << 2;
    float *d = dst + r * S + c;
    const bool ok = r0 + r < rows;
    const float *s = ok ? src + (int64_t)(r0 + r) * ld + c : src;
    const int cnt = ok ? max(0, min(4, ncols - c)) : 0;
    if (vec) {
      cp16(d, cnt ? s : src, cnt * 4);
    } else {
#pragma unroll
      for (int u = 0; u < 4; ++u) cp4(d + u, u < cnt ? s + u : src, u < cnt ? 4 : 0);
    }
    r += dr;
    q += dq;
    if (q >= nq) {
      q -= nq;
      ++r;
    }
  }
}

// One bulk (TMA) copy global -> shared, completing on an mbarrier (both addresses 16-byte aligned, bytes a
// multiple of 16).
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   tc::smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(tc::smem_u32(bar))
               : "memory");
}

// Rows [r0, r0 + R) of a matrix whose rows are contiguous (leading dimension == ncols) and whose tile start is
// 16-byte aligned (R ncols a multiple of 4): one span of R ncols floats into a dense tile (row stride ncols).
// Thread 0 issues the 16-byte-multiple prefix as one bulk copy; all threads fill the rest of the tile and a
// 16-float tail (the < 4 leftover floats from global memory, zeros past the valid rows).  Returns the bytes
// the bulk copy will deliver (the caller arms the mbarrier with them).
struct Span {
  float *dst;
  const float *src;
  uint32_t bytes;
};
__device__ __forceinline__ Span span_tile(float *dst, const float *src, int r0, int R, int rows, int ncols) {
  const int64_t base = (int64_t)r0 * ncols;
  const int span = max(0, min(R, rows - r0)) * ncols, pre = span & ~3;
  for (int f = pre + threadIdx.x; f < R * ncols + 16; f += kThreads) dst[f] = f < span ? src[base + f] : 0.f;
  return Span{dst, src + base, (uint32_t)pre * 4u};
}

// Thread 0: arm the stage's mbarrier with the spans' bytes and issue their bulk copies (spans of 0 bytes skip).
__device__ __forceinline__ void issue_spans(uint64_t *bar, Span a, Span b = Span{nullptr, nullptr, 0u}) {
  if (threadIdx.x != 0) return;
  tc::fence_proxy_async_smem();  // this stage's earlier generic accesses come before the async writes
  tc::mbar_arrive_expect_tx(bar, a.bytes + b.bytes);
  if (a.bytes) bulk_g2s(a.dst, a.src, a.bytes, bar);
  if (b.bytes) bulk_g2s(b.dst, b.src, b.bytes, bar);
}

// The row-tile ring: kStages stages in shared memory with one mbarrier each.  Every load arms its stage's
// mbarrier exactly once (with 0 bytes when it used cp.async only), so the barrier phases stay in step.
struct Ring {
  float *buf;
  uint64_t *full;
  uint32_t phase;  // bit s: parity of the next completion of stage s
};

// Stream rows [0, rows) in tiles of R rows: load(stage, r0, bar) issues one tile (cp.async by all threads and/or
// spans via issue_spans), use(stage, r0) consumes it.  Loads run kStages - 1 tiles ahead.  Thread 0 waits on the
// mbarrier (bounded: RMC_ETIMEOUT to *status) and a CTA barrier passes the tile on.
template <class Load, class Use>
__device__ __forceinline__ void stream_tiles(Ring &rg, int rows, int R, int *status, Load load, Use use) {
  const int T = (rows + R - 1) / R;
#pragma unroll 1
  for (int s = 0; s < kStages - 1; ++s) {
    if (s < T) load(rg.buf + s * kStageFloats, s * R, &rg.full[s]);
    cp_commit();
  }
#pragma unroll 1
  for (int t = 0; t < T; ++t) {
    const int st = t % kStages;
    cp_wait<kStages - 2>();
    if (threadIdx.x == 0 && !tc::mbar_wait(&rg.full[st], (rg.phase >> st) & 1u)) rmc_report(status, RMC_ETIMEOUT);
    rg.phase ^= 1u << st;
    __syncthreads();  // tile t is in; every thread is done with tile t - 1, whose stage is refilled next
    if (t + kStages - 1 < T) {
      const int sn = (t + kStages - 1) % kStages;
      load(rg.buf + sn * kStageFloats, (t + kStages - 1) * R, &rg.full[sn]);
    }
    cp_commit();
    use(rg.buf + st * kStageFloats, t * R);
  }
  cp_wait<0>();
  __syncthreads();
}

// ------------------------------------------------------------------------- products out of row tiles

// Warp-level tensor-core products in FP32 accuracy: mma.sync m16n8k8 on TF32 operands, each operand split into a
// TF32 high part and a TF32 remainder, D += A_lo B_hi + A_hi B_lo + A_hi B_hi (the A_lo B_lo term, below 2^-22 of
// the product, is dropped).  Fragment layout of m16n8k8 (g = lane / 4, t = lane % 4): A a0 (g, t), a1 (g + 8, t),
// a2 (g, t + 4), a3 (g + 8, t + 4); B b0 (k = t, n = g), b1 (k = t + 4, n = g); C c0 (g, 2t), c1 (g, 2t + 1),
// c2 (g + 8, 2t), c3 (g + 8, 2t + 1).
// TF32 rounding to nearest, ties away from zero (the rounding of cvt.rna.tf32.f32), on the bit pattern with integer
// operations, which issue at a much higher rate than the conversion instruction.  Finite inputs only.
__device__ __forceinline__ uint32_t tf32_rna(float x) { return (__float_as_uint(x) + 0x1000u) & 0xFFFFE000u; }
__device__ __forceinline__ void split_tf32(float x, uint32_t &hi, uint32_t &lo) {
  hi = tf32_rna(x);
  lo = tf32_rna(x - __uint_as_float(hi));
}
__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
__device__ __forceinline__ void mma3(float (&d)[4], const uint32_t (&ah)[4], const uint32_t (&al)[4], float b0,
                                     float b1) {
  uint32_t bh0, bl0, bh1, bl1;
  split_tf32(b0, bh0, bl0);
  split_tf32(b1, bh1, bl1);
  mma_tf32(d, al, bh0, bh1);  // small terms first
  mma_tf32(d, ah, bl0, bl1);
  mma_tf32(d, ah, bh0, bh1);
}

// P[ks] (R x LP) = A_tile[:, k-steps of slice ks] Z[those rows, :]: warp unit (16-row block mb, k slice ks),
// all LP / 8 column blocks, k-steps of 8 columns of A.
template <int TN>
__device__ __forceinline__ void tile_times_z(const float *At, int S, int R, int ksplit, int kb_per, int KB,
                                             const float *Z, float *P) {
  constexpr int LP = 4 * TN, NB = LP / 8;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int MB = R >> 4;
  for (int u = warp; u < MB * ksplit; u += kWarps) {
    const int mb = u % MB, ks = u / MB;
    const int k0 = ks * kb_per, k1 = min(KB, k0 + kb_per);
    float acc[NB][4];
#pragma unroll
    for (int nb = 0; nb < NB; ++nb) acc[nb][0] = acc[nb][1] = acc[nb][2] = acc[nb][3] = 0.f;
    const float *ap = At + (mb * 16 + g) * S + t;
    const float *zp = Z + t * LP + g;
#pragma unroll 2
    for (int kb = k0; kb < k1; ++kb) {
      const float *a = ap + kb * 8;
      uint32_t ah[4], al[4];
      split_tf32(a[0], ah[0], al[0]);
      split_tf32(a[8 * S], ah[1], al[1]);
      split_tf32(a[4], ah[2], al[2]);
      split_tf32(a[8 * S + 4], ah[3], al[3]);
      const float *z = zp + kb * 8 * LP;
#pragma unroll
      for (int nb = 0; nb < NB; ++nb) mma3(acc[nb], ah, al, z[nb * 8], z[4 * LP + nb * 8]);
    }
    float *pp = P + (size_t)ks * R * LP + (mb * 16 + g) * LP + 2 * t;
#pragma unroll
    for (int nb = 0; nb < NB; ++nb) {
      *reinterpret_cast<float2 *>(pp + nb * 8) = make_float2(acc[nb][0], acc[nb][1]);
      *reinterpret_cast<float2 *>(pp + 8 * LP + nb * 8) = make_float2(acc[nb][2], acc[nb][3]);
    }
  }
}

// acc (warp unit: 16 columns of A in block mb, k-steps kb = rs, rs + RS, ...) += A_tile^T Y_tile: the m16 x n8
// blocks of W^T (columns of A x LP).
template <int TN>
__device__ __forceinline__ void at_times_y(const float *At, int S, const float *Yt, int R, int mb, int rs, int RS,
                                           float (&acc)[TN / 2][4]) {
  constexpr int LP = 4 * TN, NB = LP / 8;
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const float *ap = At + t * S + mb * 16 + g;
  const float *yp = Yt + t * LP + g;
#pragma unroll 2
  for (int kb = rs; kb < (R >> 3); kb += RS) {
    const float *a = ap + kb * 8 * S;
    uint32_t ah[4], al[4];
    split_tf32(a[0], ah[0], al[0]);
    split_tf32(a[8], ah[1], al[1]);
    split_tf32(a[4 * S], ah[2], al[2]);
    split_tf32(a[4 * S + 8], ah[3], al[3]);
    const float *y = yp + kb * 8 * LP;
#pragma unroll
    for (int nb = 0; nb < NB; ++nb) mma3(acc[nb], ah, al, y[nb * 8], y[4 * LP + nb * 8]);
  }
}

// Sum the KS slices of P into slice 0, in slice order.
__device__ __forceinline__ void reduce_slices(float *P, int count4, int KS) {
  if (KS <= 1) return;
  float4 *P4 = reinterpret_cast<float4 *>(P);
  for (int e = threadIdx.x; e < count4; e += kThreads) {
    float4 s = P4[e];
    for (int sl = 1; sl < KS; ++sl) {
      const float4 v = P4[sl * count4 + e];
      s.x += v.x; s.y += v.y; s.z += v.z; s.w += v.w;
    }
    P4[e] = s;
  }
}

// acc += X_tile^T T_tile over the tile's rows.  Thread (jg, cq, g) owns rows jg TN .. of the result and
// columns 4 cq .. 4 cq + 3, and takes tile rows g, g + G, ...
template <int TN>
__device__ __forceinline__ void xt_accum(const float *X, int LX, const float *T, int ST, int R, int nqT, int G,
                                         float (&acc)[TN][4]) {
  const int t = threadIdx.x, jg = t & 3, rest = t >> 2, cq = rest % nqT, g = rest / nqT;
  if (g >= G) return;
  const float *x = X + jg * TN, *tt = T + 4 * cq;
#pragma unroll 2
  for (int r = g; r < R; r += G) {
    const float4 a = *reinterpret_cast<const float4 *>(tt + r * ST);
    float xv[TN];
    ld_vec<TN>(x + r * LX, xv);
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      acc[j][0] = fmaf(xv[j], a.x, acc[j][0]);
      acc[j][1] = fmaf(xv[j], a.y, acc[j][1]);
      acc[j][2] = fmaf(xv[j], a.z, acc[j][2]);
      acc[j][3] = fmaf(xv[j], a.w, acc[j][3]);
    }
  }
}

// Write each group's accumulator to scr[g] (LP x 4 nqT, row-major).
template <int TN>
__device__ __forceinline__ void dump_acc(float *scr, int nqT, int G, const float (&acc)[TN][4]) {
  constexpr int LP = 4 * TN;
  const int t = threadIdx.x, jg = t & 3, rest = t >> 2, cq = rest % nqT, g = rest / nqT;
  if (g >= G) return;
  const int W4 = 4 * nqT;
  float *d = scr + (size_t)g * LP * W4 + 4 * cq;
#pragma unroll
  for (int j = 0; j < TN; ++j)
    *reinterpret_cast<float4 *>(d + (jg * TN + j) * W4) = make_float4(acc[j][0], acc[j][1], acc[j][2], acc[j][3]);
}

template <int TN>
__device__ __forceinline__ void zero_acc(float (&acc)[TN][4]) {
#pragma unroll
  for (int j = 0; j < TN; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
}
template <int TN>
__device__ __forceinline__ void add_acc(float (&tot)[TN][4], const float (&a)[TN][4]) {
#pragma unroll
  for (int j = 0; j < TN; ++j)
#pragma unroll
    for (int c = 0; c < 4; ++c) tot[j][c] += a[j][c];
}

// G64 (ld 32) = sum over the G groups of the l x l leading block of scr, in group order, in FP64.
__device__ __forceinline__ void gram_reduce64(const float *scr, int LP, int G, int l, double *G64) {
  for (int e = threadIdx.x; e < l * l; e += kThreads) {
    const int i = e / l, j = e - i * l;
    double s = 0.0;
    for (int g = 0; g < G; ++g) s += (double)scr[((size_t)g * LP + i) * LP + j];
    G64[i * 32 + j] = s;
  }
}

// ----------------------------------------------------------------------------- small factorizations

// Upper Cholesky factor of the l x l matrix G64 (ld 32) and its inverse, both FP32 with ld 32 and zeros
// outside the leading l x l block.  All threads of the CTA: right-looking, each step's trailing update spread
// over the CTA.  A pivot that is not positive means cond(Y)^2 is beyond FP32: the factorization is repeated on
// G + sigma I with sigma = 64 l 2^-23 max_i G_ii, just above the Gram matrix's rounding (shifted CholeskyQR:
// Y R^-1 is then well conditioned though not orthonormal, and every basis the result depends on takes a
// second, unshifted pass; R = R_b R_a stays exact for B^T = Q2 R).  If that fails too, warp 0 repeats it in
// FP64 (in place in G64), and then R is NaN and the problem reports RMC_ENUMERIC.  The inverse is formed one
// column per warp (column j: x = e_j, then x_i /= R_ii and x_c -= R_ci x_i for c < i, from i = j down).
__device__ bool chol_small_attempt(const double *G64, int l, float shift, float *R, int *flag) {
  const int t = threadIdx.x;
  for (int e = t; e < 1024; e += kThreads) {
    const int i = e >> 5, j = e & 31;
    R[e] = (i < l && j < l && j >= i) ? (float)G64[i * 32 + j] + (i == j ? shift : 0.f) : 0.f;
  }
  if (t == 0) *flag = 0;
  __syncthreads();
  for (int k = 0; k < l; ++k) {
    const float d = R[k * 32 + k];
    if (!(d > 0.f) || !(d < INFINITY)) {  // every thread sees the same pivot
      if (t == 0) *flag = 1;
      break;
    }
    const float rd = sqrtf(d);
    __syncthreads();  // the pivot is read before row k changes
    if (t >= k && t < l) R[k * 32 + t] = t == k ? rd : R[k * 32 + t] / rd;
    __syncthreads();
    for (int e = t; e < 1024; e += kThreads) {
      const int i = e >> 5, j = e & 31;
      if (i > k && i <= j && j < l) R[e] = fmaf(-R[k * 32 + i], R[k * 32 + j], R[e]);
    }
    __syncthreads();
  }
  __syncthreads();
  const bool ok = *flag == 0;
  __syncthreads();
  return ok;
}

__device__ void factor_small(double *G64, int l, float *R, float *Ri, int *flag, int *status) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  bool ok = chol_small_attempt(G64, l, 0.f, R, flag);  // the same value in every thread
  if (!ok) {
    float dmax = 0.f;
    for (int i = 0; i < l; ++i) dmax = fmaxf(dmax, (float)G64[i * 32 + i]);
    ok = chol_small_attempt(G64, l, 64.f * (float)l * 1.1920929e-7f * dmax, R, flag);
  }
  if (!ok) {
    if (warp == 0) {  // FP64 retry, in place in G64's upper triangle
      ok = true;
      for (int k = 0; k < l; ++k) {
        const double d = G64[k * 32 + k];
        if (!(d > 0.0) || !(d < INFINITY)) { ok = false; break; }
        const double rd = sqrt(d);
        const double rkj = (lane > k && lane < l) ? G64[k * 32 + lane] / rd : 0.0;
        __syncwarp();
        if (lane == k) G64[k * 32 + k] = rd;
        if (lane > k && lane < l) G64[k * 32 + lane] = rkj;
        __syncwarp();
        if (lane > k && lane < l)
          for (int i = k + 1; i <= lane; ++i) G64[i * 32 + lane] -= G64[k * 32 + i] * rkj;
        __syncwarp();
      }
      for (int i = 0; i < 32; ++i)
        R[i * 32 + lane] = (i < l && lane < l && lane >= i) ? (ok ? (float)G64[i * 32 + lane] : nanf("")) : 0.f;
      if (!ok && lane == 0) rmc_report(status, RMC_ENUMERIC);
    }
    __syncthreads();
  }
  for (int j = warp; j < 32; j += kWarps) {
    float x = lane == j ? 1.f : 0.f;
    if (j < l) {
      for (int i = j; i >= 0; --i) {
        const float xi = __shfl_sync(0xffffffffu, x, i) / R[i * 32 + i];
        if (lane == i) x = xi;
        if (lane < i) x = fmaf(-R[lane * 32 + i], xi, x);
      }
    } else {
      x = 0.f;
    }
    Ri[lane * 32 + j] = lane < l ? x : 0.f;
  }
  __syncthreads();
}

// X[r, :] <- X[r, :] M for rows r < rows (LP columns, row stride LP).  M is 32 x 32 (ld 32) with zeros
// outside its leading l x l block; `upper` skips its zero lower triangle.
template <int TN, bool upper>
__device__ __forceinline__ void rows_times(float *X, int rows, const float *M) {
  constexpr int LP = 4 * TN;
  const volatile float *Mv = M;  // volatile: keeps the compiler from hoisting all of M into registers
  for (int r = threadIdx.x; r < rows; r += kThreads) {
    float v[LP];
    ld_vec<LP>(X + r * LP, v);
#pragma unroll
    for (int j = 0; j < LP; ++j) {
      float s = 0.f;
#pragma unroll
      for (int i = 0; i < LP; ++i)
        if (!upper || i <= j) s = fmaf(v[i], Mv[i * 32 + j], s);
      X[r * LP + j] = s;  // the row's inputs are all in registers already
    }
  }
}

// One-sided Jacobi on W (l x l, column j at W + 32 j), rotations accumulated into V; round-robin pairing,
// one warp per column pair.  Rotation of the one-sided (Hestenes) method with correctly rounded reciprocal
// and square root so that c^2 + s^2 does not drift below 1.
__device__ void jacobi_small(float *W, float *V, int l, int *flag, int *status) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int e = threadIdx.x; e < 1024; e += kThreads) V[e] = ((e >> 5) == (e & 31) && (e & 31) < l) ? 1.f : 0.f;
  const int lp = (l + 1) & ~1;
  const float tol = 4.f * 1.1920929e-7f * sqrtf((float)l);
  int sweep = 0;
  for (; sweep < 60; ++sweep) {
    if (threadIdx.x == 0) *flag = 0;
    __syncthreads();
    for (int round = 0; round < lp - 1; ++round) {
      if (warp < lp / 2) {
        const int a = warp, b = lp - 1 - warp;
        int p = a == 0 ? 0 : 1 + (a - 1 + round) % (lp - 1);
        int q = b == 0 ? 0 : 1 + (b - 1 + round) % (lp - 1);
        if (p > q) { const int t = p; p = q; q = t; }
        if (q < l) {
          float *wp = W + 32 * p, *wq = W + 32 * q;
          const float x = lane < l ? wp[lane] : 0.f, y = lane < l ? wq[lane] : 0.f;
          float alpha = x * x, beta = y * y, gamma = x * y;
#pragma unroll
          for (int o = 16; o; o >>= 1) {
            alpha += __shfl_xor_sync(0xffffffffu, alpha, o);
            beta += __shfl_xor_sync(0xffffffffu, beta, o);
            gamma += __shfl_xor_sync(0xffffffffu, gamma, o);
          }
          if (gamma != 0.f && fabsf(gamma) > tol * sqrtf(alpha * beta)) {
            const float zeta = (beta - alpha) * __frcp_rn(2.f * gamma);
            const float tt = copysignf(1.f, zeta) * __frcp_rn(fabsf(zeta) + __fsqrt_rn(fmaf(zeta, zeta, 1.f)));
            const float c = __frcp_rn(__fsqrt_rn(fmaf(tt, tt, 1.f))), s = c * tt;
            if (lane < l) {
              wp[lane] = c * x - s * y;
              wq[lane] = s * x + c * y;
              float *vp = V + 32 * p, *vq = V + 32 * q;
              const float u = vp[lane], v = vq[lane];
              vp[lane] = c * u - s * v;
              vq[lane] = s * u + c * v;
            }
            if (lane == 0) *flag = 1;
          }
        }
      }
      __syncthreads();
    }
    const int rotated = *flag;
    __syncthreads();
    if (!rotated) break;
  }
  if (sweep == 60 && threadIdx.x == 0) rmc_report(status, RMC_ENUMERIC);
}

// ------------------------------------------------------------------------------------- rsvd problem

struct RsvdGeo {
  int m, n, nz, S, R, MB, KB, ksplit, kb_per, GY, MBW, RS, R2, yoff;
  bool dense;
};

template <int TN>
__device__ void rsvd_problem(const BatchItem &it, float *sm, Ring &rg, int *flag, int *status) {
  constexpr int LP = 4 * TN;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int l = it.k + it.p, k = it.k;
  RsvdGeo g;
  g.m = it.m;
  g.n = it.n;
  g.nz = (g.n + 15) & ~15;  // Z rows and A tile columns, zero-padded to whole 16-column MMA blocks
  // Contiguous A: each tile is one 16-byte aligned span copied into a dense tile (row stride n); the columns
  // n..nz-1 the MMAs read then hold the next row's (finite) values, which meet zero rows of Z in A Z, and the
  // rows c >= n of A^T Y are dropped.  Otherwise rows go one by one into a zero-padded tile (stride nz + 4,
  // which puts the 8 rows of an A fragment in 8 different bank quads).
  g.dense = it.lda == it.n && (reinterpret_cast<uintptr_t>(it.A) & 15) == 0;
  g.S = g.dense ? g.n : g.nz + 4;
  g.R = min(256, (kStageFloats - 32) / (g.S + LP)) & ~15;  // A span + Y span, each with a 16-float tail
  if (it.rtile >= 16 && it.rtile < g.R) g.R = it.rtile & ~15;  // the tuned row tile of this problem's class
  g.yoff = g.R * g.S + (g.dense ? 16 : 0);  // where the W pass puts the Y tile in a stage
  g.MB = g.R >> 4;
  g.KB = g.nz >> 3;
  g.ksplit = max(1, min(kWarps / g.MB, g.KB));
  g.kb_per = (g.KB + g.ksplit - 1) / g.ksplit;
  g.ksplit = (g.KB + g.kb_per - 1) / g.kb_per;
  g.GY = kThreads / LP;           // row groups of the Gram accumulation (4 TN threads per group)
  g.MBW = g.nz >> 4;              // 16-column blocks of A in the W^T = A^T Y product
  g.RS = max(1, kWarps / g.MBW);  // k-step groups per column block
  g.R2 = min(256, (kStageFloats - 16) / LP) & ~3;

  float *ring = sm;
  float *P = sm + kStages * kStageFloats;
  float *Z = P + kPartFloats;
  float *Tinv = Z + kZFloats;
  float *Ri = Tinv + 1024;
  double *G64 = reinterpret_cast<double *>(Ri + 1024);
  float *Yg = it.ws0;
  const float *A = it.A;
  const int64_t lda = it.lda;
  const bool vec = it.vec != 0;

  // Omega (n x l): Gaussian block (r, c/4) of the same Philox stream as the single-problem path
  for (int e = t; e < g.nz * LP; e += kThreads) Z[e] = 0.f;
  __syncthreads();
  {
    const int gl = (l + 3) >> 2;
    for (int e = t; e < g.n * gl; e += kThreads) {
      const int r = e / gl, cq = e - r * gl;
      const float4 z = rmc::gaussian4(it.seed, 0, (uint64_t)e);
      const float v[4] = {z.x, z.y, z.z, z.w};
#pragma unroll
      for (int c = 0; c < 4; ++c)
        if (4 * cq + c < l) Z[r * LP + 4 * cq + c] = v[c];
    }
  }
  __syncthreads();

  // Gram matrix of the rows streamed by the last pass -> G64 -> R, R^-1 (warp 0)
  auto finish_gram = [&](const float (&acc)[TN][4], float *Rout, float *Riout) {
    dump_acc<TN>(ring, TN, g.GY, acc);
    __syncthreads();
    gram_reduce64(ring, LP, g.GY, l, G64);
    __syncthreads();
    factor_small(G64, l, Rout, Riout, flag, status);
  };

  // W^T = A^T Yg: warp unit (16-column block w_mb of A, k-step group w_rs); w_finish sums the groups in order
  // and forms Z = (Tinv^T W)^T, dropping the rows c >= n (they hold the dense tile's neighbouring values)
  const int w_mb = warp % g.MBW, w_rs = warp / g.MBW;
  const bool w_active = warp < g.MBW * g.RS;
  auto w_finish = [&](const float (&acc)[TN / 2][4]) {
    if (w_active) {
      const int gq = lane >> 2, tq = lane & 3;
      float *d = ring + (size_t)w_rs * g.nz * LP + (w_mb * 16 + gq) * LP + 2 * tq;
#pragma unroll
      for (int nb = 0; nb < TN / 2; ++nb) {
        *reinterpret_cast<float2 *>(d + nb * 8) = make_float2(acc[nb][0], acc[nb][1]);
        *reinterpret_cast<float2 *>(d + 8 * LP + nb * 8) = make_float2(acc[nb][2], acc[nb][3]);
      }
    }
    __syncthreads();
    for (int e = t; e < g.nz * LP; e += kThreads) {
      float s = 0.f;
      for (int r = 0; r < g.RS; ++r) s += ring[(size_t)r * g.nz * LP + e];
      P[e] = s;
    }
    __syncthreads();
    for (int e = t; e < g.nz * LP; e += kThreads) {
      const int c = e / LP, i = e - c * LP;
      float s = 0.f;
      for (int j = 0; j <= i && j < l; ++j) s = fmaf(Tinv[j * 32 + i], P[c * LP + j], s);
      Z[e] = c < g.n ? s : 0.f;
    }
    __syncthreads();
  };

  // Y = A Z (written to Yg) with the Gram matrix of Y accumulated on the way.  With fuse_w (the intermediate
  // bases of the power iteration, where Q = Y R^-1 stays implicit anyway), W^T = A^T Y is accumulated from the
  // same A tiles and Z = (R^-T W)^T formed at the end, which saves the separate pass over A; Tinv = R^-1.
  auto y_pass = [&](float *Rout, float *Riout, bool fuse_w) {
    float gtot[TN][4];
    zero_acc<TN>(gtot);
    float wacc[TN / 2][4];
#pragma unroll
    for (int nb = 0; nb < TN / 2; ++nb) wacc[nb][0] = wacc[nb][1] = wacc[nb][2] = wacc[nb][3] = 0.f;
    stream_tiles(
        rg, g.m, g.R, status,
        [&](float *st, int r0, uint64_t *bar) {
          if (g.dense) {
            issue_spans(bar, span_tile(st, A, r0, g.R, g.m, g.n));
          } else {
            load_rows(st, g.S, A, lda, r0, g.R, g.m, g.n, g.nz, vec);
            issue_spans(bar, Span{nullptr, nullptr, 0u});
          }
        },
        [&](float *st, int r0) {
          tile_times_z<TN>(st, g.S, g.R, g.ksplit, g.kb_per, g.KB, Z, P);
          __syncthreads();
          reduce_slices(P, g.R * LP / 4, g.ksplit);
          __syncthreads();
          const int rv = min(g.R, g.m - r0);
          float4 *dst = reinterpret_cast<float4 *>(Yg + (size_t)r0 * LP);
          const float4 *src = reinterpret_cast<const float4 *>(P);
          for (int e = t; e < rv * LP / 4; e += kThreads) dst[e] = src[e];
          float gt[TN][4];
          zero_acc<TN>(gt);
          xt_accum<TN>(P, LP, P, LP, g.R, TN, g.GY, gt);
          add_acc<TN>(gtot, gt);
          if (fuse_w && w_active) at_times_y<TN>(st, g.S, P, g.R, w_mb, w_rs, g.RS, wacc);
        });
    finish_gram(gtot, Rout, Riout);
    if (fuse_w) {
      for (int e = t; e < 1024; e += kThreads) Tinv[e] = Riout[e];
      __syncthreads();
      w_finish(wacc);
    }
  };

  // Second CholeskyQR pass over Yg: Q1 = Y R1^-1 written back in place, Gram matrix of Q1 accumulated
  auto q_pass = [&](const float *R1i, float *Rout, float *Riout) {
    float gtot[TN][4];
    zero_acc<TN>(gtot);
    stream_tiles(
        rg, g.m, g.R2, status,
        [&](float *st, int r0, uint64_t *bar) { issue_spans(bar, span_tile(st, Yg, r0, g.R2, g.m, LP)); },
        [&](float *st, int r0) {
          const int rv = min(g.R2, g.m - r0);
          rows_times<TN, true>(st, rv, R1i);
          __syncthreads();
          float4 *dst = reinterpret_cast<float4 *>(Yg + (size_t)r0 * LP);
          const float4 *src = reinterpret_cast<const float4 *>(st);
          for (int e = t; e < rv * LP / 4; e += kThreads) dst[e] = src[e];
          float gt[TN][4];
          zero_acc<TN>(gt);
          xt_accum<TN>(st, LP, st, LP, g.R2, TN, g.GY, gt);
          add_acc<TN>(gtot, gt);
        });
    finish_gram(gtot, Rout, Riout);
  };

  // Z = (Yg Tinv)^T A transposed, i.e. Z[c][i] = sum_j Tinv[j][i] (A^T Yg)[c][j]  (n x l)
  auto w_pass = [&]() {
    float acc[TN / 2][4];
#pragma unroll
    for (int nb = 0; nb < TN / 2; ++nb) acc[nb][0] = acc[nb][1] = acc[nb][2] = acc[nb][3] = 0.f;
    stream_tiles(
        rg, g.m, g.R, status,
        [&](float *st, int r0, uint64_t *bar) {
          const Span y = span_tile(st + g.yoff, Yg, r0, g.R, g.m, LP);
          if (g.dense) {
            issue_spans(bar, span_tile(st, A, r0, g.R, g.m, g.n), y);
          } else {
            load_rows(st, g.S, A, lda, r0, g.R, g.m, g.n, g.nz, vec);
            issue_spans(bar, y);
          }
        },
        [&](float *st, int r0) {
          if (w_active) at_times_y<TN>(st, g.S, st + g.yoff, g.R, w_mb, w_rs, g.RS, acc);
        });
    w_finish(acc);
  };

  // one CholeskyQR pass on Z (nz x LP, in shared memory): Z <- Z R^-1, R kept in Rout
  auto z_cholqr = [&](float *Rout) {
    float acc[TN][4];
    zero_acc<TN>(acc);
    xt_accum<TN>(Z, LP, Z, LP, g.nz, TN, g.GY, acc);
    finish_gram(acc, Rout, Ri);
    rows_times<TN, true>(Z, g.nz, Ri);
    __syncthreads();
  };

  float *Rscr = P;  // R factors of the CholeskyQR passes that are not kept
  // ---- range finder and power iteration
  if (it.q == 0) {
    y_pass(Rscr, Ri, false);  // Y = A Omega; R1^-1 in Ri
    for (int e = t; e < 1024; e += kThreads) Tinv[e] = Ri[e];
    __syncthreads();
    q_pass(Tinv, Rscr, Ri);  // Q1 = Y R1^-1; R2^-1 in Ri
    for (int e = t; e < 1024; e += kThreads) Tinv[e] = Ri[e];
    __syncthreads();
  } else {
    y_pass(Rscr, Ri, true);  // Y = A Omega and Z = (Q^T A)^T in one pass
    for (int itn = 0; itn < it.q; ++itn) {
      const bool last = itn == it.q - 1;
      z_cholqr(Rscr);           // Z = orth(A^T Q)
      y_pass(Rscr, Ri, !last);  // Y = A Z (and the next Z, except for the last basis)
      if (last) {
        for (int e = t; e < 1024; e += kThreads) Tinv[e] = Ri[e];
        __syncthreads();
        q_pass(Tinv, Rscr, Ri);
        for (int e = t; e < 1024; e += kThreads) Tinv[e] = Ri[e];
        __syncthreads();
      }
    }
  }
  w_pass();  // Z = B^T = (Q^T A)^T, n x l

  // ---- small SVD: B^T = Q2 R by CholeskyQR2, R = W V^T by one-sided Jacobi
  float *Ra = P, *Rb = P + 1024, *W = P + 2048, *V = P + 3072, *Ub = P + 4096, *M = P + 5120;
  float *Ms = P + 6144;
  double *sg = reinterpret_cast<double *>(P + 7168);
  float *sgs = P + 7232;
  z_cholqr(Ra);
  z_cholqr(Rb);
  // W = R = Rb Ra, column j at W + 32 j
  for (int e = t; e < 1024; e += kThreads) {
    const int j = e >> 5, i = e & 31;
    float s = 0.f;
    if (i < l && j < l)
      for (int c = i; c <= j; ++c) s = fmaf(Rb[i * 32 + c], Ra[c * 32 + j], s);
    W[j * 32 + i] = s;
  }
  __syncthreads();
  jacobi_small(W, V, l, flag, status);
  for (int j = t; j < 32; j += kThreads) {
    double s = 0.0;
    for (int r = 0; r < l; ++r) s += (double)W[j * 32 + r] * (double)W[j * 32 + r];
    sg[j] = j < l ? sqrt(s) : 0.0;
  }
  for (int e = t; e < 1024; e += kThreads) Ub[e] = M[e] = 0.f;
  __syncthreads();
  // Ub[:, rank j] = V[:, j], M[:, rank j] = w_j / sigma_j, sigma descending (ties by index)
  for (int j = t; j < l; j += kThreads) {
    int rank = 0;
    for (int u = 0; u < l; ++u) rank += (sg[u] > sg[j]) || (sg[u] == sg[j] && u < j);
    sgs[rank] = (float)sg[j];
    const double inv = sg[j] > 0 ? 1.0 / sg[j] : 0.0;
    for (int r = 0; r < l; ++r) {
      Ub[r * 32 + rank] = V[j * 32 + r];
      M[r * 32 + rank] = (float)((double)W[j * 32 + r] * inv);
    }
  }
  __syncthreads();
  rows_times<TN, false>(Z, g.nz, M);  // Vb = Q2 M
  __syncthreads();
  // signs: the entry of largest magnitude of Vb[:, i] (first on ties) is made positive
  for (int e = t; e < 1024; e += kThreads) Ms[e] = 0.f;
  __syncthreads();
  for (int i = warp; i < k; i += kWarps) {
    float best = -1.f;
    int where = 0;
    for (int r = lane; r < g.n; r += 32) {
      const float v = fabsf(Z[r * LP + i]);
      if (v > best) { best = v; where = r; }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      const float b2 = __shfl_xor_sync(0xffffffffu, best, o);
      const int w2 = __shfl_xor_sync(0xffffffffu, where, o);
      if (b2 > best || (b2 == best && w2 < where)) { best = b2; where = w2; }
    }
    const float sgn = Z[where * LP + i] < 0.f ? -1.f : 1.f;
    for (int r = lane; r < g.n; r += 32) it.V[(int64_t)r * k + i] = sgn * Z[r * LP + i];
    if (lane < l) Ms[lane * 32 + i] = sgn * Ub[lane * 32 + i];
    if (lane == 0) it.sigma[i] = sgs[i];
  }
  __syncthreads();
  // U = Q1 Tinv Ms: fold Tinv Ms (l x k) into Ri, then one pass over Q1
  for (int e = t; e < 1024; e += kThreads) {
    const int r = e >> 5, c = e & 31;
    float s = 0.f;
    if (r < l && c < k)
      for (int i = r; i < l; ++i) s = fmaf(Tinv[r * 32 + i], Ms[i * 32 + c], s);
    Ri[e] = s;
  }
  __syncthreads();
  stream_tiles(
      rg, g.m, g.R2, status,
      [&](float *st, int r0, uint64_t *bar) { issue_spans(bar, span_tile(st, Yg, r0, g.R2, g.m, LP)); },
      [&](float *st, int r0) {
        const int rv = min(g.R2, g.m - r0);
        for (int e = t; e < rv * k; e += kThreads) {
          const int r = e / k, c = e - r * k;
          float s = 0.f;
#pragma unroll
          for (int i = 0; i < LP; ++i) s = fmaf(st[r * LP + i], Ri[i * 32 + c], s);
          it.U[(int64_t)(r0 + r) * k + c] = s;
        }
      });
}

// -------------------------------------------------------------------------------------- lsr problem

// Packed upper triangle of an nn x nn matrix: row i holds columns i .. nn-1.
__device__ __forceinline__ int poff(int i, int nn) { return i * nn - (i * (i - 1)) / 2; }

// Block exclusive scan of one int per thread; returns the prefix, total in *total.
__device__ __forceinline__ int block_scan(int v, int *wsum, int *total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int w = lane < kWarps ? wsum[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < kWarps) wsum[lane] = w;
  }
  __syncthreads();
  const int before = (warp ? wsum[warp - 1] : 0) + x - v;
  if (total) *total = wsum[kWarps - 1];
  __syncthreads();
  return before;
}

// Triangular solves with the packed factor (row stride nn = n + 1) by one warp; index c lives in lane c % 32,
// slot c / 32.  forward: R^T y = rhs; backward: R x = rhs.  Result to out (shared memory).
template <bool forward>
__device__ void packed_solve(const float *Pk, int n, int nn, const float *rhs, float *out) {
  const int lane = threadIdx.x & 31;
  float rr[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    const int c = lane + 32 * u;
    rr[u] = c < n ? rhs[c] : 0.f;
  }
  if (forward) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      if (32 * u >= n) break;
      for (int ii = 0; ii < 32; ++ii) {
        const int i = 32 * u + ii;
        if (i >= n) break;
        const int oi = poff(i, nn);
        const float yi = __shfl_sync(0xffffffffu, rr[u], ii) / Pk[oi];
        if (lane == ii) out[i] = yi;
#pragma unroll
        for (int u2 = u; u2 < 8; ++u2) {
          const int c = lane + 32 * u2;
          if (c > i && c < n) rr[u2] = fmaf(-Pk[oi + c - i], yi, rr[u2]);
        }
      }
    }
  } else {
#pragma unroll
    for (int u = 7; u >= 0; --u) {
      if (32 * u >= n) continue;
      for (int ii = 31; ii >= 0; --ii) {
        const int i = 32 * u + ii;
        if (i >= n) continue;
        const float xi = __shfl_sync(0xffffffffu, rr[u], ii) / Pk[poff(i, nn)];
        if (lane == ii) out[i] = xi;
#pragma unroll
        for (int u2 = 0; u2 <= u; ++u2) {
          const int c = lane + 32 * u2;
          if (c < i) rr[u2] = fmaf(-Pk[poff(c, nn) + i - c], xi, rr[u2]);
        }
      }
    }
  }
  __syncwarp();
}

__device__ void lsr_problem(const BatchItem &it, float *sm, Ring &rg, int *wsum, int *status) {
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int m = it.m, n = it.n, s = it.s, n1 = n + 1, n8 = (n1 + 7) & ~7;
  const float *A = it.A, *bv = it.b;
  const int64_t lda = it.lda;
  float *SAb = it.ws0;
  uint32_t *keys = it.ws1, *perm = it.ws1 + m;

  // ---- 1. hash every row; per-warp bucket histograms (warp w takes rows [w chunk, (w+1) chunk))
  int *hs = reinterpret_cast<int *>(sm);  // hs[b * 16 + w]
  int *bstart = hs + kWarps * kMaxS;
  for (int e = t; e < kWarps * s; e += kThreads) hs[e] = 0;
  __syncthreads();
  const int chunk = (m + kWarps - 1) / kWarps;
  const int lo = min(m, warp * chunk), hi = min(m, lo + chunk);
  for (int i = lo + lane; i < hi; i += 32) {
    uint32_t b;
    float sg;
    rmc::cs_hash(it.seed, 0, (uint64_t)i, (uint32_t)s, &b, &sg);
    keys[i] = b | (sg < 0.f ? 0x80000000u : 0u);
    atomicAdd(&hs[b * kWarps + warp], 1);
  }
  __syncthreads();
  // ---- 2. exclusive scan in (bucket, warp) order: the start of each warp's run inside each bucket
  {
    const int tot = kWarps * s, per = (tot + kThreads - 1) / kThreads;
    const int a = min(tot, t * per), z = min(tot, a + per);
    int sum = 0;
    for (int e = a; e < z; ++e) sum += hs[e];
    int run = block_scan(sum, wsum, nullptr);
    for (int e = a; e < z; ++e) {
      const int v = hs[e];
      hs[e] = run;
      run += v;
    }
  }
  __syncthreads();
  for (int b = t; b < s; b += kThreads) bstart[b] = hs[b * kWarps];
  if (t == 0) bstart[s] = m;
  __syncthreads();
  // ---- 3. stable placement: rows of a bucket in increasing order
  for (int base = lo; base < hi; base += 32) {
    const int i = base + lane;
    const bool v = i < hi;
    const uint32_t key = v ? keys[i] : 0xFFFFFFFFu;
    const uint32_t b = key & 0x7FFFFFFFu;
    const unsigned peers = __match_any_sync(0xffffffffu, b);
    const int rank = __popc(peers & ((1u << lane) - 1u));
    if (v) perm[hs[b * kWarps + warp] + rank] = (uint32_t)i | (key & 0x80000000u);
    __syncwarp();
    if (v && rank == 0) hs[b * kWarps + warp] += __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  // ---- 4. gather: row b of [S^T A, S^T b] = signed sum of the rows hashed to bucket b (one warp per bucket)
  for (int b = warp; b < s; b += kWarps) {
    const int p0 = bstart[b], p1 = bstart[b + 1];
    float acc[9];
#pragma unroll
    for (int u = 0; u < 9; ++u) acc[u] = 0.f;
    for (int p = p0; p < p1; p += 8) {  // eight rows in flight per warp
      float va[8][9];
      float sgn[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const bool ok = p + j < p1;
        const uint32_t e = ok ? perm[p + j] : 0u;
        const int row = (int)(e & 0x7FFFFFFFu);
        sgn[j] = ok ? ((e >> 31) ? -1.f : 1.f) : 0.f;
        const float *ar = A + (int64_t)row * lda;
#pragma unroll
        for (int u = 0; u < 9; ++u) {
          const int c = lane + 32 * u;
          va[j][u] = !ok ? 0.f : c < n ? __ldg(ar + c) : c == n ? __ldg(bv + row) : 0.f;
        }
      }
#pragma unroll
      for (int j = 0; j < 8; ++j)
#pragma unroll
        for (int u = 0; u < 9; ++u) acc[u] = fmaf(sgn[j], va[j][u], acc[u]);
    }
    float *d = SAb + (size_t)b * n8;
#pragma unroll
    for (int u = 0; u < 9; ++u) {
      const int c = lane + 32 * u;
      if (c < n8) d[c] = c < n1 ? acc[u] : 0.f;
    }
  }
  __syncthreads();
  // ---- 5. augmented Gram matrix [SA, Sb]^T [SA, Sb] in 8 x 8 blocks (FP32), block partials to ws2
  const int nbk = n8 >> 3, blocks = nbk * (nbk + 1) / 2;
  const int splits = max(1, kThreads / blocks), items = blocks * splits;
  const int CR = min((kStageFloats - 16) / n8, (s + 3) & ~3) & ~3;  // rows per staged tile, >= 4
  for (int round = 0; round * kThreads < items; ++round) {
    const int item = round * kThreads + t;
    const bool active = item < items;
    const int sp = active ? item / blocks : 0, blk = active ? item - (item / blocks) * blocks : 0;
    int bi = 0, rem = blk;
    while (rem >= nbk - bi) { rem -= nbk - bi; ++bi; }
    const int bj = bi + rem;
    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
    stream_tiles(
        rg, s, CR, status,
        [&](float *st, int r0, uint64_t *bar) { issue_spans(bar, span_tile(st, SAb, r0, CR, s, n8)); },
        [&](float *st, int r0) {
          if (!active) return;
          const int rv = min(CR, s - r0);
          for (int r = (sp - r0 % splits + splits) % splits; r < rv; r += splits) {
            const float *row = st + r * n8;
            const float4 x0 = *reinterpret_cast<const float4 *>(row + 8 * bi);
            const float4 x1 = *reinterpret_cast<const float4 *>(row + 8 * bi + 4);
            const float4 y0 = *reinterpret_cast<const float4 *>(row + 8 * bj);
            const float4 y1 = *reinterpret_cast<const float4 *>(row + 8 * bj + 4);
            const float xv[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
            const float yv[8] = {y0.x, y0.y, y0.z, y0.w, y1.x, y1.y, y1.z, y1.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
              for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(xv[i], yv[j], acc[i][j]);
          }
        });
    if (active) {
      float4 *d = reinterpret_cast<float4 *>(it.ws2 + (size_t)item * 64);
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        d[2 * i] = make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
        d[2 * i + 1] = make_float4(acc[i][4], acc[i][5], acc[i][6], acc[i][7]);
      }
    }
  }
  __syncthreads();
  float *Pk = sm;  // packed upper triangle of the (n+1) x (n+1) augmented Gram matrix
  for (int i = warp; i < n1; i += kWarps) {
    const int bi = i >> 3, o = poff(i, n1);
    for (int j = i + lane; j < n1; j += 32) {
      const int bj = j >> 3;
      const int blk = bi * nbk - (bi * (bi - 1)) / 2 + (bj - bi);
      float v = 0.f;
      for (int sp = 0; sp < splits; ++sp) v += it.ws2[((size_t)sp * blocks + blk) * 64 + (i & 7) * 8 + (j & 7)];
      Pk[o + j - i] = v;
    }
  }
  __syncthreads();
  // ---- 6. right-looking Cholesky of the leading n x n block; the augmented column becomes R^-T S^T A^T S b
  float *vecs = sm + ((poff(n1, n1) + 63) & ~31);
  float *y = vecs, *xf = vecs + 288, *rres = vecs + 576, *gp = rres + kMaxS;
  double *x64 = reinterpret_cast<double *>(gp + 2 * 288);
  float *gsum = reinterpret_cast<float *>(x64 + 288);  // up to 64 row groups x 264 columns of SA^T r partials
  bool ok = true;
  float dprev = 0.f;
  for (int kk = 0; kk < n; ++kk) {
    const float d = Pk[poff(kk, n1)];
    if (!(d > 0.f) || !(d < INFINITY)) { ok = false; break; }
    if (kk > 0) {
      const int o = poff(kk - 1, n1);
      const float rd = sqrtf(dprev), inv = 1.f / rd;
      for (int c = kk - 1 + t; c <= n; c += kThreads) Pk[o + c - (kk - 1)] = (c == kk - 1) ? rd : Pk[o + c - (kk - 1)] * inv;
    }
    const float invd = 1.f / d;
    const int ok_ = poff(kk, n1);
    for (int i = kk + 1 + warp; i < n; i += kWarps) {
      const float f = Pk[ok_ + i - kk] * invd;
      const int oi = poff(i, n1);
      for (int c = i + lane; c <= n; c += 32) Pk[oi + c - i] = fmaf(-f, Pk[ok_ + c - kk], Pk[oi + c - i]);
    }
    dprev = d;
    __syncthreads();
  }
  if (ok) {
    const int o = poff(n - 1, n1);
    const float rd = sqrtf(dprev), inv = 1.f / rd;
    for (int c = n - 1 + t; c <= n; c += kThreads) Pk[o + c - (n - 1)] = (c == n - 1) ? rd : Pk[o + c - (n - 1)] * inv;
  }
  __syncthreads();
  if (!ok) {
    for (int c = t; c < n; c += kThreads) it.x[c] = nan("");
    if (t == 0) rmc_report(status, RMC_ENUMERIC);
    return;
  }
  // ---- 7. x0 = R^-1 (augmented column), then two refinement steps against [SA, Sb]:
  //         r = Sb - SA x, dx = (R^T R)^-1 SA^T r
  for (int i = t; i < n; i += kThreads) y[i] = Pk[poff(i, n1) + n - i];
  __syncthreads();
  if (warp == 0) packed_solve<false>(Pk, n, n1, y, xf);
  __syncthreads();
  for (int i = t; i < n; i += kThreads) x64[i] = xf[i];
  __syncthreads();
  for (int iter = 0; iter < 2; ++iter) {
    for (int i = warp; i < s; i += kWarps) {
      const float *row = SAb + (size_t)i * n8;
      float acc = 0.f;
      for (int c = lane; c < n; c += 32) acc = fmaf(row[c], xf[c], acc);
#pragma unroll
      for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) rres[i] = row[n] - acc;
    }
    __syncthreads();
    {
      // g = SA^T r: thread (column c, row group h) sums rows h, h + H, ... with eight loads in flight
      const int H = kThreads / n8, c = t % n8, h = t / n8;
      if (h < H && c < n) {
        float acc = 0.f;
#pragma unroll 8
        for (int i = h; i < s; i += H) acc = fmaf(SAb[(size_t)i * n8 + c], rres[i], acc);
        gsum[h * 264 + c] = acc;
      }
    }
    __syncthreads();
    {
      const int H = kThreads / n8;
      for (int c = t; c < n; c += kThreads) {
        float g = 0.f;
        for (int h = 0; h < H; ++h) g += gsum[h * 264 + c];
        rres[c] = g;  // reuse: SA^T r
      }
    }
    __syncthreads();
    if (warp == 0) {
      packed_solve<true>(Pk, n, n1, rres, y);
      packed_solve<false>(Pk, n, n1, y, gp);
    }
    __syncthreads();
    for (int c = t; c < n; c += kThreads) {
      x64[c] += (double)gp[c];
      xf[c] = (float)x64[c];
    }
    __syncthreads();
  }
  for (int c = t; c < n; c += kThreads) it.x[c] = x64[c];
}

// ------------------------------------------------------------------------------------------- kernel

__global__ void __launch_bounds__(kThreads, 1)
    batch_kernel(const BatchItem *__restrict__ items, const int *__restrict__ order, int nitems, int *next,
                 int *status) {
  extern __shared__ __align__(16) float sm[];
  __shared__ int s_item, s_flag;
  __shared__ int s_wsum[kWarps];
  __shared__ __align__(8) uint64_t s_full[kStages];
  if (threadIdx.x == 0) {
    for (int st = 0; st < kStages; ++st) tc::mbar_init(&s_full[st], 1);
    tc::fence_barrier_init();
  }
  __syncthreads();
  Ring rg{sm, s_full, 0u};  // the ring's stages start at the front of shared memory, for every problem
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(next, 1);
    __syncthreads();
    const int w = s_item;
    __syncthreads();
    if (w >= nitems) break;
    const BatchItem it = items[order[w]];
    if (it.kind == RMC_REQ_LSR) {
      lsr_problem(it, sm, rg, s_wsum, status);
    } else {
      const int l = it.k + it.p;
      if (l <= 8) rsvd_problem<2>(it, sm, rg, &s_flag, status);
      else if (l <= 16) rsvd_problem<4>(it, sm, rg, &s_flag, status);
      else if (l <= 24) rsvd_problem<6>(it, sm, rg, &s_flag, status);
      else rsvd_problem<8>(it, sm, rg, &s_flag, status);
    }
    __syncthreads();
  }
}

static int lp_of(int l) { return (l + 7) & ~7; }

// Rough per-problem cost in microseconds of one SM: streamed bytes at ~40 GB/s or FP32 FMAs at ~60% of one
// SM's rate, plus the fixed tail (small factorizations).  Only the ORDER matters (largest first).
static double cost_us(const rmc_request &r) {
  const double m = (double)r.m, n = (double)r.n;
  if (r.kind == RMC_REQ_LSR) {
    const double bytes = m * (n + 1) * 4 + 16 * m;
    const double fma = (double)r.s * (n + 8) * (n + 8) / 2 + 4 * (double)r.s * n + n * n * n / 6;
    return std::max(bytes / 4.0e4, fma / 1.5e5) + 0.2 * n;
  }
  const int lp = lp_of(r.k + r.p);
  const double passes = 2.0 + 2.0 * r.q;
  const double bytes = passes * m * n * 4 + (3.0 + r.q) * m * lp * 8;
  const double fma = passes * m * n * lp + (2.0 + r.q) * m * lp * lp;
  return std::max(bytes / 4.0e4, fma / 1.5e5) + 40.0;
}

// Tuning class of a k-SVD problem: n class (n in 1-64, 65-128, 129-192, 193-256) x l class (l rounded up to
// 8, 16, 24 or 32: the kernel's column tile).
static int tile_class(const rmc_request &r) {
  const int nc = (int)std::min<int64_t>(3, (r.n - 1) / 64);
  const int lc = std::min(3, lp_of(r.k + r.p) / 8 - 1);
  return nc * 4 + lc;
}

static bool bad_request(const rmc_request &r) {
  if (!r.A || r.m < 1 || r.m > kMaxM || r.n < 1 || r.n > kMaxN || r.lda < r.n) return true;
  if (r.kind == RMC_REQ_LSR) return !r.b || !r.x || r.s < r.n || r.s > kMaxS;
  if (r.kind == RMC_REQ_RSVD) {
    const int64_t l = int64_t(r.k) + r.p;
    return !r.U || !r.sigma || !r.V || r.k < 1 || r.p < 0 || r.q < 0 || r.q > 64 || l > kMaxL || l > r.n || l > r.m;
  }
  return true;
}

// Workspace of a batch: descriptors, order, queue counter, then each problem's buffers.
static void batch_carve(WsCarve &w, const rmc_request *reqs, int nreq, BatchItem *host, BatchItem **d_items,
                        int **d_order, int **d_next) {
  *d_items = w.take<BatchItem>(nreq);
  *d_order = w.take<int>(nreq);
  *d_next = w.take<int>(1);
  for (int i = 0; i < nreq; ++i) {
    const rmc_request &r = reqs[i];
    BatchItem &b = host[i];
    b.ws0 = nullptr;
    b.ws1 = nullptr;
    b.ws2 = nullptr;
    if (r.kind == RMC_REQ_RSVD) {
      b.ws0 = w.take<float>(size_t(r.m) * lp_of(r.k + r.p));
    } else {
      const int n8 = (int(r.n) + 8) & ~7;
      const int nbk = n8 / 8, blocks = nbk * (nbk + 1) / 2;
      const int items = blocks * std::max(1, kThreads / blocks);
      b.ws0 = w.take<float>(size_t(r.s) * n8);
      b.ws1 = w.take<uint32_t>(2 * size_t(r.m));
      b.ws2 = w.take<float>(size_t(items) * 64);
    }
  }
}

}  // namespace

bool rmc_batch_request_ok(const rmc_request &r) { return !bad_request(r); }

size_t rmc_batch_plan_bytes(const rmc_request *reqs, int nreq) {
  std::vector<BatchItem> host(nreq);
  BatchItem *d_items;
  int *d_order, *d_next;
  WsCarve plan;
  batch_carve(plan, reqs, nreq, host.data(), &d_items, &d_order, &d_next);
  return plan.off;
}

extern "C" int rmc_batch_run(rmc_ctx *ctx, const rmc_request *reqs, int nreq) {
  if (!ctx || nreq < 0 || (nreq > 0 && !reqs)) return RMC_EINVAL;
  if (nreq == 0) return RMC_OK;
  for (int i = 0; i < nreq; ++i)
    if (bad_request(reqs[i])) return RMC_EINVAL;

  std::vector<int> order(nreq);
  std::vector<double> cost(nreq);
  for (int i = 0; i < nreq; ++i) {
    order[i] = i;
    cost[i] = cost_us(reqs[i]);
  }
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });

  std::vector<BatchItem> host(nreq);
  BatchItem *d_items = nullptr;
  int *d_order = nullptr, *d_next = nullptr;
  auto carve = [&](WsCarve &w) { batch_carve(w, reqs, nreq, host.data(), &d_items, &d_order, &d_next); };
  WsCarve plan;
  carve(plan);
  RMC_TRY(rmc_ws_reserve(ctx, plan.off));
  WsCarve w;
  w.base = static_cast<char *>(ctx->ws);
  carve(w);
  for (int i = 0; i < nreq; ++i) {
    const rmc_request &r = reqs[i];
    BatchItem &b = host[i];
    b.kind = r.kind;
    b.k = r.k;
    b.p = r.p;
    b.q = r.q;
    b.m = (int)r.m;
    b.n = (int)r.n;
    b.s = (int)r.s;
    b.vec = ((reinterpret_cast<uintptr_t>(r.A) & 15) == 0 && (r.lda & 3) == 0) ? 1 : 0;
    b.rtile = (r.kind == RMC_REQ_RSVD) ? ctx->batch_rtile[tile_class(r)] : 0;
    b.lda = r.lda;
    b.seed = r.seed;
    b.A = r.A;
    b.b = r.b;
    b.x = r.x;
    b.U = r.U;
    b.sigma = r.sigma;
    b.V = r.V;
  }
  cudaStream_t st = ctx->stream;
  // descriptors go through the context's pinned staging buffer (an asynchronous copy that never waits on the
  // device, unlike one from pageable memory); the buffer is reused once the previous copy out of it is done
  const size_t items_bytes = sizeof(BatchItem) * nreq, stage_bytes = items_bytes + sizeof(int) * nreq;
  if (!ctx->stage_ev) RMC_TRY_CUDA(cudaEventCreateWithFlags(&ctx->stage_ev, cudaEventDisableTiming));
  else RMC_TRY_CUDA(cudaEventSynchronize(ctx->stage_ev));
  if (ctx->h_stage_bytes < stage_bytes) {
    if (ctx->h_stage) RMC_TRY_CUDA(cudaFreeHost(ctx->h_stage));
    ctx->h_stage = nullptr;
    ctx->h_stage_bytes = 0;
    RMC_TRY_CUDA(cudaMallocHost(&ctx->h_stage, stage_bytes + stage_bytes / 2));
    ctx->h_stage_bytes = stage_bytes + stage_bytes / 2;
  }
  char *stage = static_cast<char *>(ctx->h_stage);
  memcpy(stage, host.data(), items_bytes);
  memcpy(stage + items_bytes, order.data(), sizeof(int) * nreq);
  RMC_TRY_CUDA(cudaMemcpyAsync(d_items, stage, items_bytes, cudaMemcpyHostToDevice, st));
  RMC_TRY_CUDA(cudaMemcpyAsync(d_order, stage + items_bytes, sizeof(int) * nreq, cudaMemcpyHostToDevice, st));
  RMC_TRY_CUDA(cudaEventRecord(ctx->stage_ev, st));
  RMC_TRY_CUDA(cudaMemsetAsync(d_next, 0, sizeof(int), st));
  RMC_TRY_CUDA(rmc_allow_smem(batch_kernel, kSmemBytes));
  const int grid = std::min(nreq, ctx->num_sms);
  {
    RmcProf prof(ctx, RMC_K_BATCH);
    batch_kernel<<<grid, kThreads, kSmemBytes, st>>>(d_items, d_order, nreq, d_next, ctx->d_status);
  }
  rmc_note_launch();
  RMC_LAUNCH_CHECK();
  return RMC_OK;
}

// ------------------------------------------------------------------------------------------- autotuner
// The row-tile height of the k-SVD passes trades barrier count (tall tiles) against parallel k-splits and
// load balance inside a tile (short tiles); the best height depends on n and l.  The tuner times each
// candidate on the caller's own problems, class by class, and keeps the fastest in the context's table.

extern "C" int rmc_batch_autotune(rmc_ctx *ctx, const rmc_request *reqs, int nreq, int reps) {
  if (!ctx || nreq < 0 || (nreq > 0 && !reqs) || reps < 1 || reps > 100) return RMC_EINVAL;
  for (int i = 0; i < nreq; ++i)
    if (bad_request(reqs[i])) return RMC_EINVAL;
  constexpr int kCand[] = {0, 32, 64, 128};   // 0: as many rows as a stage holds
  constexpr int kSample = 256;                // problems per class that are timed
  std::vector<std::vector<rmc_request>> byclass(kBatchTileClasses);
  for (int i = 0; i < nreq; ++i)
    if (reqs[i].kind == RMC_REQ_RSVD && (int)byclass[tile_class(reqs[i])].size() < kSample)
      byclass[tile_class(reqs[i])].push_back(reqs[i]);
  cudaEvent_t e0, e1;
  RMC_TRY_CUDA(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    (void)cudaGetLastError();
    return RMC_ECUDA;
  }
  int rc = RMC_OK;
  for (int c = 0; c < kBatchTileClasses && rc == RMC_OK; ++c) {
    if (byclass[c].empty()) continue;
    float best = 0.f;
    int best_tile = 0;
    bool have = false;
    for (int cand : kCand) {
      ctx->batch_rtile[c] = cand;
      rc = rmc_batch_run(ctx, byclass[c].data(), (int)byclass[c].size());     // warm-up (and workspace)
      if (rc != RMC_OK) break;
      if (cudaEventRecord(e0, ctx->stream) != cudaSuccess) { rc = RMC_ECUDA; break; }
      for (int r = 0; r < reps && rc == RMC_OK; ++r) rc = rmc_batch_run(ctx, byclass[c].data(), (int)byclass[c].size());
      if (rc != RMC_OK) break;
      float ms = 0.f;
      if (cudaEventRecord(e1, ctx->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
          cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
        rc = RMC_ECUDA;
        break;
      }
      if (!have || ms < best) {
        have = true;
        best = ms;
        best_tile = cand;
      }
    }
    ctx->batch_rtile[c] = best_tile;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  (void)cudaGetLastError();
  if (rc == RMC_OK) rc = rmc_sync(ctx);
  return rc;
}

extern "C" int rmc_batch_get_tiles(const rmc_ctx *ctx, int *table, int count) {
  if (!ctx || !table || count < kBatchTileClasses) return RMC_EINVAL;
  for (int c = 0; c < kBatchTileClasses; ++c) table[c] = ctx->batch_rtile[c];
  return RMC_OK;
}

extern "C" int rmc_batch_set_tiles(rmc_ctx *ctx, const int *table, int count) {
  if (!ctx || !table || count < kBatchTileClasses) return RMC_EINVAL;
  for (int c = 0; c < kBatchTileClasses; ++c)
    if (table[c] < 0 || table[c] > 256 || (table[c] % 16) != 0) return RMC_EINVAL;
  for (int c = 0; c < kBatchTileClasses; ++c) ctx->batch_rtile[c] = table[c];
  return RMC_OK;
}
