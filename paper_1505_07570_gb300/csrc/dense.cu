// Dense building blocks of the randomized SVD and of the least-squares solve:
//  - the FP32 (CUDA-core) products with A: Y = A X and W = X^T A (split-K over the rows of A),
//  - CholeskyQR2 (Gram matrix accumulated in FP64 from exact FP32 products, FP64 Cholesky, triangular apply),
//  - the small SVD by one-sided Jacobi on the l x l triangular factor,
//  - the FP64 solve of the sketched least-squares problem.
#include <algorithm>
#include <cmath>

#include "rmc_internal.cuh"

namespace {

// ------------------------------------------------------------------------------------ FP32 SIMT GEMMs
constexpr int GT = 64;   // output tile edge
constexpr int GK = 16;   // reduction step

// Y (m x l) = A (m x n) X (n x l).  256 threads, 4 x 4 outputs each.
__global__ void __launch_bounds__(256) matmul_an_kernel(const float *__restrict__ A, int64_t m, int64_t n,
                                                        int64_t lda, const float *__restrict__ X, int64_t l,
                                                        int64_t ldx, float *__restrict__ Y, int64_t ldy) {
  __shared__ float As[GK][GT + 4];
  __shared__ float Xs[GK][GT + 4];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t row0 = (int64_t)blockIdx.y * GT, col0 = (int64_t)blockIdx.x * GT;
  float acc[4][4] = {};
  for (int64_t k0 = 0; k0 < n; k0 += GK) {
    for (int e = tid; e < GT * GK; e += 256) {
      const int r = e / GK, kk = e % GK;                 // A tile: 64 rows x 16 k
      const int64_t gr = row0 + r, gk = k0 + kk;
      As[kk][r] = (gr < m && gk < n) ? A[gr * lda + gk] : 0.f;
      const int kx = e / GT, c = e % GT;                 // X tile: 16 k x 64 cols
      const int64_t gkx = k0 + kx, gc = col0 + c;
      Xs[kx][c] = (gkx < n && gc < l) ? X[gkx * ldx + gc] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GK; ++kk) {
      float a[4], x[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) x[j] = Xs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], x[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t r = row0 + ty + 16 * i, c = col0 + tx + 16 * j;
      if (r < m && c < l) Y[r * ldy + c] = acc[i][j];
    }
}

// Partial W_split (l x n) = X[rows of split]^T A[rows of split]; X is m x l.
__global__ void __launch_bounds__(256) matmul_at_kernel(const float *__restrict__ A, int64_t m, int64_t n,
                                                        int64_t lda, const float *__restrict__ X, int64_t l,
                                                        int64_t ldx, int64_t rows_per_split,
                                                        float *__restrict__ out, int64_t ldo,
                                                        int64_t split_stride) {
  __shared__ float Xs[GK][GT + 4];
  __shared__ float As[GK][GT + 4];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t lrow0 = (int64_t)blockIdx.y * GT, col0 = (int64_t)blockIdx.x * GT;
  const int64_t r_begin = (int64_t)blockIdx.z * rows_per_split;
  const int64_t r_end = min(m, r_begin + rows_per_split);
  float acc[4][4] = {};
  for (int64_t k0 = r_begin; k0 < r_end; k0 += GK) {
    for (int e = tid; e < GT * GK; e += 256) {
      const int kk = e / GT, c = e % GT;
      const int64_t gk = k0 + kk;
      const bool ok = gk < r_end;
      Xs[kk][c] = (ok && lrow0 + c < l) ? X[gk * ldx + lrow0 + c] : 0.f;
      As[kk][c] = (ok && col0 + c < n) ? A[gk * lda + col0 + c] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GK; ++kk) {
      float x[4], a[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) x[i] = Xs[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) a[j] = As[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(x[i], a[j], acc[i][j]);
    }
    __syncthreads();
  }
  float *o = out + (int64_t)blockIdx.z * split_stride;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t r = lrow0 + ty + 16 * i, c = col0 + tx + 16 * j;
      if (r < l && c < n) o[r * ldo + c] = acc[i][j];
    }
}

// W = sum over splits of the partials, in split order (deterministic).
__global__ void sum_splits_kernel(const float *__restrict__ part, int splits, int64_t rows, int64_t cols,
                                  float *__restrict__ W, int64_t ldw) {
  const int64_t total = rows * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int t = 0; t < splits; ++t) s += part[t * total + e];
    W[(e / cols) * ldw + e % cols] = s;
  }
}

// ------------------------------------------------------------------------------------- FP64 Gram matrix
constexpr int GRAM_T = 32;

// Partial Gram of one chunk of rows for one 32 x 32 tile pair (ti <= tj): products of FP32 values are exact in
// FP64, and the sums are FP64.
__global__ void __launch_bounds__(256) gram_f64_kernel(const float *__restrict__ Y, int64_t m, int l, int64_t ldy,
                                                       int64_t rows_per_chunk, double *__restrict__ part,
                                                       const int *gate) {
  if (gate && !*gate) return;  // a fallback that is not needed
  __shared__ double As[GRAM_T][GRAM_T + 1];
  __shared__ double Bs[GRAM_T][GRAM_T + 1];
  // decode the tile pair
  int p = blockIdx.x, ti = 0;
  const int T = (l + GRAM_T - 1) / GRAM_T;
  while (p >= T - ti) { p -= T - ti; ++ti; }
  const int tj = ti + p;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t r_begin = (int64_t)blockIdx.y * rows_per_chunk;
  const int64_t r_end = min(m, r_begin + rows_per_chunk);
  double acc00 = 0, acc01 = 0, acc10 = 0, acc11 = 0;
  for (int64_t r0 = r_begin; r0 < r_end; r0 += GRAM_T) {
    for (int e = tid; e < GRAM_T * GRAM_T; e += 256) {
      const int rr = e / GRAM_T, cc = e % GRAM_T;
      const int64_t r = r0 + rr;
      const int ca = ti * GRAM_T + cc, cb = tj * GRAM_T + cc;
      As[rr][cc] = (r < r_end && ca < l) ? (double)Y[r * ldy + ca] : 0.0;
      Bs[rr][cc] = (r < r_end && cb < l) ? (double)Y[r * ldy + cb] : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int rr = 0; rr < GRAM_T; ++rr) {
      const double a0 = As[rr][ty], a1 = As[rr][ty + 16], b0 = Bs[rr][tx], b1 = Bs[rr][tx + 16];
      acc00 = fma(a0, b0, acc00);
      acc01 = fma(a0, b1, acc01);
      acc10 = fma(a1, b0, acc10);
      acc11 = fma(a1, b1, acc11);
    }
    __syncthreads();
  }
  double *o = part + (int64_t)blockIdx.y * l * l;
  const int i0 = ti * GRAM_T + ty, i1 = i0 + 16, j0 = tj * GRAM_T + tx, j1 = j0 + 16;
  if (i0 < l && j0 < l) o[i0 * l + j0] = acc00;
  if (i0 < l && j1 < l) o[i0 * l + j1] = acc01;
  if (i1 < l && j0 < l) o[i1 * l + j0] = acc10;
  if (i1 < l && j1 < l) o[i1 * l + j1] = acc11;
}

// a + b as hi + lo exactly (TwoSum): the running double-FP32 sums of the Gram kernel below.
__device__ __forceinline__ void two_sum_acc(float &hi, float &lo, float x) {
  const float s = hi + x, bb = s - hi;
  lo += (hi - (s - bb)) + (x - bb);
  hi = s;
}

// Partial Gram matrix of one chunk of rows for one TILE x TILE tile pair (ti <= tj): 256 threads as 16 x 16, each
// owning an R x R block (R = TILE / 16) of adjacent rows and columns; 32-row slices of both column tiles are
// staged in shared memory while the next slice is loaded into registers.  Sums are double-FP32 (hi + lo), so the
// FP64 pipe (a small fraction of the FP32 rate on this GPU) is not used:
//   EXACT = false: FP32 products summed in FP32 over a slice, slices summed in double-FP32;
//   EXACT = true:  every product split exactly as p + e (e = fma(a, b, -p)), both summed in double-FP32 — exact
//                  products with ~48-bit sums, the FP32-data equivalent of FP64 products.
template <int TILE, bool EXACT>
__global__ void __launch_bounds__(256) gram_tile_kernel(const float *__restrict__ Y, int64_t m, int l, int64_t ldy,
                                                        int64_t rows_per_chunk, double *__restrict__ part) {
  constexpr int R = TILE / 16, SLICE = 32, LD = SLICE * TILE * 2 / 256;
  __shared__ __align__(16) float As[SLICE][TILE];
  __shared__ __align__(16) float Bs[SLICE][TILE];
  int p = blockIdx.x, ti = 0;
  const int T = (l + TILE - 1) / TILE;
  while (p >= T - ti) { p -= T - ti; ++ti; }
  const int tj = ti + p;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t r_begin = (int64_t)blockIdx.y * rows_per_chunk;
  const int64_t r_end = min(m, r_begin + rows_per_chunk);
  float hi[R][R], lo[R][R];
#pragma unroll
  for (int i = 0; i < R; ++i)
#pragma unroll
    for (int j = 0; j < R; ++j) hi[i][j] = lo[i][j] = 0.f;
  float st[LD];
  auto load = [&](int64_t r0) {
#pragma unroll
    for (int u = 0; u < LD; ++u) {
      const int e = tid + 256 * u, which = e / (SLICE * TILE), ee = e % (SLICE * TILE);
      const int rr = ee / TILE, cc = ee % TILE;
      const int col = (which ? tj : ti) * TILE + cc;
      const int64_t r = r0 + rr;
      st[u] = (r < r_end && col < l) ? __ldg(Y + r * ldy + col) : 0.f;
    }
  };
  if (r_begin < r_end) load(r_begin);
  for (int64_t r0 = r_begin; r0 < r_end; r0 += SLICE) {
#pragma unroll
    for (int u = 0; u < LD; ++u) {
      const int e = tid + 256 * u, which = e / (SLICE * TILE), ee = e % (SLICE * TILE);
      (which ? &Bs[0][0] : &As[0][0])[ee] = st[u];
    }
    __syncthreads();
    if (r0 + SLICE < r_end) load(r0 + SLICE);
    float f[R][R];
#pragma unroll
    for (int i = 0; i < R; ++i)
#pragma unroll
      for (int j = 0; j < R; ++j) f[i][j] = 0.f;
#pragma unroll 4
    for (int rr = 0; rr < SLICE; ++rr) {
      float a[R], b[R];
#pragma unroll
      for (int i = 0; i < R; ++i) {
        a[i] = As[rr][ty * R + i];
        b[i] = Bs[rr][tx * R + i];
      }
#pragma unroll
      for (int i = 0; i < R; ++i)
#pragma unroll
        for (int j = 0; j < R; ++j) {
          if (EXACT) {
            const float pr = a[i] * b[j];
            f[i][j] += fmaf(a[i], b[j], -pr);
            two_sum_acc(hi[i][j], lo[i][j], pr);
          } else {
            f[i][j] = fmaf(a[i], b[j], f[i][j]);
          }
        }
    }
#pragma unroll
    for (int i = 0; i < R; ++i)
#pragma unroll
      for (int j = 0; j < R; ++j) {
        if (EXACT) lo[i][j] += f[i][j];          // the product errors of the slice
        else two_sum_acc(hi[i][j], lo[i][j], f[i][j]);
      }
    __syncthreads();
  }
  double *o = part + (int64_t)blockIdx.y * l * l;
#pragma unroll
  for (int i = 0; i < R; ++i)
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const int gi = ti * TILE + ty * R + i, gj = tj * TILE + tx * R + j;
      if (gi < l && gj < l) o[gi * l + gj] = (double)hi[i][j] + (double)lo[i][j];
    }
}

__global__ void gram_reduce_kernel(const double *__restrict__ part, int chunks, int l, int tile,
                                   double *__restrict__ G, const int *gate) {
  if (gate && !*gate) return;
  const int total = l * l;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const int i = e / l, j = e % l;
    if (i / tile > j / tile) continue;      // lower tiles are mirrored below
    double s = 0;
    for (int c = 0; c < chunks; ++c) s += part[(int64_t)c * total + e];
    G[i * l + j] = s;
    if (i / tile < j / tile) G[j * l + i] = s;
  }
}

// Rinv = R^-1 (upper triangular): one warp per column c solves R x = e_c by a column sweep.
__global__ void tri_inverse_cols_kernel(const double *R, int l, double *Rinv, float *Rinv32, const int *fail32,
                                        const int *fail64) {
  extern __shared__ double z[];   // l entries
  const int c = blockIdx.x, lane = threadIdx.x;
  if (!*fail32 || *fail64) return;   // the FP32 factor was used, or the FP64 one failed (status reported)
  for (int k = lane; k < l; k += 32) z[k] = (k == c) ? 1.0 : 0.0;
  __syncwarp();
  for (int i = c; i >= 0; --i) {
    const double xi = z[i] / R[(int64_t)i * l + i];
    __syncwarp();
    for (int k = lane; k < i; k += 32) z[k] = fma(-R[(int64_t)k * l + i], xi, z[k]);
    if (lane == 0) z[i] = xi;
    __syncwarp();
  }
  for (int k = lane; k < l; k += 32) {
    const double v = (k <= c) ? z[k] : 0.0;
    Rinv[(int64_t)k * l + c] = v;
    Rinv32[(int64_t)k * l + c] = (float)v;
  }
}

// ---------------------------------------------------- FP32 Cholesky of an FP64 Gram matrix (one block)
// On this GPU a dependent FP64 operation costs on the order of a hundred cycles, so the sequential part of a
// small factorization runs in FP32 (a few cycles per dependent operation) on the FP64 Gram matrix rounded to
// FP32, entirely in shared memory; least squares recovers FP64 accuracy by refinement against the FP64 Gram
// matrix.  The upper triangle is packed: U[i][j] (j >= i) lives at P[base[i] + j], base[i] = i*l - i(i+1)/2.
constexpr size_t kMaxPackedBytes = 200 * 1024;

__device__ __forceinline__ int pk_base(int i, int l) { return i * l - (i * (i + 1)) / 2; }

// Right-looking Cholesky of the packed matrix in place (block-wide): for each pivot j, scale row j of U, then
// update the trailing upper triangle, one warp per row, lanes along the row.  Returns false on a non-positive
// pivot.  dinv[j] receives 1 / U[j][j].
__device__ bool chol32_smem(float *P, const int *base, float *dinv, int l) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  for (int j = 0; j < l; ++j) {
    const int bj = base[j];
    const float d = P[bj + j];
    if (!(d > 0.f) || !isfinite(d)) return false;   // uniform: every thread read the same pivot
    const float r = sqrtf(d), inv = 1.f / r;
    __syncthreads();                                 // everyone has read the pivot before it changes
    for (int k = j + 1 + tid; k < l; k += blockDim.x) P[bj + k] *= inv;
    if (tid == 0) {
      P[bj + j] = r;
      dinv[j] = inv;
    }
    __syncthreads();
    for (int i = j + 1 + warp; i < l; i += nwarps) {
      const float gi = P[bj + i];
      const int bi = base[i];
      for (int k = i + lane; k < l; k += 32) P[bi + k] = fmaf(-gi, P[bj + k], P[bi + k]);
    }
    __syncthreads();
  }
  return true;
}


__device__ void load_packed(const double *G, int l, int ldg, float *P, int *base) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  for (int i = tid; i < l; i += blockDim.x) base[i] = pk_base(i, l);
  for (int i = warp; i < l; i += nwarps) {
    const int bi = pk_base(i, l);
    for (int j = i + lane; j < l; j += 32) P[bi + j] = (float)G[(int64_t)i * ldg + j];
  }
  __syncthreads();
}

// CholeskyQR step: factor G (l x l FP64) in FP32, write R (FP64, upper) into G and R^-1 in FP32 (Rinv32).
// fail[0] = 1 when the FP32 factorization broke down (the FP64 kernels below then take over).
// X_SMEM: R^-1 is built in shared memory (l x l more floats) and copied out; otherwise in Rinv32 directly.
template <bool X_SMEM>
__global__ void __launch_bounds__(512) chol32_inv_kernel(double *G, int l, float *Rinv32, int *fail) {
  extern __shared__ float smem32[];
  int *base = reinterpret_cast<int *>(smem32);
  float *dinv = smem32 + l;
  float *P = smem32 + 2 * l;
  float *X = X_SMEM ? P + (size_t)l * (l + 1) / 2 : Rinv32;   // X[i * l + c]: thread c's column
  load_packed(G, l, l, P, base);
  const bool ok = chol32_smem(P, base, dinv, l);
  if (threadIdx.x == 0) fail[0] = ok ? 0 : 1;
  if (!ok) return;
  __syncthreads();
  // R^-1, one thread per column c, rows from the bottom: X[i][c] = (delta_ic - sum_{k>i} U[i][k] X[k][c]) / U[i][i].
  // A column depends only on itself, so no synchronisation (consecutive threads, consecutive banks).
  for (int c = threadIdx.x; c < l; c += blockDim.x) {
    for (int i = l - 1; i > c; --i) X[(int64_t)i * l + c] = 0.f;
    for (int i = c; i >= 0; --i) {
      const int bi = base[i];
      float a0 = (i == c) ? 1.f : 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
      int k = i + 1;
      for (; k + 4 <= c + 1; k += 4) {
        a0 = fmaf(-P[bi + k], X[(int64_t)k * l + c], a0);
        a1 = fmaf(-P[bi + k + 1], X[(int64_t)(k + 1) * l + c], a1);
        a2 = fmaf(-P[bi + k + 2], X[(int64_t)(k + 2) * l + c], a2);
        a3 = fmaf(-P[bi + k + 3], X[(int64_t)(k + 3) * l + c], a3);
      }
      for (; k <= c; ++k) a0 = fmaf(-P[bi + k], X[(int64_t)k * l + c], a0);
      X[(int64_t)i * l + c] = ((a0 + a1) + (a2 + a3)) * dinv[i];
    }
  }
  if (X_SMEM) {
    __syncthreads();
    for (int e = threadIdx.x; e < l * l; e += blockDim.x) Rinv32[e] = X[e];
  }
  for (int e = threadIdx.x; e < l * l; e += blockDim.x) {
    const int i = e / l, j = e % l;
    G[e] = (j >= i) ? (double)P[base[i] + j] : 0.0;
  }
}

// The same factorization and inverse for l <= 128 with one barrier per pivot.  Right-looking without scaling the
// pivot row: in step j every row below it is updated from row j alone,
//   P[i][k] -= g_i P[j][k]   (k >= i),   B[i][c] -= g_i B[j][c]   (c <= j),   g_i = P[j][i] / P[j][j],  i > j,
// with B = I at the start; finally P[j][k] = r_j U[j][k] and B[j][c] = r_j Y[j][c], r_j = sqrt(P[j][j]) and
// Y = U^-T (forward substitution on U^T Y = I, row j of Y final in step j).
// The rows live in registers: warp w owns rows i = w + 16 r (r < 8), lane q holds columns 32 c + q (c < 4) of P
// and of B (entries outside a row's triangle are carried but never read).  In step j the owner of row j
// publishes it to shared memory (two buffers, alternating with j), and after the step's one barrier every warp
// reads it and updates its own rows below j in registers -- the trailing matrix never passes through shared
// memory.  The arithmetic is the packed right-looking form's, operation for operation.
constexpr int kCholFusedMaxL = 128;
constexpr int kCholFusedThreads = 512;

__global__ void __launch_bounds__(kCholFusedThreads) chol32_fused_kernel(double *G, int l, float *Rinv32, int *fail) {
  __shared__ float prow[2][kCholFusedMaxL], brow[2][kCholFusedMaxL], invr[kCholFusedMaxL];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  float P[8][4], B[8][4];
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int i = w + 16 * r;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int k = 32 * c + lane;
      P[r][c] = (i < l && k < l && k >= i) ? (float)G[(int64_t)i * l + k] : 0.f;
      B[r][c] = (i < l && k == i) ? 1.f : 0.f;
    }
  }
  for (int j = 0; j < l; ++j) {
    const int buf = j & 1;
    if (w == (j & 15)) {                       // the owner publishes row j (final since step j - 1)
      const int rj = j >> 4;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        float pv = 0.f, bv = 0.f;
#pragma unroll
        for (int r = 0; r < 8; ++r)
          if (r == rj) {
            pv = P[r][c];
            bv = B[r][c];
          }
        prow[buf][32 * c + lane] = pv;
        brow[buf][32 * c + lane] = bv;
      }
    }
    __syncthreads();
    const float d = prow[buf][j];
    if (!(d > 0.f) || !isfinite(d)) {        // uniform: every thread read the same pivot
      if (t == 0) fail[0] = 1;
      return;
    }
    const float invd = 1.f / d;
    if (t == 0) invr[j] = 1.f / sqrtf(d);
    float pjk[4], bjc[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int k = 32 * c + lane;
      pjk[c] = (k > j && k < l) ? prow[buf][k] : 0.f;
      bjc[c] = (k <= j) ? brow[buf][k] : 0.f;
    }
    // pjk is zero at k <= j and k >= l, bjc at k > j: the updates need no masks.  Where they reach entries
    // outside row i's triangle (j < k < i of P) those entries are never read again.
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int i = w + 16 * r;
      if (i > j && i < l) {                    // uniform across the warp
        const float g = prow[buf][i] * invd;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          P[r][c] = fmaf(-g, pjk[c], P[r][c]);
          B[r][c] = fmaf(-g, bjc[c], B[r][c]);
        }
      }
    }
  }
  __syncthreads();   // invr complete
  if (t == 0) fail[0] = 0;
  // R (FP64, upper, zeros below) and R^-1 = Y^T (FP32, row-major): R[i][k] = P[i][k] / r_i, R^-1[c][j] = B[j][c] / r_j
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int i = w + 16 * r;
    if (i < l) {
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int k = 32 * c + lane;
        if (k < l) {
          G[(int64_t)i * l + k] = (k >= i) ? (double)(P[r][c] * invr[i]) : 0.0;
          Rinv32[(int64_t)k * l + i] = (k <= i) ? B[r][c] * invr[i] : 0.f;
        }
      }
    }
  }
}

size_t chol32_fused_smem_bytes(int l) { (void)l; return 0; }

// Least squares on the augmented FP64 Gram matrix G ((n+1) x (n+1), last column g = [S^T A]^T S^T b):
// U = chol32(G11), then x0 = U^-1 U^-T g and x += U^-1 U^-T (g - G11 x) with FP64 residuals (iters times).
// fail[0] = 1 when the FP32 factorization broke down (the FP64 kernels below then take over).
size_t chol32_smem_bytes(int l) { return sizeof(float) * (2 * (size_t)l + (size_t)l * (l + 1) / 2); }

// The FP64 path runs only when the FP32 one failed.  Matrices whose packed triangle does not fit in shared
// memory go straight to the FP64 path.
__global__ void force_fp64_kernel(int *fail32) { *fail32 = 1; }

// FP64 fallback, one block: Cholesky of G (l x l) in place (upper), only if *fail32 is set.  A non-positive
// pivot reports RMC_ENUMERIC and sets *fail64.
__global__ void __launch_bounds__(1024) chol64_fallback_kernel(double *G, int l, const int *fail32, int *status,
                                                               int *fail64) {
  __shared__ double piv;
  __shared__ int bad;
  if (!*fail32) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  if (tid == 0) bad = 0;
  __syncthreads();
  for (int j = 0; j < l; ++j) {
    if (tid == 0) {
      const double d = G[(int64_t)j * l + j];
      if (!(d > 0.0) || !isfinite(d)) bad = 1;
      else {
        piv = sqrt(d);
        G[(int64_t)j * l + j] = piv;
      }
    }
    __syncthreads();
    if (bad) break;
    for (int i = j + 1 + tid; i < l; i += blockDim.x) G[(int64_t)j * l + i] /= piv;
    __syncthreads();
    for (int i = j + 1 + warp; i < l; i += nwarps) {
      const double gi = G[(int64_t)j * l + i];
      for (int k = i + lane; k < l; k += 32) G[(int64_t)i * l + k] = fma(-gi, G[(int64_t)j * l + k], G[(int64_t)i * l + k]);
    }
    __syncthreads();
  }
  for (int64_t e = tid; e < (int64_t)l * l; e += blockDim.x)
    if (e / l > e % l) G[e] = 0.0;
  if (tid == 0) {
    *fail64 = bad;
    if (bad) rmc_report(status, RMC_ENUMERIC);
  }
}

// C = A B for upper-triangular l x l FP64 matrices (the R of CholeskyQR2 is R2 R1); one block per row.
__global__ void tri_mul_kernel(const double *A, const double *B, int l, double *C) {
  const int i = blockIdx.x;
  for (int j = threadIdx.x; j < l; j += blockDim.x) {
    double s = 0.0;
    for (int k = i; k <= j; ++k) s = fma(A[i * l + k], B[k * l + j], s);
    C[i * l + j] = (i <= j) ? s : 0.0;
  }
}

// ------------------------------------------------------------- row block times a small matrix (in place)
// out[r, 0:lo] = in[r, 0:li] M (M li x lo, row stride ldm, FP32), 32 rows per block; with SUB,
// out[r, 0:lo] -= in[r, 0:li] M.  in and out may alias: every block reads its rows into shared memory before
// writing them.
constexpr int RB = 32;

template <bool SUB>
__global__ void __launch_bounds__(256) rowblock_mul_kernel(const float *in, int64_t m, int li, int64_t ldi,
                                                           const float *__restrict__ M, int lo, int64_t ldm,
                                                           float *out, int64_t ldo) {
  extern __shared__ float Ys[];  // RB x li
  const int64_t r0 = (int64_t)blockIdx.x * RB;
  for (int e = threadIdx.x; e < RB * li; e += blockDim.x) {
    const int rr = e / li, c = e % li;
    Ys[e] = (r0 + rr < m) ? in[(r0 + rr) * ldi + c] : 0.f;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;  // warp w: rows 4w .. 4w+3
  for (int c0 = 0; c0 < lo; c0 += 32 * 4) {
    float acc[4][4] = {};
    for (int k = 0; k < li; ++k) {
      float mv[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int c = c0 + lane + 32 * t;
        mv[t] = (c < lo) ? M[(int64_t)k * ldm + c] : 0.f;
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float y = Ys[(4 * warp + i) * li + k];
#pragma unroll
        for (int t = 0; t < 4; ++t) acc[i][t] = fmaf(y, mv[t], acc[i][t]);
      }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int64_t r = r0 + 4 * warp + i;
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int c = c0 + lane + 32 * t;
        if (r < m && c < lo) {
          if (SUB) out[r * ldo + c] -= acc[i][t];
          else out[r * ldo + c] = acc[i][t];
        }
      }
    }
  }
}

// The same product for li, lo <= 128 with register tiles: 64 rows per block, both operands in shared memory
// (the row block transposed, M padded to 128 columns with zeros), 256 threads as 16 x 16, thread (ty, tx)
// owning rows 4 ty .. 4 ty + 3 and columns 4 tx .. 4 tx + 3 and 64 + 4 tx .. 64 + 4 tx + 3: three 16-byte
// shared-memory loads per 32 FMAs.
constexpr int RB2 = 64, RB2_LD = RB2 + 4;

template <bool SUB>
__global__ void __launch_bounds__(256) rowblock_tile_kernel(const float *in, int64_t m, int li, int64_t ldi,
                                                            const float *__restrict__ M, int lo, int64_t ldm,
                                                            float *out, int64_t ldo) {
  extern __shared__ __align__(16) float rbs[];
  float *Yt = rbs, *Ms = rbs + (size_t)li * RB2_LD;   // Yt[k][r] (li x RB2_LD), Ms[k][c] (li x 128)
  const int64_t r0 = (int64_t)blockIdx.x * RB2;
  // both operands by 4-byte cp.async, all in flight at once (a load-then-store loop would wait out the
  // latency of every load in turn); out-of-range elements are zero-filled (source size 0)
  for (int e = threadIdx.x; e < RB2 * li; e += blockDim.x) {
    const int rr = e / li, k = e - rr * li;
    const bool in_range = r0 + rr < m;
    const float *src = in_range ? in + (r0 + rr) * ldi + k : in;
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"((unsigned)__cvta_generic_to_shared(
                     Yt + k * RB2_LD + rr)),
                 "l"(src), "r"(in_range ? 4 : 0)
                 : "memory");
  }
  for (int e = threadIdx.x; e < li * 128; e += blockDim.x) {
    const int k = e >> 7, c = e & 127;
    const bool in_range = c < lo;
    const float *src = in_range ? M + (int64_t)k * ldm + c : M;
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"((unsigned)__cvta_generic_to_shared(Ms + e)),
                 "l"(src), "r"(in_range ? 4 : 0)
                 : "memory");
  }
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
  __syncthreads();
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float acc[4][8] = {};
#pragma unroll 4
  for (int k = 0; k < li; ++k) {
    const float4 a = *reinterpret_cast<const float4 *>(Yt + k * RB2_LD + 4 * ty);
    const float4 b0 = *reinterpret_cast<const float4 *>(Ms + k * 128 + 4 * tx);
    const float4 b1 = *reinterpret_cast<const float4 *>(Ms + k * 128 + 64 + 4 * tx);
    const float av[4] = {a.x, a.y, a.z, a.w};
    const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t r = r0 + 4 * ty + i;
    if (r >= m) continue;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int c = (j < 4 ? 4 * tx + j : 64 + 4 * tx + j - 4);
      if (c < lo) {
        if (SUB) out[r * ldo + c] -= acc[i][j];
        else out[r * ldo + c] = acc[i][j];
      }
    }
  }
}

__global__ void transpose_kernel(const float *__restrict__ in, int64_t rows, int64_t cols, int64_t ldi,
                                 float *__restrict__ out, int64_t ldo) {
  __shared__ float tile[32][33];
  const int64_t bx = (int64_t)blockIdx.x * 32, by = (int64_t)blockIdx.y * 32;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int64_t r = by + k, c = bx + threadIdx.x;
    if (r < rows && c < cols) tile[k][threadIdx.x] = in[r * ldi + c];
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int64_t c = bx + k, r = by + threadIdx.x;
    if (r < rows && c < cols) out[c * ldo + r] = tile[threadIdx.x][k];
  }
}

// ------------------------------------------------------------------- one-sided Jacobi SVD (one block)
// W (l x l, column-major in global memory) is rotated until its columns are mutually orthogonal; V accumulates
// the rotations.  Round-robin ordering: in each of the l'-1 rounds (l' = l rounded up to even) the l'/2
// disjoint column pairs are rotated in parallel, one warp per pair.  Rotation as in the textbook one-sided
// (Hestenes) method: zeta = (beta - alpha) / (2 gamma), t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)).
template <typename T>
__global__ void __launch_bounds__(1024) jacobi_kernel(T *W, T *V, int l, T tol, int max_sweeps, int *status) {
  __shared__ int rotated;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  for (int e = threadIdx.x; e < l * l; e += blockDim.x) V[e] = (e / l == e % l) ? T(1) : T(0);
  const int lp = (l + 1) & ~1;
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    if (threadIdx.x == 0) rotated = 0;
    __syncthreads();
    for (int round = 0; round < lp - 1; ++round) {
      for (int pr = warp; pr < lp / 2; pr += nwarps) {
        // round-robin pairing: position 0 fixed, positions 1..lp-1 rotate
        const int a = pr, b = lp - 1 - pr;
        auto pos = [&](int x) { return x == 0 ? 0 : 1 + (x - 1 + round) % (lp - 1); };
        int p = pos(a), q = pos(b);
        if (p > q) { const int t = p; p = q; q = t; }
        if (q >= l) continue;  // the padding column of an odd l
        T *wp = W + (int64_t)p * l, *wq = W + (int64_t)q * l;
        T alpha = 0, beta = 0, gamma = 0;
        for (int r = lane; r < l; r += 32) {
          const T x = wp[r], y = wq[r];
          alpha += x * x;
          beta += y * y;
          gamma += x * y;
        }
        for (int o = 16; o; o >>= 1) {
          alpha += __shfl_xor_sync(0xffffffffu, alpha, o);
          beta += __shfl_xor_sync(0xffffffffu, beta, o);
          gamma += __shfl_xor_sync(0xffffffffu, gamma, o);
        }
        if (gamma == T(0) || fabs(gamma) <= tol * sqrt(alpha * beta)) continue;
        const T zeta = (beta - alpha) / (T(2) * gamma);
        const T t = copysign(T(1), zeta) / (fabs(zeta) + sqrt(T(1) + zeta * zeta));
        const T c = T(1) / sqrt(T(1) + t * t), s = c * t;
        for (int r = lane; r < l; r += 32) {
          const T x = wp[r], y = wq[r];
          wp[r] = c * x - s * y;
          wq[r] = s * x + c * y;
        }
        T *vp = V + (int64_t)p * l, *vq = V + (int64_t)q * l;
        for (int r = lane; r < l; r += 32) {
          const T x = vp[r], y = vq[r];
          vp[r] = c * x - s * y;
          vq[r] = s * x + c * y;
        }
        if (lane == 0) rotated = 1;
      }
      __syncthreads();
    }
    if (!rotated) break;
    __syncthreads();
  }
  if (sweep == max_sweeps && threadIdx.x == 0) rmc_report(status, RMC_ENUMERIC);
}

// Jacobi rotation (c, s) zeroing the inner product of a column pair.
__device__ __forceinline__ void rotation(double alpha, double beta, double gamma, double &c, double &s) {
  const double zeta = (beta - alpha) / (2.0 * gamma);
  const double t = copysign(1.0, zeta) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
  c = 1.0 / sqrt(1.0 + t * t);
  s = c * t;
}
__device__ __forceinline__ void rotation(float alpha, float beta, float gamma, float &c, float &s) {
  // correctly rounded reciprocals and square roots: an approximate rsqrt biases c^2 + s^2 below 1 and the
  // column norms (the singular values) shrink a little at every one of their ~l x sweeps rotations
  const float zeta = (beta - alpha) * __frcp_rn(2.f * gamma);
  const float t = copysignf(1.f, zeta) * __frcp_rn(fabsf(zeta) + __fsqrt_rn(fmaf(zeta, zeta, 1.f)));
  c = __frcp_rn(__fsqrt_rn(fmaf(t, t, 1.f)));
  s = c * t;
}

// The same rotations with W and V held in shared memory (used when 2 l^2 values fit): a pair costs a few
// hundred cycles instead of global-memory round trips.
template <typename T>
__global__ void __launch_bounds__(1024) jacobi_smem_kernel(T *Wg, T *Vg, int l, T tol, int max_sweeps, int *status) {
  extern __shared__ __align__(16) unsigned char jac_raw[];
  T *W = reinterpret_cast<T *>(jac_raw);
  T *V = W + (size_t)l * l;
  __shared__ int rotated;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  for (int e = threadIdx.x; e < l * l; e += blockDim.x) {
    W[e] = Wg[e];
    V[e] = (e / l == e % l) ? T(1) : T(0);
  }
  const int lp = (l + 1) & ~1;
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    if (threadIdx.x == 0) rotated = 0;
    __syncthreads();
    for (int round = 0; round < lp - 1; ++round) {
      for (int pr = warp; pr < lp / 2; pr += nwarps) {
        const int a = pr, b = lp - 1 - pr;
        int p = a == 0 ? 0 : 1 + (a - 1 + round) % (lp - 1);
        int q = b == 0 ? 0 : 1 + (b - 1 + round) % (lp - 1);
        if (p > q) { const int t = p; p = q; q = t; }
        if (q >= l) continue;
        T *wp = W + (size_t)p * l, *wq = W + (size_t)q * l;
        T alpha = 0, beta = 0, gamma = 0;
        for (int r = lane; r < l; r += 32) {
          const T x = wp[r], y = wq[r];
          alpha = fma(x, x, alpha);
          beta = fma(y, y, beta);
          gamma = fma(x, y, gamma);
        }
        for (int o = 16; o; o >>= 1) {
          alpha += __shfl_xor_sync(0xffffffffu, alpha, o);
          beta += __shfl_xor_sync(0xffffffffu, beta, o);
          gamma += __shfl_xor_sync(0xffffffffu, gamma, o);
        }
        if (gamma == T(0) || fabs(gamma) <= tol * sqrt(alpha * beta)) continue;
        T c, sn;
        rotation(alpha, beta, gamma, c, sn);
        T *vp = V + (size_t)p * l, *vq = V + (size_t)q * l;
        for (int r = lane; r < l; r += 32) {
          const T x = wp[r], y = wq[r];
          wp[r] = c * x - sn * y;
          wq[r] = sn * x + c * y;
          const T u = vp[r], v = vq[r];
          vp[r] = c * u - sn * v;
          vq[r] = sn * u + c * v;
        }
        if (lane == 0) rotated = 1;
      }
      __syncthreads();
    }
    if (!rotated) break;
    __syncthreads();
  }
  if (sweep == max_sweeps && threadIdx.x == 0) rmc_report(status, RMC_ENUMERIC);
  __syncthreads();
  for (int e = threadIdx.x; e < l * l; e += blockDim.x) {
    Wg[e] = W[e];
    Vg[e] = V[e];
  }
}

// After Jacobi on the triangular factor R of B^T (B^T = Q2 R, R = W V^T column-wise, sigma_j = ||w_j||):
//   Ub[:, rank(j)] = V[:, j]           (left singular vectors of B, l x l, row-major)
//   M[:, rank(j)]  = w_j / sigma_j     (so that Vb = Q2 M)
//   sigma[rank(j)] = sigma_j, descending (ties by index).
template <typename T>
__global__ void jacobi_finish_kernel(const T *W, const T *V, int l, float *Ub, float *M, float *sigma) {
  extern __shared__ double sg[];
  for (int j = threadIdx.x; j < l; j += blockDim.x) {
    double s = 0;
    for (int r = 0; r < l; ++r) s += (double)W[(int64_t)j * l + r] * (double)W[(int64_t)j * l + r];
    sg[j] = sqrt(s);
  }
  __syncthreads();
  for (int j = threadIdx.x; j < l; j += blockDim.x) {
    int rank = 0;
    for (int u = 0; u < l; ++u) rank += (sg[u] > sg[j]) || (sg[u] == sg[j] && u < j);
    sigma[rank] = (float)sg[j];
    const double inv = sg[j] > 0 ? 1.0 / sg[j] : 0.0;
    for (int r = 0; r < l; ++r) {
      Ub[r * l + rank] = (float)V[(int64_t)j * l + r];
      M[r * l + rank] = (float)(W[(int64_t)j * l + r] * inv);
    }
  }
}

// ---------------------------------------------------- one-sided Jacobi, a lane group per column pair
// The same round-robin rotations as jacobi_smem_kernel, with W alone in shared memory (no rotation
// accumulator: the other singular factor is recovered afterwards, see jacobi_right_kernel) and a group of G lanes
// per column pair instead of a warp: a 1024-thread block rotates up to 1024 / G disjoint pairs per round, each
// lane holding every G-th row (G = 16 up to l = 128 and 8 above in FP64; FP32 uses it above l = 128 with G = 8,
// and jacobi_oe_kernel below that).
// G lanes per pair (8 or 16; 1024 / G pairs per round at most).
template <typename T, int G>
__global__ void __launch_bounds__(1024) jacobi_grp_kernel(T *Wg, int l, T tol, int max_sweeps, int *status) {
  extern __shared__ __align__(16) unsigned char jg_raw[];
  T *W = reinterpret_cast<T *>(jg_raw);
  __shared__ int rotated;
  for (int e = threadIdx.x; e < l * l; e += blockDim.x) W[e] = Wg[e];
  const int grp = threadIdx.x / G, j = threadIdx.x % G;
  const int lp = (l + 1) & ~1;
  const T tol2 = tol * tol;
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    if (threadIdx.x == 0) rotated = 0;
    __syncthreads();
    for (int round = 0; round < lp - 1; ++round) {
      int p = -1, q = -1;
      if (grp < lp / 2) {
        const int a = grp, b = lp - 1 - grp;
        p = a == 0 ? 0 : 1 + (a - 1 + round) % (lp - 1);
        q = b == 0 ? 0 : 1 + (b - 1 + round) % (lp - 1);
        if (p > q) {
          const int t = p;
          p = q;
          q = t;
        }
        if (q >= l) p = -1;
      }
      T alpha = 0, beta = 0, gamma = 0;
      T *wp = W + (size_t)(p < 0 ? 0 : p) * l, *wq = W + (size_t)(p < 0 ? 0 : q) * l;
      if (p >= 0)
        for (int r = j; r < l; r += G) {
          const T x = wp[r], y = wq[r];
          alpha = fma(x, x, alpha);
          beta = fma(y, y, beta);
          gamma = fma(x, y, gamma);
        }
      // the G lanes of a group are aligned in the warp: xor offsets below G stay inside the group
#pragma unroll
      for (int o = 1; o < G; o <<= 1) {
        alpha += __shfl_xor_sync(0xffffffffu, alpha, o);
        beta += __shfl_xor_sync(0xffffffffu, beta, o);
        gamma += __shfl_xor_sync(0xffffffffu, gamma, o);
      }
      if (p >= 0 && gamma != T(0) && gamma * gamma > tol2 * alpha * beta) {
        T c, sn;
        rotation(alpha, beta, gamma, c, sn);
        for (int r = j; r < l; r += G) {
          const T x = wp[r], y = wq[r];
          wp[r] = c * x - sn * y;
          wq[r] = sn * x + c * y;
        }
        if (j == 0) rotated = 1;
      }
      __syncthreads();
    }
    if (!rotated) break;
    __syncthreads();
  }
  if (sweep == max_sweeps && threadIdx.x == 0) rmc_report(status, RMC_ENUMERIC);
  __syncthreads();
  for (int e = threadIdx.x; e < l * l; e += blockDim.x) Wg[e] = W[e];
}

// FP32 rotation for the vectorised kernel below.  The angle only steers convergence, so t is formed with fast
// reciprocals and square roots; c = (1 + t^2)^-1/2 is correctly rounded and s = c t, so that c^2 + s^2 - 1 is an
// unbiased rounding error and the column norms do not drift over the ~l x sweeps rotations of a column.
__device__ __forceinline__ void rotation_fast(float alpha, float beta, float gamma, float &c, float &s) {
  const float zeta = __fdividef(beta - alpha, 2.f * gamma);
  const float x = fmaf(zeta, zeta, 1.f);
  const float t = copysignf(__fdividef(1.f, fabsf(zeta) + x * rsqrtf(x)), zeta);
  c = __frsqrt_rn(fmaf(t, t, 1.f));
  s = c * t;
}


// One-sided Jacobi for l <= 128 (FP32) in the odd-even ordering: the l' = l rounded up to even columns sit on
// positions 0 .. l'-1; even rounds rotate the pairs of positions (2i, 2i+1), odd rounds (2i+1, 2i+2), and every
// rotated pair swaps positions, so that in l' rounds (one sweep) each pair of columns meets exactly once (the
// swaps of odd-even transposition reverse the order).  Group i (8 lanes, rows 4j + 32v .. +3 of each column in
// float4 registers; padding rows are zeros) takes pair i of every round, and one of its two columns stays with it
// into the next round: per round a group stores the column that leaves for its neighbour into that position's
// shared-memory slot and, after the round's barrier, loads the one that arrives -- half the shared-memory traffic
// of reloading both.  Even round: group i holds positions 2i (loaded) and 2i+1 (kept), sends 2i to group i-1 and
// receives 2i+2 from group i+1; odd round: it holds 2i+1 (kept) and 2i+2, sends 2i+2 and receives 2i (group l'/2-1
// only joins the shuffles in odd rounds; position 0 waits in its slot).  Each slot is written by one group and
// read by one group per round, on opposite sides of the barrier, so one barrier per round suffices.  A zero padding column (odd l)
// is never rotated; after an odd number of sweeps it sits at position 0, else at l'-1, and is skipped on output.
// Columns leave in position order (a permutation of the input's): the callers rank them by norm.
template <int NV>
__global__ void __launch_bounds__(512) jacobi_oe_kernel(float *Wg, int l, float tol, int max_sweeps, int *status) {
  extern __shared__ __align__(16) float jv[];
  constexpr int ldw = 32 * NV;
  __shared__ int rotated;
  const int lp = (l + 1) & ~1;
#pragma unroll 8
  for (int e = threadIdx.x; e < lp * ldw; e += blockDim.x) {
    const int col = e / ldw, r = e % ldw;
    jv[e] = (r < l && col < l) ? Wg[(int64_t)col * l + r] : 0.f;
  }
  __syncthreads();
  // The block is a whole number of warps: groups past the l'/2 pairs ("real" false) hold zeros, touch no slot
  // and only join the warp shuffles, so every lane of every warp runs the same shuffle sequence.
  const int gi = threadIdx.x >> 3, j = threadIdx.x & 7;
  const int last = lp / 2 - 1;
  const bool real = gi <= last;
  const float tol2 = tol * tol;
  float4 arr[NV], keep[NV];
  auto store = [&](int pos, const float4 (&x)[NV]) {
    float4 *d = reinterpret_cast<float4 *>(jv + (size_t)pos * ldw) + j;
#pragma unroll
    for (int v = 0; v < NV; ++v) d[8 * v] = x[v];
  };
  auto load = [&](int pos, float4 (&x)[NV]) {
    const float4 *a = reinterpret_cast<const float4 *>(jv + (size_t)pos * ldw) + j;
#pragma unroll
    for (int v = 0; v < NV; ++v) x[v] = a[8 * v];
  };
#pragma unroll
  for (int v = 0; v < NV; ++v) arr[v] = keep[v] = make_float4(0.f, 0.f, 0.f, 0.f);
  if (real) {
    load(2 * gi, arr);
    load(2 * gi + 1, keep);
  }
  // Rotate (x, y) in place (x <- c x - s y, y <- s x + c y) where live and the pair's inner products ask for it.
  // Called by every thread in every round: the inner products are reduced over the group's 8 lanes by shuffles
  // that name the whole warp.
  auto rotate = [&](float4 (&x)[NV], float4 (&y)[NV], bool live) {
    float alpha = 0.f, beta = 0.f, gamma = 0.f;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      alpha = fmaf(x[v].x, x[v].x, fmaf(x[v].y, x[v].y, fmaf(x[v].z, x[v].z, fmaf(x[v].w, x[v].w, alpha))));
      beta = fmaf(y[v].x, y[v].x, fmaf(y[v].y, y[v].y, fmaf(y[v].z, y[v].z, fmaf(y[v].w, y[v].w, beta))));
      gamma = fmaf(x[v].x, y[v].x, fmaf(x[v].y, y[v].y, fmaf(x[v].z, y[v].z, fmaf(x[v].w, y[v].w, gamma))));
    }
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) {   // the 8 lanes of a group are aligned in the warp
      alpha += __shfl_xor_sync(0xffffffffu, alpha, o);
      beta += __shfl_xor_sync(0xffffffffu, beta, o);
      gamma += __shfl_xor_sync(0xffffffffu, gamma, o);
    }
    if (live && gamma != 0.f && gamma * gamma > tol2 * alpha * beta) {
      float c, sn;
      rotation_fast(alpha, beta, gamma, c, sn);
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const float4 u = x[v], w = y[v];
        x[v] = make_float4(c * u.x - sn * w.x, c * u.y - sn * w.y, c * u.z - sn * w.z, c * u.w - sn * w.w);
        y[v] = make_float4(sn * u.x + c * w.x, sn * u.y + c * w.y, sn * u.z + c * w.z, sn * u.w + c * w.w);
      }
      if (j == 0) rotated = 1;
    }
  };
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    if (threadIdx.x == 0) rotated = 0;
    __syncthreads();
#pragma unroll 1
    for (int round = 0; round < lp; round += 2) {
      // even round: (2i, 2i+1) = (arr, keep); after the swap position 2i holds the rotated keep
      rotate(arr, keep, real);
      if (real) {
        store(2 * gi, keep);                    // leaves for group i-1 (position 2i)
#pragma unroll
        for (int v = 0; v < NV; ++v) keep[v] = arr[v];   // position 2i+1 stays
      }
      __syncthreads();
      if (real && gi < last) load(2 * gi + 2, arr);      // arrives from group i+1
      // odd round: (2i+1, 2i+2) = (keep, arr); after the swap position 2i+2 holds the rotated keep
      rotate(keep, arr, real && gi < last);
      if (real && gi < last) {
        store(2 * gi + 2, keep);                // leaves for group i+1 (position 2i+2)
#pragma unroll
        for (int v = 0; v < NV; ++v) keep[v] = arr[v];   // position 2i+1 stays
      }
      __syncthreads();
      if (real) load(2 * gi, arr);              // arrives from group i-1 (group 0: position 0, unchanged)
    }
    if (!rotated) break;
    __syncthreads();
  }
  if (sweep == max_sweeps && threadIdx.x == 0) rmc_report(status, RMC_ENUMERIC);
  const int done = sweep < max_sweeps ? sweep + 1 : max_sweeps;
  if (real) store(2 * gi + 1, keep);            // position 2i+1 lived in registers
  __syncthreads();
  const int pad = (lp == l) ? -1 : ((done & 1) ? 0 : lp - 1);
  for (int e = threadIdx.x; e < l * l; e += blockDim.x) {
    const int c = e / l, r = e % l;
    const int pos = (pad >= 0 && c >= pad) ? c + 1 : c;
    Wg[e] = jv[(size_t)pos * ldw + r];
  }
}

// After jacobi_grp_kernel on R (R V = W, columns of W orthogonal): sigma_j = ||w_j|| (FP64 sum), the columns
// ranked by descending sigma (ties by index), M[:, rank(j)] = w_j / sigma_j (the left singular vectors of R,
// row-major l x l FP32) and sigma[rank(j)].
template <typename T>
__global__ void jacobi_left_kernel(const T *W, int l, float *M, float *sigma) {
  extern __shared__ double sgl[];
  for (int jj = threadIdx.x; jj < l; jj += blockDim.x) {
    double s = 0;
    for (int r = 0; r < l; ++r) s += (double)W[(int64_t)jj * l + r] * (double)W[(int64_t)jj * l + r];
    sgl[jj] = sqrt(s);
  }
  __syncthreads();
  for (int jj = threadIdx.x; jj < l; jj += blockDim.x) {
    int rank = 0;
    for (int u = 0; u < l; ++u) rank += (sgl[u] > sgl[jj]) || (sgl[u] == sgl[jj] && u < jj);
    sigma[rank] = (float)sgl[jj];
    const double inv = sgl[jj] > 0 ? 1.0 / sgl[jj] : 0.0;
    for (int r = 0; r < l; ++r) M[r * l + rank] = (float)(W[(int64_t)jj * l + r] * inv);
  }
}

// The right singular vectors of R (upper triangular, row-major FP64) from its left ones: R = M diag(sigma) V^T
// gives V = R^T M diag(sigma)^-1, Ub[:, c] = R^T M[:, c] / sigma_c in FP64 (one block per column c).  The error
// of column c is about eps_FP32 * sigma_1 / sigma_c: FP32-level for the leading columns a k-SVD keeps.
__global__ void jacobi_right_kernel(const double *R, int l, const float *M, const float *sigma, float *Ub) {
  const int c = blockIdx.x;
  const double inv = sigma[c] > 0.f ? 1.0 / (double)sigma[c] : 0.0;
  for (int r = threadIdx.x; r < l; r += blockDim.x) {
    double acc = 0.0;
    for (int i = 0; i <= r; ++i) acc += R[(int64_t)i * l + r] * (double)M[(int64_t)i * l + c];
    Ub[(int64_t)r * l + c] = (float)(acc * inv);
  }
}

// R (row-major FP64, upper) -> column-major working copy of type T.
template <typename T>
__global__ void to_colmajor_kernel(const double *R, int l, T *W) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < l * l; e += gridDim.x * blockDim.x) {
    const int i = e / l, j = e % l;
    W[(int64_t)j * l + i] = (T)R[e];
  }
}

// ---------------------------------------------------------------- rsvd tail: signs, U = Q Ub[:, :k], V
// For column i < k: the entry of largest magnitude of Vb[:, i] (first one on ties) is made positive.
__global__ void sign_fix_kernel(const float *Vb, int64_t n, int64_t ldvb, const float *Ub, int l, int k,
                                float *Msigned, float *V, int64_t ldv, const float *sg, float *sigma) {
  __shared__ float best[1024];
  __shared__ int64_t where[1024];
  const int i = blockIdx.x;
  float b = -1.f;
  int64_t w = 0;
  for (int64_t r = threadIdx.x; r < n; r += blockDim.x) {
    const float v = fabsf(Vb[r * ldvb + i]);
    if (v > b) { b = v; w = r; }
  }
  best[threadIdx.x] = b;
  where[threadIdx.x] = w;
  __syncthreads();
  for (int o = blockDim.x / 2; o; o >>= 1) {
    if (threadIdx.x < o) {
      const float b2 = best[threadIdx.x + o];
      const int64_t w2 = where[threadIdx.x + o];
      if (b2 > best[threadIdx.x] || (b2 == best[threadIdx.x] && w2 < where[threadIdx.x])) {
        best[threadIdx.x] = b2;
        where[threadIdx.x] = w2;
      }
    }
    __syncthreads();
  }
  const float sgn = Vb[where[0] * ldvb + i] < 0.f ? -1.f : 1.f;
  for (int64_t r = threadIdx.x; r < n; r += blockDim.x) V[r * ldv + i] = sgn * Vb[r * ldvb + i];
  for (int r = threadIdx.x; r < l; r += blockDim.x) Msigned[r * k + i] = sgn * Ub[r * l + i];
  if (threadIdx.x == 0) sigma[i] = sg[i];
}

// ------------------------------------------------------------------------ least-squares back substitution
// x = R11^-1 r12 where R ((n+1) x (n+1), upper) is the Cholesky factor of the augmented Gram matrix: one warp,
// x_i = (r_i,n - sum_{k>i} R_ik x_k) / R_ii from the last row up, each dot product over the lanes.
__global__ void lsr_backsub_kernel(const double *R, int n, double *x, const int *fail32, const int *fail) {
  extern __shared__ double xs[];
  const int lda = n + 1, lane = threadIdx.x;
  if (!*fail32) return;        // the FP32 factor and refinement produced x
  if (fail && *fail) {
    for (int i = lane; i < n; i += 32) x[i] = nan("");
    return;
  }
  for (int i = n - 1; i >= 0; --i) {
    const double *row = R + (int64_t)i * lda;
    double acc = 0.0;
    for (int k = i + 1 + lane; k < n; k += 32) acc = fma(row[k], xs[k], acc);
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    const double xi = (row[n] - acc) / row[i];
    if (lane == 0) xs[i] = xi;
    __syncwarp();
  }
  for (int i = lane; i < n; i += 32) x[i] = xs[i];
}

__global__ void copy_column_kernel(const float *v, int64_t s, float *W, int64_t ldw, int64_t col) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < s; i += (int64_t)gridDim.x * blockDim.x)
    W[i * ldw + col] = v[i];
}

// ------------------------------------------------------------- least-squares solve: FP32 factor, refinement
// The normal-equation matrix SA^T SA is factored in FP32 (Gram with FP32 products summed in FP64 across
// 32-row slices; blocked right-looking Cholesky over 32-wide panels, many CTAs per step), its inverse is formed
// as M = R^-1 R^-T (R^-1 by block back substitution, one CTA per 32-column block), and x is then refined
// against SA itself: r = Sb - SA x and g = SA^T r in FP64 (FP32 x FP32 products are exact in FP64), dx = M g.
// The fixed point is the least-squares solution of the FP32 [SA, Sb] whatever the rounding of the factor and
// of M; each step shrinks the error by about cond(SA)^2 x 2^-24.  A pivot that is not positive, or a last step
// that has not converged, hands the problem to the FP64 path.
//
// flags: [0] FP32 path failed (FP64 takes over), [1] FP64 path failed, [2] refinement converged, [4 + 2 it] and
// [5 + 2 it]: bit patterns of max |dx| and max |x| after refinement step it (non-negative floats order like
// their bit patterns, so atomicMax on the words takes the maximum).
constexpr int kLsrFlagWords = 16;

// Step `it` ended the iteration: its correction is below tol ||x|| (and x is finite).
__device__ __forceinline__ bool lsr_converged(const int *flags, int it, float tol) {
  const float a = __uint_as_float((unsigned)flags[4 + 2 * it]), b = __uint_as_float((unsigned)flags[5 + 2 * it]);
  return b < INFINITY && a <= tol * b;
}

// Common early exit of the refinement kernels of step `it`: failed, or an earlier step converged.
__device__ __forceinline__ bool lsr_skip(int *flags, int it) {
  if (flags[0] || flags[2]) return true;
  if (it > 0 && lsr_converged(flags, it - 1, 1e-9f)) {
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) flags[2] = 1;
    return true;
  }
  return false;
}

constexpr int kPanel = 32;

// Rf (n x n, row-major, upper triangle used) = the leading n x n block of G (FP64, ld = ldg).
__global__ void lsr_rf_init_kernel(const double *G, int ldg, int n, float *Rf, int *flags) {
  if (blockIdx.x == 0 && threadIdx.x < kLsrFlagWords) flags[threadIdx.x] = 0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n * n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / n), j = (int)(e - (int64_t)i * n);
    Rf[e] = i <= j ? (float)G[(int64_t)i * ldg + j] : 0.f;
  }
}

// Panel j0: every CTA factors the 32 x 32 diagonal block (FP32, in shared memory), CTA 0 stores it and its
// inverse (Dinv, 32 x 32 row-major, identity in the padding of a ragged block), and each CTA forms its 256
// columns of the panel rows R[j0 : j0+32, c] = R_jj^-T Rf[j0 : j0+32, c] (thread per column).
__global__ void __launch_bounds__(256) lsr_chol_panel_kernel(float *Rf, int n, int j0, float *Dinv, int *fail) {
  __shared__ float D[kPanel][kPanel + 1];
  __shared__ int bad;
  if (*fail) return;
  const int t = threadIdx.x;
  const int b = min(kPanel, n - j0);
  for (int e = t; e < kPanel * kPanel; e += blockDim.x) {
    const int i = e / kPanel, j = e % kPanel;
    D[i][j] = (i < b && j < b && i <= j) ? Rf[(int64_t)(j0 + i) * n + j0 + j] : (i == j ? 1.f : 0.f);
  }
  if (t == 0) bad = 0;
  __syncthreads();
  // right-looking over the 32 x 32 block in one warp's registers: lane j holds column j (col[i] = D[i][j])
  if (t < 32) {
    const int lane = t;
    float col[kPanel];
#pragma unroll
    for (int i = 0; i < kPanel; ++i) col[i] = D[i][lane];
    bool ok = true;
#pragma unroll
    for (int k = 0; k < kPanel; ++k) {
      const float d = __shfl_sync(0xffffffffu, col[k], k);
      if (!(d > 0.f) || !(d < INFINITY)) ok = false;  // uniform across the warp
      const float rd = sqrtf(d), inv = 1.f / rd;
      col[k] = lane == k ? rd : (lane > k ? col[k] * inv : col[k]);
#pragma unroll
      for (int i = k + 1; i < kPanel; ++i) {
        const float rki = __shfl_sync(0xffffffffu, col[k], i);  // R[k][i]
        if (lane >= i) col[i] = fmaf(-rki, col[k], col[i]);
      }
    }
    if (!ok && lane == 0) bad = 1;
#pragma unroll
    for (int i = 0; i < kPanel; ++i) D[i][lane] = col[i];
  }
  __syncthreads();
  if (bad) {
    if (t == 0 && blockIdx.x == 0) *fail = 1;
    return;
  }
  if (blockIdx.x == 0) {
    for (int e = t; e < b * b; e += blockDim.x) {
      const int i = e / b, j = e % b;
      if (i <= j) Rf[(int64_t)(j0 + i) * n + j0 + j] = D[i][j];
    }
    if (t >= 32 && t < 64) {  // column j of D^-1 by back substitution (lane j)
      const int j = t - 32;
      float xv[kPanel];
#pragma unroll
      for (int i = kPanel - 1; i >= 0; --i) {
        float v = i == j ? 1.f : 0.f;
#pragma unroll
        for (int k = i + 1; k < kPanel; ++k) v = fmaf(-D[i][k], xv[k], v);
        xv[i] = v / D[i][i];
      }
      float *dst = Dinv + (int64_t)(j0 / kPanel) * kPanel * kPanel;
#pragma unroll
      for (int i = 0; i < kPanel; ++i) dst[i * kPanel + j] = xv[i];
    }
  }
  const int c = j0 + b + blockIdx.x * blockDim.x + t;
  if (c >= n) return;
  float x[kPanel];
#pragma unroll
  for (int k = 0; k < kPanel; ++k) x[k] = k < b ? Rf[(int64_t)(j0 + k) * n + c] : 0.f;
#pragma unroll
  for (int k = 0; k < kPanel; ++k) {
    float v = x[k];
#pragma unroll
    for (int p = 0; p < k; ++p) v = fmaf(-D[p][k], x[p], v);
    x[k] = v / D[k][k];
  }
#pragma unroll
  for (int k = 0; k < kPanel; ++k)
    if (k < b) Rf[(int64_t)(j0 + k) * n + c] = x[k];
}

// Trailing update after panel j0: Rf[i, c] -= sum_k R[j0+k, i] R[j0+k, c] for j0+32 <= i <= c < n, in 64 x 64
// tiles of the upper triangle (thread: 4 x 4 outputs).
__global__ void __launch_bounds__(256) lsr_chol_update_kernel(float *Rf, int n, int j0, const int *fail) {
  __shared__ float Pi[kPanel][64], Pc[kPanel][64];
  if (*fail) return;
  const int j1 = j0 + kPanel;
  int p = blockIdx.x, ti = 0;
  const int T = (n - j1 + 63) / 64;
  while (p >= T - ti) { p -= T - ti; ++ti; }
  const int tj = ti + p;
  const int i0 = j1 + 64 * ti, c0 = j1 + 64 * tj;
  const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
  for (int e = t; e < kPanel * 64; e += blockDim.x) {
    const int k = e / 64, q = e % 64;
    Pi[k][q] = i0 + q < n ? Rf[(int64_t)(j0 + k) * n + i0 + q] : 0.f;
    Pc[k][q] = c0 + q < n ? Rf[(int64_t)(j0 + k) * n + c0 + q] : 0.f;
  }
  __syncthreads();
  float acc[4][4] = {};
#pragma unroll 8
  for (int k = 0; k < kPanel; ++k) {
    float a[4], bb[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      a[u] = Pi[k][ty + 16 * u];
      bb[u] = Pc[k][tx + 16 * u];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(a[u], bb[v], acc[u][v]);
  }
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int i = i0 + ty + 16 * u, c = c0 + tx + 16 * v;
      if (i < n && c < n && i <= c) Rf[(int64_t)i * n + c] -= acc[u][v];
    }
}

// Column block J = blockIdx.x of R^-1 (rows 0 .. 32 J + 31) by block back substitution over the 32 x 32 blocks:
// X_JJ = D_J^-1 and X_IJ = -D_I^-1 sum_{K=I+1..J} R_IK X_KJ for I = J-1 .. 0 (thread (i, j) of the block).
__global__ void __launch_bounds__(1024) lsr_tri_inv_kernel(const float *Rf, const float *Dinv, int n, float *Ri,
                                                           const int *fail) {
  extern __shared__ float X[];  // rows 0 .. 32 (J + 1) - 1 of the column block, then T (32 x 32)
  if (*fail) return;
  const int J = blockIdx.x, t = threadIdx.x, i = t >> 5, j = t & 31;
  const int rows = kPanel * (J + 1), k1 = min(rows, n);
  float *Tm = X + (size_t)rows * kPanel;
  X[(kPanel * J + i) * kPanel + j] = Dinv[(int64_t)J * kPanel * kPanel + i * kPanel + j];
  __syncthreads();
  for (int I = J - 1; I >= 0; --I) {
    const float *rrow = Rf + (int64_t)(kPanel * I + i) * n;  // one row per warp: a broadcast load per k
    float acc = 0.f;
#pragma unroll 8
    for (int k = kPanel * (I + 1); k < k1; ++k) acc = fmaf(rrow[k], X[k * kPanel + j], acc);
    Tm[i * kPanel + j] = acc;
    __syncthreads();
    const float *drow = Dinv + (int64_t)I * kPanel * kPanel + i * kPanel;
    float v = 0.f;
#pragma unroll 8
    for (int k = 0; k < kPanel; ++k) v = fmaf(drow[k], Tm[k * kPanel + j], v);
    X[(kPanel * I + i) * kPanel + j] = -v;
    __syncthreads();
  }
  const int c = kPanel * J + j;
  if (c < n)
    for (int r = i; r < k1; r += kPanel) Ri[(int64_t)r * n + c] = X[r * kPanel + j];
}

// M = R^-1 R^-T (n x n, symmetric): M[a][c] = sum_{k >= max(a, c)} Ri[a][k] Ri[c][k], 64 x 64 tiles of the upper
// triangle (thread: 4 x 4 outputs), each written to both halves.  Ri is read only on and above its diagonal.
__global__ void __launch_bounds__(256) lsr_inv_gram_kernel(const float *Ri, int n, float *M, const int *fail) {
  __shared__ float Pa[kPanel][65], Pc[kPanel][65];
  if (*fail) return;
  int p = blockIdx.x, ta = 0;
  const int T = (n + 63) / 64;
  while (p >= T - ta) { p -= T - ta; ++ta; }
  const int tc = ta + p;
  const int a0 = 64 * ta, c0 = 64 * tc;
  const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
  float acc[4][4] = {};
  for (int k0 = c0; k0 < n; k0 += kPanel) {
    __syncthreads();
    for (int e = t; e < kPanel * 64; e += blockDim.x) {
      const int q = e >> 5, kk = e & 31, k = k0 + kk;
      const int ra = a0 + q, rc = c0 + q;
      Pa[kk][q] = (ra < n && k < n && k >= ra) ? Ri[(int64_t)ra * n + k] : 0.f;
      Pc[kk][q] = (rc < n && k < n && k >= rc) ? Ri[(int64_t)rc * n + k] : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < kPanel; ++k) {
      float av[4], cv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        av[u] = Pa[k][ty + 16 * u];
        cv[u] = Pc[k][tx + 16 * u];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(av[u], cv[v], acc[u][v]);
    }
  }
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int ia = a0 + ty + 16 * u, ic = c0 + tx + 16 * v;
      if (ia < n && ic < n && ia <= ic) {
        M[(int64_t)ia * n + ic] = acc[u][v];
        M[(int64_t)ic * n + ia] = acc[u][v];
      }
    }
}

// r = Sb - SA x (FP64), one warp per row of [SA, Sb] (s x (n+1), Sb in column n).
__global__ void lsr_resid_kernel(const float *SA, int64_t s, int n, int64_t ld, const double *x, double *r,
                                 int it, int *flags) {
  if (lsr_skip(flags, it)) return;
  const int lane = threadIdx.x & 31;
  for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; i < s;
       i += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const float *row = SA + i * ld;
    double acc = 0.0;
#pragma unroll 4
    for (int c = lane; c < n; c += 32) acc = fma((double)row[c], x[c], acc);
#pragma unroll
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) r[i] = (double)row[n] - acc;
  }
}

// part[chunk][c] = sum over the chunk's rows of SA[i, c] r_i (FP64), thread per column.
__global__ void lsr_atr_kernel(const float *SA, int64_t s, int n, int64_t ld, const double *r, int64_t rows_per,
                               double *part, int it, int *flags) {
  if (lsr_skip(flags, it)) return;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  const int64_t r0 = blockIdx.y * rows_per, r1 = min(s, r0 + rows_per);
  double acc = 0.0;
#pragma unroll 8
  for (int64_t i = r0; i < r1; ++i) acc = fma((double)SA[i * ld + c], r[i], acc);  // eight loads in flight
  part[(int64_t)blockIdx.y * n + c] = acc;
}

// dx = M g for the 32 rows of this CTA (g = sum of the chunk partials, one warp per row), x += dx, and the
// maxima of |dx| and |x| of step `it` into the flag words.
__global__ void __launch_bounds__(256) lsr_apply_kernel(const float *M, int n, const double *part, int chunks,
                                                        double *xs, int it, int *flags) {
  extern __shared__ float gsm[];  // g (n)
  if (lsr_skip(flags, it)) return;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  for (int c = t; c < n; c += blockDim.x) {
    double g = 0.0;
    for (int k = 0; k < chunks; ++k) g += part[(int64_t)k * n + c];
    gsm[c] = (float)g;
  }
  __syncthreads();
  unsigned mdx = 0u, mx = 0u;
  for (int rr = warp; rr < kPanel; rr += blockDim.x >> 5) {
    const int r = blockIdx.x * kPanel + rr;
    if (r >= n) break;
    const float *mrow = M + (int64_t)r * n;
    float acc = 0.f;
#pragma unroll 4
    for (int c = lane; c < n; c += 32) acc = fmaf(mrow[c], gsm[c], acc);
#pragma unroll
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) {
      const double nx = xs[r] + (double)acc;
      xs[r] = nx;
      const float adx = isfinite(acc) ? fabsf(acc) : INFINITY;
      const float ax = isfinite(nx) ? fabsf((float)nx) : INFINITY;
      mdx = max(mdx, __float_as_uint(adx));
      mx = max(mx, __float_as_uint(ax));
    }
  }
  if (lane == 0) {
    atomicMax(reinterpret_cast<unsigned *>(&flags[4 + 2 * it]), mdx);
    atomicMax(reinterpret_cast<unsigned *>(&flags[5 + 2 * it]), mx);
  }
}

// End of the refinement: x is written out if a step converged (correction below 1e-9 ||x||) or the last one is
// below 1e-5 ||x||; otherwise flags[0] hands the problem to the FP64 path.
__global__ void lsr_refine_finish_kernel(const double *xs, int n, int last, double *xout, int *flags) {
  if (flags[0]) return;
  const bool ok = flags[2] || lsr_converged(flags, last, 1e-5f);
  if (!ok) {
    if (threadIdx.x == 0) flags[0] = 1;
    return;
  }
  for (int c = threadIdx.x; c < n; c += blockDim.x) xout[c] = xs[c];
}

// ----------------------------------------------------------------------------------------- host helpers

// Products and sums of the Gram matrix (launch_gram): FP32 products summed in FP32 over 32-row slices and in
// double-FP32 across them; exact products in double-FP32; exact products in FP64 (least squares, refresh).
enum GramMode { kGramF32, kGramExact, kGramF64 };

static int gram_tile(int l, GramMode mode) { return (mode == kGramF64 || l <= 48) ? GRAM_T : 64; }

int gram_chunks(int64_t m, int l, int num_sms, int tile) {
  const int T = (l + tile - 1) / tile;
  const int pairs = T * (T + 1) / 2;
  int64_t chunks = (2 * (int64_t)num_sms + pairs - 1) / pairs;
  const int64_t max_chunks = (m + 255) / 256;
  if (chunks > max_chunks) chunks = max_chunks;
  if (chunks < 1) chunks = 1;
  return (int)chunks;
}

size_t gram_ws(int64_t m, int l, int num_sms) {
  const int c = std::max(gram_chunks(m, l, num_sms, GRAM_T), gram_chunks(m, l, num_sms, 64));
  return sizeof(double) * (size_t)c * l * l;
}

// G (l x l FP64) = Y^T Y with the products and sums of `mode`.
// With `gate` (kGramF64 only), the kernels run only if *gate is nonzero (decided on the device).
int launch_gram(rmc_ctx *ctx, const float *Y, int64_t m, int l, int64_t ldy, double *G, double *part,
                GramMode mode, const int *gate = nullptr) {
  if (gate && mode != kGramF64) return RMC_EINVAL;
  const int tile = gram_tile(l, mode);
  const int T = (l + tile - 1) / tile;
  const int pairs = T * (T + 1) / 2;
  const int chunks = gram_chunks(m, l, ctx->num_sms, tile);
  int64_t rows = (m + chunks - 1) / chunks;
  rows = (rows + GRAM_T - 1) / GRAM_T * GRAM_T;
  const dim3 grid(pairs, chunks);
  cudaStream_t st = ctx->stream;
  {
    RmcProf prof(ctx, RMC_K_GRAM);
    if (mode == kGramF64) gram_f64_kernel<<<grid, 256, 0, st>>>(Y, m, l, ldy, rows, part, gate);
    else if (mode == kGramExact && tile == 64) gram_tile_kernel<64, true><<<grid, 256, 0, st>>>(Y, m, l, ldy, rows, part);
    else if (mode == kGramExact) gram_tile_kernel<32, true><<<grid, 256, 0, st>>>(Y, m, l, ldy, rows, part);
    else if (tile == 64) gram_tile_kernel<64, false><<<grid, 256, 0, st>>>(Y, m, l, ldy, rows, part);
    else gram_tile_kernel<32, false><<<grid, 256, 0, st>>>(Y, m, l, ldy, rows, part);
  }
  rmc_note_launch(2);
  gram_reduce_kernel<<<rmc_blocks((int64_t)l * l, 256, 1024), 256, 0, st>>>(part, chunks, l, tile, G, gate);
  RMC_LAUNCH_CHECK();
  return RMC_OK;
}

int launch_rowblock(cudaStream_t st, const float *in, int64_t m, int li, int64_t ldi, const float *M, int lo,
                    int64_t ldm, float *out, int64_t ldo, bool subtract = false) {
  if (li >= 1 && li <= 128 && lo <= 128) {
    const size_t smem2 = sizeof(float) * ((size_t)li * RB2_LD + (size_t)li * 128);
    if (smem2 > 48 * 1024) {
      RMC_TRY_CUDA(rmc_allow_smem(rowblock_tile_kernel<false>, smem2));
      RMC_TRY_CUDA(rmc_allow_smem(rowblock_tile_kernel<true>, smem2));
    }
    if (subtract)
      rowblock_tile_kernel<true><<<rmc_blocks(m, RB2), 256, smem2, st>>>(in, m, li, ldi, M, lo, ldm, out, ldo);
    else
      rowblock_tile_kernel<false><<<rmc_blocks(m, RB2), 256, smem2, st>>>(in, m, li, ldi, M, lo, ldm, out, ldo);
    rmc_note_launch();
    RMC_LAUNCH_CHECK();
    return RMC_OK;
  }
  const size_t smem = sizeof(float) * RB * li;
  if (smem > 48 * 1024) {
    RMC_TRY_CUDA(rmc_allow_smem(rowblock_mul_kernel<false>, smem));
    RMC_TRY_CUDA(rmc_allow_smem(rowblock_mul_kernel<true>, smem));
  }
  if (subtract) rowblock_mul_kernel<true><<<rmc_blocks(m, RB), 256, smem, st>>>(in, m, li, ldi, M, lo, ldm, out, ldo);
  else rowblock_mul_kernel<false><<<rmc_blocks(m, RB), 256, smem, st>>>(in, m, li, ldi, M, lo, ldm, out, ldo);
  rmc_note_launch();
  RMC_LAUNCH_CHECK();
  return RMC_OK;
}

}  // namespace

int rmc_launch_rowblock(cudaStream_t st, const float *in, int64_t m, int li, int64_t ldi, const float *M, int lo,
                        int64_t ldm, float *out, int64_t ldo, bool subtract) {
  return launch_rowblock(st, in, m, li, ldi, M, lo, ldm, out, ldo, subtract);
}

// ------------------------------------------------------------------------------------------- matmuls

static int matmul_at_splits(int64_t m, int64_t n, int64_t l, int num_sms) {
  const int64_t tiles = ((l + GT - 1) / GT) * ((n + GT - 1) / GT);
  int64_t splits = (2 * (int64_t)num_sms + tiles - 1) / tiles;
  const int64_t max_splits = (m + 1023) / 1024;
  if (splits > max_splits) splits = max_splits;
  if (splits < 1) splits = 1;
  return (int)splits;
}

int rmc_tc_matmul_an(rmc_ctx *ctx, const float *A, int64_t m, int64_t n, int64_t lda, const float *X, int64_t l,
                     int64_t ldx, float *Y, int64_t ldy, bool x3, void *ws);
int rmc_tc_matmul_at(rmc_ctx *ctx, const float *A, int64_t m, int64_t n, int64_t lda, const float *X, int64_t l,
                     int64_t ldx, float *W, int64_t ldw, bool x3, void *ws);
size_t rmc_tc_matmul_ws(int64_t m, int64_t n, int64_t l, int which, bool x3, int num_sms);
int rmc_tc_matmul_an_bf16(rmc_ctx *ctx, const float *A, int64_t m, int64_t n, int64_t lda, const float *X, int64_t l,
                          int64_t ldx, float *Y, int64_t ldy, void *ws);
int rmc_tc_matmul_at_bf16(rmc_ctx *ctx, const float *A, int64_t m, int64_t n, int64_t lda, const float *X, int64_t l,
                          int64_t ldx, float *W, int64_t ldw, void *ws);
size_t rmc_tc_matmul_bf16_ws(int64_t m, int64_t n, int64_t l, int which, int num_sms);

size_t rmc_matmul_ws(int64_t m, int64_t n, int64_t l, int which, int prec, int num_sms) {
  size_t simt = 0;
  if (which == 1) {
    const int splits = matmul_at_splits(m, n, l, num_sms);
    simt = splits > 1 ? sizeof(float) * (size_t)splits * l * n : 0;
  }
  size_t tc = 0;
  if (prec == RMC_TF32 || prec == RMC_TF32X3) tc = rmc_tc_matmul_ws(m, n, l, which, prec == RMC_TF32X3, num_sms);
  else if (prec == RMC_BF16) tc = rmc_tc_matmul_bf16_ws(m, n, l, which, num_sms);
  return tc > simt ? tc : simt;
}

// The tensor-core products stream A with TMA (16-byte aligned rows); other layouts take the FP32 kernels.
static bool tma_rows_ok(const float *A, int64_t lda) {
  return (lda % 4 == 0) && (reinterpret_cast<uintptr_t>(A) % 16 == 0);
}

int rmc_launch_matmul_an(rmc_ctx *ctx, const float *A, int64_t m, int64_t n, int64_t lda, const float *X, int64_t l,
                         int64_t ldx, int prec, float *Y, int64_t ldy, void *ws) {
  if ((prec == RMC_TF32 || prec == RMC_TF32X3) && tma_rows_ok(A, lda))
    return rmc_tc_matmul_an(ctx, A, m, n, lda, X, l, ldx, Y, ldy, prec == RMC_TF32X3, ws);
  if (prec == RMC_BF16 && tma_rows_ok(A, lda)) return rmc_tc_matmul_an_bf16(ctx, A, m, n, lda, X, l, ldx, Y, ldy, ws);
  dim3 grid((unsigned)((l + GT - 1) / GT), (unsigned)((m + GT - 1) / GT));
  {
    RmcProf prof(ctx, RMC_K_MATMUL_AN);
    matmul_an_kernel<<<grid, 256, 0, ctx->stream>>>(A, m, n, lda, X, l, ldx, Y, ldy);
  }
  rmc_note_launch();
  RMC_LAUNCH_CHECK();
  return RMC_OK;
}

int rmc_launch_matmul_at(rmc_ctx *ctx, const float *A, int64_t m, int64_t n, int64_t lda, const float *X, int64_t l,
                         int64_t ldx, int prec, float *W, int64_t ldw, void *ws) {
  if ((prec == RMC_TF32 || prec == RMC_TF32X3) && tma_rows_ok(A, lda))
    return rmc_tc_matmul_at(ctx, A, m, n, lda, X, l, ldx, W, ldw, prec == RMC_TF32X3, ws);
  if (prec == RMC_BF16 && tma_rows_ok(A, lda)) return rmc_tc_matmul_at_bf16(ctx, A, m, n, lda, X, l, ldx, W, ldw, ws);
  const int splits = matmul_at_splits(m, n, l, ctx->num_sms);
  int64_t rows = (m + splits - 1) / splits;
  rows = (rows + GK - 1) / GK * GK;
  dim3 grid((unsigned)((n + GT - 1) / GT), (unsigned)((l + GT - 1) / GT), (unsigned)splits);
  if (splits == 1) {
    RmcProf prof(ctx, RMC_K_MATMUL_AT);
    matmul_at_kernel<<<grid, 256, 0, ctx->stream>>>(A, m, n, lda, X, l, ldx, rows, W, ldw, 0);
    rmc_note_launch();
  } else {
    float *part = static_cast<float *>(ws);
    {
      RmcProf prof(ctx, RMC_K_MATMUL_AT);
      matmul_at_kernel<<<grid, 256, 0, ctx->stream>>>(A, m, n, lda, X, l, ldx, rows, part, n, l * n);
    }
    rmc_note_launch(2);
    sum_splits_kernel<<<rmc_blocks(l * n, 256, 4096), 256, 0, ctx->stream>>>(part, splits, l, n, W, ldw);
  }
  RMC_LAUNCH_CHECK();
  return RMC_OK;
}

int rmc_launch_transpose(cudaStream_t st, const float *in, int64_t rows, int64_t cols, int64_t ldi, float *out,
                         int64_t ldo) {
  dim3 grid((unsigned)((cols + 31) / 32), (unsigned)((rows + 31) / 32));
  transpose_kernel<<<grid, dim3(32, 8), 0, st>>>(in, rows, cols, ldi, out, ldo);
  rmc_note_launch();
  RMC_LAUNCH_CHECK();
  return RMC_OK;
}

// ------------------------------------------------------------------------------------------ CholeskyQR2

// Upper factor of the FP64 Gram matrix G (l x l, overwritten by R in FP64) and R^-1 in FP32: FP32 Cholesky in
// shared memory first; only if it meets a non-positive pivot (or the matrix is too large for shared memory)
// does the FP64 factorization run (its kernels return at once otherwise), with no host round trip.
// fail[0]: the FP32 path failed; fail[1]: the FP64 path failed.
// refresh (optional): the basis whose Gram matrix G is, with the partials buffer; when G was formed with FP32
// products and the FP32 factorization fails, G is formed again with FP64 products (exact for FP32 data) before
// the FP64 factorization, so that a basis whose condition number squared is beyond FP32 but within FP64 (e.g.
// A Omega with a square, ill-conditioned Gaussian Omega) still factors.  The refresh runs only when the FP32
// path failed (decided on the device).
struct GramRefresh {
  const float *Y;
  int64_t m, ldy;
  double *part;
};

static int launch_factor(rmc_ctx *ctx, double *G, int l, double *Rinv, float *Rinv32, int *fail,
                         const GramRefresh *refresh = nullptr) {
  cudaStream_t st = ctx->stream;
  const size_t smem = chol32_smem_bytes(l);
  RmcProf prof(ctx, RMC_K_SMALL);
  if (smem > kMaxPackedBytes || ctx->small_fp64) {
    force_fp64_kernel<<<1, 1, 0, st>>>(&fail[0]);
  } else if (l <= kCholFusedMaxL) {
    const size_t smem_f = chol32_fused_smem_bytes(l);
    if (smem_f > 48 * 1024)
      RMC_TRY_CUDA(rmc_allow_smem(chol32_fused_kernel, smem_f));
    chol32_fused_kernel<<<1, kCholFusedThreads, smem_f, st>>>(G, l, Rinv32, fail);
  } else {
    const size_t smem_x = smem + sizeof(float) * (size_t)l * l;
    if (smem_x <= kMaxPackedBytes) {
      if (smem_x > 48 * 1024)
        RMC_TRY_CUDA(rmc_allow_smem(chol32_inv_kernel<true>, smem_x));
      chol32_inv_kernel<true><<<1, 512, smem_x, st>>>(G, l, Rinv32, fail);
    } else {
      if (smem > 48 * 1024)
        RMC_TRY_CUDA(rmc_allow_smem(chol32_inv_kernel<false>, smem));
      chol32_inv_kernel<false><<<1, 512, smem, st>>>(G, l, Rinv32, fail);
    }
  }
  RMC_TRY_CUDA(cudaMemsetAsync(&fail[1], 0, sizeof(int), st));
  if (refresh) RMC_TRY(launch_gram(ctx, refresh->Y, refresh->m, l, refresh->ldy, G, refresh->part, kGramF64, &fail[0]));
  chol64_fallback_kernel<<<1, 1024, 0, st>>>(G, l, &fail[0], ctx->d_status, &fail[1]);
  tri_inverse_cols_kernel<<<l, 32, sizeof(double) * l, st>>>(G, l, Rinv, Rinv32, &fail[0], &fail[1]);
  rmc_note_launch(3);
  RMC_LAUNCH_CHECK();
  return RMC_OK;
}

size_t rmc_cholqr2_ws(int64_t m, int64_t l, int num_sms) {
  WsCarve w;
  w.take<double>(l * l);        // G
  w.take<double>(l * l);        // Rinv
  w.take<float>(l * l);         // Rinv32
  w.take<double>(l * l);        // R1
  w.take<int>(4);
  w.take<char>(gram_ws(m, (int)l, num_sms));
  return w.off;
}

int rmc_launch_cholqr2(rmc_ctx *ctx, float *Y, int64_t m, int64_t l_, int64_t ldy, double *R, void *ws,
                       int passes, bool fp64_gram) {
  const int l = (int)l_;
  cudaStream_t st = ctx->stream;
  WsCarve w;
  w.base = static_cast<char *>(ws);
  double *G = w.take<double>(l * l);
  double *Rinv = w.take<double>(l * l);
  float *Rinv32 = w.take<float>(l * l);
  double *R1 = w.take<double>(l * l);
  int *fail = w.take<int>(4);
  double *part = reinterpret_cast<double *>(w.take<char>(gram_ws(m, l, ctx->num_sms)));
  for (int pass = 0; pass < passes; ++pass) {
    // FP64 products (fp64_gram) only where they decide the result: the last pass.  An earlier pass only needs a
    // well-conditioned basis, which the FP32 products (summed in FP64) give; R = R2 R1 is exact up to the FP32
    // storage of the intermediate basis either way.
    const GramMode mode = ctx->small_fp64 ? kGramF64 : (fp64_gram && pass == passes - 1) ? kGramExact : kGramF32;
    RMC_TRY(launch_gram(ctx, Y, m, l, ldy, G, part, mode));
    const GramRefresh refresh{Y, m, ldy, part};
    RMC_TRY(launch_factor(ctx, G, l, Rinv, Rinv32, fail, mode == kGramF64 ? nullptr : &refresh));
    RMC_TRY(launch_rowblock(st, Y, m, l, ldy, Rinv32, l, l, Y, ldy));
    if (R) {
      if (pass == 0) RMC_TRY_CUDA(cudaMemcpyAsync(R1, G, sizeof(double) * l * l, cudaMemcpyDeviceToDevice, st));
      else {
        tri_mul_kernel<<<l, 128, 0, st>>>(G, R1, l, R);
        rmc_note_launch();
      }
    }
  }
  RMC_LAUNCH_CHECK();
  return RMC_OK;
}

// ------------------------------------------------------------------------------------------- small SVD

static bool jacobi_in_fp64(int l) { return l <= 32; }

// The eight-lanes-per-pair Jacobi keeps W (l x l) in shared memory: FP32 up to l = 240, FP64 up to l = 120.
static bool jacobi_grp_fits(int l, bool fp64) {
  return (size_t)l * l * (fp64 ? sizeof(double) : sizeof(float)) + 64 <= 227 * 1024;
}

// FP32 Jacobi of the column-major l x l W (l <= 128) with the vectorised kernel.
static int launch_jacobi_oe(cudaStream_t st, float *W, int l, float tol, int *status) {
  const int nv = (l + 31) / 32;
  const size_t smem = sizeof(float) * 32 * nv * (size_t)((l + 1) & ~1);   // one slot per position
  // eight lanes per column pair, rounded up to whole warps (the kernel's shuffles name every lane of a warp)
  const unsigned threads = (unsigned)((((l + 1) & ~1) / 2 * 8 + 31) / 32 * 32);
  switch (nv) {
#define RMC_JV(NV)                                                                                            \
  case NV:                                                                                                    \
    if (smem > 48 * 1024)                                                                                     \
      RMC_TRY_CUDA(rmc_allow_smem(jacobi_oe_kernel<NV>, smem));                                               \
    jacobi_oe_kernel<NV><<<1, threads, smem, st>>>(W, l, tol, 60, status);                                    \
    break;
    RMC_JV(1)
    RMC_JV(2)
    RMC_JV(3)
    RMC_JV(4)
#undef RMC_JV
    default:
      return RMC_EINVAL;
  }
  return RMC_OK;
}

// R (FP64 row-major) -> W = R^T column-major in FP32, i.e. the same entries in the same order.
__global__ void rows_as_cols_kernel(const double *R, int l, float *W) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < l * l; e += gridDim.x * blockDim.x) W[e] = (float)R[e];
}

// Left singular vectors of R from its right ones: R = M diag(sigma) N^T gives M = R N diag(sigma)^-1, M[:, c] =
// R N[:, c] / sigma_c in FP64 with R upper triangular (one block per column c; the counterpart of
// jacobi_right_kernel).
__global__ void jacobi_left_from_right_kernel(const double *R, int l, const float *N, const float *sigma,
                                              float *M) {
  const int c = blockIdx.x;
  const double inv = sigma[c] > 0.f ? 1.0 / (double)sigma[c] : 0.0;
  for (int r = threadIdx.x; r < l; r += blockDim.x) {
    double acc = 0.0;
    for (int i = r; i < l; ++i) acc += R[(int64_t)r * l + i] * (double)N[(int64_t)i * l + c];
    M[(int64_t)r * l + c] = (float)(acc * inv);
  }
}

// Jacobi on R (FP64 row-major upper, l x l) with the group kernel: M (left singular vectors of R, row-major) and
// sigma, descending.  fp64: rotations in FP64 (else FP32, FP64 below l = 33 as jacobi_in_fp64 says).
// With right != nullptr and the FP32 odd-even kernel (33 <= l <= 128), the rotations run on the columns of R^T
// (the rows of R), which for a triangular factor converge in fewer sweeps (nine against eleven on a 1/i spectrum
// at l = 120): their normalised columns are then R's right singular vectors, written to right, and M follows as
// R right diag(sigma)^-1; *right_done tells the caller which of the two it still has to form.
static int launch_jacobi_grp(rmc_ctx *ctx, const double *R, int l, double *work, float *M, float *sigma,
                             bool fp64, float *right = nullptr, bool *right_done = nullptr) {
  cudaStream_t st = ctx->stream;
  if (right_done) *right_done = false;
  if (fp64 || jacobi_in_fp64(l)) {
    const double tol = 8 * 2.220446049250313e-16 * sqrt((double)l);
    const size_t smem = sizeof(double) * (size_t)l * l;
    to_colmajor_kernel<double><<<rmc_blocks(l * l, 256), 256, 0, st>>>(R, l, work);
    if (l <= 128) {
      if (smem > 48 * 1024)
        RMC_TRY_CUDA(rmc_allow_smem(jacobi_grp_kernel<double, 16>, smem));
      jacobi_grp_kernel<double, 16><<<1, 1024, smem, st>>>(work, l, tol, 60, ctx->d_status);
    } else {
      if (smem > 48 * 1024)
        RMC_TRY_CUDA(rmc_allow_smem(jacobi_grp_kernel<double, 8>, smem));
      jacobi_grp_kernel<double, 8><<<1, 1024, smem, st>>>(work, l, tol, 60, ctx->d_status);
    }
    jacobi_left_kernel<double><<<1, 256, sizeof(double) * l, st>>>(work, l, M, sigma);
  } else {
    const float tol = 4 * 1.1920929e-7f * sqrtf((float)l);
    const size_t smem = sizeof(float) * (size_t)l * l;
    float *Wf = reinterpret_cast<float *>(work);
    if (l <= 128 && right) {
      rows_as_cols_kernel<<<rmc_blocks(l * l, 256), 256, 0, st>>>(R, l, Wf);
      RMC_TRY(launch_jacobi_oe(st, Wf, l, tol, ctx->d_status));
      jacobi_left_kernel<float><<<1, 256, sizeof(double) * l, st>>>(Wf, l, right, sigma);
      jacobi_left_from_right_kernel<<<l, 128, 0, st>>>(R, l, right, sigma, M);
      rmc_note_launch(4);
      RMC_LAUNCH_CHECK();
      *right_done = true;
      return RMC_OK;
    }
    to_colmajor_kernel<float><<<rmc_blocks(l * l, 256), 256, 0, st>>>(R, l, Wf);
    if (l <= 128) {
      RMC_TRY(launch_jacobi_oe(st, Wf, l, tol, ctx->d_status));
    } else {
      if (smem > 48 * 1024)
        RMC_TRY_CUDA(rmc_allow_smem(jacobi_grp_kernel<float, 8>, smem));
      jacobi_grp_kernel<float, 8><<<1, 1024, smem, st>>>(Wf, l, tol, 60, ctx->d_status);
    }
    jacobi_left_kernel<float><<<1, 256, sizeof(double) * l, st>>>(Wf, l, M, sigma);
  }
  rmc_note_launch(3);
  RMC_LAUNCH_CHECK();
  return RMC_OK;
}

size_t rmc_svd_wide_ws(int64_t l, int64_t n, int num_sms) {
  WsCarve w;
  w.take<float>(n * l);        // Bt -> Q2
  w.take<double>(l * l);       // R
  w.take<double>(l * l);       // W
  w.take<double>(l * l);       // V
  w.take<float>(l * l);        // M
  const size_t head = w.off;
  return head + 256 + rmc_cholqr2_ws(n, l, num_sms);
}

int rmc_launch_svd_wide(rmc_ctx *ctx, const float *B, int64_t l_, int64_t n, int64_t ldb, float *Ub, float *sigma,
                        float *Vb, int64_t ldv, void *ws) {
  const int l = (int)l_;
  cudaStream_t st = ctx->stream;
  WsCarve w;
  w.base = static_cast<char *>(ws);
  float *Bt = w.take<float>(n * l);
  double *R = w.take<double>(l * l);
  double *W = w.take<double>(l * l);
  double *V = w.take<double>(l * l);
  float *M = w.take<float>(l * l);
  void *rest = static_cast<char *>(ws) + ((w.off + 255) & ~size_t(255));
  RMC_TRY(rmc_launch_transpose(st, B, l, n, ldb, Bt, l));                    // B^T, n x l
  // the singular values come from R: its Gram matrices take FP64 products
  RMC_TRY(rmc_launch_cholqr2(ctx, Bt, n, l, l, R, rest, 2, true));           // B^T = Q2 R
  RmcProf prof(ctx, RMC_K_SMALL);
  if (jacobi_grp_fits(l, ctx->small_fp64)) {
    bool ub_done = false;
    RMC_TRY(launch_jacobi_grp(ctx, R, l, W, M, sigma, ctx->small_fp64, Ub, &ub_done));
    if (!ub_done) {
      jacobi_right_kernel<<<l, 128, 0, st>>>(R, l, M, sigma, Ub);              // Ub = R^T M diag(sigma)^-1
      rmc_note_launch();
    }
  } else {
    rmc_note_launch(3);
    const size_t smem64 = 2 * sizeof(double) * (size_t)l * l, smem32 = 2 * sizeof(float) * (size_t)l * l;
    if (jacobi_in_fp64(l)) {
      const double tol = 8 * 2.220446049250313e-16 * sqrt((double)l);
      to_colmajor_kernel<double><<<rmc_blocks(l * l, 256), 256, 0, st>>>(R, l, W);
      jacobi_smem_kernel<double><<<1, 1024, smem64, st>>>(W, V, l, tol, 60, ctx->d_status);
      jacobi_finish_kernel<double><<<1, 256, sizeof(double) * l, st>>>(W, V, l, Ub, M, sigma);
    } else {
      const float tol = 4 * 1.1920929e-7f * sqrtf((float)l);
      float *Wf = reinterpret_cast<float *>(W), *Vf = reinterpret_cast<float *>(V);
      to_colmajor_kernel<float><<<rmc_blocks(l * l, 256), 256, 0, st>>>(R, l, Wf);
      if (smem32 <= 200 * 1024) {
        if (smem32 > 48 * 1024)
          RMC_TRY_CUDA(rmc_allow_smem(jacobi_smem_kernel<float>, smem32));
        jacobi_smem_kernel<float><<<1, 1024, smem32, st>>>(Wf, Vf, l, tol, 60, ctx->d_status);
      } else {
        jacobi_kernel<float><<<1, 1024, 0, st>>>(Wf, Vf, l, tol, 60, ctx->d_status);
      }
      jacobi_finish_kernel<float><<<1, 256, sizeof(double) * l, st>>>(Wf, Vf, l, Ub, M, sigma);
    }
  }
  RMC_LAUNCH_CHECK();
  return launch_rowblock(st, Bt, n, l, l, M, l, l, Vb, ldv);                 // Vb = Q2 M
}

// SVD of a square l x l matrix by one-sided Jacobi on its columns, with no QR first (for symmetric PSD
// matrices whose condition number is beyond a Cholesky-based QR, e.g. the landmark block of a kernel matrix):
// W (row-major FP64) = Ml diag(sigma) Vr^T with Ml the left and Vr the right singular vectors (row-major FP32,
// columns ordered by descending sigma; Vr is written only on the path for l beyond the shared-memory group
// kernel).  FP64 rotations for l <= 32 or with RMC_OPT_SMALL_FP64, FP32 otherwise, as the small SVD of rmc_rsvd.
size_t rmc_jacobi_square_ws(int64_t l) { return 2 * sizeof(double) * (size_t)l * l + 256; }

int rmc_launch_jacobi_square(rmc_ctx *ctx, const double *Wrm, int l, float *Ml, float *sigma, float *Vr, void *ws) {
  cudaStream_t st = ctx->stream;
  double *W = static_cast<double *>(ws);
  double *V = W + (size_t)l * l;
  const size_t smem64 = 2 * sizeof(double) * (size_t)l * l, smem32 = 2 * sizeof(float) * (size_t)l * l;
  RmcProf prof(ctx, RMC_K_SMALL);
  if (jacobi_grp_fits(l, ctx->small_fp64)) return launch_jacobi_grp(ctx, Wrm, l, W, Ml, sigma, ctx->small_fp64);
  rmc_note_launch(3);
  if (jacobi_in_fp64(l)) {
    const double tol = 8 * 2.220446049250313e-16 * sqrt((double)l);
    to_colmajor_kernel<double><<<rmc_blocks(l * l, 256), 256, 0, st>>>(Wrm, l, W);
    jacobi_smem_kernel<double><<<1, 1024, smem64, st>>>(W, V, l, tol, 60, ctx->d_status);
    jacobi_finish_kernel<double><<<1, 256, sizeof(double) * l, st>>>(W, V, l, Vr, Ml, sigma);
  } else {
    const float tol = 4 * 1.1920929e-7f * sqrtf((float)l);
    float *Wf = reinterpret_cast<float *>(W), *Vf = Wf + (size_t)l * l;
    to_colmajor_kernel<float><<<rmc_blocks(l * l, 256), 256, 0, st>>>(Wrm, l, Wf);
    if (smem32 <= 200 * 1024) {
      if (smem32 > 48 * 1024)
        RMC_TRY_CUDA(rmc_allow_smem(jacobi_smem_kernel<float>, smem32));
      jacobi_smem_kernel<float><<<1, 1024, smem32, st>>>(Wf, Vf, l, tol, 60, ctx->d_status);
    } else {
      jacobi_kernel<float><<<1, 1024, 0, st>>>(Wf, Vf, l, tol, 60, ctx->d_status);
    }
    jacobi_finish_kernel<float><<<1, 256, sizeof(double) * l, st>>>(Wf, Vf, l, Vr, Ml, sigma);
  }
  RMC_LAUNCH_CHECK();
  return RMC_OK;
}

int rmc_launch_rsvd_finish(rmc_ctx *ctx, const float *Q, int64_t m, int64_t l, const float *Ub, const float *sg,
                           const float *Vb, int64_t n, int k, float *U, int64_t ldu, float *sigma, float *V,
                           int64_t ldv, void *ws) {
  float *Ms = static_cast<float *>(ws);  // Ub[:, :k] with the column signs applied, l x k
  sign_fix_kernel<<<k, 1024, 0, ctx->stream>>>(Vb, n, l, Ub, (int)l, k, Ms, V, ldv, sg, sigma);
  rmc_note_launch();
  RMC_LAUNCH_CHECK();
  return launch_rowblock(ctx->stream, Q, m, (int)l, l, Ms, k, k, U, ldu);
}

// ------------------------------------------------------------------------------------ least-squares solve

constexpr int kRefineSteps = 4;

static int atr_chunks(int64_t s) { return (int)std::min<int64_t>(64, std::max<int64_t>(1, s / 32)); }

struct LsrBufs {
  double *G, *xs, *r, *part, *gpart, *Gsq;
  float *Rf, *Dinv, *Ri, *M;
  int *flags;  // kLsrFlagWords words, see the refinement kernels
};

static LsrBufs lsr_carve(WsCarve &w, int64_t s, int64_t n, int num_sms) {
  LsrBufs b;
  const int l = (int)n + 1;
  const int64_t nb = (n + kPanel - 1) / kPanel;
  b.G = w.take<double>((size_t)l * l);
  b.flags = w.take<int>(kLsrFlagWords);
  b.xs = w.take<double>(n);
  b.r = w.take<double>(s);
  b.part = w.take<double>((size_t)atr_chunks(s) * n);
  b.Rf = w.take<float>((size_t)n * n);
  b.Dinv = w.take<float>((size_t)nb * kPanel * kPanel);
  b.Ri = w.take<float>((size_t)n * n);
  b.M = w.take<float>((size_t)n * n);
  b.Gsq = n <= kCholFusedMaxL ? w.take<double>((size_t)n * n) : nullptr;
  b.gpart = reinterpret_cast<double *>(w.take<char>(gram_ws(s, l, num_sms)));
  return b;
}

__global__ void lsr_gsq_init_kernel(const double *G, int ldg, int n, double *Gsq, int *flags) {
  if (blockIdx.x == 0 && threadIdx.x < kLsrFlagWords) flags[threadIdx.x] = 0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n * n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / n), j = (int)(e - (int64_t)i * n);
    Gsq[e] = G[(int64_t)i * ldg + j];
  }
}

// FP32 Cholesky factor R of the n x n Gram matrix in b.G (leading dimension ldg) and R^-1 in b.Ri (row-major,
// upper); b.flags are cleared first and flags[0] = 1 marks a breakdown.  n <= 128: the single-CTA fused kernel
// on a contiguous copy (two launches); larger n: 32-column panels, trailing updates and the blocked inverse.
static void launch_lsr_cholesky(cudaStream_t st, const LsrBufs &b, int ldg, int n) {
  if (n <= kCholFusedMaxL) {
    lsr_gsq_init_kernel<<<rmc_blocks((int64_t)n * n, 256, 1024), 256, 0, st>>>(b.G, ldg, n, b.Gsq, b.flags);
    chol32_fused_kernel<<<1, kCholFusedThreads, 0, st>>>(b.Gsq, n, b.Ri, &b.flags[0]);
    rmc_note_launch(2);
    return;
  }
  lsr_rf_init_kernel<<<rmc_blocks((int64_t)n * n, 256, 1024), 256, 0, st>>>(b.G, ldg, n, b.Rf, b.flags);
  rmc_note_launch();
  for (int j0 = 0; j0 < n; j0 += kPanel) {
    const int bw = std::min(kPanel, n - j0), rest = n - j0 - bw;
    lsr_chol_panel_kernel<<<std::max(1, (rest + 255) / 256), 256, 0, st>>>(b.Rf, n, j0, b.Dinv, &b.flags[0]);
    rmc_note_launch();
    if (rest > 0) {
      const int T = (rest + 63) / 64;
      lsr_chol_update_kernel<<<T * (T + 1) / 2, 256, 0, st>>>(b.Rf, n, j0, &b.flags[0]);
      rmc_note_launch();
    }
  }
  const int nb = (n + kPanel - 1) / kPanel;
  const size_t tri_smem = sizeof(float) * ((size_t)nb * kPanel * kPanel + kPanel * kPanel);
  lsr_tri_inv_kernel<<<nb, 1024, tri_smem, st>>>(b.Rf, b.Dinv, n, b.Ri, &b.flags[0]);
  rmc_note_launch();
}

size_t rmc_lsr_solve_ws(int64_t s, int64_t n, int num_sms) {
  WsCarve w;
  lsr_carve(w, s, n, num_sms);
  return w.off;
}

int rmc_launch_lsr_solve(rmc_ctx *ctx, const float *SA, int64_t s, int64_t n_, int64_t ldsa, const float *Sb,
                         double *x, void *ws) {
  // SA is s x (n+1) with ldsa >= n+1; column n receives Sb first.
  cudaStream_t st = ctx->stream;
  const int n = (int)n_, l = n + 1;
  WsCarve w;
  w.base = static_cast<char *>(ws);
  const LsrBufs b = lsr_carve(w, s, n, ctx->num_sms);
  copy_column_kernel<<<rmc_blocks(s, 256, 1024), 256, 0, st>>>(Sb, s, const_cast<float *>(SA), ldsa, n);
  rmc_note_launch();
  // FP32 products summed in FP64 across 32-row slices: the factor only preconditions the refinement
  RMC_TRY(launch_gram(ctx, SA, s, l, ldsa, b.G, b.gpart, kGramF32));
  {
    RmcProf prof(ctx, RMC_K_SMALL);
    const int nb = (n + kPanel - 1) / kPanel;
    const size_t tri_smem = sizeof(float) * ((size_t)nb * kPanel * kPanel + kPanel * kPanel);
    if (tri_smem > 48 * 1024)
      RMC_TRY_CUDA(rmc_allow_smem(lsr_tri_inv_kernel, tri_smem));
    launch_lsr_cholesky(st, b, l, n);
    // M = R^-1 R^-T
    const int T64 = (n + 63) / 64;
    lsr_inv_gram_kernel<<<T64 * (T64 + 1) / 2, 256, 0, st>>>(b.Ri, n, b.M, &b.flags[0]);
    rmc_note_launch();
    RMC_TRY_CUDA(cudaMemsetAsync(b.xs, 0, sizeof(double) * n, st));
    const int chunks = atr_chunks(s);
    const int64_t rows_per = (s + chunks - 1) / chunks;
    for (int it = 0; it < kRefineSteps; ++it) {
      lsr_resid_kernel<<<rmc_blocks(s * 32, 256, 4096), 256, 0, st>>>(SA, s, n, ldsa, b.xs, b.r, it, b.flags);
      lsr_atr_kernel<<<dim3((n + 255) / 256, chunks), 256, 0, st>>>(SA, s, n, ldsa, b.r, rows_per, b.part, it,
                                                                    b.flags);
      lsr_apply_kernel<<<nb, 256, sizeof(float) * n, st>>>(b.M, n, b.part, chunks, b.xs, it, b.flags);
      rmc_note_launch(3);
    }
    lsr_refine_finish_kernel<<<1, 256, 0, st>>>(b.xs, n, kRefineSteps - 1, x, b.flags);
    rmc_note_launch();
  }
  // FP64 path (every kernel returns at once unless flags[0] is set): FP64 Gram, FP64 Cholesky of the augmented
  // matrix, back substitution
  RMC_TRY(launch_gram(ctx, SA, s, l, ldsa, b.G, b.gpart, kGramF64, &b.flags[0]));
  {
    RmcProf prof(ctx, RMC_K_SMALL);
    chol64_fallback_kernel<<<1, 1024, 0, st>>>(b.G, l, &b.flags[0], ctx->d_status, &b.flags[1]);
    lsr_backsub_kernel<<<1, 32, sizeof(double) * n, st>>>(b.G, n, x, &b.flags[0], &b.flags[1]);
  }
  rmc_note_launch(2);
  RMC_LAUNCH_CHECK();
  return RMC_OK;
}

// --------------------------------------------------------------------- resident least squares (request server)
// The preconditioner of rmc_launch_lsr_solve computed from S^T A alone and kept by the caller, and the solve of
// one right-hand side against it: the server keeps S^T A and this factor resident between requests on the same
// matrix and sketch, so that a request only sketches its b and refines.

__global__ void lsr_flag_out_kernel(const int *flags, int *fail) { *fail = flags[0]; }

__global__ void lsr_flags_in_kernel(int *flags, const int *fail) {
  if (threadIdx.x < kLsrFlagWords) flags[threadIdx.x] = threadIdx.x == 0 ? *fail : 0;
}

// the solve's buffers, then the partials of the n x n Gram matrix (its tiling differs from the (n+1)-column one)
size_t rmc_lsr_factor_ws(int64_t s, int64_t n, int num_sms) {
  WsCarve w;
  lsr_carve(w, s, n, num_sms);
  w.take<char>(gram_ws(s, (int)n, num_sms));
  return w.off;
}

// M (n x n FP32) = R^-1 R^-T for the FP32 Cholesky factor R of (S^T A)^T (S^T A), S^T A (s x n, ldsa); *fail
// (device) = 1 where that factor broke down (the solves then take the FP64 path).
int rmc_launch_lsr_factor(rmc_ctx *ctx, const float *SA, int64_t s, int64_t n_, int64_t ldsa, float *M, int *fail,
                          void *ws) {
  cudaStream_t st = ctx->stream;
  const int n = (int)n_;
  WsCarve w;
  w.base = static_cast<char *>(ws);
  const LsrBufs b = lsr_carve(w, s, n, ctx->num_sms);
  double *gpart = reinterpret_cast<double *>(w.take<char>(gram_ws(s, n, ctx->num_sms)));
  RMC_TRY(launch_gram(ctx, SA, s, n, ldsa, b.G, gpart, kGramF32));
  {
    RmcProf prof(ctx, RMC_K_SMALL);
    const int nb = (n + kPanel - 1) / kPanel;
    const size_t tri_smem = sizeof(float) * ((size_t)nb * kPanel * kPanel + kPanel * kPanel);
    if (tri_smem > 48 * 1024)
      RMC_TRY_CUDA(rmc_allow_smem(lsr_tri_inv_kernel, tri_smem));
    launch_lsr_cholesky(st, b, n, n);
    const int T64 = (n + 63) / 64;
    lsr_inv_gram_kernel<<<T64 * (T64 + 1) / 2, 256, 0, st>>>(b.Ri, n, M, &b.flags[0]);
    lsr_flag_out_kernel<<<1, 1, 0, st>>>(b.flags, fail);
    rmc_note_launch(2);
  }
  RMC_LAUNCH_CHECK();
  return RMC_OK;
}

size_t rmc_lsr_refine_ws(int64_t s, int64_t n, int num_sms) { return rmc_lsr_solve_ws(s, n, num_sms); }

// x = argmin ||S^T A x - S^T b|| for SAb = [S^T A, S^T b] (s x (n+1), ldsab) with the factor of
// rmc_launch_lsr_factor: refinement with FP64 residuals preconditioned by M, and the FP64 Cholesky of the
// augmented Gram matrix where the factor failed or the refinement did not converge (as rmc_launch_lsr_solve).
int rmc_launch_lsr_refine(rmc_ctx *ctx, const float *SAb, int64_t s, int64_t n_, int64_t ldsab, const float *M,
                          const int *fail, double *x, void *ws) {
  cudaStream_t st = ctx->stream;
  const int n = (int)n_, l = n + 1;
  WsCarve w;
  w.base = static_cast<char *>(ws);
  const LsrBufs b = lsr_carve(w, s, n, ctx->num_sms);
  {
    RmcProf prof(ctx, RMC_K_SMALL);
    lsr_flags_in_kernel<<<1, 32, 0, st>>>(b.flags, fail);
    rmc_note_launch();
    RMC_TRY_CUDA(cudaMemsetAsync(b.xs, 0, sizeof(double) * n, st));
    const int nb = (n + kPanel - 1) / kPanel;
    const int chunks = atr_chunks(s);
    const int64_t rows_per = (s + chunks - 1) / chunks;
    for (int it = 0; it < kRefineSteps; ++it) {
      lsr_resid_kernel<<<rmc_blocks(s * 32, 256, 4096), 256, 0, st>>>(SAb, s, n, ldsab, b.xs, b.r, it, b.flags);
      lsr_atr_kernel<<<dim3((n + 255) / 256, chunks), 256, 0, st>>>(SAb, s, n, ldsab, b.r, rows_per, b.part, it,
                                                                    b.flags);
      lsr_apply_kernel<<<nb, 256, sizeof(float) * n, st>>>(M, n, b.part, chunks, b.xs, it, b.flags);
      rmc_note_launch(3);
    }
    lsr_refine_finish_kernel<<<1, 256, 0, st>>>(b.xs, n, kRefineSteps - 1, x, b.flags);
    rmc_note_launch();
  }
  RMC_TRY(launch_gram(ctx, SAb, s, l, ldsab, b.G, b.gpart, kGramF64, &b.flags[0]));
  {
    RmcProf prof(ctx, RMC_K_SMALL);
    chol64_fallback_kernel<<<1, 1024, 0, st>>>(b.G, l, &b.flags[0], ctx->d_status, &b.flags[1]);
    lsr_backsub_kernel<<<1, 32, sizeof(double) * n, st>>>(b.G, n, x, &b.flags[0], &b.flags[1]);
  }
  rmc_note_launch(2);
  RMC_LAUNCH_CHECK();
  return RMC_OK;
}
