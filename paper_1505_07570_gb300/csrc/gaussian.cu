// Gaussian projection (Sec. 3.2.1, row orientation): C = S^T A with S = G / sqrt(s), G (m x s) iid N(0, 1).
//
// G is never stored: every tile of G is drawn from Philox where the product needs it (the sketch stream, 4, of
// rmc.h: eight normals per Philox block from 16-bit uniforms).  The reduction runs over the m rows of A, so the work is split over row ranges (split-K) and the
// partial products are summed in a fixed order afterwards.
//   RMC_FP32: CUDA-core FMAs (the plain form), this file.
//   RMC_TF32: tcgen05 tensor-core kernel (tc_gemm.cu).
#include "rmc_internal.cuh"
#include "philox.cuh"

using namespace rmc;

namespace {

constexpr int TS = 64;    // sketch rows (columns of G) per tile
constexpr int TN = 128;   // columns of [A | b] per tile
constexpr int TK = 16;    // rows of A per step

__global__ void __launch_bounds__(256) gauss_simt_kernel(const float *__restrict__ A, int64_t m, int64_t n,
                                                         int64_t lda, const float *__restrict__ b, int64_t s,
                                                         uint64_t seed, uint32_t instance, int64_t rows_per_split,
                                                         float *__restrict__ part) {
  __shared__ __align__(16) float Os[TK][TS];
  __shared__ float As[TK][TN + 4];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t ntot = n + (b ? 1 : 0);
  const int64_t s0 = (int64_t)blockIdx.y * TS, c0 = (int64_t)blockIdx.x * TN;
  const int64_t r_begin = (int64_t)blockIdx.z * rows_per_split;
  const int64_t r_end = min(m, r_begin + rows_per_split);
  const int64_t groups = (s + 7) / 8;
  // Blocked summation: acc collects 16 steps (256 rows), then folds into tot, so no FP32 chain is longer than
  // 256 + rows / 256 terms (a split may span 2^18 rows of a 2^20-row matrix).
  float acc[4][8] = {}, tot[4][8] = {};
  int step = 0;
  for (int64_t k0 = r_begin; k0 < r_end; k0 += TK) {
    if (tid < TK * TS / 8) {  // G tile: one Philox block (8 normals) per thread of the first 128
      const int kk = tid >> 3, g = tid & 7;
      const int64_t row = k0 + kk;
      float z[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      if (row < r_end) gaussian8(seed, instance, (uint64_t)(row * groups + s0 / 8 + g), z);
      *reinterpret_cast<float4 *>(&Os[kk][8 * g]) = make_float4(z[0], z[1], z[2], z[3]);
      *reinterpret_cast<float4 *>(&Os[kk][8 * g + 4]) = make_float4(z[4], z[5], z[6], z[7]);
    }
    for (int e = tid; e < TK * TN; e += 256) {
      const int kk = e / TN, c = e % TN;
      const int64_t row = k0 + kk, col = c0 + c;
      float x = 0.f;
      if (row < r_end) {
        if (col < n) x = A[row * lda + col];
        else if (col == n && b) x = b[row];
      }
      As[kk][c] = x;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
      const float4 o = *reinterpret_cast<const float4 *>(&Os[kk][4 * ty]);
      const float g[4] = {o.x, o.y, o.z, o.w};
      float x[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) x[j] = As[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(g[i], x[j], acc[i][j]);
    }
    __syncthreads();
    if (++step == 16) {
      step = 0;
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          tot[i][j] += acc[i][j];
          acc[i][j] = 0.f;
        }
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) tot[i][j] += acc[i][j];
  float *o = part + (int64_t)blockIdx.z * s * ntot;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int64_t r = s0 + 4 * ty + i, c = c0 + tx + 16 * j;
      if (r < s && c < ntot) o[r * ntot + c] = tot[i][j];
    }
}

__global__ void gauss_reduce_kernel(const float *__restrict__ part, int splits, int64_t s, int64_t n, int64_t ntot,
                                    float scale, float *__restrict__ C, int64_t ldc, float *__restrict__ Cb) {
  const int64_t total = s * ntot;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    float acc = 0.f;
    for (int t = 0; t < splits; ++t) acc += part[t * total + e];
    const int64_t r = e / ntot, c = e - r * ntot;
    if (c < n) C[r * ldc + c] = acc * scale;
    else Cb[r] = acc * scale;
  }
}

int gauss_splits(int64_t m, int64_t ntot, int64_t s, int num_sms) {
  const int64_t tiles = ((s + TS - 1) / TS) * ((ntot + TN - 1) / TN);
  int64_t splits = (4 * (int64_t)num_sms + tiles - 1) / tiles;
  const int64_t max_splits = (m + 255) / 256;
  if (splits > max_splits) splits = max_splits;
  if (splits < 1) splits = 1;
  return (int)splits;
}

}  // namespace

size_t rmc_tc_gauss_ws(int64_t m, int64_t ntot, int64_t s, int prec, int num_sms);
int rmc_tc_gauss_sketch(rmc_ctx *ctx, const float *A, int64_t m, int64_t n, int64_t lda, const float *b, int64_t s,
                        uint64_t seed, uint32_t instance, int prec, float *C, int64_t ldc, float *Cb, void *ws);

size_t rmc_gauss_ws(int64_t m, int64_t ntot, int64_t s, int prec, int num_sms) {
  const size_t simt = sizeof(float) * (size_t)gauss_splits(m, ntot, s, num_sms) * s * ntot;
  if (prec == RMC_FP32) return simt;
  const size_t tc = rmc_tc_gauss_ws(m, ntot, s, prec, num_sms);
  return tc > simt ? tc : simt;   // rows that TMA cannot stream take the FP32 kernel
}

int rmc_launch_gauss_sketch(rmc_ctx *ctx, const float *A, int64_t m, int64_t n, int64_t lda, const float *b,
                            int64_t s, uint64_t seed, uint32_t instance, int prec, float *C, int64_t ldc, float *Cb,
                            void *ws) {
  // The tensor-core kernel streams A with TMA, which needs 16-byte aligned rows; other layouts take the FP32
  // CUDA-core kernel (same operator, FP32 operands).
  const bool tma_ok = (lda % 4 == 0) && (reinterpret_cast<uintptr_t>(A) % 16 == 0);
  if (prec != RMC_FP32 && tma_ok)
    return rmc_tc_gauss_sketch(ctx, A, m, n, lda, b, s, seed, instance, prec, C, ldc, Cb, ws);
  const int64_t ntot = n + (b ? 1 : 0);
  const int splits = gauss_splits(m, ntot, s, ctx->num_sms);
  int64_t rows = (m + splits - 1) / splits;
  rows = (rows + TK - 1) / TK * TK;
  float *part = static_cast<float *>(ws);
  dim3 grid((unsigned)((ntot + TN - 1) / TN), (unsigned)((s + TS - 1) / TS), (unsigned)splits);
  {
    RmcProf prof(ctx, RMC_K_GAUSSIAN);
    gauss_simt_kernel<<<grid, 256, 0, ctx->stream>>>(A, m, n, lda, b, s, seed, instance, rows, part);
  }
  rmc_note_launch(2);
  gauss_reduce_kernel<<<rmc_blocks(s * ntot, 256, 8192), 256, 0, ctx->stream>>>(
      part, splits, s, n, ntot, 1.0f / sqrtf((float)s), C, ldc, Cb);
  RMC_LAUNCH_CHECK();
  return RMC_OK;
}
