// The Nystrom method on the Gaussian RBF kernel (Sec. 6.1 kernel, Sec. 6.4 method and listing):
//
//   S = sort(randsample(n, s))  (the s landmarks: the SRHT sample rule over [0, n), Philox stream 3);
//   C = K(:, S) with K_ij = exp(-||x_i - x_j||^2 / (2 sigma^2))       (n x s, the only part of K formed);
//   W = C(S, :) = U_W diag(lam) U_W^T                                  (one-sided Jacobi on W, no QR first);
//   L = C U_W[:, :k] diag(lam[:k])^-1/2                                (n x k, K ~ L L^T = C W_k^+ C^T).
//
// The kernel tile computes ||x_i - x_j||^2 as a sum of squared differences (not |x|^2 + |y|^2 - 2 x.y), so
// nearby points keep their accuracy; the points are staged in shared memory 64 x 16 at a time.
#include <cmath>

#include "rmc_internal.cuh"

namespace {

constexpr int kT = 64;     // points per tile edge
constexpr int kD = 16;     // coordinates per step

// C[i, j] = exp(-||X_i - Y_j||^2 * inv2s2) for i < n1, j < n2: 256 threads, 4 x 4 outputs each.
__global__ void __launch_bounds__(256) rbf_kernel(const float *__restrict__ X, int64_t n1, int64_t ldx,
                                                  const float *__restrict__ Y, int64_t n2, int64_t ldy, int64_t d,
                                                  float inv2s2, float *__restrict__ C, int64_t ldc) {
  __shared__ float Xs[kD][kT + 1];
  __shared__ float Ys[kD][kT + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int64_t i0 = (int64_t)blockIdx.x * kT, j0 = (int64_t)blockIdx.y * kT;
  float acc[4][4] = {};
  for (int64_t c0 = 0; c0 < d; c0 += kD) {
    for (int e = threadIdx.x; e < kT * kD; e += 256) {
      const int r = e / kD, c = e % kD;
      Xs[c][r] = (i0 + r < n1 && c0 + c < d) ? X[(i0 + r) * ldx + c0 + c] : 0.f;
      Ys[c][r] = (j0 + r < n2 && c0 + c < d) ? Y[(j0 + r) * ldy + c0 + c] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < kD; ++c) {
      float x[4], y[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        x[u] = Xs[c][ty + 16 * u];
        y[u] = Ys[c][tx + 16 * u];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const float df = x[u] - y[v];
          acc[u][v] = fmaf(df, df, acc[u][v]);
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int64_t i = i0 + ty + 16 * u, j = j0 + tx + 16 * v;
      if (i < n1 && j < n2) C[i * ldc + j] = expf(-acc[u][v] * inv2s2);
    }
}

// Rows idx[0..s) of X (n x d) into Xs (s x d, row stride d).
__global__ void gather_rows_kernel(const float *X, int64_t ldx, int64_t d, const int64_t *idx, int64_t s, float *Xs,
                                   int64_t ldo) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < s * d; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / d, c = e % d;
    Xs[r * ldo + c] = X[idx[r] * ldx + c];
  }
}

// W (s x s, FP64 row-major) = C(S, :) from the n x s FP32 C.
__global__ void landmark_block_kernel(const float *C, int64_t ldc, const int64_t *idx, int s, double *W) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < s * s; e += gridDim.x * blockDim.x) {
    const int r = e / s, c = e % s;
    W[e] = (double)C[idx[r] * ldc + c];
  }
}

// Mk (s x k) = U_W[:, :k] diag(lam)^-1/2 with each column signed so its largest-magnitude entry (first on ties)
// is positive; lam[:k] copied out.  One warp per column.  A non-positive eigenvalue among the k kept means W_k
// is not positive definite (the landmarks repeat a point, or sigma is far too small): RMC_ENUMERIC.
__global__ void nystrom_scale_kernel(const float *U, int s, const float *sg, int k, float *Mk, float *lam_out,
                                     int *status) {
  const int j = blockIdx.x, lane = threadIdx.x;
  float best = -1.f;
  int at = 0;
  for (int r = lane; r < s; r += 32) {
    const float a = fabsf(U[r * s + j]);
    if (a > best) {
      best = a;
      at = r;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float b2 = __shfl_xor_sync(0xffffffffu, best, o);
    const int a2 = __shfl_xor_sync(0xffffffffu, at, o);
    if (b2 > best || (b2 == best && a2 < at)) {
      best = b2;
      at = a2;
    }
  }
  const float lam = sg[j];
  if (lane == 0) {
    if (!(lam > 0.f)) rmc_report(status, RMC_ENUMERIC);
    if (lam_out) lam_out[j] = lam;
  }
  const float scale = (U[at * s + j] < 0.f ? -1.f : 1.f) * rsqrtf(lam);
  for (int r = lane; r < s; r += 32) Mk[r * k + j] = U[r * s + j] * scale;
}

struct NysBufs {
  int64_t *idx;
  float *Xs, *C, *Ml, *sg, *Vr, *Mk;
  double *W;
  void *rest;
};

NysBufs nys_carve(WsCarve &w, int64_t n, int64_t d, int64_t s, int k, size_t rest) {
  NysBufs b;
  b.idx = w.take<int64_t>(s);
  b.Xs = w.take<float>((size_t)s * d);
  b.C = w.take<float>((size_t)n * s);
  b.W = w.take<double>((size_t)s * s);
  b.Ml = w.take<float>((size_t)s * s);
  b.sg = w.take<float>(s);
  b.Vr = w.take<float>((size_t)s * s);
  b.Mk = w.take<float>((size_t)s * k);
  b.rest = w.take<char>(rest);
  return b;
}

}  // namespace

int rmc_launch_rbf(rmc_ctx *ctx, const float *X, int64_t n1, int64_t ldx, const float *Y, int64_t n2, int64_t ldy,
                   int64_t d, double sigma, float *C, int64_t ldc) {
  dim3 grid((unsigned)((n1 + kT - 1) / kT), (unsigned)((n2 + kT - 1) / kT));
  if (grid.y > 65535u) return RMC_EINVAL;
  {
    RmcProf prof(ctx, RMC_K_RBF);
    rbf_kernel<<<grid, 256, 0, ctx->stream>>>(X, n1, ldx, Y, n2, ldy, d, (float)(0.5 / (sigma * sigma)), C, ldc);
  }
  rmc_note_launch();
  RMC_LAUNCH_CHECK();
  return RMC_OK;
}

extern "C" int rmc_rbf(rmc_ctx *ctx, const float *X, int64_t n1, int64_t ldx, const float *Y, int64_t n2,
                       int64_t ldy, int64_t d, double sigma, float *K, int64_t ldk) {
  if (!ctx || !X || !Y || !K || n1 < 1 || n2 < 1 || d < 1 || ldx < d || ldy < d || ldk < n2 || !(sigma > 0.0))
    return RMC_EINVAL;
  return rmc_launch_rbf(ctx, X, n1, ldx, Y, n2, ldy, d, sigma, K, ldk);
}

extern "C" int rmc_nystrom(rmc_ctx *ctx, const float *X, int64_t n, int64_t d, int64_t ldx, double sigma, int64_t s,
                           int k, uint64_t seed, float *L, int64_t ldl, float *lam, int64_t *landmarks) {
  if (!ctx || !X || !L || n < 1 || d < 1 || ldx < d || !(sigma > 0.0) || s < 1 || s > 256 || s > n) return RMC_EINVAL;
  if (k == 0) k = (int)std::ceil(0.8 * (double)s);
  if (k < 1 || k > s || ldl < k || n > (int64_t(1) << 31)) return RMC_EINVAL;
  size_t rest = rmc_srht_sample_ws(n);
  if (rmc_jacobi_square_ws(s) > rest) rest = rmc_jacobi_square_ws(s);
  WsCarve plan;
  nys_carve(plan, n, d, s, k, rest);
  RMC_TRY(rmc_ws_reserve(ctx, plan.off));
  WsCarve w;
  w.base = static_cast<char *>(ctx->ws);
  const NysBufs b = nys_carve(w, n, d, s, k, rest);
  cudaStream_t st = ctx->stream;
  RMC_TRY(rmc_launch_srht_sample(ctx, seed, 0, n, s, b.idx, b.rest));                   // S, ascending
  gather_rows_kernel<<<rmc_blocks(s * d, 256, 1024), 256, 0, st>>>(X, ldx, d, b.idx, s, b.Xs, d);
  rmc_note_launch();
  RMC_TRY(rmc_launch_rbf(ctx, X, n, ldx, b.Xs, s, d, d, sigma, b.C, s));                // C = K(:, S)
  landmark_block_kernel<<<rmc_blocks(s * s, 256, 256), 256, 0, st>>>(b.C, s, b.idx, (int)s, b.W);
  rmc_note_launch();
  RMC_TRY(rmc_launch_jacobi_square(ctx, b.W, (int)s, b.Ml, b.sg, b.Vr, b.rest));        // W = U diag(lam) U^T
  nystrom_scale_kernel<<<k, 32, 0, st>>>(b.Ml, (int)s, b.sg, k, b.Mk, lam, ctx->d_status);
  rmc_note_launch();
  RMC_LAUNCH_CHECK();
  if (landmarks) RMC_TRY_CUDA(cudaMemcpyAsync(landmarks, b.idx, sizeof(int64_t) * s, cudaMemcpyDeviceToDevice, st));
  return rmc_launch_rowblock(st, b.C, n, (int)s, s, b.Mk, k, k, L, ldl);                 // L = C Mk
}
