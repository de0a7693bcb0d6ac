// Machine-precision least squares by sketch preconditioning (Algorithm 4.1, Sec. 4.3):
//
//   Y = S^T A and S^T b from one sketch of [A, b];  Y = Q_Y R_Y (CholeskyQR2);  T = R_Y^-1 (FP64);
//   z = Q_Y^T (S^T b);   repeat:  r = b - A (T z);  z += theta T^T (A^T r);   x = T z.
//
// A T is never formed (the remark that closes Sec. 4.3): each step is one pass over A that computes, row by
// row, r_i = b_i - A_i v with v = T z, and accumulates A_i^T r_i from the same registers, so A is read once per
// step.  The residual is where the accuracy goes: b - A v cancels to a few parts in a thousand of |A_i| |v| on a
// well-fitted problem, so the row dot product is a compensated one (Ogita, Rump and Oishi, "Accurate sum and
// dot product", SIAM J. Sci. Comput. 2005, algorithm Dot2: Dekker's error-free product through an FMA and
// Knuth's error-free sum), as accurate as a dot product in twice FP32's precision, with v split into an FP32
// head and tail.  The gradient A^T r takes plain FP32 products (their rounding is relative to the gradient, which
// goes to zero) summed in FP32 within a warp's rows and in FP64 across warps and blocks, in a fixed order.
// The small n x n steps (T^T g, T z) run in FP64.
#include <cmath>

#include "rmc_internal.cuh"

namespace {

constexpr int kPassThreads = 256;           // 8 warps, one row per warp at a time
constexpr int kMaxN = 256;                  // columns: 8 per lane (two float4)

// ------------------------------------------------------------------------------ error-free transformations
// a + b = s + e exactly (Knuth's TwoSum, no branch, any magnitudes).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  const float z = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z));
}

// (s, c) += a * x in the manner of Dot2: the product's rounding error comes from an FMA, the sum's from TwoSum,
// and both go into the compensation c.
__device__ __forceinline__ void dot2_step(float a, float x, float &s, float &c) {
  const float p = __fmul_rn(a, x);
  const float pe = __fmaf_rn(a, x, -p);
  float t, te;
  two_sum(s, p, t, te);
  s = t;
  c = __fadd_rn(c, __fadd_rn(pe, te));
}

// Warp sum of (s, c) pairs with TwoSum at every level; returns s + c (all lanes).
__device__ __forceinline__ void warp_dot2_reduce(float &s, float &c) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float s2 = __shfl_xor_sync(0xffffffffu, s, o);
    const float c2 = __shfl_xor_sync(0xffffffffu, c, o);
    float t, te;
    two_sum(s, s2, t, te);
    s = t;
    c = __fadd_rn(c, __fadd_rn(c2, te));
  }
}

struct PassArgs {
  const float *A;
  int64_t m, lda;
  int n;
  const float *b;
  const float *vh, *vl;     // v = T z split into an FP32 head and tail (n entries each)
  double *part;             // [gridDim.x][n] FP64 partial gradients
  const int *done;          // non-zero: the iteration has converged, nothing to do
};

// One step's pass over A: every warp takes rows warp_id, warp_id + W, ...; lane l owns the columns
// 4 l .. 4 l + 3 and 128 + 4 l .. 128 + 4 l + 3 (VEC: two float4 loads per row) or l + 32 j (scalar loads).
// The next row is loaded while the current one is reduced.
template <bool VEC>
__global__ void __launch_bounds__(kPassThreads) lsrp_pass_kernel(PassArgs a) {
  if (*a.done) return;
  __shared__ float red[kPassThreads / 32][kMaxN];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t warps = (int64_t)gridDim.x * (kPassThreads / 32);
  const int64_t w0 = (int64_t)blockIdx.x * (kPassThreads / 32) + wib;
  const int n = a.n;

  auto col = [&](int j) -> int { return VEC ? 4 * lane + 128 * (j >> 2) + (j & 3) : lane + 32 * j; };
  float vh[8], vl[8], g[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int c = col(j);
    vh[j] = c < n ? a.vh[c] : 0.f;
    vl[j] = c < n ? a.vl[c] : 0.f;
    g[j] = 0.f;
  }

  auto load_row = [&](int64_t row, float (&x)[8]) {
    const float *p = a.A + row * a.lda;
    if (VEC) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int c = 4 * lane + 128 * h;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (c < n) v = __ldcs(reinterpret_cast<const float4 *>(p + c));   // n % 4 == 0 on this path
        x[4 * h + 0] = v.x;
        x[4 * h + 1] = v.y;
        x[4 * h + 2] = v.z;
        x[4 * h + 3] = v.w;
      }
    } else {
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int c = col(j);
        x[j] = c < n ? __ldcs(p + c) : 0.f;
      }
    }
  };

  float cur[8], nxt[8];
  int64_t row = w0;
  if (row < a.m) load_row(row, cur);
  while (row < a.m) {
    const int64_t next = row + warps;
    if (next < a.m) load_row(next, nxt);
    const float bi = __ldg(a.b + row);
    // r_i = b_i - A_i (vh + vl): Dot2 over the head, plain FMAs over the tail (2^-24 of the head's size)
    float s = 0.f, c = 0.f, tail = 0.f;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      dot2_step(cur[j], vh[j], s, c);
      tail = __fmaf_rn(cur[j], vl[j], tail);
    }
    c = __fadd_rn(c, tail);
    warp_dot2_reduce(s, c);
    float rh, re;
    two_sum(bi, -s, rh, re);
    const float r = __fadd_rn(rh, __fsub_rn(re, c));
#pragma unroll
    for (int j = 0; j < 8; ++j) g[j] = __fmaf_rn(cur[j], r, g[j]);
    row = next;
#pragma unroll
    for (int j = 0; j < 8; ++j) cur[j] = nxt[j];
  }
  // block sum of the warps' gradients in FP64, in warp order
#pragma unroll
  for (int j = 0; j < 8; ++j) red[wib][col(j)] = g[j];
  __syncthreads();
  for (int cc = threadIdx.x; cc < n; cc += kPassThreads) {
    double acc = 0.0;
#pragma unroll
    for (int w = 0; w < kPassThreads / 32; ++w) acc += (double)red[w][cc];
    a.part[(int64_t)blockIdx.x * n + cc] = acc;
  }
}

// ---------------------------------------------------------------------------------------- small FP64 steps

// Tinv = R^-1 for the upper-triangular FP64 R (n x n, row-major): one warp per column j solves R x = e_j from
// the last row up, the dot products over the lanes.
__global__ void lsrp_tri_inv_kernel(const double *R, int n, double *Tinv, int *status) {
  const int j = blockIdx.x, lane = threadIdx.x;
  extern __shared__ double xcol[];
  for (int i = lane; i < n; i += 32) xcol[i] = 0.0;
  __syncwarp();
  for (int i = j; i >= 0; --i) {
    double acc = 0.0;
    for (int k = i + 1 + lane; k <= j; k += 32) acc += R[(int64_t)i * n + k] * xcol[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) {
      const double d = R[(int64_t)i * n + i];
      if (!(d > 0.0) && status) rmc_report(status, RMC_ENUMERIC);
      xcol[i] = ((i == j ? 1.0 : 0.0) - acc) / d;
    }
    __syncwarp();
  }
  for (int i = lane; i < n; i += 32) Tinv[(int64_t)i * n + j] = xcol[i];
}

// z0 = Q^T Sb (Q s x n FP32 with row stride ldq): thread per column, FP64 sums in row order.
__global__ void lsrp_qt_b_kernel(const float *Q, int64_t s, int n, int64_t ldq, const float *Sb, double *z) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  double acc = 0.0;
  for (int64_t i = 0; i < s; ++i) acc += (double)Q[i * ldq + c] * (double)Sb[i];
  z[c] = acc;
}

// v = T z (T upper), written as FP64 x and as an FP32 head + tail for the pass kernel.
__device__ void lsrp_apply_T(const double *T, const double *z, int n, double *x, float *vh, float *vl) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double acc = 0.0;
    for (int j = i; j < n; ++j) acc += T[(int64_t)i * n + j] * z[j];
    x[i] = acc;
    const float h = (float)acc;
    vh[i] = h;
    vl[i] = (float)(acc - (double)h);
  }
}

__global__ void lsrp_init_kernel(const double *T, const double *z, int n, double *x, float *vh, float *vl,
                                 int *done, int *iters) {
  lsrp_apply_T(T, z, n, x, vh, vl);
  if (threadIdx.x == 0) {
    *done = 0;
    if (iters) *iters = 0;
  }
}

// One gradient step: g = sum of the partials (block order), w = T^T g, z += theta w, v = T z.  Converged when
// max |theta w| <= tol max |z|: the later passes and steps then return at once.
__global__ void __launch_bounds__(1024) lsrp_step_kernel(const double *part, int nblk, const double *T, int n,
                                                         double theta, double tol, double *z, double *g,
                                                         double *x, float *vh, float *vl, int *done,
                                                         int *iters) {
  if (*done) return;
  __shared__ double smax[2][32];
  for (int c = threadIdx.x; c < n; c += blockDim.x) {
    double acc = 0.0;
    for (int bk = 0; bk < nblk; ++bk) acc += part[(int64_t)bk * n + c];
    g[c] = acc;
  }
  __syncthreads();
  double dmax = 0.0, zmax = 0.0;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    double acc = 0.0;
    for (int i = 0; i <= j; ++i) acc += T[(int64_t)i * n + j] * g[i];   // (T^T g)_j, T upper
    const double dz = theta * acc;
    const double zn = z[j] + dz;
    z[j] = zn;
    dmax = fmax(dmax, fabs(dz));
    zmax = fmax(zmax, fabs(zn));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
    zmax = fmax(zmax, __shfl_xor_sync(0xffffffffu, zmax, o));
  }
  if ((threadIdx.x & 31) == 0) {
    smax[0][threadIdx.x >> 5] = dmax;
    smax[1][threadIdx.x >> 5] = zmax;
  }
  __syncthreads();
  lsrp_apply_T(T, z, n, x, vh, vl);
  if (threadIdx.x == 0) {
    double d = 0.0, zz = 0.0;
    for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) {
      d = fmax(d, smax[0][w]);
      zz = fmax(zz, smax[1][w]);
    }
    if (iters) *iters += 1;
    if (!(d > tol * zz)) *done = 1;     // also stops on NaN
  }
}

// Blocks of the pass: as many as fit on the GPU at once (one wave; every warp then strides over the same
// number of rows), at most one warp per row.  The count depends only on the SM count, so the workspace plan
// and the launch agree.
int pass_blocks(int num_sms, int64_t m) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, lsrp_pass_kernel<true>, kPassThreads, 0) !=
          cudaSuccess ||
      per_sm < 1) {
    (void)cudaGetLastError();
    per_sm = 4;
  }
  int64_t b = (int64_t)num_sms * per_sm;
  const int64_t need = (m + (kPassThreads / 32) - 1) / (kPassThreads / 32);
  if (b > need) b = need;
  return (int)(b < 1 ? 1 : b);
}

struct LsrpBufs {
  float *SAb, *Sb;
  double *R, *T, *z, *g, *x, *part;
  float *vh, *vl;
  int *flags;   // [0] done, [1] iterations
  void *rest;
};

LsrpBufs lsrp_carve(WsCarve &w, int64_t n, int64_t s, int nblk, size_t rest_bytes) {
  LsrpBufs b;
  b.SAb = w.take<float>((size_t)s * (n + 1));
  b.Sb = w.take<float>((size_t)s);
  b.R = w.take<double>((size_t)n * n);
  b.T = w.take<double>((size_t)n * n);
  b.z = w.take<double>(n);
  b.g = w.take<double>(n);
  b.x = w.take<double>(n);
  b.part = w.take<double>((size_t)nblk * n);
  b.vh = w.take<float>(n);
  b.vl = w.take<float>(n);
  b.flags = w.take<int>(4);
  b.rest = w.take<char>(rest_bytes);
  return b;
}


}  // namespace

// Launch the preconditioned iteration on an already sketched problem (SAb = [S^T A, S^T b], s x (n+1)).
static int lsrp_run(rmc_ctx *ctx, const float *A, int64_t m, int n, int64_t lda, const float *b, int64_t s,
                    double theta, int max_iters, double tol, double *x_out, int *iters_out, LsrpBufs &B) {
  cudaStream_t st = ctx->stream;
  // Q_Y R_Y = S^T A (CholeskyQR2 in place on the first n columns), T = R^-1, z0 = Q_Y^T S^T b, x0 = T z0
  RMC_TRY(rmc_launch_cholqr2(ctx, B.SAb, s, n, n + 1, B.R, B.rest, 2, true));
  lsrp_tri_inv_kernel<<<n, 32, sizeof(double) * n, st>>>(B.R, n, B.T, ctx->d_status);
  lsrp_qt_b_kernel<<<(n + 127) / 128, 128, 0, st>>>(B.SAb, s, n, n + 1, B.Sb, B.z);
  lsrp_init_kernel<<<1, 256, 0, st>>>(B.T, B.z, n, B.x, B.vh, B.vl, &B.flags[0], iters_out);
  rmc_note_launch(3);
  RMC_LAUNCH_CHECK();
  const int nblk = pass_blocks(ctx->num_sms, m);
  PassArgs pa;
  pa.A = A;
  pa.m = m;
  pa.lda = lda;
  pa.n = n;
  pa.b = b;
  pa.vh = B.vh;
  pa.vl = B.vl;
  pa.part = B.part;
  pa.done = &B.flags[0];
  const bool vec = (n % 4 == 0) && (lda % 4 == 0) && (reinterpret_cast<uintptr_t>(A) % 16 == 0);
  for (int it = 0; it < max_iters; ++it) {
    {
      RmcProf prof(ctx, RMC_K_LSR_PASS);
      if (vec) lsrp_pass_kernel<true><<<nblk, kPassThreads, 0, st>>>(pa);
      else lsrp_pass_kernel<false><<<nblk, kPassThreads, 0, st>>>(pa);
    }
    lsrp_step_kernel<<<1, 1024, 0, st>>>(B.part, nblk, B.T, n, theta, tol, B.z, B.g, B.x, B.vh, B.vl,
                                         &B.flags[0], iters_out);
    rmc_note_launch(2);
    RMC_LAUNCH_CHECK();
  }
  RMC_TRY_CUDA(cudaMemcpyAsync(x_out, B.x, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
  return RMC_OK;
}

// The step size when the caller passes theta <= 0: optimal for singular values of A T at the Marchenko-Pastur
// edges 1 -+ sqrt(n/s) of a Gaussian sketch (e capped at 0.9).
static double lsrp_default_theta(int64_t n, int64_t s) {
  double e = std::sqrt((double)n / (double)s);
  if (e > 0.9) e = 0.9;
  return 2.0 / (1.0 / ((1.0 - e) * (1.0 - e)) + 1.0 / ((1.0 + e) * (1.0 + e)));
}

size_t rmc_lsrp_plan_bytes(rmc_ctx *ctx, int64_t m, int64_t n, int64_t s, int kind, int prec) {
  size_t rest = rmc_sketch_plan_bytes(ctx, m, n + 1, s, kind, prec);
  const size_t q = rmc_cholqr2_ws(s, n, ctx->num_sms);
  if (q > rest) rest = q;
  WsCarve w;
  lsrp_carve(w, n, s, pass_blocks(ctx->num_sms, m), rest);
  return w.off;
}

extern "C" int rmc_lsr_precise(rmc_ctx *ctx, const float *A, int64_t m, int64_t n, int64_t lda, const float *b,
                               int64_t s, int kind, uint64_t seed, int prec, double theta, int max_iters,
                               double tol, double *x, int *iters) {
  if (!ctx || !b || !x || max_iters < 0 || max_iters > 100000 || !(tol >= 0.0)) return RMC_EINVAL;
  RMC_TRY(rmc_check_sketch_args(A, m, n, lda, s, kind, prec));
  if (s < n || n > kMaxN || m < n) return RMC_EINVAL;
  if (!(theta > 0.0)) theta = lsrp_default_theta(n, s);
  size_t rest = rmc_sketch_plan_bytes(ctx, m, n + 1, s, kind, prec);
  const size_t q = rmc_cholqr2_ws(s, n, ctx->num_sms);
  if (q > rest) rest = q;
  const int nblk = pass_blocks(ctx->num_sms, m);
  WsCarve plan;
  lsrp_carve(plan, n, s, nblk, rest);
  RMC_TRY(rmc_ws_reserve(ctx, plan.off));
  WsCarve w;
  w.base = static_cast<char *>(ctx->ws);
  LsrpBufs B = lsrp_carve(w, n, s, nblk, rest);
  // one sketch of [A, b]: S^T A into the first n columns of SAb, S^T b into its own vector
  RMC_TRY(rmc_run_sketch(ctx, A, m, n, lda, b, s, kind, seed, prec, B.SAb, n + 1, B.Sb, B.rest));
  return lsrp_run(ctx, A, m, (int)n, lda, b, s, theta, max_iters, tol, x, iters, B);
}
