// Count sketch (Sec. 3.2.3, Algorithm 3.1 in the row orientation): C[h(i), :] += g(i) A[i, :].
//
// GPU form: rather than scattering every row into C (m * n atomic adds), the rows are first grouped by bucket
// with a counting sort of the m hashes (a few MB of traffic), and then one warp per bucket gathers its rows and
// sums them in registers.  A is read exactly once, with whole-row coalesced loads, and C is written once.
// The counting sort is stable (rows are ranked within their chunk with warp match operations), so each
// bucket's rows are visited in increasing row order, and the sums are formed in a fixed order: results are
// bit-identical from run to run.
#include "rmc_internal.cuh"
#include "philox.cuh"

using namespace rmc;

namespace {

constexpr int kChunk = 1024;   // rows per block in the hash/rank passes (one row per thread)

// Pass 1: hash every row (bucket in bits 1.., sign in bit 0) and count rows per (bucket, chunk).
// count is bucket-major: count[b * nchunks + c].
__global__ void __launch_bounds__(kChunk) cs_hash_count_kernel(uint64_t seed, uint32_t instance, int64_t m,
                                                               uint32_t s, uint32_t *code, uint32_t *count,
                                                               int64_t nchunks) {
  const int64_t i = (int64_t)blockIdx.x * kChunk + threadIdx.x;
  if (i >= m) return;
  uint32_t h;
  float g;
  cs_hash(seed, instance, (uint64_t)i, s, &h, &g);
  code[i] = (h << 1) | (g < 0.f ? 1u : 0u);
  atomicAdd(&count[(int64_t)h * nchunks + blockIdx.x], 1u);
}

// Exclusive scan over the bucket-major counts (reduce-then-scan, three passes).
constexpr int kScanTile = 4096;

__global__ void scan_tile_sum_kernel(const uint32_t *in, int64_t len, uint64_t *tile_sum) {
  __shared__ unsigned long long warp_sum[32];
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  unsigned long long s = 0;
  for (int k = threadIdx.x; k < kScanTile; k += blockDim.x)
    if (base + k < len) s += in[base + k];
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) warp_sum[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    unsigned long long v = threadIdx.x < (blockDim.x >> 5) ? warp_sum[threadIdx.x] : 0;
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) tile_sum[blockIdx.x] = v;
  }
}

__global__ void scan_tile_offsets_kernel(uint64_t *tile_sum, int64_t ntiles) {
  __shared__ unsigned long long part[1024];
  const int64_t per = (ntiles + 1023) / 1024;
  const int64_t lo = threadIdx.x * per, hi = min(ntiles, lo + per);
  unsigned long long sum = 0;
  for (int64_t t = lo; t < hi; ++t) sum += tile_sum[t];
  part[threadIdx.x] = sum;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    unsigned long long v = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  unsigned long long run = threadIdx.x ? part[threadIdx.x - 1] : 0;
  for (int64_t t = lo; t < hi; ++t) {
    const unsigned long long v = tile_sum[t];
    tile_sum[t] = run;
    run += v;
  }
}

// In-place exclusive scan of one tile, offset by the tile's start (1024 threads, 4 values each).
__global__ void __launch_bounds__(1024) scan_tile_apply_kernel(uint32_t *data, int64_t len, const uint64_t *tile_off) {
  __shared__ uint32_t warp_sum[32];
  const int64_t base = (int64_t)blockIdx.x * kScanTile + 4 * threadIdx.x;
  uint32_t v[4];
  uint32_t local = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    v[k] = (base + k < len) ? data[base + k] : 0u;
    local += v[k];
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t incl = local;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) warp_sum[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = warp_sum[lane];
    uint32_t wi = w;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += y;
    }
    warp_sum[lane] = wi - w;   // exclusive prefix of the warp totals
  }
  __syncthreads();
  uint32_t run = (uint32_t)tile_off[blockIdx.x] + warp_sum[warp] + (incl - local);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if (base + k < len) data[base + k] = run;
    run += v[k];
  }
}

// Pass 3: stable placement.  Rows of one chunk are visited in increasing order, 32 at a time; a row's slot is
// its chunk's offset for its bucket plus the number of earlier rows of the chunk in the same bucket.
__global__ void __launch_bounds__(kChunk) cs_place_kernel(const uint32_t *code, int64_t m, const uint32_t *offset,
                                                          int64_t nchunks, uint32_t *perm) {
  const int64_t i = (int64_t)blockIdx.x * kChunk + threadIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool valid = i < m;
  const uint32_t b = valid ? (code[i] >> 1) : 0xFFFFFFFFu;
  const uint32_t peers = __match_any_sync(0xffffffffu, b);
  const uint32_t rank_in_warp = __popc(peers & ((1u << lane) - 1));
  // rows of earlier warps of this chunk with the same bucket
  __shared__ uint32_t buckets[kChunk];
  buckets[threadIdx.x] = b;
  __syncthreads();
  uint32_t before = 0;
  if (valid) {
    for (int k = 0; k < warp * 32; ++k) before += (buckets[k] == b);
    perm[offset[(int64_t)b * nchunks + blockIdx.x] + before + rank_in_warp] = (uint32_t)i;
  }
}

// Pass 4: one block per bucket.  Warp w of the block sums rows w, w + 4, w + 8, ... of the bucket (rows in
// increasing order within each warp, eight in flight), then the four partial rows are added in warp order
// through shared memory: deterministic.  Columns are split in blocks of 32 * 4 * NV (float4 loads when the
// rows are 16-byte aligned); b, when given, is one more column.
constexpr int kGatherWarps = 4;
constexpr int kRowsInFlight = 8;

template <int NV, bool VEC>
__global__ void __launch_bounds__(32 * kGatherWarps) cs_gather_kernel(const float *__restrict__ A, int64_t n,
                                                                      int64_t lda, const float *__restrict__ bvec,
                                                                      const uint32_t *__restrict__ code,
                                                                      const uint32_t *__restrict__ bucket_start,
                                                                      const uint32_t *__restrict__ perm, int64_t s,
                                                                      float *__restrict__ C, int64_t ldc,
                                                                      float *__restrict__ Cb, int64_t col0) {
  constexpr int W = VEC ? 4 : 1;               // floats per load
  constexpr int COLS = 32 * W * NV;            // columns per block of this launch
  __shared__ float red[kGatherWarps][COLS + 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int64_t bk = blockIdx.x; bk < s; bk += gridDim.x) {
    const uint32_t beg = bucket_start[bk], end = bucket_start[bk + 1];
    float acc[NV][W];
#pragma unroll
    for (int v = 0; v < NV; ++v)
#pragma unroll
      for (int w = 0; w < W; ++w) acc[v][w] = 0.f;
    float accb = 0.f;
    for (uint32_t j0 = beg + warp; j0 < end; j0 += kGatherWarps * kRowsInFlight) {
      uint32_t row[kRowsInFlight];
      float sg[kRowsInFlight];
#pragma unroll
      for (int u = 0; u < kRowsInFlight; ++u) {
        const uint32_t j = j0 + kGatherWarps * u;
        const bool ok = j < end;
        row[u] = ok ? perm[j] : 0u;
        sg[u] = ok ? ((code[row[u]] & 1u) ? -1.f : 1.f) : 0.f;
      }
      float val[kRowsInFlight][NV][W];
#pragma unroll
      for (int u = 0; u < kRowsInFlight; ++u) {
        const float *ar = A + (int64_t)row[u] * lda + col0;
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          const int64_t c = (int64_t)W * (lane + 32 * v);
          if (VEC) {
            float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
            if (sg[u] != 0.f && col0 + c + 3 < n) x = __ldg(reinterpret_cast<const float4 *>(ar + c));
            else if (sg[u] != 0.f) {
              if (col0 + c < n) x.x = __ldg(ar + c);
              if (col0 + c + 1 < n) x.y = __ldg(ar + c + 1);
              if (col0 + c + 2 < n) x.z = __ldg(ar + c + 2);
            }
            val[u][v][0] = x.x;
            if (W > 1) { val[u][v][1 % W] = x.y; val[u][v][2 % W] = x.z; val[u][v][3 % W] = x.w; }
          } else {
            val[u][v][0] = (sg[u] != 0.f && col0 + c < n) ? __ldg(ar + c) : 0.f;
          }
        }
      }
#pragma unroll
      for (int u = 0; u < kRowsInFlight; ++u) {
#pragma unroll
        for (int v = 0; v < NV; ++v)
#pragma unroll
          for (int w = 0; w < W; ++w) acc[v][w] = fmaf(sg[u], val[u][v][w], acc[v][w]);
        if (bvec && lane == 0 && col0 == 0 && sg[u] != 0.f) accb = fmaf(sg[u], __ldg(bvec + row[u]), accb);
      }
    }
    // fixed-order combination of the warps' partial rows
#pragma unroll
    for (int v = 0; v < NV; ++v)
#pragma unroll
      for (int w = 0; w < W; ++w) red[warp][W * (lane + 32 * v) + w] = acc[v][w];
    if (lane == 0) red[warp][COLS] = accb;
    __syncthreads();
    for (int c = threadIdx.x; c <= COLS; c += blockDim.x) {
      float t = 0.f;
#pragma unroll
      for (int q = 0; q < kGatherWarps; ++q) t += red[q][c];
      if (c < COLS) {
        if (col0 + c < n) C[bk * ldc + col0 + c] = t;
      } else if (bvec && col0 == 0) {
        Cb[bk] = t;
      }
    }
    __syncthreads();
  }
}

struct CsBufs {
  uint32_t *code, *count, *perm, *bucket_start;
  uint64_t *tile;
};

int64_t cs_chunks(int64_t m) { return (m + kChunk - 1) / kChunk; }

CsBufs cs_carve(WsCarve &w, int64_t m, int64_t s) {
  CsBufs b;
  const int64_t nch = cs_chunks(m);
  const int64_t len = s * nch;
  b.code = w.take<uint32_t>(m);
  b.count = w.take<uint32_t>(len + 1);
  b.perm = w.take<uint32_t>(m);
  b.bucket_start = w.take<uint32_t>(s + 1);
  b.tile = w.take<uint64_t>((len + kScanTile - 1) / kScanTile + 1);
  return b;
}

__global__ void bucket_start_kernel(const uint32_t *offset, int64_t s, int64_t nchunks, int64_t m, uint32_t *start) {
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b <= s; b += (int64_t)gridDim.x * blockDim.x)
    start[b] = (b < s) ? offset[b * nchunks] : (uint32_t)m;
}

}  // namespace

size_t rmc_countsketch_ws(int64_t m, int64_t s) {
  WsCarve w;
  cs_carve(w, m, s);
  return w.off;
}

int rmc_launch_countsketch(rmc_ctx *ctx, const float *A, int64_t m, int64_t n, int64_t lda, const float *b, int64_t s,
                           uint64_t seed, uint32_t instance, float *C, int64_t ldc, float *Cb, void *ws) {
  cudaStream_t st = ctx->stream;
  WsCarve w;
  w.base = static_cast<char *>(ws);
  const CsBufs bf = cs_carve(w, m, s);
  const int64_t nch = cs_chunks(m);
  const int64_t len = s * nch;
  const int64_t ntiles = (len + kScanTile - 1) / kScanTile;

  RMC_TRY_CUDA(cudaMemsetAsync(bf.count, 0, sizeof(uint32_t) * len, st));
  cs_hash_count_kernel<<<(unsigned)nch, kChunk, 0, st>>>(seed, instance, m, (uint32_t)s, bf.code, bf.count, nch);
  scan_tile_sum_kernel<<<(unsigned)ntiles, 1024, 0, st>>>(bf.count, len, bf.tile);
  scan_tile_offsets_kernel<<<1, 1024, 0, st>>>(bf.tile, ntiles);
  scan_tile_apply_kernel<<<(unsigned)ntiles, 1024, 0, st>>>(bf.count, len, bf.tile);
  bucket_start_kernel<<<rmc_blocks(s + 1, 256, 4096), 256, 0, st>>>(bf.count, s, nch, m, bf.bucket_start);
  cs_place_kernel<<<(unsigned)nch, kChunk, 0, st>>>(bf.code, m, bf.count, nch, bf.perm);
  rmc_note_launch(6);
  RMC_LAUNCH_CHECK();
  RmcProf prof(ctx, RMC_K_COUNTSKETCH);

  const bool vec = (lda % 4 == 0) && (reinterpret_cast<uintptr_t>(A) % 16 == 0);
  const unsigned grid = (unsigned)(s < (int64_t)1 << 30 ? s : (int64_t)1 << 30);
  rmc_note_launch((int)((n + (vec ? 255 : 127)) / (vec ? 256 : 128)));
  if (vec) {
    for (int64_t c0 = 0; c0 < n; c0 += 256) {
      if (n - c0 > 128)
        cs_gather_kernel<2, true><<<grid, 32 * kGatherWarps, 0, st>>>(A, n, lda, b, bf.code, bf.bucket_start, bf.perm, s, C, ldc,
                                                        Cb, c0);
      else
        cs_gather_kernel<1, true><<<grid, 32 * kGatherWarps, 0, st>>>(A, n, lda, b, bf.code, bf.bucket_start, bf.perm, s, C, ldc,
                                                        Cb, c0);
    }
  } else {
    for (int64_t c0 = 0; c0 < n; c0 += 128)
      cs_gather_kernel<4, false><<<grid, 32 * kGatherWarps, 0, st>>>(A, n, lda, b, bf.code, bf.bucket_start, bf.perm, s, C, ldc,
                                                       Cb, c0);
  }
  RMC_LAUNCH_CHECK();
  return RMC_OK;
}
