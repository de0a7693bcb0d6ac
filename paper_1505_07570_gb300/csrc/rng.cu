// Random draws of the sketches: raw Philox words, Gaussian matrices, count-sketch hashes and the SRHT sample.
#include "rmc_internal.cuh"
#include "philox.cuh"

using namespace rmc;

namespace {

__global__ void philox_words_kernel(uint64_t seed, uint32_t stream_id, uint32_t instance, uint64_t first,
                                    int64_t count, uint4 *out) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < count;
       t += (int64_t)gridDim.x * blockDim.x)
    out[t] = philox_block(seed, stream_id, instance, first + (uint64_t)t);
}

// One thread per Gaussian block (row i, column group g): up to four entries of row i.
__global__ void gaussian_kernel(uint64_t seed, uint32_t instance, int64_t rows, int64_t cols, float *out,
                                int64_t ld, float scale, bool transposed) {
  const int64_t groups = (cols + 3) / 4;
  const int64_t total = rows * groups;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / groups, g = t - i * groups;
    const float4 z = gaussian4(seed, instance, (uint64_t)t);
    const float v[4] = {z.x, z.y, z.z, z.w};
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int64_t j = 4 * g + c;
      if (j < cols) {
        if (transposed) out[j * ld + i] = scale * v[c];
        else out[i * ld + j] = scale * v[c];
      }
    }
  }
}

__global__ void cs_hash_kernel(uint64_t seed, uint32_t instance, int64_t m, uint32_t s, int32_t *bucket,
                               float *sign) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t h;
    float g;
    cs_hash(seed, instance, (uint64_t)i, s, &h, &g);
    bucket[i] = (int32_t)h;
    sign[i] = g;
  }
}

// ---------------------------------------------------------------------------- SRHT sample (radix select)
// The s smallest keys are found in one histogram pass over the top `bits` bits of the keys: every key in a
// bin below the bin that holds the s-th smallest key is selected, and the few keys inside that bin are
// ranked exactly by (key, index).  The selected flags are then compacted in index order.

constexpr int kCandCap = 16384;

struct SampleCtl {
  uint32_t bin;    // bin holding the s-th smallest key
  uint32_t need;   // how many keys of that bin are selected
  uint32_t ncand;  // keys found in that bin
  uint32_t pad;
};

__global__ void srht_hist_kernel(uint64_t seed, uint32_t instance, int64_t N, int bits, uint32_t *hist) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < N; j += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&hist[srht_key(seed, instance, (uint64_t)j) >> (64 - bits)], 1u);
}

// One block of 1024 threads: scan the histogram and locate the bin of the s-th smallest key.
__global__ void srht_find_bin_kernel(const uint32_t *hist, int nbins, int64_t s, SampleCtl *ctl) {
  __shared__ unsigned long long part[1024];
  const int per = (nbins + 1023) / 1024;
  const int lo = threadIdx.x * per, hi = min(nbins, lo + per);
  unsigned long long sum = 0;
  for (int b = lo; b < hi; ++b) sum += hist[b];
  part[threadIdx.x] = sum;
  __syncthreads();
  // inclusive Hillis-Steele scan over 1024 partial sums
  for (int off = 1; off < 1024; off <<= 1) {
    unsigned long long v = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  unsigned long long before = threadIdx.x ? part[threadIdx.x - 1] : 0;
  if (before < (unsigned long long)s && (unsigned long long)s <= part[threadIdx.x]) {
    for (int b = lo; b < hi; ++b) {
      if (before + hist[b] >= (unsigned long long)s) {
        ctl->bin = b;
        ctl->need = (uint32_t)(s - before);
        ctl->ncand = 0;
        break;
      }
      before += hist[b];
    }
  }
}

__global__ void srht_mark_kernel(uint64_t seed, uint32_t instance, int64_t N, int bits, SampleCtl *ctl,
                                 uint8_t *flag, unsigned long long *cand_key, uint32_t *cand_idx) {
  const uint32_t bstar = ctl->bin;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < N; j += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t key = srht_key(seed, instance, (uint64_t)j);
    const uint32_t bin = (uint32_t)(key >> (64 - bits));
    flag[j] = bin < bstar ? 1 : 0;
    if (bin == bstar) {
      const uint32_t slot = atomicAdd(&ctl->ncand, 1u);
      if (slot < kCandCap) {
        cand_key[slot] = key;
        cand_idx[slot] = (uint32_t)j;
      }
    }
  }
}

// Exact ranking of the candidates of the boundary bin by (key, index).
__global__ void srht_resolve_kernel(SampleCtl *ctl, const unsigned long long *cand_key, const uint32_t *cand_idx,
                                    uint8_t *flag, int *status) {
  const uint32_t c = ctl->ncand, need = ctl->need;
  if (c > (uint32_t)kCandCap) {
    if (threadIdx.x == 0) rmc_report(status, RMC_ENUMERIC);
    return;
  }
  for (uint32_t t = threadIdx.x; t < c; t += blockDim.x) {
    const unsigned long long kt = cand_key[t];
    const uint32_t jt = cand_idx[t];
    uint32_t rank = 0;
    for (uint32_t u = 0; u < c; ++u) {
      const unsigned long long ku = cand_key[u];
      rank += (ku < kt) || (ku == kt && cand_idx[u] < jt);
    }
    if (rank < need) flag[jt] = 1;
  }
}

constexpr int kCompactTile = 4096;  // flags per block in the compaction passes (1024 threads x 4)

__global__ void flag_count_kernel(const uint8_t *flag, int64_t N, uint32_t *tile_count) {
  __shared__ uint32_t warp_sum[32];
  const int64_t base = blockIdx.x * (int64_t)kCompactTile;
  uint32_t c = 0;
  for (int k = 0; k < 4; ++k) {
    const int64_t j = base + k * 1024 + threadIdx.x;
    if (j < N) c += flag[j];
  }
  for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0) warp_sum[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x < 32) {
    uint32_t v = warp_sum[threadIdx.x];
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) tile_count[blockIdx.x] = v;
  }
}

// Exclusive scan of the tile counts (one block; each thread scans a contiguous segment).
__global__ void tile_scan_kernel(const uint32_t *count, int64_t ntiles, uint64_t *offset) {
  __shared__ unsigned long long part[1024];
  const int64_t per = (ntiles + 1023) / 1024;
  const int64_t lo = threadIdx.x * per, hi = min(ntiles, lo + per);
  unsigned long long sum = 0;
  for (int64_t t = lo; t < hi; ++t) sum += count[t];
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
    offset[t] = run;
    run += count[t];
  }
}

// Write the selected indices in ascending order: block-wide exclusive scan of the flags of one tile.
__global__ void flag_compact_kernel(const uint8_t *flag, int64_t N, const uint64_t *tile_off, int64_t *idx,
                                    int64_t s) {
  __shared__ uint32_t warp_sum[32];
  const int64_t base = blockIdx.x * (int64_t)kCompactTile;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint64_t run = tile_off[blockIdx.x];
  for (int k = 0; k < 4; ++k) {
    const int64_t j = base + k * 1024 + threadIdx.x;
    const uint32_t f = (j < N) ? flag[j] : 0;
    const uint32_t ballot = __ballot_sync(0xffffffffu, f);
    if (lane == 0) warp_sum[warp] = __popc(ballot);
    __syncthreads();
    uint32_t before = 0, total = 0;
    for (int w = 0; w < 32; ++w) {
      const uint32_t v = warp_sum[w];
      before += (w < warp) ? v : 0;
      total += v;
    }
    const uint64_t pos = run + before + __popc(ballot & ((1u << lane) - 1));
    if (f && pos < (uint64_t)s) idx[pos] = j;
    run += total;
    __syncthreads();
  }
}

}  // namespace

int rmc_launch_philox(cudaStream_t st, uint64_t seed, uint32_t stream_id, uint32_t instance, uint64_t first,
                      int64_t count, uint32_t *out) {
  if (count <= 0) return RMC_OK;
  philox_words_kernel<<<rmc_blocks(count, 256, 65536), 256, 0, st>>>(seed, stream_id, instance, first, count,
                                                                     reinterpret_cast<uint4 *>(out));
  rmc_note_launch();
  RMC_LAUNCH_CHECK();
  return RMC_OK;
}

int rmc_launch_gaussian(cudaStream_t st, uint64_t seed, uint32_t instance, int64_t rows, int64_t cols, float *out,
                        int64_t ld, float scale) {
  if (rows <= 0 || cols <= 0) return RMC_OK;
  gaussian_kernel<<<rmc_blocks(rows * ((cols + 3) / 4), 256, 65536), 256, 0, st>>>(seed, instance, rows, cols,
                                                                                    out, ld, scale, false);
  rmc_note_launch();
  RMC_LAUNCH_CHECK();
  return RMC_OK;
}

int rmc_launch_gaussian_t(cudaStream_t st, uint64_t seed, uint32_t instance, int64_t rows, int64_t cols,
                          float *out_t, int64_t ld_t, float scale) {
  if (rows <= 0 || cols <= 0) return RMC_OK;
  gaussian_kernel<<<rmc_blocks(rows * ((cols + 3) / 4), 256, 65536), 256, 0, st>>>(seed, instance, rows, cols,
                                                                                    out_t, ld_t, scale, true);
  rmc_note_launch();
  RMC_LAUNCH_CHECK();
  return RMC_OK;
}

int rmc_launch_cs_hash(cudaStream_t st, uint64_t seed, uint32_t instance, int64_t m, int64_t s, int32_t *bucket,
                       float *sign) {
  if (m <= 0) return RMC_OK;
  cs_hash_kernel<<<rmc_blocks(m, 256, 65536), 256, 0, st>>>(seed, instance, m, (uint32_t)s, bucket, sign);
  rmc_note_launch();
  RMC_LAUNCH_CHECK();
  return RMC_OK;
}

static int sample_bits(int64_t N) {
  int lg = 0;
  while ((int64_t(1) << lg) < N) ++lg;
  int bits = lg - 4;  // about 16 keys per bin
  return bits < 4 ? 4 : (bits > 20 ? 20 : bits);
}

size_t rmc_srht_sample_ws(int64_t N) {
  WsCarve w;
  w.take<uint32_t>(size_t(1) << sample_bits(N));
  w.take<SampleCtl>(1);
  w.take<uint8_t>(N);
  w.take<unsigned long long>(kCandCap);
  w.take<uint32_t>(kCandCap);
  const int64_t ntiles = (N + kCompactTile - 1) / kCompactTile;
  w.take<uint32_t>(ntiles);
  w.take<uint64_t>(ntiles);
  return w.off;
}

int rmc_launch_srht_sample(rmc_ctx *ctx, uint64_t seed, uint32_t instance, int64_t N, int64_t s, int64_t *idx,
                           void *ws) {
  cudaStream_t st = ctx->stream;
  const int bits = sample_bits(N);
  const int nbins = 1 << bits;
  WsCarve w;
  w.base = static_cast<char *>(ws);
  uint32_t *hist = w.take<uint32_t>(nbins);
  SampleCtl *ctl = w.take<SampleCtl>(1);
  uint8_t *flag = w.take<uint8_t>(N);
  unsigned long long *ckey = w.take<unsigned long long>(kCandCap);
  uint32_t *cidx = w.take<uint32_t>(kCandCap);
  const int64_t ntiles = (N + kCompactTile - 1) / kCompactTile;
  uint32_t *tcount = w.take<uint32_t>(ntiles);
  uint64_t *toff = w.take<uint64_t>(ntiles);

  RMC_TRY_CUDA(cudaMemsetAsync(hist, 0, sizeof(uint32_t) * nbins, st));
  RMC_TRY_CUDA(cudaMemsetAsync(ctl, 0, sizeof(SampleCtl), st));
  const unsigned grid = rmc_blocks(N, 256, 8 * ctx->num_sms);
  srht_hist_kernel<<<grid, 256, 0, st>>>(seed, instance, N, bits, hist);
  srht_find_bin_kernel<<<1, 1024, 0, st>>>(hist, nbins, s, ctl);
  srht_mark_kernel<<<grid, 256, 0, st>>>(seed, instance, N, bits, ctl, flag, ckey, cidx);
  srht_resolve_kernel<<<1, 1024, 0, st>>>(ctl, ckey, cidx, flag, ctx->d_status);
  flag_count_kernel<<<(unsigned)ntiles, 1024, 0, st>>>(flag, N, tcount);
  tile_scan_kernel<<<1, 1024, 0, st>>>(tcount, ntiles, toff);
  flag_compact_kernel<<<(unsigned)ntiles, 1024, 0, st>>>(flag, N, toff, idx, s);
  rmc_note_launch(7);
  RMC_LAUNCH_CHECK();
  return RMC_OK;
}
