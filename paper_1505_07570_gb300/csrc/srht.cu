// SRHT (Sec. 3.2.2, row orientation): C = (1/sqrt(s)) P^T H_N D A_pad.
//
// The N-point Walsh-Hadamard transform factors over the bits of the row index: with i = (i1, i2), r = (r1, r2)
// and N = N1 * N2, (H_N)[r, i] = (H_N1)[r1, i1] (H_N2)[r2, i2].  So
//     C[r] = (1/sqrt(s)) sum_{i1} (H_N1)[r1, i1] T[i1, r2],   T[i1, r2] = sum_{i2} (H_N2)[r2, i2] g_i A[i],
// and only the r2 that occur among the s sampled rows are needed.
//
// Stage 1 (persistent CTAs, one 4096-row block of one 4-column slab per item, N2 = 4096): each CTA takes items in
//   turn, streams the next item's 4096 x 4 tile into shared memory with cp.async while it transforms the current
//   one (sign flip, then its 12 index bits in three register phases of four bits separated by shared-memory
//   transposes), and writes the transformed rows whose index r2 occurs in the sample to T[i1, slot(r2), slab].
// Stage 2: C[r] = (1/sqrt(s)) sum over the N1 = N / N2 blocks of +-T[i1, slot(r2)], one thread per (row,
//   4 columns), eight loads in flight.
// A is read once; T holds N1 * |R2| rows (|R2| <= min(s, N2)), written once and read about s / |R2| times.
#include <algorithm>

#include "rmc_internal.cuh"
#include "philox.cuh"

using namespace rmc;

namespace {

constexpr int kRowsCta = 4096;   // rows transformed by one CTA (12 index bits)
constexpr int kThreads = 512;    // per phase: 16 rows x 2 columns per thread

// shared-memory slot of local row r: XOR the low 3 bits with bits 4..6 (conflict-free float4 phases)
__device__ __forceinline__ int swz(int r) { return r ^ ((r >> 4) & 7); }

__device__ __forceinline__ void bfly(float2 &a, float2 &b) {
  const float2 x = a, y = b;
  a = make_float2(x.x + y.x, x.y + y.y);
  b = make_float2(x.x - y.x, x.y - y.y);
}

// 16-point transform over the register index (4 bits).
__device__ __forceinline__ void fwht16(float2 (&v)[16]) {
#pragma unroll
  for (int h = 1; h < 16; h <<= 1)
#pragma unroll
    for (int j = 0; j < 16; ++j)
      if ((j & h) == 0) bfly(v[j], v[j | h]);
}

__device__ __forceinline__ float4 load_slab(const float *__restrict__ A, int64_t m, int64_t n, int64_t lda,
                                            const float *__restrict__ b, int64_t row, int64_t c0, bool vec) {
  float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
  if (row >= m) return x;
  const float *ar = A + row * lda;
  if (vec && c0 + 3 < n) return __ldg(reinterpret_cast<const float4 *>(ar + c0));
  float t[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int64_t c = c0 + k;
    t[k] = (c < n) ? __ldg(ar + c) : ((c == n && b) ? __ldg(b + row) : 0.f);
  }
  return make_float4(t[0], t[1], t[2], t[3]);
}

// D as packed bits: bit (i mod 32) of word i / 32 set means g_i = -1.
__global__ void srht_signs_kernel(uint64_t seed, uint32_t instance, int64_t m, uint32_t *bits) {
  const int64_t words = (m + 31) / 32;
  for (int64_t base = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) & ~int64_t(31); base < words * 32;
       base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = base + (threadIdx.x & 31);
    const bool neg = i < m && srht_sign(seed, instance, (uint64_t)i) < 0.f;
    const uint32_t word = __ballot_sync(0xffffffffu, neg);
    if ((threadIdx.x & 31) == 0) bits[base / 32] = word;
  }
}

__device__ __forceinline__ void cp_async16(float4 *dst, const void *src, int bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
               "l"(src), "r"(bytes)
               : "memory");
}

// Persistent stage 1.  CTA k takes items k, k + gridDim.x, ... where an item is one (slab, i1) pair: rows
// [i1 4096, +4096) of the 4-column slab.  Each CTA double-buffers its 4096 x 4 tile in shared memory: the rows of
// the next item stream in with cp.async while the current one is transformed.  Thread (q, h) = (t / 2, t % 2)
// transforms column pair h (a float2) of 16 rows per phase, so 16 warps share the work, and the last phase writes
// the rows that occur in the sample straight from registers.  T out: [N1][umax][slabs] float4.
__global__ void __launch_bounds__(kThreads, 1) srht_stage1_kernel(const float *__restrict__ A, int64_t m, int64_t n,
                                                                   int64_t lda, const float *__restrict__ b,
                                                                   const uint32_t *__restrict__ sign_bits,
                                                                   const uint32_t *__restrict__ mark,
                                                                   const uint32_t *__restrict__ slot, int64_t umax,
                                                                   int64_t slabs, int64_t N1, float4 *__restrict__ T,
                                                                   bool vec) {
  extern __shared__ float4 sm[];   // two buffers of kRowsCta float4, swizzled; sign words; row -> slot table
  uint32_t *sgn = reinterpret_cast<uint32_t *>(sm + 2 * kRowsCta);  // 2 x kRowsCta / 32 sign words
  int *rslot = reinterpret_cast<int *>(sgn + 2 * (kRowsCta / 32));   // slot of local row r2 in T, or -1
  const int64_t items = slabs * N1;
  const int t = threadIdx.x, q = t >> 1, h = t & 1;
  for (int r = t; r < kRowsCta; r += kThreads) rslot[r] = mark[r] ? (int)slot[r] : -1;

  auto issue = [&](int64_t item, float4 *buf, uint32_t *sw) {
    const int64_t slab = item % slabs, i1 = item / slabs;
    const int64_t row8 = i1 * kRowsCta + t * 8;
    const int64_t c0 = slab * 4;
    if (t < kRowsCta / 32) {  // this tile's sign words, with the tile (rows past m read as +1)
      const int64_t w = i1 * (kRowsCta / 32) + t;
      const bool in = w * 32 < m;
      asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"((unsigned)__cvta_generic_to_shared(sw + t)),
                   "l"(in ? sign_bits + w : sign_bits), "r"(in ? 4 : 0)
                   : "memory");
    }
    if (vec && c0 + 3 < n) {
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int64_t row = row8 + j;
        cp_async16(buf + swz(t * 8 + j), row < m ? (const void *)(A + row * lda + c0) : (const void *)A,
                   row < m ? 16 : 0);
      }
    } else {  // the slab holding b, or unaligned rows: plain loads
#pragma unroll
      for (int j = 0; j < 8; ++j) buf[swz(t * 8 + j)] = load_slab(A, m, n, lda, b, row8 + j, c0, vec);
    }
  };

  int64_t item = blockIdx.x;
  int cur = 0;
  if (item < items) issue(item, sm, sgn);
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  for (; item < items; item += gridDim.x, cur ^= 1) {
    float4 *S = sm + cur * kRowsCta;
    float2 *S2 = reinterpret_cast<float2 *>(S) + h;   // column pair h of float4 slot k: S2[2 k]
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    // the tile is in, and every thread is done with the other buffer (the previous combine) before it is refilled
    __syncthreads();
    if (item + gridDim.x < items) issue(item + gridDim.x, sm + (cur ^ 1) * kRowsCta, sgn + (cur ^ 1) * (kRowsCta / 32));
    asm volatile("cp.async.commit_group;\n" ::: "memory");

    const int64_t slab = item % slabs, i1 = item / slabs;
    float2 v[16];
    // phase 1: rows q*16 + j, sign flip, bits 0..3
    {
      const uint32_t gw = sgn[cur * (kRowsCta / 32) + (q >> 1)] >> ((q & 1) * 16);  // rows q*16 .. q*16 + 15
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        float2 x = S2[2 * swz(q * 16 + j)];
        if ((gw >> j) & 1u) x = make_float2(-x.x, -x.y);
        v[j] = x;
      }
      fwht16(v);
#pragma unroll
      for (int j = 0; j < 16; ++j) S2[2 * swz(q * 16 + j)] = v[j];
    }
    __syncthreads();
    // phase 2: bits 4..7 (each thread rewrites exactly the slots it read)
    {
      const int lo = q & 15, hi = q >> 4;
#pragma unroll
      for (int j = 0; j < 16; ++j) v[j] = S2[2 * swz(lo | (j << 4) | (hi << 8))];
      fwht16(v);
#pragma unroll
      for (int j = 0; j < 16; ++j) S2[2 * swz(lo | (j << 4) | (hi << 8))] = v[j];
    }
    __syncthreads();
    // phase 3: bits 8..11, then the rows whose index occurs among the sampled low parts r2 go to T
    {
#pragma unroll
      for (int j = 0; j < 16; ++j) v[j] = S2[2 * swz(q | (j << 8))];
      fwht16(v);
      float2 *Tout = reinterpret_cast<float2 *>(T + i1 * umax * slabs + slab) + h;
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int u = rslot[q | (j << 8)];
        if (u >= 0) Tout[(int64_t)u * slabs * 2] = v[j];
      }
    }
  }
}

// C[k, :] for sampled row r = idx[k]: (1/sqrt(s)) sum_{i1} (-1)^popc(r1 & i1) T[i1, slot(r2)].
__global__ void srht_stage2_kernel(const float4 *__restrict__ T, int64_t N1, int64_t umax, int64_t slabs,
                                   const int64_t *__restrict__ idx, int64_t s, const uint32_t *__restrict__ slot,
                                   int64_t N2, float scale, int64_t n, float *__restrict__ C, int64_t ldc,
                                   float *__restrict__ Cb) {
  const int64_t total = s * slabs;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = e / slabs, sl = e - k * slabs;
    const int64_t r = idx[k];
    const int64_t r1 = r / N2;
    const uint32_t u = slot[r % N2];
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 8
    for (int64_t i1 = 0; i1 < N1; ++i1) {  // unrolled: eight independent loads in flight per thread
      const float4 x = __ldg(&T[(i1 * umax + u) * slabs + sl]);
      const float sg = (__popcll(r1 & i1) & 1) ? -1.f : 1.f;
      acc = make_float4(fmaf(sg, x.x, acc.x), fmaf(sg, x.y, acc.y), fmaf(sg, x.z, acc.z), fmaf(sg, x.w, acc.w));
    }
    const float out[4] = {acc.x * scale, acc.y * scale, acc.z * scale, acc.w * scale};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int64_t c = sl * 4 + q;
      if (c < n) C[k * ldc + c] = out[q];
      else if (c == n && Cb) Cb[k] = out[q];
    }
  }
}

// Distinct low parts r2 = idx & (N2 - 1) of the sample: mark, then number them in ascending order in one block
// (N2 <= 32768): slot[r2] = the row of T that holds r2.
__global__ void srht_mark_r2_kernel(const int64_t *idx, int64_t s, int64_t N2, uint32_t *mark) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < s; k += (int64_t)gridDim.x * blockDim.x)
    mark[idx[k] & (N2 - 1)] = 1u;
}

__global__ void __launch_bounds__(1024) srht_compact_r2_kernel(const uint32_t *mark, int64_t N2, uint32_t *slot) {
  __shared__ uint32_t part[1024];
  const int per = (int)((N2 + 1023) / 1024);
  const int lo = threadIdx.x * per;
  uint32_t c = 0;
  for (int k = 0; k < per; ++k)
    if (lo + k < N2) c += mark[lo + k];
  part[threadIdx.x] = c;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    const uint32_t y = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
    __syncthreads();
    part[threadIdx.x] += y;
    __syncthreads();
  }
  uint32_t run = threadIdx.x ? part[threadIdx.x - 1] : 0;
  for (int k = 0; k < per; ++k) {
    const int64_t r = lo + k;
    if (r < N2 && mark[r]) slot[r] = run++;
  }
}

struct SrhtPlan {
  int64_t N, N2, N1, slabs;
};

SrhtPlan srht_plan(int64_t m, int64_t ntot) {
  SrhtPlan p;
  p.N = 1;
  while (p.N < m) p.N <<= 1;
  // One CTA per 4096-row block: combining several blocks in a thread-block cluster over DSMEM moves about as many
  // bytes between shared memories as the CTAs read from HBM and adds two cluster barriers per tile, which measured
  // slower than writing the needed rows of each block and combining the N / 4096 blocks in stage 2.
  p.N2 = kRowsCta;
  p.N1 = p.N > p.N2 ? p.N / p.N2 : 1;
  p.slabs = (ntot + 3) / 4;
  return p;
}

struct SrhtBufs {
  int64_t *idx;
  uint32_t *sign_bits;
  uint32_t *mark, *slot;
  float4 *T;
  void *sample_ws;
};

SrhtBufs srht_carve(WsCarve &w, const SrhtPlan &p, int64_t s) {
  SrhtBufs b;
  b.idx = w.take<int64_t>(s);
  b.sign_bits = w.take<uint32_t>(p.N / 32 + 1);
  b.mark = w.take<uint32_t>(p.N2);
  b.slot = w.take<uint32_t>(p.N2);
  const int64_t umax = s < p.N2 ? s : p.N2;
  b.T = w.take<float4>(p.N1 * umax * p.slabs);
  b.sample_ws = w.take<char>(rmc_srht_sample_ws(p.N));
  return b;
}

}  // namespace

size_t rmc_srht_ws(int64_t m, int64_t ntot, int64_t s) {
  WsCarve w;
  srht_carve(w, srht_plan(m, ntot), s);
  return w.off;
}

int rmc_launch_srht(rmc_ctx *ctx, const float *A, int64_t m, int64_t n, int64_t lda, const float *b, int64_t s,
                    uint64_t seed, uint32_t instance, float *C, int64_t ldc, float *Cb, void *ws) {
  cudaStream_t st = ctx->stream;
  const int64_t ntot = n + (b ? 1 : 0);
  const SrhtPlan p = srht_plan(m, ntot);
  WsCarve w;
  w.base = static_cast<char *>(ws);
  const SrhtBufs bf = srht_carve(w, p, s);

  RMC_TRY(rmc_launch_srht_sample(ctx, seed, instance, p.N, s, bf.idx, bf.sample_ws));
  RMC_TRY_CUDA(cudaMemsetAsync(bf.mark, 0, sizeof(uint32_t) * p.N2, st));
  srht_mark_r2_kernel<<<rmc_blocks(s, 256, 1024), 256, 0, st>>>(bf.idx, s, p.N2, bf.mark);
  srht_compact_r2_kernel<<<1, 1024, 0, st>>>(bf.mark, p.N2, bf.slot);
  srht_signs_kernel<<<rmc_blocks(m, 256, 4096), 256, 0, st>>>(seed, instance, m, bf.sign_bits);
  rmc_note_launch(3);
  RMC_LAUNCH_CHECK();
  const int64_t umax = s < p.N2 ? s : p.N2;

  const bool vec = (lda % 4 == 0) && (reinterpret_cast<uintptr_t>(A) % 16 == 0);
  const size_t smem = 2 * sizeof(float4) * kRowsCta + sizeof(uint32_t) * (2 * (kRowsCta / 32) + (size_t)p.N2);
  RMC_TRY_CUDA(cudaFuncSetAttribute(srht_stage1_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  // as many CTAs as are co-resident (one per SM), each looping over (slab, i1) items
  const int64_t items = p.slabs * p.N1;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, srht_stage1_kernel, kThreads, smem) != cudaSuccess ||
      per_sm < 1) {
    (void)cudaGetLastError();
    per_sm = 1;
  }
  const int64_t grid = std::min<int64_t>(items, (int64_t)per_sm * ctx->num_sms);
  rmc_note_launch(2);
  {
    RmcProf prof(ctx, RMC_K_SRHT);
    srht_stage1_kernel<<<(unsigned)grid, kThreads, smem, st>>>(A, m, n, lda, b, (const uint32_t *)bf.sign_bits,
                                                               (const uint32_t *)bf.mark, (const uint32_t *)bf.slot,
                                                               umax, p.slabs, p.N1, bf.T, vec);
  }
  const float scale = 1.0f / sqrtf((float)s);
  RmcProf prof(ctx, RMC_K_SRHT_REDUCE);
  srht_stage2_kernel<<<rmc_blocks(s * p.slabs, 256, 65536), 256, 0, st>>>(bf.T, p.N1, umax, p.slabs, bf.idx, s,
                                                                            bf.slot, p.N2, scale, n, C, ldc, Cb);
  RMC_LAUNCH_CHECK();
  return RMC_OK;
}
