// SRHT (Sec. 3.2.2, row orientation): C = (1/sqrt(s)) P^T H_N D A_pad.
//
// The N-point Walsh-Hadamard transform factors over the bits of the row index: with i = (i1, i2), r = (r1, r2)
// and N = N1 * N2, (H_N)[r, i] = (H_N1)[r1, i1] (H_N2)[r2, i2].  So
//     C[r] = (1/sqrt(s)) sum_{i1} (H_N1)[r1, i1] T[i1, r2],   T[i1, r2] = sum_{i2} (H_N2)[r2, i2] g_i A[i],
// and only the r2 that occur among the s sampled rows are needed.
//
// Stage 1 (persistent CTAs, N2 = 4096): a work unit is one 4-column slab of G consecutive 4096-row blocks
//   i1 = G a + b, b = 0 .. G-1.  Each CTA streams the next block's 4096 x 4 tile into shared memory with cp.async
//   while it transforms the current one (sign flip, then its 12 index bits in three register phases of four bits
//   separated by shared-memory transposes).  The high index bits split as r1 = (r1_hi, c) with c = r1 mod G, so
//       C[r] = (1/sqrt(s)) sum_a (-1)^popc(r1_hi & a) T'[a, (c, r2)],
//       T'[a, (c, r2)] = sum_b (-1)^popc(c & b) T[G a + b, r2],
//   and the CTA folds its G blocks into T' in shared memory: for every pair (c, r2) that occurs among the sampled
//   rows (|R2'| <= min(s, 4096 G) pairs), the transformed row r2 of block b is added with the sign of (c, b); the
//   last block writes the pairs to T'.  G = min(8, N / 4096) when s <= 4096 (the accumulators fit), else 1.
// Stage 2: C[r] = (1/sqrt(s)) sum over the N1 / G groups of +-T'[a, (c, r2)], one thread per (row, 4 columns),
//   eight loads in flight.
// A is read once; T' holds (N1 / G) |R2'| rows, written once and read about s / |R2'| times.
#include <algorithm>
#include <cstring>

#include "rmc_internal.cuh"
#include "philox.cuh"
#include "tc_common.cuh"

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

// Persistent stage 1.  CTA k takes work units k, k + gridDim.x, ... (unit = (a, slab)), each as G items
// (blocks b = 0 .. G-1 of rows [(G a + b) 4096, +4096) of the slab).  Each CTA double-buffers its 4096 x 4 tile
// in shared memory: the next item's rows stream in while the current one is transformed.
//   kTma (A 16-byte aligned): the tile arrives by 16 TMA loads of 256 x 4 boxes, rows packed densely (row r at
//     16 r bytes), plus the tile's 512 bytes of sign words by one bulk copy, all on the buffer's mbarrier.  The
//     first phase takes the index bits 3-6 into registers (lanes along bits 0-2: conflict-free reads of the dense
//     rows) and writes the rows back at their swizzled slots after a barrier; the second takes bits 0-2 and 7,
//     the third bits 8-11.
//   otherwise: cp.async of 16 bytes per row straight into the swizzled slots (plain loads for unaligned rows),
//     and the phases take bits 0-3, 4-7, 8-11.
// Swizzled slot of row r: r ^ ((r >> 4) & 7) (16-byte units).  Thread (q, h) = (t / 2, t % 2) transforms column
// pair h (a float2) of 16 rows per phase, so 16 warps share the work; after the last phase the thread owns rows
// r2 = q + 256 j (j < 16); the pairs (c, r2) of the sample (pinfo[p] = (r2 << 3) | c) are then folded
// pair-major: pair p, column pair h belongs to thread (p mod 256, h) in every block, so the accumulators need no
// synchronisation.  Every wait is bounded (RMC_ETIMEOUT).  T out: [N1 / G][umax][slabs].
template <bool kTma>
__global__ void __launch_bounds__(kThreads, 1) srht_stage1_kernel(const __grid_constant__ CUtensorMap tmap,
                                                                   const float *__restrict__ A, int64_t m, int64_t n,
                                                                   int64_t lda, const float *__restrict__ b,
                                                                   const uint32_t *__restrict__ sign_bits,
                                                                   const uint32_t *__restrict__ npairs_g,
                                                                   const uint16_t *__restrict__ pinfo_g, int64_t umax,
                                                                   int64_t slabs, int64_t N1, int G,
                                                                   float4 *__restrict__ T, bool vec, int *status) {
  // two tile buffers, sign words, pair records, accumulators; the base is aligned by hand (TMA destinations
  // must be 128-byte aligned, and the static shared variables below come first)
  extern __shared__ __align__(16) unsigned char srht_raw[];
  float4 *sm = reinterpret_cast<float4 *>((reinterpret_cast<uintptr_t>(srht_raw) + 1023) & ~uintptr_t(1023));
  uint32_t *sgn = reinterpret_cast<uint32_t *>(sm + 2 * kRowsCta);   // 2 x kRowsCta / 32 sign words
  uint16_t *pinfo = reinterpret_cast<uint16_t *>(sgn + 2 * (kRowsCta / 32));   // (r2 << 3) | c of each pair
  float2 *acc = reinterpret_cast<float2 *>(pinfo + kRowsCta);          // kRowsCta pairs x 2 halves (G > 1)
  __shared__ __align__(8) uint64_t full[2];
  __shared__ int go;
  const int64_t units = slabs * (N1 / G);
  const int t = threadIdx.x, q = t >> 1, h = t & 1;
  const int npairs = (int)*npairs_g;
  for (int p = t; p < npairs; p += kThreads) pinfo[p] = pinfo_g[p];
  if (kTma && t == 0) {
    tc::mbar_init(&full[0], 1);
    tc::mbar_init(&full[1], 1);
    tc::fence_barrier_init();
  }
  __syncthreads();

  // item n of this CTA: unit blockIdx.x + (n / G) gridDim.x, block b = n mod G
  auto unit_of = [&](int64_t nn) { return (int64_t)blockIdx.x + (nn / G) * gridDim.x; };
  auto issue = [&](int64_t nn, int buf) {
    const int64_t unit = unit_of(nn);
    const int64_t slab = unit % slabs, i1 = (unit / slabs) * G + nn % G;
    const int64_t c0 = slab * 4;
    float4 *tile = sm + buf * kRowsCta;
    uint32_t *sw = sgn + buf * (kRowsCta / 32);
    if (kTma) {
      if (t == 0) {
        tc::fence_proxy_async_smem();
        tc::mbar_arrive_expect_tx(&full[buf], (uint32_t)(kRowsCta * 16 + (kRowsCta / 32) * 4));
#pragma unroll
        for (int k = 0; k < kRowsCta / 256; ++k)
          tc::tma_load_2d(tile + 256 * k, &tmap, (int32_t)c0, (int32_t)(i1 * kRowsCta + 256 * k), &full[buf]);
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                tc::smem_u32(sw)),
            "l"(sign_bits + i1 * (kRowsCta / 32)), "r"((kRowsCta / 32) * 4), "r"(tc::smem_u32(&full[buf]))
            : "memory");
      }
      return;
    }
    const int64_t row8 = i1 * kRowsCta + t * 8;
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
        cp_async16(tile + swz(t * 8 + j), row < m ? (const void *)(A + row * lda + c0) : (const void *)A,
                   row < m ? 16 : 0);
      }
    } else {  // the slab holding b, or unaligned rows: plain loads
#pragma unroll
      for (int j = 0; j < 8; ++j) tile[swz(t * 8 + j)] = load_slab(A, m, n, lda, b, row8 + j, c0, vec);
    }
  };
  int64_t nn = 0;
  int cur = 0;
  int64_t issued = 0;
  if (unit_of(0) < units) {
    issue(0, 0);
    issued = 1;
  }
  if (!kTma) asm volatile("cp.async.commit_group;\n" ::: "memory");
  for (; unit_of(nn) < units; ++nn, cur ^= 1) {
    float4 *S = sm + cur * kRowsCta;
    float2 *S2 = reinterpret_cast<float2 *>(S) + h;   // column pair h of float4 slot k: S2[2 k]
    if (kTma) {
      if (t == 0) go = tc::mbar_wait(&full[cur], (uint32_t)((nn >> 1) & 1)) ? 1 : 0;
    } else {
      asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    }
    // the tile is in, and every thread is done with the other buffer (the previous fold) before it is refilled
    __syncthreads();
    if (kTma && !go) {
      if (t == 0) rmc_report(status, RMC_ETIMEOUT);
      break;
    }
    if (unit_of(nn + 1) < units) {
      issue(nn + 1, cur ^ 1);
      issued = nn + 2;
    }
    if (!kTma) asm volatile("cp.async.commit_group;\n" ::: "memory");

    const int64_t unit = unit_of(nn);
    const int64_t slab = unit % slabs, a = unit / slabs;
    const int bb = (int)(nn % G);
    const int64_t i1 = a * G + bb;
    float2 v[16];
    if (kTma) {
      if (b != nullptr && slab * 4 <= n && n < slab * 4 + 4) {
        // b is column n: the TMA filled it with zeros (past A's columns)
        float *tf = reinterpret_cast<float *>(S);
        const int cb = (int)(n - slab * 4);
        for (int r = t; r < kRowsCta; r += kThreads) {
          const int64_t row = i1 * kRowsCta + r;
          tf[4 * r + cb] = row < m ? __ldg(b + row) : 0.f;
        }
        __syncthreads();
      }
      // phase 1: rows r = (q mod 8) + 8 j + 128 (q / 8): sign flip and bits 3..6, read from the dense rows
      const int lo3 = q & 7, hi5 = q >> 3;
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int r = lo3 | (j << 3) | (hi5 << 7);
        float2 x = S2[2 * r];
        const uint32_t word = sgn[cur * (kRowsCta / 32) + (r >> 5)];
        if ((word >> (r & 31)) & 1u) x = make_float2(-x.x, -x.y);
        v[j] = x;
      }
      fwht16(v);
      __syncthreads();   // every dense row is read before any slot is rewritten
#pragma unroll
      for (int j = 0; j < 16; ++j) S2[2 * swz(lo3 | (j << 3) | (hi5 << 7))] = v[j];
      __syncthreads();
      // phase 2: rows r = (j mod 8) + 8 (q mod 16) + 128 (j / 8) + 256 (q / 16): bits 0..2 and 7
      const int qa = q & 15, qb = q >> 4;
#pragma unroll
      for (int j = 0; j < 16; ++j) v[j] = S2[2 * swz((j & 7) | (qa << 3) | ((j >> 3) << 7) | (qb << 8))];
      fwht16(v);
#pragma unroll
      for (int j = 0; j < 16; ++j) S2[2 * swz((j & 7) | (qa << 3) | ((j >> 3) << 7) | (qb << 8))] = v[j];
      __syncthreads();
    } else {
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
    }
    // phase 3: bits 8..11, written back; then, after a barrier, thread (q, h) folds pairs q, q + 256, ... of the
    // sample (column pair h): the same amount of work on every thread, whichever rows the pairs fall on
    {
#pragma unroll
      for (int j = 0; j < 16; ++j) v[j] = S2[2 * swz(q | (j << 8))];
      fwht16(v);
#pragma unroll
      for (int j = 0; j < 16; ++j) S2[2 * swz(q | (j << 8))] = v[j];
      __syncthreads();
      float2 *Tout = reinterpret_cast<float2 *>(T + a * umax * slabs + slab) + h;
      const bool first = bb == 0, last = bb == G - 1;
      for (int p = q; p < npairs; p += kThreads / 2) {
        const uint32_t info = pinfo[p];
        const float2 xv = S2[2 * swz((int)(info >> 3))];
        const float sg = (__popc(info & 7u & (uint32_t)bb) & 1) ? -1.f : 1.f;
        float2 y = first ? make_float2(0.f, 0.f) : acc[2 * p + h];
        y = make_float2(fmaf(sg, xv.x, y.x), fmaf(sg, xv.y, y.y));
        if (last) Tout[(int64_t)p * slabs * 2] = y;
        else acc[2 * p + h] = y;
      }
    }
  }
  // no copy may still be landing when the CTA exits: after a timeout, wait (bounded) once more for the items
  // issued and not consumed
  if (kTma && t == 0)
    for (int64_t k = nn; k < issued; ++k) (void)tc::mbar_wait(&full[k & 1], (uint32_t)((k >> 1) & 1));
}

// C[k, :] for sampled row r = idx[k]: (1/sqrt(s)) sum_a (-1)^popc(r1_hi & a) T'[a, slot(r mod 4096 G)], with
// r1_hi = r / (4096 G).
__global__ void srht_stage2_kernel(const float4 *__restrict__ T, int64_t groups, int64_t umax, int64_t slabs,
                                   const int64_t *__restrict__ idx, int64_t s, const uint32_t *__restrict__ slotv,
                                   int64_t span, float scale, int64_t n, float *__restrict__ C, int64_t ldc,
                                   float *__restrict__ Cb) {
  const int64_t total = s * slabs;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = e / slabs, sl = e - k * slabs;
    const int64_t r = idx[k];
    const int64_t r1 = r / span;
    const uint32_t u = slotv[r % span];
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 8
    for (int64_t a = 0; a < groups; ++a) {  // unrolled: eight independent loads in flight per thread
      const float4 x = __ldg(&T[(a * umax + u) * slabs + sl]);
      const float sg = (__popcll(r1 & a) & 1) ? -1.f : 1.f;
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

// The pairs (c, r2) of the sample: v = r mod (4096 G) = c 4096 + r2 for every sampled row r.  mark[v] = 1, then in
// one block: off[r2] = number of pairs with a smaller r2 (pairs ordered by r2, then c; off[4096] = their count),
// pinfo[p] = (r2 << 3) | c of pair p, slotv[v] = that pair's position.
__global__ void srht_mark_pairs_kernel(const int64_t *idx, int64_t s, int64_t span, uint32_t *mark) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < s; k += (int64_t)gridDim.x * blockDim.x)
    mark[idx[k] % span] = 1u;
}

__global__ void __launch_bounds__(1024) srht_pairs_kernel(const uint32_t *mark, int G, uint32_t *off,
                                                          uint32_t *slotv, uint16_t *pinfo) {
  __shared__ uint32_t part[1024];
  constexpr int per = kRowsCta / 1024;
  const int lo = threadIdx.x * per;
  uint32_t cnt = 0;
  for (int k = 0; k < per; ++k)
    for (int c = 0; c < G; ++c) cnt += mark[c * kRowsCta + lo + k];
  part[threadIdx.x] = cnt;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    const uint32_t y = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
    __syncthreads();
    part[threadIdx.x] += y;
    __syncthreads();
  }
  uint32_t run = threadIdx.x ? part[threadIdx.x - 1] : 0;
  for (int k = 0; k < per; ++k) {
    const int r2 = lo + k;
    off[r2] = run;
    for (int c = 0; c < G; ++c)
      if (mark[c * kRowsCta + r2]) {
        pinfo[run] = (uint16_t)((r2 << 3) | c);
        slotv[c * kRowsCta + r2] = run;
        ++run;
      }
  }
  if (threadIdx.x == 1023) off[kRowsCta] = run;
}

struct SrhtPlan {
  int64_t N, N2, N1, slabs;
  int G;            // 4096-row blocks folded per work unit
  int64_t umax;     // rows of T' per group (an upper bound on the pairs of the sample)
};

SrhtPlan srht_plan(int64_t m, int64_t ntot, int64_t s, int64_t num_ctas) {
  SrhtPlan p;
  p.N = 1;
  while (p.N < m) p.N <<= 1;
  // One CTA per 4096-row block: combining several blocks in a thread-block cluster over DSMEM moves about as many
  // bytes between shared memories as the CTAs read from HBM and adds two cluster barriers per tile, which measured
  // slower than writing the needed rows of each block and combining the N / 4096 blocks in stage 2.  Folding G
  // consecutive blocks in one CTA's shared memory instead cuts the intermediate T' by about G (its pairs fit in
  // the 4096 accumulators when s <= 4096).
  p.N2 = kRowsCta;
  p.N1 = p.N > p.N2 ? p.N / p.N2 : 1;
  p.slabs = (ntot + 3) / 4;
  p.G = s <= kRowsCta ? (int)std::min<int64_t>(8, p.N1) : 1;
  // fewer blocks per unit where 8 would leave the last wave of units uneven (the CTAs with one more unit set the
  // time): within 5% of the per-CTA average, on the number of CTAs that can be co-resident
  const int64_t items = p.slabs * p.N1;
  while (p.G > 1) {
    const int64_t units = items / p.G;
    const int64_t per = (units + num_ctas - 1) / num_ctas * p.G;
    if ((double)per <= 1.05 * (double)items / (double)num_ctas) break;
    p.G >>= 1;
  }
  p.umax = std::min<int64_t>(s, p.N2 * p.G);
  return p;
}

struct SrhtBufs {
  int64_t *idx;
  uint32_t *sign_bits;
  uint32_t *mark, *off, *slotv;
  uint16_t *pinfo;
  float4 *T;
  void *sample_ws;
};

SrhtBufs srht_carve(WsCarve &w, const SrhtPlan &p, int64_t s) {
  SrhtBufs b;
  b.idx = w.take<int64_t>(s);
  b.sign_bits = w.take<uint32_t>(p.N / 32 + 1);
  b.mark = w.take<uint32_t>(p.N2 * p.G);
  b.off = w.take<uint32_t>(p.N2 + 4);
  b.slotv = w.take<uint32_t>(p.N2 * p.G);
  b.pinfo = w.take<uint16_t>(p.N2);
  b.T = w.take<float4>((p.N1 / p.G) * p.umax * p.slabs);
  b.sample_ws = w.take<char>(rmc_srht_sample_ws(p.N));
  return b;
}

}  // namespace

size_t rmc_srht_ws(int64_t m, int64_t ntot, int64_t s, int num_sms) {
  WsCarve w;
  srht_carve(w, srht_plan(m, ntot, s, num_sms), s);
  return w.off;
}

int rmc_launch_srht(rmc_ctx *ctx, const float *A, int64_t m, int64_t n, int64_t lda, const float *b, int64_t s,
                    uint64_t seed, uint32_t instance, float *C, int64_t ldc, float *Cb, void *ws) {
  cudaStream_t st = ctx->stream;
  const int64_t ntot = n + (b ? 1 : 0);
  const SrhtPlan p = srht_plan(m, ntot, s, ctx->num_sms);
  WsCarve w;
  w.base = static_cast<char *>(ws);
  const SrhtBufs bf = srht_carve(w, p, s);
  const int64_t span = p.N2 * p.G;

  RMC_TRY(rmc_launch_srht_sample(ctx, seed, instance, p.N, s, bf.idx, bf.sample_ws));
  RMC_TRY_CUDA(cudaMemsetAsync(bf.mark, 0, sizeof(uint32_t) * span, st));
  srht_mark_pairs_kernel<<<rmc_blocks(s, 256, 1024), 256, 0, st>>>(bf.idx, s, span, bf.mark);
  srht_pairs_kernel<<<1, 1024, 0, st>>>(bf.mark, p.G, bf.off, bf.slotv, bf.pinfo);
  srht_signs_kernel<<<rmc_blocks(m, 256, 4096), 256, 0, st>>>(seed, instance, m, bf.sign_bits);
  rmc_note_launch(3);
  RMC_LAUNCH_CHECK();

  const bool vec = (lda % 4 == 0) && (reinterpret_cast<uintptr_t>(A) % 16 == 0);
  // aligned rows stream in by TMA (256 x 4 boxes, rows packed densely); the map covers A's n columns, b (column
  // n) is added on chip
  CUtensorMap map;
  memset(&map, 0, sizeof(map));
  const bool tma = vec && rmc_make_tmap_dense(&map, A, m, n, lda, 4, 256) == RMC_OK;
  // alignment slack, tiles, sign words, pair records and (G > 1) the accumulators of 4096 pairs
  const size_t smem = 1024 + 2 * sizeof(float4) * kRowsCta + sizeof(uint32_t) * 2 * (kRowsCta / 32) +
                      sizeof(uint16_t) * kRowsCta + (p.G > 1 ? sizeof(float4) * kRowsCta : 0);
  auto kern = tma ? srht_stage1_kernel<true> : srht_stage1_kernel<false>;
  RMC_TRY_CUDA(rmc_allow_smem(kern, smem));
  // as many CTAs as are co-resident (one per SM), each looping over (a, slab) units of G items
  const int64_t units = p.slabs * (p.N1 / p.G);
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem) != cudaSuccess || per_sm < 1) {
    (void)cudaGetLastError();
    per_sm = 1;
  }
  const int64_t grid = std::min<int64_t>(units, (int64_t)per_sm * ctx->num_sms);
  rmc_note_launch(2);
  {
    RmcProf prof(ctx, RMC_K_SRHT);
    kern<<<(unsigned)grid, kThreads, smem, st>>>(map, A, m, n, lda, b, (const uint32_t *)bf.sign_bits,
                                                 (const uint32_t *)(bf.off + p.N2), (const uint16_t *)bf.pinfo, p.umax, p.slabs,
                                                 p.N1, p.G, bf.T, vec, ctx->d_status);
  }
  const float scale = 1.0f / sqrtf((float)s);
  RmcProf prof(ctx, RMC_K_SRHT_REDUCE);
  srht_stage2_kernel<<<rmc_blocks(s * p.slabs, 256, 65536), 256, 0, st>>>(bf.T, p.N1 / p.G, p.umax, p.slabs, bf.idx,
                                                                            s, bf.slotv, span, scale, n, C, ldc, Cb);
  RMC_LAUNCH_CHECK();
  return RMC_OK;
}
