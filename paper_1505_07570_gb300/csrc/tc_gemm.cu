// tcgen05 tensor-core kernels (sm_103a): TF32 operands, FP32 accumulation in tensor memory.
//
// kind::tf32 takes both operands K-major, so the product with A over its rows needs A transposed on chip.
//
// Gaussian sketch C = (1/sqrt(s)) G^T [A | b] (Sec. 3.2.1), one CTA per (256 sketch rows, 256 columns of A,
// range of rows of A):
//   warp 1      allocates 512 TMEM columns (two 128 x 256 FP32 accumulators) and issues tcgen05.mma
//               (M=128, N=256, K=8) from one lane
//   warps 2-3   transpose the 32 x 256 tile of A (staged by TMA) into the K-major, 128-byte-swizzled layout
//               (BF16: rounding to BF16 on the way)
//   warps 4-19  per stage of 32 rows: draw G^T (32 x 256) from Philox (the sketch stream: eight normals per
//               block) straight into the same K-major layout, and fold the b column in with FP32 FMAs
//   8 of them   epilogue: tcgen05.ld of the accumulators, written as this row range's partial sum
// Both sketch tiles share each transposed A tile.  Three stages of 64 KB are in flight; every wait is bounded
// (RMC_ETIMEOUT after one second).
#include <cuda.h>
#include <cudaTypedefs.h>

#include "rmc_internal.cuh"
#include "philox.cuh"
#include "tc_common.cuh"

using namespace rmc;

namespace {

constexpr int kKStage = 32;                       // rows of A per stage (128 bytes of TF32 along K)
constexpr int kM = 128, kN = 256;
constexpr int kMT = 2;                            // 128-row sketch tiles per CTA sharing one A tile
constexpr int kOmegaBytes = kM * kKStage * 4;     // 16 KB per sketch tile
constexpr int kBBytes = kN * kKStage * 4;         // 32 KB: 256 columns of A, K-major (also the staging size)
constexpr int kAtomBytes = kKStage * 128;         // staging: 32 rows x 32 columns, 128-byte swizzle
constexpr int kStgStages = 2;                     // TMA staging buffers (A rows, row-major)
constexpr int kStages = 2;                        // operand buffers (G^T tiles + transposed A)
constexpr int kStageBytes = kMT * kOmegaBytes + kBBytes;
constexpr int kTransWarp0 = 2;                    // the transposers (staging -> K-major) start at warp 2
constexpr int kRngWarps = 16;                     // the warps that draw G^T follow them
constexpr int kTmemCols = kMT * kN;               // 512

// TF32: an operand stage holds 32 rows of A (128 bytes of TF32 along K).  BF16: the same bytes hold 64 rows
// (128 bytes of BF16), filled from two 32-row staging buffers.
template <bool BF16>
struct GaussCfg {
  static constexpr int kTransWarps = 2;               // warps 2-3 transpose (four measured slower for TF32)
  static constexpr int kRngWarp0 = kTransWarp0 + kTransWarps;
  static constexpr int kThreads = 32 * (kRngWarp0 + kRngWarps);
  static constexpr int kKOp = BF16 ? 64 : 32;         // rows of A per operand stage
  static constexpr int kStgPer = kKOp / kKStage;      // staging buffers per operand stage
  static constexpr int kStg = BF16 ? 3 : kStgStages;  // staging ring
  // barriers (256 bytes), then the b-column partials of the two producer groups (TF32)
  static constexpr size_t kSmem = 1024 + (size_t)kStg * kBBytes + (size_t)kStages * kStageBytes + 256 +
                                  sizeof(float) * kM * kMT;
};
static_assert(GaussCfg<true>::kSmem <= 227 * 1024, "shared memory");

// Approximate special functions (PTX .approx with flush-to-zero).  Every argument here is a normal number (u in
// [2^-24, 1), -2 ln u >= 2^-24, angles in (-pi, pi)), so the subnormal handling of the default forms is skipped.
__device__ __forceinline__ float lg2_ftz(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rsqrt_ftz(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float sin_ftz(float x) {
  float y;
  asm("sin.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float cos_ftz(float x) {
  float y;
  asm("cos.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Box-Muller with the hardware approximations: the operands are rounded to TF32 (10-bit mantissa) before they
// reach the tensor cores, far coarser than these approximations' ~2^-21 error.  -2 ln u = (-2 ln 2) log2 u; the
// angle is shifted by -pi into (-pi, pi) and both outputs negated to compensate.
// The Box-Muller pair of one word of the sketch stream (its low and high 16-bit halves).
__device__ __forceinline__ float2 box_muller16_fast(uint32_t w) {
  const float t = -1.3862943611198906f * lg2_ftz(unit16_f32(w & 0xFFFFu));
  const float r = t * rsqrt_ftz(t);
  const float a = 6.283185307179586f * (unit16_f32(w >> 16) - 0.5f);
  return make_float2(-r * cos_ftz(a), -r * sin_ftz(a));
}

// Round to TF32 (10-bit mantissa), to nearest with ties away from zero, as cvt.rna.tf32.f32 does, with integer
// operations on the bit pattern (add half of the dropped range, clear the 13 dropped bits): the conversion
// instruction runs at a fraction of the integer rate and this kernel converts every draw.  Finite inputs only.
__device__ __forceinline__ float to_tf32(float x) {
  return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

// Two FP32 values as BF16 (round to nearest even), the first in the low half (the lower K index).
__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  uint32_t r;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}

// Byte offset of (row r, 16-byte chunk q) in a tile with 128-byte rows and 128-byte swizzle.
__device__ __forceinline__ int swz_off(int r, int q) { return r * 128 + ((q ^ (r & 7)) << 4); }

// v with its 13 low mantissa bits cleared (the TF32 head), and the exact remainder.
__device__ __forceinline__ float tf32_head(float v) { return __uint_as_float(__float_as_uint(v) & 0xFFFFE000u); }

__device__ __forceinline__ void split4(float4 v, float4 &h, float4 &l) {
  h = make_float4(tf32_head(v.x), tf32_head(v.y), tf32_head(v.z), tf32_head(v.w));
  l = make_float4(v.x - h.x, v.y - h.y, v.z - h.z, v.w - h.w);
}

// Transpose one staged tile of 32 rows of A x (32 kAtoms) columns -- kAtoms column atoms of 32 rows x 128 bytes,
// 128-byte swizzled, as a 32 x 32 TMA box writes them -- into the K-major, 128-byte-swizzled operand tile (row c
// = column c of A, its 32 K values in one 128-byte row).  The 8 kHalves lanes-groups of 8 split the work: unit
// (kq, cq) = rows 4kq..4kq+3 x columns 4cq..4cq+3; lane lq of group g = 8 gh + gl takes kq = lq and the units
// cq = c0 + 8 (gh + kHalves i), c0 = (gl + lq) mod 8.  Within a group the reads (chunk c0 ^ (4 (lq & 1) + t) of a
// row) and the writes (chunk lq ^ (4 (c0 & 1) + t)) of the 8 lanes fall on 8 distinct 16-byte bank groups, and
// every address is a per-thread constant plus a multiple of 4096 bytes (one column atom), so the loop carries
// no address arithmetic.  X3: the remainder tile (the exact v - head) is written half_off bytes after the head.
template <int kAtoms, int kHalves, bool X3>
__device__ __forceinline__ void transpose_tile_tf32(const unsigned char *src, unsigned char *dst, int half_off,
                                                    int tl) {
  const int lq = tl & 7, gl = (tl >> 3) & 7, gh = tl >> 6;
  const int c0 = (gl + lq) & 7;
  int roff[4], woff[4];
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    roff[t] = swz_off(4 * lq + t, c0);
    woff[t] = swz_off(4 * c0 + t, lq);
  }
#pragma unroll
  for (int i = 0; i < kAtoms / kHalves; ++i) {
    const int atom = gh + kHalves * i;
    const unsigned char *sa = src + atom * (32 * 128);
    unsigned char *da = dst + atom * (32 * 128);
    float4 v[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) v[t] = *reinterpret_cast<const float4 *>(sa + roff[t]);
    const float4 o[4] = {make_float4(v[0].x, v[1].x, v[2].x, v[3].x), make_float4(v[0].y, v[1].y, v[2].y, v[3].y),
                         make_float4(v[0].z, v[1].z, v[2].z, v[3].z), make_float4(v[0].w, v[1].w, v[2].w, v[3].w)};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (X3) {
        float4 h, lo;
        split4(o[j], h, lo);
        *reinterpret_cast<float4 *>(da + woff[j]) = h;
        *reinterpret_cast<float4 *>(da + half_off + woff[j]) = lo;
      } else {
        *reinterpret_cast<float4 *>(da + woff[j]) = o[j];
      }
    }
  }
}

struct GaussArgs {
  const float *b;  // the extra column folded in by the drawing warps: b[row * ldb] (nullptr: none)
  int64_t ldb;
  int64_t m, n, ntot, s;
  uint64_t seed;
  uint32_t instance;
  int64_t rows_per_split;
  float *part;     // [splits][s][ntot]
  int *status;
};

__device__ __forceinline__ bool warp_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag, int *status) {
  int ok = 1;
  if ((threadIdx.x & 31) == 0) ok = !*abort_flag && tc::mbar_wait(bar, parity);
  ok = __shfl_sync(0xffffffffu, ok, 0);
  if (!ok && (threadIdx.x & 31) == 0) {
    *abort_flag = 1;
    rmc_report(status, RMC_ETIMEOUT);
  }
  return ok != 0;
}

// grid: x = 256-row sketch range, y = 256-column tile of A, z = row range of A.
template <bool BF16>
__global__ void __launch_bounds__(GaussCfg<BF16>::kThreads, 1) tc_gauss_kernel(const __grid_constant__ CUtensorMap tmap_a,
                                                               GaussArgs args) {
  using C = GaussCfg<BF16>;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char *smem = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                          ~uintptr_t(1023));
  unsigned char *staging = smem;                                   // C::kStg x 32 KB
  unsigned char *operands = smem + C::kStg * kBBytes;              // kStages x (2 x 16 KB + 32 KB)
  uint64_t *stg_full = reinterpret_cast<uint64_t *>(operands + kStages * kStageBytes);
  uint64_t *stg_empty = stg_full + C::kStg;
  uint64_t *full = stg_empty + C::kStg;
  uint64_t *empty = full + kStages;
  uint64_t *done = empty + kStages;
  uint32_t *tmem_base_slot = reinterpret_cast<uint32_t *>(done + 1);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_base_slot + 1);
  float *bsum = reinterpret_cast<float *>(operands + kStages * kStageBytes + 256);   // kM kMT floats (TF32 b column)

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t s0 = (int64_t)blockIdx.x * (kM * kMT);
  const int64_t n0 = (int64_t)blockIdx.y * kN;
  const int64_t k_begin = (int64_t)blockIdx.z * args.rows_per_split;
  const int64_t k_end = min(args.m, k_begin + args.rows_per_split);
  const int num_it = k_end > k_begin ? (int)((k_end - k_begin + C::kKOp - 1) / C::kKOp) : 0;
  const int64_t groups = (args.s + 7) / 8;     // Philox blocks per row of the sketch stream

  if (threadIdx.x == 0) {
    for (int i = 0; i < C::kStg; ++i) {
      tc::mbar_init(&stg_full[i], 1);
      tc::mbar_init(&stg_empty[i], C::kTransWarps);
    }
    for (int i = 0; i < kStages; ++i) {
      tc::mbar_init(&full[i], C::kTransWarps + kRngWarps / (BF16 ? 1 : 2));   // transposers + the stage's drawers
      tc::mbar_init(&empty[i], 1);
    }
    tc::mbar_init(done, 1);
    *abort_flag = 0;
    tc::fence_barrier_init();
  }
  if (warp == 0 && lane == 0) tc::prefetch_tmap(&tmap_a);
  if (warp == 1) tc::tmem_alloc(tmem_base_slot, kTmemCols);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *tmem_base_slot;

  if (warp == 0) {
    // ---------------------------------------------------------------- TMA: A rows into staging (row-major)
    if (lane == 0) {
      int issued = 0;
      for (int is = 0; is < num_it * C::kStgPer; ++is) {
        const int st = is % C::kStg;
        const uint32_t ph = (is / C::kStg) & 1;
        if (*abort_flag || !tc::mbar_wait(&stg_empty[st], ph ^ 1)) {
          *abort_flag = 1;
          rmc_report(args.status, RMC_ETIMEOUT);
          break;
        }
        unsigned char *dst = staging + st * kBBytes;
        tc::mbar_arrive_expect_tx(&stg_full[st], kBBytes);
        const int32_t y = (int32_t)(k_begin + (int64_t)is * kKStage);
#pragma unroll
        for (int atom = 0; atom < kN / 32; ++atom)
          tc::tma_load_2d(dst + atom * kAtomBytes, &tmap_a, (int32_t)(n0 + atom * 32), y, &stg_full[st]);
        ++issued;
      }
      // copies still in flight land before the CTA may exit
      for (int is = issued > C::kStg ? issued - C::kStg : 0; is < issued; ++is)
        (void)tc::mbar_wait(&stg_full[is % C::kStg], (is / C::kStg) & 1);
    }
  } else if (warp == 1) {
    // ---------------------------------------------------------------- MMA issuer
    if (lane == 0) {
      constexpr uint32_t idesc = BF16 ? tc::instr_desc(1, 1, 0, 0, kN, kM) : tc::instr_desc(2, 2, 0, 0, kN, kM);
      for (int it = 0; it < num_it; ++it) {
        const int st = it % kStages;
        const uint32_t ph = (it / kStages) & 1;
        if (*abort_flag || !tc::mbar_wait(&full[st], ph)) {
          *abort_flag = 1;
          rmc_report(args.status, RMC_ETIMEOUT);
          break;
        }
        tc::tc_fence_after();
        const uint32_t base = tc::smem_u32(operands + st * kStageBytes);
        const uint32_t b_addr = base + kMT * kOmegaBytes;
#pragma unroll
        for (int mt = 0; mt < kMT; ++mt)
#pragma unroll
          for (int kk = 0; kk < kKStage / 8; ++kk) {
            const uint64_t adesc = tc::smem_desc(base + mt * kOmegaBytes + kk * 32, 16, 1024, tc::kSwizzle128B);
            const uint64_t bdesc = tc::smem_desc(b_addr + kk * 32, 16, 1024, tc::kSwizzle128B);
            // K = 8 (TF32) or 16 (BF16) per instruction: 32 bytes of each 128-byte row either way
            if (BF16) tc::mma_f16(tmem + mt * kN, adesc, bdesc, idesc, (it > 0 || kk > 0) ? 1u : 0u);
            else tc::mma_tf32(tmem + mt * kN, adesc, bdesc, idesc, (it > 0 || kk > 0) ? 1u : 0u);
          }
        tc::mma_commit(&empty[st]);
      }
      tc::mma_commit(done);   // also issued after an abort: completes once the issued MMAs have
    }
  } else if (warp < C::kRngWarp0) {
    // ---------------------------------------------------------------- transposers: staging -> K-major
    const int tl = (warp - kTransWarp0) * 32 + lane;       // 0 .. 32 kTransWarps - 1
    const int l = tl & 7, grp = tl >> 3;                   // 8 groups of 8 lanes
    int is = 0;                                            // staging buffers consumed
    for (int it = 0; it < num_it; ++it) {
      const int st = it % kStages;
      unsigned char *btile = operands + st * kStageBytes + kMT * kOmegaBytes;
      bool ok = true;
      for (int h = 0; h < C::kStgPer; ++h, ++is) {
        const int sst = is % C::kStg;
        // the first staging buffer of the stage, then the operand buffer (free once its MMAs completed)
        if (!warp_wait(&stg_full[sst], (is / C::kStg) & 1, abort_flag, args.status) ||
            (h == 0 && !warp_wait(&empty[st], ((it / kStages) & 1) ^ 1, abort_flag, args.status))) {
          ok = false;
          break;
        }
        const unsigned char *src = staging + sst * kBBytes;
        if (!BF16) {
          transpose_tile_tf32<kN / 32, C::kTransWarps / 2, false>(src, btile, 0, tl);
        } else {
          // Unit (qk, cq): staging rows 8qk..8qk+7 x columns 4cq..4cq+3, written as BF16 into 16-byte K-chunk
          // 4h + qk of rows 4cq..4cq+3 of the K-major tile.  Lane l of group grp takes cq = 8 grp + 2 (l & 3) +
          // (l >> 2) and qk = (l + d) & 3 in pass d: the 8 lanes read 8 distinct 16-byte chunks (cq mod 8
          // distinct) and write 8 distinct ones ((qk, cq & 1) distinct), so neither side has bank conflicts.
          const int cq = 8 * grp + 2 * (l & 3) + (l >> 2);
          const int cc = cq & 7;
#pragma unroll 2
          for (int d = 0; d < 4; ++d) {
            const int qk = (l + d) & 3;
            float4 v[8];
#pragma unroll
            for (int t = 0; t < 8; ++t)
              v[t] = *reinterpret_cast<const float4 *>(src + grp * kAtomBytes + swz_off(8 * qk + t, cc));
            const int q = 4 * h + qk;
            *reinterpret_cast<uint4 *>(btile + swz_off(4 * cq + 0, q)) =
                make_uint4(pack_bf16x2(v[0].x, v[1].x), pack_bf16x2(v[2].x, v[3].x), pack_bf16x2(v[4].x, v[5].x),
                           pack_bf16x2(v[6].x, v[7].x));
            *reinterpret_cast<uint4 *>(btile + swz_off(4 * cq + 1, q)) =
                make_uint4(pack_bf16x2(v[0].y, v[1].y), pack_bf16x2(v[2].y, v[3].y), pack_bf16x2(v[4].y, v[5].y),
                           pack_bf16x2(v[6].y, v[7].y));
            *reinterpret_cast<uint4 *>(btile + swz_off(4 * cq + 2, q)) =
                make_uint4(pack_bf16x2(v[0].z, v[1].z), pack_bf16x2(v[2].z, v[3].z), pack_bf16x2(v[4].z, v[5].z),
                           pack_bf16x2(v[6].z, v[7].z));
            *reinterpret_cast<uint4 *>(btile + swz_off(4 * cq + 3, q)) =
                make_uint4(pack_bf16x2(v[0].w, v[1].w), pack_bf16x2(v[2].w, v[3].w), pack_bf16x2(v[4].w, v[5].w),
                           pack_bf16x2(v[6].w, v[7].w));
          }
        }
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&stg_empty[sst]);   // this warp's reads of the staging buffer are done
      }
      if (!ok) break;
      tc::fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&full[st]);
    }
  } else {
    // ---------------------------------------------------------------- G^T producers (+ b column)
    // Each K-row of a stage takes one Philox block of the sketch stream per group of 8 sketch rows (8 normals),
    // and each thread draws 4 K-rows of one group, so a sketch row's 4 values land together in the K-major tile.
    //   TF32: 32 K-rows per stage, covered by 8 warps: warps 4-11 draw the even stages and warps 12-19 the odd
    //         ones (four independent Philox blocks per thread, and two stage times to draw them).  Thread = (K-row
    //         quad kq = lane mod 8: one whole 16-byte K-chunk; group 4 (warp mod 8) + lane / 8 of the 32 groups of
    //         the two tiles).
    //   BF16: 64 K-rows per stage, all 16 warps on every stage.  Thread = (K-row quad kq = lane mod 16: one 8-byte
    //         half of a 16-byte K-chunk; group 2 (warp mod 8) + lane / 16 of tile warp / 8).
    const int rw = warp - C::kRngWarp0;                        // 0..15
    constexpr int kTurns = BF16 ? 1 : 2;                    // warp groups taking turns on the stages
    const int turn = BF16 ? 0 : rw >> 3;
    const int kq = BF16 ? (lane & 15) : (lane & 7);
    const int g8all = BF16 ? (rw >> 3) * 16 + 2 * (rw & 7) + (lane >> 4) : 4 * (rw & 7) + (lane >> 3);
    const int mt = g8all >> 4, g8 = g8all & 15;             // sketch tile, group of 8 sketch rows within it
    const bool with_b = args.b != nullptr && blockIdx.y == 0;
    const uint64_t gidx = (uint64_t)((s0 + mt * kM) / 8 + g8);
    float bacc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int it = turn; it < num_it; it += kTurns) {
      const int st = it % kStages;
      const int64_t row0 = k_begin + (int64_t)it * C::kKOp + 4 * kq;
      // b for this stage's rows, loaded first so its latency hides behind the draws
      float bv[4] = {0.f, 0.f, 0.f, 0.f};
      if (with_b) {
#pragma unroll
        for (int t = 0; t < 4; ++t)
          if (row0 + t < k_end) bv[t] = __ldg(args.b + (row0 + t) * args.ldb);
      }
      float z[4][8];
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int64_t row = row0 + t;
        if (row < k_end) {
          const uint4 w =
              philox_block_wide(args.seed, kStreamGaussSketch, args.instance, (uint64_t)row * groups + gidx);
          const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const float2 p = box_muller16_fast(ws[q]);
            z[t][2 * q] = p.x;
            z[t][2 * q + 1] = p.y;
          }
        } else {
#pragma unroll
          for (int q = 0; q < 8; ++q) z[t][q] = 0.f;
        }
      }
      if (with_b) {
#pragma unroll
        for (int t = 0; t < 4; ++t)
#pragma unroll
          for (int jj = 0; jj < 8; ++jj) bacc[jj] = fmaf(z[t][jj], bv[t], bacc[jj]);
      }
      if (!warp_wait(&empty[st], ((it / kStages) & 1) ^ 1, abort_flag, args.status)) break;
      unsigned char *otile = operands + st * kStageBytes + mt * kOmegaBytes;
#pragma unroll
      for (int jj = 0; jj < 8; ++jj) {
        const int r = 8 * g8 + jj;
        if (BF16)
          *reinterpret_cast<uint2 *>(otile + swz_off(r, kq >> 1) + 8 * (kq & 1)) =
              make_uint2(pack_bf16x2(z[0][jj], z[1][jj]), pack_bf16x2(z[2][jj], z[3][jj]));
        else
          *reinterpret_cast<float4 *>(otile + swz_off(r, kq)) =
              make_float4(to_tf32(z[0][jj]), to_tf32(z[1][jj]), to_tf32(z[2][jj]), to_tf32(z[3][jj]));
      }
      tc::fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&full[st]);
    }
    if (with_b) {
      // sum over the lanes (K-row quads) that share a group, then over the warp groups that took turns, and
      // write the b column of the partial
      constexpr int kLanes = BF16 ? 16 : 8;
#pragma unroll
      for (int jj = 0; jj < 8; ++jj)
#pragma unroll
        for (int o = 1; o < kLanes; o <<= 1) bacc[jj] += __shfl_xor_sync(0xffffffffu, bacc[jj], o);
      if (!BF16) {
        if (turn == 0 && kq == 0) {
#pragma unroll
          for (int jj = 0; jj < 8; ++jj) bsum[mt * kM + 8 * g8 + jj] = bacc[jj];
        }
        asm volatile("bar.sync 1, %0;" ::"r"(32 * kRngWarps) : "memory");   // the producer warps only
        if (turn == 1 && kq == 0) {
#pragma unroll
          for (int jj = 0; jj < 8; ++jj) bacc[jj] += bsum[mt * kM + 8 * g8 + jj];
        }
      }
      if (turn == kTurns - 1 && kq == 0) {
        float *pb = args.part + ((int64_t)blockIdx.z * args.s) * args.ntot;
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) {
          const int64_t srow = s0 + mt * kM + 8 * g8 + jj;
          if (srow < args.s) pb[srow * args.ntot + args.n] = bacc[jj];
        }
      }
    }
    // ---------------------------------------------------------------- epilogue: warps 4-7 tile 0, 8-11 tile 1
    if ((rw & 7) < 4) {
      const int et = rw >> 3;                    // accumulator (sketch tile) this warp drains
      const int q = warp & 3;                    // TMEM lane quarter this warp may access
      const bool ok = warp_wait(done, 0, abort_flag, args.status);
      tc::tc_fence_after();
      const int64_t ncols = min((int64_t)kN, args.n - n0);
      if (ok) {
        const int64_t srow = s0 + et * kM + q * 32 + lane;
        float *prow = args.part + ((int64_t)blockIdx.z * args.s + srow) * args.ntot + n0;
#pragma unroll 1
        for (int c0 = 0; c0 < kN; c0 += 32) {
          float v[32];
          if (num_it > 0) {
            tc::tmem_ld32(tmem + (uint32_t)(et * kN) + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, v);
          } else {
#pragma unroll
            for (int i = 0; i < 32; ++i) v[i] = 0.f;   // empty row range: nothing was accumulated
          }
          if (srow < args.s) {
#pragma unroll
            for (int i = 0; i < 32; ++i)
              if (c0 + i < ncols) prow[c0 + i] = v[i];
          }
        }
      }
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, kTmemCols);
  }
}

// Drawing alone (the bound of the sketch kernel's producers): Philox blocks b = 0 .. m ceil(s / 8) - 1 of the
// sketch stream (block b is (row b / ceil(s / 8), group b mod ceil(s / 8)) of the operator), each turned into
// eight normals as the producers do and rounded to TF32, summed per thread; 16 warps per CTA, one CTA per SM.
__global__ void __launch_bounds__(512, 1) draw_floor_kernel(uint64_t seed, int64_t blocks, double *part) {
  float acc = 0.f;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t blk = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; blk < blocks; blk += stride) {
    const uint4 w = philox_block(seed, kStreamGaussSketch, 0, (uint64_t)blk);
    const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float2 p = box_muller16_fast(ws[q]);
      acc += to_tf32(p.x) + to_tf32(p.y);
    }
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) part[blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32] = acc;
}

__global__ void draw_floor_sum_kernel(const double *part, int n, double *sum) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += part[i];
    *sum = s;
  }
}

__global__ void tc_reduce_kernel(const float *__restrict__ part, int splits, int64_t s, int64_t n, int64_t ntot,
                                 float scale, float *__restrict__ C, int64_t ldc, float *__restrict__ Cb,
                                 int64_t ldcb) {
  const int64_t total = s * ntot;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    float acc = 0.f;
    for (int t = 0; t < splits; ++t) acc += part[t * total + e];
    const int64_t r = e / ntot, c = e - r * ntot;
    if (c < n) C[r * ldc + c] = acc * scale;
    else Cb[r * ldcb] = acc * scale;
  }
}

// ------------------------------------------------------------------------------------------ host side

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    else
      (void)cudaGetLastError();
  }
  return fn;
}

// Row-major FP32 matrix (rows x cols, leading dimension ld) as a 2-D tensor with a 32 x box_rows box and
// 128-byte swizzle.
int make_tmap(CUtensorMap *map, const float *base, int64_t rows, int64_t cols, int64_t ld, int box_rows) {
  PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
  if (!fn) return RMC_ECUDA;
  if ((reinterpret_cast<uintptr_t>(base) & 15) || ((ld * 4) & 15)) return RMC_EALIGN;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * 4)};
  cuuint32_t box[2] = {32, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? RMC_OK : RMC_EALIGN;
}

// Row ranges per output tile so that tiles x splits fills whole waves of one CTA per SM.
int tc_splits(int64_t m, int64_t tiles, int num_sms) {
  const int64_t max_splits = (m + 2047) / 2048;
  for (int waves = 1; waves <= 8; ++waves) {
    int64_t sp = (int64_t)waves * num_sms / tiles;
    if (sp < 1) sp = 1;
    if (sp > max_splits) return (int)(max_splits < 1 ? 1 : max_splits);
    const int64_t ctas = sp * tiles;
    const int64_t w = (ctas + num_sms - 1) / num_sms;
    if ((double)ctas / (double)(w * num_sms) >= 0.95) return (int)sp;
  }
  int64_t sp = 8LL * num_sms / tiles;
  if (sp > max_splits) sp = max_splits;
  return (int)(sp < 1 ? 1 : sp);
}

}  // namespace

int rmc_tc_available(void) { return encode_fn() != nullptr; }

// Row-major FP32 matrix as a 2-D tensor with a box_cols x box_rows box and no swizzle (rows of the box packed
// densely in shared memory); box_cols * 4 must be a multiple of 16 bytes.
int rmc_make_tmap_dense(CUtensorMap *map, const float *base, int64_t rows, int64_t cols, int64_t ld, int box_cols,
                        int box_rows) {
  PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
  if (!fn) return RMC_ECUDA;
  if ((reinterpret_cast<uintptr_t>(base) & 15) || ((ld * 4) & 15) || ((box_cols * 4) & 15)) return RMC_EALIGN;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * 4)};
  cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? RMC_OK : RMC_EALIGN;
}

// Split count for a sketch of s rows and ntot output columns (the same formula sizes the workspace).
// Split count from the number of output tiles; ntot may include the b column, so the column-tile count is
// estimated as floor(ntot / 256) (exact for the usual n = 256 * k with or without b).  The workspace and the
// launch use this same function, so they always agree.
int gauss_splits_tc(int64_t m, int64_t ntot, int64_t s, int num_sms) {
  const int64_t nt = ntot / kN > 0 ? ntot / kN : 1;
  return tc_splits(m, ((s + kM * kMT - 1) / (kM * kMT)) * nt, num_sms);
}

// ntot = n + 1 when b is sketched as well; the b column does not change the tiling.
size_t rmc_tc_gauss_ws(int64_t m, int64_t ntot, int64_t s, int prec, int num_sms) {
  (void)prec;
  return sizeof(float) * (size_t)gauss_splits_tc(m, ntot, s, num_sms) * s * ntot + 256;
}

int rmc_tc_gauss_sketch(rmc_ctx *ctx, const float *A, int64_t m, int64_t n, int64_t lda, const float *b, int64_t s,
                        uint64_t seed, uint32_t instance, int prec, float *C, int64_t ldc, float *Cb, void *ws) {
  if (prec != RMC_TF32 && prec != RMC_BF16) return RMC_EINVAL;
  const bool bf16 = prec == RMC_BF16;
  const int kop = bf16 ? GaussCfg<true>::kKOp : GaussCfg<false>::kKOp;
  const int64_t ntot = n + (b ? 1 : 0);
  // A matrix with one column past a multiple of 256 (an augmented [A, b] sketched as one matrix): its last column
  // is folded in by the drawing warps like b, instead of a second column tile that would draw every normal again
  int64_t ldb = 1, ldcb = 1;
  if (!b && n > kN && n % kN == 1) {
    b = A + (n - 1);
    ldb = lda;
    Cb = C + (n - 1);
    ldcb = ldc;
    --n;
  }
  CUtensorMap map;
  RMC_TRY(make_tmap(&map, A, m, n, lda, kKStage));
  const int64_t mt = (s + kM * kMT - 1) / (kM * kMT), nt = (n + kN - 1) / kN;
  // the same count the workspace was sized with (gauss_splits_tc of ntot)
  const int splits = gauss_splits_tc(m, ntot, s, ctx->num_sms);
  int64_t rows = (m + splits - 1) / splits;
  rows = (rows + kop - 1) / kop * kop;
  GaussArgs a;
  a.b = b;
  a.ldb = ldb;
  a.m = m;
  a.n = n;
  a.ntot = ntot;
  a.s = s;
  a.seed = seed;
  a.instance = instance;
  a.rows_per_split = rows;
  a.part = static_cast<float *>(ws);
  a.status = ctx->d_status;
  const dim3 grid((unsigned)mt, (unsigned)nt, (unsigned)splits);
  if (bf16) {
    constexpr size_t smem = GaussCfg<true>::kSmem;
    RMC_TRY_CUDA(rmc_allow_smem(tc_gauss_kernel<true>, smem));
    RmcProf prof(ctx, RMC_K_GAUSSIAN);
    tc_gauss_kernel<true><<<grid, GaussCfg<true>::kThreads, smem, ctx->stream>>>(map, a);
  } else {
    constexpr size_t smem = GaussCfg<false>::kSmem;
    RMC_TRY_CUDA(rmc_allow_smem(tc_gauss_kernel<false>, smem));
    RmcProf prof(ctx, RMC_K_GAUSSIAN);
    tc_gauss_kernel<false><<<grid, GaussCfg<false>::kThreads, smem, ctx->stream>>>(map, a);
  }
  tc_reduce_kernel<<<rmc_blocks(s * ntot, 256, 8192), 256, 0, ctx->stream>>>(
      static_cast<float *>(ws), splits, s, n, ntot, 1.0f / sqrtf((float)s), C, ldc, Cb, ldcb);
  rmc_note_launch(2);
  RMC_LAUNCH_CHECK();
  return RMC_OK;
}

extern "C" int rmc_gaussian_draw_floor(rmc_ctx *ctx, int64_t m, int64_t s, uint64_t seed, double *sum) {
  if (!ctx || !sum || m < 1 || s < 1 || m > (int64_t(1) << 31) || s > (int64_t(1) << 31)) return RMC_EINVAL;
  const int grid = ctx->num_sms;
  const int nparts = grid * 16;
  RMC_TRY(rmc_ws_reserve(ctx, sizeof(double) * (size_t)nparts));
  double *part = static_cast<double *>(ctx->ws);
  draw_floor_kernel<<<grid, 512, 0, ctx->stream>>>(seed, m * ((s + 7) / 8), part);
  draw_floor_sum_kernel<<<1, 32, 0, ctx->stream>>>(part, nparts, sum);
  rmc_note_launch(2);
  RMC_LAUNCH_CHECK();
  return RMC_OK;
}

namespace {

// =========================================================================== products with A for the rSVD
// Y = A X (rmc_matmul_an): A tiles (128 rows x 32 columns) and X^T tiles (N rows x 32) both arrive K-major
// through TMA; one CTA owns 128 rows of Y and runs the whole reduction over the n columns of A.
// W = X^T A (rmc_matmul_at): X^T tiles by TMA (K-major), A tiles staged by TMA and transposed on chip (as in
// the Gaussian kernel); split-K over the rows of A with a fixed-order reduction.
//
// X3 (RMC_TF32X3): every FP32 operand v is split into a TF32 head h (v with its 13 low mantissa bits cleared,
// exactly what the tensor core reads) and the remainder v - h (exact in FP32), and each k-step issues three
// MMAs: A_h X_h into one accumulator, the cross terms A_h X_l + A_l X_h into a second (their own rounding is
// then ~2^-11 smaller than the main chain's), summed with round-to-nearest in the epilogue.  The dropped A_l X_l and the TF32 reading of the
// remainders leave about 2^-21 relative error per product instead of TF32's 2^-11.  X's head and remainder are
// split once in global memory; A's are split on chip (converter warps for Y = A X, the transposer warps for
// W = X^T A, which write both parts of the transposed tile).


constexpr int kAnThreads = 256;   // warp 0 TMA, warp 1 MMA, warps 4-7 epilogue (X3: warps 2-7 also split A)
constexpr int kAnConvWarps = 6;   // warps 2-7
constexpr size_t kSmemCap = 227 * 1024;

template <int NPAD, bool X3>
struct AnCfg {
  static constexpr int kA = 128 * 128;                 // 128 rows x 32 TF32
  static constexpr int kX = NPAD * 128;                // NPAD rows x 32 TF32
  static constexpr int kStage = (X3 ? 2 : 1) * (kA + kX);
  static constexpr int kFit = (int)((kSmemCap - 2048) / kStage);
  static constexpr int kStages = kFit > 4 ? 4 : kFit;
  static constexpr size_t kSmem = 1024 + (size_t)kStages * kStage + 256;
};

template <int NPAD, bool X3>
__global__ void __launch_bounds__(kAnThreads, 1) tc_an_kernel(const __grid_constant__ CUtensorMap tmap_a,
                                                              const __grid_constant__ CUtensorMap tmap_xt,
                                                              const __grid_constant__ CUtensorMap tmap_xl,
                                                              int64_t m, int64_t n, int64_t l, float *Y,
                                                              int64_t ldy, int64_t cols_per_split, int *status) {
  using Cfg = AnCfg<NPAD, X3>;
  constexpr int kS = Cfg::kStages;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char *smem = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                          ~uintptr_t(1023));
  // stage: A head | X^T head | (X3) A remainder | X^T remainder
  uint64_t *full = reinterpret_cast<uint64_t *>(smem + kS * Cfg::kStage);
  uint64_t *conv = full + kS;
  uint64_t *empty = conv + kS;
  uint64_t *done = empty + kS;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done + 1);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t row0 = (int64_t)blockIdx.x * 128;
  // split-K: this CTA reduces over columns [k0, k1) of A; its partial goes to Y + blockIdx.y * m * ldy
  const int64_t k0 = (int64_t)blockIdx.y * cols_per_split, k1 = min(n, k0 + cols_per_split);
  const int num_it = k1 > k0 ? (int)((k1 - k0 + kKStage - 1) / kKStage) : 0;
  Y += (int64_t)blockIdx.y * m * ldy;
  // X3: the cross terms accumulate in a second accumulator (columns NPAD..2 NPAD-1), see tc_an's epilogue
  constexpr uint32_t kCols = (X3 ? 2 : 1) * (NPAD < 32 ? 32 : NPAD);
  constexpr int kHalf = Cfg::kA + Cfg::kX;

  if (threadIdx.x == 0) {
    for (int i = 0; i < kS; ++i) {
      tc::mbar_init(&full[i], 1);
      tc::mbar_init(&conv[i], kAnConvWarps);
      tc::mbar_init(&empty[i], 1);
    }
    tc::mbar_init(done, 1);
    *abort_flag = 0;
    tc::fence_barrier_init();
  }
  if (warp == 0 && lane == 0) {
    tc::prefetch_tmap(&tmap_a);
    tc::prefetch_tmap(&tmap_xt);
    if (X3) tc::prefetch_tmap(&tmap_xl);
  }
  if (warp == 1) tc::tmem_alloc(tmem_slot, kCols);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      int issued = 0;
      for (int it = 0; it < num_it; ++it) {
        const int st = it % kS;
        if (*abort_flag || !tc::mbar_wait(&empty[st], ((it / kS) & 1) ^ 1)) {
          *abort_flag = 1;
          rmc_report(status, RMC_ETIMEOUT);
          break;
        }
        unsigned char *stage = smem + st * Cfg::kStage;
        tc::mbar_arrive_expect_tx(&full[st], X3 ? Cfg::kA + 2 * Cfg::kX : Cfg::kA + Cfg::kX);
        const int32_t kx = (int32_t)(k0 + (int64_t)it * kKStage);
        tc::tma_load_2d(stage, &tmap_a, kx, (int32_t)row0, &full[st]);
        tc::tma_load_2d(stage + Cfg::kA, &tmap_xt, kx, 0, &full[st]);
        if (X3) tc::tma_load_2d(stage + kHalf + Cfg::kA, &tmap_xl, kx, 0, &full[st]);
        ++issued;
      }
      for (int it = issued > kS ? issued - kS : 0; it < issued; ++it)
        (void)tc::mbar_wait(&full[it % kS], (it / kS) & 1);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = tc::instr_desc(2, 2, 0, 0, NPAD, 128);
      for (int it = 0; it < num_it; ++it) {
        const int st = it % kS;
        if (*abort_flag || !tc::mbar_wait(X3 ? &conv[st] : &full[st], (it / kS) & 1)) {
          *abort_flag = 1;
          rmc_report(status, RMC_ETIMEOUT);
          break;
        }
        tc::tc_fence_after();
        const uint32_t a_addr = tc::smem_u32(smem + st * Cfg::kStage);
        const uint32_t x_addr = a_addr + Cfg::kA;
#pragma unroll
        for (int kk = 0; kk < kKStage / 8; ++kk) {
          const uint64_t ah = tc::smem_desc(a_addr + kk * 32, 16, 1024, tc::kSwizzle128B);
          const uint64_t xh = tc::smem_desc(x_addr + kk * 32, 16, 1024, tc::kSwizzle128B);
          tc::mma_tf32(tmem, ah, xh, idesc, (it > 0 || kk > 0) ? 1u : 0u);
          if (X3) {
            const uint64_t al = tc::smem_desc(a_addr + kHalf + kk * 32, 16, 1024, tc::kSwizzle128B);
            const uint64_t xl = tc::smem_desc(x_addr + kHalf + kk * 32, 16, 1024, tc::kSwizzle128B);
            tc::mma_tf32(tmem + NPAD, ah, xl, idesc, (it > 0 || kk > 0) ? 1u : 0u);
            tc::mma_tf32(tmem + NPAD, al, xh, idesc, 1u);
          }
        }
        tc::mma_commit(&empty[st]);
      }
      tc::mma_commit(done);
    }
  } else {
    if (X3) {
      // warps 2-7: split each landed A tile into its TF32 head (in place) and remainder (second half)
      const int ct = threadIdx.x - 64;
      for (int it = 0; it < num_it; ++it) {
        const int st = it % kS;
        if (!warp_wait(&full[st], (it / kS) & 1, abort_flag, status)) break;
        unsigned char *a_tile = smem + st * Cfg::kStage;
        for (int c = ct; c < Cfg::kA / 16; c += 32 * kAnConvWarps) {
          float4 *hp = reinterpret_cast<float4 *>(a_tile) + c;
          float4 h, lo;
          split4(*hp, h, lo);
          *hp = h;
          *(reinterpret_cast<float4 *>(a_tile + kHalf) + c) = lo;
        }
        tc::fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&conv[st]);
      }
    }
    if (warp >= 4) {
      const int q = warp & 3;
      const bool ok = warp_wait(done, 0, abort_flag, status);
      tc::tc_fence_after();
      const int64_t row = row0 + q * 32 + lane;
      if (ok) {
#pragma unroll 1
        for (int c0 = 0; c0 < NPAD; c0 += 32) {
          float v[32];
          if (num_it > 0) {
            tc::tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, v);
            if (X3) {
              // main chain + cross terms, added with round-to-nearest
              float w[32];
              tc::tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(NPAD + c0), w);
#pragma unroll
              for (int i = 0; i < 32; ++i) v[i] += w[i];
            }
          } else {
#pragma unroll
            for (int i = 0; i < 32; ++i) v[i] = 0.f;   // an empty column range accumulated nothing
          }
          if (row < m) {
#pragma unroll
            for (int i = 0; i < 32; ++i)
              if (c0 + i < l) Y[row * ldy + c0 + i] = v[i];
          }
        }
      }
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, kCols);
  }
}

// W = X^T A over a row range of A: A_op = X^T tiles (MT x 128 rows of l, K-major via TMA), B_op = A tile
// (NC columns) staged by TMA and transposed to K-major by warps 2-3.  Partial sums per row range.  X3: the
// X^T remainder arrives by a second TMA, the transposers write the A tile's head and remainder.
constexpr int kAtTrans = 4;       // transposer warps of tc_at_kernel (warps 2-5; 4 and 5 join the epilogue)

template <int MT, bool X3>
struct AtCfg {
  static constexpr int NC = X3 ? 128 : 256;            // columns of A per CTA (the MMA's N)
  static constexpr int kStg = NC * kKStage * 4;        // staging / transposed tile bytes
  static constexpr int kXt = MT * kOmegaBytes;         // MT x (128 rows x 32 TF32)
  static constexpr int kHalf = kXt + kStg;
  static constexpr int kStage = (X3 ? 2 : 1) * kHalf;
  // staging ring: as many 32-row buffers of A as fit beside the operand stages, up to four, so that the loads of
  // A run ahead of the transpose by more than the two operand stages
  static constexpr int kFitRing = (int)((kSmemCap - 1024 - 256 - (size_t)kStages * kStage) / kStg);
  static constexpr int kRing = kFitRing > 4 ? 4 : kFitRing;
  static constexpr size_t kSmem = 1024 + (size_t)kRing * kStg + (size_t)kStages * kStage + 256;
  static_assert(kRing >= 2 && kSmem <= kSmemCap, "tc_at_kernel shared memory");
};

template <int MT, bool X3>
__global__ void __launch_bounds__(32 * (4 + 4 * MT), 1) tc_at_kernel(const __grid_constant__ CUtensorMap tmap_a,
                                                                     const __grid_constant__ CUtensorMap tmap_xt,
                                                                     const __grid_constant__ CUtensorMap tmap_xl,
                                                                     int64_t m, int64_t n, int64_t l,
                                                                     int64_t rows_per_split, float *part,
                                                                     int *status) {
  using Cfg = AtCfg<MT, X3>;
  constexpr int NC = Cfg::NC;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char *smem = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                          ~uintptr_t(1023));
  unsigned char *staging = smem;
  constexpr int R = Cfg::kRing;
  unsigned char *operands = smem + R * Cfg::kStg;
  uint64_t *stg_full = reinterpret_cast<uint64_t *>(operands + kStages * Cfg::kStage);
  uint64_t *stg_empty = stg_full + R;
  uint64_t *full = stg_empty + R;
  uint64_t *empty = full + kStages;
  uint64_t *done = empty + kStages;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done + 1);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t n0 = (int64_t)blockIdx.x * NC;
  const int64_t k_begin = (int64_t)blockIdx.z * rows_per_split;
  const int64_t k_end = min(m, k_begin + rows_per_split);
  const int num_it = k_end > k_begin ? (int)((k_end - k_begin + kKStage - 1) / kKStage) : 0;
  // X3: the cross terms accumulate in a second set of accumulators (columns MT NC .. 2 MT NC - 1)
  constexpr uint32_t kCols = (X3 ? 2 : 1) * MT * NC;

  if (threadIdx.x == 0) {
    for (int i = 0; i < R; ++i) {
      tc::mbar_init(&stg_full[i], 1);
      tc::mbar_init(&stg_empty[i], kAtTrans);
    }
    for (int i = 0; i < kStages; ++i) {
      tc::mbar_init(&full[i], kAtTrans + 1);         // the transposer warps + the X^T TMA arrival
      tc::mbar_init(&empty[i], 1);
    }
    tc::mbar_init(done, 1);
    *abort_flag = 0;
    tc::fence_barrier_init();
  }
  if (warp == 0 && lane == 0) {
    tc::prefetch_tmap(&tmap_a);
    tc::prefetch_tmap(&tmap_xt);
    if (X3) tc::prefetch_tmap(&tmap_xl);
  }
  if (warp == 1) tc::tmem_alloc(tmem_slot, kCols);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      int ia = 0;   // A tiles issued into the staging ring (up to R - 1 stages ahead of the operand stage)
      bool ok = true;
      for (int it = 0; it < num_it && ok; ++it) {
        const int st = it % kStages;
        for (; ia < num_it && ia < it + R; ++ia) {
          const int sst = ia % R;
          if (*abort_flag || !tc::mbar_wait(&stg_empty[sst], ((ia / R) & 1) ^ 1)) {
            ok = false;
            break;
          }
          const int32_t ya = (int32_t)(k_begin + (int64_t)ia * kKStage);
          unsigned char *dst = staging + sst * Cfg::kStg;
          tc::mbar_arrive_expect_tx(&stg_full[sst], Cfg::kStg);
#pragma unroll
          for (int atom = 0; atom < NC / 32; ++atom)
            tc::tma_load_2d(dst + atom * kAtomBytes, &tmap_a, (int32_t)(n0 + atom * 32), ya, &stg_full[sst]);
        }
        if (!ok || *abort_flag || !tc::mbar_wait(&empty[st], ((it / kStages) & 1) ^ 1)) {
          ok = false;
          break;
        }
        const int32_t y = (int32_t)(k_begin + (int64_t)it * kKStage);
        unsigned char *xt = operands + st * Cfg::kStage;
        tc::mbar_arrive_expect_tx(&full[st], (X3 ? 2 : 1) * Cfg::kXt);
#pragma unroll
        for (int mt = 0; mt < MT; ++mt) {
          tc::tma_load_2d(xt + mt * kOmegaBytes, &tmap_xt, y, mt * 128, &full[st]);
          if (X3) tc::tma_load_2d(xt + Cfg::kHalf + mt * kOmegaBytes, &tmap_xl, y, mt * 128, &full[st]);
        }
      }
      if (!ok) {
        *abort_flag = 1;
        rmc_report(status, RMC_ETIMEOUT);
      }
      // copies still in flight land before the CTA may exit
      for (int k = ia > R ? ia - R : 0; k < ia; ++k) (void)tc::mbar_wait(&stg_full[k % R], (k / R) & 1);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = tc::instr_desc(2, 2, 0, 0, NC, kM);
      for (int it = 0; it < num_it; ++it) {
        const int st = it % kStages;
        if (*abort_flag || !tc::mbar_wait(&full[st], (it / kStages) & 1)) {
          *abort_flag = 1;
          rmc_report(status, RMC_ETIMEOUT);
          break;
        }
        tc::tc_fence_after();
        const uint32_t base = tc::smem_u32(operands + st * Cfg::kStage);
        const uint32_t b_addr = base + Cfg::kXt;
#pragma unroll
        for (int mt = 0; mt < MT; ++mt)
#pragma unroll
          for (int kk = 0; kk < kKStage / 8; ++kk) {
            const uint64_t xh = tc::smem_desc(base + mt * kOmegaBytes + kk * 32, 16, 1024, tc::kSwizzle128B);
            const uint64_t ah = tc::smem_desc(b_addr + kk * 32, 16, 1024, tc::kSwizzle128B);
            tc::mma_tf32(tmem + mt * NC, xh, ah, idesc, (it > 0 || kk > 0) ? 1u : 0u);
            if (X3) {
              const uint64_t xl =
                  tc::smem_desc(base + Cfg::kHalf + mt * kOmegaBytes + kk * 32, 16, 1024, tc::kSwizzle128B);
              const uint64_t al = tc::smem_desc(b_addr + Cfg::kHalf + kk * 32, 16, 1024, tc::kSwizzle128B);
              tc::mma_tf32(tmem + (MT + mt) * NC, xh, al, idesc, (it > 0 || kk > 0) ? 1u : 0u);
              tc::mma_tf32(tmem + (MT + mt) * NC, xl, ah, idesc, 1u);
            }
          }
        tc::mma_commit(&empty[st]);
      }
      tc::mma_commit(done);
    }
  } else {
   if (warp < 2 + kAtTrans) {
    // transposers: staging (row-major, swizzled) -> K-major B tile, 16 groups of 8 lanes in two halves; X3 also
    // writes the remainder tile
    static_assert(kAtTrans == 4, "two halves of 8 lane groups");
    const int tl = (warp - 2) * 32 + lane;
    for (int it = 0; it < num_it; ++it) {
      const int st = it % kStages, sst = it % R;
      if (!warp_wait(&stg_full[sst], (it / R) & 1, abort_flag, status)) break;
      if (!warp_wait(&empty[st], ((it / kStages) & 1) ^ 1, abort_flag, status)) break;
      const unsigned char *src = staging + sst * Cfg::kStg;
      unsigned char *btile = operands + st * Cfg::kStage + Cfg::kXt;
      transpose_tile_tf32<NC / 32, 2, X3>(src, btile, Cfg::kHalf, tl);
      tc::fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) {
        tc::mbar_arrive(&stg_empty[sst]);
        tc::mbar_arrive(&full[st]);
      }
    }
   }
   if (warp >= 4) {
    // epilogue: warps 4.. (MT x 4 warps), accumulator et, lane quarter q
    const int ew = warp - 4, et = ew >> 2, q = warp & 3;
    const bool ok = warp_wait(done, 0, abort_flag, status);
    tc::tc_fence_after();
    const int64_t row = (int64_t)et * kM + q * 32 + lane;    // row of W (index into l)
    const int64_t ncols = min((int64_t)NC, n - n0);
    if (ok) {
      float *prow = part + ((int64_t)blockIdx.z * l + row) * n + n0;
#pragma unroll 1
      for (int c0 = 0; c0 < NC; c0 += 32) {
        float v[32];
        if (num_it > 0) {
          tc::tmem_ld32(tmem + (uint32_t)(et * NC) + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, v);
          if (X3) {
            float w[32];
            tc::tmem_ld32(tmem + (uint32_t)((MT + et) * NC) + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, w);
#pragma unroll
            for (int i = 0; i < 32; ++i) v[i] += w[i];
          }
        } else {
#pragma unroll
          for (int i = 0; i < 32; ++i) v[i] = 0.f;
        }
        if (row < l) {
#pragma unroll
          for (int i = 0; i < 32; ++i)
            if (c0 + i < ncols) prow[c0 + i] = v[i];
        }
      }
    }
  }
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, kCols);
  }
}

// ============================================================================ BF16 products with A
// RMC_BF16: both operands rounded to BF16 (8-bit mantissa), FP32 accumulation in tensor memory (kind::f16).
// A stays FP32 in HBM and is converted on chip; X^T is converted once in global memory.  An operand stage holds
// 64 values of K per 128-byte row (the TF32 stage holds 32), so the MMA issue and the descriptors are those of
// the TF32 kernels with K = 16 per instruction.

// Y = A X: A arrives as two 128 x 32 FP32 boxes per stage; warps 2-7 write its BF16 K-major tile (row r, 16-byte
// K-chunk q from the FP32 chunks 2(q mod 4), 2(q mod 4) + 1 of half q / 4; 8 lanes on 8 rows, so reads and
// writes both hit 8 distinct bank groups); the X^T tile arrives in BF16 by TMA.
template <int NPAD>
struct AnBfCfg {
  static constexpr int kA32 = 128 * 64 * 4;            // FP32 staging: 128 rows x 64 values of K
  static constexpr int kA16 = 128 * 128;               // BF16 operand: 128 rows x 64 values
  static constexpr int kX = NPAD * 128;                // X^T: NPAD rows x 64 BF16
  static constexpr int kStage = kA32 + kA16 + kX;
  static constexpr int kFit = (int)((kSmemCap - 2048) / kStage);
  static constexpr int kStages = kFit > 4 ? 4 : kFit;
  static constexpr size_t kSmem = 1024 + (size_t)kStages * kStage + 256;
};

template <int NPAD>
__global__ void __launch_bounds__(kAnThreads, 1) tc_an_bf16_kernel(const __grid_constant__ CUtensorMap tmap_a,
                                                                   const __grid_constant__ CUtensorMap tmap_x16,
                                                                   int64_t m, int64_t n, int64_t l, float *Y,
                                                                   int64_t ldy, int *status) {
  using Cfg = AnBfCfg<NPAD>;
  constexpr int kS = Cfg::kStages;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char *smem = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                          ~uintptr_t(1023));
  // stage: A FP32 (two 16 KB halves) | A BF16 | X^T BF16
  uint64_t *full = reinterpret_cast<uint64_t *>(smem + kS * Cfg::kStage);
  uint64_t *conv = full + kS;
  uint64_t *empty = conv + kS;
  uint64_t *done = empty + kS;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done + 1);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t row0 = (int64_t)blockIdx.x * 128;
  const int num_it = (int)((n + 63) / 64);
  constexpr uint32_t kCols = NPAD < 32 ? 32 : NPAD;

  if (threadIdx.x == 0) {
    for (int i = 0; i < kS; ++i) {
      tc::mbar_init(&full[i], 1);
      tc::mbar_init(&conv[i], kAnConvWarps);
      tc::mbar_init(&empty[i], 1);
    }
    tc::mbar_init(done, 1);
    *abort_flag = 0;
    tc::fence_barrier_init();
  }
  if (warp == 0 && lane == 0) {
    tc::prefetch_tmap(&tmap_a);
    tc::prefetch_tmap(&tmap_x16);
  }
  if (warp == 1) tc::tmem_alloc(tmem_slot, kCols);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      int issued = 0;
      for (int it = 0; it < num_it; ++it) {
        const int st = it % kS;
        if (*abort_flag || !tc::mbar_wait(&empty[st], ((it / kS) & 1) ^ 1)) {
          *abort_flag = 1;
          rmc_report(status, RMC_ETIMEOUT);
          break;
        }
        unsigned char *stage = smem + st * Cfg::kStage;
        tc::mbar_arrive_expect_tx(&full[st], Cfg::kA32 + Cfg::kX);
        const int32_t kx = (int32_t)((int64_t)it * 64);
        tc::tma_load_2d(stage, &tmap_a, kx, (int32_t)row0, &full[st]);
        tc::tma_load_2d(stage + Cfg::kA32 / 2, &tmap_a, kx + 32, (int32_t)row0, &full[st]);
        tc::tma_load_2d(stage + Cfg::kA32 + Cfg::kA16, &tmap_x16, kx, 0, &full[st]);
        ++issued;
      }
      for (int it = issued > kS ? issued - kS : 0; it < issued; ++it)
        (void)tc::mbar_wait(&full[it % kS], (it / kS) & 1);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = tc::instr_desc(1, 1, 0, 0, NPAD, 128);
      for (int it = 0; it < num_it; ++it) {
        const int st = it % kS;
        if (*abort_flag || !tc::mbar_wait(&conv[st], (it / kS) & 1)) {
          *abort_flag = 1;
          rmc_report(status, RMC_ETIMEOUT);
          break;
        }
        tc::tc_fence_after();
        const uint32_t a_addr = tc::smem_u32(smem + st * Cfg::kStage + Cfg::kA32);
        const uint32_t x_addr = a_addr + Cfg::kA16;
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          const uint64_t ad = tc::smem_desc(a_addr + kk * 32, 16, 1024, tc::kSwizzle128B);
          const uint64_t xd = tc::smem_desc(x_addr + kk * 32, 16, 1024, tc::kSwizzle128B);
          tc::mma_f16(tmem, ad, xd, idesc, (it > 0 || kk > 0) ? 1u : 0u);
        }
        tc::mma_commit(&empty[st]);
      }
      tc::mma_commit(done);
    }
  } else {
    // warps 2-7: FP32 staging -> BF16 K-major operand
    const int ct = threadIdx.x - 64;
    for (int it = 0; it < num_it; ++it) {
      const int st = it % kS;
      if (!warp_wait(&full[st], (it / kS) & 1, abort_flag, status)) break;
      const unsigned char *a32 = smem + st * Cfg::kStage;
      unsigned char *a16 = smem + st * Cfg::kStage + Cfg::kA32;
      for (int e = ct; e < 1024; e += 32 * kAnConvWarps) {
        const int r = ((e >> 6) << 3) | (e & 7), q = (e >> 3) & 7;
        const unsigned char *src = a32 + (q >> 2) * (Cfg::kA32 / 2);
        const float4 u = *reinterpret_cast<const float4 *>(src + swz_off(r, 2 * (q & 3)));
        const float4 v = *reinterpret_cast<const float4 *>(src + swz_off(r, 2 * (q & 3) + 1));
        *reinterpret_cast<uint4 *>(a16 + swz_off(r, q)) =
            make_uint4(pack_bf16x2(u.x, u.y), pack_bf16x2(u.z, u.w), pack_bf16x2(v.x, v.y), pack_bf16x2(v.z, v.w));
      }
      tc::fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&conv[st]);
    }
    if (warp >= 4) {
      const int q = warp & 3;
      const bool ok = warp_wait(done, 0, abort_flag, status);
      tc::tc_fence_after();
      const int64_t row = row0 + q * 32 + lane;
      if (ok) {
#pragma unroll 1
        for (int c0 = 0; c0 < NPAD; c0 += 32) {
          float v[32];
          tc::tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, v);
          if (row < m) {
#pragma unroll
            for (int i = 0; i < 32; ++i)
              if (c0 + i < l) Y[row * ldy + c0 + i] = v[i];
          }
        }
      }
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, kCols);
  }
}

// W = X^T A over a row range of A: the X^T tiles arrive in BF16 by TMA; A is staged in FP32 32 rows at a time
// (two staging buffers per 64-row operand stage) and converted + transposed by warps 2-5 into the BF16 K-major
// tile, with the lane mapping of the BF16 Gaussian kernel (conflict-free reads and writes).
template <int MT>
struct AtBfCfg {
  static constexpr int NC = 256;
  static constexpr int kStg = NC * kKStage * 4;        // 32 KB of FP32 staging per 32 rows
  static constexpr int kXt = MT * 128 * 128;           // MT x (128 rows x 64 BF16)
  static constexpr int kB = NC * 128;                  // NC rows x 64 BF16
  static constexpr int kStage = kXt + kB;
  // staging ring: as many 32-row FP32 buffers as fit beside the operand stages, up to four (two operand stages)
  static constexpr int kFitRing = (int)((kSmemCap - 1024 - 256 - (size_t)kStages * kStage) / kStg);
  static constexpr int kStgRing = kFitRing > 4 ? 4 : kFitRing;
  static constexpr size_t kSmem = 1024 + (size_t)kStgRing * kStg + (size_t)kStages * kStage + 256;
  static_assert(kStgRing >= 2 && kSmem <= kSmemCap, "tc_at_bf16_kernel shared memory");
};

template <int MT>
__global__ void __launch_bounds__(32 * (4 + 4 * MT), 1) tc_at_bf16_kernel(
    const __grid_constant__ CUtensorMap tmap_a, const __grid_constant__ CUtensorMap tmap_x16, int64_t m, int64_t n,
    int64_t l, int64_t rows_per_split, float *part, int *status) {
  using Cfg = AtBfCfg<MT>;
  constexpr int NC = Cfg::NC, kR = Cfg::kStgRing;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char *smem = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                          ~uintptr_t(1023));
  unsigned char *staging = smem;
  unsigned char *operands = smem + kR * Cfg::kStg;
  uint64_t *stg_full = reinterpret_cast<uint64_t *>(operands + kStages * Cfg::kStage);
  uint64_t *stg_empty = stg_full + kR;
  uint64_t *full = stg_empty + kR;
  uint64_t *empty = full + kStages;
  uint64_t *done = empty + kStages;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done + 1);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t n0 = (int64_t)blockIdx.x * NC;
  const int64_t k_begin = (int64_t)blockIdx.z * rows_per_split;
  const int64_t k_end = min(m, k_begin + rows_per_split);
  const int num_it = k_end > k_begin ? (int)((k_end - k_begin + 63) / 64) : 0;
  constexpr uint32_t kCols = MT * NC;

  if (threadIdx.x == 0) {
    for (int i = 0; i < kR; ++i) {
      tc::mbar_init(&stg_full[i], 1);
      tc::mbar_init(&stg_empty[i], kAtTrans);
    }
    for (int i = 0; i < kStages; ++i) {
      tc::mbar_init(&full[i], kAtTrans + 1);         // the transposer warps + the X^T TMA arrival
      tc::mbar_init(&empty[i], 1);
    }
    tc::mbar_init(done, 1);
    *abort_flag = 0;
    tc::fence_barrier_init();
  }
  if (warp == 0 && lane == 0) {
    tc::prefetch_tmap(&tmap_a);
    tc::prefetch_tmap(&tmap_x16);
  }
  if (warp == 1) tc::tmem_alloc(tmem_slot, kCols);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // 32-row staging buffers issued: buffers 2 it and 2 it + 1 hold rows k_begin + 64 it .. +63 of A (row
      // ranges are whole 64-row stages, so a stage never reaches into the next range; rows past m arrive as
      // zeros).  The loads of A run up to kR - 2 buffers ahead of the operand stage, so they do not wait for the
      // MMAs that free the next X^T buffer.
      int issued = 0;
      bool failed = false;
      for (int it = 0; it < num_it && !failed; ++it) {
        const int st = it % kStages;
        for (; issued < 2 * num_it && issued < 2 * it + kR; ++issued) {
          const int sst = issued % kR;
          if (*abort_flag || !tc::mbar_wait(&stg_empty[sst], ((issued / kR) & 1) ^ 1)) {
            failed = true;
            break;
          }
          tc::mbar_arrive_expect_tx(&stg_full[sst], Cfg::kStg);
          const int32_t y = (int32_t)(k_begin + (int64_t)issued * kKStage);
#pragma unroll
          for (int atom = 0; atom < NC / 32; ++atom)
            tc::tma_load_2d(staging + sst * Cfg::kStg + atom * kAtomBytes, &tmap_a, (int32_t)(n0 + atom * 32), y,
                            &stg_full[sst]);
        }
        if (failed || *abort_flag || !tc::mbar_wait(&empty[st], ((it / kStages) & 1) ^ 1)) {
          failed = true;
          break;
        }
        unsigned char *xt = operands + st * Cfg::kStage;
        tc::mbar_arrive_expect_tx(&full[st], Cfg::kXt);
        const int32_t y = (int32_t)(k_begin + (int64_t)it * 64);
#pragma unroll
        for (int mt = 0; mt < MT; ++mt) tc::tma_load_2d(xt + mt * 128 * 128, &tmap_x16, y, mt * 128, &full[st]);
      }
      if (failed) {
        *abort_flag = 1;
        rmc_report(status, RMC_ETIMEOUT);
      }
      for (int is = issued > kR ? issued - kR : 0; is < issued; ++is)
        (void)tc::mbar_wait(&stg_full[is % kR], (is / kR) & 1);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = tc::instr_desc(1, 1, 0, 0, NC, kM);
      for (int it = 0; it < num_it; ++it) {
        const int st = it % kStages;
        if (*abort_flag || !tc::mbar_wait(&full[st], (it / kStages) & 1)) {
          *abort_flag = 1;
          rmc_report(status, RMC_ETIMEOUT);
          break;
        }
        tc::tc_fence_after();
        const uint32_t base = tc::smem_u32(operands + st * Cfg::kStage);
        const uint32_t b_addr = base + Cfg::kXt;
#pragma unroll
        for (int mt = 0; mt < MT; ++mt)
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            const uint64_t xd = tc::smem_desc(base + mt * 128 * 128 + kk * 32, 16, 1024, tc::kSwizzle128B);
            const uint64_t ad = tc::smem_desc(b_addr + kk * 32, 16, 1024, tc::kSwizzle128B);
            tc::mma_f16(tmem + mt * NC, xd, ad, idesc, (it > 0 || kk > 0) ? 1u : 0u);
          }
        tc::mma_commit(&empty[st]);
      }
      tc::mma_commit(done);
    }
  } else {
    if (warp < 2 + kAtTrans) {
      const int tl = (warp - 2) * 32 + lane;             // 0..127
      const int l8 = tl & 7, grp = tl >> 3;              // 16 groups of 8 lanes
      const int atom = grp & 7, dset = grp >> 3;         // two groups per 32-column atom, two passes each
      const int cq = 8 * atom + 2 * (l8 & 3) + (l8 >> 2);
      const int cc = cq & 7;
      int is = 0;
      for (int it = 0; it < num_it; ++it) {
        const int st = it % kStages;
        if (!warp_wait(&empty[st], ((it / kStages) & 1) ^ 1, abort_flag, status)) break;
        unsigned char *btile = operands + st * Cfg::kStage + Cfg::kXt;
        bool ok = true;
        for (int h = 0; h < 2; ++h, ++is) {
          const int sst = is % kR;
          if (!warp_wait(&stg_full[sst], (is / kR) & 1, abort_flag, status)) {
            ok = false;
            break;
          }
          const unsigned char *src = staging + sst * Cfg::kStg;
#pragma unroll
          for (int dd = 0; dd < 2; ++dd) {
            const int qk = (l8 + 2 * dset + dd) & 3;
            float4 v[8];
#pragma unroll
            for (int t = 0; t < 8; ++t)
              v[t] = *reinterpret_cast<const float4 *>(src + atom * kAtomBytes + swz_off(8 * qk + t, cc));
            const int q = 4 * h + qk;
            *reinterpret_cast<uint4 *>(btile + swz_off(4 * cq + 0, q)) =
                make_uint4(pack_bf16x2(v[0].x, v[1].x), pack_bf16x2(v[2].x, v[3].x), pack_bf16x2(v[4].x, v[5].x),
                           pack_bf16x2(v[6].x, v[7].x));
            *reinterpret_cast<uint4 *>(btile + swz_off(4 * cq + 1, q)) =
                make_uint4(pack_bf16x2(v[0].y, v[1].y), pack_bf16x2(v[2].y, v[3].y), pack_bf16x2(v[4].y, v[5].y),
                           pack_bf16x2(v[6].y, v[7].y));
            *reinterpret_cast<uint4 *>(btile + swz_off(4 * cq + 2, q)) =
                make_uint4(pack_bf16x2(v[0].z, v[1].z), pack_bf16x2(v[2].z, v[3].z), pack_bf16x2(v[4].z, v[5].z),
                           pack_bf16x2(v[6].z, v[7].z));
            *reinterpret_cast<uint4 *>(btile + swz_off(4 * cq + 3, q)) =
                make_uint4(pack_bf16x2(v[0].w, v[1].w), pack_bf16x2(v[2].w, v[3].w), pack_bf16x2(v[4].w, v[5].w),
                           pack_bf16x2(v[6].w, v[7].w));
          }
          __syncwarp();
          if (lane == 0) tc::mbar_arrive(&stg_empty[sst]);
        }
        if (!ok) break;
        tc::fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&full[st]);
      }
    }
    if (warp >= 4) {
      const int ew = warp - 4, et = ew >> 2, q = warp & 3;
      const bool ok = warp_wait(done, 0, abort_flag, status);
      tc::tc_fence_after();
      const int64_t row = (int64_t)et * kM + q * 32 + lane;    // row of W (index into l)
      const int64_t ncols = min((int64_t)NC, n - n0);
      if (ok) {
        float *prow = part + ((int64_t)blockIdx.z * l + row) * n + n0;
#pragma unroll 1
        for (int c0 = 0; c0 < NC; c0 += 32) {
          float v[32];
          if (num_it > 0) {
            tc::tmem_ld32(tmem + (uint32_t)(et * NC) + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, v);
          } else {
#pragma unroll
            for (int i = 0; i < 32; ++i) v[i] = 0.f;
          }
          if (row < l) {
#pragma unroll
            for (int i = 0; i < 32; ++i)
              if (c0 + i < ncols) prow[c0 + i] = v[i];
          }
        }
      }
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, kCols);
  }
}

__global__ void sum_parts_kernel(const float *__restrict__ part, int splits, int64_t rows, int64_t cols,
                                 float *__restrict__ W, int64_t ldw) {
  const int64_t total = rows * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    float acc = 0.f;
    for (int t = 0; t < splits; ++t) acc += part[t * total + e];
    W[(e / cols) * ldw + e % cols] = acc;
  }
}

__global__ void transpose32_kernel(const float *__restrict__ in, int64_t rows, int64_t cols, int64_t ldi,
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

// Longest reduction one tensor-memory accumulator takes in the 3xTF32 form.  The tensor core adds each k-step
// into its FP32 accumulator without round-to-nearest, so the rounding error grows with the number of k-steps
// rather than with its square root; capping every chain at 4096 terms (512 k-steps) keeps it near 3e-5 relative,
// and the chains are then summed with ordinary FP32 adds.  The single-TF32 form, whose operand rounding is
// coarser, takes whole reductions.
constexpr int64_t kX3Chain = 4096;

// Column tile of W = X^T A: 128 columns in the 3xTF32 form (both operand halves must fit), 256 otherwise.
int at_cols(bool x3) { return x3 ? 128 : 256; }

int at_splits(int64_t m, int64_t n, bool x3, int num_sms) {
  int sp = tc_splits(m, (n + at_cols(x3) - 1) / at_cols(x3), num_sms);
  // 3xTF32: no accumulator chain longer than kX3Chain rows of A (each split's rows are rounded up to whole
  // 32-row stages, so aim below the cap)
  if (x3) {
    const int64_t need = (m + kX3Chain - 32 - 1) / (kX3Chain - 32);
    if (sp < need) sp = (int)need;
  }
  return sp;
}

int64_t xt_ld(int64_t rows) { return (rows + 3) / 4 * 4; }   // 16-byte row pitch for TMA

// In place: Xt (rows x cols, ld) <- its TF32 head; Xl <- the remainder (3xTF32 operand split).
__global__ void split_tf32_kernel(float *Xt, int64_t rows, int64_t cols, int64_t ld, float *Xl) {
  const int64_t total = rows * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / cols, c = e - r * cols;
    const float v = Xt[r * ld + c], h = tf32_head(v);
    Xt[r * ld + c] = h;
    Xl[r * ld + c] = v - h;
  }
}

int an_splits(int64_t n, bool x3) { return x3 ? (int)((n + kX3Chain - 1) / kX3Chain) : 1; }

template <int NP, bool X3>
int an_launch(rmc_ctx *ctx, const CUtensorMap &ma, const CUtensorMap &mx, const CUtensorMap &ml, int64_t m,
              int64_t n, int64_t l, float *Y, int64_t ldy, int splits) {
  const size_t smem = AnCfg<NP, X3>::kSmem;
  RMC_TRY_CUDA(rmc_allow_smem(tc_an_kernel<NP, X3>, smem));
  int64_t per = (n + splits - 1) / splits;
  per = (per + kKStage - 1) / kKStage * kKStage;
  tc_an_kernel<NP, X3><<<dim3((unsigned)((m + 127) / 128), (unsigned)splits), kAnThreads, smem, ctx->stream>>>(
      ma, mx, ml, m, n, l, Y, ldy, per, ctx->d_status);
  return RMC_OK;
}

// Launch Y = A X with X^T (l x n) given (X3: Xt holds the heads, Xl the remainders); l <= 256.  With more
// than one K split the partial products go to part (splits x m x l) and are summed into Y in split order.
int launch_an_t(rmc_ctx *ctx, const float *A, int64_t m, int64_t n, int64_t lda, const float *Xt, const float *Xl,
                int64_t l, int64_t ldxt, float *Y, int64_t ldy, bool x3, float *part) {
  const int splits = an_splits(n, x3);
  CUtensorMap ma, mx, ml;
  const int npad = l <= 32 ? 32 : l <= 64 ? 64 : l <= 128 ? 128 : 256;
  RMC_TRY(make_tmap(&ma, A, m, n, lda, 128));
  RMC_TRY(make_tmap(&mx, Xt, l, n, ldxt, npad));
  if (x3) RMC_TRY(make_tmap(&ml, Xl, l, n, ldxt, npad));
  else ml = mx;
  float *outp = splits > 1 ? part : Y;
  const int64_t ldo = splits > 1 ? l : ldy;
  {
    RmcProf prof(ctx, RMC_K_MATMUL_AN);
    int rc = RMC_OK;
    switch (npad * 2 + (x3 ? 1 : 0)) {
      case 64: rc = an_launch<32, false>(ctx, ma, mx, ml, m, n, l, outp, ldo, splits); break;
      case 65: rc = an_launch<32, true>(ctx, ma, mx, ml, m, n, l, outp, ldo, splits); break;
      case 128: rc = an_launch<64, false>(ctx, ma, mx, ml, m, n, l, outp, ldo, splits); break;
      case 129: rc = an_launch<64, true>(ctx, ma, mx, ml, m, n, l, outp, ldo, splits); break;
      case 256: rc = an_launch<128, false>(ctx, ma, mx, ml, m, n, l, outp, ldo, splits); break;
      case 257: rc = an_launch<128, true>(ctx, ma, mx, ml, m, n, l, outp, ldo, splits); break;
      case 512: rc = an_launch<256, false>(ctx, ma, mx, ml, m, n, l, outp, ldo, splits); break;
      default: rc = an_launch<256, true>(ctx, ma, mx, ml, m, n, l, outp, ldo, splits); break;
    }
    RMC_TRY(rc);
  }
  rmc_note_launch();
  if (splits > 1) {
    sum_parts_kernel<<<rmc_blocks(m * l, 256, 8192), 256, 0, ctx->stream>>>(part, splits, m, l, Y, ldy);
    rmc_note_launch();
  }
  RMC_LAUNCH_CHECK();
  return RMC_OK;
}

template <int MT, bool X3>
int at_launch(rmc_ctx *ctx, const CUtensorMap &ma, const CUtensorMap &mx, const CUtensorMap &ml, int64_t m,
              int64_t n, int64_t l, int64_t rows, int splits, float *part) {
  const size_t smem = AtCfg<MT, X3>::kSmem;
  RMC_TRY_CUDA(rmc_allow_smem(tc_at_kernel<MT, X3>, smem));
  dim3 grid((unsigned)((n + AtCfg<MT, X3>::NC - 1) / AtCfg<MT, X3>::NC), 1, (unsigned)splits);
  tc_at_kernel<MT, X3><<<grid, 32 * (4 + 4 * MT), smem, ctx->stream>>>(ma, mx, ml, m, n, l, rows, part,
                                                                       ctx->d_status);
  return RMC_OK;
}

// Launch W = X^T A with X^T (l x m) given (X3: Xt heads, Xl remainders); l <= 256; part: workspace for the
// row-range partial sums.
int launch_at_t(rmc_ctx *ctx, const float *A, int64_t m, int64_t n, int64_t lda, const float *Xt, const float *Xl,
                int64_t l, int64_t ldxt, float *W, int64_t ldw, float *part, bool x3) {
  CUtensorMap ma, mx, ml;
  RMC_TRY(make_tmap(&ma, A, m, n, lda, kKStage));
  RMC_TRY(make_tmap(&mx, Xt, l, m, ldxt, 128));
  if (x3) RMC_TRY(make_tmap(&ml, Xl, l, m, ldxt, 128));
  else ml = mx;
  const int splits = at_splits(m, n, x3, ctx->num_sms);
  int64_t rows = (m + splits - 1) / splits;
  rows = (rows + kKStage - 1) / kKStage * kKStage;
  {
    RmcProf prof(ctx, RMC_K_MATMUL_AT);
    int rc;
    if (l <= 128) rc = x3 ? at_launch<1, true>(ctx, ma, mx, ml, m, n, l, rows, splits, part)
                          : at_launch<1, false>(ctx, ma, mx, ml, m, n, l, rows, splits, part);
    else rc = x3 ? at_launch<2, true>(ctx, ma, mx, ml, m, n, l, rows, splits, part)
                 : at_launch<2, false>(ctx, ma, mx, ml, m, n, l, rows, splits, part);
    RMC_TRY(rc);
  }
  sum_parts_kernel<<<rmc_blocks(l * n, 256, 8192), 256, 0, ctx->stream>>>(part, splits, l, n, W, ldw);
  rmc_note_launch(2);
  RMC_LAUNCH_CHECK();
  return RMC_OK;
}

// Row-major BF16 matrix (rows x cols, leading dimension ld elements) as a 2-D tensor with a 64 x box_rows box
// (128 bytes along the row) and 128-byte swizzle: the K-major BF16 operand layout.
int make_tmap_bf16(CUtensorMap *map, const uint16_t *base, int64_t rows, int64_t cols, int64_t ld, int box_rows) {
  PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
  if (!fn) return RMC_ECUDA;
  if ((reinterpret_cast<uintptr_t>(base) & 15) || ((ld * 2) & 15)) return RMC_EALIGN;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * 2)};
  cuuint32_t box[2] = {64, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<uint16_t *>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? RMC_OK : RMC_EALIGN;
}

int64_t x16_ld(int64_t cols) { return (cols + 7) / 8 * 8; }   // 16-byte row pitch for TMA

// X (rows x cols, row-major FP32, ldx) transposed and rounded to BF16: X16[c][r] (cols x rows, ld16).
__global__ void transpose_bf16_kernel(const float *__restrict__ X, int64_t rows, int64_t cols, int64_t ldx,
                                      uint16_t *__restrict__ X16, int64_t ld16) {
  __shared__ float tile[32][33];
  const int64_t bx = (int64_t)blockIdx.x * 32, by = (int64_t)blockIdx.y * 32;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int64_t r = by + k, c = bx + threadIdx.x;
    if (r < rows && c < cols) tile[k][threadIdx.x] = X[r * ldx + c];
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int64_t c = bx + k, r = by + threadIdx.x;
    if (r < rows && c < cols) X16[c * ld16 + r] = (uint16_t)(pack_bf16x2(tile[threadIdx.x][k], 0.f) & 0xFFFFu);
  }
}

template <int NP>
int an_bf16_launch(rmc_ctx *ctx, const CUtensorMap &ma, const CUtensorMap &mx, int64_t m, int64_t n, int64_t l,
                   float *Y, int64_t ldy) {
  const size_t smem = AnBfCfg<NP>::kSmem;
  RMC_TRY_CUDA(rmc_allow_smem(tc_an_bf16_kernel<NP>, smem));
  tc_an_bf16_kernel<NP><<<(unsigned)((m + 127) / 128), kAnThreads, smem, ctx->stream>>>(ma, mx, m, n, l, Y, ldy,
                                                                                         ctx->d_status);
  return RMC_OK;
}

template <int MT>
int at_bf16_launch(rmc_ctx *ctx, const CUtensorMap &ma, const CUtensorMap &mx, int64_t m, int64_t n, int64_t l,
                   int64_t rows, int splits, float *part) {
  const size_t smem = AtBfCfg<MT>::kSmem;
  RMC_TRY_CUDA(rmc_allow_smem(tc_at_bf16_kernel<MT>, smem));
  dim3 grid((unsigned)((n + AtBfCfg<MT>::NC - 1) / AtBfCfg<MT>::NC), 1, (unsigned)splits);
  tc_at_bf16_kernel<MT><<<grid, 32 * (4 + 4 * MT), smem, ctx->stream>>>(ma, mx, m, n, l, rows, part, ctx->d_status);
  return RMC_OK;
}

}  // namespace

// Workspace of the public tensor-core products: X^T (padded pitch; 3xTF32 also its remainder) plus the split
// partials of W = X^T A.
size_t rmc_tc_matmul_ws(int64_t m, int64_t n, int64_t l, int which, bool x3, int num_sms) {
  WsCarve w;
  const int64_t ld = xt_ld(which == 0 ? n : m);
  w.take<float>((size_t)l * ld);
  if (x3) w.take<float>((size_t)l * ld);
  if (which == 1) w.take<float>((size_t)at_splits(m, n, x3, num_sms) * l * n);
  else if (an_splits(n, x3) > 1) w.take<float>((size_t)an_splits(n, x3) * m * l);
  return w.off;
}

int rmc_tc_matmul_an(rmc_ctx *ctx, const float *A, int64_t m, int64_t n, int64_t lda, const float *X, int64_t l,
                     int64_t ldx, float *Y, int64_t ldy, bool x3, void *ws) {
  WsCarve w;
  w.base = static_cast<char *>(ws);
  const int64_t ld = xt_ld(n);
  float *Xt = w.take<float>((size_t)l * ld);
  float *Xl = x3 ? w.take<float>((size_t)l * ld) : nullptr;
  float *part = an_splits(n, x3) > 1 ? w.take<float>((size_t)an_splits(n, x3) * m * l) : nullptr;
  dim3 grid((unsigned)((l + 31) / 32), (unsigned)((n + 31) / 32));
  transpose32_kernel<<<grid, dim3(32, 8), 0, ctx->stream>>>(X, n, l, ldx, Xt, ld);
  rmc_note_launch();
  if (x3) {
    split_tf32_kernel<<<rmc_blocks(l * n, 256, 4096), 256, 0, ctx->stream>>>(Xt, l, n, ld, Xl);
    rmc_note_launch();
  }
  return launch_an_t(ctx, A, m, n, lda, Xt, Xl, l, ld, Y, ldy, x3, part);
}

int rmc_tc_matmul_at(rmc_ctx *ctx, const float *A, int64_t m, int64_t n, int64_t lda, const float *X, int64_t l,
                     int64_t ldx, float *W, int64_t ldw, bool x3, void *ws) {
  WsCarve w;
  w.base = static_cast<char *>(ws);
  const int64_t ld = xt_ld(m);
  float *Xt = w.take<float>((size_t)l * ld);
  float *Xl = x3 ? w.take<float>((size_t)l * ld) : nullptr;
  float *part = w.take<float>((size_t)at_splits(m, n, x3, ctx->num_sms) * l * n);
  dim3 grid((unsigned)((l + 31) / 32), (unsigned)((m + 31) / 32));
  transpose32_kernel<<<grid, dim3(32, 8), 0, ctx->stream>>>(X, m, l, ldx, Xt, ld);
  rmc_note_launch();
  if (x3) {
    split_tf32_kernel<<<rmc_blocks(l * m, 256, 4096), 256, 0, ctx->stream>>>(Xt, l, m, ld, Xl);
    rmc_note_launch();
  }
  return launch_at_t(ctx, A, m, n, lda, Xt, Xl, l, ld, W, ldw, part, x3);
}

// BF16 operands (RMC_BF16): X^T rounded to BF16 in the workspace, A converted on chip.  Workspace: X^T in BF16
// (padded pitch) and, for W = X^T A, the split partials.
size_t rmc_tc_matmul_bf16_ws(int64_t m, int64_t n, int64_t l, int which, int num_sms) {
  WsCarve w;
  w.take<uint16_t>((size_t)l * x16_ld(which == 0 ? n : m));
  if (which == 1) w.take<float>((size_t)at_splits(m, n, false, num_sms) * l * n);
  return w.off;
}

int rmc_tc_matmul_an_bf16(rmc_ctx *ctx, const float *A, int64_t m, int64_t n, int64_t lda, const float *X, int64_t l,
                          int64_t ldx, float *Y, int64_t ldy, void *ws) {
  WsCarve w;
  w.base = static_cast<char *>(ws);
  const int64_t ld = x16_ld(n);
  uint16_t *X16 = w.take<uint16_t>((size_t)l * ld);
  dim3 grid((unsigned)((l + 31) / 32), (unsigned)((n + 31) / 32));
  transpose_bf16_kernel<<<grid, dim3(32, 8), 0, ctx->stream>>>(X, n, l, ldx, X16, ld);
  rmc_note_launch();
  CUtensorMap ma, mx;
  const int npad = l <= 32 ? 32 : l <= 64 ? 64 : l <= 128 ? 128 : 256;
  RMC_TRY(make_tmap(&ma, A, m, n, lda, 128));
  RMC_TRY(make_tmap_bf16(&mx, X16, l, n, ld, npad));
  {
    RmcProf prof(ctx, RMC_K_MATMUL_AN);
    int rc;
    switch (npad) {
      case 32: rc = an_bf16_launch<32>(ctx, ma, mx, m, n, l, Y, ldy); break;
      case 64: rc = an_bf16_launch<64>(ctx, ma, mx, m, n, l, Y, ldy); break;
      case 128: rc = an_bf16_launch<128>(ctx, ma, mx, m, n, l, Y, ldy); break;
      default: rc = an_bf16_launch<256>(ctx, ma, mx, m, n, l, Y, ldy); break;
    }
    RMC_TRY(rc);
  }
  rmc_note_launch();
  RMC_LAUNCH_CHECK();
  return RMC_OK;
}

int rmc_tc_matmul_at_bf16(rmc_ctx *ctx, const float *A, int64_t m, int64_t n, int64_t lda, const float *X, int64_t l,
                          int64_t ldx, float *W, int64_t ldw, void *ws) {
  WsCarve w;
  w.base = static_cast<char *>(ws);
  const int64_t ld = x16_ld(m);
  uint16_t *X16 = w.take<uint16_t>((size_t)l * ld);
  const int splits = at_splits(m, n, false, ctx->num_sms);
  float *part = w.take<float>((size_t)splits * l * n);
  dim3 grid((unsigned)((l + 31) / 32), (unsigned)((m + 31) / 32));
  transpose_bf16_kernel<<<grid, dim3(32, 8), 0, ctx->stream>>>(X, m, l, ldx, X16, ld);
  rmc_note_launch();
  CUtensorMap ma, mx;
  RMC_TRY(make_tmap(&ma, A, m, n, lda, kKStage));
  RMC_TRY(make_tmap_bf16(&mx, X16, l, m, ld, 128));
  int64_t rows = (m + splits - 1) / splits;
  rows = (rows + 63) / 64 * 64;
  {
    RmcProf prof(ctx, RMC_K_MATMUL_AT);
    RMC_TRY(l <= 128 ? at_bf16_launch<1>(ctx, ma, mx, m, n, l, rows, splits, part)
                     : at_bf16_launch<2>(ctx, ma, mx, m, n, l, rows, splits, part));
  }
  sum_parts_kernel<<<rmc_blocks(l * n, 256, 8192), 256, 0, ctx->stream>>>(part, splits, l, n, W, ldw);
  rmc_note_launch(2);
  RMC_LAUNCH_CHECK();
  return RMC_OK;
}
