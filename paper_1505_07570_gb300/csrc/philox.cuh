// Philox4x32-10 on the device (Salmon, Moraes, Dror and Shaw, "Parallel random numbers: as easy as 1, 2,
// 3", SC'11) and the draws the sketches take from it.  The stream layout is the one stated in rmc.h.
#pragma once
#include <stdint.h>

namespace rmc {

constexpr uint32_t kPhiloxM0 = 0xD2511F53u;  // round multipliers of the published generator
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u;  // Weyl key increments
constexpr uint32_t kPhiloxW1 = 0xBB67AE85u;

enum : uint32_t {
  kStreamGaussian = 0,       // range-finder test matrices (four normals per block, 32-bit uniforms)
  kStreamSrhtSign = 1,
  kStreamCountSketch = 2,
  kStreamSrhtKey = 3,
  kStreamGaussSketch = 4     // Gaussian sketching matrix (eight normals per block, 16-bit uniforms)
};

// Ten rounds of the Philox S-P network on one 128-bit counter block.
__device__ __forceinline__ uint4 philox10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(kPhiloxM0, c.x), lo0 = kPhiloxM0 * c.x;
    const uint32_t hi1 = __umulhi(kPhiloxM1, c.z), lo1 = kPhiloxM1 * c.z;
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += kPhiloxW0;
    k1 += kPhiloxW1;
  }
  return c;
}

__device__ __forceinline__ uint4 philox_block(uint64_t seed, uint32_t stream, uint32_t instance, uint64_t index) {
  return philox10(make_uint4((uint32_t)index, (uint32_t)(index >> 32), stream, instance), (uint32_t)seed,
                  (uint32_t)(seed >> 32));
}

// The same rounds with each product written as one 32 x 32 -> 64-bit multiply (bit-identical results).  The
// instruction selection differs: inside the tensor-core Gaussian sketch, where the draws share the SM with the
// transposes and MMAs, this form measured about 4% faster; in a kernel that only draws, about 12% slower.
__device__ __forceinline__ uint4 philox10_wide(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = (uint64_t)kPhiloxM0 * c.x, p1 = (uint64_t)kPhiloxM1 * c.z;
    c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ k0, (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ k1, (uint32_t)p0);
    k0 += kPhiloxW0;
    k1 += kPhiloxW1;
  }
  return c;
}

__device__ __forceinline__ uint4 philox_block_wide(uint64_t seed, uint32_t stream, uint32_t instance,
                                                   uint64_t index) {
  return philox10_wide(make_uint4((uint32_t)index, (uint32_t)(index >> 32), stream, instance), (uint32_t)seed,
                       (uint32_t)(seed >> 32));
}

// ((w >> 9) + 1/2) * 2^-23: exact in FP32, strictly inside (0, 1).  Built from the bit pattern of
// 1 + (w >> 9) 2^-23 in [1, 2) minus (1 - 2^-24): the difference (2 (w >> 9) + 1) 2^-24 has at most 24
// significant bits, so the subtraction is exact and no integer-to-float conversion is needed.
__device__ __forceinline__ float unit_f32(uint32_t w) {
  return __fsub_rn(__uint_as_float(0x3F800000u | (w >> 9)), 0.999999940395355224609375f);
}

// Box-Muller pair from two words: r = sqrt(-2 ln u_a), (r cos 2 pi u_b, r sin 2 pi u_b).
__device__ __forceinline__ float2 box_muller(uint32_t wa, uint32_t wb) {
  const float r = sqrtf(-2.0f * logf(unit_f32(wa)));
  float sn, cs;
  sincospif(2.0f * unit_f32(wb), &sn, &cs);  // 2 u_b is exact, so the angle carries no extra rounding
  return make_float2(r * cs, r * sn);
}

// (h + 1/2) * 2^-16 for a 16-bit h: the bit pattern of 1 + h 2^-16 minus (1 - 2^-17), exact in FP32.
__device__ __forceinline__ float unit16_f32(uint32_t h) {
  return __fsub_rn(__uint_as_float(0x3F800000u | (h << 7)), 0.9999923706054688f);
}

// The eight normals of sketch block `index` (columns 8b .. 8b+7 of one row of the Gaussian sketching matrix):
// halves (lo, hi) of word w form the Box-Muller pair of columns 8b + 2w, 8b + 2w + 1.
__device__ __forceinline__ void gaussian8(uint64_t seed, uint32_t instance, uint64_t index, float (&z)[8]) {
  const uint4 w = philox_block(seed, kStreamGaussSketch, instance, index);
  const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    const float r = sqrtf(-2.0f * logf(unit16_f32(ws[t] & 0xFFFFu)));
    float sn, cs;
    sincospif(2.0f * unit16_f32(ws[t] >> 16), &sn, &cs);   // 2 u is exact: the angle carries no extra rounding
    z[2 * t] = r * cs;
    z[2 * t + 1] = r * sn;
  }
}

// The four normals of Gaussian block `index` (columns 4t .. 4t+3 of one row).
__device__ __forceinline__ float4 gaussian4(uint64_t seed, uint32_t instance, uint64_t index) {
  const uint4 w = philox_block(seed, kStreamGaussian, instance, index);
  const float2 a = box_muller(w.x, w.y);
  const float2 b = box_muller(w.z, w.w);
  return make_float4(a.x, a.y, b.x, b.y);
}

__device__ __forceinline__ float srht_sign(uint64_t seed, uint32_t instance, uint64_t row) {
  const uint4 w = philox_block(seed, kStreamSrhtSign, instance, row);
  return (w.x >> 31) ? -1.0f : 1.0f;
}

// Count-sketch hash: bucket in [0, s) (high half of word0 * s), sign from bit 31 of word 1.
__device__ __forceinline__ void cs_hash(uint64_t seed, uint32_t instance, uint64_t row, uint32_t s,
                                        uint32_t *bucket, float *sign) {
  const uint4 w = philox_block(seed, kStreamCountSketch, instance, row);
  *bucket = __umulhi(w.x, s);
  *sign = (w.y >> 31) ? -1.0f : 1.0f;
}

__device__ __forceinline__ uint64_t srht_key(uint64_t seed, uint32_t instance, uint64_t j) {
  const uint4 w = philox_block(seed, kStreamSrhtKey, instance, j);
  return ((uint64_t)w.x << 32) | w.y;
}

}  // namespace rmc
