// tcgen05 tensor-core kernels (TF32 / BF16 operands, FP32 accumulation in tensor memory).
#include "rmc_internal.cuh"

int rmc_tc_available(void) { return 0; }

size_t rmc_tc_gauss_ws(int64_t, int64_t, int64_t, int, int) { return 0; }
int rmc_tc_gauss_sketch(rmc_ctx *, const float *, int64_t, int64_t, int64_t, const float *, int64_t, uint64_t,
                        uint32_t, int, float *, int64_t, float *, void *) {
  return RMC_EINVAL;
}
size_t rmc_tc_matmul_ws(int64_t, int64_t, int64_t, int, int) { return 0; }
int rmc_tc_matmul_an(rmc_ctx *, const float *, int64_t, int64_t, int64_t, const float *, int64_t, int64_t, float *,
                     int64_t, void *) {
  return RMC_EINVAL;
}
int rmc_tc_matmul_at(rmc_ctx *, const float *, int64_t, int64_t, int64_t, const float *, int64_t, int64_t, float *,
                     int64_t, void *) {
  return RMC_EINVAL;
}
