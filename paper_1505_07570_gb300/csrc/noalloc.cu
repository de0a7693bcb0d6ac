// Count sketch without any device allocation (rmc_countsketch_noalloc in rmc.h).
//
// The scratch that the count-sketch path normally takes from a context's workspace (row hashes, the
// bucket-by-chunk counters, the row permutation) lives here in one file-scope device array.  Host code
// cannot use the array's name as a device address, so every call looks the address up with
// cudaGetSymbolAddress on the current device (a host-side query that enqueues nothing), which stays correct
// after the device or this module has been torn down and reloaded.  All calls share the array: overlapping
// calls race on it.
#include "rmc_internal.cuh"

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[RMC_NOALLOC_SCRATCH_BYTES];

// The array's device address and the SM count of the current device.
int noalloc_setup(int device, void **scratch, int *num_sms) {
  void *p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || !p) {
    (void)cudaGetLastError();
    return RMC_ECUDA;
  }
  int sms = 0;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  if (e != cudaSuccess || sms < 1) {
    (void)cudaGetLastError();
    return RMC_ECUDA;
  }
  *scratch = p;
  *num_sms = sms;
  return RMC_OK;
}

}  // namespace

extern "C" int rmc_countsketch_noalloc(void *cuda_stream, const float *A, int64_t m, int64_t n, int64_t lda,
                                       int64_t s, uint64_t seed, float *C, int64_t ldc) {
  if (!A || !C || m < 1 || n < 1 || lda < n || s < 1 || ldc < n) return RMC_EINVAL;
  if (m > (int64_t(1) << 31) || s > (int64_t(1) << 31)) return RMC_EINVAL;
  if (rmc_countsketch_ws(m, s) > (size_t)RMC_NOALLOC_SCRATCH_BYTES) return RMC_ESCRATCH;
  int device = -1;
  if (cudaGetDevice(&device) != cudaSuccess) {
    (void)cudaGetLastError();
    return RMC_ECUDA;
  }
  void *scratch = nullptr;
  int num_sms = 0;
  RMC_TRY(noalloc_setup(device, &scratch, &num_sms));
  // A context-shaped view for the shared launcher: stream and SM count only (no workspace, no status word,
  // no profiling); it lives on the host stack and owns nothing.
  rmc_ctx view = {};
  view.stream = static_cast<cudaStream_t>(cuda_stream);
  view.device = device;
  view.num_sms = num_sms;
  return rmc_launch_countsketch(&view, A, m, n, lda, nullptr, s, seed, 0, C, ldc, nullptr, scratch);
}
