// Count sketch without any device allocation (rmc_countsketch_noalloc in rmc.h).
//
// The scratch that the count-sketch path normally takes from a context's workspace (row hashes, the
// bucket-by-chunk counters, the row permutation) lives here in one file-scope device array.  Host code
// cannot use the array's name as a device address, so its address is looked up once per device with
// cudaGetSymbolAddress and cached.  All calls share the array: overlapping calls race on it.
#include <mutex>

#include "rmc_internal.cuh"

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[RMC_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void *g_scratch_ptr[kMaxDevices] = {};
int g_num_sms[kMaxDevices] = {};

// First call on a device (that device current): find the array's device address and the SM count.
int noalloc_setup(int device, void **scratch, int *num_sms) {
  if (device < 0 || device >= kMaxDevices) return RMC_EINVAL;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[device]) {
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
    g_num_sms[device] = sms;
    g_scratch_ptr[device] = p;
  }
  *scratch = g_scratch_ptr[device];
  *num_sms = g_num_sms[device];
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
