// grest_gram_noalloc: the Gram product C = X^T Y with its split-K scratch in a
// file-scope device array instead of memory allocated by a context, for
// callers that cannot allocate device memory (see include/grest.h).
//
// The scratch is one static __device__ array of kNoAllocScratchDoubles
// doubles (4 MiB) that every GPU loading this library holds until the
// process exits.  Host code must not use the array's name as a device
// address: on the host it is only a stand-in symbol.  The device address is
// obtained once per device with cudaGetSymbolAddress, with that device
// current, on the first call made on that device.
#include <mutex>

#include "common.cuh"

namespace {

constexpr int64_t kNoAllocScratchDoubles = int64_t(1) << 19;  // 4 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_gram_scratch[kNoAllocScratchDoubles];

std::mutex g_setup_mutex;
double* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array for the current device (set-up on first use).
cudaError_t scratch_for_current_device(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_gram_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" grest_status grest_gram_noalloc(const double* X, int64_t ldx, int32_t a, const double* Y, int64_t ldy,
                                           int32_t b, int64_t n, double* C, int64_t ldc, void* cuda_stream) {
  if (!X || !Y || !C || a < 1 || b < 1 || n < 1 || ldx < a || ldy < b || ldc < b) return GREST_ERR_INVALID_ARG;
  if (a > 256 || b > 256) return GREST_ERR_CAPACITY;  // a * b partials must fit the fixed scratch
  // a launch error left pending on this host thread by earlier work is
  // reported as such before anything is enqueued (and is not cleared)
  if (cudaPeekAtLastError() != cudaSuccess) return GREST_ERR_CUDA;
  double* scratch = nullptr;
  cudaError_t e = scratch_for_current_device(&scratch);
  if (e != cudaSuccess) return GREST_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  // with a, b <= 256 one chunk's partials (a * b <= 65,536 doubles) always
  // fit, so the capped launcher takes every shape accepted above
  if (grest::gram_f64_capped(X, ldx, a, Y, ldy, b, n, C, ldc, scratch, kNoAllocScratchDoubles, s) != 0)
    return GREST_ERR_INVALID_ARG;
  e = cudaGetLastError();  // only this call's launches can have set it
  return e == cudaSuccess ? GREST_OK : GREST_ERR_CUDA;
}
