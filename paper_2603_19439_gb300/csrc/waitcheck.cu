// grest_check_bounded_wait: exercises the bounded wait that every mbarrier
// wait of the tensor-core kernels uses (tc_util.cuh, mbar_wait).  One thread
// waits on a freshly initialized barrier that nothing arrives on; the wait
// gives up after its iteration limit (about a second), records
// DERR_TIMEOUT in the error word and the kernel returns, holding no tensor
// memory and no copies in flight.  The host reads the word, so a caller (or
// a test) can see that an expired wait turns into GREST_ERR_TIMEOUT and that
// the device stays usable afterwards.
//
// grest_check_fast_recip: evaluates the Newton reciprocal of the small
// factorizations (common.cuh, rcp_newton) on caller-given inputs, so that a
// test can hold it to its error bound against correctly rounded 1 / x.
#include "tc_util.cuh"

namespace grest {
namespace {

__global__ void k_wait_never_arrives(int32_t* err) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  __syncthreads();
  // phase 0 completes only after one arrival, which never comes
  if (threadIdx.x == 0 && !tc::mbar_wait(&bar, 0)) atomicCAS(err, 0, DERR_TIMEOUT);
}

__global__ void k_fast_recip(const double* __restrict__ x, int64_t n, double* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = rcp_newton(x[i]);
}

}  // namespace
}  // namespace grest

extern "C" grest_status grest_check_fast_recip(const double* x, int64_t n, double* out, void* cuda_stream) {
  if (n < 0 || (n > 0 && (!x || !out))) return GREST_ERR_INVALID_ARG;
  if (n == 0) return GREST_OK;
  cudaError_t e = cudaPeekAtLastError();
  if (e != cudaSuccess) return GREST_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const int64_t blocks = (n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024;
  grest::k_fast_recip<<<(unsigned)blocks, 256, 0, s>>>(x, n, out);
  e = cudaPeekAtLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e == cudaSuccess ? GREST_OK : GREST_ERR_CUDA;
}

extern "C" grest_status grest_check_bounded_wait(void* cuda_stream) {
  int32_t* err = nullptr;
  if (cudaMalloc(&err, sizeof(int32_t)) != cudaSuccess) return GREST_ERR_OOM;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  int32_t h = -1;
  cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int32_t), s);
  if (e == cudaSuccess) {
    grest::k_wait_never_arrives<<<1, 32, 0, s>>>(err);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, err, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(err);
  if (e != cudaSuccess) return GREST_ERR_CUDA;
  return h == grest::DERR_TIMEOUT ? GREST_ERR_TIMEOUT : (h == 0 ? GREST_OK : GREST_ERR_CUDA);
}
