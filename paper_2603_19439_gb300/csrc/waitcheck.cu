// grest_check_bounded_wait: exercises the bounded wait that every mbarrier
// wait of the tensor-core kernels uses (tc_util.cuh, mbar_wait).  One thread
// waits on a freshly initialized barrier that nothing arrives on; the wait
// gives up after its iteration limit (about a second), records
// DERR_TIMEOUT in the error word and the kernel returns, holding no tensor
// memory and no copies in flight.  The host reads the word, so a caller (or
// a test) can see that an expired wait turns into GREST_ERR_TIMEOUT and that
// the device stays usable afterwards.
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

}  // namespace
}  // namespace grest

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
