// Probe: issue rate of tcgen05.mma kind::tf32 (M = 128, K = 8) against N, with
// the A operand in shared memory (ss) or tensor memory (ts).  One CTA per SM,
// one thread issues a dependent chain of accumulating MMAs; every wait is
// bounded.  Build: nvcc -gencode arch=compute_103a,code=sm_103a -O3 -std=c++17
// -I include -o mma_rate paper_2603_19439_gb300/probe/mma_rate_probe.cu
#include "../csrc/tc_util.cuh"
#include <cstdio>
using namespace grest::tc;

__global__ void __launch_bounds__(128, 1) k_rate(int N, int ts, int niter, long long* out, int* err) {
  extern __shared__ uint8_t smraw[];
  uint8_t* sm = (uint8_t*)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tbase;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // zero operands: A 16 KB, B up to 32 KB
  for (int i = threadIdx.x; i < (48 * 1024) / 16; i += blockDim.x) ((float4*)sm)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (threadIdx.x == 0) { mbar_init(&bar, 1); asm volatile("fence.mbarrier_init.release.cluster;"); }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(smem_u32(&tbase)), "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tbase;
  if (warp == 0 && lane == 0) {
    const uint32_t idesc = idesc_tf32(128, N);
    const uint32_t a = smem_u32(sm), b = smem_u32(sm + 16384);
    long long t0 = clock64();
    for (int it = 0; it < niter; ++it) {
#pragma unroll
      for (int k4 = 0; k4 < 4; ++k4) {
        if (ts) {
          mma_tf32_ts(tmem, tmem + 256 + 8 * k4, sdesc(b + 32 * k4), idesc, 1u);
          mma_tf32_ts(tmem, tmem + 256 + 8 * k4, sdesc(b + 32 * k4), idesc, 1u);
          mma_tf32_ts(tmem, tmem + 288 + 8 * k4, sdesc(b + 32 * k4), idesc, 1u);
        } else {
          mma_tf32(tmem, sdesc(a + 32 * k4), sdesc(b + 32 * k4), idesc, 1u);
          mma_tf32(tmem, sdesc(a + 32 * k4), sdesc(b + 32 * k4), idesc, 1u);
          mma_tf32(tmem, sdesc(a + 32 * k4), sdesc(b + 32 * k4), idesc, 1u);
        }
      }
    }
    long long t1 = clock64();
    mma_commit(&bar);
    if (!mbar_wait(&bar, 0)) atomicExch(err, 1);
    long long t2 = clock64();
    if (blockIdx.x == 0) { out[0] = t1 - t0; out[1] = t2 - t0; }
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(512));
}

int main() {
  long long* out; int* err;
  cudaMalloc(&out, 16); cudaMalloc(&err, 4); cudaMemset(err, 0, 4);
  const size_t smem = 48 * 1024 + 1024 + 72 * 1024;  // extra to force one CTA per SM
  cudaFuncSetAttribute(k_rate, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const int niter = 2000;
  for (int ts = 0; ts < 2; ++ts)
    for (int N : {32, 64, 128, 256}) {
      k_rate<<<152, 128, smem>>>(N, ts, niter, out, err);
      cudaError_t e = cudaDeviceSynchronize();
      long long h[2]; int he;
      cudaMemcpy(h, out, 16, cudaMemcpyDeviceToHost); cudaMemcpy(&he, err, 4, cudaMemcpyDeviceToHost);
      const double per = (double)h[1] / (niter * 12.0);
      const double macs = 128.0 * N * 8;
      printf("%s N=%3d: issue %.1f clk/mma, complete %.1f clk/mma, %.0f MAC/clk/SM  (%s err %d)\n", ts ? "ts" : "ss", N,
             (double)h[0] / (niter * 12.0), per, macs / per, cudaGetErrorString(e), he);
    }
  return 0;
}
