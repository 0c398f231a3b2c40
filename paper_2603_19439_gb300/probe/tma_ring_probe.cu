// Probe: sustained TMA 2D load bandwidth with a ring of R stages per CTA (one
// CTA per SM), no compute: the consumer warp waits for a stage and releases it.
#include <cstdio>
#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  uint32_t done = 0;
  for (uint32_t it = 0; it < (1u << 22) && !done; ++it)
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.b32 %0, 1, 0, p;\n}\n"
                 : "=r"(done) : "r"(smem_u32(bar)), "r"(parity) : "memory");
  return done != 0;
}
__global__ void __launch_bounds__(64, 1) k_stream(const __grid_constant__ CUtensorMap map, int64_t n, int rows_box, int box_bytes,
                                                 int R, int64_t rows_per_cta, int ntile_x, int* err, float* sink) {
  extern __shared__ uint8_t raw[];
  uint8_t* sm = (uint8_t*)(((uintptr_t)raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full[16], empty[16];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int q = 0; q < R; ++q) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&full[q])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&empty[q])));
    }
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  __syncthreads();
  const int64_t r0 = blockIdx.x * rows_per_cta;
  int64_t r1 = r0 + rows_per_cta; if (r1 > n) r1 = n;
  const int nch = r1 > r0 ? (int)((r1 - r0 + rows_box - 1) / rows_box) * ntile_x : 0;
  bool bad = false;
  if (warp == 0 && lane == 0) {
    for (int q = 0; q < nch; ++q) {
      const int s = q % R;
      if (q >= R && !mbar_wait(&empty[s], ((q / R) - 1) & 1)) { bad = true; break; }
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(smem_u32(&full[s])), "r"(box_bytes) : "memory");
      const int x = (q % ntile_x) * 128, y = (int)(r0 + (int64_t)(q / ntile_x) * rows_box);
      asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
                   :: "r"(smem_u32(sm + (size_t)s * box_bytes)), "l"(&map), "r"(x), "r"(y), "r"(smem_u32(&full[s])) : "memory");
    }
    for (int q = nch - R > 0 ? nch - R : 0; q < nch; ++q) mbar_wait(&full[q % R], (q / R) & 1);
  } else if (warp == 1) {
    float acc = 0.f;
    for (int q = 0; q < nch; ++q) {
      const int s = q % R;
      if (!mbar_wait(&full[s], (q / R) & 1)) { bad = true; break; }
      acc += ((const float*)(sm + (size_t)s * box_bytes))[lane];
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(smem_u32(&empty[s])) : "memory");
    }
    if (acc == 1234.5f) sink[blockIdx.x] = acc;
  }
  if (bad) atomicExch(err, 1);
  __syncthreads();
}

typedef CUresult (*EncodeFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*, const cuuint64_t*,
                             const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                             CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
int main() {
  void* fp = nullptr; cudaDriverEntryPointQueryResult qr;
  cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &fp, cudaEnableDefault, &qr);
  EncodeFn enc = (EncodeFn)fp;
  const int64_t n = 1 << 20; const int cols = 256;
  float* X; cudaMalloc(&X, n * cols * 4); cudaMemset(X, 0, n * cols * 4);
  int* err; cudaMalloc(&err, 4); cudaMemset(err, 0, 4);
  float* sink; cudaMalloc(&sink, 4096);
  int nsm = 0; cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, 0);
  cudaFuncSetAttribute(k_stream, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
  cudaEvent_t a, b; cudaEventCreate(&a); cudaEventCreate(&b);
  for (int rows_box : {32, 64, 128}) {
    CUtensorMap map;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)n};
    cuuint64_t strides[1] = {(cuuint64_t)cols * 4};
    cuuint32_t box[2] = {128, (cuuint32_t)rows_box};
    cuuint32_t es[2] = {1, 1};
    if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, X, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS) {
      printf("encode failed\n"); return 1; }
    const int box_bytes = 128 * rows_box * 4;
    for (int R : {2, 3, 4, 6, 8, 12}) {
      if ((size_t)R * box_bytes + 1024 > 220 * 1024 || R > 16) continue;
      const int64_t rows_per = (n + nsm - 1) / nsm;
      for (int rep = 0; rep < 2; ++rep) {
        cudaEventRecord(a);
        k_stream<<<nsm, 64, R * box_bytes + 1024>>>(map, n, rows_box, box_bytes, R, rows_per, 2, err, sink);
        cudaEventRecord(b);
        cudaEventSynchronize(b);
      }
      float ms; cudaEventElapsedTime(&ms, a, b);
      int herr = 0; cudaMemcpy(&herr, err, 4, cudaMemcpyDeviceToHost);
      const double bytes = (double)n * cols * 4;
      printf("box %3d rows x 512 B (%3d KB), R=%2d (%4d KB in flight): %.3f ms  %.0f GB/s  (%.1f GB/s/SM) err=%d\n", rows_box,
             box_bytes / 1024, R, R * box_bytes / 1024, ms, bytes / ms / 1e6, bytes / ms / 1e6 / nsm, herr);
    }
  }
  cudaError_t e = cudaDeviceSynchronize();
  printf("status %s\n", cudaGetErrorString(e));
  return e == cudaSuccess ? 0 : 1;
}
