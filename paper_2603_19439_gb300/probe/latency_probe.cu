// Probe: latency and throughput facts of GB300 that shape the small dense
// kernels (FP64 chains vs active lanes and warps per SM, FP64 division, FP32
// chains, cluster barrier, distributed shared memory load latency).
// Probe: FP64 chain cost vs active lanes and warps/SM; FP64 division chain;
// cluster barrier latency; DSMEM load latency.  All loops bounded.
#include <cstdio>
#include <cooperative_groups.h>
namespace cg = cooperative_groups;

template <int ACTIVE>
__global__ void k_fma_chain(double* out, int iters, double a, double b) {
  const int lane = threadIdx.x & 31;
  double x = threadIdx.x * 1e-3;
  if (lane < ACTIVE) {
    for (int i = 0; i < iters; ++i) x = fma(x, a, b);
  }
  if (x == 12345.0) out[threadIdx.x] = x;
}

template <int ACTIVE>
__global__ void k_div_chain(double* out, int iters, double b) {
  const int lane = threadIdx.x & 31;
  double x = 1.0 + threadIdx.x * 1e-3;
  if (lane < ACTIVE) {
    for (int i = 0; i < iters; ++i) x = b - 0.25 / x;
  }
  if (x == 12345.0) out[threadIdx.x] = x;
}

__global__ void k_f32_chain(float* out, int iters, float a, float b) {
  float x = threadIdx.x * 1e-3f;
  for (int i = 0; i < iters; ++i) x = fmaf(x, a, b);
  if (x == 12345.0f) out[threadIdx.x] = x;
}

__global__ void k_cluster_sync(int iters, int* out) {
  cg::cluster_group cl = cg::this_cluster();
  for (int i = 0; i < iters; ++i) cl.sync();
  if (threadIdx.x == 0 && cl.block_rank() == 0) out[0] = iters;
}

__global__ void k_dsmem_chase(int iters, int* out) {
  __shared__ int nxt[256];
  cg::cluster_group cl = cg::this_cluster();
  for (int i = threadIdx.x; i < 256; i += blockDim.x) nxt[i] = (i * 17 + 5) & 255;
  cl.sync();
  if (cl.block_rank() == 0 && threadIdx.x == 0) {
    const int* rem = cl.map_shared_rank(nxt, 1);
    int p = 0;
    for (int i = 0; i < iters; ++i) p = rem[p];
    out[0] = p;
  }
  cl.sync();
}

template <typename F>
float time_it(F f, int reps = 5) {
  cudaEvent_t a, b;
  cudaEventCreate(&a); cudaEventCreate(&b);
  f();
  cudaDeviceSynchronize();
  float best = 1e30f;
  for (int r = 0; r < reps; ++r) {
    cudaEventRecord(a);
    f();
    cudaEventRecord(b);
    cudaEventSynchronize(b);
    float ms; cudaEventElapsedTime(&ms, a, b);
    if (ms < best) best = ms;
  }
  return best;
}

template <typename K>
void launch_cluster(K kern, int C, int threads, int iters, int* out) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C); cfg.blockDim = dim3(threads);
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = C; at[0].val.clusterDim.y = 1; at[0].val.clusterDim.z = 1;
  cfg.attrs = at; cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kern, iters, out);
}

int main() {
  double* d; float* f; int* o;
  cudaMalloc(&d, 1 << 20); cudaMalloc(&f, 1 << 20); cudaMalloc(&o, 64);
  const double clk = 2.07e9;
  int iters = 20000;
  for (int threads : {32, 128, 256, 1024}) {
    float t32 = time_it([&] { k_fma_chain<32><<<152, threads>>>(d, iters, 0.999, 1e-3); });
    float t8 = time_it([&] { k_fma_chain<8><<<152, threads>>>(d, iters, 0.999, 1e-3); });
    float t1 = time_it([&] { k_fma_chain<1><<<152, threads>>>(d, iters, 0.999, 1e-3); });
    printf("dfma chain 152 blocks x %4d thr: active32 %.2f clk/iter, active8 %.2f, active1 %.2f\n", threads,
           t32 * 1e-3 * clk / iters, t8 * 1e-3 * clk / iters, t1 * 1e-3 * clk / iters);
  }
  iters = 4000;
  for (int threads : {32, 128}) {
    float t32 = time_it([&] { k_div_chain<32><<<152, threads>>>(d, iters, 1.5); });
    float t1 = time_it([&] { k_div_chain<1><<<152, threads>>>(d, iters, 1.5); });
    printf("ddiv chain 152 blocks x %4d thr: active32 %.2f clk/iter, active1 %.2f\n", threads,
           t32 * 1e-3 * clk / iters, t1 * 1e-3 * clk / iters);
  }
  iters = 20000;
  for (int threads : {32, 1024}) {
    float t = time_it([&] { k_f32_chain<<<152, threads>>>(f, iters, 0.999f, 1e-3f); });
    printf("ffma chain 152 blocks x %4d thr: %.2f clk/iter\n", threads, t * 1e-3 * clk / iters);
  }
  cudaFuncSetAttribute(k_cluster_sync, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  for (int C : {2, 4, 8, 16}) {
    for (int threads : {256, 1024}) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(C); cfg.blockDim = dim3(threads);
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = C; at[0].val.clusterDim.y = 1; at[0].val.clusterDim.z = 1;
      cfg.attrs = at; cfg.numAttrs = 1;
      int ncl = 0;
      cudaError_t e = cudaOccupancyMaxActiveClusters(&ncl, k_cluster_sync, &cfg);
      if (e != cudaSuccess || ncl == 0) { printf("cluster %d x %d: not launchable (%s, %d)\n", C, threads, cudaGetErrorString(e), ncl); cudaGetLastError(); continue; }
      int it = 10000;
      float t = time_it([&] { launch_cluster(k_cluster_sync, C, threads, it, o); });
      cudaError_t le = cudaGetLastError();
      printf("cluster.sync C=%2d threads=%4d: %.1f ns (%.0f clk) per barrier [max active clusters %d] %s\n", C, threads,
             t * 1e6 / it, t * 1e-3 * clk / it, ncl, cudaGetErrorString(le));
    }
  }
  {
    int it = 10000;
    float t = time_it([&] { launch_cluster(k_dsmem_chase, 2, 128, it, o); });
    printf("dsmem dependent load latency: %.0f clk\n", t * 1e-3 * clk / it);
  }
  cudaError_t e = cudaDeviceSynchronize();
  printf("status %s\n", cudaGetErrorString(e));
  return e == cudaSuccess ? 0 : 1;
}
