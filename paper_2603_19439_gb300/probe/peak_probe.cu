// Arithmetic and gather-bandwidth probe for the roofline denominators of the FP64 path:
// DFMA, FFMA and DMMA (mma.sync f64) throughput, device properties, and the
// bandwidth of warp-per-row random row gathers (the SpMM access pattern).
// Build and run: nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o /tmp/peak_probe peak_probe.cu && /tmp/peak_probe
#include <cstdio>
#include <cstdlib>
#include <cstdint>
#include <vector>
#include <cuda_runtime.h>
#define CK(x) do{cudaError_t e=(x); if(e!=cudaSuccess){printf("CUDA %s at %d: %s\n",#x,__LINE__,cudaGetErrorString(e)); exit(1);}}while(0)

template<int CH>
__global__ void k_dfma(double* out, int iters, double a, double b){
  double x[CH];
  #pragma unroll
  for(int c=0;c<CH;c++) x[c]=threadIdx.x*1e-9+c;
  for(int i=0;i<iters;i++){
    #pragma unroll
    for(int c=0;c<CH;c++) x[c]=fma(x[c],a,b);
  }
  double s=0;
  #pragma unroll
  for(int c=0;c<CH;c++) s+=x[c];
  if(s==1234.5) out[threadIdx.x]=s;
}
template<int CH>
__global__ void k_ffma(float* out, int iters, float a, float b){
  float x[CH];
  #pragma unroll
  for(int c=0;c<CH;c++) x[c]=threadIdx.x*1e-9f+c;
  for(int i=0;i<iters;i++){
    #pragma unroll
    for(int c=0;c<CH;c++) x[c]=fmaf(x[c],a,b);
  }
  float s=0;
  #pragma unroll
  for(int c=0;c<CH;c++) s+=x[c];
  if(s==1234.5f) out[threadIdx.x]=s;
}
__global__ void k_dmma(double* out, int iters){
  double a0 = 1.0 + threadIdx.x*1e-6, b0 = 0.5;
  double acc[4][2];
  for(int c=0;c<4;c++){acc[c][0]=0;acc[c][1]=0;}
  for(int i=0;i<iters;i++){
    #pragma unroll
    for(int c=0;c<4;c++){
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
        : "+d"(acc[c][0]), "+d"(acc[c][1]) : "d"(a0), "d"(b0));
    }
  }
  double s=0; for(int c=0;c<4;c++) s+=acc[c][0]+acc[c][1];
  if(s==1234.5) out[threadIdx.x]=s;
}
// gather: out[i, :] = sum_j X[idx[i*deg+j], :], X rows of W doubles, warp per row
template<int W>
__global__ void k_gather(const double* __restrict__ X, const int* __restrict__ idx, double* __restrict__ out, int n, int deg){
  int warp=(blockIdx.x*blockDim.x+threadIdx.x)>>5, lane=threadIdx.x&31;
  if(warp>=n) return;
  double acc[W/32>0?W/32:1];
  constexpr int PL = W/32>0?W/32:1;
  for(int c=0;c<PL;c++) acc[c]=0;
  for(int j=0;j<deg;j++){
    int r=__ldg(idx+(size_t)warp*deg+j);
    const double* xr=X+(size_t)r*W;
    #pragma unroll
    for(int c=0;c<PL;c++) acc[c]+=__ldg(xr+c*32+lane);
  }
  for(int c=0;c<PL;c++) out[(size_t)warp*W+c*32+lane]=acc[c];
}
int main(){
  cudaDeviceProp p; CK(cudaGetDeviceProperties(&p,0));
  printf("name=%s sms=%d cc=%d.%d l2=%d smem_optin=%zu smem_per_sm=%zu regs_per_sm=%d clock_khz=%d memclk_khz=%d busw=%d\n",
    p.name,p.multiProcessorCount,p.major,p.minor,p.l2CacheSize,p.sharedMemPerBlockOptin,p.sharedMemPerMultiprocessor,p.regsPerMultiprocessor,0,0,p.memoryBusWidth);
  int clk=0; cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, 0); printf("clock_khz=%d\n",clk);
  double* dout; CK(cudaMalloc(&dout, 1<<20));
  cudaEvent_t e0,e1; CK(cudaEventCreate(&e0)); CK(cudaEventCreate(&e1));
  int sms=p.multiProcessorCount;
  float ms;
  // DFMA
  for(int rep=0;rep<2;rep++){
    int iters=4096; int blocks=sms*4, thr=256;
    CK(cudaEventRecord(e0)); k_dfma<8><<<blocks,thr>>>(dout,iters,1.0000001,1e-9); CK(cudaEventRecord(e1)); CK(cudaEventSynchronize(e1));
    CK(cudaEventElapsedTime(&ms,e0,e1)); CK(cudaGetLastError());
    double fl=2.0*8*iters*(double)blocks*thr; printf("DFMA: %.3f TFLOP/s (%.3f ms)\n", fl/ms/1e9, ms);
  }
  for(int rep=0;rep<2;rep++){
    int iters=8192; int blocks=sms*8, thr=256;
    CK(cudaEventRecord(e0)); k_ffma<8><<<blocks,thr>>>((float*)dout,iters,1.0000001f,1e-9f); CK(cudaEventRecord(e1)); CK(cudaEventSynchronize(e1));
    CK(cudaEventElapsedTime(&ms,e0,e1)); CK(cudaGetLastError());
    double fl=2.0*8*iters*(double)blocks*thr; printf("FFMA: %.3f TFLOP/s (%.3f ms)\n", fl/ms/1e9, ms);
  }
  for(int rep=0;rep<2;rep++){
    int iters=2048; int blocks=sms*4, thr=256;
    CK(cudaEventRecord(e0)); k_dmma<<<blocks,thr>>>(dout,iters); CK(cudaEventRecord(e1)); CK(cudaEventSynchronize(e1));
    CK(cudaEventElapsedTime(&ms,e0,e1)); CK(cudaGetLastError());
    double fl=2.0*8*8*4*4.0*iters*(double)blocks*(thr/32); printf("DMMA m8n8k4: %.3f TFLOP/s (%.3f ms)\n", fl/ms/1e9, ms);
  }
  // gather bandwidth: n rows, X random, deg neighbors uniform random
  {
    const int n=1<<20, deg=32;
    std::vector<int> h(n*(size_t)deg); uint64_t s=88172645463325252ull;
    for(size_t i=0;i<h.size();i++){ s^=s<<13; s^=s>>7; s^=s<<17; h[i]=(int)(s%n);}
    int* didx; CK(cudaMalloc(&didx,h.size()*4)); CK(cudaMemcpy(didx,h.data(),h.size()*4,cudaMemcpyHostToDevice));
    double *X,*O; CK(cudaMalloc(&X,(size_t)n*128*8)); CK(cudaMalloc(&O,(size_t)n*128*8));
    CK(cudaMemset(X,0,(size_t)n*128*8));
    for(int rep=0;rep<3;rep++){
      CK(cudaEventRecord(e0)); k_gather<32><<<(n*32+255)/256,256>>>(X,didx,O,n,deg); CK(cudaEventRecord(e1)); CK(cudaEventSynchronize(e1));
      CK(cudaEventElapsedTime(&ms,e0,e1));
      double gb=(double)n*deg*32*8/1e9; printf("gather W=32 f64: %.3f ms gathered %.1f GB/s  compulsory %.1f GB/s\n",ms,gb/ms*1e3,((double)n*32*8*2+n*deg*4.0)/1e6/ms);
    }
    for(int rep=0;rep<3;rep++){
      CK(cudaEventRecord(e0)); k_gather<128><<<(n*32+255)/256,256>>>(X,didx,O,n,deg); CK(cudaEventRecord(e1)); CK(cudaEventSynchronize(e1));
      CK(cudaEventElapsedTime(&ms,e0,e1));
      double gb=(double)n*deg*128*8/1e9; printf("gather W=128 f64: %.3f ms gathered %.1f GB/s\n",ms,gb/ms*1e3);
    }
    CK(cudaGetLastError());
  }
  printf("probe done\n");
  return 0;
}
