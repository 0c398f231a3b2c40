// Check: TF32 rounding by integer operations (tc_util.cuh, tf32_rna) against
// the cvt.rna.tf32.f32 instruction, including ties and carries into the exponent.
#include <cstdio>
#include <cstdint>
__global__ void k(uint32_t seed, int64_t n, unsigned long long* mism) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t h = (uint32_t)i * 2654435761u ^ seed;
    h ^= h >> 13; h *= 0x5bd1e995u; h ^= h >> 15;
    // finite values with exponents in [2^-60, 2^60]; every 4th a tie, every 8th just below a carry
    uint32_t e = 67 + (h % 120);
    uint32_t m = (h * 2246822519u) & 0x7fffff;
    if ((i & 3) == 0) m = (m & ~0x1fffu) | 0x1000u;
    if ((i & 7) == 1) m = 0x7fffffu;
    uint32_t bits = ((h >> 31) << 31) | (e << 23) | m;
    float x = __uint_as_float(bits);
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    uint32_t mine = (bits + 0x1000u) & 0xffffe000u;
    if (r != mine) atomicAdd(mism, 1ull);
  }
}
int main() {
  unsigned long long* d; cudaMalloc(&d, 8); cudaMemset(d, 0, 8);
  k<<<1024, 256>>>(12345u, 1ll << 26, d);
  unsigned long long h = 0; cudaMemcpy(&h, d, 8, cudaMemcpyDeviceToHost);
  cudaError_t e = cudaDeviceSynchronize();
  printf("tf32 rounding mismatches over 2^26 values: %llu (%s)\n", h, cudaGetErrorString(e));
  return (h == 0 && e == cudaSuccess) ? 0 : 1;
}
