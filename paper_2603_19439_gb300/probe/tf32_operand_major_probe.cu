// Probe: tcgen05.mma kind::tf32 with MN-major (transposed) A and B operands in
// the 128B-swizzled layout that a TMA box {32 elements, 32 rows} produces.
// Checks which descriptor stride field carries the MN-atom stride.  All smem
// reads stay inside the two 16 KB tiles for either interpretation.
#include <cstdio>
#include <cstdint>
#include <cstdlib>
#include <cmath>

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint32_t sw128(int row, int kbyte) {
  return (row >> 3) * 1024 + (row & 7) * 128 + ((((kbyte >> 4) ^ (row & 7)) & 7) << 4) + (kbyte & 15);
}
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}
__global__ void __launch_bounds__(128) k_probe(const float* A, const float* B, float* D, uint32_t lbo, uint32_t sbo, int mnA, int mnB, int steps) {
  extern __shared__ uint8_t raw[];
  uint8_t* sm = (uint8_t*)(((uintptr_t)raw + 1023) & ~(uintptr_t)1023);
  uint8_t* As = sm;
  uint8_t* Bs = sm + 16384;
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tbase;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // fill: element (m, k), m < 128, k < 32
  for (int e = tid; e < 128 * 32; e += 128) {
    const int m = e / 32, k = e % 32;
    const uint32_t offmn = (m / 32) * 4096 + sw128(k, 4 * (m % 32));   // MN-major: rows = k, 32 m per 128 B
    const uint32_t offk = sw128(m, 4 * k);                              // K-major
    *(float*)(As + (mnA ? offmn : offk)) = A[m * 32 + k];
    *(float*)(Bs + (mnB ? offmn : offk)) = B[m * 32 + k];
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&bar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" :: "r"(smem_u32(&tbase)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tm = tbase;
  if (tid == 0) {
    uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((128u >> 3) << 17) | ((128u >> 4) << 24);
    if (mnA) idesc |= (1u << 15);
    if (mnB) idesc |= (1u << 16);
    for (int s = 0; s < steps; ++s) {
      const uint64_t da = mnA ? sdesc(smem_u32(As) + 1024 * s, lbo, sbo) : sdesc(smem_u32(As) + 32 * s, 16, 1024);
      const uint64_t db = mnB ? sdesc(smem_u32(Bs) + 1024 * s, lbo, sbo) : sdesc(smem_u32(Bs) + 32 * s, 16, 1024);
      const uint32_t acc = s > 0;
      asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
                   :: "r"(tm), "l"(da), "l"(db), "r"(idesc), "r"(acc));
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" :: "r"(smem_u32(&bar)) : "memory");
  }
  __syncwarp();
  uint32_t done = 0;
  for (uint32_t it = 0; it < (1u << 22) && !done; ++it)
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.b32 %0, 1, 0, p;\n}\n"
                 : "=r"(done) : "r"(smem_u32(&bar)), "r"(0) : "memory");
  asm volatile("tcgen05.fence::after_thread_sync;");
  for (int c0 = 0; c0 < 128; c0 += 32) {
    uint32_t r[32];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                 "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
                   "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
                   "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                 : "r"(tm + ((uint32_t)(warp * 32) << 16) + c0));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    for (int j = 0; j < 32; ++j) D[(warp * 32 + lane) * 128 + c0 + j] = __uint_as_float(r[j]);
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" :: "r"(tm));
  if (tid == 0 && !done) D[0] = NAN;
}

int main() {
  const int M = 128, K = 32;
  float *hA = (float*)malloc(M * K * 4), *hB = (float*)malloc(M * K * 4), *hD = (float*)malloc(M * M * 4);
  srand(7);
  for (int i = 0; i < M * K; ++i) { hA[i] = (float)(rand() % 9 - 4); hB[i] = (float)(rand() % 9 - 4); }
  float *A, *B, *D;
  cudaMalloc(&A, M * K * 4); cudaMalloc(&B, M * K * 4); cudaMalloc(&D, M * M * 4);
  cudaMemcpy(A, hA, M * K * 4, cudaMemcpyHostToDevice);
  cudaMemcpy(B, hB, M * K * 4, cudaMemcpyHostToDevice);
  cudaFuncSetAttribute(k_probe, cudaFuncAttributeMaxDynamicSharedMemorySize, 40 * 1024);
  struct V { uint32_t lbo, sbo; int mnA, mnB, steps; } vs[] = {
      {16, 1024, 0, 0, 1}, {4096, 1024, 1, 0, 1}, {1024, 4096, 1, 0, 1}, {4096, 1024, 0, 1, 1}, {1024, 4096, 0, 1, 1},
      {4096, 1024, 1, 1, 1}, {1024, 4096, 1, 1, 1}, {4096, 1024, 1, 1, 4}};
  for (auto& v : vs) {
    cudaMemset(D, 0, M * M * 4);
    k_probe<<<1, 128, 40 * 1024>>>(A, B, D, v.lbo, v.sbo, v.mnA, v.mnB, v.steps);
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) { printf("CUDA error %s\n", cudaGetErrorString(e)); return 1; }
    cudaMemcpy(hD, D, M * M * 4, cudaMemcpyDeviceToHost);
    const int Kuse = 8 * v.steps;
    printf("mnA=%d mnB=%d lbo=%u sbo=%u steps=%d  block max err (rows: M atom, cols: N atom):\n", v.mnA, v.mnB, v.lbo, v.sbo, v.steps);
    for (int bm = 0; bm < 4; ++bm) {
      printf("   ");
      for (int bn = 0; bn < 4; ++bn) {
        double me = 0;
        for (int m = bm * 32; m < bm * 32 + 32; ++m)
          for (int n = bn * 32; n < bn * 32 + 32; ++n) {
            double ref = 0;
            for (int k = 0; k < Kuse; ++k) ref += (double)hA[m * K + k] * hB[n * K + k];
            me = fmax(me, fabs(ref - hD[m * M + n]));
          }
        printf(" %6.0f", me);
      }
      printf("\n");
    }
    // does D match A^T-style misreads? check a few alternative hypotheses for mnA only, steps=1
    if (v.mnA && !v.mnB && v.steps == 1) {
      // hypothesis: hardware reads element (m, k) from the K-major position of (m, k) in an MN tile?
      double best = 1e30; int bestp = -1;
      for (int p = 0; p < 4; ++p) {  // k offset within the atom rows
        double me = 0;
        for (int m = 0; m < 32; ++m) for (int n = 0; n < 32; ++n) {
          double ref = 0;
          for (int k = 0; k < 8; ++k) ref += (double)hA[m * K + ((k + 8 * p) % 32)] * hB[n * K + k];
          me = fmax(me, fabs(ref - hD[m * M + n]));
        }
        if (me < best) { best = me; bestp = p; }
      }
      printf("   [M atom 0: best k-offset hypothesis p=%d err=%g]\n", bestp, best);
    }
  }
  return 0;
}
