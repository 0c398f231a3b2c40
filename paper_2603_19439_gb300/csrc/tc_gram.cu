// Tensor-core Gram product C = X^T Y for tall-skinny FP32 blocks (the
// projection and CholQR Gram matrices of the mixed-precision step and
// H = Z^T (M Z) of Alg. 1), on tcgen05 with accumulators in tensor memory.
//
// Precision: each FP32 value x is split into x_hi = tf32(x) and
// x_lo = tf32(x - x_hi) (round to nearest), and x y ~ x_hi y_hi + x_hi y_lo +
// x_lo y_hi (three kind::tf32 MMAs), which keeps products at about 2^-22
// relative error; the FP32 accumulator in tensor memory is drained into FP64
// partial sums every kFlushChunks x 32 rows.
//
// Per CTA: one 128-column tile of X (rows of the MMA's M) against all of Y
// (N <= 256), over a contiguous range of rows (the MMA's K).  TMA copies raw
// 32-row tiles of X and Y into a ring of staging buffers; the CTA's threads
// transpose them into K-major, 128B-swizzled hi / lo operand tiles; one
// thread issues the MMAs and commits them to mbarriers.  Every wait on an
// mbarrier is bounded; on timeout the kernel records an error and leaves.
#include <cuda.h>

#include "common.cuh"

namespace grest {

namespace {

constexpr int kRows = 32;         // rows (MMA K) per chunk: 128 B of TF32 per operand row
constexpr int kFlushChunks = 8;   // FP32 accumulation spans 256 rows before the FP64 flush
constexpr int kThreads = 128;
constexpr uint32_t kSpinLimit = 1u << 22;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of element (row, k) in a K-major tile with 128-byte rows, 128B swizzle
__device__ __forceinline__ uint32_t sw128(int row, int kbyte) {
  return (row >> 3) * 1024 + (row & 7) * 128 + ((((kbyte >> 4) ^ (row & 7)) & 7) << 4) + (kbyte & 15);
}

// tcgen05 shared-memory matrix descriptor: K-major, 128B swizzle, 8-row groups 1024 B apart
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)1 << 16;            // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;  // stride byte offset
  d |= (uint64_t)1 << 46;            // descriptor version for tcgen05
  d |= (uint64_t)2 << 61;            // SWIZZLE_128B
  return d;
}

// instruction descriptor: D F32, A and B TF32, both K-major, M x N
__device__ __forceinline__ uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  uint32_t done = 0;
  for (uint32_t it = 0; it < kSpinLimit && !done; ++it) {
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.b32 %0, 1, 0, p;\n}\n"
                 : "=r"(done) : "r"(smem_u32(bar)), "r"(parity) : "memory");
  }
  return done != 0;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
               :: "r"(smem_u32(dst)), "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
               :: "r"(tmem), "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t* r) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
               "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                 "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
                 "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
                 "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

constexpr int kMaxStages = 6;
constexpr int kSmemBudget = 225 * 1024;

// Convert 16-row half h of a staged raw tile (rows x `pitch` floats, row-major)
// into the hi / lo K-major swizzled operand tiles: operand row r = raw column r.
__device__ __forceinline__ void convert_half(const float* __restrict__ raw, int pitch, int rows_op, int r_begin,
                                             int r_step, int h, uint8_t* __restrict__ hi_t, uint8_t* __restrict__ lo_t) {
  for (int r = r_begin; r < rows_op; r += r_step) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int kq = 4 * h + q;
      float4 hi, lo;
      const float v0 = raw[(4 * kq + 0) * pitch + r], v1 = raw[(4 * kq + 1) * pitch + r];
      const float v2 = raw[(4 * kq + 2) * pitch + r], v3 = raw[(4 * kq + 3) * pitch + r];
      hi.x = tf32_rna(v0); lo.x = tf32_rna(v0 - hi.x);
      hi.y = tf32_rna(v1); lo.y = tf32_rna(v1 - hi.y);
      hi.z = tf32_rna(v2); lo.z = tf32_rna(v2 - hi.z);
      hi.w = tf32_rna(v3); lo.w = tf32_rna(v3 - hi.w);
      *(float4*)(hi_t + sw128(r, 16 * kq)) = hi;
      *(float4*)(lo_t + sw128(r, 16 * kq)) = lo;
    }
  }
}

// partT[chunk][j][i] (b x a doubles per chunk, transposed so that lanes, which
// own rows i, store contiguously) receives the CTA's partial X^T Y.
//
// Shared memory: `stages` raw TMA buffers of kRows x (bx + by) floats (a ring,
// refilled as soon as a chunk has been converted), then the hi / lo operand
// tiles A (128 x 128 B) and B (by x 128 B).  Each 32-row chunk is converted and
// multiplied in two 16-row halves (16-byte chunks 0-3 and 4-7 of the swizzled
// 128-byte operand rows), so converting one half overlaps the MMAs of the
// other; threads 0-127 convert X, threads 128-255 convert Y.
__global__ void __launch_bounds__(2 * kThreads, 1)
    k_gram_tc(const __grid_constant__ CUtensorMap mapX, const __grid_constant__ CUtensorMap mapY, int a, int b,
              int bx, int by, int stages, int64_t n, int64_t rows_per_cta, double* __restrict__ partT, int32_t* err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* sm = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full[kMaxStages];
  __shared__ __align__(8) uint64_t mma_bar[2];
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ta = blockIdx.x;
  const int64_t chunk = blockIdx.y;
  const int64_t r0 = chunk * rows_per_cta;
  int64_t r1 = r0 + rows_per_cta;
  if (r1 > n) r1 = n;
  const int nloc = r1 > r0 ? (int)((r1 - r0 + kRows - 1) / kRows) : 0;
  const int ncols = by <= 32 ? 32 : by <= 64 ? 64 : by <= 128 ? 128 : 256;
  const int raw_stage = kRows * (bx + by) * 4;
  const int raw_total = ((stages * raw_stage + 1023) / 1024) * 1024;
  uint8_t* Ahi = sm + raw_total;
  uint8_t* Alo = Ahi + 128 * 128;
  uint8_t* Bhi = Alo + 128 * 128;
  uint8_t* Blo = Bhi + by * 128;
  if (tid == 0) {
    for (int q = 0; q < stages; ++q) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&full[q])));
    for (int q = 0; q < 2; ++q) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&mma_bar[q])));
    asm volatile("fence.mbarrier_init.release.cluster;");
    abort_flag = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(smem_u32(&tmem_base)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;
  const uint32_t idesc = idesc_tf32(128, by);
  const uint32_t tx_bytes = (uint32_t)raw_stage;
  // prologue: fill the ring
  if (tid == 0) {
    for (int i = 0; i < stages && i < nloc; ++i) {
      uint8_t* dst = sm + i * raw_stage;
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(smem_u32(&full[i])), "r"(tx_bytes)
                   : "memory");
      tma_load_2d(dst, &mapX, ta * 128, (int)(r0 + (int64_t)i * kRows), &full[i]);
      tma_load_2d(dst + kRows * bx * 4, &mapY, 0, (int)(r0 + (int64_t)i * kRows), &full[i]);
    }
  }
  bool first_flush = true;
  for (int i = 0; i < nloc; ++i) {
    const int s = i % stages;
    const float* rawx = (const float*)(sm + s * raw_stage);
    const float* rawy = rawx + kRows * bx;
    if (!mbar_wait(&full[s], (uint32_t)((i / stages) & 1))) abort_flag = 1;
    for (int h = 0; h < 2; ++h) {
      // this half of the operand tiles is free once its MMAs of the previous chunk are done
      if (i > 0 && !mbar_wait(&mma_bar[h], (uint32_t)((i - 1) & 1))) abort_flag = 1;
      if (tid < kThreads)
        convert_half(rawx, bx, bx, tid, kThreads, h, Ahi, Alo);
      else
        convert_half(rawy, by, by, tid - kThreads, kThreads, h, Bhi, Blo);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncthreads();
      if (abort_flag) break;
      asm volatile("tcgen05.fence::after_thread_sync;");
      if (tid == 0) {
        const uint32_t acc0 = (h == 1 || (i % kFlushChunks) != 0) ? 1u : 0u;
        const uint32_t ah = smem_u32(Ahi), al = smem_u32(Alo), bh = smem_u32(Bhi), bl = smem_u32(Blo);
#pragma unroll
        for (int kk = 2 * h; kk < 2 * h + 2; ++kk) {
          mma_tf32(tmem, sdesc(ah + 32 * kk), sdesc(bh + 32 * kk), idesc, kk == 2 * h ? acc0 : 1u);
          mma_tf32(tmem, sdesc(ah + 32 * kk), sdesc(bl + 32 * kk), idesc, 1u);
          mma_tf32(tmem, sdesc(al + 32 * kk), sdesc(bh + 32 * kk), idesc, 1u);
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                     :: "r"(smem_u32(&mma_bar[h])) : "memory");
        if (h == 1 && i + stages < nloc) {
          // raw stage s is fully converted: refill it with chunk i + stages
          uint8_t* dst = sm + s * raw_stage;
          const int y = (int)(r0 + (int64_t)(i + stages) * kRows);
          asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(smem_u32(&full[s])),
                       "r"(tx_bytes) : "memory");
          tma_load_2d(dst, &mapX, ta * 128, y, &full[s]);
          tma_load_2d(dst + kRows * bx * 4, &mapY, 0, y, &full[s]);
        }
      }
    }
    if (abort_flag) break;
    if ((i + 1) % kFlushChunks == 0 || i + 1 == nloc) {
      // drain the FP32 accumulator into the FP64 partial sums (all MMAs so far
      // are complete once the last commit of this chunk has arrived)
      if (!mbar_wait(&mma_bar[1], (uint32_t)(i & 1))) abort_flag = 1;
      __syncthreads();
      if (abort_flag) break;
      asm volatile("tcgen05.fence::after_thread_sync;");
      const int quarter = warp & 3, half = warp >> 2;
      const int row = ta * 128 + quarter * 32 + lane;
      for (int c0 = 32 * half; c0 < by; c0 += 64) {
        uint32_t r[32];
        tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)c0, r);
        if (row < a) {
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const int col = c0 + j;
            if (col < b) {
              double* q = partT + (chunk * (int64_t)b + col) * a + row;
              *q = (first_flush ? 0.0 : *q) + (double)__uint_as_float(r[j]);
            }
          }
        }
      }
      first_flush = false;
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncthreads();
    }
  }
  if (nloc == 0) {
    for (int row = ta * 128 + tid; row < a && row < ta * 128 + 128; row += 2 * kThreads)
      for (int col = 0; col < b; ++col) partT[(chunk * (int64_t)b + col) * a + row] = 0.0;
  }
  if (abort_flag && tid == 0) atomicCAS(err, 0, DERR_TIMEOUT);
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(ncols));
}

// ---- host: tensor maps through the driver entry point (no link-time libcuda dependency)
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
    else
      cudaGetLastError();
  }
  return fn;
}

bool make_map(CUtensorMap* m, const float* base, int64_t rows, int cols, int64_t ld, int box_cols) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * sizeof(float)};
  cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)kRows};
  cuuint32_t estr[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

bool gram_tc_supported(const float* X, int64_t ldx, int a, const float* Y, int64_t ldy, int b) {
  if (a < 1 || b < 1 || a > 256 || b > 256) return false;
  if (((uintptr_t)X & 15) || ((uintptr_t)Y & 15) || (ldx & 3) || (ldy & 3)) return false;
  return encode_fn() != nullptr;
}

int gram_f32_tc(const float* X, int64_t ldx, int a, const float* Y, int64_t ldy, int b, int64_t n, double* C,
                int64_t ldc, double* part, int64_t part_cap, int32_t* err, cudaStream_t s) {
  if (n <= 0) return -1;
  const int by = ((b + 15) / 16) * 16;               // MMA N, multiple of 16
  const int nta = (a + 127) / 128;
  const int bx = nta > 1 ? 128 : ((a + 15) / 16) * 16;  // TMA box width of the X tile
  const int operands = 2 * 128 * 128 + 2 * by * 128;
  const int raw_stage = kRows * (bx + by) * 4;
  int stages = (kSmemBudget - operands - 1024) / raw_stage;
  if (stages > kMaxStages) stages = kMaxStages;
  if (stages < 2) return -1;
  CUtensorMap mx, my;
  if (!make_map(&mx, X, n, a, ldx, bx) || !make_map(&my, Y, n, b, ldy, by)) return -1;
  int64_t per_ta = (152 + nta - 1) / nta;
  const int64_t cap_chunks = part_cap / ((int64_t)a * b);
  if (per_ta > cap_chunks) per_ta = cap_chunks;
  const int64_t max_chunks = (n + kRows - 1) / kRows;
  if (per_ta > max_chunks) per_ta = max_chunks;
  if (per_ta < 1) return -1;
  int64_t rows = (n + per_ta - 1) / per_ta;
  rows = ((rows + kRows - 1) / kRows) * kRows;
  const int64_t chunks = (n + rows - 1) / rows;
  const size_t smem = (size_t)((stages * raw_stage + 1023) / 1024) * 1024 + operands + 1024;
  if (!reserve_dynamic_smem(k_gram_tc, smem)) return -1;
  dim3 grid((unsigned)nta, (unsigned)chunks);
  k_gram_tc<<<grid, 2 * kThreads, smem, s>>>(mx, my, a, b, bx, by, stages, n, rows, part, err);
  gram_reduce_launch(part, chunks, a, b, C, ldc, s, true);
  return 0;
}

}  // namespace grest
