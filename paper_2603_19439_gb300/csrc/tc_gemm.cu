// Tensor-core tall-skinny GEMM Out = beta Cin + alpha X B for the FP32 N x w
// blocks of the mixed-precision step (projections X - U (U^T X), the CholQR
// applications V T, the RSVD lift R = M U_hat of Sec. 3.5, and X = Z F_K of
// Alg. 2), on tcgen05 with accumulators in tensor memory.
//
// Each MMA takes a 128-row tile of X as its A operand (M = 128 rows), all of
// B's c <= 256 columns as its B operand (N = c rounded up to 16) and 8 of X's
// columns as K; a tcgen05 kind::tf32 instruction costs about the same up to
// N = 128 and only ~1.45x that at N = 256, so covering every output column in
// one instruction halves the instruction count against 128-column tiles.  X
// is row-major, so its row tiles are already K-major: TMA writes them straight
// into the 128B-swizzled operand layout and the TF32 hi / lo split (3xTF32:
// x y ~ x_hi y_hi + x_hi y_lo + x_lo y_hi) is an in-place elementwise pass.
// B^T (output column = operand row, K contiguous) is scaled by alpha, split
// and laid out as shared-memory images once per call (k_gemm_prep); it stays
// resident when small, else it is re-read from L2 with each 32-column chunk
// of X.
//
// Warp roles (192 threads, one CTA per SM, persistent over row tiles):
//   warp 0     TMA producer (X chunks, B^T images) into a ring of stages
//   warp 1     tensor-memory owner and MMA issuer (one thread)
//   warps 2-5  split each X chunk into hi / lo, then drain the previous
//              tile's accumulator to Out: warp w owns TMEM lanes (= tile
//              rows) 32 (w mod 4) .. + 31 and moves 32-column blocks of them
// Accumulators are double-buffered in tensor memory (2 x 256 columns), so
// the epilogue of tile t overlaps the MMAs of tile t + 1.  Every mbarrier
// wait is bounded; on a timeout the kernel records an error, waits (bounded)
// for its own copies and MMAs in flight, frees its tensor memory and returns.
#include <string.h>

#include "tc_util.cuh"

namespace grest {

using namespace tc;

namespace {

constexpr int kTile = 128;               // X rows per tile (MMA M)
constexpr int kChunkBytes = 128 * 128;   // 128 rows x 32 FP32 (128 B), swizzled
constexpr int kBlkBytes = 32 * 128;      // epilogue block: 32 rows x 32 FP32, swizzled
constexpr uint32_t kAccCols = 256;       // tensor-memory columns per accumulator buffer
constexpr int kGemmThreads = 192;
constexpr int kMaxStagesG = 4;
constexpr int kSmemBudgetG = 225 * 1024;

// B^T images: K chunk kc, part (0 hi, 1 lo) at (kc * 2 + part) * Np * 128
// bytes, element (j, k) (j = output column, k = row of B) at
// sw128(j, 4 (k mod 32)): an Np-row K-major operand tile.  Rows j >= c and
// columns k >= a are zero.
__global__ void k_gemm_prep(const double* __restrict__ B, int64_t ldb, int a, int c, double alpha, int Np, int Kc,
                            uint8_t* __restrict__ img) {
  const int64_t total = (int64_t)Kc * Np * 32;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int kk = (int)(e & 31);
    const int j = (int)((e >> 5) % Np);
    const int kc = (int)((e >> 5) / Np);
    const int k = kc * 32 + kk;
    const double v = (j < c && k < a) ? alpha * B[(int64_t)k * ldb + j] : 0.0;
    const float hi = tf32_rna((float)v);
    const float lo = tf32_rna((float)(v - (double)hi));
    uint8_t* base = img + (size_t)kc * 2 * Np * 128;
    *(float*)(base + sw128(j, 4 * kk)) = hi;
    *(float*)(base + (size_t)Np * 128 + sw128(j, 4 * kk)) = lo;
  }
}

struct GemmArgs {
  const uint8_t* img;  // B^T images
  int64_t n;
  int a, c, Np, Kc, stages, a_res;
  int eslots;          // staging slots per epilogue warp (0: direct stores)
  const float* Cin;
  int64_t ldc;
  float beta;
  float* Out;
  int64_t ldo;
  int32_t* err;
};

// Drain accumulator buffer (it & 1) of the CTA's tile `it` into Out (and add
// beta Cin): TMEM lane = row of the tile, TMEM column = output column, so each
// thread moves 32 consecutive columns of its row per block.
__device__ __forceinline__ bool drain_tile(const GemmArgs& p, uint32_t tmem, int it, int quarter, int lane,
                                           uint64_t* accf, uint64_t* acce) {
  const int b = it & 1;
  if (!mbar_wait(&accf[b], (uint32_t)((it >> 1) & 1))) return false;
  asm volatile("tcgen05.fence::after_thread_sync;");
  const int64_t row = (blockIdx.x + (int64_t)it * gridDim.x) * kTile + quarter * 32 + lane;
  for (int j0 = 0; j0 < p.c; j0 += 32) {
    uint32_t r[32];
    tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * kAccCols + j0), r);
    if (row < p.n) {
      // Cin may be Out (in-place update): read the whole fragment first
      float cin[32];
#pragma unroll
      for (int i = 0; i < 32; ++i) cin[i] = (p.beta != 0.0f && j0 + i < p.c) ? p.Cin[row * p.ldc + j0 + i] : 0.0f;
#pragma unroll
      for (int i = 0; i < 32; ++i)
        if (j0 + i < p.c) p.Out[row * p.ldo + j0 + i] = fmaf(p.beta, cin[i], __uint_as_float(r[i]));
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncwarp();
  if (lane == 0) mbar_arrive(&acce[b]);
  return true;
}

// Staged drain: the warp's 32-row x 32-column output blocks go through
// 4 KB shared-memory slots (128B-swizzled rows): beta Cin arrives there by TMA
// (issued ahead of time), the accumulator is added in place, and one TMA
// store writes the block (rows >= n and columns >= c are clipped).  Block kb
// of this warp is column block kb mod nvb of its tile kb / nvb; slot kb mod
// eslots.
__device__ __forceinline__ void cin_prefetch(const GemmArgs& p, const CUtensorMap* mapCin, uint8_t* E,
                                             uint64_t* cin_bar, int quarter, int nvb, int64_t kb) {
  const int it = (int)(kb / nvb), jb = (int)(kb % nvb);
  const int slot = (int)(kb % p.eslots);
  const int64_t row0 = (blockIdx.x + (int64_t)it * gridDim.x) * kTile + quarter * 32;
  mbar_expect_tx(&cin_bar[slot], (uint32_t)kBlkBytes);
  tma_load_2d(E + (size_t)slot * kBlkBytes, mapCin, jb * 32, (int)row0, &cin_bar[slot]);
}

__device__ __forceinline__ bool drain_tile_staged(const GemmArgs& p, const CUtensorMap* mapOut,
                                                  const CUtensorMap* mapCin, uint32_t tmem, int it, int quarter,
                                                  int lane, uint64_t* accf, uint64_t* acce, uint8_t* E,
                                                  uint64_t* cin_bar, int nvb, int64_t nblocks, int64_t& cin_issued,
                                                  int64_t& cin_waited) {
  const int b = it & 1;
  if (!mbar_wait(&accf[b], (uint32_t)((it >> 1) & 1))) return false;
  asm volatile("tcgen05.fence::after_thread_sync;");
  const int64_t row0 = (blockIdx.x + (int64_t)it * gridDim.x) * kTile + quarter * 32;
  const bool has_cin = p.beta != 0.0f;
  for (int jb = 0; jb < nvb; ++jb) {
    const int64_t kb = (int64_t)it * nvb + jb;
    const int slot = (int)(kb % p.eslots);
    uint8_t* Es = E + (size_t)slot * kBlkBytes;
    if (has_cin) {
      if (!mbar_wait(&cin_bar[slot], (uint32_t)((kb / p.eslots) & 1))) return false;
      cin_waited = kb + 1;
    } else {
      // the slot's previous store must have finished reading it (one store per block, in order)
      if (lane == 0) {
        if (p.eslots == 4) bulk_wait_read<3>();
        else if (p.eslots == 3) bulk_wait_read<2>();
        else if (p.eslots == 2) bulk_wait_read<1>();
        else bulk_wait_read<0>();
      }
      __syncwarp();
    }
    uint32_t r[32];
    tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * kAccCols + jb * 32), r);
#pragma unroll
    for (int q4 = 0; q4 < 8; ++q4) {
      float4* e = (float4*)(Es + sw128(lane, 16 * q4));
      float4 v = has_cin ? *e : make_float4(0.f, 0.f, 0.f, 0.f);
      v.x = fmaf(p.beta, v.x, __uint_as_float(r[4 * q4 + 0]));
      v.y = fmaf(p.beta, v.y, __uint_as_float(r[4 * q4 + 1]));
      v.z = fmaf(p.beta, v.z, __uint_as_float(r[4 * q4 + 2]));
      v.w = fmaf(p.beta, v.w, __uint_as_float(r[4 * q4 + 3]));
      *e = v;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncwarp();
    if (lane == 0) {
      tma_store_2d(mapOut, Es, jb * 32, (int)row0);
      bulk_commit();
      if (has_cin && kb + p.eslots < nblocks) {
        bulk_wait_read<0>();  // this slot is free once the store has read it
        cin_prefetch(p, mapCin, E, cin_bar, quarter, nvb, kb + p.eslots);
      }
    }
    if (has_cin && kb + p.eslots < nblocks) cin_issued = kb + p.eslots + 1;
    __syncwarp();
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncwarp();
  if (lane == 0) mbar_arrive(&acce[b]);
  return true;
}

__global__ void __launch_bounds__(kGemmThreads, 1)
    k_gemm_tc(const __grid_constant__ CUtensorMap mapX, const __grid_constant__ CUtensorMap mapOut,
              const __grid_constant__ CUtensorMap mapCin, const GemmArgs p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* sm = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full[kMaxStagesG], conv[kMaxStagesG], empty[kMaxStagesG];
  __shared__ __align__(8) uint64_t accf[2], acce[2], abar, donebar;
  __shared__ __align__(8) uint64_t cin_bar[4][4];
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int Np = p.Np, Kc = p.Kc, stages = p.stages;
  const int64_t ntiles = (p.n + kTile - 1) / kTile;
  const int my_tiles = blockIdx.x < ntiles ? (int)((ntiles - 1 - blockIdx.x) / gridDim.x + 1) : 0;
  const int64_t nchunks = (int64_t)my_tiles * Kc;
  const uint32_t a_tile_bytes = (uint32_t)(2 * Np * 128);  // hi + lo B^T images of one K chunk
  uint8_t* Ares = sm;
  const size_t ares_bytes = p.a_res ? (size_t)Kc * a_tile_bytes : 0;
  const size_t stage_bytes = 2 * kChunkBytes + (p.a_res ? 0 : a_tile_bytes);
  uint8_t* stage0 = sm + ares_bytes;
  if (tid == 0) {
    for (int q = 0; q < stages; ++q) {
      mbar_init(&full[q], 1);
      mbar_init(&conv[q], 4);
      mbar_init(&empty[q], 1);
    }
    for (int q = 0; q < 2; ++q) {
      mbar_init(&accf[q], 1);
      mbar_init(&acce[q], 4);
    }
    mbar_init(&abar, 1);
    mbar_init(&donebar, 1);
    for (int q = 0; q < 4; ++q)
      for (int e = 0; e < 4; ++e) mbar_init(&cin_bar[q][e], 1);
    asm volatile("fence.mbarrier_init.release.cluster;");
    abort_flag = 0;
  }
  const uint32_t ncols = 2 * kAccCols;
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(smem_u32(&tmem_base)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;

  if (warp == 0) {
    // ---------------- TMA producer
    if (lane == 0 && nchunks > 0) {
      if (p.a_res) {
        mbar_expect_tx(&abar, (uint32_t)ares_bytes);
        bulk_load(Ares, p.img, (uint32_t)ares_bytes, &abar);
      }
      int64_t issued = 0;
      for (int64_t q = 0; q < nchunks; ++q) {
        const int s = (int)(q % stages);
        const int64_t u = q / stages;
        if (u > 0 && !mbar_wait(&empty[s], (uint32_t)((u - 1) & 1))) { abort_flag = 1; break; }
        if (abort_flag) break;
        const int it = (int)(q / Kc), kc = (int)(q % Kc);
        const int64_t tile = blockIdx.x + (int64_t)it * gridDim.x;
        uint8_t* st = stage0 + (size_t)s * stage_bytes;
        mbar_expect_tx(&full[s], (uint32_t)kChunkBytes + (p.a_res ? 0u : a_tile_bytes));
        tma_load_2d(st, &mapX, kc * 32, (int)(tile * kTile), &full[s]);
        if (!p.a_res) bulk_load(st + 2 * kChunkBytes, p.img + (size_t)kc * a_tile_bytes, a_tile_bytes, &full[s]);
        issued = q + 1;
      }
      // wait for the copies still in flight (all of them on the normal path
      // were consumed already, so these waits return at once)
      for (int64_t q = issued - stages > 0 ? issued - stages : 0; q < issued; ++q)
        mbar_wait(&full[q % stages], (uint32_t)((q / stages) & 1));
      if (p.a_res) mbar_wait(&abar, 0);
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer
    if (lane == 0 && nchunks > 0) {
      const uint32_t idesc = idesc_tf32(kTile, Np);
      bool ok = !p.a_res || mbar_wait(&abar, 0);
      for (int it = 0; ok && it < my_tiles; ++it) {
        const int b = it & 1;
        if (it >= 2 && !mbar_wait(&acce[b], (uint32_t)(((it - 2) >> 1) & 1))) { ok = false; break; }
        asm volatile("tcgen05.fence::after_thread_sync;");
        for (int kc = 0; kc < Kc; ++kc) {
          const int64_t q = (int64_t)it * Kc + kc;
          const int s = (int)(q % stages);
          if (!mbar_wait(&conv[s], (uint32_t)((q / stages) & 1)) || abort_flag) { ok = false; break; }
          asm volatile("tcgen05.fence::after_thread_sync;");
          uint8_t* st = stage0 + (size_t)s * stage_bytes;
          const uint32_t xh = smem_u32(st), xl = smem_u32(st + kChunkBytes);
          const uint8_t* bbase = p.a_res ? Ares + (size_t)kc * a_tile_bytes : st + 2 * kChunkBytes;
          const uint32_t bh = smem_u32(bbase), bl = bh + (uint32_t)(Np * 128);
          const uint32_t d = tmem + (uint32_t)(b * kAccCols);
#pragma unroll
          for (int k4 = 0; k4 < 4; ++k4) {
            mma_tf32(d, sdesc(xh + 32 * k4), sdesc(bh + 32 * k4), idesc, (kc > 0 || k4 > 0) ? 1u : 0u);
            mma_tf32(d, sdesc(xh + 32 * k4), sdesc(bl + 32 * k4), idesc, 1u);
            mma_tf32(d, sdesc(xl + 32 * k4), sdesc(bh + 32 * k4), idesc, 1u);
          }
          mma_commit(&empty[s]);
        }
        if (!ok) break;
        mma_commit(&accf[b]);
      }
      if (!ok) abort_flag = 1;
      // every MMA issued so far has completed once this commit arrives
      mma_commit(&donebar);
      mbar_wait(&donebar, 0);
    }
  } else {
    // ---------------- split X into hi / lo, drain accumulators to Out
    const int ct = tid - 64;  // 0..127
    const int quarter = warp & 3;
    uint8_t* E = stage0 + (size_t)stages * stage_bytes + (size_t)quarter * p.eslots * kBlkBytes;
    const int nvb = (p.c + 31) / 32;  // 32-column output blocks per tile row group
    const int64_t nblocks = (int64_t)my_tiles * nvb;
    int64_t cin_issued = 0, cin_waited = 0;  // Cin blocks loaded / consumed by this warp
    if (p.eslots > 0 && p.beta != 0.0f) {
      for (int64_t kb = 0; kb < p.eslots && kb < nblocks; ++kb) {
        if (lane == 0) cin_prefetch(p, &mapCin, E, cin_bar[quarter], quarter, nvb, kb);
        cin_issued = kb + 1;
      }
    }
    bool ok = true;
    for (int it = 0; ok && it < my_tiles; ++it) {
      for (int kc = 0; kc < Kc; ++kc) {
        const int64_t q = (int64_t)it * Kc + kc;
        const int s = (int)(q % stages);
        if (!mbar_wait(&full[s], (uint32_t)((q / stages) & 1)) || abort_flag) { ok = false; break; }
        uint8_t* st = stage0 + (size_t)s * stage_bytes;
#pragma unroll
        for (int u = 0; u < kChunkBytes / 16 / 128; ++u) {
          const int off = (u * 128 + ct) * 16;
          float4 v = *(const float4*)(st + off), hi, lo;
          hi.x = tf32_rna(v.x); lo.x = tf32_rna(v.x - hi.x);
          hi.y = tf32_rna(v.y); lo.y = tf32_rna(v.y - hi.y);
          hi.z = tf32_rna(v.z); lo.z = tf32_rna(v.z - hi.z);
          hi.w = tf32_rna(v.w); lo.w = tf32_rna(v.w - hi.w);
          *(float4*)(st + off) = hi;
          *(float4*)(st + kChunkBytes + off) = lo;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(&conv[s]);
      }
      if (ok && it > 0)
        ok = p.eslots ? drain_tile_staged(p, &mapOut, &mapCin, tmem, it - 1, quarter, lane, accf, acce, E,
                                          cin_bar[quarter], nvb, nblocks, cin_issued, cin_waited)
                      : drain_tile(p, tmem, it - 1, quarter, lane, accf, acce);
    }
    if (ok && my_tiles > 0)
      ok = p.eslots ? drain_tile_staged(p, &mapOut, &mapCin, tmem, my_tiles - 1, quarter, lane, accf, acce, E,
                                        cin_bar[quarter], nvb, nblocks, cin_issued, cin_waited)
                    : drain_tile(p, tmem, my_tiles - 1, quarter, lane, accf, acce);
    if (!ok) abort_flag = 1;
    if (p.eslots > 0 && lane == 0) {
      // Cin loads issued but not consumed (abort path only), then every store complete
      for (int64_t kb = cin_waited; kb < cin_issued; ++kb)
        mbar_wait(&cin_bar[quarter][kb % p.eslots], (uint32_t)((kb / p.eslots) & 1));
      bulk_wait_all();
    }
  }
  __syncthreads();
  if (abort_flag && tid == 0) atomicCAS(p.err, 0, DERR_TIMEOUT);
  asm volatile("tcgen05.fence::before_thread_sync;");
  if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(ncols));
}

}  // namespace

size_t gemm_tc_img_bytes(int a, int c) {
  const int Np = (c + 15) / 16 * 16, Kc = (a + 31) / 32;
  return (size_t)Kc * 2 * Np * 128;
}

bool gemm_tc_supported(int64_t n, int a, int c, const float* X, int64_t ldx, const float* Cin, int64_t ldc,
                       const float* Out, int64_t ldo) {
  if (n < 1 || a < 1 || c < 1 || c > 256 || a > 512) return false;
  if (((uintptr_t)X & 15) || (ldx & 3)) return false;
  (void)Cin; (void)ldc; (void)Out; (void)ldo;
  return encode_fn() != nullptr;
}

// Returns 0 on success (two kernels enqueued), -1 when the tensor-core path
// cannot take the call (nothing enqueued).
int gemm_f32_tc(int64_t n, int a, int c, double alpha, const float* X, int64_t ldx, const double* B, int64_t ldb,
                double beta, const float* Cin, int64_t ldc, float* Out, int64_t ldo, uint8_t* img, size_t img_cap,
                int32_t* err, cudaStream_t s) {
  if (!gemm_tc_supported(n, a, c, X, ldx, Cin, ldc, Out, ldo)) return -1;
  const int Np = (c + 15) / 16 * 16, Kc = (a + 31) / 32;
  const size_t img_bytes = (size_t)Kc * 2 * Np * 128;
  if (img_bytes > img_cap) return -1;
  const size_t a_tile = (size_t)2 * Np * 128;
  CUtensorMap mx, mout, mcin;
  memset(&mout, 0, sizeof(mout));
  memset(&mcin, 0, sizeof(mcin));
  if (!make_map_f32(&mx, X, n, a, ldx, 32, kTile, true)) return -1;
  // output staging through shared memory needs TMA-compatible Out (and Cin)
  bool can_stage = ((uintptr_t)Out & 15) == 0 && (ldo & 3) == 0 && make_map_f32(&mout, Out, n, c, ldo, 32, 32, true);
  if (beta != 0.0)
    can_stage = can_stage && ((uintptr_t)Cin & 15) == 0 && (ldc & 3) == 0 &&
                make_map_f32(&mcin, Cin, n, c, ldc, 32, 32, true);
  else
    mcin = mout;
  // pick (resident B^T images?, staging slots, stages) within the budget
  const bool res_fits = img_bytes + 2 * kChunkBytes + 1024 <= (size_t)kSmemBudgetG;
  const int min_stages = Kc > 1 ? 2 : 1;
  int a_res = 0, stages = 0, eslots = 0;
  for (int es = can_stage ? 4 : 0; es >= 0 && stages == 0; --es) {
    const size_t ebytes = (size_t)4 * es * kBlkBytes;
    for (int res = res_fits ? 1 : 0; res >= 0 && stages == 0; --res) {
      const size_t fixed = 1024 + ebytes + (res ? img_bytes : 0);
      if (fixed >= (size_t)kSmemBudgetG) continue;
      int st = (int)((kSmemBudgetG - fixed) / (2 * kChunkBytes + (res ? 0 : a_tile)));
      if (st > kMaxStagesG) st = kMaxStagesG;
      if (st >= (res ? min_stages : 2) && (es > 0 || st >= 2)) {
        stages = st;
        a_res = res;
        eslots = es;
      }
    }
  }
  if (stages == 0) return -1;
  size_t smem = (a_res ? img_bytes : 0) + (size_t)stages * (2 * kChunkBytes + (a_res ? 0 : a_tile)) +
                (size_t)4 * eslots * kBlkBytes + 1024;
  // the kernel takes all 512 tensor-memory columns: keep one CTA per SM
  if (smem < 116 * 1024) smem = 116 * 1024;
  if (!reserve_dynamic_smem(k_gemm_tc, smem)) return -1;
  const int64_t total = (int64_t)Kc * Np * 32;
  k_gemm_prep<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(B, ldb, a, c, alpha, Np, Kc, img);
  GemmArgs p;
  p.img = img;
  p.n = n;
  p.a = a;
  p.c = c;
  p.Np = Np;
  p.Kc = Kc;
  p.stages = stages;
  p.a_res = a_res;
  p.eslots = eslots;
  p.Cin = Cin;
  p.ldc = ldc;
  p.beta = (float)beta;
  p.Out = Out;
  p.ldo = ldo;
  p.err = err;
  const int64_t ntiles = (n + kTile - 1) / kTile;
  int dev = 0, nsm = 152;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const unsigned grid = (unsigned)(ntiles < nsm ? ntiles : nsm);
  k_gemm_tc<<<grid, kGemmThreads, smem, s>>>(mx, mout, mcin, p);
  return 0;
}

}  // namespace grest
