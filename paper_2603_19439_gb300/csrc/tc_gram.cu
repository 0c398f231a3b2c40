// Tensor-core Gram product C = X^T Y for tall-skinny FP32 blocks (the CholQR
// Gram matrices of the mixed-precision step and H = Z^T (M Z) of Alg. 1; the
// products with a side of at most 32 columns go to narrow_gram.cu), on
// tcgen05 with accumulators in tensor memory.
//
// Precision: each FP32 value x is split into x_hi = tf32(x) and
// x_lo = tf32(x - x_hi) (round to nearest), and x y ~ x_hi y_hi + x_hi y_lo +
// x_lo y_hi (three kind::tf32 MMAs), which keeps products at about 2^-22
// relative error.  The FP32 accumulator in tensor memory spans 256 rows; it
// is then added into double-float (FP32 hi + lo, two-sum) accumulators held
// in registers, and each CTA's result is written once as FP64.
//
// Each CTA owns a 128 x 128 tile of C (the upper tiles only when X = Y) and a
// contiguous range of rows (the MMA's K).  The contraction runs over rows, so
// the operands (K-major: each operand row is one column of X or Y with its
// rows contiguous) are transposes of the row-major blocks; kind::tf32 takes
// K-major operands only (a transposed-operand descriptor produced no result
// on this part), so the transpose is done by the CTA's threads, pipelined:
//   warp 0     TMA producer: raw 32-row tiles of X and Y into a ring
//   warp 1     tensor-memory owner and MMA issuer (one thread)
//   warps 2-5  transpose + hi / lo split of X into the A operand, written
//              straight into tensor memory (lane = operand row)
//   warps 6-9  the same for Y into the B operand (shared memory, 128B
//              swizzle); every 256 rows all eight warps drain the previous
//              span's accumulator (double-buffered in tensor memory) into
//              double-float registers
// Tensor memory: two 128-column accumulators and four 64-column A stages
// (hi, lo); shared memory: the raw ring and four B stages.
// Every mbarrier wait is bounded; on a timeout the kernel records an error,
// waits (bounded) for its own copies and MMAs in flight, frees its tensor
// memory and returns.
#include "tc_util.cuh"

namespace grest {

using namespace tc;

namespace {

constexpr int kRows = 32;          // rows (MMA K) per chunk: 128 B of TF32 per operand row
constexpr int kSpan = 8;           // chunks per FP32 accumulation span (256 rows)
constexpr int kTileG = 128;        // C tile edge
constexpr int kGramThreads = 320;  // 10 warps
constexpr int kOpBytes = 128 * 128;  // one 128-row K-major operand tile (32 TF32 per row), swizzled
constexpr int kMaxRaw = 4, kMaxOp = 4;
constexpr uint32_t kAcol = 256;  // first tensor-memory column of the A stages (64 columns each)
constexpr int kSmemBudget = 225 * 1024;

struct GramArgs {
  int a, b, n_tiles_m, sym;
  int bxw, byw;          // TMA box widths (columns) of X and Y
  int N;                 // MMA N (multiple of 16, <= 128)
  int raw_stages, op_stages;
  int64_t n, rows_per_split;
  double* partT;         // [split][col][row]: b x a doubles per split
  int32_t* err;
};

__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float x) {
  const float s = hi + x;
  const float bb = s - hi;
  const float e = (hi - (s - bb)) + (x - bb);
  hi = s;
  lo += e;
}

// Transpose + split one raw tile (kRows rows x w columns, row-major) into the
// hi / lo operand tiles: operand row r = raw column r, K = raw row.
template <int Q0, int Q1>
__device__ __forceinline__ void convert_tile(const float* __restrict__ raw, int w, int r, uint8_t* __restrict__ hi_t,
                                             uint8_t* __restrict__ lo_t) {
  if (r >= w) return;
#pragma unroll
  for (int q = Q0; q < Q1; ++q) {
    float4 hi, lo;
    const float v0 = raw[(4 * q + 0) * w + r], v1 = raw[(4 * q + 1) * w + r];
    const float v2 = raw[(4 * q + 2) * w + r], v3 = raw[(4 * q + 3) * w + r];
    hi.x = tf32_rna(v0); lo.x = tf32_rna(v0 - hi.x);
    hi.y = tf32_rna(v1); lo.y = tf32_rna(v1 - hi.y);
    hi.z = tf32_rna(v2); lo.z = tf32_rna(v2 - hi.z);
    hi.w = tf32_rna(v3); lo.w = tf32_rna(v3 - hi.w);
    *(float4*)(hi_t + sw128(r, 16 * q)) = hi;
    *(float4*)(lo_t + sw128(r, 16 * q)) = lo;
  }
}

// Add span sp's FP32 accumulator (buffer sp & 1) into the double-float
// accumulators of this thread's C row and 64 columns.
__device__ __forceinline__ bool drain_span(int sp, uint32_t tmem, int N, int quarter, int colhalf, int lane,
                                           uint64_t* accf, uint64_t* acce, float (&hi)[64], float (&lo)[64]) {
  const int b = sp & 1;
  if (!mbar_wait(&accf[b], (uint32_t)((sp >> 1) & 1))) return false;
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (colhalf * 64 < N) {
    uint32_t v[32];
    tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * 128 + colhalf * 64), v);
#pragma unroll
    for (int j = 0; j < 32; ++j) two_sum_acc(hi[j], lo[j], __uint_as_float(v[j]));
    if (colhalf * 64 + 32 < N) {
      tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * 128 + colhalf * 64 + 32), v);
#pragma unroll
      for (int j = 0; j < 32; ++j) two_sum_acc(hi[32 + j], lo[32 + j], __uint_as_float(v[j]));
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncwarp();
  if (lane == 0) mbar_arrive(&acce[b]);
  return true;
}

// Transpose + split of one raw tile column r (operand row r, K = raw rows)
// into tensor memory: hi at columns [acol, acol + 32), lo at [acol + 32,
// acol + 64) of this warp's lanes; rows beyond the tile width are zero.
__device__ __forceinline__ void convert_a_tmem(const float* __restrict__ raw, int w, int r, uint32_t taddr) {
#pragma unroll
  for (int q = 0; q < kRows / 8; ++q) {
    uint32_t h[8], l[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const float v = r < w ? raw[(8 * q + i) * w + r] : 0.f;
      const float hv = tf32_rna(v);
      h[i] = __float_as_uint(hv);
      l[i] = __float_as_uint(tf32_rna(v - hv));
    }
    tmem_st8(taddr + 8 * q, h);
    tmem_st8(taddr + 32 + 8 * q, l);
  }
  tmem_wait_st();
}

__global__ void __launch_bounds__(kGramThreads, 1)
    k_gram_tc(const __grid_constant__ CUtensorMap mapX, const __grid_constant__ CUtensorMap mapY, const GramArgs p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* sm = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t raw_full[kMaxRaw], raw_empty[kMaxRaw], op_full[kMaxOp], op_empty[kMaxOp];
  __shared__ __align__(8) uint64_t accf[2], acce[2], donebar;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // tile of C
  int tm = 0, tn = 0;
  {
    int t = blockIdx.x;
    if (p.sym) {
      // upper-triangular enumeration: row tm holds tiles tm..T-1
      const int T = p.n_tiles_m;
      while (t >= T - tm) { t -= T - tm; ++tm; }
      tn = tm + t;
    } else {
      tm = t % p.n_tiles_m;
      tn = t / p.n_tiles_m;
    }
  }
  const int m0 = tm * kTileG, n0 = tn * kTileG;
  const bool diag = p.sym && tm == tn;  // X = Y and the same columns: load and convert X only
  const int64_t r0 = (int64_t)blockIdx.y * p.rows_per_split;
  int64_t r1 = r0 + p.rows_per_split;
  if (r1 > p.n) r1 = p.n;
  const int nloc = r1 > r0 ? (int)((r1 - r0 + kRows - 1) / kRows) : 0;
  const int R = p.raw_stages, S = p.op_stages, N = p.N;
  const int raw_bytes = kRows * (p.bxw + p.byw) * 4;
  const int raw_stride = ((raw_bytes + 1023) / 1024) * 1024;
  const int op_b_bytes = N * 128;
  const int op_stride = 2 * op_b_bytes;  // B hi, B lo (A lives in tensor memory)
  uint8_t* raw0 = sm;
  uint8_t* op0 = sm + (size_t)R * raw_stride;
  if (tid == 0) {
    for (int q = 0; q < R; ++q) {
      mbar_init(&raw_full[q], 1);
      mbar_init(&raw_empty[q], 8);
    }
    for (int q = 0; q < S; ++q) {
      mbar_init(&op_full[q], 8);
      mbar_init(&op_empty[q], 1);
    }
    for (int q = 0; q < 2; ++q) {
      mbar_init(&accf[q], 1);
      mbar_init(&acce[q], 8);
    }
    mbar_init(&donebar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;");
    abort_flag = 0;
  }
  const uint32_t ncols = 512u;
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(smem_u32(&tmem_base)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;
  const int nspans = (nloc + kSpan - 1) / kSpan;

  if (warp == 0) {
    // ---------------- TMA producer
    if (lane == 0 && nloc > 0) {
      int issued = 0;
      for (int q = 0; q < nloc; ++q) {
        const int st = q % R;
        if (q >= R && !mbar_wait(&raw_empty[st], (uint32_t)(((q / R) - 1) & 1))) { abort_flag = 1; break; }
        if (abort_flag) break;
        uint8_t* dst = raw0 + (size_t)st * raw_stride;
        const int y = (int)(r0 + (int64_t)q * kRows);
        mbar_expect_tx(&raw_full[st], (uint32_t)(diag ? kRows * p.bxw * 4 : raw_bytes));
        tma_load_2d(dst, &mapX, m0, y, &raw_full[st]);
        if (!diag) tma_load_2d(dst + kRows * p.bxw * 4, &mapY, n0, y, &raw_full[st]);
        issued = q + 1;
      }
      for (int q = issued - R > 0 ? issued - R : 0; q < issued; ++q)
        mbar_wait(&raw_full[q % R], (uint32_t)((q / R) & 1));
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer
    if (lane == 0 && nloc > 0) {
      const uint32_t idesc = idesc_tf32(128, N);
      bool ok = true;
      for (int q = 0; ok && q < nloc; ++q) {
        const int sp = q / kSpan, b = sp & 1;
        if (q % kSpan == 0 && sp >= 2 && !mbar_wait(&acce[b], (uint32_t)(((sp - 2) >> 1) & 1))) { ok = false; break; }
        const int st = q % S;
        if (!mbar_wait(&op_full[st], (uint32_t)((q / S) & 1)) || abort_flag) { ok = false; break; }
        asm volatile("tcgen05.fence::after_thread_sync;");
        uint8_t* op = op0 + (size_t)st * op_stride;
        const uint32_t bh = smem_u32(op), bl = bh + op_b_bytes;
        const uint32_t ah = tmem + kAcol + 64u * st, al = ah + 32u;
        const uint32_t d = tmem + (uint32_t)(b * 128);
#pragma unroll
        for (int k4 = 0; k4 < 4; ++k4) {
          mma_tf32_ts(d, ah + 8 * k4, sdesc(bh + 32 * k4), idesc, (q % kSpan != 0 || k4 > 0) ? 1u : 0u);
          mma_tf32_ts(d, ah + 8 * k4, sdesc(bl + 32 * k4), idesc, 1u);
          mma_tf32_ts(d, al + 8 * k4, sdesc(bh + 32 * k4), idesc, 1u);
        }
        mma_commit(&op_empty[st]);
        if (q % kSpan == kSpan - 1 || q == nloc - 1) mma_commit(&accf[b]);
      }
      if (!ok) abort_flag = 1;
      mma_commit(&donebar);
      mbar_wait(&donebar, 0);
    }
  } else {
    // ---------------- transpose / split, then drain spans into double-float registers
    const int quarter = warp & 3, colhalf = (warp - 2) >> 2;  // colhalf 0: A from X, 1: B from Y
    const int row = quarter * 32 + lane;     // operand row / C row within the tile (TMEM lane)
    const int r = row;
    float hi[64], lo[64];
#pragma unroll
    for (int j = 0; j < 64; ++j) { hi[j] = 0.f; lo[j] = 0.f; }
    bool ok = true;
    for (int q = 0; ok && q < nloc; ++q) {
      const int rs = q % R, os = q % S;
      if (!mbar_wait(&raw_full[rs], (uint32_t)((q / R) & 1))) { ok = false; break; }
      if (q >= S && !mbar_wait(&op_empty[os], (uint32_t)(((q / S) - 1) & 1))) { ok = false; break; }
      if (abort_flag) { ok = false; break; }
      const float* raw = (const float*)(raw0 + (size_t)rs * raw_stride);
      uint8_t* op = op0 + (size_t)os * op_stride;
      if (colhalf == 0) {
        // A (from X) into tensor memory, this warp's lane quarter
        convert_a_tmem(raw, p.bxw, r, tmem + ((uint32_t)(quarter * 32) << 16) + kAcol + 64u * os);
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      } else {
        // B (from Y, or from X on a diagonal tile) into shared memory
        if (r < N) {
          if (diag)
            convert_tile<0, kRows / 4>(raw, p.bxw, r, op, op + op_b_bytes);
          else
            convert_tile<0, kRows / 4>(raw + kRows * p.bxw, p.byw, r, op, op + op_b_bytes);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      }
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(&raw_empty[rs]);
        mbar_arrive(&op_full[os]);
      }
      if (q % kSpan == kSpan - 1 && q / kSpan >= 1) ok = drain_span(q / kSpan - 1, tmem, N, quarter, colhalf, lane, accf, acce, hi, lo);
    }
    if (ok && nspans >= 2 && (nloc % kSpan) != 0)  // the span before a partial last one
      ok = drain_span(nspans - 2, tmem, N, quarter, colhalf, lane, accf, acce, hi, lo);
    if (ok && nspans >= 1) ok = drain_span(nspans - 1, tmem, N, quarter, colhalf, lane, accf, acce, hi, lo);
    if (!ok) abort_flag = 1;
    // write this CTA's partial tile (zeros for an empty row range)
    const int col0 = n0 + colhalf * 64;
    const int ci = m0 + row;
    if (ci < p.a) {
      double* out = p.partT + (int64_t)blockIdx.y * p.b * p.a;
#pragma unroll
      for (int j = 0; j < 64; ++j) {
        const int cj = col0 + j;
        if (cj < p.b && cj < n0 + kTileG) out[(int64_t)cj * p.a + ci] = (double)hi[j] + (double)lo[j];
      }
    }
  }
  __syncthreads();
  if (abort_flag && tid == 0) atomicCAS(p.err, 0, DERR_TIMEOUT);
  asm volatile("tcgen05.fence::before_thread_sync;");
  if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(ncols));
}

// C[i][j] = sum over splits of the partial tiles; with sym, tiles below the
// diagonal were not computed and are read mirrored.
__global__ void k_gram_tc_reduce(const double* __restrict__ partT, int64_t splits, int a, int b, int sym, double* C,
                                 int64_t ldc) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)a * b) return;
  const int j = (int)(e / a), i = (int)(e % a);  // consecutive threads read consecutive rows of a partial
  const bool mirror = sym && (i / kTileG) > (j / kTileG);
  const int64_t off = mirror ? (int64_t)i * a + j : (int64_t)j * a + i;
  double s = 0.0;
  for (int64_t c = 0; c < splits; ++c) s += partT[c * (int64_t)a * b + off];
  C[(int64_t)i * ldc + j] = s;
}

}  // namespace

bool gram_tc_supported(const float* X, int64_t ldx, int a, const float* Y, int64_t ldy, int b) {
  if (a < 1 || b < 1 || a > 256 || b > 256) return false;
  if (((uintptr_t)X & 15) || ((uintptr_t)Y & 15) || (ldx & 3) || (ldy & 3)) return false;
  return encode_fn() != nullptr;
}

int gram_f32_tc(const float* X, int64_t ldx, int a, const float* Y, int64_t ldy, int b, int64_t n, double* C,
                int64_t ldc, double* part, int64_t part_cap, int32_t* err, cudaStream_t s) {
  if (n <= 0 || !gram_tc_supported(X, ldx, a, Y, ldy, b)) return -1;
  GramArgs p;
  p.a = a;
  p.b = b;
  p.sym = (X == Y && a == b && ldx == ldy) ? 1 : 0;
  const int tma = (a + kTileG - 1) / kTileG, tnb = (b + kTileG - 1) / kTileG;
  p.n_tiles_m = tma;
  const int ntiles = p.sym ? tma * (tma + 1) / 2 : tma * tnb;
  p.bxw = a >= kTileG ? kTileG : ((a + 3) / 4) * 4;
  p.byw = b >= kTileG ? kTileG : ((b + 3) / 4) * 4;
  p.N = b >= kTileG ? kTileG : ((b + 15) / 16) * 16;
  const int raw_stride = ((kRows * (p.bxw + p.byw) * 4 + 1023) / 1024) * 1024;
  const int op_stride = 2 * p.N * 128;
  p.op_stages = kMaxOp;
  int R = (kSmemBudget - 1024 - kMaxOp * op_stride) / raw_stride;
  if (R > kMaxRaw) R = kMaxRaw;
  if (R < 2) return -1;
  p.raw_stages = R;
  int dev = 0, nsm = 152;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  // one CTA per SM (shared memory): all tiles x splits in a single wave
  int64_t splits = nsm / ntiles > 0 ? nsm / ntiles : 1;
  const int64_t cap_splits = part_cap / ((int64_t)a * b);
  if (splits > cap_splits) splits = cap_splits;
  const int64_t max_chunks = (n + kRows - 1) / kRows;
  if (splits > max_chunks) splits = max_chunks;
  if (splits < 1) return -1;
  int64_t rows = (n + splits - 1) / splits;
  rows = ((rows + kRows - 1) / kRows) * kRows;
  splits = (n + rows - 1) / rows;
  p.n = n;
  p.rows_per_split = rows;
  p.partT = part;
  p.err = err;
  CUtensorMap mx, my;
  if (!make_map_f32(&mx, X, n, a, ldx, p.bxw, kRows, false) || !make_map_f32(&my, Y, n, b, ldy, p.byw, kRows, false))
    return -1;
  const size_t smem = (size_t)R * raw_stride + (size_t)kMaxOp * op_stride + 1024;
  if (!reserve_dynamic_smem(k_gram_tc, smem)) return -1;
  dim3 grid((unsigned)ntiles, (unsigned)splits);
  k_gram_tc<<<grid, kGramThreads, smem, s>>>(mx, my, p);
  const int64_t tot = (int64_t)a * b;
  k_gram_tc_reduce<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(part, splits, a, b, p.sym, C, ldc);
  return 0;
}

namespace tc {

EncodeTiledFn encode_fn() {
  // initialized once, thread-safely (function-local static)
  static const EncodeTiledFn fn = []() -> EncodeTiledFn {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return reinterpret_cast<EncodeTiledFn>(p);
    cudaGetLastError();
    return nullptr;
  }();
  return fn;
}

bool make_map_f32(CUtensorMap* m, const float* base, int64_t rows, int cols, int64_t ld, int box_cols, int box_rows,
                  bool swizzle128) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * sizeof(float)};
  cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace tc

}  // namespace grest
