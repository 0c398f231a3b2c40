// CSR SpMM Y = M X over tall-skinny row-major blocks, with the operator of
// Sec. 4.2 applied in the epilogue:
//   ADJ   y_r = sum_j a_rj x_j
//   LAP   y_r = (alpha - d_r) x_r + sum_j a_rj x_j,   alpha = 2 d_max
//   NLAP  y_r = x_r + s_r sum_j a_rj s_j x_j,          s = d^-1/2
// Tombstoned rows give zero (principal submatrix on live nodes).
//
// Scheduling: one warp per row; the warp loads 32 column indices at a time
// (coalesced) and broadcasts them by shuffle, then every lane gathers its
// columns of the neighbour's row (a whole row of X is one contiguous run, so
// a gather is fully coalesced).  Rows longer than kLongRow (hubs of power-law
// graphs) go to a second kernel where a block of 16 warps splits the
// neighbour list and reduces in shared memory in a fixed order, so results
// are deterministic.
#include "common.cuh"

namespace grest {

namespace {

template <typename T, int NCH>
struct Acc {
  T v[NCH];
};

template <typename Tx, typename T, int NCH, bool HASVAL>
__device__ __forceinline__ void gather_range(const int32_t* __restrict__ col, const double* __restrict__ val,
                                             int64_t beg, int64_t end, const OpParams& op, const Tx* __restrict__ X,
                                             int64_t ldx, int w, int64_t col_lo, int lane, Acc<T, NCH>& acc) {
  const bool nl = op.op == GREST_OP_NLAP;
  if (!HASVAL && !nl) {
    // unit weights: the same sums as below with a = 1 (fma(1, y, t) = t + y
    // exactly), without the multiplications, which cost a full FP64 pipe
    // slot each when T is double
    for (int64_t j0 = beg; j0 < end; j0 += 32) {
      const int64_t j = j0 + lane;
      const int32_t mc = j < end ? col[j] : 0;
      const int cnt = (int)((end - j0) < 32 ? (end - j0) : 32);
      int k = 0;
      for (; NCH <= 2 && k + 8 <= cnt; k += 8) {
        int32_t cc[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) cc[q] = __shfl_sync(0xffffffffu, mc, k + q);
#pragma unroll
        for (int ch = 0; ch < NCH; ++ch) {
          const int c = ch * 32 + lane;
          if (c < w) {
            T y[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) y[q] = (T)__ldg(X + (int64_t)(cc[q] - col_lo) * ldx + c);
            acc.v[ch] += ((y[0] + y[1]) + y[2]) + y[3];
            acc.v[ch] += ((y[4] + y[5]) + y[6]) + y[7];
          }
        }
      }
      for (; k + 4 <= cnt; k += 4) {
        const int32_t c0 = __shfl_sync(0xffffffffu, mc, k), c1 = __shfl_sync(0xffffffffu, mc, k + 1);
        const int32_t c2 = __shfl_sync(0xffffffffu, mc, k + 2), c3 = __shfl_sync(0xffffffffu, mc, k + 3);
#pragma unroll
        for (int ch = 0; ch < NCH; ++ch) {
          const int c = ch * 32 + lane;
          if (c < w) {
            const T y0 = (T)__ldg(X + (int64_t)(c0 - col_lo) * ldx + c), y1 = (T)__ldg(X + (int64_t)(c1 - col_lo) * ldx + c);
            const T y2 = (T)__ldg(X + (int64_t)(c2 - col_lo) * ldx + c), y3 = (T)__ldg(X + (int64_t)(c3 - col_lo) * ldx + c);
            acc.v[ch] += ((y0 + y1) + y2) + y3;
          }
        }
      }
      for (; k < cnt; ++k) {
        const int32_t c0 = __shfl_sync(0xffffffffu, mc, k);
#pragma unroll
        for (int ch = 0; ch < NCH; ++ch) {
          const int c = ch * 32 + lane;
          if (c < w) acc.v[ch] += (T)__ldg(X + (int64_t)(c0 - col_lo) * ldx + c);
        }
      }
    }
    return;
  }
  for (int64_t j0 = beg; j0 < end; j0 += 32) {
    int64_t j = j0 + lane;
    int32_t mc = 0;
    T ma = 0;
    if (j < end) {
      mc = col[j];
      double a = HASVAL ? val[j] : 1.0;
      if (nl) a *= op.dis[mc];
      ma = (T)a;
    }
    const int cnt = (int)((end - j0) < 32 ? (end - j0) : 32);
    int k = 0;
    if (NCH <= 2) {
      // narrow blocks: eight neighbours' loads in flight per lane, added as
      // two groups of four in order (the same sums as the loop below)
      for (; k + 8 <= cnt; k += 8) {
        int32_t cc[8];
        T aa[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          cc[q] = __shfl_sync(0xffffffffu, mc, k + q);
          aa[q] = __shfl_sync(0xffffffffu, ma, k + q);
        }
#pragma unroll
        for (int ch = 0; ch < NCH; ++ch) {
          int c = ch * 32 + lane;
          if (c < w) {
            T y[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) y[q] = (T)__ldg(X + (int64_t)(cc[q] - col_lo) * ldx + c);
            acc.v[ch] += aa[0] * y[0] + aa[1] * y[1] + aa[2] * y[2] + aa[3] * y[3];
            acc.v[ch] += aa[4] * y[4] + aa[5] * y[5] + aa[6] * y[6] + aa[7] * y[7];
          }
        }
      }
    }
    for (; k + 4 <= cnt; k += 4) {
      int32_t c0 = __shfl_sync(0xffffffffu, mc, k), c1 = __shfl_sync(0xffffffffu, mc, k + 1);
      int32_t c2 = __shfl_sync(0xffffffffu, mc, k + 2), c3 = __shfl_sync(0xffffffffu, mc, k + 3);
      T a0 = __shfl_sync(0xffffffffu, ma, k), a1 = __shfl_sync(0xffffffffu, ma, k + 1);
      T a2 = __shfl_sync(0xffffffffu, ma, k + 2), a3 = __shfl_sync(0xffffffffu, ma, k + 3);
      const Tx* x0 = X + (int64_t)(c0 - col_lo) * ldx;
      const Tx* x1 = X + (int64_t)(c1 - col_lo) * ldx;
      const Tx* x2 = X + (int64_t)(c2 - col_lo) * ldx;
      const Tx* x3 = X + (int64_t)(c3 - col_lo) * ldx;
#pragma unroll
      for (int ch = 0; ch < NCH; ++ch) {
        int c = ch * 32 + lane;
        if (c < w) {
          T y0 = (T)__ldg(x0 + c), y1 = (T)__ldg(x1 + c), y2 = (T)__ldg(x2 + c), y3 = (T)__ldg(x3 + c);
          acc.v[ch] += a0 * y0 + a1 * y1 + a2 * y2 + a3 * y3;
        }
      }
    }
    for (; k < cnt; ++k) {
      int32_t c0 = __shfl_sync(0xffffffffu, mc, k);
      T a0 = __shfl_sync(0xffffffffu, ma, k);
      const Tx* x0 = X + (int64_t)(c0 - col_lo) * ldx;
#pragma unroll
      for (int ch = 0; ch < NCH; ++ch) {
        int c = ch * 32 + lane;
        if (c < w) acc.v[ch] += a0 * (T)__ldg(x0 + c);
      }
    }
  }
}

__device__ __forceinline__ int64_t lower_bound_i32(const int32_t* a, int64_t lo, int64_t hi, int64_t x) {
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if (a[mid] < x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// diagonal coefficient of row r (Sec. 4.2); the sum term is scaled by `scale`
__device__ __forceinline__ void diag_terms(const OpParams& op, int64_t r, double& dcoef, double& scale) {
  dcoef = 0.0;
  scale = 1.0;
  if (op.op == GREST_OP_LAP) dcoef = 2.0 * (*op.dmax) - op.deg[r];
  else if (op.op == GREST_OP_NLAP) { dcoef = 1.0; scale = op.dis[r]; }
}

template <typename Tx, typename T, int NCH, bool HASVAL>
__global__ void __launch_bounds__(256) k_spmm_rows(const int64_t* __restrict__ row_off, const int32_t* __restrict__ row_len,
                                                   const int32_t* __restrict__ col, const double* __restrict__ val,
                                                   OpParams op, const Tx* __restrict__ X, int64_t ldx, T* __restrict__ Y,
                                                   int64_t ldy, int w, int64_t r0, int64_t r1, int64_t col_lo) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t r = r0 + (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < r1; r += warps) {
    const int len = row_len[r];
    if (col_lo == 0 && len > kLongRow) continue;  // hub rows: k_spmm_long
    T* yr = Y + (r - r0) * ldy;
    if (!op.live[r]) {
#pragma unroll
      for (int ch = 0; ch < NCH; ++ch) {
        int c = ch * 32 + lane;
        if (c < w) yr[c] = 0;
      }
      continue;
    }
    const int64_t beg = row_off[r], end = beg + len;
    int64_t s = beg;
    if (col_lo > 0) s = lower_bound_i32(col, beg, end, col_lo);
    Acc<T, NCH> acc;
#pragma unroll
    for (int ch = 0; ch < NCH; ++ch) acc.v[ch] = 0;
    gather_range<Tx, T, NCH, HASVAL>(col, val, s, end, op, X, ldx, w, col_lo, lane, acc);
    double dcoef, scale;
    diag_terms(op, r, dcoef, scale);
    const bool has_diag = dcoef != 0.0 && r >= col_lo;
    const Tx* xr = X + (r - col_lo) * ldx;
#pragma unroll
    for (int ch = 0; ch < NCH; ++ch) {
      int c = ch * 32 + lane;
      if (c < w) {
        T y = (T)scale * acc.v[ch];
        if (has_diag) y += (T)dcoef * (T)xr[c];
        yr[c] = y;
      }
    }
  }
}

// one block (kLongWarps warps) per long row; fixed-order reduction in shared memory
constexpr int kLongWarps = 16;

template <typename Tx, typename T, int NCH, bool HASVAL>
__global__ void __launch_bounds__(kLongWarps * 32) k_spmm_long(const int64_t* __restrict__ row_off, const int32_t* __restrict__ row_len,
                                                   const int32_t* __restrict__ col, const double* __restrict__ val,
                                                   OpParams op, const int32_t* __restrict__ rows,
                                                   const int64_t* __restrict__ n_rows, const Tx* __restrict__ X,
                                                   int64_t ldx, T* __restrict__ Y, int64_t ldy, int w, int64_t r0,
                                                   int64_t r1) {
  __shared__ T part[kLongWarps][NCH * 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t nr = *n_rows;
  for (int64_t t = blockIdx.x; t < nr; t += gridDim.x) {
    const int64_t r = rows[t];
    if (r < r0 || r >= r1) continue;
    T* yr = Y + (r - r0) * ldy;
    if (!op.live[r]) {
      for (int c = threadIdx.x; c < w; c += blockDim.x) yr[c] = 0;
      continue;
    }
    const int64_t beg = row_off[r], len = row_len[r];
    const int64_t per = ((len + kLongWarps - 1) / kLongWarps + 31) & ~(int64_t)31;
    int64_t s = beg + wid * per, e = s + per;
    if (e > beg + len) e = beg + len;
    Acc<T, NCH> acc;
#pragma unroll
    for (int ch = 0; ch < NCH; ++ch) acc.v[ch] = 0;
    if (s < e) gather_range<Tx, T, NCH, HASVAL>(col, val, s, e, op, X, ldx, w, 0, lane, acc);
#pragma unroll
    for (int ch = 0; ch < NCH; ++ch) part[wid][ch * 32 + lane] = acc.v[ch];
    __syncthreads();
    double dcoef, scale;
    diag_terms(op, r, dcoef, scale);
    const Tx* xr = X + r * ldx;
    for (int c = threadIdx.x; c < w; c += blockDim.x) {
      T sum = 0;
#pragma unroll
      for (int q = 0; q < kLongWarps; ++q) sum += part[q][c];
      T y = (T)scale * sum;
      if (dcoef != 0.0) y += (T)dcoef * (T)xr[c];
      yr[c] = y;
    }
    __syncthreads();
  }
}

template <typename Tx, typename T, int NCH>
void launch_nch(const Csr& g, const OpParams& op, const int32_t* long_rows, const int64_t* n_long_dev, const Tx* X,
                int64_t ldx, T* Y, int64_t ldy, int w, int64_t r0, int64_t r1, int64_t col_lo, cudaStream_t s) {
  const int64_t rows = r1 - r0;
  int64_t blocks = (rows + 7) / 8;
  const int64_t cap = 152 * 64;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  if (g.val) {
    k_spmm_rows<Tx, T, NCH, true><<<(unsigned)blocks, 256, 0, s>>>(g.row_off, g.row_len, g.col, g.val, op, X, ldx, Y,
                                                                   ldy, w, r0, r1, col_lo);
    if (col_lo == 0)
      k_spmm_long<Tx, T, NCH, true><<<152 * 2, kLongWarps * 32, 0, s>>>(g.row_off, g.row_len, g.col, g.val, op, long_rows,
                                                             n_long_dev, X, ldx, Y, ldy, w, r0, r1);
  } else {
    k_spmm_rows<Tx, T, NCH, false><<<(unsigned)blocks, 256, 0, s>>>(g.row_off, g.row_len, g.col, nullptr, op, X, ldx,
                                                                    Y, ldy, w, r0, r1, col_lo);
    if (col_lo == 0)
      k_spmm_long<Tx, T, NCH, false><<<152 * 2, kLongWarps * 32, 0, s>>>(g.row_off, g.row_len, g.col, nullptr, op, long_rows,
                                                              n_long_dev, X, ldx, Y, ldy, w, r0, r1);
  }
}

template <typename Tx, typename T>
void spmm_dispatch(const Csr& g, const OpParams& op, const int32_t* long_rows, const int64_t* n_long_dev, const Tx* X,
                   int64_t ldx, T* Y, int64_t ldy, int w, int64_t r0, int64_t r1, int64_t col_lo, cudaStream_t s) {
  if (r1 <= r0 || w <= 0) return;
  switch ((w + 31) / 32) {
    case 1: launch_nch<Tx, T, 1>(g, op, long_rows, n_long_dev, X, ldx, Y, ldy, w, r0, r1, col_lo, s); break;
    case 2: launch_nch<Tx, T, 2>(g, op, long_rows, n_long_dev, X, ldx, Y, ldy, w, r0, r1, col_lo, s); break;
    case 3: launch_nch<Tx, T, 3>(g, op, long_rows, n_long_dev, X, ldx, Y, ldy, w, r0, r1, col_lo, s); break;
    case 4: launch_nch<Tx, T, 4>(g, op, long_rows, n_long_dev, X, ldx, Y, ldy, w, r0, r1, col_lo, s); break;
    case 5: launch_nch<Tx, T, 5>(g, op, long_rows, n_long_dev, X, ldx, Y, ldy, w, r0, r1, col_lo, s); break;
    case 6: launch_nch<Tx, T, 6>(g, op, long_rows, n_long_dev, X, ldx, Y, ldy, w, r0, r1, col_lo, s); break;
    case 7: launch_nch<Tx, T, 7>(g, op, long_rows, n_long_dev, X, ldx, Y, ldy, w, r0, r1, col_lo, s); break;
    case 8: launch_nch<Tx, T, 8>(g, op, long_rows, n_long_dev, X, ldx, Y, ldy, w, r0, r1, col_lo, s); break;
    default: launch_nch<Tx, T, 9>(g, op, long_rows, n_long_dev, X, ldx, Y, ldy, w, r0, r1, col_lo, s); break;
  }
}

}  // namespace

void spmm_f64(const Csr& g, const OpParams& op, const int32_t* long_rows, const int64_t* n_long_dev,
              const double* X, int64_t ldx, double* Y, int64_t ldy, int w, int64_t r0, int64_t r1, int64_t col_lo,
              cudaStream_t s) {
  spmm_dispatch<double, double>(g, op, long_rows, n_long_dev, X, ldx, Y, ldy, w, r0, r1, col_lo, s);
}

void spmm_f32(const Csr& g, const OpParams& op, const int32_t* long_rows, const int64_t* n_long_dev,
              const float* X, int64_t ldx, float* Y, int64_t ldy, int w, int64_t r0, int64_t r1, int64_t col_lo,
              cudaStream_t s) {
  spmm_dispatch<float, float>(g, op, long_rows, n_long_dev, X, ldx, Y, ldy, w, r0, r1, col_lo, s);
}

void spmm_f32_f64(const Csr& g, const OpParams& op, const int32_t* long_rows, const int64_t* n_long_dev,
                  const float* X, int64_t ldx, double* Y, int64_t ldy, int w, int64_t r0, int64_t r1, int64_t col_lo,
                  cudaStream_t s) {
  spmm_dispatch<float, double>(g, op, long_rows, n_long_dev, X, ldx, Y, ldy, w, r0, r1, col_lo, s);
}

}  // namespace grest
