// FP64-accurate products of the mixed-precision refinement (A11: Rayleigh-
// Ritz in span(U), U the FP32 Ritz vectors of Alg. 2) in double-float
// arithmetic on the FP32 pipes.
//
// On GB300 an FP64 warp instruction costs ~68 clocks per SM sub-partition,
// about 64x an FP32 one, so the refinement's N x K products (M U, U^T U,
// U^T (M U), U S) would be FP64-pipe bound.  U holds FP32 values exactly, so
// every product of two FP32 numbers is recovered exactly by the FMA two-
// product (p = a b, e = fma(a, b, -p)), and sums are kept as unevaluated pairs
// hi + lo with |lo| <= ulp(hi) / 2 (two-sum, then fast two-sum), which carries
// about 48 significant bits.  FP64 coefficients (edge weights, D^-1/2, the
// small K x K matrix) are split once into hi + lo FP32 parts.  Partial sums run
// over at most a few thousand terms before they are combined in FP64, which
// keeps the accumulated error near 1e-14 relative.
//
// All double-float steps use explicitly rounded intrinsics so the compiler
// cannot contract them into FMAs (which would break the error terms).
#include "common.cuh"

namespace grest {

namespace {

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// (hi, lo) += p + q with q a small correction of p
__device__ __forceinline__ void df_add(float& hi, float& lo, float p, float q) {
  float s, e;
  two_sum(hi, p, s, e);
  e = __fadd_rn(e, __fadd_rn(lo, q));
  hi = __fadd_rn(s, e);
  lo = __fsub_rn(e, __fsub_rn(hi, s));
}

// (hi, lo) += (ah + al) x
__device__ __forceinline__ void df_madd(float& hi, float& lo, float ah, float al, float x) {
  const float p = __fmul_rn(ah, x);
  const float pe = __fmaf_rn(ah, x, -p);
  df_add(hi, lo, p, __fmaf_rn(al, x, pe));
}

__device__ __forceinline__ void split(double v, float& h, float& l) {
  h = __double2float_rn(v);
  l = __double2float_rn(v - (double)h);
}

// ---------------------------------------------------------------- M U
// Y (hi, lo) = M X for FP32 X (n x w, w <= 64), the operator of Sec. 4.2:
//   ADJ   y_r = sum_j a_rj x_j
//   LAP   y_r = (alpha - d_r) x_r + sum_j a_rj x_j
//   NLAP  y_r = x_r + s_r sum_j a_rj s_j x_j,  s = d^-1/2
// one warp per row (lane = column), hub rows (> kLongRow) in k_spmm_df_long.
template <int NCH, bool COEF>
__device__ __forceinline__ void df_gather(const int32_t* __restrict__ col, const double* __restrict__ val,
                                          int64_t beg, int64_t end, const OpParams& op, const float* __restrict__ X,
                                          int64_t ldx, int w, int lane, float (&hi)[NCH], float (&lo)[NCH]) {
  const bool nl = op.op == GREST_OP_NLAP;
  for (int64_t j0 = beg; j0 < end; j0 += 32) {
    const int64_t j = j0 + lane;
    int32_t mc = 0;
    float mh = 0.f, ml = 0.f;
    if (j < end) {
      mc = col[j];
      if (COEF) {
        double a = val ? val[j] : 1.0;
        if (nl) a *= op.dis[mc];
        split(a, mh, ml);
      }
    }
    const int cnt = (int)((end - j0) < 32 ? (end - j0) : 32);
    // eight neighbours' rows are loaded before they are added (in order), so
    // a warp keeps eight gathers in flight instead of one
    for (int k0 = 0; k0 < cnt; k0 += 8) {
      float xv[8][NCH], ahv[8], alv[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int k = k0 + q;
        const int32_t c0 = __shfl_sync(0xffffffffu, mc, k & 31);
        if (COEF) {
          ahv[q] = __shfl_sync(0xffffffffu, mh, k & 31);
          alv[q] = __shfl_sync(0xffffffffu, ml, k & 31);
        }
        const float* x0 = X + (int64_t)c0 * ldx;
#pragma unroll
        for (int ch = 0; ch < NCH; ++ch) {
          const int c = ch * 32 + lane;
          xv[q][ch] = (k < cnt && c < w) ? __ldg(x0 + c) : 0.f;
        }
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        if (k0 + q >= cnt) break;  // warp-uniform
#pragma unroll
        for (int ch = 0; ch < NCH; ++ch) {
          const int c = ch * 32 + lane;
          if (c < w) {
            if (COEF)
              df_madd(hi[ch], lo[ch], ahv[q], alv[q], xv[q][ch]);
            else
              df_add(hi[ch], lo[ch], xv[q][ch], 0.f);
          }
        }
      }
    }
  }
}

// y = scale S + dcoef x_r, S = (hi, lo), in double-float; stored as hi / lo
__device__ __forceinline__ void df_epilogue(const OpParams& op, int64_t r, float xr, float& hi, float& lo) {
  if (op.op == GREST_OP_LAP) {
    float dh, dl;
    split(2.0 * (*op.dmax) - op.deg[r], dh, dl);
    df_madd(hi, lo, dh, dl, xr);
  } else if (op.op == GREST_OP_NLAP) {
    float sh, sl;
    split(op.dis[r], sh, sl);
    // (hi + lo)(sh + sl) ~ hi sh (exact two-product) + hi sl + lo sh
    const float p = __fmul_rn(hi, sh);
    const float pe = __fmaf_rn(hi, sh, -p);
    const float q = __fmaf_rn(hi, sl, __fmaf_rn(lo, sh, pe));
    hi = 0.f;
    lo = 0.f;
    df_add(hi, lo, p, q);
    df_add(hi, lo, xr, 0.f);
  }
}

template <int NCH, bool COEF>
__global__ void __launch_bounds__(256) k_spmm_df_rows(const int64_t* __restrict__ row_off,
                                                      const int32_t* __restrict__ row_len,
                                                      const int32_t* __restrict__ col, const double* __restrict__ val,
                                                      OpParams op, const float* __restrict__ X, int64_t ldx,
                                                      float* __restrict__ Yh, float* __restrict__ Yl, int64_t ldy,
                                                      int w, int64_t n) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < n; r += warps) {
    const int len = row_len[r];
    if (len > kLongRow) continue;  // hub rows: k_spmm_df_long
    float hi[NCH], lo[NCH];
#pragma unroll
    for (int ch = 0; ch < NCH; ++ch) { hi[ch] = 0.f; lo[ch] = 0.f; }
    const bool live = op.live[r] != 0;
    if (live) {
      const int64_t beg = row_off[r];
      df_gather<NCH, COEF>(col, val, beg, beg + len, op, X, ldx, w, lane, hi, lo);
    }
#pragma unroll
    for (int ch = 0; ch < NCH; ++ch) {
      const int c = ch * 32 + lane;
      if (c < w) {
        if (live) df_epilogue(op, r, X[r * ldx + c], hi[ch], lo[ch]);
        Yh[r * ldy + c] = hi[ch];
        Yl[r * ldy + c] = lo[ch];
      }
    }
  }
}

// one block (8 warps) per hub row; partials combined in a fixed order
template <int NCH, bool COEF>
__global__ void __launch_bounds__(256) k_spmm_df_long(const int64_t* __restrict__ row_off,
                                                      const int32_t* __restrict__ row_len,
                                                      const int32_t* __restrict__ col, const double* __restrict__ val,
                                                      OpParams op, const int32_t* __restrict__ rows,
                                                      const int64_t* __restrict__ n_rows, const float* __restrict__ X,
                                                      int64_t ldx, float* __restrict__ Yh, float* __restrict__ Yl,
                                                      int64_t ldy, int w, int64_t n) {
  __shared__ float ph[8][NCH * 32], pl[8][NCH * 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t nr = *n_rows;
  for (int64_t t = blockIdx.x; t < nr; t += gridDim.x) {
    const int64_t r = rows[t];
    if (r < 0 || r >= n) continue;
    const bool live = op.live[r] != 0;
    const int64_t beg = row_off[r], len = row_len[r];
    const int64_t per = ((len + 7) / 8 + 31) & ~(int64_t)31;
    int64_t s = beg + wid * per, e = s + per;
    if (e > beg + len) e = beg + len;
    float hi[NCH], lo[NCH];
#pragma unroll
    for (int ch = 0; ch < NCH; ++ch) { hi[ch] = 0.f; lo[ch] = 0.f; }
    if (live && s < e) df_gather<NCH, COEF>(col, val, s, e, op, X, ldx, w, lane, hi, lo);
#pragma unroll
    for (int ch = 0; ch < NCH; ++ch) {
      ph[wid][ch * 32 + lane] = hi[ch];
      pl[wid][ch * 32 + lane] = lo[ch];
    }
    __syncthreads();
    for (int c = threadIdx.x; c < w; c += blockDim.x) {
      float h = 0.f, l = 0.f;
      if (live) {
#pragma unroll
        for (int q = 0; q < 8; ++q) df_add(h, l, ph[q][c], pl[q][c]);
        df_epilogue(op, r, X[r * ldx + c], h, l);
      }
      Yh[r * ldy + c] = h;
      Yl[r * ldy + c] = l;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- Grams
// part[block][i][j] = sum over the block's rows of x_i (yh_j + yl_j) (FP64),
// Yl may be null; 32-row tiles of X and Y staged in shared memory.
// Each dot product is accumulated by Dot2 (Ogita, Rump and Oishi, "Accurate
// sum and dot product", SIAM J. Sci. Comput. 26(6), 2005): the product
// x yh is split exactly into p + pe by an FMA, p enters the running sum s by
// an exact two-sum whose error goes, with pe and x yl, into a separate FP32
// correction c; s + c is as accurate as a sum carried in twice the working
// precision, at 11 FP32 operations per product.
constexpr int kDfRows = 32;

__device__ __forceinline__ void dot2_madd(float& s, float& c, float x, float yh, float yl) {
  const float p = __fmul_rn(x, yh);
  const float pe = __fmaf_rn(x, yh, -p);  // x yh = p + pe exactly
  const float t = __fadd_rn(s, p);
  const float z = __fsub_rn(t, s);
  const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z));  // s + p = t + e exactly
  s = t;
  c = __fadd_rn(c, __fadd_rn(e, __fmaf_rn(x, yl, pe)));
}

// Thread t owns C entries (i, j) with i = t / 8 + 32 u and j = 4 (t mod 8) +
// 32 v + 0..3 (u, v < k / 32 rounded up): per staged row, one x_i and a float4
// of y_h (and y_l) serve four products.
template <int NU>
__global__ void __launch_bounds__(256) k_gram_df(const float* __restrict__ X, int64_t ldx, const float* __restrict__ Yh,
                                                 const float* __restrict__ Yl, int64_t ldy, int k, int64_t n,
                                                 int64_t rows_per_block, double* __restrict__ part) {
  __shared__ __align__(16) float xs[kDfRows][64], yhs[kDfRows][64], yls[kDfRows][64];
  const int tid = threadIdx.x;
  const int ti = tid >> 3, tj = (tid & 7) * 4;
  float hi[NU][NU][4], lo[NU][NU][4];
#pragma unroll
  for (int u = 0; u < NU; ++u)
#pragma unroll
    for (int v = 0; v < NU; ++v)
#pragma unroll
      for (int q = 0; q < 4; ++q) { hi[u][v][q] = 0.f; lo[u][v][q] = 0.f; }
  const int64_t rb = blockIdx.x * rows_per_block;
  int64_t re = rb + rows_per_block;
  if (re > n) re = n;
  for (int64_t r0 = rb; r0 < re; r0 += kDfRows) {
    const int rows = (int)((re - r0) < kDfRows ? (re - r0) : kDfRows);
    __syncthreads();
    for (int e = tid; e < kDfRows * 64; e += 256) {
      const int rr = e >> 6, c = e & 63;
      const bool in = rr < rows && c < k;
      const int64_t r = r0 + rr;
      xs[rr][c] = in ? X[r * ldx + c] : 0.f;
      yhs[rr][c] = in ? Yh[r * ldy + c] : 0.f;
      yls[rr][c] = (in && Yl) ? Yl[r * ldy + c] : 0.f;
    }
    __syncthreads();
    for (int rr = 0; rr < rows; ++rr) {
#pragma unroll
      for (int u = 0; u < NU; ++u) {
        const float xv = xs[rr][ti + 32 * u];
#pragma unroll
        for (int v = 0; v < NU; ++v) {
          const float4 yh = *(const float4*)&yhs[rr][tj + 32 * v];
          const float4 yl = *(const float4*)&yls[rr][tj + 32 * v];
          dot2_madd(hi[u][v][0], lo[u][v][0], xv, yh.x, yl.x);
          dot2_madd(hi[u][v][1], lo[u][v][1], xv, yh.y, yl.y);
          dot2_madd(hi[u][v][2], lo[u][v][2], xv, yh.z, yl.z);
          dot2_madd(hi[u][v][3], lo[u][v][3], xv, yh.w, yl.w);
        }
      }
    }
  }
  double* out = part + (int64_t)blockIdx.x * k * k;
#pragma unroll
  for (int u = 0; u < NU; ++u)
#pragma unroll
    for (int v = 0; v < NU; ++v)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int i = ti + 32 * u, j = tj + 32 * v + q;
        if (i < k && j < k) out[i * k + j] = (double)hi[u][v][q] + (double)lo[u][v][q];
      }
}

// C = sum of the partials in FP64: one warp per entry, lanes over blocks,
// then a fixed shuffle tree (deterministic)
__global__ void k_gram_df_reduce(const double* __restrict__ part, int64_t nb, int k, double* C, int64_t ldc) {
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= (int64_t)k * k) return;
  double s = 0.0;
  for (int64_t b = lane; b < nb; b += 32) s += part[b * (int64_t)k * k + w];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) C[(w / k) * ldc + (w % k)] = s;
}

// ---------------------------------------------------------------- U S
// Out (n x k, FP64) = X (n x k, FP32) S (k x k, FP64): one warp per row,
// lane = output column (two columns for k > 32).
// k <= 32: column `lane` of S (split into hi + lo) in registers; each output
// is a Dot2 sum over the k products.
__global__ void __launch_bounds__(256) k_lift_df32(const float* __restrict__ X, int64_t ldx,
                                                   const double* __restrict__ S, int k, int64_t n,
                                                   double* __restrict__ Out, int64_t ldo) {
  const int lane = threadIdx.x & 31;
  float sh[32], sl[32];
#pragma unroll
  for (int q = 0; q < 32; ++q) {
    sh[q] = sl[q] = 0.f;
    if (q < k && lane < k) split(S[q * k + lane], sh[q], sl[q]);
  }
  // two rows per pass (independent Dot2 chains), rows r and r + warps
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < n; r += 2 * warps) {
    const int64_t r2 = r + warps;
    const bool two = r2 < n;
    const float xv = lane < k ? X[r * ldx + lane] : 0.f;
    const float xv2 = (two && lane < k) ? X[r2 * ldx + lane] : 0.f;
    float h = 0.f, l = 0.f, h2 = 0.f, l2 = 0.f;
#pragma unroll
    for (int q = 0; q < 32; ++q) {
      const float xq = __shfl_sync(0xffffffffu, xv, q);
      const float xq2 = __shfl_sync(0xffffffffu, xv2, q);
      if (q < k) {
        dot2_madd(h, l, xq, sh[q], sl[q]);
        dot2_madd(h2, l2, xq2, sh[q], sl[q]);
      }
    }
    if (lane < k) {
      Out[r * ldo + lane] = (double)h + (double)l;
      if (two) Out[r2 * ldo + lane] = (double)h2 + (double)l2;
    }
  }
}

// 32 < k <= 64: S split into shared memory, two output columns per lane.
__global__ void __launch_bounds__(256) k_lift_df64(const float* __restrict__ X, int64_t ldx,
                                                   const double* __restrict__ S, int k, int64_t n,
                                                   double* __restrict__ Out, int64_t ldo) {
  __shared__ float sh[64][64], sl[64][64];
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) split(S[e], sh[e / k][e % k], sl[e / k][e % k]);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < n; r += warps) {
    const float* xr = X + r * ldx;
    const float xv0 = lane < k ? xr[lane] : 0.f;
    const float xv1 = lane + 32 < k ? xr[lane + 32] : 0.f;
    float h0 = 0.f, l0 = 0.f, h1 = 0.f, l1 = 0.f;
    for (int q = 0; q < k; ++q) {
      const float xq = __shfl_sync(0xffffffffu, q < 32 ? xv0 : xv1, q & 31);
      df_madd(h0, l0, sh[q][lane], sl[q][lane], xq);
      if (lane + 32 < k) df_madd(h1, l1, sh[q][lane + 32], sl[q][lane + 32], xq);
    }
    Out[r * ldo + lane] = (double)h0 + (double)l0;
    if (lane + 32 < k) Out[r * ldo + lane + 32] = (double)h1 + (double)l1;
  }
}

// ---------------------------------------------------------------- signs
// Per column, the row of the largest |x| (lowest row on ties) and the sign of
// that entry; |x| is compared through its bit pattern (sign cleared), which
// orders non-negative doubles like their values.
__global__ void __launch_bounds__(256) k_sign_part(const double* __restrict__ X, int64_t ldx, int w, int64_t n,
                                                   int64_t rows_per_block, unsigned long long* __restrict__ pkey,
                                                   int64_t* __restrict__ prow) {
  __shared__ unsigned long long sk[8][64];
  __shared__ int64_t sr[8][64];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t rb = blockIdx.x * rows_per_block;
  int64_t re = rb + rows_per_block;
  if (re > n) re = n;
  unsigned long long bk0 = 0, bk1 = 0;
  int64_t br0 = INT64_MAX, br1 = INT64_MAX;
  for (int64_t r = rb + wid; r < re; r += 8) {
    const unsigned long long* xr = reinterpret_cast<const unsigned long long*>(X + r * ldx);
    if (lane < w) {
      const unsigned long long key = xr[lane] & 0x7fffffffffffffffull;
      if (key > bk0 || br0 == INT64_MAX) { bk0 = key; br0 = r; }
    }
    if (lane + 32 < w) {
      const unsigned long long key = xr[lane + 32] & 0x7fffffffffffffffull;
      if (key > bk1 || br1 == INT64_MAX) { bk1 = key; br1 = r; }
    }
  }
  sk[wid][lane] = bk0;
  sr[wid][lane] = br0;
  sk[wid][lane + 32] = bk1;
  sr[wid][lane + 32] = br1;
  __syncthreads();
  if (wid == 0) {
    for (int c = lane; c < w; c += 32) {
      unsigned long long bk = 0;
      int64_t br = INT64_MAX;
      for (int q = 0; q < 8; ++q) {
        const unsigned long long kq = sk[q][c];
        const int64_t rq = sr[q][c];
        if (rq == INT64_MAX) continue;
        if (br == INT64_MAX || kq > bk || (kq == bk && rq < br)) { bk = kq; br = rq; }
      }
      pkey[(int64_t)blockIdx.x * w + c] = bk;
      prow[(int64_t)blockIdx.x * w + c] = br;
    }
  }
}

// one warp per column: lanes scan the block partials, then a shuffle reduction
__global__ void k_sign_final(const double* __restrict__ X, int64_t ldx, int w, int64_t nb,
                             const unsigned long long* __restrict__ pkey, const int64_t* __restrict__ prow,
                             int* __restrict__ flip) {
  const int lane = threadIdx.x & 31;
  const int c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (c >= w) return;
  unsigned long long bk = 0;
  int64_t br = INT64_MAX;
  for (int64_t b = lane; b < nb; b += 32) {
    const unsigned long long kq = pkey[b * w + c];
    const int64_t rq = prow[b * w + c];
    if (rq == INT64_MAX) continue;
    if (br == INT64_MAX || kq > bk || (kq == bk && rq < br)) { bk = kq; br = rq; }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long ok = __shfl_down_sync(0xffffffffu, bk, o);
    const int64_t orow = __shfl_down_sync(0xffffffffu, br, o);
    if (orow != INT64_MAX && (br == INT64_MAX || ok > bk || (ok == bk && orow < br))) { bk = ok; br = orow; }
  }
  if (lane == 0) {
    int f = 0;
    if (br != INT64_MAX) {
      const long long bits = reinterpret_cast<const long long*>(X + br * ldx)[c];
      f = (bits < 0 && (bits & 0x7fffffffffffffffll) != 0) ? 1 : 0;  // strictly negative
    }
    flip[c] = f;
  }
}

__global__ void k_sign_apply(double* __restrict__ X, int64_t ldx, int w, int64_t n, const int* __restrict__ flip) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const bool f0 = lane < w && flip[lane], f1 = lane + 32 < w && flip[lane + 32];
  if (!__any_sync(0xffffffffu, f0 || f1)) return;  // same flags in every warp
  for (int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < n; r += warps) {
    unsigned long long* xr = reinterpret_cast<unsigned long long*>(X + r * ldx);
    if (f0) xr[lane] ^= 0x8000000000000000ull;
    if (f1) xr[lane + 32] ^= 0x8000000000000000ull;
  }
}

template <int NCH, bool COEF>
void launch_spmm_df(const Csr& g, const OpParams& op, const int32_t* long_rows, const int64_t* n_long_dev,
                    const float* X, int64_t ldx, float* Yh, float* Yl, int64_t ldy, int w, int64_t n, cudaStream_t s) {
  int64_t blocks = (n + 7) / 8;
  if (blocks > 152 * 64) blocks = 152 * 64;
  if (blocks < 1) blocks = 1;
  k_spmm_df_rows<NCH, COEF><<<(unsigned)blocks, 256, 0, s>>>(g.row_off, g.row_len, g.col, g.val, op, X, ldx, Yh, Yl,
                                                             ldy, w, n);
  k_spmm_df_long<NCH, COEF><<<152 * 4, 256, 0, s>>>(g.row_off, g.row_len, g.col, g.val, op, long_rows, n_long_dev, X,
                                                    ldx, Yh, Yl, ldy, w, n);
}

}  // namespace

int spmm_df(const Csr& g, const OpParams& op, const int32_t* long_rows, const int64_t* n_long_dev, const float* X,
            int64_t ldx, float* Yh, float* Yl, int64_t ldy, int w, int64_t n, cudaStream_t s) {
  if (n <= 0 || w <= 0 || w > 64) return 0;
  const bool coef = g.val != nullptr || op.op == GREST_OP_NLAP;
  if (w <= 32) {
    if (coef) launch_spmm_df<1, true>(g, op, long_rows, n_long_dev, X, ldx, Yh, Yl, ldy, w, n, s);
    else launch_spmm_df<1, false>(g, op, long_rows, n_long_dev, X, ldx, Yh, Yl, ldy, w, n, s);
  } else {
    if (coef) launch_spmm_df<2, true>(g, op, long_rows, n_long_dev, X, ldx, Yh, Yl, ldy, w, n, s);
    else launch_spmm_df<2, false>(g, op, long_rows, n_long_dev, X, ldx, Yh, Yl, ldy, w, n, s);
  }
  return 2;
}

int gram_df(const float* X, int64_t ldx, const float* Yh, const float* Yl, int64_t ldy, int k, int64_t n, double* C,
            int64_t ldc, double* part, int64_t part_cap, cudaStream_t s) {
  if (n <= 0 || k <= 0 || k > 64) return 0;
  int64_t nb = 152 * 8;
  const int64_t cap = part_cap / ((int64_t)k * k);
  if (nb > cap) nb = cap;
  int64_t rpb = (n + nb - 1) / nb;
  rpb = ((rpb + kDfRows - 1) / kDfRows) * kDfRows;
  nb = (n + rpb - 1) / rpb;
  if (k <= 32)
    k_gram_df<1><<<(unsigned)nb, 256, 0, s>>>(X, ldx, Yh, Yl, ldy, k, n, rpb, part);
  else
    k_gram_df<2><<<(unsigned)nb, 256, 0, s>>>(X, ldx, Yh, Yl, ldy, k, n, rpb, part);
  k_gram_df_reduce<<<(unsigned)(((int64_t)k * k * 32 + 255) / 256), 256, 0, s>>>(part, nb, k, C, ldc);
  return 2;
}

int lift_df(const float* X, int64_t ldx, const double* S, int k, int64_t n, double* Out, int64_t ldo, cudaStream_t s) {
  if (n <= 0 || k <= 0 || k > 64) return 0;
  int64_t blocks = (n + 7) / 8;
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (k <= 32)
    k_lift_df32<<<(unsigned)blocks, 256, 0, s>>>(X, ldx, S, k, n, Out, ldo);
  else
    k_lift_df64<<<(unsigned)blocks, 256, 0, s>>>(X, ldx, S, k, n, Out, ldo);
  return 1;
}

int sign_normalize_fast(double* X, int64_t ldx, int w, int64_t n, double* part, int64_t* ipart, cudaStream_t s) {
  if (n <= 0 || w <= 0 || w > 64) return 0;
  int64_t nb = 304;
  int64_t rpb = (n + nb - 1) / nb;
  nb = (n + rpb - 1) / rpb;
  unsigned long long* pkey = reinterpret_cast<unsigned long long*>(part);
  int* flip = reinterpret_cast<int*>(part + nb * w);
  k_sign_part<<<(unsigned)nb, 256, 0, s>>>(X, ldx, w, n, rpb, pkey, ipart);
  k_sign_final<<<(unsigned)((w + 7) / 8), 256, 0, s>>>(X, ldx, w, nb, pkey, ipart, flip);
  int64_t blocks = (n + 7) / 8;
  if (blocks > 152 * 16) blocks = 152 * 16;
  k_sign_apply<<<(unsigned)blocks, 256, 0, s>>>(X, ldx, w, n, flip);
  return 3;
}

}  // namespace grest
