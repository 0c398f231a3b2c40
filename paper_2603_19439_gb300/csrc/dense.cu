// Dense FP64 kernels of the G-REST step on tall-skinny row-major blocks:
//   gram_f64      C = X^T Y (projections C = X_bar^T Y1, Gram matrices of the
//                 CholQR2 passes, H = Z^T (M Z) of Alg. 1)
//   gemm_nn_f64   Out = beta Cin + alpha X B (P_perp updates, V T, lift Z F_K)
//   pchol_inverse pivoted Cholesky with a drop tolerance and the triangular
//                 inverse, giving T with (V T)^T (V T) = I on the kept columns
// plus small helpers (sign normalization, residual norms).
//
// The Gram is split over row chunks; each CTA writes a partial tile and a
// second kernel sums the partials in a fixed order (deterministic results).
// FP64 on GB300 runs on the CUDA-core DFMA pipe (about 1.2 TFLOP/s measured
// for the whole GPU); 4x4 register tiles keep it the bound.
#include "common.cuh"

namespace grest {

namespace {

constexpr int TM = 64, TN = 64, TK = 32;  // CTA tile (outputs) and row slab

inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// partial Gram of one (ta, tb) tile over rows [rbeg, rend); (TMv/4) x (TNv/4)
// threads, 4 x 4 outputs each
template <int TMv, int TNv>
__global__ void __launch_bounds__(256) k_gram_part(const double* __restrict__ X, int64_t ldx, int a,
                                                   const double* __restrict__ Y, int64_t ldy, int b, int64_t n,
                                                   int64_t rows_per_chunk, bool upper, double* __restrict__ part) {
  __shared__ double Xs[TK][TMv + 1];
  __shared__ double Ys[TK][TNv + 1];
  constexpr int NT = (TMv / 4) * (TNv / 4);
  // tile (ta, tb) from the block index; upper-triangular enumeration when symmetric
  const int ntb = (b + TNv - 1) / TNv;
  int bid = blockIdx.x, ta = 0, tb;
  if (!upper) {
    ta = bid / ntb;
    tb = bid % ntb;
  } else {
    while (bid >= ntb - ta) { bid -= ntb - ta; ++ta; }
    tb = ta + bid;
  }
  const int i0 = ta * TMv, j0 = tb * TNv;
  const int64_t chunk = blockIdx.y;
  const int64_t rbeg = chunk * rows_per_chunk;
  int64_t rend = rbeg + rows_per_chunk;
  if (rend > n) rend = n;
  const int tx = threadIdx.x % (TNv / 4), ty = threadIdx.x / (TNv / 4);
  double acc[4][4] = {};
  for (int64_t r0 = rbeg; r0 < rend; r0 += TK) {
    for (int e = threadIdx.x; e < TK * TMv; e += NT) {
      int rr = e / TMv, cc = e % TMv;
      int64_t r = r0 + rr;
      Xs[rr][cc] = (r < rend && i0 + cc < a) ? X[r * ldx + i0 + cc] : 0.0;
    }
    for (int e = threadIdx.x; e < TK * TNv; e += NT) {
      int rr = e / TNv, cc = e % TNv;
      int64_t r = r0 + rr;
      Ys[rr][cc] = (r < rend && j0 + cc < b) ? Y[r * ldy + j0 + cc] : 0.0;
    }
    __syncthreads();
#pragma unroll 4
    for (int k = 0; k < TK; ++k) {
      double xa[4], yb[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        xa[u] = Xs[k][ty * 4 + u];
        yb[u] = Ys[k][tx * 4 + u];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fma(xa[u], yb[v], acc[u][v]);
    }
    __syncthreads();
  }
  double* P = part + chunk * (int64_t)a * b;
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      int i = i0 + ty * 4 + u, j = j0 + tx * 4 + v;
      if (i < a && j < b) P[(int64_t)i * b + j] = acc[u][v];
    }
}

// FP32 inputs: products and 32-row slab sums in FP32, slab sums added into
// FP64 accumulators, partials written in FP64.
template <int TMv, int TNv>
__global__ void __launch_bounds__(256) k_gram_part_f32(const float* __restrict__ X, int64_t ldx, int a,
                                                       const float* __restrict__ Y, int64_t ldy, int b, int64_t n,
                                                       int64_t rows_per_chunk, bool upper, double* __restrict__ part) {
  __shared__ float Xs[TK][TMv + 4];
  __shared__ float Ys[TK][TNv + 4];
  constexpr int NT = (TMv / 4) * (TNv / 4);
  const int ntb = (b + TNv - 1) / TNv;
  int bid = blockIdx.x, ta = 0, tb;
  if (!upper) {
    ta = bid / ntb;
    tb = bid % ntb;
  } else {
    while (bid >= ntb - ta) { bid -= ntb - ta; ++ta; }
    tb = ta + bid;
  }
  const int i0 = ta * TMv, j0 = tb * TNv;
  const int64_t chunk = blockIdx.y;
  const int64_t rbeg = chunk * rows_per_chunk;
  int64_t rend = rbeg + rows_per_chunk;
  if (rend > n) rend = n;
  const int tx = threadIdx.x % (TNv / 4), ty = threadIdx.x / (TNv / 4);
  double acc[4][4] = {};
  float sl[4][4] = {};
  int slabs = 0;
  for (int64_t r0 = rbeg; r0 < rend; r0 += TK) {
    for (int e = threadIdx.x; e < TK * TMv; e += NT) {
      int rr = e / TMv, cc = e % TMv;
      int64_t r = r0 + rr;
      Xs[rr][cc] = (r < rend && i0 + cc < a) ? X[r * ldx + i0 + cc] : 0.f;
    }
    for (int e = threadIdx.x; e < TK * TNv; e += NT) {
      int rr = e / TNv, cc = e % TNv;
      int64_t r = r0 + rr;
      Ys[rr][cc] = (r < rend && j0 + cc < b) ? Y[r * ldy + j0 + cc] : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < TK; ++k) {
      float xa[4], yb[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        xa[u] = Xs[k][ty * 4 + u];
        yb[u] = Ys[k][tx * 4 + u];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) sl[u][v] = fmaf(xa[u], yb[v], sl[u][v]);
    }
    // FP32 sums of 4 slabs (128 rows), then FP64: the FP64 pipe is 1/64 of FP32 here
    if (++slabs == 4) {
      slabs = 0;
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          acc[u][v] += (double)sl[u][v];
          sl[u][v] = 0.f;
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[u][v] += (double)sl[u][v];
  double* P = part + chunk * (int64_t)a * b;
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      int i = i0 + ty * 4 + u, j = j0 + tx * 4 + v;
      if (i < a && j < b) P[(int64_t)i * b + j] = acc[u][v];
    }
}

__global__ void k_gram_reduce(const double* __restrict__ part, int64_t chunks, int a, int b, double* C, int64_t ldc,
                              bool symmetric, int tm, int tn) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)a * b) return;
  int i = (int)(e / b), j = (int)(e % b);
  int si = i, sj = j;
  if (symmetric && (i / tm) > (j / tn)) { si = j; sj = i; }  // only upper tiles were computed
  double s = 0.0;
  for (int64_t c = 0; c < chunks; ++c) s += part[c * (int64_t)a * b + (int64_t)si * b + sj];
  C[(int64_t)i * ldc + j] = s;
}

template <int TNv>
__global__ void __launch_bounds__(256) k_gemm_nn(int64_t n, int a, int c, double alpha, const double* __restrict__ X,
                                                 int64_t ldx, const double* __restrict__ B, int64_t ldb, double beta,
                                                 const double* Cin, int64_t ldc, double* Out, int64_t ldo) {
  __shared__ double Xs[TM][TK + 1];
  __shared__ double Bs[TK][TNv + 1];
  constexpr int NT = (TM / 4) * (TNv / 4);
  const int64_t r0 = blockIdx.x * (int64_t)TM;
  const int j0 = blockIdx.y * TNv;
  const int tx = threadIdx.x % (TNv / 4), ty = threadIdx.x / (TNv / 4);
  double acc[4][4] = {};
  for (int k0 = 0; k0 < a; k0 += TK) {
    for (int e = threadIdx.x; e < TM * TK; e += NT) {
      int rr = e / TK, kk = e % TK;
      int64_t r = r0 + rr;
      Xs[rr][kk] = (r < n && k0 + kk < a) ? X[r * ldx + k0 + kk] : 0.0;
    }
    for (int e = threadIdx.x; e < TK * TNv; e += NT) {
      int kk = e / TNv, cc = e % TNv;
      Bs[kk][cc] = (k0 + kk < a && j0 + cc < c) ? B[(int64_t)(k0 + kk) * ldb + j0 + cc] : 0.0;
    }
    __syncthreads();
#pragma unroll 4
    for (int k = 0; k < TK; ++k) {
      double xa[4], bb[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        xa[u] = Xs[ty * 4 + u][k];
        bb[u] = Bs[k][tx * 4 + u];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fma(xa[u], bb[v], acc[u][v]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    int64_t r = r0 + ty * 4 + u;
    if (r >= n) continue;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      int j = j0 + tx * 4 + v;
      if (j >= c) continue;
      double y = alpha * acc[u][v];
      if (beta != 0.0) y += beta * Cin[r * ldc + j];
      Out[r * ldo + j] = y;
    }
  }
}

// FP32 tall-skinny update: Out = beta Cin + alpha X B with B given in FP64
template <int TNv>
__global__ void __launch_bounds__(256) k_gemm_nn_f32(int64_t n, int a, int c, float alpha, const float* __restrict__ X,
                                                     int64_t ldx, const double* __restrict__ B, int64_t ldb, float beta,
                                                     const float* Cin, int64_t ldc, float* Out, int64_t ldo) {
  __shared__ float Xs[TM][TK + 1];
  __shared__ float Bs[TK][TNv + 4];
  constexpr int NT = (TM / 4) * (TNv / 4);
  const int64_t r0 = blockIdx.x * (int64_t)TM;
  const int j0 = blockIdx.y * TNv;
  const int tx = threadIdx.x % (TNv / 4), ty = threadIdx.x / (TNv / 4);
  float acc[4][4] = {};
  for (int k0 = 0; k0 < a; k0 += TK) {
    for (int e = threadIdx.x; e < TM * TK; e += NT) {
      int rr = e / TK, kk = e % TK;
      int64_t r = r0 + rr;
      Xs[rr][kk] = (r < n && k0 + kk < a) ? X[r * ldx + k0 + kk] : 0.f;
    }
    for (int e = threadIdx.x; e < TK * TNv; e += NT) {
      int kk = e / TNv, cc = e % TNv;
      Bs[kk][cc] = (k0 + kk < a && j0 + cc < c) ? (float)B[(int64_t)(k0 + kk) * ldb + j0 + cc] : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < TK; ++k) {
      float xa[4], bb[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        xa[u] = Xs[ty * 4 + u][k];
        bb[u] = Bs[k][tx * 4 + u];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(xa[u], bb[v], acc[u][v]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    int64_t r = r0 + ty * 4 + u;
    if (r >= n) continue;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      int j = j0 + tx * 4 + v;
      if (j >= c) continue;
      float y = alpha * acc[u][v];
      if (beta != 0.f) y += beta * Cin[r * ldc + j];
      Out[r * ldo + j] = y;
    }
  }
}

template <typename Ts, typename Td>
__global__ void k_convert(const Ts* src, int64_t lds, Td* dst, int64_t ldd, int64_t n, int w) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * w; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t r = e / w;
    int c = (int)(e % w);
    dst[r * ldd + c] = (Td)src[r * lds + c];
  }
}

// ---------------------------------------------------------------- pivoted Cholesky
// One CTA.  G (c x c) is overwritten: after step k, row k holds row k of R
// (in pivot order) and the trailing block holds the Schur complement.  A
// column is dropped when its pivot R_kk <= drop_tol * max(R_00, abs_ref)
// (R_00 is the largest column norm, abs_ref a magnitude of the operator); the
// loop stops there, so the kept rank is k.
__global__ void __launch_bounds__(1024) k_pchol(double* G, int64_t ld, int c, double drop_tol, double abs_ref,
                                                const double* abs_ref_ptr, double* T, int64_t ldt, double* info) {
  extern __shared__ int perm[];  // c entries
  __shared__ double sval[32];
  __shared__ int sidx[32];
  __shared__ double ref, rkk;
  __shared__ int piv, rank_s, stop;
  const int tid = threadIdx.x, nth = blockDim.x, lane = tid & 31, wid = tid >> 5;
  for (int i = tid; i < c; i += nth) perm[i] = i;
  if (tid == 0) { rank_s = c; stop = 0; ref = 0.0; }
  __syncthreads();
  double kept_min = 1.0, dropped_max = 0.0;
  for (int k = 0; k < c; ++k) {
    // pivot: largest remaining diagonal (lowest index on ties)
    double bv = -1.0;
    int bi = c;
    for (int i = k + tid; i < c; i += nth) {
      double d = G[(int64_t)i * ld + i];
      if (d > bv || (d == bv && i < bi)) { bv = d; bi = i; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      double ov = __shfl_down_sync(0xffffffffu, bv, o);
      int oi = __shfl_down_sync(0xffffffffu, bi, o);
      if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
    }
    if (lane == 0) { sval[wid] = bv; sidx[wid] = bi; }
    __syncthreads();
    if (tid == 0) {
      double v = sval[0];
      int idx = sidx[0];
      for (int w = 1; w < (nth + 31) / 32; ++w)
        if (sval[w] > v || (sval[w] == v && sidx[w] < idx)) { v = sval[w]; idx = sidx[w]; }
      if (k == 0) {
        // drop reference: max(R_00, |theta_1|)^2 where |theta_1| ~ ||M||_2 (abs_ref_ptr)
        double a = abs_ref_ptr ? fabs(*abs_ref_ptr) : abs_ref;
        ref = fmax(v, a * a);
      }
      if (!(v > 0.0) || !(v > drop_tol * drop_tol * ref) || !isfinite(v)) {
        stop = 1;
        rank_s = k;
      }
      piv = idx;
      rkk = sqrt(v > 0.0 ? v : 0.0);
    }
    __syncthreads();
    if (stop) {
      double v = piv < c ? G[(int64_t)piv * ld + piv] : 0.0;
      dropped_max = (ref > 0.0 && v > 0.0) ? sqrt(v / ref) : 0.0;
      break;
    }
    const int p = piv;
    // symmetric swap of rows/columns k and p
    if (p != k) {
      for (int j = tid; j < c; j += nth) {
        double t = G[(int64_t)k * ld + j];
        G[(int64_t)k * ld + j] = G[(int64_t)p * ld + j];
        G[(int64_t)p * ld + j] = t;
      }
      __syncthreads();
      for (int i = tid; i < c; i += nth) {
        double t = G[(int64_t)i * ld + k];
        G[(int64_t)i * ld + k] = G[(int64_t)i * ld + p];
        G[(int64_t)i * ld + p] = t;
      }
      if (tid == 0) { int t = perm[k]; perm[k] = perm[p]; perm[p] = t; }
      __syncthreads();
    }
    const double r = rkk;
    kept_min = ref > 0.0 ? r / sqrt(ref) : 0.0;
    // row k of R
    for (int j = k + 1 + tid; j < c; j += nth) G[(int64_t)k * ld + j] /= r;
    __syncthreads();
    if (tid == 0) G[(int64_t)k * ld + k] = r;
    // trailing update of the upper triangle (and mirror for the diagonal scan)
    const int m = c - k - 1;
    for (int64_t e = tid; e < (int64_t)m * m; e += nth) {
      int i = k + 1 + (int)(e / m), j = k + 1 + (int)(e % m);
      if (j < i) continue;
      double v = G[(int64_t)i * ld + j] - G[(int64_t)k * ld + i] * G[(int64_t)k * ld + j];
      G[(int64_t)i * ld + j] = v;
      G[(int64_t)j * ld + i] = v;
    }
    __syncthreads();
  }
  __syncthreads();
  const int rk = rank_s;
  // T = P R^-1 (c x c, zero columns >= rk): thread j solves R x = e_j
  for (int64_t e = tid; e < (int64_t)c * c; e += nth) T[(e / c) * ldt + (e % c)] = 0.0;
  __syncthreads();
  for (int j = tid; j < rk; j += nth) {
    // x_j = 1/R_jj, x_i = -(sum_{l=i+1..j} R_il x_l) / R_ii
    T[(int64_t)perm[j] * ldt + j] = 1.0 / G[(int64_t)j * ld + j];
    for (int i = j - 1; i >= 0; --i) {
      double s = 0.0;
      for (int l = i + 1; l <= j; ++l) s = fma(G[(int64_t)i * ld + l], T[(int64_t)perm[l] * ldt + j], s);
      T[(int64_t)perm[i] * ldt + j] = -s / G[(int64_t)i * ld + i];
    }
  }
  if (tid == 0) {
    info[0] = rk;
    info[1] = rk > 0 ? kept_min : 0.0;
    info[2] = dropped_max;
    info[3] = 0.0;
  }
}

// Shared-memory variant: the upper triangle of G is packed row by row in
// shared memory (element (i, j >= i) at off(i) + j - i, off(i) = i c - i(i-1)/2),
// which holds c <= 237 in FP64.  Same pivoting and drop rule as k_pchol.
__device__ __forceinline__ int poff(int i, int c) { return i * c - (i * (i - 1)) / 2; }
__device__ __forceinline__ double& pat(double* A, int i, int j, int c) { return A[poff(i, c) + (j - i)]; }

__global__ void __launch_bounds__(1024) k_pchol_smem(const double* G, int64_t ld, int c, double drop_tol,
                                                     double abs_ref, const double* abs_ref_ptr, double* T,
                                                     int64_t ldt, double* info) {
  extern __shared__ double A[];  // packed upper triangle, then perm (ints)
  int* perm = reinterpret_cast<int*>(A + (c * (c + 1)) / 2);
  __shared__ double sval[32];
  __shared__ int sidx[32];
  __shared__ double ref, rkk;
  __shared__ int piv, rank_s, stop;
  const int tid = threadIdx.x, nth = blockDim.x, lane = tid & 31, wid = tid >> 5;
  for (int i = tid; i < c; i += nth) {
    perm[i] = i;
    for (int j = i; j < c; ++j) pat(A, i, j, c) = G[(int64_t)i * ld + j];
  }
  if (tid == 0) { rank_s = c; stop = 0; ref = 0.0; }
  __syncthreads();
  double kept_min = 1.0, dropped_max = 0.0;
  for (int k = 0; k < c; ++k) {
    double bv = -1.0;
    int bi = c;
    for (int i = k + tid; i < c; i += nth) {
      double d = A[poff(i, c)];
      if (d > bv || (d == bv && i < bi)) { bv = d; bi = i; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      double ov = __shfl_down_sync(0xffffffffu, bv, o);
      int oi = __shfl_down_sync(0xffffffffu, bi, o);
      if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
    }
    if (lane == 0) { sval[wid] = bv; sidx[wid] = bi; }
    __syncthreads();
    if (tid == 0) {
      double v = sval[0];
      int idx = sidx[0];
      for (int w = 1; w < (nth + 31) / 32; ++w)
        if (sval[w] > v || (sval[w] == v && sidx[w] < idx)) { v = sval[w]; idx = sidx[w]; }
      if (k == 0) {
        double a = abs_ref_ptr ? fabs(*abs_ref_ptr) : abs_ref;
        ref = fmax(v, a * a);
      }
      if (!(v > 0.0) || !(v > drop_tol * drop_tol * ref) || !isfinite(v)) {
        stop = 1;
        rank_s = k;
      }
      piv = idx;
      rkk = sqrt(v > 0.0 ? v : 0.0);
    }
    __syncthreads();
    if (stop) {
      double v = piv < c ? A[poff(piv, c)] : 0.0;
      dropped_max = (ref > 0.0 && v > 0.0) ? sqrt(v / ref) : 0.0;
      break;
    }
    const int p = piv;
    if (p != k) {
      // symmetric swap of indices k and p in the packed upper triangle
      for (int j = tid; j < c; j += nth) {
        if (j < k) {
          double t = pat(A, j, k, c); pat(A, j, k, c) = pat(A, j, p, c); pat(A, j, p, c) = t;
        } else if (j > k && j < p) {
          double t = pat(A, k, j, c); pat(A, k, j, c) = pat(A, j, p, c); pat(A, j, p, c) = t;
        } else if (j > p) {
          double t = pat(A, k, j, c); pat(A, k, j, c) = pat(A, p, j, c); pat(A, p, j, c) = t;
        } else if (j == k) {
          double t = pat(A, k, k, c); pat(A, k, k, c) = pat(A, p, p, c); pat(A, p, p, c) = t;
          int q = perm[k]; perm[k] = perm[p]; perm[p] = q;
        }
      }
      __syncthreads();
    }
    const double r = rkk;
    kept_min = ref > 0.0 ? r / sqrt(ref) : 0.0;
    for (int j = k + 1 + tid; j < c; j += nth) pat(A, k, j, c) /= r;
    if (tid == 0) pat(A, k, k, c) = r;
    __syncthreads();
    // trailing update of the upper triangle: A[i][j] -= R[k][i] R[k][j], k < i <= j
    const int m = c - k - 1;
    const double* Rk = A + poff(k, c) - k;  // Rk[j] = R[k][j]
    for (int i = k + 1 + wid; i < c; i += nth / 32) {
      const double rki = Rk[i];
      double* Ai = A + poff(i, c) - i;
      for (int j = i + lane; j < c; j += 32) Ai[j] = fma(-rki, Rk[j], Ai[j]);
    }
    (void)m;
    __syncthreads();
  }
  __syncthreads();
  const int rk = rank_s;
  for (int64_t e = tid; e < (int64_t)c * c; e += nth) T[(e / c) * ldt + (e % c)] = 0.0;
  __syncthreads();
  // T = P R^-1: thread j solves R x = e_j (x_j = 1/R_jj, x_i = -(sum_{l=i+1..j} R_il x_l)/R_ii)
  for (int j = tid; j < rk; j += nth) {
    T[(int64_t)perm[j] * ldt + j] = 1.0 / pat(A, j, j, c);
    for (int i = j - 1; i >= 0; --i) {
      double s2 = 0.0;
      const double* Ri = A + poff(i, c) - i;
      for (int l = i + 1; l <= j; ++l) s2 = fma(Ri[l], T[(int64_t)perm[l] * ldt + j], s2);
      T[(int64_t)perm[i] * ldt + j] = -s2 / Ri[i];
    }
  }
  if (tid == 0) {
    info[0] = rk;
    info[1] = rk > 0 ? kept_min : 0.0;
    info[2] = dropped_max;
    info[3] = 0.0;
  }
}

__global__ void k_symmetrize(double* H, int64_t ld, int m) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)m * m) return;
  int i = (int)(e / m), j = (int)(e % m);
  if (j <= i) return;
  double v = 0.5 * (H[(int64_t)i * ld + j] + H[(int64_t)j * ld + i]);
  H[(int64_t)i * ld + j] = v;
  H[(int64_t)j * ld + i] = v;
}

__global__ void k_fill(double* p, double v, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) p[i] = v;
}

__global__ void k_copy_cols(const double* src, int64_t lds, double* dst, int64_t ldd, int64_t n, int w) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * w; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t r = e / w;
    int c = (int)(e % w);
    dst[r * ldd + c] = src[r * lds + c];
  }
}

template <typename T>
__global__ void k_zero_dead(T* X, int64_t ldx, int w, const uint8_t* live, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * w; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t r = e / w;
    if (!live[r]) {
      T& x = X[r * ldx + (e % w)];
      if (x != (T)0) x = (T)0;  // zeros of either sign stay as they are (restored states keep their bytes)
    }
  }
}

// per column: the entry of largest magnitude, lowest index on ties
template <typename T>
__global__ void k_argmax_part(const T* X, int64_t ldx, int w, int64_t n, int64_t rows_per_block, double* part,
                              int64_t* ipart) {
  __shared__ double sv[256];
  __shared__ int64_t si[256];
  const int64_t rb = blockIdx.x * rows_per_block;
  int64_t re = rb + rows_per_block;
  if (re > n) re = n;
  for (int c = 0; c < w; ++c) {
    double bv = -1.0;
    int64_t bi = INT64_MAX;
    for (int64_t r = rb + threadIdx.x; r < re; r += blockDim.x) {
      double v = fabs((double)X[r * ldx + c]);
      if (v > bv) { bv = v; bi = r; }
    }
    sv[threadIdx.x] = bv;
    si[threadIdx.x] = bi;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
      if (threadIdx.x < o) {
        double ov = sv[threadIdx.x + o];
        int64_t oi = si[threadIdx.x + o];
        if (ov > sv[threadIdx.x] || (ov == sv[threadIdx.x] && oi < si[threadIdx.x])) {
          sv[threadIdx.x] = ov;
          si[threadIdx.x] = oi;
        }
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      part[(int64_t)blockIdx.x * w + c] = sv[0];
      ipart[(int64_t)blockIdx.x * w + c] = si[0];
    }
    __syncthreads();
  }
}

template <typename T>
__global__ void k_argmax_final(const T* X, int64_t ldx, int w, int64_t nb, const double* part,
                               const int64_t* ipart, double* sign) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= w) return;
  double bv = -1.0;
  int64_t bi = INT64_MAX;
  for (int64_t b = 0; b < nb; ++b) {
    double v = part[b * w + c];
    int64_t i = ipart[b * w + c];
    if (v > bv || (v == bv && i < bi)) { bv = v; bi = i; }
  }
  sign[c] = (bi != INT64_MAX && (double)X[bi * ldx + c] < 0.0) ? -1.0 : 1.0;
}

template <typename T>
__global__ void k_scale_cols(T* X, int64_t ldx, int w, int64_t n, const double* sign) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * w; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t r = e / w;
    int c = (int)(e % w);
    X[r * ldx + c] *= (T)sign[c];
  }
}

__global__ void k_resid_part(const double* MX, const double* X, int64_t ld, int w, const double* theta, int64_t n,
                             int64_t rows_per_block, double* part) {
  __shared__ double red[256];
  const int64_t rb = blockIdx.x * rows_per_block;
  int64_t re = rb + rows_per_block;
  if (re > n) re = n;
  for (int c = 0; c < w; ++c) {
    double s = 0.0;
    const double th = theta[c];
    for (int64_t r = rb + threadIdx.x; r < re; r += blockDim.x) {
      double d = MX[r * ld + c] - th * X[r * ld + c];
      s = fma(d, d, s);
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
      if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) part[(int64_t)blockIdx.x * w + c] = red[0];
    __syncthreads();
  }
}

__global__ void k_resid_final(const double* part, int64_t nb, int w, double* out) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= w) return;
  double s = 0.0;
  for (int64_t b = 0; b < nb; ++b) s += part[b * w + c];
  out[c] = sqrt(s);
}

int64_t gram_chunks(int64_t n, int ntiles) {
  int64_t target = (152 * 4 + ntiles - 1) / ntiles;
  int64_t maxc = cdiv(n, 256);
  if (target > maxc) target = maxc;
  if (target < 1) target = 1;
  return target;
}

}  // namespace

// tile shape: 32-wide tiles for widths <= 32 (K-wide products), else 64
inline int tile_of(int w) { return w <= 32 ? 32 : 64; }

int64_t gram_parts(int64_t n, int a, int b) {
  int nt = (int)(cdiv(a, tile_of(a)) * cdiv(b, tile_of(b)));
  return gram_chunks(n, nt);
}

template <typename T>
void launch_gram_part(dim3 grid, int tm, int tn, const T* X, int64_t ldx, int a, const T* Y, int64_t ldy, int b,
                      int64_t n, int64_t rpc, bool upper, double* part, cudaStream_t s) {
  const int nthr = (tm / 4) * (tn / 4);
  if constexpr (sizeof(T) == sizeof(double)) {
    if (tm == 32 && tn == 32) k_gram_part<32, 32><<<grid, nthr, 0, s>>>(X, ldx, a, Y, ldy, b, n, rpc, upper, part);
    else if (tm == 32) k_gram_part<32, 64><<<grid, nthr, 0, s>>>(X, ldx, a, Y, ldy, b, n, rpc, upper, part);
    else if (tn == 32) k_gram_part<64, 32><<<grid, nthr, 0, s>>>(X, ldx, a, Y, ldy, b, n, rpc, upper, part);
    else k_gram_part<64, 64><<<grid, nthr, 0, s>>>(X, ldx, a, Y, ldy, b, n, rpc, upper, part);
  } else {
    if (tm == 32 && tn == 32) k_gram_part_f32<32, 32><<<grid, nthr, 0, s>>>(X, ldx, a, Y, ldy, b, n, rpc, upper, part);
    else if (tm == 32) k_gram_part_f32<32, 64><<<grid, nthr, 0, s>>>(X, ldx, a, Y, ldy, b, n, rpc, upper, part);
    else if (tn == 32) k_gram_part_f32<64, 32><<<grid, nthr, 0, s>>>(X, ldx, a, Y, ldy, b, n, rpc, upper, part);
    else k_gram_part_f32<64, 64><<<grid, nthr, 0, s>>>(X, ldx, a, Y, ldy, b, n, rpc, upper, part);
  }
}

// CTAs of one launch of the variant that fit on the device at once
template <typename T>
int gram_wave(int tm, int tn) {
  const int nthr = (tm / 4) * (tn / 4);
  int occ = 0, dev = 0, nsm = 152;
  cudaError_t e;
  if constexpr (sizeof(T) == sizeof(double)) {
    if (tm == 32 && tn == 32) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_gram_part<32, 32>, nthr, 0);
    else if (tm == 32) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_gram_part<32, 64>, nthr, 0);
    else if (tn == 32) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_gram_part<64, 32>, nthr, 0);
    else e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_gram_part<64, 64>, nthr, 0);
  } else {
    if (tm == 32 && tn == 32) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_gram_part_f32<32, 32>, nthr, 0);
    else if (tm == 32) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_gram_part_f32<32, 64>, nthr, 0);
    else if (tn == 32) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_gram_part_f32<64, 32>, nthr, 0);
    else e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_gram_part_f32<64, 64>, nthr, 0);
  }
  if (e != cudaSuccess || occ < 1) {
    cudaGetLastError();
    occ = 4;
  }
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  return nsm * occ;
}

// partial-sum buffer of the callers that pass no capacity (a context's part buffer)
constexpr int64_t kDefaultPartCap = 8'000'000;

template <typename T>
void gram_t(const T* X, int64_t ldx, int a, const T* Y, int64_t ldy, int b, int64_t n, double* C, int64_t ldc,
            double* part, bool symmetric, int64_t part_cap, cudaStream_t s) {
  if (a <= 0 || b <= 0) return;
  if (n <= 0) {
    for (int i = 0; i < a; ++i) cudaMemsetAsync(C + (int64_t)i * ldc, 0, sizeof(double) * b, s);
    return;
  }
  symmetric = symmetric && (X == Y) && (a == b) && (ldx == ldy);
  int tm = tile_of(a), tn = tile_of(b);
  if (symmetric) tm = tn = tile_of(a);
  const int nta = (int)cdiv(a, tm), ntb = (int)cdiv(b, tn);
  const int nt = symmetric ? nta * (nta + 1) / 2 : nta * ntb;
  // one full wave of CTAs: row chunks x computed tiles ~ the CTAs that fit at once
  int64_t chunks = gram_wave<T>(tm, tn) / nt;
  if (chunks > cdiv(n, 256)) chunks = cdiv(n, 256);
  const int64_t cap = (part_cap > 0 ? part_cap : kDefaultPartCap) / ((int64_t)a * b);
  if (chunks > cap) chunks = cap;
  if (chunks < 1) chunks = 1;
  int64_t rpc = cdiv(n, chunks);
  chunks = cdiv(n, rpc);
  dim3 grid((unsigned)nt, (unsigned)chunks);
  launch_gram_part<T>(grid, tm, tn, X, ldx, a, Y, ldy, b, n, rpc, symmetric, part, s);
  int64_t tot = (int64_t)a * b;
  k_gram_reduce<<<(unsigned)cdiv(tot, 256), 256, 0, s>>>(part, chunks, a, b, C, ldc, symmetric, tm, tn);
}

__global__ void k_gram_reduce_t(const double* __restrict__ partT, int64_t chunks, int a, int b, double* C,
                                int64_t ldc) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)a * b) return;
  int j = (int)(e / a), i = (int)(e % a);  // consecutive threads read consecutive rows of a partial
  double s = 0.0;
  for (int64_t c = 0; c < chunks; ++c) s += partT[(c * b + j) * (int64_t)a + i];
  C[(int64_t)i * ldc + j] = s;
}

void gram_reduce_launch(const double* part, int64_t chunks, int a, int b, double* C, int64_t ldc, cudaStream_t s,
                        bool transposed) {
  int64_t tot = (int64_t)a * b;
  if (transposed)
    k_gram_reduce_t<<<(unsigned)cdiv(tot, 256), 256, 0, s>>>(part, chunks, a, b, C, ldc);
  else
    k_gram_reduce<<<(unsigned)cdiv(tot, 256), 256, 0, s>>>(part, chunks, a, b, C, ldc, false, 64, 64);
}

namespace {

// Upper triangles of G = X^T X and H = X^T Y (k <= 64 columns) over one row
// chunk.  The work is split into 4 x 4 blocks (bi <= bj) of G and of H, one
// per thread, so every warp except the last does only needed products: on
// this part an FP64 warp instruction costs its sub-partition the same
// whatever its active lanes.
constexpr int kPairRows = 32;

__global__ void __launch_bounds__(512) k_gram_pair_upper(const double* __restrict__ X, const double* __restrict__ Y,
                                                         int64_t ld, int k, int64_t n, int64_t rows_per_chunk, int R,
                                                         double* __restrict__ part) {
  __shared__ double XYs[2][kPairRows][64 + 1];
  double (*Xs)[64 + 1] = XYs[0];
  double (*Ys)[64 + 1] = XYs[1];
  const int nb = (k + 3) / 4, npairs = nb * (nb + 1) / 2, ntask = 2 * npairs;
  // R row groups of ntask threads each (R chosen so that whole warps are
  // busy); row group g takes the rows g, g + R, ... of every slab
  const int t = threadIdx.x % ntask, rg = threadIdx.x / ntask;
  const bool active = rg < R;
  const int which = t < npairs ? 0 : 1;  // 0: X^T X, 1: X^T Y
  int pi = t - which * npairs, bi = 0;
  while (pi >= nb - bi) { pi -= nb - bi; ++bi; }
  const int bj = bi + pi;
  const int64_t chunk = blockIdx.x;
  const int64_t rbeg = chunk * rows_per_chunk;
  const int64_t rend = rbeg + rows_per_chunk < n ? rbeg + rows_per_chunk : n;
  double acc[4][4] = {};
  for (int64_t r0 = rbeg; r0 < rend; r0 += kPairRows) {
    for (int e = threadIdx.x; e < kPairRows * k; e += blockDim.x) {
      const int rr = e / k, cc = e % k;
      const int64_t r = r0 + rr;
      Xs[rr][cc] = r < rend ? X[r * ld + cc] : 0.0;
      Ys[rr][cc] = r < rend ? Y[r * ld + cc] : 0.0;
    }
    for (int e = threadIdx.x; e < kPairRows * (nb * 4 - k); e += blockDim.x) {  // zero the padding columns
      const int rr = e / (nb * 4 - k), cc = k + e % (nb * 4 - k);
      Xs[rr][cc] = 0.0;
      Ys[rr][cc] = 0.0;
    }
    __syncthreads();
    if (active) {
      double (*B)[64 + 1] = which ? Ys : Xs;
      for (int kk = rg; kk < kPairRows; kk += R) {
        double xa[4], yb[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          xa[u] = Xs[kk][bi * 4 + u];
          yb[u] = B[kk][bj * 4 + u];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) acc[u][v] = fma(xa[u], yb[v], acc[u][v]);
      }
    }
    __syncthreads();
  }
  // groups 1..R-1 stage their sums in the (now free) slab buffer and group 0
  // adds them in group order, so the result does not depend on timing
  double* stage = &XYs[0][0][0];
  if (active && rg > 0) {
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) stage[((rg - 1) * ntask + t) * 16 + u * 4 + v] = acc[u][v];
  }
  __syncthreads();
  if (rg != 0) return;
  for (int g = 1; g < R; ++g)
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) acc[u][v] += stage[((g - 1) * ntask + t) * 16 + u * 4 + v];
  double* P = part + (chunk * 2 + which) * (int64_t)k * k;
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int i = bi * 4 + u, j = bj * 4 + v;
      if (i < k && j < k) P[(int64_t)i * k + j] = acc[u][v];
    }
}

// G and H in full: entry (i, j) is read from the computed block of the upper
// triangle, (j, i) when block (i/4, j/4) lies below the diagonal
__global__ void k_gram_pair_reduce(const double* __restrict__ part, int64_t chunks, int k, double* G, double* H) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 2 * k * k) return;
  const int which = e / (k * k), ij = e % (k * k), i = ij / k, j = ij % k;
  const int src = (i / 4 <= j / 4) ? ij : j * k + i;
  double sum = 0.0;
  for (int64_t c = 0; c < chunks; ++c) sum += part[(c * 2 + which) * (int64_t)k * k + src];
  (which ? H : G)[ij] = sum;
}

}  // namespace

int gram_pair_sym_f64(const double* X, const double* Y, int64_t ld, int k, int64_t n, double* G, double* H,
                      double* part, int64_t part_cap, cudaStream_t s) {
  if (k < 1 || k > 64 || n < 1) return -1;
  const int nb = (k + 3) / 4, ntask = nb * (nb + 1);
  // row groups: the R (<= 8, R ntask <= 512, R - 1 staged groups fit in the
  // slab buffer) that leaves the fewest idle lanes in the last warp
  int R = 1;
  double best = 2.0;
  for (int r = 1; r <= 8 && r * ntask <= 512 && (r - 1) * ntask * 16 <= 2 * kPairRows * 65; ++r) {
    const int th = (r * ntask + 31) / 32 * 32;
    const double idle = (double)(th - r * ntask) / th;
    if (idle < best - 1e-12) { best = idle; R = r; }
  }
  const int threads = (R * ntask + 31) / 32 * 32;
  int64_t chunks = 152 * 4;
  const int64_t slabs = cdiv(n, kPairRows);
  if (chunks > slabs) chunks = slabs;
  if (chunks > part_cap / (2 * (int64_t)k * k)) chunks = part_cap / (2 * (int64_t)k * k);
  if (chunks < 1) return -1;
  const int64_t rpc = cdiv(cdiv(n, chunks), kPairRows) * kPairRows;
  chunks = cdiv(n, rpc);
  k_gram_pair_upper<<<(unsigned)chunks, threads, 0, s>>>(X, Y, ld, k, n, rpc, R, part);
  k_gram_pair_reduce<<<(unsigned)cdiv(2 * (int64_t)k * k, 256), 256, 0, s>>>(part, chunks, k, G, H);
  return 2;
}

void gram_f64(const double* X, int64_t ldx, int a, const double* Y, int64_t ldy, int b, int64_t n, double* C,
              int64_t ldc, double* part, bool symmetric, cudaStream_t s) {
  gram_t<double>(X, ldx, a, Y, ldy, b, n, C, ldc, part, symmetric, 0, s);
}

int gram_f64_capped(const double* X, int64_t ldx, int a, const double* Y, int64_t ldy, int b, int64_t n, double* C,
                    int64_t ldc, double* part, int64_t part_cap, cudaStream_t s) {
  if (a <= 0 || b <= 0 || n <= 0) return -1;
  if ((int64_t)a * b > part_cap) return -1;
  gram_t<double>(X, ldx, a, Y, ldy, b, n, C, ldc, part, false, part_cap, s);
  return 0;
}

void gemm_nn_f64(int64_t n, int a, int c, double alpha, const double* X, int64_t ldx, const double* B, int64_t ldb,
                 double beta, const double* Cin, int64_t ldc, double* Out, int64_t ldo, cudaStream_t s) {
  if (n <= 0 || c <= 0) return;
  if (c <= 32) {
    dim3 grid((unsigned)cdiv(n, TM), (unsigned)cdiv(c, 32));
    k_gemm_nn<32><<<grid, (TM / 4) * 8, 0, s>>>(n, a, c, alpha, X, ldx, B, ldb, beta, Cin, ldc, Out, ldo);
  } else {
    dim3 grid((unsigned)cdiv(n, TM), (unsigned)cdiv(c, TN));
    k_gemm_nn<64><<<grid, 256, 0, s>>>(n, a, c, alpha, X, ldx, B, ldb, beta, Cin, ldc, Out, ldo);
  }
}

bool pchol_cluster(double* G, int64_t ldg, int c, double drop_tol, double abs_ref, const double* abs_ref_ptr,
                   double* T, int64_t ldt, int* piv, double* info, bool f32, cudaStream_t s);

bool pchol_f32_1cta(const double* G, int64_t ldg, int c, double drop_tol, double abs_ref, const double* abs_ref_ptr,
                    double* Tm, int64_t ldt, int* piv, double* info, cudaStream_t s);

int pchol_inverse(double* G, int64_t ldg, int c, double drop_tol, double abs_ref, const double* abs_ref_ptr,
                  double* T, int64_t ldt, int* piv, double* info, bool f32, cudaStream_t s) {
  // one SM for small problems (barrier latency dominates), a cluster for large
  // ones (the Schur updates are bound by shared-memory bandwidth on one SM)
  if (f32 && c <= 64 && pchol_f32_1cta(G, ldg, c, drop_tol, abs_ref, abs_ref_ptr, T, ldt, piv, info, s)) return 1;
  if (pchol_cluster(G, ldg, c, drop_tol, abs_ref, abs_ref_ptr, T, ldt, piv, info, f32, s)) return 2;
  const size_t smem = sizeof(double) * ((size_t)c * (c + 1) / 2) + sizeof(int) * (c + 1) + 16;
  if (reserve_dynamic_smem(k_pchol_smem, smem)) {
    k_pchol_smem<<<1, 1024, smem, s>>>(G, ldg, c, drop_tol, abs_ref, abs_ref_ptr, T, ldt, info);
  } else {
    k_pchol<<<1, 1024, sizeof(int) * (c + 1), s>>>(G, ldg, c, drop_tol, abs_ref, abs_ref_ptr, T, ldt, info);
  }
  return 1;
}

void symmetrize(double* H, int64_t ld, int m, cudaStream_t s) {
  int64_t t = (int64_t)m * m;
  k_symmetrize<<<(unsigned)cdiv(t, 256), 256, 0, s>>>(H, ld, m);
}

void fill_f64(double* p, double v, int64_t n, cudaStream_t s) {
  if (n > 0) k_fill<<<(unsigned)(cdiv(n, 256) < 4096 ? cdiv(n, 256) : 4096), 256, 0, s>>>(p, v, n);
}

void copy_cols_f64(const double* src, int64_t lds, double* dst, int64_t ldd, int64_t n, int w, cudaStream_t s) {
  int64_t t = n * w;
  if (t > 0) k_copy_cols<<<(unsigned)(cdiv(t, 256) < 8192 ? cdiv(t, 256) : 8192), 256, 0, s>>>(src, lds, dst, ldd, n, w);
}

template <typename T>
void zero_dead_rows_t(T* X, int64_t ldx, int w, const uint8_t* live, int64_t n, cudaStream_t s) {
  int64_t t = n * w;
  if (t > 0) k_zero_dead<T><<<(unsigned)(cdiv(t, 256) < 8192 ? cdiv(t, 256) : 8192), 256, 0, s>>>(X, ldx, w, live, n);
}
void zero_dead_rows(double* X, int64_t ldx, int w, const uint8_t* live, int64_t n, cudaStream_t s) {
  zero_dead_rows_t(X, ldx, w, live, n, s);
}
void zero_dead_rows(float* X, int64_t ldx, int w, const uint8_t* live, int64_t n, cudaStream_t s) {
  zero_dead_rows_t(X, ldx, w, live, n, s);
}

template <typename T>
void sign_normalize_t(T* X, int64_t ldx, int w, int64_t n, double* part, int64_t* ipart, cudaStream_t s) {
  if (n <= 0 || w <= 0) return;
  int64_t nb = 304;
  int64_t rpb = cdiv(n, nb);
  nb = cdiv(n, rpb);
  k_argmax_part<T><<<(unsigned)nb, 256, 0, s>>>(X, ldx, w, n, rpb, part, ipart);
  double* sign = part + nb * w;
  k_argmax_final<T><<<(unsigned)cdiv(w, 64), 64, 0, s>>>(X, ldx, w, nb, part, ipart, sign);
  int64_t t = n * w;
  k_scale_cols<T><<<(unsigned)(cdiv(t, 256) < 8192 ? cdiv(t, 256) : 8192), 256, 0, s>>>(X, ldx, w, n, sign);
}
void sign_normalize(double* X, int64_t ldx, int w, int64_t n, double* part, int64_t* ipart, cudaStream_t s) {
  sign_normalize_t(X, ldx, w, n, part, ipart, s);
}
void sign_normalize(float* X, int64_t ldx, int w, int64_t n, double* part, int64_t* ipart, cudaStream_t s) {
  sign_normalize_t(X, ldx, w, n, part, ipart, s);
}

void gram_f32(const float* X, int64_t ldx, int a, const float* Y, int64_t ldy, int b, int64_t n, double* C,
              int64_t ldc, double* part, bool symmetric, cudaStream_t s) {
  gram_t<float>(X, ldx, a, Y, ldy, b, n, C, ldc, part, symmetric, 0, s);
}

void gemm_nn_f32(int64_t n, int a, int c, double alpha, const float* X, int64_t ldx, const double* B, int64_t ldb,
                 double beta, const float* Cin, int64_t ldc, float* Out, int64_t ldo, cudaStream_t s) {
  if (n <= 0 || c <= 0) return;
  if (c <= 32) {
    dim3 grid((unsigned)cdiv(n, TM), (unsigned)cdiv(c, 32));
    k_gemm_nn_f32<32><<<grid, (TM / 4) * 8, 0, s>>>(n, a, c, (float)alpha, X, ldx, B, ldb, (float)beta, Cin, ldc, Out, ldo);
  } else {
    dim3 grid((unsigned)cdiv(n, TM), (unsigned)cdiv(c, TN));
    k_gemm_nn_f32<64><<<grid, 256, 0, s>>>(n, a, c, (float)alpha, X, ldx, B, ldb, (float)beta, Cin, ldc, Out, ldo);
  }
}

void convert_f32_to_f64(const float* src, int64_t lds, double* dst, int64_t ldd, int64_t n, int w, cudaStream_t s) {
  int64_t t = n * w;
  if (t > 0) k_convert<float, double><<<(unsigned)(cdiv(t, 256) < 8192 ? cdiv(t, 256) : 8192), 256, 0, s>>>(src, lds, dst, ldd, n, w);
}
void convert_f64_to_f32(const double* src, int64_t lds, float* dst, int64_t ldd, int64_t n, int w, cudaStream_t s) {
  int64_t t = n * w;
  if (t > 0) k_convert<double, float><<<(unsigned)(cdiv(t, 256) < 8192 ? cdiv(t, 256) : 8192), 256, 0, s>>>(src, lds, dst, ldd, n, w);
}

void residual_norms(const double* MX, const double* X, int64_t ld, int w, const double* theta, int64_t n,
                    double* part, double* out, cudaStream_t s) {
  if (n <= 0 || w <= 0) return;
  int64_t nb = 304;
  int64_t rpb = cdiv(n, nb);
  nb = cdiv(n, rpb);
  k_resid_part<<<(unsigned)nb, 256, 0, s>>>(MX, X, ld, w, theta, n, rpb, part);
  k_resid_final<<<(unsigned)cdiv(w, 64), 64, 0, s>>>(part, nb, w, out);
}

}  // namespace grest
