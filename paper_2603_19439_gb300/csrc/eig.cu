// Symmetric eigensolver for the small projected matrix H = Z^T M Z (Alg. 1,
// first step: leading eigenpairs of Z^T A_hat Z), FP64 throughout.
//
//   1. Householder reduction H = Q T Q^T to tridiagonal form (one CTA; the
//      reflectors stay in H's rows).
//   2. All m eigenvalues of T by Sturm-count multisection: one warp per
//      eigenvalue, its 32 lanes probe 32 points of the bracket at once, so
//      the work spreads over the whole GPU (FP64 throughput per SM on GB300
//      is only about 2 DFMA per clock).
//   3. Tracking order (|theta| descending for the adjacency, theta descending
//      for the shifted Laplacians) and the K leading values.
//   4. Their eigenvectors of T by inverse iteration (tridiagonal LU with
//      partial pivoting), re-orthogonalized inside clusters of close values.
//   5. Back-transformation F = Q Y (one warp per vector).
#include <float.h>

#include "common.cuh"

namespace grest {

namespace {

constexpr int kMaxK = 256;  // selected pairs per call (RSVD basis: L <= 256)

struct EigWork {
  double *d, *e, *beta, *ev, *scr;
  int* ord;
};

__device__ __host__ inline EigWork eig_layout(double* w, int mmax) {
  EigWork L;
  L.d = w;
  L.e = w + mmax;
  L.beta = w + 2 * mmax;
  L.ev = w + 3 * mmax;
  L.ord = reinterpret_cast<int*>(w + 4 * mmax);
  L.scr = w + 5 * mmax;
  return L;
}

__device__ double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double s = 0.0;
  for (int i = 0; i < nw; ++i) s += red[i];  // fixed order
  return s;
}

// --- 1. tridiagonalization (one CTA)
__global__ void __launch_bounds__(1024) k_tridiag(double* H, int64_t ld, int m, double* work, int mmax) {
  extern __shared__ double sm[];  // v[m], p[m]
  __shared__ double red[32];
  EigWork L = eig_layout(work, mmax);
  double* v = sm;
  double* p = sm + m;
  const int tid = threadIdx.x, nth = blockDim.x, lane = tid & 31, wid = tid >> 5, nw = nth >> 5;
  for (int j = 0; j + 2 < m; ++j) {
    const int n = m - j - 1;
    const double* x = H + (int64_t)j * ld + j + 1;  // row j right of the diagonal
    double s = 0.0;
    for (int i = tid; i < n; i += nth) s = fma(x[i], x[i], s);
    const double nrm2 = block_sum(s, red);
    const double x0 = x[0];
    const double alpha = nrm2 > 0.0 ? -copysign(sqrt(nrm2), x0) : 0.0;
    const double beta = nrm2 > 0.0 ? 1.0 / (nrm2 - alpha * x0) : 0.0;
    for (int i = tid; i < n; i += nth) v[i] = (i == 0) ? x0 - alpha : x[i];
    if (tid == 0) {
      L.d[j] = H[(int64_t)j * ld + j];
      L.e[j] = alpha;
      L.beta[j] = beta;
    }
    __syncthreads();
    if (beta != 0.0) {
      // p = beta B v, one warp per row of B = H[j+1:, j+1:]
      for (int i = wid; i < n; i += nw) {
        const double* row = H + (int64_t)(j + 1 + i) * ld + j + 1;
        double a = 0.0;
        for (int l = lane; l < n; l += 32) a = fma(row[l], v[l], a);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
        if (lane == 0) p[i] = beta * a;
      }
      __syncthreads();
      double t = 0.0;
      for (int i = tid; i < n; i += nth) t = fma(p[i], v[i], t);
      const double K = 0.5 * beta * block_sum(t, red);
      for (int i = tid; i < n; i += nth) p[i] -= K * v[i];  // p becomes w
      __syncthreads();
      for (int64_t e = tid; e < (int64_t)n * n; e += nth) {
        int i = (int)(e / n), l = (int)(e % n);
        double* h = H + (int64_t)(j + 1 + i) * ld + j + 1 + l;
        *h -= v[i] * p[l] + p[i] * v[l];
      }
    }
    __syncthreads();
    // keep the reflector in row j for the back-transformation
    for (int i = tid; i < n; i += nth) H[(int64_t)j * ld + j + 1 + i] = v[i];
    __syncthreads();
  }
  if (tid == 0) {
    if (m >= 2) {
      L.d[m - 2] = H[(int64_t)(m - 2) * ld + m - 2];
      L.d[m - 1] = H[(int64_t)(m - 1) * ld + m - 1];
      L.e[m - 2] = H[(int64_t)(m - 2) * ld + m - 1];
    } else if (m == 1) {
      L.d[0] = H[0];
    }
    L.e[m - 1] = 0.0;
  }
}

// Shared-memory variant of step 1: the upper triangle of H is packed row by
// row (element (i, j >= i) at off(i) + j - i, off(i) = i m - i(i-1)/2), so the
// reduction runs out of shared memory for m <= 235.  Reflectors go to H's rows.
__device__ __forceinline__ int poff(int i, int m) { return i * m - (i * (i - 1)) / 2; }

__global__ void __launch_bounds__(1024) k_tridiag_smem(double* H, int64_t ld, int m, double* work, int mmax) {
  extern __shared__ double sm[];
  __shared__ double red[32];
  EigWork L = eig_layout(work, mmax);
  double* A = sm;
  double* v = sm + (m * (m + 1)) / 2;
  double* p = v + m;
  const int tid = threadIdx.x, nth = blockDim.x, lane = tid & 31, wid = tid >> 5, nw = nth >> 5;
  for (int i = wid; i < m; i += nw)
    for (int j = i + lane; j < m; j += 32) A[poff(i, m) + j - i] = H[(int64_t)i * ld + j];
  __syncthreads();
  for (int j = 0; j + 2 < m; ++j) {
    const int n = m - j - 1;
    const double* x = A + poff(j, m) + 1;  // row j right of the diagonal
    double s = 0.0;
    for (int i = tid; i < n; i += nth) s = fma(x[i], x[i], s);
    const double nrm2 = block_sum(s, red);
    const double x0 = x[0];
    const double alpha = nrm2 > 0.0 ? -copysign(sqrt(nrm2), x0) : 0.0;
    const double beta = nrm2 > 0.0 ? 1.0 / (nrm2 - alpha * x0) : 0.0;
    for (int i = tid; i < n; i += nth) v[i] = (i == 0) ? x0 - alpha : x[i];
    if (tid == 0) {
      L.d[j] = A[poff(j, m)];
      L.e[j] = alpha;
      L.beta[j] = beta;
    }
    __syncthreads();
    const int b0 = j + 1;  // B = trailing block, B(i, l) = A(b0 + min, b0 + max)
    if (beta != 0.0) {
      for (int i = wid; i < n; i += nw) {
        const int gi = b0 + i;
        double a = 0.0;
        for (int l = lane; l < n; l += 32) {
          const int gl = b0 + l;
          const double bil = l >= i ? A[poff(gi, m) + gl - gi] : A[poff(gl, m) + gi - gl];
          a = fma(bil, v[l], a);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
        if (lane == 0) p[i] = beta * a;
      }
      __syncthreads();
      double t = 0.0;
      for (int i = tid; i < n; i += nth) t = fma(p[i], v[i], t);
      const double K = 0.5 * beta * block_sum(t, red);
      for (int i = tid; i < n; i += nth) p[i] -= K * v[i];  // p becomes w
      __syncthreads();
      for (int i = wid; i < n; i += nw) {
        const int gi = b0 + i;
        double* row = A + poff(gi, m) - gi;
        const double vi = v[i], wi = p[i];
        for (int l = i + lane; l < n; l += 32) row[b0 + l] -= vi * p[l] + wi * v[l];
      }
    }
    __syncthreads();
    for (int i = tid; i < n; i += nth) H[(int64_t)j * ld + j + 1 + i] = v[i];
    __syncthreads();
  }
  if (tid == 0) {
    if (m >= 2) {
      L.d[m - 2] = A[poff(m - 2, m)];
      L.d[m - 1] = A[poff(m - 1, m)];
      L.e[m - 2] = A[poff(m - 2, m) + 1];
    } else if (m == 1) {
      L.d[0] = A[0];
    }
    L.e[m - 1] = 0.0;
  }
}

__device__ __forceinline__ int sturm_count(const double* d, const double* e, int m, double x, double pivmin) {
  int c = 0;
  double q = d[0] - x;
  if (fabs(q) < pivmin) q = -pivmin;
  c += q < 0.0;
  for (int t = 1; t < m; ++t) {
    double et = e[t - 1];
    q = (d[t] - x) - et * et / q;
    if (fabs(q) < pivmin) q = -pivmin;
    c += q < 0.0;
  }
  return c;
}

// --- 2. eigenvalue number i (ascending) by 32-way multisection, one warp each
__global__ void __launch_bounds__(256) k_multisect(int m, double* work, int mmax) {
  EigWork L = eig_layout(work, mmax);
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (i >= m) return;
  double gl = DBL_MAX, gu = -DBL_MAX, emax2 = 0.0;
  for (int t = lane; t < m; t += 32) {
    double r = (t > 0 ? fabs(L.e[t - 1]) : 0.0) + (t + 1 < m ? fabs(L.e[t]) : 0.0);
    gl = fmin(gl, L.d[t] - r);
    gu = fmax(gu, L.d[t] + r);
    if (t + 1 < m) emax2 = fmax(emax2, L.e[t] * L.e[t]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    gl = fmin(gl, __shfl_xor_sync(0xffffffffu, gl, o));
    gu = fmax(gu, __shfl_xor_sync(0xffffffffu, gu, o));
    emax2 = fmax(emax2, __shfl_xor_sync(0xffffffffu, emax2, o));
  }
  const double tnorm = fmax(fabs(gl), fabs(gu));
  const double pivmin = DBL_MIN * fmax(1.0, emax2);
  double lo = gl - 2.0 * DBL_EPSILON * tnorm - pivmin, hi = gu + 2.0 * DBL_EPSILON * tnorm + pivmin;
  for (int it = 0; it < 40; ++it) {
    if (hi - lo <= 2.0 * DBL_EPSILON * fmax(fabs(lo), fabs(hi)) + pivmin) break;
    const double x = lo + (hi - lo) * (double)(lane + 1) / 33.0;
    const int c = sturm_count(L.d, L.e, m, x, pivmin);
    // first probe holding more than i eigenvalues below it
    unsigned above = __ballot_sync(0xffffffffu, c > i);
    double nlo = lo, nhi = hi;
    if (above) {
      int f = __ffs(above) - 1;
      nhi = __shfl_sync(0xffffffffu, x, f);
      if (f > 0) nlo = __shfl_sync(0xffffffffu, x, f - 1);
    } else {
      nlo = __shfl_sync(0xffffffffu, x, 31);
    }
    lo = nlo;
    hi = nhi;
  }
  if (lane == 0) L.ev[i] = 0.5 * (lo + hi);
}

__device__ __forceinline__ double order_key_cmp(double a, int ia, double b, int ib, int op) {
  // returns < 0 when (a, ia) precedes (b, ib) in tracking order
  if (op == GREST_OP_ADJ) {
    if (fabs(a) != fabs(b)) return fabs(a) > fabs(b) ? -1.0 : 1.0;
  }
  if (a != b) return a > b ? -1.0 : 1.0;
  return ia < ib ? -1.0 : (ia > ib ? 1.0 : 0.0);
}

__device__ __forceinline__ double hash_unit(uint32_t a, uint32_t b) {
  uint32_t h = a * 0x9E3779B1u ^ (b + 0x7F4A7C15u) * 0x85EBCA77u;
  h ^= h >> 15;
  h *= 0x2C1B3C6Du;
  h ^= h >> 12;
  h *= 0x297A2D39u;
  h ^= h >> 15;
  return ((double)h / 4294967296.0) - 0.5;
}

// --- 3 + 4. order, select, inverse iteration, cluster re-orthogonalization
__global__ void __launch_bounds__(256) k_select_invit(int m, int k, int op, double* work, int mmax, double* theta,
                                                      double* F, int64_t ldf, double* ritz, double* info) {
  __shared__ double lam[kMaxK];
  __shared__ int sel_sorted[kMaxK];
  __shared__ double red[32];
  EigWork L = eig_layout(work, mmax);
  const int tid = threadIdx.x, nth = blockDim.x;
  for (int i = tid; i < m; i += nth) {
    double a = L.ev[i];
    int pos = 0;
    for (int j = 0; j < m; ++j)
      if (order_key_cmp(L.ev[j], j, a, i, op) < 0) ++pos;
    L.ord[pos] = i;
    ritz[pos] = a;
  }
  __syncthreads();
  double tnorm = 0.0;
  for (int i = 0; i < m; ++i) tnorm = fmax(tnorm, fabs(L.ev[i]));
  if (tid == 0) {
    for (int t = 0; t < k; ++t) theta[t] = L.ev[L.ord[t]];
    if (m > k) {
      double a = L.ev[L.ord[k - 1]], b = L.ev[L.ord[k]];
      double g = op == GREST_OP_ADJ ? fabs(fabs(a) - fabs(b)) : fabs(a - b);
      info[0] = tnorm > 0.0 ? g / tnorm : 0.0;
    } else {
      info[0] = INFINITY;
    }
    // selected values sorted ascending, pulled apart by at least 10 eps ||T||
    for (int t = 0; t < k; ++t) sel_sorted[t] = t;
    for (int a = 1; a < k; ++a) {
      int x = sel_sorted[a], b = a - 1;
      while (b >= 0 && L.ev[L.ord[sel_sorted[b]]] > L.ev[L.ord[x]]) {
        sel_sorted[b + 1] = sel_sorted[b];
        --b;
      }
      sel_sorted[b + 1] = x;
    }
    const double sep = 10.0 * DBL_EPSILON * fmax(tnorm, DBL_MIN);
    for (int a = 0; a < k; ++a) {
      double v = L.ev[L.ord[sel_sorted[a]]];
      if (a > 0 && v < lam[sel_sorted[a - 1]] + sep) v = lam[sel_sorted[a - 1]] + sep;
      lam[sel_sorted[a]] = v;
    }
  }
  __syncthreads();
  // inverse iteration on T - lambda I, one thread per selected pair
  if (tid < k) {
    const int t = tid;
    // per-thread arrays interleaved across threads (coalesced): element i at [i * kMaxK]
    struct Strided {
      double* b;
      __device__ double& operator[](int i) const { return b[(int64_t)i * kMaxK]; }
    };
    const Strided a{L.scr + t}, c{L.scr + (int64_t)mmax * kMaxK + t}, c2{L.scr + (int64_t)2 * mmax * kMaxK + t},
        l{L.scr + (int64_t)3 * mmax * kMaxK + t}, y{L.scr + (int64_t)4 * mmax * kMaxK + t};
    const double lm = lam[t];
    const double eps = DBL_EPSILON * fmax(tnorm, DBL_MIN);
    for (int i = 0; i < m; ++i) {
      a[i] = L.d[i] - lm;
      c[i] = (i + 1 < m) ? L.e[i] : 0.0;
      c2[i] = 0.0;
    }
    // LU with partial pivoting (row swaps recorded in y, then moved to `flags`)
    for (int i = 0; i + 1 < m; ++i) {
      const double b = L.e[i];  // sub-diagonal entry below a[i]
      if (fabs(a[i]) >= fabs(b)) {
        if (a[i] == 0.0) a[i] = eps;
        const double f = b / a[i];
        l[i] = f;
        a[i + 1] -= f * c[i];
        y[i] = 0.0;  // not swapped
      } else {
        const double f = a[i] / b;
        l[i] = f;
        a[i] = b;
        const double t1 = a[i + 1];
        a[i + 1] = c[i] - f * t1;
        if (i + 2 < m) {
          c2[i] = c[i + 1];
          c[i + 1] = -f * c[i + 1];
        }
        c[i] = t1;
        y[i] = 1.0;  // swapped
      }
    }
    if (a[m - 1] == 0.0) a[m - 1] = eps;
    const Strided flags{L.scr + (int64_t)5 * mmax * kMaxK + t};
    for (int i = 0; i < m; ++i) flags[i] = y[i];
    for (int i = 0; i < m; ++i) y[i] = hash_unit((uint32_t)i, (uint32_t)(t * 7919 + 13)) + 0.5 / (1 + i % 7);
    for (int it = 0; it < 3; ++it) {
      // forward: apply L with row swaps
      for (int i = 0; i + 1 < m; ++i) {
        if (flags[i] != 0.0) {
          const double t1 = y[i];
          y[i] = y[i + 1];
          y[i + 1] = t1 - l[i] * y[i];
        } else {
          y[i + 1] -= l[i] * y[i];
        }
      }
      // backward: U y = rhs
      y[m - 1] /= a[m - 1];
      if (m >= 2) y[m - 2] = (y[m - 2] - c[m - 2] * y[m - 1]) / a[m - 2];
      for (int i = m - 3; i >= 0; --i) y[i] = (y[i] - c[i] * y[i + 1] - c2[i] * y[i + 2]) / a[i];
      double nr = 0.0;
      for (int i = 0; i < m; ++i) nr = fma(y[i], y[i], nr);
      nr = 1.0 / sqrt(nr);
      for (int i = 0; i < m; ++i) y[i] *= nr;
    }
    for (int i = 0; i < m; ++i) F[(int64_t)i * ldf + t] = y[i];
  }
  __syncthreads();
  // clusters of close selected values: block classical Gram-Schmidt, applied
  // twice, in ascending order; all projections of one vector run in parallel
  // (one warp per earlier cluster member), so a cluster of c vectors costs
  // O(c) block synchronizations instead of O(c^2)
  __shared__ double dots[kMaxK];
  const double ortol = 1e-3 * tnorm;
  const int lane = tid & 31, wid = tid >> 5, nw = nth >> 5;
  for (int a = 1; a < k; ++a) {
    const int ta = sel_sorted[a];
    int b0 = a;
    while (b0 > 0 && lam[sel_sorted[b0]] - lam[sel_sorted[b0 - 1]] < ortol) --b0;
    if (b0 == a) continue;
    for (int pass = 0; pass < 2; ++pass) {
      for (int b = b0 + wid; b < a; b += nw) {
        const int tb = sel_sorted[b];
        double d = 0.0;
        for (int i = lane; i < m; i += 32) d = fma(F[(int64_t)i * ldf + tb], F[(int64_t)i * ldf + ta], d);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
        if (lane == 0) dots[b - b0] = d;
      }
      __syncthreads();
      for (int i = tid; i < m; i += nth) {
        double y = F[(int64_t)i * ldf + ta];
        for (int b = b0; b < a; ++b) y = fma(-dots[b - b0], F[(int64_t)i * ldf + sel_sorted[b]], y);
        F[(int64_t)i * ldf + ta] = y;
      }
      __syncthreads();
    }
    double s2 = 0.0;
    for (int i = tid; i < m; i += nth) s2 = fma(F[(int64_t)i * ldf + ta], F[(int64_t)i * ldf + ta], s2);
    s2 = block_sum(s2, red);
    const double inv = s2 > 0.0 ? 1.0 / sqrt(s2) : 0.0;
    for (int i = tid; i < m; i += nth) F[(int64_t)i * ldf + ta] *= inv;
    __syncthreads();
  }
}

// --- 5. F = Q Y, Q = P_0 P_1 ... P_{m-3}; one warp per selected vector
__global__ void __launch_bounds__(256) k_backtransform(const double* H, int64_t ld, int m, int k, double* work,
                                                       int mmax, double* F, int64_t ldf) {
  extern __shared__ double xs[];  // 8 warps x m
  EigWork L = eig_layout(work, mmax);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int t = blockIdx.x * 8 + wid;
  if (t >= k) return;
  double* x = xs + wid * m;
  for (int i = lane; i < m; i += 32) x[i] = F[(int64_t)i * ldf + t];
  __syncwarp();
  for (int j = m - 3; j >= 0; --j) {
    const double b = L.beta[j];
    if (b == 0.0) continue;
    const double* v = H + (int64_t)j * ld + j + 1;
    const int n = m - j - 1;
    double s = 0.0;
    for (int i = lane; i < n; i += 32) s = fma(v[i], x[j + 1 + i], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    s *= b;
    for (int i = lane; i < n; i += 32) x[j + 1 + i] -= s * v[i];
    __syncwarp();
  }
  for (int i = lane; i < m; i += 32) F[(int64_t)i * ldf + t] = x[i];
}

}  // namespace

size_t eig_work_doubles(int mmax) { return (size_t)5 * mmax + (size_t)kMaxK * 6 * mmax + 64; }

void sym_eig_select(double* H, int64_t ld, int m, int k, int op, double* theta, double* F, int64_t ldf, double* ritz,
                    double* info, double* work, cudaStream_t s) {
  const int mmax = m;
  const size_t smem = sizeof(double) * ((size_t)m * (m + 1) / 2 + 2 * (size_t)m + 2);
  if (reserve_dynamic_smem(k_tridiag_smem, smem)) {
    k_tridiag_smem<<<1, 1024, smem, s>>>(H, ld, m, work, mmax);
  } else {
    k_tridiag<<<1, 1024, sizeof(double) * 2 * (m + 1), s>>>(H, ld, m, work, mmax);
  }
  k_multisect<<<(m + 7) / 8, 256, 0, s>>>(m, work, mmax);
  k_select_invit<<<1, 256, 0, s>>>(m, k, op, work, mmax, theta, F, ldf, ritz, info);
  k_backtransform<<<(k + 7) / 8, 256, sizeof(double) * 8 * m, s>>>(H, ld, m, k, work, mmax, F, ldf);
}

}  // namespace grest
