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

constexpr int kMaxM = 512;  // largest projected problem (K + 2 (L + P) <= 576 is rejected earlier)

struct EigWork {
  double *d, *e, *ds, *e2, *beta, *ev, *lam, *tnorm, *scr;
  float *dsf, *e2f;          // FP32 copies of ds, e2 for the FP32 multisection
  float *df, *ef, *betaf;    // FP32 copies of d, e, beta
  float* vf;                 // FP32 reflectors (row j, ld m) of the FP32 path
  int *ord, *sel, *cl0;      // cl0[a]: first member of the cluster of sorted selected value a
};

// d, e, scaled d, scaled e^2, beta, ev: mmax each; ord: mmax ints; lam: kMaxK;
// sel: kMaxK ints; tnorm[8]; FP32 copies of ds, e2, d, e, beta; cl0 (kMaxK
// ints); FP32 reflectors (mmax x mmax floats); then the inverse-iteration
// scratch (6 mmax kMaxK).
__device__ __host__ inline EigWork eig_layout(double* w, int mmax) {
  EigWork L;
  L.d = w;
  L.e = w + mmax;
  L.ds = w + 2 * mmax;
  L.e2 = w + 3 * mmax;
  L.beta = w + 4 * mmax;
  L.ev = w + 5 * mmax;
  L.ord = reinterpret_cast<int*>(w + 6 * mmax);
  L.lam = w + 7 * mmax;
  L.sel = reinterpret_cast<int*>(w + 7 * mmax + kMaxK);
  L.tnorm = w + 7 * mmax + 2 * kMaxK;
  double* f0 = w + 7 * mmax + 2 * kMaxK + 8;  // FP32 region: 5 mmax floats (3 mmax doubles)
  L.dsf = reinterpret_cast<float*>(f0);
  L.e2f = L.dsf + mmax;
  L.df = L.e2f + mmax;
  L.ef = L.df + mmax;
  L.betaf = L.ef + mmax;
  L.cl0 = reinterpret_cast<int*>(f0 + 3 * mmax);  // kMaxK ints
  L.vf = reinterpret_cast<float*>(f0 + 3 * mmax + kMaxK / 2);
  L.scr = f0 + 3 * mmax + kMaxK / 2 + ((size_t)mmax * mmax + 1) / 2;
  return L;
}

template <typename T>
__device__ T block_sum(T v, T* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  T s = 0;
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

// Sturm count: the number of eigenvalues of T below x equals the number of
// sign changes in p_0 = 1, p_1, ..., p_m with p_t = (d_t - x) p_{t-1} -
// e_{t-1}^2 p_{t-2} (the leading principal minors of T - x I).  This
// product form needs no division, which matters on GB300, where one FP64
// warp instruction costs ~68 clocks and a division about ten of them.  T is
// pre-scaled by a power of two to norm ~1, an exact zero p_t is replaced by
// -floor_q p_{t-1} (the minor ratio q_t = p_t / p_{t-1} pushed just below
// zero), and the pair (p_t, p_{t-1}) is rescaled by a power of two (exact)
// whenever p_t leaves [2^-400, 2^400].
__device__ __forceinline__ int sturm_count(const double* d, const double* e2, int m, double x, double floor_q) {
  double pm2 = 0.0, pm1 = 1.0;
  int cnt = 0;
  bool neg_prev = false;
  for (int t = 0; t < m; ++t) {
    double pt = fma(-(t > 0 ? e2[t - 1] : 0.0), pm2, (d[t] - x) * pm1);
    if (((__double2hiint(pt) & 0x7fffffff) | __double2loint(pt)) == 0) pt = -floor_q * pm1;
    const int hw = __double2hiint(pt);
    const bool neg = hw < 0;
    cnt += neg != neg_prev;
    neg_prev = neg;
    const int ex = (hw >> 20) & 0x7ff;
    if (ex > 1023 + 400 || ex < 1023 - 400) {
      const int field = max(2046 - ex, 1);  // 2^(1023 - ex)
      const double sc = __hiloint2double(field << 20, 0);
      pt *= sc;
      pm1 *= sc;
    }
    pm2 = pm1;
    pm1 = pt;
  }
  return cnt;
}

// The same count in FP32 (the projected problems of the mixed path): the
// narrow FP32 exponent range calls for renormalizing p_t to [1, 2) at every
// step (two FP32 multiplies by an exact power of two).
__device__ __forceinline__ int sturm_count_f(const float* d, const float* e2, int m, float x, float floor_q) {
  float pm2 = 0.f, pm1 = 1.f;
  int cnt = 0;
  bool neg_prev = false;
  for (int t = 0; t < m; ++t) {
    float pt = fmaf(-(t > 0 ? e2[t - 1] : 0.f), pm2, (d[t] - x) * pm1);
    if ((__float_as_int(pt) & 0x7fffffff) == 0) pt = -floor_q * pm1;
    const int bits = __float_as_int(pt);
    const bool neg = bits < 0;
    cnt += neg != neg_prev;
    neg_prev = neg;
    const int ex = (bits >> 23) & 0xff;
    if (ex != 0) {
      const float sc = __int_as_float(max(254 - ex, 1) << 23);  // 2^(127 - ex)
      pt *= sc;
      pm1 *= sc;
    }
    pm2 = pm1;
    pm1 = pt;
  }
  return cnt;
}

// Gershgorin bounds of T and the exact power-of-two scaling used by the
// multisection: ds = s d, e2 = (s e)^2, tnorm[1..4] = s gl, s gu, 1/s, s ||T||.
__global__ void __launch_bounds__(256) k_sturm_prep(int m, double* work, int mmax) {
  __shared__ double rlo[32], rhi[32];
  __shared__ double bs[2];
  EigWork L = eig_layout(work, mmax);
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  double gl = DBL_MAX, gu = -DBL_MAX;
  for (int t = tid; t < m; t += blockDim.x) {
    const double r = (t > 0 ? fabs(L.e[t - 1]) : 0.0) + (t + 1 < m ? fabs(L.e[t]) : 0.0);
    gl = fmin(gl, L.d[t] - r);
    gu = fmax(gu, L.d[t] + r);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    gl = fmin(gl, __shfl_down_sync(0xffffffffu, gl, o));
    gu = fmax(gu, __shfl_down_sync(0xffffffffu, gu, o));
  }
  if (lane == 0) {
    rlo[wid] = gl;
    rhi[wid] = gu;
  }
  __syncthreads();
  if (tid == 0) {
    for (int w = 1; w < nw; ++w) {
      gl = fmin(gl, rlo[w]);
      gu = fmax(gu, rhi[w]);
    }
    const double tn = fmax(fmax(fabs(gl), fabs(gu)), DBL_MIN);
    const int E = min(((__double2hiint(tn) >> 20) & 0x7ff) - 1023, 1022);
    const double sc = __hiloint2double((1023 - E) << 20, 0);  // 2^-E
    bs[0] = sc;
    L.tnorm[1] = gl * sc;
    L.tnorm[2] = gu * sc;
    L.tnorm[3] = __hiloint2double((1023 + E) << 20, 0);  // 2^E
    L.tnorm[4] = tn * sc;
  }
  __syncthreads();
  const double sc = bs[0];
  for (int t = tid; t < m; t += blockDim.x) {
    L.ds[t] = L.d[t] * sc;
    const double es = L.e[t] * sc;
    L.e2[t] = es * es;
    L.dsf[t] = (float)L.ds[t];
    L.e2f[t] = (float)L.e2[t];
    L.df[t] = (float)L.d[t];
    L.ef[t] = (float)L.e[t];
    L.betaf[t] = (float)L.beta[t];
  }
}

// --- 2. eigenvalue number i (ascending) by 32-way multisection on the scaled
// T; one warp per block so the warps land on separate SM sub-partitions.  The
// bracket is refined to an absolute width of 4 eps ||T|| (eps of the
// arithmetic type).
template <typename T>
__global__ void __launch_bounds__(32) k_multisect(int m, double* work, int mmax) {
  EigWork L = eig_layout(work, mmax);
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x;
  if (i >= m) return;
  constexpr bool F32 = sizeof(T) == 4;
  const T eps = F32 ? (T)FLT_EPSILON : (T)DBL_EPSILON;
  const T tnorm = (T)L.tnorm[4];
  const T floor_q = F32 ? eps * T(1.0 / 1024.0) * tnorm : eps * eps * tnorm;
  const T tol = T(4) * eps * tnorm;
  T lo = (T)L.tnorm[1] - tol, hi = (T)L.tnorm[2] + tol;
  for (int it = 0; it < 40 && hi - lo > tol; ++it) {
    const T x = lo + (hi - lo) * (T)(lane + 1) / T(33);
    int c;
    if constexpr (F32) c = sturm_count_f(L.dsf, L.e2f, m, x, floor_q);
    else c = sturm_count(L.ds, L.e2, m, x, floor_q);
    // first probe holding more than i eigenvalues below it
    const unsigned above = __ballot_sync(0xffffffffu, c > i);
    T nlo = lo, nhi = hi;
    if (above) {
      const int f = __ffs(above) - 1;
      nhi = __shfl_sync(0xffffffffu, x, f);
      if (f > 0) nlo = __shfl_sync(0xffffffffu, x, f - 1);
    } else {
      nlo = __shfl_sync(0xffffffffu, x, 31);
    }
    lo = nlo;
    hi = nhi;
  }
  if (lane == 0) L.ev[i] = 0.5 * ((double)lo + (double)hi) * L.tnorm[3];
}

// Order-preserving integer image of a double (-0 and +0 equal).
__device__ __forceinline__ long long ord_key(double x) {
  long long b = __double_as_longlong(x);
  if ((b & 0x7fffffffffffffffll) == 0) return 0;
  return b >= 0 ? b : -(b & 0x7fffffffffffffffll);
}

// --- 3. tracking order (|theta| descending for the adjacency, theta
// descending otherwise, lower index first on ties), the K leading values, the
// boundary gap, and the selected values sorted ascending and pulled apart by
// at least 10 eps ||T|| for the inverse iteration.
__global__ void __launch_bounds__(256) k_select(int m, int k, int op, double* work, int mmax, double* theta,
                                                double* ritz, double* info, double eps) {
  __shared__ long long k1[kMaxM], k2[kMaxM];
  __shared__ int sel_i[kMaxK];
  EigWork L = eig_layout(work, mmax);
  const int tid = threadIdx.x, nth = blockDim.x;
  for (int i = tid; i < m; i += nth) {
    const double a = L.ev[i];
    k1[i] = op == GREST_OP_ADJ ? ord_key(fabs(a)) : 0;
    k2[i] = ord_key(a);
  }
  __syncthreads();
  for (int i = tid; i < m; i += nth) {
    int pos = 0;
    const long long a1 = k1[i], a2 = k2[i];
    for (int j = 0; j < m; ++j) {
      const long long b1 = k1[j], b2 = k2[j];
      pos += (b1 > a1) || (b1 == a1 && (b2 > a2 || (b2 == a2 && j < i)));
    }
    L.ord[pos] = i;
    ritz[pos] = L.ev[i];
  }
  __syncthreads();
  // selected indices sorted ascending by value = ascending by index (ev is
  // ascending in its index up to the bracket width)
  for (int t = tid; t < k; t += nth) {
    const int it = L.ord[t];
    int pos = 0;
    for (int u = 0; u < k; ++u) pos += L.ord[u] < it;
    sel_i[pos] = t;
  }
  for (int t = tid; t < k; t += nth) theta[t] = L.ev[L.ord[t]];
  __syncthreads();
  if (tid == 0) {
    const double tnorm = fmax(fabs(L.ev[0]), fabs(L.ev[m - 1]));
    if (m > k) {
      const double a = L.ev[L.ord[k - 1]], b = L.ev[L.ord[k]];
      const double g = op == GREST_OP_ADJ ? fabs(fabs(a) - fabs(b)) : fabs(a - b);
      info[0] = tnorm > 0.0 ? g / tnorm : 0.0;
    } else {
      info[0] = INFINITY;
    }
    const double sep = 10.0 * eps * fmax(tnorm, DBL_MIN);
    double prev = -DBL_MAX;
    const double ortol = 1e-3 * tnorm;
    int c0 = 0;
    for (int a = 0; a < k; ++a) {
      const int t = sel_i[a];
      double v = L.ev[L.ord[t]];
      if (a > 0 && v < prev + sep) v = prev + sep;
      if (a > 0 && !(v - prev < ortol)) c0 = a;  // a starts a new cluster
      L.lam[t] = v;
      L.sel[a] = t;
      L.cl0[a] = c0;
      prev = v;
    }
    L.tnorm[0] = tnorm;
  }
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

// --- 4. eigenvectors of T by inverse iteration (tridiagonal LU with partial
// pivoting, three solves from a fixed pseudo-random start), one thread per
// selected pair and LANES pairs per block: the chains are serial, so the
// blocks are spread over the SMs (an FP64 warp instruction costs the same
// for 8 active lanes as for 32, so the FP64 path takes 8 pairs per block and
// keeps their arrays in shared memory).  The reciprocal of each U pivot is
// formed once in the LU and reused by the solves.
template <typename T>
__device__ __forceinline__ T recip(T a) {
  if constexpr (sizeof(T) == sizeof(double)) return rcp_newton(a);
  else return T(1) / a;
}

template <typename T, bool SMEM, int LANES>
__global__ void __launch_bounds__(32) k_invit(int m, int k, double* work, int mmax, double* F, int64_t ldf) {
  EigWork L = eig_layout(work, mmax);
  extern __shared__ __align__(16) unsigned char iv_raw[];
  const int t = blockIdx.x * LANES + threadIdx.x;
  if (threadIdx.x >= LANES || t >= k) return;
  // per-thread arrays interleaved across threads (coalesced / conflict-free):
  // element i at [i * stride], in shared memory (stride LANES, planes of m)
  // or global scratch (stride kMaxK, planes of mmax)
  struct Strided {
    T* b;
    int64_t st;
    __device__ T& operator[](int i) const { return b[(int64_t)i * st]; }
  };
  T* scr;
  int64_t st;
  if (SMEM) {
    scr = reinterpret_cast<T*>(iv_raw) + threadIdx.x;
    st = LANES;
  } else {
    scr = reinterpret_cast<T*>(L.scr) + t;
    st = kMaxK;
  }
  const int64_t pl = (int64_t)(SMEM ? m : mmax) * st;
  const Strided ur{scr, st}, c{scr + pl, st}, c2{scr + 2 * pl, st}, l{scr + 3 * pl, st}, y{scr + 4 * pl, st},
      flags{scr + 5 * pl, st};
  constexpr bool F32 = sizeof(T) == 4;
  auto dd = [&](int i) -> T { return F32 ? (T)L.df[i] : (T)L.d[i]; };
  auto ee = [&](int i) -> T { return F32 ? (T)L.ef[i] : (T)L.e[i]; };
  const T lm = (T)L.lam[t];
  const T eps = (F32 ? (T)FLT_EPSILON : (T)DBL_EPSILON) * (T)fmax(L.tnorm[0], DBL_MIN);
  // LU of T - lambda I with partial pivoting; ur[i] = 1 / U_ii
  T ai = dd(0) - lm;  // running diagonal entry of the active row
  T ci = m > 1 ? ee(0) : T(0);
  for (int i = 0; i + 1 < m; ++i) {
    const T b = ee(i);  // sub-diagonal entry below a_i
    const T an = dd(i + 1) - lm;
    const T cn = i + 2 < m ? ee(i + 1) : T(0);
    if (fabs(ai) >= fabs(b)) {
      if (ai == T(0)) ai = eps;
      const T r = recip(ai);
      ur[i] = r;
      const T f = b * r;
      l[i] = f;
      c[i] = ci;
      c2[i] = 0;
      flags[i] = 0;
      ai = an - f * ci;
      ci = cn;
    } else {
      const T r = recip(b);
      ur[i] = r;
      const T f = ai * r;
      l[i] = f;
      c[i] = an;
      c2[i] = cn;
      flags[i] = 1;
      ai = ci - f * an;
      ci = -f * cn;
    }
  }
  if (ai == T(0)) ai = eps;
  ur[m - 1] = recip(ai);
  c[m - 1] = 0;
  c2[m - 1] = 0;
  for (int i = 0; i < m; ++i) y[i] = (T)(hash_unit((uint32_t)i, (uint32_t)(t * 7919 + 13)) + 0.5 / (1 + i % 7));
  for (int it = 0; it < 3; ++it) {
    // forward: apply L with row swaps
    for (int i = 0; i + 1 < m; ++i) {
      if (flags[i] != T(0)) {
        const T t1 = y[i];
        y[i] = y[i + 1];
        y[i + 1] = t1 - l[i] * y[i];
      } else {
        y[i + 1] -= l[i] * y[i];
      }
    }
    // backward: U y = rhs
    T y1 = y[m - 1] * ur[m - 1], y2 = 0;
    y[m - 1] = y1;
    for (int i = m - 2; i >= 0; --i) {
      const T yi = (y[i] - c[i] * y1 - c2[i] * y2) * ur[i];
      y[i] = yi;
      y2 = y1;
      y1 = yi;
    }
    T nr = 0;
    for (int i = 0; i < m; ++i) nr = fma(y[i], y[i], nr);
    if constexpr (sizeof(T) == sizeof(double)) nr = rsqrt(nr);
    else nr = T(1) / sqrt(nr);
    for (int i = 0; i < m; ++i) y[i] *= nr;
  }
  for (int i = 0; i < m; ++i) F[(int64_t)i * ldf + t] = (double)y[i];
}

// --- clusters of close selected values: block classical Gram-Schmidt, applied
// twice, in ascending order; all projections of one vector run in parallel
// (one warp per earlier cluster member), so a cluster of c vectors costs
// O(c) block synchronizations instead of O(c^2).
template <typename T, bool SMEM>
__global__ void __launch_bounds__(256) k_cluster_orth(int m, int k, double* work, int mmax, double* Fg,
                                                      int64_t ldg) {
  __shared__ T dots[kMaxK];
  __shared__ T red[32];
  extern __shared__ __align__(16) double co_sm[];
  EigWork L = eig_layout(work, mmax);
  const int tid = threadIdx.x, nth = blockDim.x, lane = tid & 31, wid = tid >> 5, nw = nth >> 5;
  // the k vectors (m x k) in shared memory when they fit: every dot product
  // and update below then runs on shared memory instead of global loads
  double* F = SMEM ? co_sm : Fg;
  const int64_t ldf = SMEM ? k : ldg;
  if (SMEM) {
    for (int e = tid; e < m * k; e += nth) co_sm[e] = Fg[(int64_t)(e / k) * ldg + (e % k)];
    __syncthreads();
  }
  for (int a = 1; a < k; ++a) {
    const int ta = L.sel[a];
    const int b0 = L.cl0[a];
    if (b0 == a) continue;
    for (int pass = 0; pass < 2; ++pass) {
      for (int b = b0 + wid; b < a; b += nw) {
        const int tb = L.sel[b];
        T d = 0;
        for (int i = lane; i < m; i += 32) d = fma((T)F[(int64_t)i * ldf + tb], (T)F[(int64_t)i * ldf + ta], d);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
        if (lane == 0) dots[b - b0] = d;
      }
      __syncthreads();
      for (int i = tid; i < m; i += nth) {
        T y = (T)F[(int64_t)i * ldf + ta];
        for (int b = b0; b < a; ++b) y = fma(-dots[b - b0], (T)F[(int64_t)i * ldf + L.sel[b]], y);
        F[(int64_t)i * ldf + ta] = (double)y;
      }
      __syncthreads();
    }
    T s2 = 0;
    for (int i = tid; i < m; i += nth) s2 = fma((T)F[(int64_t)i * ldf + ta], (T)F[(int64_t)i * ldf + ta], s2);
    s2 = block_sum(s2, red);
    T inv = 0;
    if (s2 > T(0)) {
      if constexpr (sizeof(T) == sizeof(double)) inv = rsqrt(s2);
      else inv = T(1) / sqrt(s2);
    }
    for (int i = tid; i < m; i += nth) F[(int64_t)i * ldf + ta] = (double)((T)F[(int64_t)i * ldf + ta] * inv);
    __syncthreads();
  }
  if (SMEM)
    for (int e = tid; e < m * k; e += nth) Fg[(int64_t)(e / k) * ldg + (e % k)] = co_sm[e];
}

// --- 5. F = Q Y, Q = P_0 P_1 ... P_{m-3}; one warp per selected vector, four
// warps per block (one per SM sub-partition).
constexpr int kBtWarps = 4;

// Row j of the packed reflector block starts at off(j) = j (2m - j - 1) / 2
// (row r holds the m - r - 1 entries right of the diagonal).
__device__ __forceinline__ int64_t refl_off(int m, int j) { return (int64_t)j * (2 * m - j - 1) / 2; }
inline int64_t refl_off_host(int m, int j) { return (int64_t)j * (2 * m - j - 1) / 2; }

template <typename T, bool SMEM>
__global__ void __launch_bounds__(kBtWarps * 32) k_backtransform(const double* H, int64_t ld, int m, int k,
                                                                double* work, int mmax, double* F, int64_t ldf) {
  extern __shared__ __align__(16) unsigned char bt_raw[];  // kBtWarps x m, then (SMEM) the packed reflectors
  EigWork L = eig_layout(work, mmax);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int t = blockIdx.x * kBtWarps + wid;
  constexpr bool F32 = sizeof(T) == 4;
  T* vs = reinterpret_cast<T*>(bt_raw) + kBtWarps * m;
  if (SMEM) {
    // every reflector once into shared memory (independent loads, all in
    // flight together), so the serial chain below waits on no global load
    const int64_t total = refl_off(m, m - 1);
    for (int64_t e = threadIdx.x; e < total; e += blockDim.x) {
      const float q = (float)(2 * m - 1);
      int j = (int)((q - sqrtf(fmaxf(q * q - 8.f * (float)e, 0.f))) * 0.5f);
      j = j < 0 ? 0 : (j > m - 2 ? m - 2 : j);
      while (j > 0 && refl_off(m, j) > e) --j;
      while (j < m - 2 && refl_off(m, j + 1) <= e) ++j;
      const int i = (int)(e - refl_off(m, j));
      vs[e] = F32 ? (T)L.vf[(size_t)j * m + j + 1 + i] : (T)H[(int64_t)j * ld + j + 1 + i];
    }
    __syncthreads();
  }
  if (t >= k) return;
  T* x = reinterpret_cast<T*>(bt_raw) + wid * m;
  for (int i = lane; i < m; i += 32) x[i] = (T)F[(int64_t)i * ldf + t];
  __syncwarp();
  for (int j = m - 3; j >= 0; --j) {
    const T b = F32 ? (T)L.betaf[j] : (T)L.beta[j];
    if (b == T(0)) continue;
    const double* v = H + (int64_t)j * ld + j + 1;
    const float* vfj = L.vf + (size_t)j * m + j + 1;
    const T* vj = vs + refl_off(m, j);
    const int n = m - j - 1;
    auto vat = [&](int i) -> T { return SMEM ? vj[i] : (F32 ? (T)vfj[i] : (T)v[i]); };
    T s = 0;
    for (int i = lane; i < n; i += 32) s = fma(vat(i), x[j + 1 + i], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    s *= b;
    for (int i = lane; i < n; i += 32) x[j + 1 + i] -= s * vat(i);
    __syncwarp();
  }
  for (int i = lane; i < m; i += 32) F[(int64_t)i * ldf + t] = (double)x[i];
}

// FP32 copies of reflectors stored in H's rows (cluster / fallback reductions)
__global__ void k_reflectors_f32(const double* H, int64_t ld, int m, double* work, int mmax) {
  EigWork L = eig_layout(work, mmax);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)m * m; e += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(e / m), l = (int)(e % m);
    if (l > j) L.vf[e] = (float)H[(int64_t)j * ld + l];
  }
}

}  // namespace

size_t eig_work_doubles(int mmax) {
  return (size_t)10 * mmax + 2 * kMaxK + 8 + kMaxK / 2 + ((size_t)mmax * mmax + 1) / 2 + (size_t)kMaxK * 6 * mmax + 64;
}

bool tridiag_cluster(double* H, int64_t ld, int m, double* d, double* e, double* beta, bool f32, cudaStream_t s);
bool tridiag_f32_1cta(const double* H, int64_t ld, int m, double* d, double* e, double* beta, float* df, float* ef,
                      float* betaf, float* vf, cudaStream_t s);

template <typename T>
void backtransform(const double* H, int64_t ld, int m, int k, double* work, int mmax, double* F, int64_t ldf,
                   cudaStream_t s) {
  const unsigned nbt = (unsigned)((k + kBtWarps - 1) / kBtWarps);
  const size_t vec = sizeof(T) * kBtWarps * (size_t)m;
  const size_t refl = m >= 2 ? sizeof(T) * (size_t)refl_off_host(m, m - 1) : 0;
  if (m >= 3 && reserve_dynamic_smem(k_backtransform<T, true>, vec + refl))
    k_backtransform<T, true><<<nbt, kBtWarps * 32, vec + refl, s>>>(H, ld, m, k, work, mmax, F, ldf);
  else
    k_backtransform<T, false><<<nbt, kBtWarps * 32, vec, s>>>(H, ld, m, k, work, mmax, F, ldf);
}

template <typename T>
void cluster_orth(int m, int k, double* work, int mmax, double* F, int64_t ldf, cudaStream_t s) {
  const size_t smem = sizeof(double) * (size_t)m * k;
  if (reserve_dynamic_smem(k_cluster_orth<T, true>, smem))
    k_cluster_orth<T, true><<<1, 256, smem, s>>>(m, k, work, mmax, F, ldf);
  else
    k_cluster_orth<T, false><<<1, 256, 0, s>>>(m, k, work, mmax, F, ldf);
}

int sym_eig_select(double* H, int64_t ld, int m, int k, int op, double* theta, double* F, int64_t ldf, double* ritz,
                   double* info, double* work, bool f32, cudaStream_t s) {
  const int mmax = m;
  EigWork L = eig_layout(work, mmax);
  int launches = 6;
  // one SM for small problems, a cluster for large ones (as for the pivoted Cholesky)
  if (f32 && m <= 64 && tridiag_f32_1cta(H, ld, m, L.d, L.e, L.beta, L.df, L.ef, L.betaf, L.vf, s)) {
    launches += 1;
  } else if (tridiag_cluster(H, ld, m, L.d, L.e, L.beta, f32, s)) {
    launches += 1;
    if (f32) {
      k_reflectors_f32<<<64, 256, 0, s>>>(H, ld, m, work, mmax);
      launches += 1;
    }
  } else {
    const size_t smem = sizeof(double) * ((size_t)m * (m + 1) / 2 + 2 * (size_t)m + 2);
    if (reserve_dynamic_smem(k_tridiag_smem, smem)) {
      k_tridiag_smem<<<1, 1024, smem, s>>>(H, ld, m, work, mmax);
    } else {
      k_tridiag<<<1, 1024, sizeof(double) * 2 * (m + 1), s>>>(H, ld, m, work, mmax);
    }
    launches += 1;
    if (f32) {
      k_reflectors_f32<<<64, 256, 0, s>>>(H, ld, m, work, mmax);
      launches += 1;
    }
  }
  k_sturm_prep<<<1, 256, 0, s>>>(m, work, mmax);
  const unsigned niv = (unsigned)((k + 31) / 32);
  if (f32) {
    k_multisect<float><<<m, 32, 0, s>>>(m, work, mmax);
    k_select<<<1, 256, 0, s>>>(m, k, op, work, mmax, theta, ritz, info, (double)FLT_EPSILON);
    const size_t ism = sizeof(float) * 6 * 32 * (size_t)m;
    if (reserve_dynamic_smem(k_invit<float, true, 32>, ism))
      k_invit<float, true, 32><<<niv, 32, ism, s>>>(m, k, work, mmax, F, ldf);
    else
      k_invit<float, false, 32><<<niv, 32, 0, s>>>(m, k, work, mmax, F, ldf);
    cluster_orth<float>(m, k, work, mmax, F, ldf, s);
    backtransform<float>(H, ld, m, k, work, mmax, F, ldf, s);
  } else {
    k_multisect<double><<<m, 32, 0, s>>>(m, work, mmax);
    k_select<<<1, 256, 0, s>>>(m, k, op, work, mmax, theta, ritz, info, DBL_EPSILON);
    const size_t dsm = sizeof(double) * 6 * 8 * (size_t)m;
    if (reserve_dynamic_smem(k_invit<double, true, 8>, dsm))
      k_invit<double, true, 8><<<(unsigned)((k + 7) / 8), 8, dsm, s>>>(m, k, work, mmax, F, ldf);
    else
      k_invit<double, false, 32><<<niv, 32, 0, s>>>(m, k, work, mmax, F, ldf);
    cluster_orth<double>(m, k, work, mmax, F, ldf, s);
    backtransform<double>(H, ld, m, k, work, mmax, F, ldf, s);
  }
  return launches;
}

}  // namespace grest
