// Small dense FP64 factorizations spread over a thread-block cluster.
//
// The projected problems of a G-REST step are m x m with m ~ 30..320
// (H = Z^T M Z of Eq. main2, the CholQR Gram matrices of the orthonormal
// bases, the RSVD Gram B_s B_s^T of Sec. 3.5).  On GB300 one SM retires only
// about two FP64 FMAs per clock (one warp instruction per ~68 clocks on each
// of its four sub-partitions), so a single-CTA factorization is bound by one
// SM's FP64 pipe.  Here the rows of the symmetric matrix are dealt
// cyclically over the CTAs of a cluster (row i lives in CTA i mod C); every
// CTA keeps its rows in shared memory, reads the few vectors it needs from
// the others through distributed shared memory, and applies the rank-1 / 2
// updates to its own rows.  Scalars (norms, pivots, reflector coefficients)
// are computed redundantly and identically in every CTA from the same data
// in the same order, so no broadcast step is needed.
//
// Storage (inputs, reflectors, R, T, d, e) is FP64 in every case; the
// arithmetic type T is double for the FP64 path and float for the projected
// problems of the mixed path, whose entries come from FP32 blocks and carry
// FP32-level errors already (the FP64 Rayleigh-Ritz refinement that ends a
// mixed step solves its K x K problem with T = double).
//
//   k_tridiag_cl : Householder reduction to tridiagonal form (Alg. 1, first
//                  step of the eigensolve of H), two cluster barriers per
//                  column.
//   k_pchol_cl   : Cholesky with symmetric (diagonal) pivoting of a Gram
//                  matrix, with the drop rule of the orthonormalization
//                  (CholQR with pivoting), one cluster barrier per pivot.
//   k_trinv      : T = P R^{-1}, one warp per column (right-looking back
//                  substitution), spread over many SMs.
#include <cooperative_groups.h>
#include <float.h>

#include <mutex>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace grest {

namespace {

constexpr int kClThreads = 256;

// Fixed-order block sum (lane 0 of each warp, then warp 0); the result is
// returned to every thread.  Identical inputs give identical results in every
// CTA of the cluster.
template <typename T>
__device__ T cl_block_sum(T v, T* red, T* out) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if (lane == 0) red[wid] = v;
  __syncthreads();
  if (wid == 0) {
    T s = lane < nw ? red[lane] : T(0);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) *out = s;
  }
  __syncthreads();
  return *out;
}

// --- Householder tridiagonalization, rows cyclic over the cluster.
// Input: H (m x m, ld), only the upper triangle is read (mirrored).
// Output: d[0..m), e[0..m) (e[m-1] = 0), beta[0..m-2); the reflector of
// column j (v with v_0 = x_0 - alpha) is stored in row j of H right of the
// diagonal, as the back-transformation expects.
template <typename T>
__global__ void __launch_bounds__(kClThreads) k_tridiag_cl(double* H, int64_t ld, int m, double* d_out,
                                                           double* e_out, double* beta_out) {
  cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks(), r = (int)cl.block_rank();
  const int tid = threadIdx.x, nth = blockDim.x, lane = tid & 31, wid = tid >> 5, nw = nth >> 5;
  const int nl = (m + C - 1) / C;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  T* A = reinterpret_cast<T*>(sm_raw);  // nl x m: local row li is global row r + C li
  T* v = A + (size_t)nl * m;           // reflector (global column index)
  T* w = v + m;                        // p, then w = p - K v
  T* pl = w + m;                       // p_i of the owned rows
  __shared__ T red[32];
  __shared__ T bc[4];
  for (int li = wid; li < nl; li += nw) {
    const int i = r + C * li;
    if (i >= m) break;
    for (int l = lane; l < m; l += 32)
      A[(size_t)li * m + l] = (T)(i <= l ? H[(int64_t)i * ld + l] : H[(int64_t)l * ld + i]);
  }
  for (int j = 0; j + 2 < m; ++j) {
    cl.sync();  // row j final; every CTA done with the previous step's p
    const int o = j % C;
    const T* Aj = cl.map_shared_rank(A, o) + (size_t)(j / C) * m;
    T s = 0;
    for (int l = j + 1 + tid; l < m; l += nth) {
      const T x = Aj[l];
      v[l] = x;
      s = fma(x, x, s);
    }
    const T nrm2 = cl_block_sum(s, red, bc);
    if (tid == 0) {
      const T x0 = v[j + 1];
      T alpha = 0, beta = 0;
      if (nrm2 > T(0)) {
        if constexpr (sizeof(T) == sizeof(double)) {
          // FP64: reciprocal square root and Newton reciprocal (short latency
          // chains); nrm2 - alpha x0 = nrm2 + |x0| sqrt(nrm2) > 0
          alpha = -copysign(nrm2 * rsqrt(nrm2), x0);
          beta = rcp_newton(nrm2 - alpha * x0);
        } else {
          alpha = -copysign(sqrt(nrm2), x0);
          beta = T(1) / (nrm2 - alpha * x0);
        }
      }
      v[j + 1] = x0 - alpha;
      bc[1] = alpha;
      bc[2] = beta;
    }
    __syncthreads();
    const T beta = bc[2];
    if (r == o) {
      for (int l = j + 1 + tid; l < m; l += nth) H[(int64_t)j * ld + l] = (double)v[l];
      if (tid == 0) {
        d_out[j] = (double)A[(size_t)(j / C) * m + j];
        e_out[j] = (double)bc[1];
        beta_out[j] = (double)beta;
      }
    }
    if (beta == T(0)) continue;  // same decision in every CTA
    // p_i = beta (B v)_i for the owned rows i > j, one warp per row
    const int f = j + 1 - r;
    const int li0 = f <= 0 ? 0 : (f + C - 1) / C;
    for (int li = li0 + wid; li < nl; li += nw) {
      if (r + C * li >= m) break;
      const T* row = A + (size_t)li * m;
      T a = 0;
      for (int l = j + 1 + lane; l < m; l += 32) a = fma(row[l], v[l], a);
#pragma unroll
      for (int o2 = 16; o2 > 0; o2 >>= 1) a += __shfl_down_sync(0xffffffffu, a, o2);
      if (lane == 0) pl[li] = beta * a;
    }
    cl.sync();  // all p_i written
    T t = 0;
    for (int i = j + 1 + tid; i < m; i += nth) {
      const T pi = cl.map_shared_rank(pl, i % C)[i / C];
      w[i] = pi;
      t = fma(pi, v[i], t);
    }
    const T K = T(0.5) * beta * cl_block_sum(t, red, bc);
    for (int i = j + 1 + tid; i < m; i += nth) w[i] -= K * v[i];
    __syncthreads();
    // rank-2 update of the owned rows: B -= v w^T + w v^T
    for (int li = li0 + wid; li < nl; li += nw) {
      const int i = r + C * li;
      if (i >= m) break;
      T* row = A + (size_t)li * m;
      const T vi = v[i], wi = w[i];
      for (int l = j + 1 + lane; l < m; l += 32) row[l] -= vi * w[l] + wi * v[l];
    }
  }
  cl.sync();
  if (tid == 0) {
    if (m >= 2) {
      if ((m - 2) % C == r) {
        d_out[m - 2] = (double)A[(size_t)((m - 2) / C) * m + m - 2];
        e_out[m - 2] = (double)A[(size_t)((m - 2) / C) * m + m - 1];
      }
      if ((m - 1) % C == r) d_out[m - 1] = (double)A[(size_t)((m - 1) / C) * m + m - 1];
    } else if (r == 0) {
      d_out[0] = (double)A[0];
    }
    if (r == 0) e_out[m - 1] = 0.0;
  }
}

// Order-preserving integer image of a non-negative double (negative values,
// which cannot win a pivot search, map to -1).
__device__ __forceinline__ long long pivot_key(double x) { return x >= 0.0 ? __double_as_longlong(x) : -1ll; }

// Warp-wide (key, index) argmax, largest key and the lowest index among the
// lanes that hold it, in every lane: three redux.sync steps on the key's two
// halves and the index (exact, the same result as a shuffle tree).  Keys are
// >= -2 (no candidate: -2).
__device__ __forceinline__ void warp_argmax_key(long long& bk, int& bi) {
  const unsigned long long u = (unsigned long long)(bk + 2);
  const unsigned hi = (unsigned)(u >> 32), lo = (unsigned)u;
  const unsigned mhi = __reduce_max_sync(0xffffffffu, hi);
  const unsigned mlo = __reduce_max_sync(0xffffffffu, hi == mhi ? lo : 0u);
  const unsigned midx = __reduce_min_sync(0xffffffffu, (hi == mhi && lo == mlo) ? (unsigned)bi : 0xffffffffu);
  bk = (long long)(((unsigned long long)mhi << 32) | mlo) - 2;
  bi = (int)midx;
}

// --- Cholesky with diagonal pivoting of the Gram matrix G (c x c, upper
// triangle read), rows cyclic over the cluster.  Pivot k is the largest
// remaining Schur-complement diagonal (lowest index on ties); factorization
// stops at the first pivot with R_kk^2 <= drop_tol^2 max(R_00^2, abs_ref^2)
// (|abs_ref_ptr[0]| if given).  No rows are swapped: the Schur row of pivot
// k stays in its owner's shared memory and becomes row k of R.
// Output: Rt (in place of G): Rt[t][k] = R_{k,t} for k < t < rank and
// Rt[k][k] = 1 / R_kk (pivot order); piv[0..c) (kept pivots first, then the
// dropped indices ascending); info[0..3] = rank, kept_min, dropped_max, 0.
template <typename T>
__global__ void __launch_bounds__(kClThreads) k_pchol_cl(double* G, int64_t ld, int c, double drop_tol,
                                                         double abs_ref, const double* abs_ref_ptr, int* piv_out,
                                                         double* info) {
  cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks(), r = (int)cl.block_rank();
  const int tid = threadIdx.x, nth = blockDim.x, lane = tid & 31, wid = tid >> 5, nw = nth >> 5;
  const int nl = (c + C - 1) / C;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  T* A = reinterpret_cast<T*>(sm_raw);  // nl x c Schur rows (original index space)
  T* Rk = A + (size_t)nl * c;          // current row of R (original index space)
  T* rinv = Rk + c;                    // 1 / R_kk
  int* piv = reinterpret_cast<int*>(rinv + c);
  int* done = piv + c;                 // pivoted already
  __shared__ long long slot_key[2];
  __shared__ int slot_idx[2];
  __shared__ double s_ref, s_thr, s_vlast, s_vdrop;
  __shared__ T s_rinv;
  __shared__ int s_p, s_stop, s_rank;
  for (int li = wid; li < nl; li += nw) {
    const int i = r + C * li;
    if (i >= c) break;
    for (int l = lane; l < c; l += 32)
      A[(size_t)li * c + l] = (T)(i <= l ? G[(int64_t)i * ld + l] : G[(int64_t)l * ld + i]);
  }
  for (int l = tid; l < c; l += nth) done[l] = 0;
  if (tid == 0) {
    s_rank = c;
    s_vlast = 0.0;
    s_vdrop = 0.0;
  }
  __syncthreads();
  for (int k = 0; k < c; ++k) {
    // local candidate: largest diagonal of the owned, not yet pivoted rows
    if (wid == 0) {
      long long bk = -2;
      int bi = c;
      for (int li = lane; li < nl; li += 32) {
        const int i = r + C * li;
        if (i < c && !done[i]) {
          const long long key = pivot_key((double)A[(size_t)li * c + i]);
          if (key > bk || (key == bk && i < bi)) { bk = key; bi = i; }
        }
      }
      warp_argmax_key(bk, bi);
      if (lane == 0) {
        slot_key[k & 1] = bk;
        slot_idx[k & 1] = bi;
      }
    }
    cl.sync();  // candidates posted; the previous step's updates are complete
    if (wid == 0) {
      long long bk = -2;
      int bi = c;
      if (lane < C) {
        bk = cl.map_shared_rank(slot_key, lane)[k & 1];
        bi = cl.map_shared_rank(slot_idx, lane)[k & 1];
      }
      warp_argmax_key(bk, bi);
      if (lane == 0) {
        const double v = bk >= 0 ? __longlong_as_double(bk) : -1.0;  // exact value of the pivot
        if (k == 0) {
          const double a = abs_ref_ptr ? fabs(*abs_ref_ptr) : abs_ref;
          s_ref = fmax(v, a * a);
          s_thr = drop_tol * drop_tol * s_ref;
        }
        if (bi >= c || !(v > 0.0) || !(v > s_thr) || !isfinite(v)) {
          s_stop = 1;
          s_rank = k;
          s_vdrop = v > 0.0 ? v : 0.0;
        } else {
          s_stop = 0;
          T ri;
          if constexpr (sizeof(T) == sizeof(double)) ri = rsqrt(v);  // one short FP64 chain
          else ri = T(1) / sqrt((T)v);
          s_rinv = ri;
          s_vlast = v;
          s_p = bi;
          piv[k] = bi;
          rinv[k] = ri;
          done[bi] = 1;
        }
      }
    }
    __syncthreads();
    if (s_stop) break;  // same decision in every CTA
    const int p = s_p;
    const T ri = s_rinv;
    const T* Ap = cl.map_shared_rank(A, p % C) + (size_t)(p / C) * c;
    for (int l = tid; l < c; l += nth) Rk[l] = done[l] ? T(0) : Ap[l] * ri;
    __syncthreads();
    // Schur update of the owned rows that are not pivoted yet
    for (int li = wid; li < nl; li += nw) {
      const int i = r + C * li;
      if (i >= c) break;
      if (done[i]) continue;
      const T rki = Rk[i];
      T* row = A + (size_t)li * c;
      for (int l = lane; l < c; l += 32) row[l] = fma(-rki, Rk[l], row[l]);
    }
    __syncthreads();
  }
  cl.sync();  // no CTA leaves while its rows may still be read
  const int rk = s_rank;
  // dropped indices (ascending) complete the permutation
  if (tid == 0) {
    int t = rk;
    for (int l = 0; l < c; ++l)
      if (!done[l]) piv[t++] = l;
  }
  __syncthreads();
  // Rt[t][k] = R_{k,t} = S_k[piv[t]] / R_kk for the rows k this CTA owns
  for (int k = 0; k < rk; ++k) {
    const int p = piv[k];
    if (p % C != r) continue;
    const T* Sk = A + (size_t)(p / C) * c;
    for (int t = k + tid; t < rk; t += nth)
      G[(int64_t)t * ld + k] = (double)(t == k ? rinv[k] : Sk[piv[t]] * rinv[k]);
  }
  if (r == 0) {
    for (int l = tid; l < c; l += nth) piv_out[l] = piv[l];
    if (tid == 0) {
      const double ref = s_ref;
      info[0] = rk;
      info[1] = (rk > 0 && ref > 0.0) ? sqrt(s_vlast / ref) : 0.0;  // last kept pivot / reference
      info[2] = (ref > 0.0 && s_vdrop > 0.0) ? sqrt(s_vdrop / ref) : 0.0;
      info[3] = 0.0;
    }
  }
}

// --- T = P R^{-1} (c x c, zero columns >= rank): warp j solves R x = e_j by
// a right-looking back substitution, x_j = 1/R_jj, and for t = j..1 the
// partial sums s_i += R_{i,t} x_t (i < t) give x_{t-1} = -s_{t-1} / R_{t-1,t-1}.
// Rt holds R transposed with reciprocal diagonal (k_pchol_cl).
constexpr int kTrinvWarps = 4;

template <typename T>
__global__ void __launch_bounds__(kTrinvWarps * 32) k_trinv(const double* Rt, int64_t ld, const int* piv,
                                                            const double* info, int c, double* Tm, int64_t ldt) {
  extern __shared__ __align__(16) unsigned char xs_raw[];  // kTrinvWarps x c
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int j = blockIdx.x * kTrinvWarps + wid;
  if (j >= c) return;
  const int rk = (int)info[0];
  if (j >= rk) {
    for (int i = lane; i < c; i += 32) Tm[(int64_t)i * ldt + j] = 0.0;
    return;
  }
  T* s = reinterpret_cast<T*>(xs_raw) + (size_t)wid * c;
  for (int i = lane; i < j; i += 32) s[i] = 0;
  T xt = (T)Rt[(int64_t)j * ld + j];
  if (lane == 0) s[j] = xt;
  __syncwarp();
  for (int t = j; t >= 1; --t) {
    const double* col = Rt + (int64_t)t * ld;  // col[i] = R_{i,t}, i < t
    for (int i = lane; i < t; i += 32) s[i] = fma((T)col[i], xt, s[i]);
    __syncwarp();
    xt = -s[t - 1] * (T)Rt[(int64_t)(t - 1) * ld + (t - 1)];
    __syncwarp();
    if (lane == 0) s[t - 1] = xt;
    __syncwarp();
  }
  for (int i = lane; i < c; i += 32) Tm[(int64_t)piv[i] * ldt + j] = i <= j ? (double)s[i] : 0.0;
}

// True when `kern` can be launched as one cluster of C CTAs with `smem` bytes
// of dynamic shared memory each (answers are cached per kernel, size, C).
template <typename K>
bool cluster_ok(K kern, size_t smem, int C) {
  struct Entry {
    const void* k;
    size_t smem;
    int C;
    bool ok;
  };
  static Entry cache[128];
  static int n_cache = 0;
  static std::mutex mu;  // contexts may step concurrently (grest_batch_apply_updates)
  std::lock_guard<std::mutex> lock(mu);
  for (int i = 0; i < n_cache; ++i)
    if (cache[i].k == (const void*)kern && cache[i].smem == smem && cache[i].C == C) return cache[i].ok;
  bool ok = false;
  int dev = 0, optin = 0;
  cudaFuncAttributes fa;
  if (cudaGetDevice(&dev) == cudaSuccess &&
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) == cudaSuccess &&
      cudaFuncGetAttributes(&fa, kern) == cudaSuccess && smem + fa.sharedSizeBytes <= (size_t)optin &&
      reserve_dynamic_smem(kern, smem) &&
      (C <= 8 || cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess)) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C);
    cfg.blockDim = dim3(kClThreads);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int n = 0;
    ok = cudaOccupancyMaxActiveClusters(&n, kern, &cfg) == cudaSuccess && n > 0;
  }
  cudaGetLastError();
  if (n_cache < 128) cache[n_cache++] = Entry{(const void*)kern, smem, C, ok};
  return ok;
}

template <typename K, typename... Args>
bool launch_cl(K kern, int C, size_t smem, cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C);
  cfg.blockDim = dim3(kClThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  if (cudaLaunchKernelEx(&cfg, kern, args...) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return true;
}

int want_cluster(int m) { return m >= 96 ? 16 : 8; }

template <typename T>
bool tridiag_cluster_t(double* H, int64_t ld, int m, double* d, double* e, double* beta, cudaStream_t s) {
  for (int C = want_cluster(m); C >= 2; C >>= 1) {
    const int nl = (m + C - 1) / C;
    const size_t smem = sizeof(T) * ((size_t)nl * m + 2 * (size_t)m + nl);
    if (!cluster_ok(k_tridiag_cl<T>, smem, C)) continue;
    if (launch_cl(k_tridiag_cl<T>, C, smem, s, H, ld, m, d, e, beta)) return true;
  }
  return false;
}

template <typename T>
bool pchol_cluster_t(double* G, int64_t ldg, int c, double drop_tol, double abs_ref, const double* abs_ref_ptr,
                     double* Tm, int64_t ldt, int* piv, double* info, cudaStream_t s) {
  const size_t tsmem = sizeof(T) * kTrinvWarps * (size_t)c;
  if (!reserve_dynamic_smem(k_trinv<T>, tsmem)) return false;
  for (int C = want_cluster(c); C >= 2; C >>= 1) {
    const int nl = (c + C - 1) / C;
    const size_t smem = sizeof(T) * ((size_t)nl * c + 2 * (size_t)c) + sizeof(int) * 2 * (size_t)c;
    if (!cluster_ok(k_pchol_cl<T>, smem, C)) continue;
    if (!launch_cl(k_pchol_cl<T>, C, smem, s, G, ldg, c, drop_tol, abs_ref, abs_ref_ptr, piv, info)) continue;
    k_trinv<T><<<(unsigned)((c + kTrinvWarps - 1) / kTrinvWarps), kTrinvWarps * 32, tsmem, s>>>(G, ldg, piv, info,
                                                                                                  c, Tm, ldt);
    return true;
  }
  return false;
}

}  // namespace

bool tridiag_cluster(double* H, int64_t ld, int m, double* d, double* e, double* beta, bool f32, cudaStream_t s) {
  if (m < 1) return true;
  return f32 ? tridiag_cluster_t<float>(H, ld, m, d, e, beta, s) : tridiag_cluster_t<double>(H, ld, m, d, e, beta, s);
}

bool pchol_cluster(double* G, int64_t ldg, int c, double drop_tol, double abs_ref, const double* abs_ref_ptr,
                   double* Tm, int64_t ldt, int* piv, double* info, bool f32, cudaStream_t s) {
  if (c < 1) return false;
  return f32 ? pchol_cluster_t<float>(G, ldg, c, drop_tol, abs_ref, abs_ref_ptr, Tm, ldt, piv, info, s)
             : pchol_cluster_t<double>(G, ldg, c, drop_tol, abs_ref, abs_ref_ptr, Tm, ldt, piv, info, s);
}

}  // namespace grest
