// Downstream task of Sec. 5, with the matrix-function tracking of Sec. 4.1:
// approximate subgraph centrality from the tracked pairs,
// exp(M) 1 ~= X_K exp(Lambda_K) X_K^T 1, and the J most central nodes.
//
//   s = X_K^T 1                      column sums over live rows (fixed-order reduction)
//   w_j = exp(theta_j - theta_max) s_j
//   c_i = sum_j X_ij w_j             = exp(-theta_max) (X_K exp(Lambda_K) X_K^T 1)_i
//
// The common factor exp(-theta_max) keeps every term finite for any spectrum
// and leaves the ranking unchanged.  The top-J set is found by an 8-pass
// radix select on order-preserving 64-bit keys of c, ties at the threshold
// broken towards lower node ids (an exclusive scan ranks them), and the J
// winners are sorted in one CTA by (c descending, id ascending), so the
// result is unique and independent of launch order.
#include <float.h>

#include <algorithm>

#include "common.cuh"

namespace grest {
namespace {

constexpr int kCentBlocks = 608;     // 4 CTAs per SM
constexpr int kMaxTopJ = 4096;

struct CentState {
  unsigned long long prefix;  // key bits fixed so far
  long long remaining;        // winners still to find at or below the prefix
  long long n_live;
  unsigned int hist[256];
};

__device__ __forceinline__ unsigned long long order_key(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

__device__ __forceinline__ double key_value(unsigned long long k) {
  const unsigned long long b = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
  return __longlong_as_double((long long)b);
}

// per-CTA column sums of the live rows (K <= 64): part[blockIdx.x * K + j]
__global__ void k_colsum_part(const double* __restrict__ X, int64_t ldx, int K, const uint8_t* __restrict__ live,
                              int64_t n, double* __restrict__ part) {
  __shared__ double red[8][64];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double a0 = 0.0, a1 = 0.0;
  for (int64_t i = blockIdx.x * 8ll + warp; i < n; i += (int64_t)gridDim.x * 8) {
    if (!live[i]) continue;
    const double* r = X + i * ldx;
    if (lane < K) a0 += r[lane];
    if (lane + 32 < K) a1 += r[lane + 32];
  }
  red[warp][lane] = a0;
  red[warp][lane + 32] = a1;
  __syncthreads();
  if (threadIdx.x < K) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w][threadIdx.x];
    part[(int64_t)blockIdx.x * K + threadIdx.x] = t;
  }
}

// w_j = exp(theta_j - theta_max) * sum_b part[b][j]; resets the live count
__global__ void k_colsum_final(const double* __restrict__ part, int nb, int K, const double* __restrict__ theta,
                               double* __restrict__ wv, CentState* st) {
  __shared__ double tmax;
  if (threadIdx.x == 0) {
    double m = -DBL_MAX;
    for (int j = 0; j < K; ++j) m = fmax(m, theta[j]);
    tmax = m;
    st->n_live = 0;
  }
  __syncthreads();
  if (threadIdx.x < K) {
    double t = 0.0;
    for (int b = 0; b < nb; ++b) t += part[(int64_t)b * K + threadIdx.x];
    wv[threadIdx.x] = exp(theta[threadIdx.x] - tmax) * t;
  }
}

// c_i (0 for removed nodes) and its order key (0 for removed nodes, below any value)
__global__ void k_cent(const double* __restrict__ X, int64_t ldx, int K, const uint8_t* __restrict__ live,
                       int64_t n, const double* __restrict__ wv, double* __restrict__ cent,
                       unsigned long long* __restrict__ key, CentState* st, int32_t* err) {
  __shared__ double w[64];
  if (threadIdx.x < K) w[threadIdx.x] = wv[threadIdx.x];
  __syncthreads();
  long long cnt = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double v = 0.0;
    unsigned long long k = 0ull;
    if (live[i]) {
      const double* r = X + i * ldx;
      for (int j = 0; j < K; ++j) v = fma(r[j], w[j], v);
      if (v == 0.0) v = 0.0;  // one key for +0 and -0
      if (v != v) {
        set_err(err, DERR_NUMERIC);
        v = 0.0;
      }
      k = order_key(v);
      ++cnt;
    }
    cent[i] = v;
    key[i] = k;
  }
  for (int o = 16; o; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  if ((threadIdx.x & 31) == 0 && cnt) atomicAdd((unsigned long long*)&st->n_live, (unsigned long long)cnt);
}

__global__ void k_select_init(CentState* st, int J, unsigned int* counter) {
  if (threadIdx.x == 0) {
    st->prefix = 0ull;
    st->remaining = J;
    *counter = 0u;
  }
  for (int t = threadIdx.x; t < 256; t += blockDim.x) st->hist[t] = 0u;
}

// histogram of digit `pass` (bits 8 pass .. 8 pass + 7) over keys matching the prefix above it
__global__ void k_radix_hist(const unsigned long long* __restrict__ key, int64_t n, int pass, CentState* st) {
  __shared__ unsigned int h[256];
  for (int t = threadIdx.x; t < 256; t += blockDim.x) h[t] = 0u;
  __syncthreads();
  const int sh = 8 * pass;
  const unsigned long long hi_mask = pass == 7 ? 0ull : (~0ull << (sh + 8));
  const unsigned long long want = st->prefix & hi_mask;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long k = key[i];
    if ((k & hi_mask) == want) atomicAdd(&h[(k >> sh) & 255u], 1u);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < 256; t += blockDim.x)
    if (h[t]) atomicAdd(&st->hist[t], h[t]);
}

// fix digit `pass`: the largest digit d with (keys above d) < remaining
__global__ void k_radix_pick(int pass, CentState* st) {
  if (threadIdx.x == 0) {
    long long above = 0;
    const long long rem = st->remaining;
    int d = 255;
    for (; d > 0; --d) {
      const long long hd = st->hist[d];
      if (above + hd >= rem) break;
      above += hd;
    }
    st->prefix |= (unsigned long long)d << (8 * pass);
    st->remaining = rem - above;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < 256; t += blockDim.x) st->hist[t] = 0u;
}

__global__ void k_tie_flags(const unsigned long long* __restrict__ key, int64_t n, const CentState* st,
                            int64_t* __restrict__ flag) {
  const unsigned long long T = st->prefix;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    flag[i] = key[i] == T ? 1 : 0;
}

// winners: every key above the threshold (in any order), then the `remaining`
// lowest-id keys equal to it
__global__ void k_collect(const unsigned long long* __restrict__ key, int64_t n, const CentState* st,
                          const int64_t* __restrict__ tie_rank, int J, unsigned int* counter,
                          unsigned long long* __restrict__ sel_key, int32_t* __restrict__ sel_id) {
  const unsigned long long T = st->prefix;
  const long long r = st->remaining;
  const long long g = J - r;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long k = key[i];
    long long slot = -1;
    if (k > T) {
      slot = atomicAdd(counter, 1u);
      if (slot >= g) slot = -1;  // cannot happen for a consistent select; keeps the store in range
    } else if (k == T && tie_rank[i] < r) {
      slot = g + tie_rank[i];
    }
    if (slot >= 0) {
      sel_key[slot] = k;
      sel_id[slot] = (int32_t)i;
    }
  }
}

// one CTA: bitonic sort of the J winners by (key descending, id ascending)
__global__ void k_top_sort(const unsigned long long* __restrict__ sel_key, const int32_t* __restrict__ sel_id, int J,
                           int P, int32_t* __restrict__ top_ids, double* __restrict__ top_vals) {
  extern __shared__ unsigned long long sk[];
  int32_t* sid = reinterpret_cast<int32_t*>(sk + P);
  for (int t = threadIdx.x; t < P; t += blockDim.x) {
    sk[t] = t < J ? sel_key[t] : 0ull;
    sid[t] = t < J ? sel_id[t] : 0x7fffffff;
  }
  __syncthreads();
  for (int len = 2; len <= P; len <<= 1) {
    for (int stride = len >> 1; stride > 0; stride >>= 1) {
      for (int t = threadIdx.x; t < P; t += blockDim.x) {
        const int u = t ^ stride;
        if (u > t) {
          // "before" = larger key, then smaller id
          const bool t_first = sk[t] > sk[u] || (sk[t] == sk[u] && sid[t] < sid[u]);
          const bool desc = (t & len) == 0;
          if (t_first != desc) {
            const unsigned long long kk = sk[t];
            sk[t] = sk[u];
            sk[u] = kk;
            const int32_t ii = sid[t];
            sid[t] = sid[u];
            sid[u] = ii;
          }
        }
      }
      __syncthreads();
    }
  }
  for (int t = threadIdx.x; t < J; t += blockDim.x) {
    if (top_ids) top_ids[t] = sid[t];
    if (top_vals) top_vals[t] = key_value(sk[t]);
  }
}

struct CentLayout {
  double* part;
  double* wv;
  CentState* st;
  unsigned long long* key;
  int64_t* flag;  // n + 1
  unsigned long long* sel_key;
  int32_t* sel_id;
  unsigned int* counter;
  void* scan_tmp;
};

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

CentLayout cent_layout(void* work, int64_t n) {
  char* p = static_cast<char*>(work);
  CentLayout L;
  L.part = reinterpret_cast<double*>(p);
  p += align256(sizeof(double) * kCentBlocks * 64);
  L.wv = reinterpret_cast<double*>(p);
  p += align256(sizeof(double) * 64);
  L.st = reinterpret_cast<CentState*>(p);
  p += align256(sizeof(CentState));
  L.key = reinterpret_cast<unsigned long long*>(p);
  p += align256(sizeof(unsigned long long) * (size_t)n);
  L.flag = reinterpret_cast<int64_t*>(p);
  p += align256(sizeof(int64_t) * (size_t)(n + 1));
  L.sel_key = reinterpret_cast<unsigned long long*>(p);
  p += align256(sizeof(unsigned long long) * kMaxTopJ);
  L.sel_id = reinterpret_cast<int32_t*>(p);
  p += align256(sizeof(int32_t) * kMaxTopJ);
  L.counter = reinterpret_cast<unsigned int*>(p);
  p += 256;
  L.scan_tmp = p;
  return L;
}

}  // namespace

int central_max_j() { return kMaxTopJ; }

size_t central_work_bytes(int64_t n) {
  return align256(sizeof(double) * kCentBlocks * 64) + align256(sizeof(double) * 64) + align256(sizeof(CentState)) +
         align256(sizeof(unsigned long long) * (size_t)n) + align256(sizeof(int64_t) * (size_t)(n + 1)) +
         align256(sizeof(unsigned long long) * kMaxTopJ) + align256(sizeof(int32_t) * kMaxTopJ) + 256 +
         align256(scan_temp_bytes(n + 1));
}

int central_values(const double* X, int64_t ldx, int K, const double* theta, const uint8_t* live, int64_t n,
                   double* cent, void* work, int64_t* n_live_host, int32_t* err, cudaStream_t s) {
  CentLayout L = cent_layout(work, n);
  const int nb = (int)std::min<int64_t>(kCentBlocks, std::max<int64_t>(1, (n + 7) / 8));
  k_colsum_part<<<nb, 256, 0, s>>>(X, ldx, K, live, n, L.part);
  k_colsum_final<<<1, 256, 0, s>>>(L.part, nb, K, theta, L.wv, L.st);
  const unsigned g = (unsigned)std::min<int64_t>(kCentBlocks, std::max<int64_t>(1, (n + 255) / 256));
  k_cent<<<g, 256, 0, s>>>(X, ldx, K, live, n, L.wv, cent, L.key, L.st, err);
  cudaMemcpyAsync(n_live_host, &L.st->n_live, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
  return 3;
}

int central_top(int64_t n, int J, int32_t* top_ids, double* top_vals, void* work, cudaStream_t s) {
  CentLayout L = cent_layout(work, n);
  const unsigned g = (unsigned)std::min<int64_t>(kCentBlocks, std::max<int64_t>(1, (n + 255) / 256));
  k_select_init<<<1, 256, 0, s>>>(L.st, J, L.counter);
  int launches = 1;
  for (int pass = 7; pass >= 0; --pass) {
    k_radix_hist<<<g, 256, 0, s>>>(L.key, n, pass, L.st);
    k_radix_pick<<<1, 256, 0, s>>>(pass, L.st);
    launches += 2;
  }
  k_tie_flags<<<g, 256, 0, s>>>(L.key, n, L.st, L.flag);
  launches += 1 + exclusive_scan_i64(L.flag, L.flag, n, L.scan_tmp, s);
  k_collect<<<g, 256, 0, s>>>(L.key, n, L.st, L.flag, J, L.counter, L.sel_key, L.sel_id);
  int P = 1;
  while (P < J) P <<= 1;
  const size_t smem = (size_t)P * (sizeof(unsigned long long) + sizeof(int32_t));
  reserve_dynamic_smem(k_top_sort, smem);
  k_top_sort<<<1, 1024, smem, s>>>(L.sel_key, L.sel_id, J, P, top_ids, top_vals);
  return launches + 2;
}

}  // namespace grest
