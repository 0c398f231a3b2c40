// In-place update of the device slack-CSR by one batch Delta (Eq. adj_update,
// Sec. 2): +1 / -1 entries of K, the new-node blocks G and C, and node
// removal (tombstones).  Every row touched by the batch is rebuilt as a
// sorted merge of its old entries and its batch entries:
//
//   count    per-row number of batch entries (both directions of each edge)
//   scan     segment offsets; compact list of touched rows; staging offsets
//   scatter  batch entries into per-row segments
//   sort     each segment by (column, tag)           -> duplicate check
//   merge    old row (-) deletions (+) insertions     -> existence checks
//   alloc    rows that outgrow their slot get space at the arena top
//   commit   staged rows copied into place, degrees refreshed
//
// Validation finishes before commit; every state-changing kernel returns at
// once when the error word is set, so a rejected batch changes nothing.
#include <algorithm>

#include "common.cuh"

namespace grest {

namespace {

constexpr uint64_t kTagDel = 1, kTagNdel = 2, kTagIns = 3;
constexpr int kSortSmem = 2048;  // segment length sorted in shared memory

__device__ __forceinline__ uint64_t make_key(int32_t col, uint64_t tag, int64_t idx) {
  return ((uint64_t)(uint32_t)col << 33) | (tag << 31) | (uint64_t)(idx & 0x7fffffff);
}
__device__ __forceinline__ int32_t key_col(uint64_t k) { return (int32_t)(k >> 33); }
__device__ __forceinline__ uint64_t key_tag(uint64_t k) { return (k >> 31) & 3u; }
__device__ __forceinline__ int64_t key_idx(uint64_t k) { return (int64_t)(k & 0x7fffffff); }

__device__ __forceinline__ bool bad_weight(double w) { return !(w > 0.0) || !isfinite(w); }

// --- node removal: marks, range / duplicate / liveness checks
__global__ void k_mark_removed(const int32_t* dn, int64_t n_dn, int64_t N, const uint8_t* live, int32_t* mark,
                               uint8_t* delflag, int32_t* err) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_dn; i += (int64_t)gridDim.x * blockDim.x) {
    int32_t d = dn[i];
    if (d < 0 || d >= N) { set_err(err, DERR_NODE); continue; }
    if (atomicAdd(&mark[d], 1) != 0) { set_err(err, DERR_NODE); continue; }
    if (!live[d]) { set_err(err, DERR_NODE); continue; }
    delflag[d] = 1;
  }
}

__device__ __forceinline__ bool node_ok(int32_t x, int64_t N, const uint8_t* live, const uint8_t* delflag) {
  return !((x < N && !live[x]) || delflag[x]);
}

// --- count both directions of every edge edit
__global__ void k_count_edges(const int32_t* u, const int32_t* v, const double* w, int64_t ne, int64_t lim,
                              int64_t N, const uint8_t* live, const uint8_t* delflag, int32_t* cnt, int32_t* err) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ne; i += (int64_t)gridDim.x * blockDim.x) {
    int32_t a = u[i], b = v[i];
    if (a < 0 || b < 0 || a >= lim || b >= lim) { set_err(err, DERR_RANGE); continue; }
    if (a == b) { set_err(err, DERR_SELF); continue; }
    if (!node_ok(a, N, live, delflag) || !node_ok(b, N, live, delflag)) { set_err(err, DERR_DEAD); continue; }
    if (w && bad_weight(w[i])) { set_err(err, DERR_WEIGHT); continue; }
    atomicAdd(&cnt[a], 1);
    atomicAdd(&cnt[b], 1);
  }
}

// --- every neighbour x of a removed node d gets an entry (x, d) to delete
__global__ void k_count_removed(const int32_t* dn, int64_t n_dn, const int64_t* row_off, const int32_t* row_len,
                                const int32_t* col, int32_t* cnt, const int32_t* err) {
  if (*err) return;
  for (int64_t i = blockIdx.x; i < n_dn; i += gridDim.x) {
    int32_t d = dn[i];
    const int32_t* c = col + row_off[d];
    for (int j = threadIdx.x; j < row_len[d]; j += blockDim.x) atomicAdd(&cnt[c[j]], 1);
  }
}

__global__ void k_init_new_rows(int64_t N, int64_t N2, int64_t* row_off, int32_t* row_len, int32_t* row_cap) {
  int64_t r = N + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r < N2) { row_off[r] = 0; row_len[r] = 0; row_cap[r] = 0; }
}

__global__ void k_cnt_to_i64(const int32_t* cnt, int64_t* out, int64_t n) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) out[i] = cnt[i];
}

// touched = rows with batch entries or removed; staging size old_len + cnt
__global__ void k_touch_flags(const int32_t* cnt, const uint8_t* delflag, const int32_t* row_len, int64_t n,
                              int64_t* flag, int64_t* tmpsz) {
  int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r < n) {
    bool t = cnt[r] > 0 || delflag[r];
    flag[r] = t ? 1 : 0;
    tmpsz[r] = t ? (int64_t)row_len[r] + cnt[r] : 0;
  }
}

__global__ void k_compact(const int64_t* flag_scan, int64_t n, int32_t* list, int64_t* count_out) {
  int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r < n && flag_scan[r + 1] != flag_scan[r]) list[flag_scan[r]] = (int32_t)r;
  if (r == 0) *count_out = flag_scan[n];
}

__global__ void k_check_sizes(const int64_t* seg, const int64_t* tmp_off, int64_t n, int64_t ent_cap,
                              int64_t tmp_cap, int32_t* err) {
  if (seg[n] > ent_cap || tmp_off[n] > tmp_cap) set_err(err, DERR_CAPACITY);
}

// --- scatter entries into their row segments (unordered within a segment)
__global__ void k_scatter_edges(const int32_t* u, const int32_t* v, const double* w, int64_t ne, uint64_t tag,
                                const int64_t* seg, int32_t* cursor, uint64_t* ekey, double* ew, const int32_t* err) {
  if (*err) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ne; i += (int64_t)gridDim.x * blockDim.x) {
    int32_t a = u[i], b = v[i];
    double wt = w ? w[i] : 1.0;
    int64_t p = atomicAdd(&cursor[a], 1);
    ekey[seg[a] + p] = make_key(b, tag, p);
    ew[seg[a] + p] = wt;
    p = atomicAdd(&cursor[b], 1);
    ekey[seg[b] + p] = make_key(a, tag, p);
    ew[seg[b] + p] = wt;
  }
}

__global__ void k_scatter_removed(const int32_t* dn, int64_t n_dn, const int64_t* row_off, const int32_t* row_len,
                                  const int32_t* col, const int64_t* seg, int32_t* cursor, uint64_t* ekey, double* ew,
                                  const int32_t* err) {
  if (*err) return;
  for (int64_t i = blockIdx.x; i < n_dn; i += gridDim.x) {
    int32_t d = dn[i];
    const int32_t* c = col + row_off[d];
    for (int j = threadIdx.x; j < row_len[d]; j += blockDim.x) {
      int32_t x = c[j];
      int64_t p = atomicAdd(&cursor[x], 1);
      ekey[seg[x] + p] = make_key(d, kTagNdel, p);
      ew[seg[x] + p] = 0.0;
    }
  }
}

// Ascending sort of keys[0, len) by a bitonic network whose merge steps all
// sort ascending (reversal compare, then half-cleaners).  Indices >= len act
// as +infinity and are never touched, so len need not be a power of two.
__device__ void block_sort_u64(uint64_t* keys, int64_t len) {
  int64_t np2 = 1;
  while (np2 < len) np2 <<= 1;
  for (int64_t k = 2; k <= np2; k <<= 1) {
    int64_t h = k >> 1;
    for (int64_t t = threadIdx.x; t < np2 / 2; t += blockDim.x) {
      int64_t blk = t / h, off = t % h;
      int64_t a = blk * k + off, b = blk * k + k - 1 - off;
      if (b < len) {
        uint64_t x = keys[a], y = keys[b];
        if (x > y) { keys[a] = y; keys[b] = x; }
      }
    }
    __syncthreads();
    for (int64_t j = h >> 1; j >= 1; j >>= 1) {
      for (int64_t t = threadIdx.x; t < np2 / 2; t += blockDim.x) {
        int64_t blk = t / j, off = t % j;
        int64_t a = blk * 2 * j + off, b = a + j;
        if (b < len) {
          uint64_t x = keys[a], y = keys[b];
          if (x > y) { keys[a] = y; keys[b] = x; }
        }
      }
      __syncthreads();
    }
  }
}

// Block-wide inclusive scan helper over blockDim (<= 1024) int values.
__device__ int block_scan_excl_int(int v, int* total) {
  __shared__ int ws[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  int inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) ws[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    int t = lane < nw ? ws[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int u = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += u;
    }
    if (lane < nw) ws[lane] = t;
  }
  __syncthreads();
  int before = wid ? ws[wid - 1] : 0;
  *total = ws[nw - 1];
  __syncthreads();
  return before + inc - v;
}

// --- sort each touched segment; prefix count of inserts; duplicate check
__global__ void __launch_bounds__(256) k_sort_segments(const int32_t* touched, const int64_t* n_touched,
                                                        const int64_t* seg, uint64_t* ekey, int32_t* eins,
                                                        int32_t* err) {
  if (*err) return;
  __shared__ uint64_t sk[kSortSmem];
  const int64_t nt = *n_touched;
  for (int64_t t = blockIdx.x; t < nt; t += gridDim.x) {
    const int32_t r = touched[t];
    const int64_t s0 = seg[r], len = seg[r + 1] - s0;
    if (len == 0) continue;
    uint64_t* keys;
    if (len <= kSortSmem) {
      for (int64_t i = threadIdx.x; i < len; i += blockDim.x) sk[i] = ekey[s0 + i];
      __syncthreads();
      keys = sk;
    } else {
      keys = ekey + s0;
    }
    block_sort_u64(keys, len);
    // prefix count of inserts and duplicate check, in chunks of blockDim
    int carry = 0;
    for (int64_t c0 = 0; c0 < len; c0 += blockDim.x) {
      int64_t i = c0 + threadIdx.x;
      uint64_t k = i < len ? keys[i] : 0;
      int isins = (i < len && key_tag(k) == kTagIns) ? 1 : 0;
      if (i < len && i > 0 && key_col(keys[i - 1]) == key_col(k)) set_err(err, DERR_DUP);
      int tot;
      int ex = block_scan_excl_int(isins, &tot);
      if (i < len) eins[s0 + i] = carry + ex;
      carry += tot;
    }
    if (len <= kSortSmem)
      for (int64_t i = threadIdx.x; i < len; i += blockDim.x) ekey[s0 + i] = sk[i];
    __syncthreads();
  }
}

__device__ __forceinline__ int64_t lower_bound_col(const int32_t* a, int64_t n, int32_t c) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if (a[mid] < c) lo = mid + 1; else hi = mid;
  }
  return lo;
}
__device__ __forceinline__ int64_t lower_bound_key(const uint64_t* a, int64_t n, int32_t c) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if (key_col(a[mid]) < c) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// --- merge: old row minus deletions plus insertions, into the staging area
__global__ void __launch_bounds__(256) k_merge_rows(const int32_t* touched, const int64_t* n_touched,
                                                     const int64_t* seg, const uint64_t* ekey, const double* ew,
                                                     const int32_t* eins, const uint8_t* delflag, const int64_t* row_off,
                                                     const int32_t* row_len, const int32_t* col, const double* val,
                                                     const int64_t* tmp_off, int32_t* tmp_col, double* tmp_val,
                                                     int32_t* new_len, double* edel, int32_t* err) {
  if (*err) return;
  const int64_t nt = *n_touched;
  for (int64_t t = blockIdx.x; t < nt; t += gridDim.x) {
    const int32_t r = touched[t];
    const int64_t s0 = seg[r], L = seg[r + 1] - s0;
    const uint64_t* K = ekey + s0;
    const int32_t* P = eins + s0;
    const int32_t* old = col + row_off[r];
    const int64_t olen = row_len[r];
    const int64_t nins = L ? (int64_t)P[L - 1] + (key_tag(K[L - 1]) == kTagIns ? 1 : 0) : 0;
    const bool drop_row = delflag[r] != 0;
    if (threadIdx.x == 0) new_len[r] = drop_row ? 0 : (int32_t)(olen - (L - nins) + nins);
    // existence checks for the batch entries
    for (int64_t i = threadIdx.x; i < L; i += blockDim.x) {
      uint64_t k = K[i];
      int32_t c = key_col(k);
      int64_t p = lower_bound_col(old, olen, c);
      bool ex = p < olen && old[p] == c;
      if (key_tag(k) == kTagIns) {
        if (ex) set_err(err, DERR_EXISTS);
      } else if (!ex) {
        set_err(err, DERR_MISSING);
      }
    }
    if (drop_row) continue;
    int32_t* oc = tmp_col + tmp_off[r];
    double* ov = tmp_val ? tmp_val + tmp_off[r] : nullptr;
    const double* oldv = val ? val + row_off[r] : nullptr;
    for (int64_t j = threadIdx.x; j < olen; j += blockDim.x) {
      int32_t c = old[j];
      int64_t l = lower_bound_key(K, L, c);
      if (l < L && key_col(K[l]) == c && key_tag(K[l]) != kTagIns) {  // deleted: keep its old weight
        edel[s0 + l] = oldv ? oldv[j] : 1.0;
        continue;
      }
      int64_t ins_before = l < L ? P[l] : nins;
      int64_t del_before = l - ins_before;
      int64_t pos = j - del_before + ins_before;
      if (pos < 0 || pos >= olen + L) continue;  // only reachable by an invalid batch (error already set)
      oc[pos] = c;
      if (ov) ov[pos] = oldv[j];
    }
    for (int64_t i = threadIdx.x; i < L; i += blockDim.x) {
      uint64_t k = K[i];
      if (key_tag(k) != kTagIns) continue;
      int32_t c = key_col(k);
      int64_t lb = lower_bound_col(old, olen, c);
      int64_t del_before = i - P[i];
      int64_t pos = P[i] + lb - del_before;
      if (pos < 0 || pos >= olen + L) continue;
      oc[pos] = c;
      if (ov) ov[pos] = ew[s0 + key_idx(k)];
    }
  }
}

// --- slot sizes for rows that outgrow their capacity
__global__ void k_need(const int32_t* touched, const int64_t* n_touched, int64_t max_t, const int32_t* new_len,
                       const int32_t* row_cap, int64_t* need, const int32_t* err) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= max_t) return;
  int64_t v = 0;
  if (!*err && t < *n_touched) {
    int32_t r = touched[t];
    int64_t nl = new_len[r];
    if (nl > row_cap[r]) v = ((nl + nl / 2 + 16) + 7) & ~(int64_t)7;
  }
  need[t] = v;
}

__global__ void k_check_arena(const int64_t* need_scan, int64_t max_t, const int64_t* arena_top, int64_t nnz_cap,
                              int32_t* err) {
  if (*arena_top + need_scan[max_t] > nnz_cap) set_err(err, DERR_ARENA);
}

// --- commit staged rows (only reached by a fully valid batch)
__global__ void __launch_bounds__(256) k_commit_rows(const int32_t* touched, const int64_t* n_touched,
                                                      const int64_t* need_scan, const int64_t* arena_top,
                                                      const int32_t* new_len, const int64_t* tmp_off,
                                                      const int32_t* tmp_col, const double* tmp_val, int64_t* row_off,
                                                      int32_t* row_len, int32_t* row_cap, int32_t* col, double* val,
                                                      double* deg, const int32_t* err) {
  if (*err) return;
  const int64_t nt = *n_touched;
  __shared__ double red[256];
  for (int64_t t = blockIdx.x; t < nt; t += gridDim.x) {
    const int32_t r = touched[t];
    const int64_t nl = new_len[r];
    int64_t grow = need_scan[t + 1] - need_scan[t];
    int64_t off = row_off[r];
    if (grow > 0) off = *arena_top + need_scan[t];
    const int32_t* sc = tmp_col + tmp_off[r];
    double s = 0.0;
    for (int64_t j = threadIdx.x; j < nl; j += blockDim.x) {
      col[off + j] = sc[j];
      if (val) {
        double x = tmp_val[tmp_off[r] + j];
        val[off + j] = x;
        s += x;
      }
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
      if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      row_off[r] = off;
      row_len[r] = (int32_t)nl;
      if (grow > 0) row_cap[r] = (int32_t)grow;
      deg[r] = val ? red[0] : (double)nl;
    }
    __syncthreads();
  }
}

// --- arena compaction: fresh slots of len + len/4 + 4 entries, in row order
__global__ void k_compact_caps(const int32_t* row_len, int64_t n, int64_t* caps) {
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r < n) {
    const int64_t l = row_len[r];
    caps[r] = l + l / 4 + 4;
  }
}

// one warp per row; a row's offset is rewritten by the warp that read it
__global__ void __launch_bounds__(256) k_compact_copy(int64_t n, const int64_t* off_scan, int64_t* row_off,
                                                      const int32_t* row_len, int32_t* row_cap, const int32_t* col,
                                                      const double* val, int32_t* ncol, double* nval) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; r < n; r += warps) {
    const int64_t o = row_off[r], no = off_scan[r];
    const int32_t l = row_len[r];
    for (int32_t j = lane; j < l; j += 32) {
      ncol[no + j] = col[o + j];
      if (val) nval[no + j] = val[o + j];
    }
    __syncwarp();
    if (lane == 0) {
      row_off[r] = no;
      row_cap[r] = (int32_t)(off_scan[r + 1] - no);
    }
  }
}

__global__ void k_set_top(int64_t* arena_top, const int64_t* off_scan, int64_t n) { *arena_top = off_scan[n]; }

__global__ void k_bump_arena(int64_t* arena_top, const int64_t* need_scan, int64_t max_t, const int32_t* err) {
  if (!*err) *arena_top += need_scan[max_t];
}

__global__ void k_commit_nodes(int64_t N, int64_t N2, uint8_t* live, double* deg, const int32_t* dn, int64_t n_dn,
                               const int32_t* err) {
  if (*err) return;
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (N + i < N2) live[N + i] = 1;
  if (i < n_dn) {
    live[dn[i]] = 0;
    deg[dn[i]] = 0.0;
  }
}

// --- derived per-node quantities: d^-1/2, d_max over live nodes, long rows
__global__ void k_derived(int64_t n, const uint8_t* live, const double* deg, const int32_t* row_len, double* dis,
                          int64_t* longflag, double* block_max) {
  __shared__ double red[256];
  int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double m = 0.0;
  if (r < n) {
    double d = live[r] ? deg[r] : 0.0;
    dis[r] = d > 0.0 ? rsqrt(d) : 0.0;
    longflag[r] = row_len[r] > kLongRow ? 1 : 0;
    m = d;
  }
  red[threadIdx.x] = m;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) block_max[blockIdx.x] = red[0];
}

__global__ void k_max_reduce(const double* part, int64_t n, double* out) {
  __shared__ double red[1024];
  double m = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, part[i]);
  red[threadIdx.x] = m;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }
inline unsigned capped(int64_t n, int64_t cap) { return (unsigned)(n < 1 ? 1 : (n < cap ? n : cap)); }

__global__ void k_sum_len(const int32_t* row_len, int64_t n, unsigned long long* out) {
  __shared__ unsigned long long red[256];
  unsigned long long v = 0;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
    v += (unsigned long long)row_len[r];
  red[threadIdx.x] = v;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(out, red[0]);
}


// --- Delta X = (M_new - M_old) X for the paper's W block (P_perp Delta X_bar,
// Sec. 3.3) and the low-rank projection (Eq. main3), ADJ and LAP.  M_old is
// padded with zero rows and columns for the S new nodes.
//   diagonal: delta_r = alpha_new - d_r (new rows), alpha_new - alpha_old
//             (old live rows; the degree change is added per touched row),
//             zero for ADJ and for tombstoned rows
//   touched rows: sum over the row's batch entries of (+w insert | -w_old
//             delete) x_c, and for LAP old rows - (d_new - d_old) x_r
template <typename T>
__global__ void k_delta_diag(const T* __restrict__ X, int64_t ldx, T* __restrict__ Y, int64_t ldy, int w, int64_t N,
                             int64_t N2, int op, const double* __restrict__ deg, const uint8_t* __restrict__ live,
                             const double* __restrict__ dmax_new, const double* __restrict__ dmax_old) {
  const double an = 2.0 * (*dmax_new), ao = 2.0 * (*dmax_old);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < N2 * w; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / w;
    const int c = (int)(e % w);
    double dl = 0.0;
    if (op == GREST_OP_LAP && live[r]) dl = r >= N ? an - deg[r] : an - ao;
    Y[r * ldy + c] = (T)(dl * (double)X[r * ldx + c]);
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_delta_rows(const T* __restrict__ X, int64_t ldx, T* __restrict__ Y,
                                                    int64_t ldy, int w, int64_t N, int op,
                                                    const int32_t* __restrict__ touched,
                                                    const int64_t* __restrict__ n_touched,
                                                    const int64_t* __restrict__ seg, const uint64_t* __restrict__ ekey,
                                                    const double* __restrict__ ew, const double* __restrict__ edel) {
  const int lane = threadIdx.x & 31;
  const int64_t nt = *n_touched;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t t = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); t < nt; t += warps) {
    const int32_t r = touched[t];
    const int64_t s0 = seg[r], L = seg[r + 1] - s0;
    for (int c0 = 0; c0 < w; c0 += 32) {
      const int c = c0 + lane;
      double acc = 0.0, dd = 0.0;
      for (int64_t i = 0; i < L; ++i) {
        const uint64_t k = ekey[s0 + i];
        const double v = key_tag(k) == kTagIns ? ew[s0 + key_idx(k)] : -edel[s0 + i];
        dd += v;
        if (c < w) acc = fma(v, (double)X[(int64_t)key_col(k) * ldx + c], acc);
      }
      if (c < w) {
        if (op == GREST_OP_LAP && r < N) acc -= dd * (double)X[(int64_t)r * ldx + c];
        Y[(int64_t)r * ldy + c] += (T)acc;
      }
    }
  }
}

}  // namespace

int graph_count_nnz(const Csr& g, int64_t n, int64_t* out, cudaStream_t s) {
  cudaMemsetAsync(out, 0, sizeof(int64_t), s);
  unsigned nb = blocks_for(n, 256);
  if (nb > 1024) nb = 1024;
  if (nb < 1) nb = 1;
  k_sum_len<<<nb, 256, 0, s>>>(g.row_len, n, reinterpret_cast<unsigned long long*>(out));
  return 1;
}

int graph_compact_plan(const Csr& g, GraphWork& w, int64_t n, cudaStream_t s) {
  const int T = 256;
  k_compact_caps<<<blocks_for(n, T), T, 0, s>>>(g.row_len, n, w.rowflag);
  return 1 + exclusive_scan_i64(w.rowflag, w.rowflag, n, w.scan_tmp, s);
}

int graph_compact_copy(Csr& g, const GraphWork& w, int64_t n, int32_t* new_col, double* new_val, cudaStream_t s) {
  k_compact_copy<<<capped(blocks_for(n * 32, 256), 152 * 8), 256, 0, s>>>(n, w.rowflag, g.row_off, g.row_len,
                                                                          g.row_cap, g.col, g.val, new_col, new_val);
  k_set_top<<<1, 1, 0, s>>>(g.arena_top, w.rowflag, n);
  return 2;
}

int graph_refresh_derived(Csr& g, GraphWork& w, int64_t n, cudaStream_t s) {
  if (n <= 0) return 0;
  int nk = 0;
  const int T = 256;
  unsigned nb = blocks_for(n, T);
  double* bmax = reinterpret_cast<double*>(w.need);  // n_cap+1 int64 scratch reused as doubles
  k_derived<<<nb, T, 0, s>>>(n, g.live, g.deg, g.row_len, g.dis, w.rowflag, bmax);
  ++nk;
  k_max_reduce<<<1, 1024, 0, s>>>(bmax, nb, g.dmax);
  ++nk;
  nk += exclusive_scan_i64(w.rowflag, w.rowflag, n, w.scan_tmp, s);
  k_compact<<<nb, T, 0, s>>>(w.rowflag, n, w.long_rows, w.scalars + 1);
  ++nk;
  return nk;
}

int graph_apply_batch(Csr& g, GraphWork& w, const BatchDev& b, int32_t* err, cudaStream_t s) {
  int nk = 0;
  const int64_t N = g.n, N2 = g.n + b.S;
  const int T = 256;
  const unsigned gsz = 152 * 8;
  cudaMemsetAsync(w.cnt, 0, sizeof(int32_t) * (N2 + 1), s);
  cudaMemsetAsync(w.cursor, 0, sizeof(int32_t) * N2, s);
  cudaMemsetAsync(w.delflag, 0, N2, s);
  if (b.S > 0) {
    k_init_new_rows<<<blocks_for(b.S, T), T, 0, s>>>(N, N2, g.row_off, g.row_len, g.row_cap);
    ++nk;
  }
  if (b.n_dn > 0) {
    k_mark_removed<<<capped(blocks_for(b.n_dn, T), gsz), T, 0, s>>>(b.dn, b.n_dn, N, g.live, w.cursor, w.delflag, err);
    ++nk;
    cudaMemsetAsync(w.cursor, 0, sizeof(int32_t) * N2, s);
  }
  if (b.n_ins > 0) {
    k_count_edges<<<capped(blocks_for(b.n_ins, T), gsz), T, 0, s>>>(b.ins_u, b.ins_v, b.ins_w, b.n_ins, N2, N, g.live,
                                                                   w.delflag, w.cnt, err);
    ++nk;
  }
  if (b.n_del > 0) {
    k_count_edges<<<capped(blocks_for(b.n_del, T), gsz), T, 0, s>>>(b.del_u, b.del_v, nullptr, b.n_del, N, N, g.live,
                                                                   w.delflag, w.cnt, err);
    ++nk;
  }
  if (b.n_dn > 0) {
    k_count_removed<<<capped(b.n_dn, gsz), T, 0, s>>>(b.dn, b.n_dn, g.row_off, g.row_len, g.col, w.cnt, err);
    ++nk;
  }
  // segment offsets and staging offsets
  k_cnt_to_i64<<<blocks_for(N2, T), T, 0, s>>>(w.cnt, w.seg, N2);
  ++nk;
  nk += exclusive_scan_i64(w.seg, w.seg, N2, w.scan_tmp, s);
  k_touch_flags<<<blocks_for(N2, T), T, 0, s>>>(w.cnt, w.delflag, g.row_len, N2, w.rowflag, w.tmp_off);
  ++nk;
  nk += exclusive_scan_i64(w.tmp_off, w.tmp_off, N2, w.scan_tmp, s);
  nk += exclusive_scan_i64(w.rowflag, w.rowflag, N2, w.scan_tmp, s);
  k_compact<<<blocks_for(N2, T), T, 0, s>>>(w.rowflag, N2, w.touched, w.scalars + 0);
  ++nk;
  k_check_sizes<<<1, 1, 0, s>>>(w.seg, w.tmp_off, N2, w.ent_cap, w.tmp_cap, err);
  ++nk;
  // scatter, sort, merge
  if (b.n_ins > 0) {
    k_scatter_edges<<<capped(blocks_for(b.n_ins, T), gsz), T, 0, s>>>(b.ins_u, b.ins_v, b.ins_w, b.n_ins, kTagIns,
                                                                     w.seg, w.cursor, w.ekey, w.ew, err);
    ++nk;
  }
  if (b.n_del > 0) {
    k_scatter_edges<<<capped(blocks_for(b.n_del, T), gsz), T, 0, s>>>(b.del_u, b.del_v, nullptr, b.n_del, kTagDel,
                                                                     w.seg, w.cursor, w.ekey, w.ew, err);
    ++nk;
  }
  if (b.n_dn > 0) {
    k_scatter_removed<<<capped(b.n_dn, gsz), T, 0, s>>>(b.dn, b.n_dn, g.row_off, g.row_len, g.col, w.seg, w.cursor,
                                                        w.ekey, w.ew, err);
    ++nk;
  }
  k_sort_segments<<<gsz, 256, 0, s>>>(w.touched, w.scalars + 0, w.seg, w.ekey, w.eins, err);
  ++nk;
  k_merge_rows<<<gsz, 256, 0, s>>>(w.touched, w.scalars + 0, w.seg, w.ekey, w.ew, w.eins, w.delflag, g.row_off,
                                    g.row_len, g.col, g.val, w.tmp_off, w.tmp_col, g.val ? w.tmp_val : nullptr,
                                    w.new_len, w.edel, err);
  ++nk;
  // capacity: touched rows that outgrow their slot
  const int64_t max_t = N2;  // upper bound of the touched count
  k_need<<<blocks_for(max_t, T), T, 0, s>>>(w.touched, w.scalars + 0, max_t, w.new_len, g.row_cap, w.need, err);
  ++nk;
  nk += exclusive_scan_i64(w.need, w.need, max_t, w.scan_tmp, s);
  k_check_arena<<<1, 1, 0, s>>>(w.need, max_t, g.arena_top, g.nnz_cap, err);
  ++nk;
  k_commit_rows<<<gsz, 256, 0, s>>>(w.touched, w.scalars + 0, w.need, g.arena_top, w.new_len, w.tmp_off, w.tmp_col,
                                     w.tmp_val, g.row_off, g.row_len, g.row_cap, g.col, g.val, g.deg, err);
  ++nk;
  k_bump_arena<<<1, 1, 0, s>>>(g.arena_top, w.need, max_t, err);
  ++nk;
  int64_t nc = b.S > b.n_dn ? b.S : b.n_dn;
  if (nc > 0) {
    k_commit_nodes<<<blocks_for(nc, T), T, 0, s>>>(N, N2, g.live, g.deg, b.dn, b.n_dn, err);
    ++nk;
  }
  return nk;
}

template <typename T>
int delta_apply_t(const Csr& g, const GraphWork& w, int op, const T* X, int64_t ldx, T* Y, int64_t ldy, int wd,
                  int64_t N, int64_t N2, const double* dmax_old, cudaStream_t s) {
  if (N2 <= 0 || wd <= 0) return 0;
  const int64_t tot = N2 * wd;
  k_delta_diag<T><<<(unsigned)std::min<int64_t>((tot + 255) / 256, 152 * 32), 256, 0, s>>>(
      X, ldx, Y, ldy, wd, N, N2, op, g.deg, g.live, g.dmax, dmax_old);
  k_delta_rows<T><<<152 * 8, 256, 0, s>>>(X, ldx, Y, ldy, wd, N, op, w.touched, w.scalars + 0, w.seg, w.ekey, w.ew,
                                          w.edel);
  return 2;
}

int delta_apply(const Csr& g, const GraphWork& w, int op, const double* X, int64_t ldx, double* Y, int64_t ldy, int wd,
                int64_t N, int64_t N2, const double* dmax_old, cudaStream_t s) {
  return delta_apply_t<double>(g, w, op, X, ldx, Y, ldy, wd, N, N2, dmax_old, s);
}

int delta_apply(const Csr& g, const GraphWork& w, int op, const float* X, int64_t ldx, float* Y, int64_t ldy, int wd,
                int64_t N, int64_t N2, const double* dmax_old, cudaStream_t s) {
  return delta_apply_t<float>(g, w, op, X, ldx, Y, ldy, wd, N, N2, dmax_old, s);
}

}  // namespace grest
