// Grouped update, part 1: the graph update of every graph of a group (one CTA
// per graph) and the per-node stages around the dense products: the padded
// basis [X; 0] (Alg. 2), the exact new-node block E = M_new[:, N:N'] and the
// RSVD test matrix Omega (Sec. 3.5), and the final sign normalization.
//
// Graph update of graph g, following Eq. (adj_update) / Sec. 2 as the
// single-graph update does (graph.cu), inside one CTA:
//   count    both directions of every edit per row (ids checked: range, self loop)
//   scan     segment offsets, the list of touched rows, staging offsets
//   scatter  batch entries into per-row segments, then sort each segment
//   merge    old row (-) deletions (+) insertions; an inserted edge that
//            exists, a deleted one that does not, or an edge twice in the
//            batch rejects the whole batch
//   commit   only when the whole batch is valid and fits the edge arena:
//            rows that outgrow their slot move to the arena top
// A rejected batch leaves the graph unchanged and marks the graph's status,
// which every later stage of the round checks before doing anything.
#include "group.cuh"
#include "philox.cuh"

namespace grest {
namespace grp {

namespace {

constexpr int kUpdThreads = 1024;

// exclusive prefix sum of a[0..n) in place (one CTA); a[n] receives the total
__device__ int64_t block_scan(int64_t* a, int64_t n, int64_t* red) {
  const int tid = threadIdx.x, nth = blockDim.x, lane = tid & 31, wid = tid >> 5;
  const int64_t per = (n + nth - 1) / nth;
  const int64_t b = tid * per, e = b + per < n ? b + per : n;
  int64_t loc = 0;
  for (int64_t i = b; i < e; ++i) loc += a[i];
  int64_t x = loc;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) red[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int64_t w = lane < (nth >> 5) ? red[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    red[lane] = w;  // inclusive sums over warps
  }
  __syncthreads();
  int64_t run = x - loc + (wid > 0 ? red[wid - 1] : 0);
  for (int64_t i = b; i < e; ++i) {
    const int64_t v = a[i];
    a[i] = run;
    run += v;
  }
  const int64_t total = red[(nth >> 5) - 1];
  __syncthreads();
  if (tid == 0) a[n] = total;
  __syncthreads();
  return total;
}

__device__ __forceinline__ void fail(int* s_err, int code) { atomicCAS(s_err, 0, code); }

// keys of batch entries: column in the high bits, insertion flag in bit 0
__device__ __forceinline__ uint64_t ent_key(int32_t col, int ins) { return ((uint64_t)(uint32_t)col << 1) | (uint64_t)ins; }

__device__ void shell_sort(uint64_t* a, int n) {
  for (int gap = n / 2; gap > 0; gap /= 2)
    for (int i = gap; i < n; ++i) {
      const uint64_t v = a[i];
      int j = i;
      for (; j >= gap && a[j - gap] > v; j -= gap) a[j] = a[j - gap];
      a[j] = v;
    }
}

__global__ void __launch_bounds__(kUpdThreads) k_g_update(GPools P) {
  const int g = blockIdx.x, tid = threadIdx.x, nth = blockDim.x;
  GState& st = P.st[g];
  const GMeta mt = P.meta[g];
  const GRound rd = P.round[g];
  __shared__ int s_err;
  __shared__ int64_t red[32];
  __shared__ double dred[32];
  const int64_t N = st.N, S = rd.S, N2 = N + S, ni = rd.n_ins, nd = rd.n_del;
  if (tid == 0) s_err = 0;
  __syncthreads();
  if (S < 0 || ni < 0 || nd < 0) fail(&s_err, GREST_ERR_INVALID_ARG);
  else if (N2 > mt.node_cap || 2 * (ni + nd) > mt.ent_cap) fail(&s_err, GREST_ERR_CAPACITY);
  __syncthreads();
  if (s_err) {
    if (tid == 0) st.status = s_err;
    return;
  }
  const int64_t no = mt.node_off;
  int64_t* row_off = P.row_off + no;
  int32_t* row_len = P.row_len + no;
  int32_t* row_cap = P.row_cap + no;
  int32_t* col = P.col + mt.edge_off;
  int32_t* cnt = P.cnt + no;
  int64_t* seg = P.seg + no + g;      // node_cap + 1 entries per graph
  int64_t* stg = P.stg_off + no + g;
  int64_t* need = P.need + no + g;
  int32_t* touched = P.touched + no;
  int32_t* new_len = P.new_len + no;
  uint64_t* ent = P.ent + mt.ent_off;
  int32_t* stage = P.stage + mt.stage_off;
  const int32_t* iu = P.edits + rd.edit_off;
  const int32_t* iv = iu + ni;
  const int32_t* du = iv + ni;
  const int32_t* dv = du + nd;
  // count
  for (int64_t r = tid; r < N2; r += nth) cnt[r] = 0;
  __syncthreads();
  for (int64_t e = tid; e < ni + nd; e += nth) {
    const bool ins = e < ni;
    const int32_t a = ins ? iu[e] : du[e - ni], b = ins ? iv[e] : dv[e - ni];
    const int64_t lim = ins ? N2 : N;
    if (a < 0 || b < 0 || a >= lim || b >= lim || a == b) { fail(&s_err, GREST_ERR_INVALID_UPDATE); continue; }
    atomicAdd(&cnt[a], 1);
    atomicAdd(&cnt[b], 1);
  }
  __syncthreads();
  if (s_err) {
    if (tid == 0) st.status = s_err;
    return;
  }
  // segment offsets; touched rows (flags scanned in `need`)
  for (int64_t r = tid; r < N2; r += nth) {
    seg[r] = cnt[r];
    need[r] = cnt[r] > 0 ? 1 : 0;
  }
  __syncthreads();
  block_scan(seg, N2, red);
  const int64_t nt = block_scan(need, N2, red);
  for (int64_t r = tid; r < N2; r += nth) {
    if (need[r + 1] != need[r]) touched[need[r]] = (int32_t)r;
    cnt[r] = 0;  // becomes the scatter cursor
  }
  __syncthreads();
  // staging offsets of the merged rows
  for (int64_t t = tid; t < nt; t += nth) {
    const int32_t r = touched[t];
    stg[t] = (r < N ? row_len[r] : 0) + (seg[r + 1] - seg[r]);
  }
  __syncthreads();
  const int64_t staged = block_scan(stg, nt, red);
  if (staged > mt.stage_cap) fail(&s_err, GREST_ERR_CAPACITY);
  // scatter both directions of every edit
  for (int64_t e = tid; e < ni + nd; e += nth) {
    const bool ins = e < ni;
    const int32_t a = ins ? iu[e] : du[e - ni], b = ins ? iv[e] : dv[e - ni];
    ent[seg[a] + atomicAdd(&cnt[a], 1)] = ent_key(b, ins);
    ent[seg[b] + atomicAdd(&cnt[b], 1)] = ent_key(a, ins);
  }
  __syncthreads();
  if (s_err) {
    if (tid == 0) st.status = s_err;
    return;
  }
  // sort each segment, merge it with the old row, validate
  for (int64_t t = tid; t < nt; t += nth) {
    const int32_t r = touched[t];
    uint64_t* e = ent + seg[r];
    const int ne = (int)(seg[r + 1] - seg[r]);
    shell_sort(e, ne);
    const int ol = r < N ? row_len[r] : 0;
    const int32_t* old = col + (r < N ? row_off[r] : 0);
    int32_t* out = stage + stg[t];
    int i = 0, j = 0, o = 0;
    int64_t prev = -1;
    bool bad = false;
    while (!bad && (i < ol || j < ne)) {
      if (j >= ne || (i < ol && old[i] < (int32_t)(e[j] >> 1))) {
        out[o++] = old[i++];
        continue;
      }
      const int32_t c = (int32_t)(e[j] >> 1);
      const int ins = (int)(e[j] & 1);
      if (c == prev) { bad = true; break; }  // the same edge twice in the batch
      prev = c;
      ++j;
      if (i < ol && old[i] == c) {
        if (ins) bad = true;  // inserted edge exists
        else ++i;             // deleted
      } else if (!ins) {
        bad = true;           // deleted edge is missing
      } else {
        out[o++] = c;
      }
    }
    if (bad) fail(&s_err, GREST_ERR_INVALID_UPDATE);
    new_len[r] = o;
  }
  __syncthreads();
  if (s_err) {
    if (tid == 0) st.status = s_err;
    return;
  }
  // arena space of the rows that outgrow their slot
  for (int64_t t = tid; t < nt; t += nth) {
    const int32_t r = touched[t];
    const int64_t nl = new_len[r], cap = r < N ? row_cap[r] : 0;
    need[t] = nl > cap ? ((nl + nl / 2 + 16) + 7) & ~(int64_t)7 : 0;
  }
  __syncthreads();
  const int64_t grow = block_scan(need, nt, red);
  const int64_t top = st.arena_top;
  if (top + grow > mt.edge_cap) {
    if (tid == 0) st.status = GREST_ERR_CAPACITY;
    return;
  }
  // commit (the batch is valid and fits)
  for (int64_t r = N + tid; r < N2; r += nth) {
    row_off[r] = 0;
    row_len[r] = 0;
    row_cap[r] = 0;
    P.deg[no + r] = 0.0;
  }
  __syncthreads();
  for (int64_t t = tid; t < nt; t += nth) {
    const int32_t r = touched[t];
    const int64_t nl = new_len[r], gr = need[t + 1] - need[t];
    const int64_t off = gr > 0 ? top + need[t] : row_off[r];
    const int32_t* src = stage + stg[t];
    for (int64_t j = 0; j < nl; ++j) col[off + j] = src[j];
    row_off[r] = off;
    row_len[r] = (int32_t)nl;
    if (gr > 0) row_cap[r] = (int32_t)gr;
    P.deg[no + r] = (double)nl;
  }
  __syncthreads();
  // derived per-node values: d^-1/2, d_max, nnz
  double mx = 0.0;
  int64_t nz = 0;
  for (int64_t r = tid; r < N2; r += nth) {
    const double d = P.deg[no + r];
    P.dis[no + r] = d > 0.0 ? 1.0 / sqrt(d) : 0.0;
    mx = fmax(mx, d);
    nz += row_len[r];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
    nz += __shfl_down_sync(0xffffffffu, nz, o);
  }
  if ((tid & 31) == 0) {
    dred[tid >> 5] = mx;
    red[tid >> 5] = nz;
  }
  __syncthreads();
  if (tid == 0) {
    for (int w = 1; w < (nth >> 5); ++w) {
      mx = fmax(mx, dred[w]);
      nz += red[w];
    }
    const SmallLayout L = small_layout(P.K, P.q, P.L, P.cmax, P.mmax);
    st.N = N2;
    st.S = (int32_t)S;
    st.arena_top = top + grow;
    st.nnz = nz;
    st.dmax = mx;
    st.ref = fabs(gsmall(P, g)[L.theta]);
    // the step's subspace (Table 1): no block, the exact block, or the RSVD block
    int mode = 2;
    if (S > 0 && P.subspace != GREST_SUB_GREST2) {
      const bool rsvd = P.subspace == GREST_SUB_RSVD || (P.subspace == GREST_SUB_AUTO && S > P.q);
      mode = rsvd ? 4 : 3;
    }
    st.status = (mode == 3 && S > P.q) ? GREST_ERR_UNSUPPORTED : 0;
    st.mode = mode;
    st.Ku = P.K;
    st.cb = mode == 3 ? (int32_t)S : 0;
    st.cw = st.Ku + st.cb;
    st.r = st.r2 = st.rY = st.rY2 = st.Lp = st.m = 0;
    st.kept_min = st.dropped_max = st.boundary_gap = 0.0;
  }
}

// Z[:, 0:K] = [X; 0] over the graph's N' rows (Alg. 2's padded basis)
__global__ void __launch_bounds__(256) k_g_pad(GPools P) {
  const int g = blockIdx.y;
  const GState& st = P.st[g];
  if (st.status) return;
  const int64_t ro = P.meta[g].node_off, N = st.N - st.S, N2 = st.N, K = st.Ku;
  const double* U = P.U + ro * P.ldu;
  double* Z = P.Z + ro * P.ldz;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < N2 * K; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / K;
    const int c = (int)(e % K);
    Z[r * P.ldz + c] = r < N ? U[r * P.ldu + c] : 0.0;
  }
}

// diagonal coefficient and off-diagonal scale of row r (Sec. 4.2)
__device__ __forceinline__ void op_row(const GPools& P, const GState& st, int64_t gr, double& dcoef, double& scale) {
  dcoef = 0.0;
  scale = 1.0;
  if (P.op == GREST_OP_LAP) dcoef = 2.0 * st.dmax - P.deg[gr];
  else if (P.op == GREST_OP_NLAP) { dcoef = 1.0; scale = P.dis[gr]; }
}

// exact new-node block: Z[:, 2K : 2K + S] = M_new[:, N:N'] (one warp per row)
__global__ void __launch_bounds__(256) k_g_newcols(GPools P) {
  const int g = blockIdx.y;
  const GState& st = P.st[g];
  if (st.status || st.mode != 3) return;
  const int lane = threadIdx.x & 31;
  const int64_t ro = P.meta[g].node_off, N = st.N - st.S, N2 = st.N, S = st.S;
  double* B = P.Z + ro * P.ldz + 2 * st.Ku;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; r < N2; r += warps) {
    double* br = B + r * P.ldz;
    for (int64_t j = lane; j < S; j += 32) br[j] = 0.0;
    __syncwarp();
    double dcoef, scale;
    op_row(P, st, ro + r, dcoef, scale);
    const int32_t* c = P.col + P.meta[g].edge_off + P.row_off[ro + r];
    const int len = P.row_len[ro + r];
    for (int j = lane; j < len; j += 32) {
      const int32_t nb = c[j];
      if (nb >= N) br[nb - N] = P.op == GREST_OP_NLAP ? scale * P.dis[ro + nb] : 1.0;
    }
    __syncwarp();
    if (lane == 0 && r >= N && dcoef != 0.0) br[r - N] += dcoef;
  }
}

// Omega (S x q) of graph g at its step counter: the same generator and
// element layout as the single-graph update (rsvd.cu)
__global__ void __launch_bounds__(256) k_g_omega(GPools P) {
  const int g = blockIdx.y;
  const GState& st = P.st[g];
  if (st.status || st.mode != 4) return;
  const int64_t ro = P.meta[g].node_off, total = (int64_t)st.S * P.q, nblk = (total + 3) / 4;
  double* Om = P.Om + ro * P.ldq;
  const uint64_t seed = P.meta[g].seed, step = (uint64_t)st.step;
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nblk; b += (int64_t)gridDim.x * blockDim.x) {
    uint64_t c[4] = {(uint64_t)b, step, 0ull, 0ull};
    rng::philox4x64_10(c, seed, 0x47524553ull);
    double z[4];
    rng::box_muller(c[0], c[1], z[0], z[1]);
    rng::box_muller(c[2], c[3], z[2], z[3]);
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int64_t e = 4 * b + t;
      if (e < total) Om[(e / P.q) * P.ldq + (e % P.q)] = z[t];
    }
  }
}

// X = Un with each column flipped so that its largest-magnitude entry
// (lowest row on ties) is positive; Lambda = Theta_K; step + 1 (one CTA per graph)
__global__ void __launch_bounds__(256) k_g_finish(GPools P) {
  const int g = blockIdx.x, tid = threadIdx.x, nth = blockDim.x;
  GState& st = P.st[g];
  if (st.status) return;
  const int64_t ro = P.meta[g].node_off, N2 = st.N;
  const int K = P.K;
  const double* Un = P.Un + ro * P.ldu;
  double* U = P.U + ro * P.ldu;
  __shared__ double bv[8][256 / 32];
  __shared__ int64_t bi[8][256 / 32];
  __shared__ double sgn[kMaxW];
  for (int c0 = 0; c0 < K; c0 += 8) {
    double v[8];
    int64_t ix[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) { v[q] = -1.0; ix[q] = INT64_MAX; }
    for (int64_t r = tid; r < N2; r += nth)
#pragma unroll
      for (int q = 0; q < 8; ++q)
        if (c0 + q < K) {
          const double a = fabs(Un[r * P.ldu + c0 + q]);
          if (a > v[q]) { v[q] = a; ix[q] = r; }  // rows ascend per thread: strict > keeps the lowest
        }
#pragma unroll
    for (int q = 0; q < 8; ++q)
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_down_sync(0xffffffffu, v[q], o);
        const int64_t oi = __shfl_down_sync(0xffffffffu, ix[q], o);
        if (ov > v[q] || (ov == v[q] && oi < ix[q])) { v[q] = ov; ix[q] = oi; }
      }
    if ((tid & 31) == 0)
#pragma unroll
      for (int q = 0; q < 8; ++q) { bv[q][tid >> 5] = v[q]; bi[q][tid >> 5] = ix[q]; }
    __syncthreads();
    if (tid < 8 && c0 + tid < K) {
      double bvv = -1.0;
      int64_t bii = INT64_MAX;
      for (int w = 0; w < nth / 32; ++w)
        if (bv[tid][w] > bvv || (bv[tid][w] == bvv && bi[tid][w] < bii)) { bvv = bv[tid][w]; bii = bi[tid][w]; }
      sgn[c0 + tid] = (bii < N2 && Un[bii * P.ldu + c0 + tid] < 0.0) ? -1.0 : 1.0;
    }
    __syncthreads();
  }
  for (int64_t e = tid; e < N2 * K; e += nth) {
    const int64_t r = e / K;
    const int c = (int)(e % K);
    U[r * P.ldu + c] = sgn[c] * Un[r * P.ldu + c];
  }
  if (tid == 0) {
    const SmallLayout L = small_layout(P.K, P.q, P.L, P.cmax, P.mmax);
    double* sm = gsmall(P, g);
    for (int j = 0; j < K; ++j) sm[L.theta + j] = sm[L.thnew + j];
    st.step += 1;
  }
}

}  // namespace

int launch_update(const GPools& P, cudaStream_t s) {
  k_g_update<<<P.G, kUpdThreads, 0, s>>>(P);
  return 1;
}

int launch_pad(const GPools& P, const LaunchShape& ls, cudaStream_t s) {
  k_g_pad<<<dim3(ls.row_blocks, P.G), 256, 0, s>>>(P);
  return 1;
}

int launch_newcols(const GPools& P, const LaunchShape& ls, cudaStream_t s) {
  k_g_newcols<<<dim3(ls.row_blocks, P.G), 256, 0, s>>>(P);
  return 1;
}

int launch_omega(const GPools& P, const LaunchShape& ls, cudaStream_t s) {
  k_g_omega<<<dim3(ls.row_blocks, P.G), 256, 0, s>>>(P);
  return 1;
}

int launch_finish(const GPools& P, cudaStream_t s) {
  k_g_finish<<<P.G, 256, 0, s>>>(P);
  return 1;
}

}  // namespace grp
}  // namespace grest
