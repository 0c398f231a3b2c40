// Grouped update, part 2: the dense stages of Alg. 2 for every graph of a
// group, one launch per stage, each graph's operands and widths taken from
// its device-resident state (group.cuh selectors):
//   SpMM   Y = M X over the graph's rows (Sec. 4.2 operators in the epilogue)
//   Gram   C = X^T Y, kPch row chunks per graph, partial sums reduced in a
//          fixed order (the result does not depend on the group)
//   GEMM   Out = beta Cin + alpha X B, one warp per row, B in shared memory
//   CholQR pivoted Cholesky with the drop rule of the single-graph update
//          (largest remaining diagonal first, stop at R_kk^2 <= tol^2
//          max(R_00^2, ref^2)) and the inverse T = P R^-1 of the kept part
//   eig    cyclic Jacobi (parallel round-robin ordering, Brent and Luk) on
//          the m x m projected problem, then Alg. 1's selection of the K
//          leading pairs in the tracking order
// Every problem here has at most 64 columns (group.cuh).
#include "group.cuh"

namespace grest {
namespace grp {

namespace {

// ------------------------------------------------------------------ SpMM
// LPR lanes per row (32, 16 or 8: narrow blocks put several rows in a warp,
// since an FP64 warp instruction costs the same for any active lanes); the
// autotuned rows-per-warp factor only changes which warp takes which rows
template <int SEL, int NCH, int LPR>
__global__ void __launch_bounds__(256) k_g_spmm(GPools P) {
  const int g = blockIdx.y;
  const SpmmOp op = spmm_op(SEL, P, g);
  if (!op.on) return;
  const GState& st = P.st[g];
  const GMeta& mt = P.meta[g];
  const int lane = (threadIdx.x & 31) % LPR, sub = (threadIdx.x & 31) / LPR;
  constexpr int SUBS = 32 / LPR;
  const int rpw = P.spmm_rows_per_warp;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int32_t* colb = P.col + mt.edge_off;
  const bool nl = P.op == GREST_OP_NLAP;
  const int64_t step = warps * SUBS * rpw;
  for (int64_t r00 = op.r0 + (((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5) * SUBS + sub) * rpw;
       r00 < op.r1; r00 += step) {
    for (int64_t r = r00; r < r00 + rpw && r < op.r1; ++r) {
      const int64_t gr = mt.node_off + r;
      const int32_t* c = colb + P.row_off[gr];
      const int len = P.row_len[gr];
      double acc[NCH];
#pragma unroll
      for (int ch = 0; ch < NCH; ++ch) acc[ch] = 0.0;
      for (int j = 0; j < len; ++j) {
        const int32_t nb = c[j];
        if (nb < op.col_lo) continue;
        const double a = nl ? P.dis[mt.node_off + nb] : 1.0;
        const double* xr = op.X + (int64_t)(nb - op.col_lo) * op.ldx;
#pragma unroll
        for (int ch = 0; ch < NCH; ++ch) {
          const int cc = ch * LPR + lane;
          if (cc < op.w) acc[ch] = nl ? fma(a, xr[cc], acc[ch]) : acc[ch] + xr[cc];
        }
      }
      double dcoef = 0.0, scale = 1.0;
      if (P.op == GREST_OP_LAP) dcoef = 2.0 * st.dmax - P.deg[gr];
      else if (nl) { dcoef = 1.0; scale = P.dis[gr]; }
      const bool diag = dcoef != 0.0 && r >= op.col_lo;
      const double* xd = op.X + (r - op.col_lo) * op.ldx;
      double* y = op.Y + (r - op.r0) * op.ldy;
#pragma unroll
      for (int ch = 0; ch < NCH; ++ch) {
        const int cc = ch * LPR + lane;
        if (cc < op.w) {
          double v = scale * acc[ch];
          if (diag) v += dcoef * xd[cc];
          y[cc] = v;
        }
      }
    }
  }
}

// ------------------------------------------------------------------ Gram
// An FP64 warp instruction costs its sub-partition the same whatever its
// active lanes, so the 4 x 4 output tiles are packed densely onto threads
// (only tiles bi <= bj for a symmetric product: X^T X, and H = Z^T M Z with
// M symmetric), and narrow products spread the slab's rows over R thread
// groups whose sums are added in a fixed order at the end.
__device__ __forceinline__ bool gram_sym(int sel, const GramOp& op) {
  return sel == GR_H || (op.X == op.Y && op.a == op.b && op.ldx == op.ldy);
}

struct GramTiling {
  int nbi, nbj, ntask, R;
};
__device__ __forceinline__ GramTiling gram_tiling(const GramOp& op, bool sym) {
  GramTiling t;
  t.nbi = (op.a + 3) / 4;
  t.nbj = (op.b + 3) / 4;
  t.ntask = sym ? t.nbi * (t.nbi + 1) / 2 : t.nbi * t.nbj;
  t.R = 256 / t.ntask;
  if (t.R > kGramRows) t.R = kGramRows;
  if (t.R < 1) t.R = 1;
  return t;
}

template <int SEL>
__global__ void __launch_bounds__(256) k_g_gram(GPools P) {
  const int g = blockIdx.y, p = blockIdx.x;
  const GramOp op = gram_op(SEL, P, g);
  if (!op.on) return;
  __shared__ double stg[2 * kGramRows * (kMaxW + 1)];  // X and Y slabs, then the row groups' sums
  double (*Xs)[kMaxW + 1] = reinterpret_cast<double (*)[kMaxW + 1]>(stg);
  double (*Ys)[kMaxW + 1] = reinterpret_cast<double (*)[kMaxW + 1]>(stg + kGramRows * (kMaxW + 1));
  const bool sym = gram_sym(SEL, op);
  const GramTiling tl = gram_tiling(op, sym);
  const int t = threadIdx.x, task = t % tl.ntask, rg = t / tl.ntask;
  const bool active = rg < tl.R;
  int bi = 0, bj = 0;
  if (sym) {
    int x = task;
    while (x >= tl.nbi - bi) { x -= tl.nbi - bi; ++bi; }
    bj = bi + x;
  } else {
    bi = task / tl.nbj;
    bj = task % tl.nbj;
  }
  const int aw = tl.nbi * 4, bw = tl.nbj * 4;  // staged widths, zero beyond a and b
  int64_t rpc = (op.n + kPch - 1) / kPch;
  rpc = (rpc + kGramRows - 1) / kGramRows * kGramRows;
  const int64_t rb = p * rpc, re = rb + rpc < op.n ? rb + rpc : op.n;
  double acc[4][4] = {};
  for (int64_t r0 = rb; r0 < re; r0 += kGramRows) {
    for (int e = threadIdx.x; e < kGramRows * aw; e += blockDim.x) {
      const int rr = e / aw, cc = e % aw;
      const int64_t r = r0 + rr;
      Xs[rr][cc] = (r < re && cc < op.a) ? op.X[r * op.ldx + cc] : 0.0;
    }
    for (int e = threadIdx.x; e < kGramRows * bw; e += blockDim.x) {
      const int rr = e / bw, cc = e % bw;
      const int64_t r = r0 + rr;
      Ys[rr][cc] = (r < re && cc < op.b) ? op.Y[r * op.ldy + cc] : 0.0;
    }
    __syncthreads();
    if (active) {
      for (int k = rg; k < kGramRows; k += tl.R) {
        double xa[4], yb[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          xa[u] = Xs[k][bi * 4 + u];
          yb[u] = Ys[k][bj * 4 + u];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) acc[u][v] = fma(xa[u], yb[v], acc[u][v]);
      }
    }
    __syncthreads();
  }
  // the row groups' sums, added in group order
  double* red = stg;  // R * ntask <= 256 tiles of 16 values fit the staging array
  if (active)
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) red[(rg * tl.ntask + task) * 16 + u * 4 + v] = acc[u][v];
  __syncthreads();
  if (t < tl.ntask) {
    double* part = P.part + ((int64_t)g * kPch + p) * kMaxW * kMaxW;
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        double sum = 0.0;
        for (int q = 0; q < tl.R; ++q) sum += red[(q * tl.ntask + t) * 16 + u * 4 + v];
        const int i = bi * 4 + u, j = bj * 4 + v;
        if (i < op.a && j < op.b) part[i * kMaxW + j] = sum;
      }
  }
}

template <int SEL>
__global__ void __launch_bounds__(256) k_g_gram_reduce(GPools P) {
  const int g = blockIdx.x;
  const GramOp op = gram_op(SEL, P, g);
  if (!op.on) return;
  const bool sym = gram_sym(SEL, op);
  const double* part = P.part + (int64_t)g * kPch * kMaxW * kMaxW;
  for (int e = threadIdx.x; e < op.a * op.b; e += blockDim.x) {
    const int i = e / op.b, j = e % op.b;
    const int src = (!sym || i / 4 <= j / 4) ? i * kMaxW + j : j * kMaxW + i;  // lower tiles mirrored
    double s = 0.0;
#pragma unroll
    for (int p = 0; p < kPch; ++p) s += part[(int64_t)p * kMaxW * kMaxW + src];
    op.C[i * op.ldc + j] = s;
  }
}

// ------------------------------------------------------------------ GEMM
// one output element per thread ((row, column) pairs laid out linearly, so
// narrow outputs keep every lane busy); B in shared memory
template <int SEL>
__global__ void __launch_bounds__(256) k_g_gemm(GPools P) {
  const int g = blockIdx.y;
  const GemmOp op = gemm_op(SEL, P, g);
  if (!op.on) return;
  __shared__ double Bs[kMaxW][kMaxW + 1];
  for (int e = threadIdx.x; e < op.a * op.c; e += blockDim.x) Bs[e / op.c][e % op.c] = op.B[(e / op.c) * op.ldb + e % op.c];
  __syncthreads();
  const int64_t total = op.n * op.c;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / op.c;
    const int j = (int)(e % op.c);
    const double* x = op.X + r * op.ldx;
    double s = 0.0;
    for (int k = 0; k < op.a; ++k) s = fma(x[k], Bs[k][j], s);
    double v = op.alpha * s;
    if (op.beta != 0.0) v += op.beta * op.Cin[r * op.ldc + j];
    op.Out[r * op.ldo + j] = v;
  }
}

// ------------------------------------------------------------------ CholQR
__device__ inline PcholOp pchol_op(int sel, const GPools& P, int g) {
  GState& s = P.st[g];
  const SmallLayout L = small_layout(P.K, P.q, P.L, P.cmax, P.mmax);
  double* sm = gsmall(P, g);
  PcholOp o{};
  o.G = sm + L.Gm;
  o.T = sm + L.Tm;
  o.ldg = o.ldt = P.cmax;
  o.on = s.status == 0;
  switch (sel) {
    case PC_Y1: o.c = P.q; o.tol = P.drop_tol; o.abs_ref = s.ref; o.rank_out = &s.rY; o.on = o.on && s.mode == 4; break;
    case PC_Y2: o.c = s.rY; o.tol = 1e-14; o.abs_ref = 0.0; o.rank_out = &s.rY2; o.on = o.on && s.mode == 4; break;
    case PC_V1: o.c = s.cw; o.tol = P.drop_tol; o.abs_ref = s.ref; o.rank_out = &s.r; o.stats = true; break;
    default: /* PC_V2 */ o.c = s.r; o.tol = 1e-14; o.abs_ref = 0.0; o.rank_out = &s.r2; break;
  }
  o.on = o.on && o.c > 0;
  return o;
}

// Pivoted Cholesky of G (c x c, upper triangle read) in one CTA, smem =
// 2 kMaxW (kMaxW + 1) doubles.  Pivot k is the largest remaining diagonal
// (lowest index on ties); the factorization stops at the first pivot with
// R_kk^2 <= tol^2 max(R_00^2, abs_ref^2).  T (c x c, ldt) = P R^-1 on the kept
// pivots, zero elsewhere.  Returns the rank; *ref, *vlast, *vdrop: the
// reference and the last kept and first dropped squared pivots.
struct PcholResult {
  int rank;
  double ref, vlast, vdrop;
};

__device__ PcholResult pchol_block(const double* G, int ldg, int c, double tol, double abs_ref, double* T, int ldt,
                                   double* smem) {
  const int tid = threadIdx.x, nth = blockDim.x;
  double (*A)[kMaxW + 1] = reinterpret_cast<double (*)[kMaxW + 1]>(smem);
  double (*Rs)[kMaxW + 1] = reinterpret_cast<double (*)[kMaxW + 1]>(smem + kMaxW * (kMaxW + 1));  // row k of R, original indices
  __shared__ int done[kMaxW], piv[kMaxW];
  __shared__ double rinv[kMaxW];  // 1 / R_kk
  __shared__ double s_ref, s_thr, s_vlast, s_vdrop, s_rkk;
  __shared__ int s_p, s_stop, s_rank;
  for (int e = tid; e < c * c; e += nth) {
    const int i = e / c, l = e % c;
    A[i][l] = i <= l ? G[i * ldg + l] : G[l * ldg + i];
  }
  for (int l = tid; l < c; l += nth) done[l] = 0;
  if (tid == 0) { s_rank = c; s_vlast = 0.0; s_vdrop = 0.0; s_ref = 0.0; }
  __syncthreads();
  for (int k = 0; k < c; ++k) {
    if (tid < 32) {
      double bv = -1.0;
      int bi = c;
      for (int i = tid; i < c; i += 32)
        if (!done[i] && (A[i][i] > bv || (A[i][i] == bv && i < bi))) { bv = A[i][i]; bi = i; }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_down_sync(0xffffffffu, bv, o);
        const int oi = __shfl_down_sync(0xffffffffu, bi, o);
        if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
      }
      if (tid == 0) {
        if (k == 0) {
          s_ref = fmax(bv, abs_ref * abs_ref);
          s_thr = tol * tol * s_ref;
        }
        if (bi >= c || !(bv > 0.0) || !(bv > s_thr) || !isfinite(bv)) {
          s_stop = 1;
          s_rank = k;
          s_vdrop = bv > 0.0 ? bv : 0.0;
        } else {
          s_stop = 0;
          s_p = bi;
          s_vlast = bv;
          piv[k] = bi;
          done[bi] = 1;
          // once per pivot (a short FP64 chain): 1 / R_kk and R_kk = v / sqrt(v)
          const double ri = rsqrt(bv);
          rinv[k] = ri;
          s_rkk = bv * ri;
        }
      }
    }
    __syncthreads();
    if (s_stop) break;
    const int p = s_p;
    const double ri = rinv[k], rkk = s_rkk;
    for (int l = tid; l < c; l += nth) Rs[k][l] = (l == p) ? rkk : (done[l] ? 0.0 : A[p][l] * ri);
    __syncthreads();
    for (int e = tid; e < c * c; e += nth) {
      const int i = e / c, l = e % c;
      if (!done[i] && !done[l]) A[i][l] = fma(-Rs[k][i], Rs[k][l], A[i][l]);
    }
    __syncthreads();
  }
  const int rk = s_rank;
  // T = P R^-1: column j by back substitution, x_t for t = j .. 0, kept in A[t][j]
  for (int j = tid; j < rk; j += nth) {
    for (int t = j; t >= 0; --t) {
      double sum = t == j ? 1.0 : 0.0;
      for (int u = t + 1; u <= j; ++u) sum = fma(-Rs[t][piv[u]], A[u][j], sum);
      A[t][j] = sum * rinv[t];
    }
  }
  __syncthreads();
  for (int e = tid; e < c * c; e += nth) T[(e / c) * ldt + (e % c)] = 0.0;
  __syncthreads();
  for (int e = tid; e < rk * rk; e += nth) {
    const int t = e / rk, j = e % rk;
    if (t <= j) T[piv[t] * ldt + j] = A[t][j];
  }
  __syncthreads();
  return PcholResult{rk, s_ref, s_vlast, s_vdrop};
}

template <int SEL>
__global__ void __launch_bounds__(256) k_g_pchol(GPools P) {
  const int g = blockIdx.x, tid = threadIdx.x;
  GState& st = P.st[g];
  const PcholOp op = pchol_op(SEL, P, g);
  extern __shared__ __align__(16) double pc_sm[];
  if (!op.on) {
    // no columns: the widths that follow from an empty basis
    if (tid == 0 && st.status == 0) {
      if (SEL == PC_V1) { st.r = 0; st.r2 = 0; st.m = st.Ku; if (st.m < P.K) st.status = GREST_ERR_NUMERIC; }
      if (SEL == PC_Y2 && st.mode == 4) st.rY2 = 0;
    }
    return;
  }
  const PcholResult res = pchol_block(op.G, op.ldg, op.c, op.tol, op.abs_ref, op.T, op.ldt, pc_sm);
  const int rk = res.rank;
  if (tid == 0) {
    *op.rank_out = rk;
    if (op.stats) {
      st.kept_min = (rk > 0 && res.ref > 0.0) ? sqrt(res.vlast / res.ref) : 0.0;
      st.dropped_max = (res.ref > 0.0 && res.vdrop > 0.0) ? sqrt(res.vdrop / res.ref) : 0.0;
    }
    if (SEL == PC_V1 && rk == 0) { st.r2 = 0; st.m = st.Ku; }
    if (SEL == PC_V2) st.m = st.Ku + rk;
    if ((SEL == PC_V1 || SEL == PC_V2) && st.m < P.K && (SEL == PC_V2 || rk == 0)) st.status = GREST_ERR_NUMERIC;
  }
}

// one problem: info[0] = rank, info[1] = kept_min, info[2] = dropped_max, info[3] = 0
__global__ void __launch_bounds__(256) k_pchol_small(const double* G, int ldg, int c, double tol, double abs_ref,
                                                     const double* abs_ref_ptr, double* T, int ldt, double* info) {
  extern __shared__ __align__(16) double pc_sm[];
  const double ref = abs_ref_ptr ? fabs(abs_ref_ptr[0]) : abs_ref;
  const PcholResult res = pchol_block(G, ldg, c, tol, ref, T, ldt, pc_sm);
  if (threadIdx.x == 0 && info) {
    info[0] = res.rank;
    info[1] = (res.rank > 0 && res.ref > 0.0) ? sqrt(res.vlast / res.ref) : 0.0;
    info[2] = (res.ref > 0.0 && res.vdrop > 0.0) ? sqrt(res.vdrop / res.ref) : 0.0;
    info[3] = 0.0;
  }
}

// ------------------------------------------------------------------ eig
__device__ inline EigOp eig_op(int sel, const GPools& P, int g) {
  const GState& s = P.st[g];
  const SmallLayout L = small_layout(P.K, P.q, P.L, P.cmax, P.mmax);
  double* sm = gsmall(P, g);
  EigOp o{};
  o.on = s.status == 0;
  if (sel == EG_GS) {
    o.A = sm + L.Gs; o.lda = P.q; o.m = s.rY2; o.k = s.rY2 < P.L ? s.rY2 : P.L; o.op = GREST_OP_LAP;
    o.F = sm + L.Uh; o.ldf = P.L; o.theta = sm + L.tmp; o.ritz = nullptr; o.gap = false;
    o.on = o.on && s.mode == 4;
  } else {
    o.A = sm + L.Hm; o.lda = P.mmax; o.m = s.m; o.k = P.K; o.op = P.op;
    o.F = sm + L.Fm; o.ldf = P.K; o.theta = sm + L.thnew; o.ritz = sm + L.ritz; o.gap = true;
  }
  o.on = o.on && o.m > 0 && o.k > 0;
  return o;
}

constexpr int kJacobiSweeps = 40;

// Leading op.k eigenpairs of the symmetric op.m x op.m matrix (symmetrized
// on load) by cyclic Jacobi in one CTA, smem = 2 kMaxW (kMaxW + 1) doubles:
// theta (k), F (m x k) and all m values in tracking order (ritz, nullable).
// Returns the relative gap between tracked values k-1 and k (0 when m <= k).
__device__ double jacobi_block(const EigOp& op, double* eig_sm) {
  const int tid = threadIdx.x, nth = blockDim.x;
  double (*A)[kMaxW + 1] = reinterpret_cast<double (*)[kMaxW + 1]>(eig_sm);
  double (*V)[kMaxW + 1] = reinterpret_cast<double (*)[kMaxW + 1]>(eig_sm + kMaxW * (kMaxW + 1));
  __shared__ double cs[kMaxW / 2], sn[kMaxW / 2];
  __shared__ int pp[kMaxW / 2], qq[kMaxW / 2];
  __shared__ double red[8];
  __shared__ double d[kMaxW];
  __shared__ int asc[kMaxW], trk[kMaxW];
  __shared__ int s_done, s_rot;
  const int m = op.m, mm = (m + 1) & ~1, np = mm / 2;
  for (int e = tid; e < m * m; e += nth) {
    const int i = e / m, j = e % m;
    A[i][j] = 0.5 * (op.A[i * op.lda + j] + op.A[j * op.lda + i]);
    V[i][j] = i == j ? 1.0 : 0.0;
  }
  __syncthreads();
  // ||A||_F^2 (fixed)
  double loc = 0.0;
  for (int e = tid; e < m * m; e += nth) loc += A[e / m][e % m] * A[e / m][e % m];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) loc += __shfl_down_sync(0xffffffffu, loc, o);
  if ((tid & 31) == 0) red[tid >> 5] = loc;
  __syncthreads();
  double fro2 = 0.0;
  for (int w = 0; w < nth / 32; ++w) fro2 += red[w];
  __syncthreads();
  for (int sweep = 0; sweep < kJacobiSweeps && m > 1; ++sweep) {
    double off = 0.0;
    for (int e = tid; e < m * m; e += nth) {
      const int i = e / m, j = e % m;
      if (i != j) off += A[i][j] * A[i][j];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) off += __shfl_down_sync(0xffffffffu, off, o);
    if ((tid & 31) == 0) red[tid >> 5] = off;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int w = 0; w < nth / 32; ++w) t += red[w];
      s_done = !(t > 1e-30 * fro2);
      s_rot = 0;
    }
    __syncthreads();
    if (s_done) break;
    for (int round = 0; round < mm - 1; ++round) {
      if (tid < np) {
        // round-robin tournament: player 0 fixed, players 1..mm-1 rotate
        const int x = tid, y = mm - 1 - tid;
        const int a = x == 0 ? 0 : 1 + (x - 1 + round) % (mm - 1);
        const int b = 1 + (y - 1 + round) % (mm - 1);
        const int p = a < b ? a : b, q = a < b ? b : a;
        double c = 1.0, s = 0.0;
        if (q < m) {
          const double apq = A[p][q];
          // threshold Jacobi: entries below the rounding level of their
          // diagonal are left alone (|apq| > 1e-18 sqrt|a_pp a_qq|, squared)
          if (apq * apq > 1e-36 * fabs(A[p][p] * A[q][q]) && apq != 0.0) {
            s_rot = 1;
            // the rotation's scalars with reciprocal square roots and Newton
            // reciprocals, whose serial chain is several times shorter than
            // IEEE square roots and divisions on the FP64 pipe
            const double tau = (A[q][q] - A[p][p]) * rcp_newton(2.0 * apq);
            const double at = fabs(tau);
            // t = sign(tau) / (|tau| + sqrt(1 + tau^2)); for |tau| >= 2^500,
            // 1 / (2 |tau|) (tau^2 would overflow; the relative error is below 2^-1000)
            double t;
            if (at < 0x1p500) {
              const double u = fma(tau, tau, 1.0);
              t = rcp_newton(fma(u, rsqrt(u), at));
            } else {
              t = rcp_newton(2.0 * at);
            }
            t = tau >= 0.0 ? t : -t;
            c = rsqrt(fma(t, t, 1.0));
            s = t * c;
          }
        }
        pp[tid] = p;
        qq[tid] = q;
        cs[tid] = c;
        sn[tid] = s;
      }
      __syncthreads();
      // rows p, q <- J^T A
      for (int e = tid; e < np * m; e += nth) {
        const int i = e / m, l = e % m, p = pp[i], q = qq[i];
        if (q >= m || sn[i] == 0.0) continue;
        const double ap = A[p][l], aq = A[q][l];
        A[p][l] = cs[i] * ap - sn[i] * aq;
        A[q][l] = sn[i] * ap + cs[i] * aq;
      }
      __syncthreads();
      // columns p, q <- A J, V J
      for (int e = tid; e < np * m; e += nth) {
        const int i = e / m, l = e % m, p = pp[i], q = qq[i];
        if (q >= m || sn[i] == 0.0) continue;
        const double ap = A[l][p], aq = A[l][q];
        A[l][p] = cs[i] * ap - sn[i] * aq;
        A[l][q] = sn[i] * ap + cs[i] * aq;
        const double vp = V[l][p], vq = V[l][q];
        V[l][p] = cs[i] * vp - sn[i] * vq;
        V[l][q] = sn[i] * vp + cs[i] * vq;
      }
      __syncthreads();
      if (tid < np && qq[tid] < m && sn[tid] != 0.0) {
        A[pp[tid]][qq[tid]] = 0.0;
        A[qq[tid]][pp[tid]] = 0.0;
      }
      __syncthreads();
    }
    if (!s_rot) break;  // a sweep without rotations changes nothing more
    __syncthreads();
  }
  for (int i = tid; i < m; i += nth) d[i] = A[i][i];
  __syncthreads();
  // ascending positions (ties: lower index), then the tracking order of Alg. 1 / Sec. 2
  for (int i = tid; i < m; i += nth) {
    int a = 0;
    for (int j = 0; j < m; ++j) a += (d[j] < d[i] || (d[j] == d[i] && j < i)) ? 1 : 0;
    asc[i] = a;
  }
  __syncthreads();
  for (int i = tid; i < m; i += nth) {
    int t = 0;
    for (int j = 0; j < m; ++j) {
      bool before;
      if (op.op == GREST_OP_ADJ)
        before = fabs(d[j]) > fabs(d[i]) || (fabs(d[j]) == fabs(d[i]) && (d[j] > d[i] || (d[j] == d[i] && asc[j] < asc[i])));
      else
        before = d[j] > d[i] || (d[j] == d[i] && asc[j] < asc[i]);
      t += before ? 1 : 0;
    }
    trk[i] = t;
  }
  __syncthreads();
  for (int i = tid; i < m; i += nth) {
    const int t = trk[i];
    if (op.ritz) op.ritz[t] = d[i];
    if (t < op.k) op.theta[t] = d[i];
  }
  for (int e = tid; e < m * m; e += nth) {
    const int l = e / m, i = e % m, t = trk[i];
    if (t < op.k) op.F[l * op.ldf + t] = V[l][i];
  }
  __syncthreads();
  double gap = 0.0;
  if (op.gap && m > op.k) {
    int ia = 0, ib = 0;
    for (int i = 0; i < m; ++i) {
      if (trk[i] == op.k - 1) ia = i;
      if (trk[i] == op.k) ib = i;
    }
    double top = 0.0;
    for (int i = 0; i < m; ++i)
      if (trk[i] == 0) top = fabs(d[i]);
    const double x = op.op == GREST_OP_ADJ ? fabs(d[ia]) : d[ia], y = op.op == GREST_OP_ADJ ? fabs(d[ib]) : d[ib];
    gap = fabs(x - y) / fmax(top, 1e-300);
  }
  __syncthreads();
  return gap;
}

template <int SEL>
__global__ void __launch_bounds__(256) k_g_eig(GPools P) {
  const int g = blockIdx.x;
  GState& st = P.st[g];
  const EigOp op = eig_op(SEL, P, g);
  if (!op.on) return;
  extern __shared__ __align__(16) double eig_sm[];
  const double gap = jacobi_block(op, eig_sm);
  if (threadIdx.x == 0) {
    if (SEL == EG_GS) {
      st.Lp = op.k;
      st.cb = op.k;
      st.cw = st.Ku + op.k;
    } else {
      st.boundary_gap = gap;
    }
  }
}

// one problem (plain pointers): info[0] = the gap, when info is given
__global__ void __launch_bounds__(256) k_eig_small(EigOp op, double* info) {
  extern __shared__ __align__(16) double eig_sm[];
  const double gap = jacobi_block(op, eig_sm);
  if (threadIdx.x == 0 && info) info[0] = gap;
}

template <int SEL>
int gram_one(const GPools& P, cudaStream_t s) {
  k_g_gram<SEL><<<dim3(kPch, P.G), 256, 0, s>>>(P);
  k_g_gram_reduce<SEL><<<P.G, 256, 0, s>>>(P);
  return 2;
}

template <int SEL>
int gemm_one(const GPools& P, const LaunchShape& ls, cudaStream_t s) {
  k_g_gemm<SEL><<<dim3(ls.gemm_blocks, P.G), 256, 0, s>>>(P);
  return 1;
}

template <int SEL>
int spmm_one(const GPools& P, const LaunchShape& ls, cudaStream_t s) {
  const int w = SEL == SP_Y1 ? P.K : (SEL == SP_OM ? P.q : P.cmax);  // the widest the stage can be
  const dim3 grid(ls.row_blocks, P.G);
  if (w <= 8)
    k_g_spmm<SEL, 1, 8><<<grid, 256, 0, s>>>(P);
  else if (w <= 16)
    k_g_spmm<SEL, 1, 16><<<grid, 256, 0, s>>>(P);
  else if (w <= 32)
    k_g_spmm<SEL, 1, 32><<<grid, 256, 0, s>>>(P);
  else
    k_g_spmm<SEL, 2, 32><<<grid, 256, 0, s>>>(P);
  return 1;
}

constexpr size_t kEigSmem = sizeof(double) * 2 * kMaxW * (kMaxW + 1);

}  // namespace

bool prepare_kernels() {
  return reserve_dynamic_smem(k_g_eig<EG_GS>, kEigSmem) && reserve_dynamic_smem(k_g_eig<EG_H>, kEigSmem) &&
         reserve_dynamic_smem(k_g_pchol<PC_Y1>, kEigSmem) && reserve_dynamic_smem(k_g_pchol<PC_Y2>, kEigSmem) &&
         reserve_dynamic_smem(k_g_pchol<PC_V1>, kEigSmem) && reserve_dynamic_smem(k_g_pchol<PC_V2>, kEigSmem);
}

}  // namespace grp

int pchol_small_f64(const double* G, int ldg, int c, double tol, double abs_ref, const double* abs_ref_ptr, double* T,
                    int ldt, double* info, cudaStream_t s) {
  if (c < 1 || c > grp::kMaxW || !reserve_dynamic_smem(grp::k_pchol_small, grp::kEigSmem)) return -1;
  grp::k_pchol_small<<<1, 256, grp::kEigSmem, s>>>(G, ldg, c, tol, abs_ref, abs_ref_ptr, T, ldt, info);
  return 1;
}

int eig_small_f64(const double* A, int lda, int m, int k, int op, double* theta, double* F, int ldf, double* ritz,
                  double* info, cudaStream_t s) {
  if (m < 1 || m > grp::kMaxW || k < 1 || k > m || !reserve_dynamic_smem(grp::k_eig_small, grp::kEigSmem)) return -1;
  grp::EigOp o{};
  o.A = A;
  o.lda = lda;
  o.m = m;
  o.k = k;
  o.op = op;
  o.F = F;
  o.ldf = ldf;
  o.theta = theta;
  o.ritz = ritz;
  o.gap = info != nullptr;
  o.on = true;
  grp::k_eig_small<<<1, 256, grp::kEigSmem, s>>>(o, info);
  return 1;
}

namespace grp {

int launch_spmm(int sel, const GPools& P, const LaunchShape& ls, cudaStream_t s) {
  switch (sel) {
    case SP_Y1: return spmm_one<SP_Y1>(P, ls, s);
    case SP_OM: return spmm_one<SP_OM>(P, ls, s);
    case SP_S2: return spmm_one<SP_S2>(P, ls, s);
    default: return spmm_one<SP_MQ>(P, ls, s);
  }
}

int launch_gram(int sel, const GPools& P, cudaStream_t s) {
  switch (sel) {
    case GR_C: return gram_one<GR_C>(P, s);
    case GR_PW: return gram_one<GR_PW>(P, s);
    case GR_PB: return gram_one<GR_PB>(P, s);
    case GR_PY: return gram_one<GR_PY>(P, s);
    case GR_GY: return gram_one<GR_GY>(P, s);
    case GR_GY2: return gram_one<GR_GY2>(P, s);
    case GR_XTM: return gram_one<GR_XTM>(P, s);
    case GR_GS: return gram_one<GR_GS>(P, s);
    case GR_PV: return gram_one<GR_PV>(P, s);
    case GR_GV: return gram_one<GR_GV>(P, s);
    case GR_PV2: return gram_one<GR_PV2>(P, s);
    case GR_GV2: return gram_one<GR_GV2>(P, s);
    default: return gram_one<GR_H>(P, s);
  }
}

int launch_gemm(int sel, const GPools& P, const LaunchShape& ls, cudaStream_t s) {
  switch (sel) {
    case GM_W: return gemm_one<GM_W>(P, ls, s);
    case GM_PW: return gemm_one<GM_PW>(P, ls, s);
    case GM_PB: return gemm_one<GM_PB>(P, ls, s);
    case GM_PY: return gemm_one<GM_PY>(P, ls, s);
    case GM_QY: return gemm_one<GM_QY>(P, ls, s);
    case GM_QY2: return gemm_one<GM_QY2>(P, ls, s);
    case GM_ETM: return gemm_one<GM_ETM>(P, ls, s);
    case GM_R: return gemm_one<GM_R>(P, ls, s);
    case GM_PV: return gemm_one<GM_PV>(P, ls, s);
    case GM_QV: return gemm_one<GM_QV>(P, ls, s);
    case GM_PV2: return gemm_one<GM_PV2>(P, ls, s);
    case GM_QV2: return gemm_one<GM_QV2>(P, ls, s);
    default: return gemm_one<GM_LIFT>(P, ls, s);
  }
}

int launch_pchol(int sel, const GPools& P, cudaStream_t s) {
  switch (sel) {
    case PC_Y1: k_g_pchol<PC_Y1><<<P.G, 256, kEigSmem, s>>>(P); break;
    case PC_Y2: k_g_pchol<PC_Y2><<<P.G, 256, kEigSmem, s>>>(P); break;
    case PC_V1: k_g_pchol<PC_V1><<<P.G, 256, kEigSmem, s>>>(P); break;
    default: k_g_pchol<PC_V2><<<P.G, 256, kEigSmem, s>>>(P); break;
  }
  return 1;
}

int launch_eig(int sel, const GPools& P, cudaStream_t s) {
  if (sel == EG_GS) k_g_eig<EG_GS><<<P.G, 256, kEigSmem, s>>>(P);
  else k_g_eig<EG_H><<<P.G, 256, kEigSmem, s>>>(P);
  return 1;
}

}  // namespace grp
}  // namespace grest
