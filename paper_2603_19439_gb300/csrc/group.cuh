// Grouped update of many small graphs (grest_group_*): one launch per stage
// of Alg. 2 for every graph of the group, with each graph's shapes (node
// count, ranks, basis width m) kept on the device, so that a whole update of
// the group has no host synchronization and is captured once as a CUDA
// graph.  Graph g's rows live at node_off[g] in packed per-node pools; its
// small matrices in a fixed per-graph slot; every kernel takes the problem
// index from the grid and resolves its operands through the stage selectors
// below.  FP64 throughout; unweighted graphs; no node removal.
#pragma once
#include "common.cuh"

namespace grest {
namespace grp {

constexpr int kMaxW = 64;     // largest block width (q, cmax, mmax <= 64)
constexpr int kPch = 8;       // row chunks of a grouped Gram (fixed: results do not depend on the group)
constexpr int kGramRows = 32; // rows per staged slab

struct GMeta {                // per graph, fixed at creation
  uint64_t seed;              // key of the generator of Omega (the graph's configuration)
  int64_t node_off, node_cap; // rows in the per-node pools
  int64_t edge_off, edge_cap; // entries in the column arena
  int64_t stage_off, stage_cap;  // merged-row staging
  int64_t ent_off, ent_cap;   // batch entries (both directions of every edit)
};

struct GRound {               // per graph and round, written by the host
  int64_t edit_off;           // [ins_u | ins_v | del_u | del_v] in the edit buffer
  int32_t S, n_ins, n_del, pad;
};

struct GState {               // per graph, device resident
  int64_t N, nnz, arena_top, step;
  int32_t status;             // grest_status of the round (graph unchanged when set before the commit)
  int32_t S, mode;            // mode: 2 no new-node block, 3 exact block, 4 RSVD block
  int32_t Ku, cb, cw, r, r2, rY, rY2, Lp, m;
  double dmax, ref, kept_min, dropped_max, boundary_gap;
};

struct GPools {               // passed by value to every grouped kernel
  int G, K, q, L, op, subspace;
  int ldu, ldz, ldq, cmax, mmax;
  int64_t small_stride;
  double drop_tol;
  uint64_t seed;
  const GMeta* meta;
  const GRound* round;
  GState* st;
  const int32_t* edits;
  // graph (per-node pools and arena)
  int64_t* row_off;
  int32_t *row_len, *row_cap, *col;
  double *deg, *dis;
  // graph-update scratch
  int32_t *cnt, *touched, *new_len;
  int64_t *seg, *stg_off, *need;
  uint64_t* ent;
  int32_t* stage;
  // dense per-node pools (row-major)
  double *U, *Un, *Z, *MZ, *V2, *Yr, *Yr2, *Om, *EtM;
  double* small;              // per-graph small matrices
  double* part;               // per-graph Gram partials: kPch x kMaxW x kMaxW
  // launch shapes chosen by the autotuner (bit-identical alternatives)
  int spmm_rows_per_warp;
};

// per-graph small-matrix slot layout (offsets in doubles)
struct SmallLayout {
  int64_t Cm, Cv, Gm, Tm, Hm, Fm, XtM, Gs, Uh, ritz, theta, thnew, tmp, total;
};
__host__ __device__ inline SmallLayout small_layout(int K, int q, int L, int cmax, int mmax) {
  SmallLayout s;
  int64_t o = 0;
  s.Cm = o; o += (int64_t)K * K;
  s.Cv = o; o += (int64_t)K * cmax;
  s.Gm = o; o += (int64_t)cmax * cmax;
  s.Tm = o; o += (int64_t)cmax * cmax;
  s.Hm = o; o += (int64_t)mmax * mmax;
  s.Fm = o; o += (int64_t)mmax * K;
  s.XtM = o; o += (int64_t)K * q;
  s.Gs = o; o += (int64_t)q * q;
  s.Uh = o; o += (int64_t)q * L;
  s.ritz = o; o += mmax;
  s.theta = o; o += K;
  s.thnew = o; o += K;
  s.tmp = o; o += kMaxW;
  s.total = (o + 31) / 32 * 32;
  return s;
}

// ---------------------------------------------------------------- selectors
enum GramSel { GR_C, GR_PW, GR_PB, GR_PY, GR_GY, GR_GY2, GR_XTM, GR_GS, GR_PV, GR_GV, GR_PV2, GR_GV2, GR_H };
enum GemmSel { GM_W, GM_PW, GM_PB, GM_PY, GM_QY, GM_QY2, GM_ETM, GM_R, GM_PV, GM_QV, GM_PV2, GM_QV2, GM_LIFT };
enum SpmmSel { SP_Y1, SP_OM, SP_S2, SP_MQ };
enum PcholSel { PC_Y1, PC_Y2, PC_V1, PC_V2 };
enum EigSel { EG_GS, EG_H };

struct GramOp {               // C (a x b, ldc) = X^T Y over rows [0, n)
  const double *X, *Y;
  int64_t ldx, ldy, n;
  int a, b, ldc;
  double* C;
  bool on;
};
struct GemmOp {               // Out = beta Cin + alpha X B over rows [0, n)
  const double *X, *B, *Cin;
  double* Out;
  int64_t ldx, ldo, ldc, n;
  int a, c, ldb;
  double alpha, beta;
  bool on;
};
struct SpmmOp {               // Y = M X (rows r0..r1 of M, X rows shifted by col_lo)
  const double* X;
  double* Y;
  int64_t ldx, ldy, r0, r1, col_lo;
  int w;
  bool on;
};
struct PcholOp {              // pivoted Cholesky of G (c x c, ldg) -> T (c x rank, ldt)
  const double* G;
  double* T;
  int c, ldg, ldt;
  double tol, abs_ref;
  int32_t* rank_out;
  bool stats;
  bool on;
};
struct EigOp {                // leading k pairs of A (m x m) in the tracking order of `op`
  const double* A;
  int m, lda, k, op;
  double *F, *theta, *ritz;
  int ldf;
  bool gap;
  bool on;
};

__device__ __forceinline__ double* gsmall(const GPools& P, int g) { return P.small + (int64_t)g * P.small_stride; }

__device__ inline GramOp gram_op(int sel, const GPools& P, int g) {
  const GState& s = P.st[g];
  const GMeta& mt = P.meta[g];
  const SmallLayout L = small_layout(P.K, P.q, P.L, P.cmax, P.mmax);
  double* sm = gsmall(P, g);
  const int64_t ro = mt.node_off;
  double* Z = P.Z + ro * P.ldz;
  double* MZ = P.MZ + ro * P.ldz;
  GramOp o{};
  o.on = s.status == 0;
  o.n = s.N;
  o.ldx = P.ldz;
  o.ldy = P.ldz;
  o.X = Z;
  o.a = s.Ku;
  switch (sel) {
    case GR_C: o.Y = MZ; o.b = s.Ku; o.C = sm + L.Cm; o.ldc = P.K; break;
    case GR_PW: o.Y = Z + s.Ku; o.b = s.Ku; o.C = sm + L.Cv; o.ldc = P.cmax; break;
    case GR_PB: o.Y = Z + 2 * s.Ku; o.b = s.cb; o.C = sm + L.Cv; o.ldc = P.cmax; o.on = o.on && s.mode == 3; break;
    case GR_PY: o.Y = P.Yr + ro * P.ldq; o.ldy = P.ldq; o.b = P.q; o.C = sm + L.Cv; o.ldc = P.cmax;
      o.on = o.on && s.mode == 4; break;
    case GR_GY: o.X = o.Y = P.Yr + ro * P.ldq; o.ldx = o.ldy = P.ldq; o.a = o.b = P.q; o.C = sm + L.Gm; o.ldc = P.cmax;
      o.on = o.on && s.mode == 4; break;
    case GR_GY2: o.X = o.Y = P.Yr2 + ro * P.ldq; o.ldx = o.ldy = P.ldq; o.a = o.b = s.rY; o.C = sm + L.Gm;
      o.ldc = P.cmax; o.on = o.on && s.mode == 4; break;
    case GR_XTM: o.Y = P.Yr + ro * P.ldq; o.ldy = P.ldq; o.b = s.rY2; o.C = sm + L.XtM; o.ldc = P.q;
      o.on = o.on && s.mode == 4; break;
    case GR_GS: o.X = o.Y = P.EtM + ro * P.ldq; o.ldx = o.ldy = P.ldq; o.a = o.b = s.rY2; o.n = s.S; o.C = sm + L.Gs;
      o.ldc = P.q; o.on = o.on && s.mode == 4; break;
    case GR_PV: o.Y = Z + s.Ku; o.b = s.cw; o.C = sm + L.Cv; o.ldc = P.cmax; break;
    case GR_GV: o.X = o.Y = Z + s.Ku; o.a = o.b = s.cw; o.C = sm + L.Gm; o.ldc = P.cmax; break;
    case GR_PV2: o.Y = P.V2 + ro * P.ldz; o.b = s.r; o.C = sm + L.Cv; o.ldc = P.cmax; break;
    case GR_GV2: o.X = o.Y = P.V2 + ro * P.ldz; o.a = o.b = s.r; o.C = sm + L.Gm; o.ldc = P.cmax; break;
    default: /* GR_H */ o.Y = MZ; o.a = o.b = s.m; o.C = sm + L.Hm; o.ldc = P.mmax; break;
  }
  o.on = o.on && o.a > 0 && o.b > 0 && o.n > 0;
  return o;
}

__device__ inline GemmOp gemm_op(int sel, const GPools& P, int g) {
  const GState& s = P.st[g];
  const GMeta& mt = P.meta[g];
  const SmallLayout L = small_layout(P.K, P.q, P.L, P.cmax, P.mmax);
  double* sm = gsmall(P, g);
  const int64_t ro = mt.node_off;
  double* Z = P.Z + ro * P.ldz;
  double* MZ = P.MZ + ro * P.ldz;
  double* Yr = P.Yr + ro * P.ldq;
  double* Yr2 = P.Yr2 + ro * P.ldq;
  double* V2 = P.V2 + ro * P.ldz;
  GemmOp o{};
  o.on = s.status == 0;
  o.n = s.N;
  o.X = Z;
  o.ldx = P.ldz;
  o.ldo = o.ldc = P.ldz;
  o.a = s.Ku;
  o.alpha = -1.0;
  o.beta = 1.0;
  switch (sel) {
    case GM_W: o.Cin = MZ; o.Out = Z + s.Ku; o.B = sm + L.Cm; o.ldb = P.K; o.c = s.Ku; break;
    case GM_PW: o.Cin = o.Out = Z + s.Ku; o.B = sm + L.Cv; o.ldb = P.cmax; o.c = s.Ku; break;
    case GM_PB: o.Cin = o.Out = Z + 2 * s.Ku; o.B = sm + L.Cv; o.ldb = P.cmax; o.c = s.cb; o.on = o.on && s.mode == 3;
      break;
    case GM_PY: o.Cin = o.Out = Yr; o.ldo = o.ldc = P.ldq; o.B = sm + L.Cv; o.ldb = P.cmax; o.c = P.q;
      o.on = o.on && s.mode == 4; break;
    case GM_QY: o.X = Yr; o.ldx = P.ldq; o.a = P.q; o.Out = Yr2; o.ldo = P.ldq; o.Cin = nullptr; o.B = sm + L.Tm;
      o.ldb = P.cmax; o.c = s.rY; o.alpha = 1.0; o.beta = 0.0; o.on = o.on && s.mode == 4; break;
    case GM_QY2: o.X = Yr2; o.ldx = P.ldq; o.a = s.rY; o.Out = Yr; o.ldo = P.ldq; o.Cin = nullptr; o.B = sm + L.Tm;
      o.ldb = P.cmax; o.c = s.rY2; o.alpha = 1.0; o.beta = 0.0; o.on = o.on && s.mode == 4; break;
    case GM_ETM: o.X = MZ + (int64_t)(s.N - s.S) * P.ldz; o.n = s.S; o.Cin = o.Out = P.EtM + ro * P.ldq;
      o.ldo = o.ldc = P.ldq;
      o.B = sm + L.XtM; o.ldb = P.q; o.c = s.rY2; o.on = o.on && s.mode == 4; break;
    case GM_R: o.X = Yr; o.ldx = P.ldq; o.a = s.rY2; o.Out = Z + 2 * s.Ku; o.Cin = nullptr; o.B = sm + L.Uh;
      o.ldb = P.L; o.c = s.Lp; o.alpha = 1.0; o.beta = 0.0; o.on = o.on && s.mode == 4; break;
    case GM_PV: o.Cin = o.Out = Z + s.Ku; o.B = sm + L.Cv; o.ldb = P.cmax; o.c = s.cw; break;
    case GM_QV: o.X = Z + s.Ku; o.a = s.cw; o.Out = V2; o.Cin = nullptr; o.B = sm + L.Tm; o.ldb = P.cmax; o.c = s.r;
      o.alpha = 1.0; o.beta = 0.0; break;
    case GM_PV2: o.Cin = o.Out = V2; o.B = sm + L.Cv; o.ldb = P.cmax; o.c = s.r; break;
    case GM_QV2: o.X = V2; o.a = s.r; o.Out = Z + s.Ku; o.Cin = nullptr; o.B = sm + L.Tm; o.ldb = P.cmax; o.c = s.r2;
      o.alpha = 1.0; o.beta = 0.0; break;
    default: /* GM_LIFT */ o.a = s.m; o.Out = P.Un + ro * P.ldu; o.ldo = P.ldu; o.Cin = nullptr; o.B = sm + L.Fm;
      o.ldb = P.K; o.c = P.K; o.alpha = 1.0; o.beta = 0.0; break;
  }
  o.on = o.on && o.n > 0 && o.c > 0;
  return o;
}

__device__ inline SpmmOp spmm_op(int sel, const GPools& P, int g) {
  const GState& s = P.st[g];
  const int64_t ro = P.meta[g].node_off;
  SpmmOp o{};
  o.on = s.status == 0;
  o.r0 = 0;
  o.r1 = s.N;
  o.col_lo = 0;
  switch (sel) {
    case SP_Y1: o.X = P.Z + ro * P.ldz; o.ldx = P.ldz; o.Y = P.MZ + ro * P.ldz; o.ldy = P.ldz; o.w = s.Ku; break;
    case SP_OM: o.X = P.Om + ro * P.ldq; o.ldx = P.ldq; o.Y = P.Yr + ro * P.ldq; o.ldy = P.ldq; o.w = P.q;
      o.col_lo = s.N - s.S; o.on = o.on && s.mode == 4; break;
    case SP_S2: o.X = P.Yr + ro * P.ldq; o.ldx = P.ldq; o.Y = P.EtM + ro * P.ldq; o.ldy = P.ldq; o.w = s.rY2;
      o.r0 = s.N - s.S; o.on = o.on && s.mode == 4; break;
    default: /* SP_MQ */ o.X = P.Z + ro * P.ldz + s.Ku; o.ldx = P.ldz; o.Y = P.MZ + ro * P.ldz + s.Ku; o.ldy = P.ldz;
      o.w = s.r2; break;
  }
  o.on = o.on && o.w > 0 && o.r1 > o.r0;
  return o;
}

}  // namespace grp

// group_kernels.cu: launchers of the grouped stages (each returns its launch count)
namespace grp {
struct LaunchShape {
  int row_blocks;   // grid.x of the row-parallel stages (SpMM, pad, new-node columns, Omega)
  int gemm_blocks;  // grid.x of the grouped GEMMs
};
int launch_update(const GPools& P, cudaStream_t s);
int launch_pad(const GPools& P, const LaunchShape& ls, cudaStream_t s);
int launch_spmm(int sel, const GPools& P, const LaunchShape& ls, cudaStream_t s);
int launch_newcols(const GPools& P, const LaunchShape& ls, cudaStream_t s);
int launch_omega(const GPools& P, const LaunchShape& ls, cudaStream_t s);
int launch_gram(int sel, const GPools& P, cudaStream_t s);
int launch_gemm(int sel, const GPools& P, const LaunchShape& ls, cudaStream_t s);
int launch_pchol(int sel, const GPools& P, cudaStream_t s);
int launch_eig(int sel, const GPools& P, cudaStream_t s);
int launch_finish(const GPools& P, cudaStream_t s);
bool prepare_kernels();  // dynamic shared memory limits; false when the device cannot run them
}  // namespace grp

}  // namespace grest
