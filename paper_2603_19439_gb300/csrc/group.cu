// grest_group_*: the grouped update of many small graphs (declared in
// include/grest.h).  A group is loaded from checkpoints (grest_checkpoint) of
// contexts that share K, the operator and L, P; each update of the group is
// Alg. 2's step for every graph at once, as a fixed sequence of grouped
// launches (group_update.cu, group_dense.cu) that reads every shape from
// device memory.  The sequence is captured once as a CUDA graph and replayed
// for every later update; the host copies the batches in before the replay
// and reads the per-graph states back after it (one synchronization per
// update of the whole group).  After the first update an autotuner times the
// launch shapes of the SpMM and GEMM stages that give bit-identical results
// (which warp takes which rows) and keeps the fastest per shape bucket.
#include <string.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "group.cuh"

using namespace grest;
using namespace grest::grp;

struct grest_group {
  int dev = 0;
  cudaStream_t stream = nullptr;
  GPools P{};
  std::vector<GMeta> meta;
  std::vector<void*> bufs;
  GRound* round_h = nullptr;
  GRound* round_d = nullptr;
  GState* st_h = nullptr;
  int32_t* edits_h = nullptr;
  int32_t* edits_d = nullptr;
  int64_t edit_cap = 0;
  LaunchShape ls{};
  cudaGraphExec_t exec = nullptr;
  int launches = 0;
  bool tuned = false;
  int64_t total_rows = 0;
};

namespace {

inline int64_t rup(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

template <typename T>
cudaError_t galloc(grest_group* G, T** p, size_t count) {
  *p = nullptr;
  void* q = nullptr;
  const cudaError_t e = cudaMalloc(&q, sizeof(T) * (count ? count : 1));
  if (e != cudaSuccess) return e;
  G->bufs.push_back(q);
  *p = static_cast<T*>(q);
  return cudaMemsetAsync(q, 0, sizeof(T) * (count ? count : 1), G->stream);
}

void free_group(grest_group* G) {
  if (!G) return;
  if (G->exec) cudaGraphExecDestroy(G->exec);
  for (void* p : G->bufs) cudaFree(p);
  if (G->round_h) cudaFreeHost(G->round_h);
  if (G->st_h) cudaFreeHost(G->st_h);
  if (G->edits_h) cudaFreeHost(G->edits_h);
  if (G->edits_d) cudaFree(G->edits_d);
  if (G->stream) cudaStreamDestroy(G->stream);
  delete G;
}

grest_status from_cuda(cudaError_t e) {
  if (e == cudaSuccess) return GREST_OK;
  if (e == cudaErrorMemoryAllocation) return GREST_ERR_OOM;
  return GREST_ERR_CUDA;
}

#define GK(x)                                    \
  do {                                           \
    cudaError_t e_ = (x);                        \
    if (e_ != cudaSuccess) return from_cuda(e_); \
  } while (0)

// Launch shapes by shape bucket (graphs, rows, widths), chosen by the
// autotuner; process-wide so later groups of the same shape reuse them.
struct TuneKey {
  int G, K, q, rows_log2;
  bool operator==(const TuneKey& o) const { return G == o.G && K == o.K && q == o.q && rows_log2 == o.rows_log2; }
};
struct TuneVal {
  int spmm_blocks, rows_per_warp, gemm_blocks;
};
std::mutex& tune_mutex() {
  static std::mutex m;
  return m;
}
std::vector<std::pair<TuneKey, TuneVal>>& tune_table() {
  static std::vector<std::pair<TuneKey, TuneVal>> t;
  return t;
}

TuneKey tune_key(const grest_group* G) {
  int l = 0;
  while ((int64_t(1) << (l + 1)) <= G->total_rows) ++l;
  return TuneKey{G->P.G, G->P.K, G->P.q, l};
}

}  // namespace

// ------------------------------------------------------------------ creation

grest_status grest_group_create(int32_t n_graphs, const void* const* ckpts, const int64_t* ckpt_bytes,
                                double capacity_factor, grest_group** out) {
  if (!out || n_graphs < 1 || !ckpts || !ckpt_bytes) return GREST_ERR_INVALID_ARG;
  *out = nullptr;
  if (!(capacity_factor >= 1.0) || capacity_factor > 64.0) return GREST_ERR_INVALID_ARG;
  std::vector<CkptView> v(n_graphs);
  for (int g = 0; g < n_graphs; ++g)
    if (!ckpts[g] || !ckpt_view(ckpts[g], ckpt_bytes[g], &v[g])) return GREST_ERR_INVALID_ARG;
  const grest_config& c0 = v[0].cfg;
  for (int g = 0; g < n_graphs; ++g) {
    const grest_config& c = v[g].cfg;
    if (c.k != c0.k || c.op != c0.op || c.L != c0.L || c.P != c0.P || c.subspace != c0.subspace ||
        c.drop_tol != c0.drop_tol)
      return GREST_ERR_INVALID_ARG;
    if (v[g].has_val || c.projection != GREST_PROJ_EXACT || c.w_block != GREST_WB_RESID) return GREST_ERR_UNSUPPORTED;
    for (int64_t i = 0; i < v[g].n; ++i)
      if (!v[g].live[i]) return GREST_ERR_UNSUPPORTED;  // removed nodes: the single-graph path only
  }
  const int K = c0.k, q = c0.L + c0.P, L = c0.L;
  const int cmax = K + std::max(q, L), mmax = K + cmax;
  if (mmax > kMaxW || q > kMaxW) return GREST_ERR_UNSUPPORTED;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return GREST_ERR_CUDA;
  if (!prepare_kernels()) return GREST_ERR_UNSUPPORTED;
  grest_group* G = new grest_group();
  G->dev = dev;
#define IK(x)                     \
  do {                            \
    cudaError_t e_ = (x);         \
    if (e_ != cudaSuccess) {      \
      free_group(G);              \
      return from_cuda(e_);       \
    }                             \
  } while (0)
  IK(cudaStreamCreateWithFlags(&G->stream, cudaStreamNonBlocking));
  GPools& P = G->P;
  P.G = n_graphs;
  P.K = K;
  P.q = q;
  P.L = L;
  P.op = c0.op;
  P.subspace = c0.subspace;
  P.drop_tol = c0.drop_tol;
  P.seed = c0.seed;
  P.cmax = cmax;
  P.mmax = mmax;
  P.ldu = (int)rup(K, 4);
  P.ldz = (int)rup(mmax, 4);
  P.ldq = (int)rup(q, 4);
  P.spmm_rows_per_warp = 1;
  const SmallLayout SL = small_layout(K, q, L, cmax, mmax);
  P.small_stride = SL.total;
  // per-graph capacities: ids and edge slots grow by capacity_factor; a batch
  // may carry up to a quarter of the graph's nonzeros (both directions)
  G->meta.resize(n_graphs);
  int64_t node_tot = 0, edge_tot = 0, stage_tot = 0, ent_tot = 0;
  std::vector<int64_t> slack(n_graphs);
  for (int g = 0; g < n_graphs; ++g) {
    int64_t tot = 0;
    for (int64_t i = 0; i < v[g].n; ++i) {
      const int64_t l = v[g].rowptr[i + 1] - v[g].rowptr[i];
      tot += l + l / 4 + 4;
    }
    slack[g] = tot;
    GMeta& m = G->meta[g];
    m.seed = v[g].cfg.seed;
    m.node_cap = rup((int64_t)(v[g].n * capacity_factor) + 64, 32);
    m.edge_cap = rup((int64_t)(2 * tot * capacity_factor) + 4096, 32);
    m.ent_cap = std::max<int64_t>(8192, v[g].nnz / 4);
    m.stage_cap = m.edge_cap + m.ent_cap;
    m.node_off = node_tot;
    m.edge_off = edge_tot;
    m.stage_off = stage_tot;
    m.ent_off = ent_tot;
    node_tot += m.node_cap;
    edge_tot += m.edge_cap;
    stage_tot += m.stage_cap;
    ent_tot += m.ent_cap;
  }
  G->total_rows = node_tot;
  GMeta* meta_d = nullptr;
  IK(galloc(G, &meta_d, n_graphs));
  IK(cudaMemcpyAsync(meta_d, G->meta.data(), sizeof(GMeta) * n_graphs, cudaMemcpyHostToDevice, G->stream));
  P.meta = meta_d;
  IK(galloc(G, &G->round_d, n_graphs));
  P.round = G->round_d;
  IK(galloc(G, &P.st, n_graphs));
  IK(cudaMallocHost((void**)&G->round_h, sizeof(GRound) * n_graphs));
  IK(cudaMallocHost((void**)&G->st_h, sizeof(GState) * n_graphs));
  IK(galloc(G, &P.row_off, node_tot));
  IK(galloc(G, &P.row_len, node_tot));
  IK(galloc(G, &P.row_cap, node_tot));
  IK(galloc(G, &P.deg, node_tot));
  IK(galloc(G, &P.dis, node_tot));
  IK(galloc(G, &P.cnt, node_tot));
  IK(galloc(G, &P.touched, node_tot));
  IK(galloc(G, &P.new_len, node_tot));
  IK(galloc(G, &P.seg, node_tot + n_graphs));
  IK(galloc(G, &P.stg_off, node_tot + n_graphs));
  IK(galloc(G, &P.need, node_tot + n_graphs));
  IK(galloc(G, &P.col, edge_tot));
  IK(galloc(G, &P.stage, stage_tot));
  IK(galloc(G, &P.ent, ent_tot));
  IK(galloc(G, &P.U, node_tot * P.ldu));
  IK(galloc(G, &P.Un, node_tot * P.ldu));
  IK(galloc(G, &P.Z, node_tot * P.ldz));
  IK(galloc(G, &P.MZ, node_tot * P.ldz));
  IK(galloc(G, &P.V2, node_tot * P.ldz));
  IK(galloc(G, &P.Yr, node_tot * P.ldq));
  IK(galloc(G, &P.Yr2, node_tot * P.ldq));
  IK(galloc(G, &P.Om, node_tot * P.ldq));
  IK(galloc(G, &P.EtM, node_tot * P.ldq));
  IK(galloc(G, &P.small, (size_t)n_graphs * SL.total));
  IK(galloc(G, &P.part, (size_t)n_graphs * kPch * kMaxW * kMaxW));
  IK(cudaStreamSynchronize(G->stream));  // the zero fills above precede the uploads below
  // graphs, pairs and states
  std::vector<GState> st(n_graphs);
  for (int g = 0; g < n_graphs; ++g) {
    const CkptView& w = v[g];
    const GMeta& m = G->meta[g];
    const int64_t n = w.n;
    std::vector<int64_t> off(n);
    std::vector<int32_t> len(n), cap(n), col((size_t)slack[g], 0);
    std::vector<double> Upad((size_t)n * P.ldu, 0.0);
    int64_t o = 0;
    for (int64_t i = 0; i < n; ++i) {
      const int64_t l = w.rowptr[i + 1] - w.rowptr[i];
      off[i] = o;
      len[i] = (int32_t)l;
      cap[i] = (int32_t)(l + l / 4 + 4);
      memcpy(col.data() + o, w.col + w.rowptr[i], sizeof(int32_t) * l);
      o += cap[i];
      for (int j = 0; j < K; ++j) Upad[(size_t)i * P.ldu + j] = w.U[(size_t)i * K + j];
    }
    IK(cudaMemcpy(P.row_off + m.node_off, off.data(), sizeof(int64_t) * n, cudaMemcpyHostToDevice));
    IK(cudaMemcpy(P.row_len + m.node_off, len.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice));
    IK(cudaMemcpy(P.row_cap + m.node_off, cap.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice));
    IK(cudaMemcpy(P.col + m.edge_off, col.data(), sizeof(int32_t) * o, cudaMemcpyHostToDevice));
    IK(cudaMemcpy(P.deg + m.node_off, w.deg, sizeof(double) * n, cudaMemcpyHostToDevice));
    IK(cudaMemcpy(P.U + m.node_off * P.ldu, Upad.data(), sizeof(double) * Upad.size(), cudaMemcpyHostToDevice));
    IK(cudaMemcpy(P.small + (size_t)g * SL.total + SL.theta, w.theta, sizeof(double) * K, cudaMemcpyHostToDevice));
    GState& s = st[g];
    memset(&s, 0, sizeof(s));
    s.N = n;
    s.nnz = w.nnz;
    s.arena_top = o;
    s.step = w.step;
    s.Ku = K;
  }
  IK(cudaMemcpy(P.st, st.data(), sizeof(GState) * n_graphs, cudaMemcpyHostToDevice));
  IK(cudaStreamSynchronize(G->stream));
#undef IK
  int nsm = 152;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  G->ls.row_blocks = nsm * 8;
  G->ls.gemm_blocks = nsm * 8;
  {
    std::lock_guard<std::mutex> lock(tune_mutex());
    const TuneKey k = tune_key(G);
    for (auto& e : tune_table())
      if (e.first == k) {
        G->ls.row_blocks = e.second.spmm_blocks;
        G->ls.gemm_blocks = e.second.gemm_blocks;
        P.spmm_rows_per_warp = e.second.rows_per_warp;
        G->tuned = true;
      }
  }
  *out = G;
  return GREST_OK;
}

// ------------------------------------------------------------------ one update

namespace {

// Alg. 2's step for every graph, in the order of the single-graph update
// (grest.cu): A1 graph update; A2 pad; A3 Y1 = M X_bar; A4 C, W = P_perp Y1
// (projected twice); A5 the exact block P_perp M[:, N:N'] or the RSVD basis
// (S.1 Y = P_perp Delta_2 Omega, CholQR2 with pivoting, S.2 B_s^T, its L
// leading left singular vectors, S.4 R); A6 Q = orth(P_perp [W, B]) by
// CholQR2; A7 MQ; A8 H = Z^T M Z; A9 eig; A10 lift and signs.
int enqueue_step(grest_group* G, cudaStream_t s) {
  const GPools& P = G->P;
  const LaunchShape& ls = G->ls;
  int n = 0;
  n += launch_update(P, s);
  n += launch_pad(P, ls, s);
  n += launch_spmm(SP_Y1, P, ls, s);
  n += launch_gram(GR_C, P, s);
  n += launch_gemm(GM_W, P, ls, s);
  n += launch_gram(GR_PW, P, s);
  n += launch_gemm(GM_PW, P, ls, s);
  // exact new-node block (graphs in mode 3)
  n += launch_newcols(P, ls, s);
  n += launch_gram(GR_PB, P, s);
  n += launch_gemm(GM_PB, P, ls, s);
  // RSVD new-node block (graphs in mode 4)
  n += launch_omega(P, ls, s);
  n += launch_spmm(SP_OM, P, ls, s);
  n += launch_gram(GR_PY, P, s);  // one projection, as in the single-graph update
  n += launch_gemm(GM_PY, P, ls, s);
  n += launch_gram(GR_GY, P, s);
  n += launch_pchol(PC_Y1, P, s);
  n += launch_gemm(GM_QY, P, ls, s);
  n += launch_gram(GR_GY2, P, s);
  n += launch_pchol(PC_Y2, P, s);
  n += launch_gemm(GM_QY2, P, ls, s);
  n += launch_spmm(SP_S2, P, ls, s);
  n += launch_gram(GR_XTM, P, s);
  n += launch_gemm(GM_ETM, P, ls, s);
  n += launch_gram(GR_GS, P, s);
  n += launch_eig(EG_GS, P, s);
  n += launch_gemm(GM_R, P, ls, s);
  // A6: Q = orth(P_perp [W, B]), CholQR2 with pivoting
  n += launch_gram(GR_PV, P, s);
  n += launch_gemm(GM_PV, P, ls, s);
  n += launch_gram(GR_GV, P, s);
  n += launch_pchol(PC_V1, P, s);
  n += launch_gemm(GM_QV, P, ls, s);
  n += launch_gram(GR_PV2, P, s);
  n += launch_gemm(GM_PV2, P, ls, s);
  n += launch_gram(GR_GV2, P, s);
  n += launch_pchol(PC_V2, P, s);
  n += launch_gemm(GM_QV2, P, ls, s);
  // A7 - A10
  n += launch_spmm(SP_MQ, P, ls, s);
  n += launch_gram(GR_H, P, s);
  n += launch_eig(EG_H, P, s);
  n += launch_gemm(GM_LIFT, P, ls, s);
  n += launch_finish(P, s);
  return n;
}

grest_status capture(grest_group* G) {
  if (G->exec) {
    cudaGraphExecDestroy(G->exec);
    G->exec = nullptr;
  }
  cudaGraph_t graph = nullptr;
  GK(cudaStreamBeginCapture(G->stream, cudaStreamCaptureModeThreadLocal));
  const int n = enqueue_step(G, G->stream);
  const cudaError_t e = cudaStreamEndCapture(G->stream, &graph);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return GREST_ERR_CUDA;
  }
  const cudaError_t e2 = cudaGraphInstantiate(&G->exec, graph, 0);
  cudaGraphDestroy(graph);
  GK(e2);
  G->launches = n;
  return GREST_OK;
}

float time_ms(cudaStream_t s, cudaEvent_t a, cudaEvent_t b) {
  cudaEventSynchronize(b);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, a, b);
  (void)s;
  return ms;
}

// Autotuner: on the group's current state (after an update, so every
// graph's shapes are real), time the SpMM of A3 for each (grid, rows per
// warp) and the lift GEMM of A10 for each grid.  Both stages are idempotent
// here (they rewrite outputs that no later stage of the finished update
// reads), and every candidate computes each row with the same arithmetic in
// the same order, so the choice cannot change a result.
grest_status autotune(grest_group* G) {
  int nsm = 152;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, G->dev);
  cudaEvent_t a, b;
  GK(cudaEventCreate(&a));
  GK(cudaEventCreate(&b));
  const int grids[] = {2, 4, 8, 16, 32};
  const int rpws[] = {1, 2, 4};
  float best = 1e30f;
  LaunchShape ls = G->ls;
  int best_rpw = G->P.spmm_rows_per_warp, best_sb = ls.row_blocks, best_gb = ls.gemm_blocks;
  for (int gm : grids)
    for (int rpw : rpws) {
      LaunchShape t = ls;
      t.row_blocks = nsm * gm;
      GPools P = G->P;
      P.spmm_rows_per_warp = rpw;
      float tot = 0.f;
      for (int rep = 0; rep < 4; ++rep) {
        cudaEventRecord(a, G->stream);
        launch_spmm(SP_Y1, P, t, G->stream);
        cudaEventRecord(b, G->stream);
        const float ms = time_ms(G->stream, a, b);
        if (rep > 0) tot += ms;
      }
      if (tot < best) { best = tot; best_rpw = rpw; best_sb = t.row_blocks; }
    }
  best = 1e30f;
  for (int gm : grids) {
    LaunchShape t = ls;
    t.gemm_blocks = nsm * gm;
    float tot = 0.f;
    for (int rep = 0; rep < 4; ++rep) {
      cudaEventRecord(a, G->stream);
      launch_gemm(GM_LIFT, G->P, t, G->stream);
      cudaEventRecord(b, G->stream);
      const float ms = time_ms(G->stream, a, b);
      if (rep > 0) tot += ms;
    }
    if (tot < best) { best = tot; best_gb = t.gemm_blocks; }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  GK(cudaGetLastError());
  G->ls.row_blocks = best_sb;
  G->ls.gemm_blocks = best_gb;
  G->P.spmm_rows_per_warp = best_rpw;
  G->tuned = true;
  std::lock_guard<std::mutex> lock(tune_mutex());
  const TuneKey k = tune_key(G);
  for (auto& e : tune_table())
    if (e.first == k) {
      e.second = TuneVal{best_sb, best_rpw, best_gb};
      return GREST_OK;
    }
  tune_table().push_back({k, TuneVal{best_sb, best_rpw, best_gb}});
  return GREST_OK;
}

}  // namespace

grest_status grest_group_apply_updates(grest_group* G, const grest_update* ups, grest_status* status,
                                       grest_stats* stats) {
  if (!G || !ups) return GREST_ERR_INVALID_ARG;
  const int n = G->P.G;
  int64_t total = 0;
  for (int g = 0; g < n; ++g) {
    const grest_update& u = ups[g];
    if (u.n_new_nodes < 0 || u.n_ins < 0 || u.n_del < 0 || u.n_del_nodes != 0 || u.ins_w || u.on_device)
      return u.n_del_nodes != 0 || u.ins_w || u.on_device ? GREST_ERR_UNSUPPORTED : GREST_ERR_INVALID_ARG;
    if ((u.n_ins > 0 && (!u.ins_u || !u.ins_v)) || (u.n_del > 0 && (!u.del_u || !u.del_v)))
      return GREST_ERR_INVALID_ARG;
    if (u.n_new_nodes > INT32_MAX || u.n_ins > INT32_MAX / 2 || u.n_del > INT32_MAX / 2) return GREST_ERR_CAPACITY;
    total += 2 * (u.n_ins + u.n_del);
  }
  if (cudaSetDevice(G->dev) != cudaSuccess) return GREST_ERR_CUDA;
  cudaStream_t s = G->stream;
  GK(cudaStreamSynchronize(s));
  if (total > G->edit_cap) {  // the edit buffer is read through GPools: a new one needs a new graph
    const int64_t cap = std::max<int64_t>(total, 2 * G->edit_cap);
    if (G->edits_h) cudaFreeHost(G->edits_h);
    if (G->edits_d) cudaFree(G->edits_d);
    G->edits_h = nullptr;
    G->edits_d = nullptr;
    G->edit_cap = 0;
    GK(cudaMallocHost((void**)&G->edits_h, sizeof(int32_t) * cap));
    GK(cudaMalloc((void**)&G->edits_d, sizeof(int32_t) * cap));
    G->edit_cap = cap;
    G->P.edits = G->edits_d;
    if (G->exec) {
      cudaGraphExecDestroy(G->exec);
      G->exec = nullptr;
    }
  }
  int64_t o = 0;
  for (int g = 0; g < n; ++g) {
    const grest_update& u = ups[g];
    GRound& r = G->round_h[g];
    r.edit_off = o;
    r.S = (int32_t)u.n_new_nodes;
    r.n_ins = (int32_t)u.n_ins;
    r.n_del = (int32_t)u.n_del;
    r.pad = 0;
    if (u.n_ins) {
      memcpy(G->edits_h + o, u.ins_u, sizeof(int32_t) * u.n_ins);
      memcpy(G->edits_h + o + u.n_ins, u.ins_v, sizeof(int32_t) * u.n_ins);
    }
    o += 2 * u.n_ins;
    if (u.n_del) {
      memcpy(G->edits_h + o, u.del_u, sizeof(int32_t) * u.n_del);
      memcpy(G->edits_h + o + u.n_del, u.del_v, sizeof(int32_t) * u.n_del);
    }
    o += 2 * u.n_del;
  }
  GK(cudaMemcpyAsync(G->round_d, G->round_h, sizeof(GRound) * n, cudaMemcpyHostToDevice, s));
  if (o > 0) GK(cudaMemcpyAsync(G->edits_d, G->edits_h, sizeof(int32_t) * o, cudaMemcpyHostToDevice, s));
  if (!G->edits_d) {  // no edits yet: any valid pointer will do, nothing is read
    G->P.edits = reinterpret_cast<const int32_t*>(G->round_d);
  }
  if (!G->exec) {
    const grest_status cs = capture(G);
    if (cs != GREST_OK) return cs;
  }
  GK(cudaGraphLaunch(G->exec, s));
  GK(cudaMemcpyAsync(G->st_h, G->P.st, sizeof(GState) * n, cudaMemcpyDeviceToHost, s));
  GK(cudaStreamSynchronize(s));
  GK(cudaGetLastError());
  grest_status first = GREST_OK;
  bool all_ok = true;
  for (int g = 0; g < n; ++g) {
    const GState& st = G->st_h[g];
    const grest_status code = (grest_status)st.status;
    if (status) status[g] = code;
    if (code != GREST_OK) {
      all_ok = false;
      if (first == GREST_OK) first = code;
    }
    if (stats) {
      grest_stats& S = stats[g];
      memset(&S, 0, sizeof(S));
      S.step = st.step;
      S.n_nodes = st.N;
      S.nnz = st.nnz;
      S.m = st.m;
      S.k_u = st.Ku;
      S.rank_q = st.r;
      S.rank_y = st.rY;
      S.mode = st.mode;
      S.pivot_kept_min = st.kept_min;
      S.pivot_dropped_max = st.dropped_max;
      S.boundary_gap = st.boundary_gap;
      S.kernel_launches = G->launches;
    }
  }
  if (!G->tuned && all_ok) {
    const grest_status ts = autotune(G);
    if (ts != GREST_OK) return ts;
    if (G->exec) {  // the next update is captured with the chosen shapes
      cudaGraphExecDestroy(G->exec);
      G->exec = nullptr;
    }
  }
  return first;
}

grest_status grest_group_get_embedding(grest_group* G, int32_t i, double* U, double* theta, int64_t* n_out) {
  if (!G || !n_out || i < 0 || i >= G->P.G) return GREST_ERR_INVALID_ARG;
  if (cudaSetDevice(G->dev) != cudaSuccess) return GREST_ERR_CUDA;
  cudaStream_t s = G->stream;
  GK(cudaStreamSynchronize(s));
  GState st;
  GK(cudaMemcpy(&st, G->P.st + i, sizeof(GState), cudaMemcpyDeviceToHost));
  *n_out = st.N;
  const int K = G->P.K;
  const GMeta& m = G->meta[i];
  if (U && G->P.ldu == K)  // contiguous rows: one linear copy
    GK(cudaMemcpy(U, G->P.U + m.node_off * G->P.ldu, sizeof(double) * K * st.N, cudaMemcpyDeviceToHost));
  else if (U)
    GK(cudaMemcpy2D(U, sizeof(double) * K, G->P.U + m.node_off * G->P.ldu, sizeof(double) * G->P.ldu,
                    sizeof(double) * K, st.N, cudaMemcpyDeviceToHost));
  if (theta) {
    const SmallLayout L = small_layout(K, G->P.q, G->P.L, G->P.cmax, G->P.mmax);
    GK(cudaMemcpy(theta, G->P.small + (size_t)i * G->P.small_stride + L.theta, sizeof(double) * K,
                  cudaMemcpyDeviceToHost));
  }
  return GREST_OK;
}

grest_status grest_group_get_ritz_values(grest_group* G, int32_t i, double* ritz, int32_t* m) {
  if (!G || !m || i < 0 || i >= G->P.G) return GREST_ERR_INVALID_ARG;
  if (cudaSetDevice(G->dev) != cudaSuccess) return GREST_ERR_CUDA;
  GK(cudaStreamSynchronize(G->stream));
  GState st;
  GK(cudaMemcpy(&st, G->P.st + i, sizeof(GState), cudaMemcpyDeviceToHost));
  *m = st.m;
  if (ritz && st.m > 0) {
    const SmallLayout L = small_layout(G->P.K, G->P.q, G->P.L, G->P.cmax, G->P.mmax);
    GK(cudaMemcpy(ritz, G->P.small + (size_t)i * G->P.small_stride + L.ritz, sizeof(double) * st.m,
                  cudaMemcpyDeviceToHost));
  }
  return GREST_OK;
}

grest_status grest_group_info(grest_group* G, int32_t* captured, int32_t* launches_per_update, int32_t* tuned,
                              int32_t* spmm_blocks, int32_t* spmm_rows_per_warp, int32_t* gemm_blocks) {
  if (!G) return GREST_ERR_INVALID_ARG;
  if (captured) *captured = G->exec != nullptr;
  if (launches_per_update) *launches_per_update = G->launches;
  if (tuned) *tuned = G->tuned;
  if (spmm_blocks) *spmm_blocks = G->ls.row_blocks;
  if (spmm_rows_per_warp) *spmm_rows_per_warp = G->P.spmm_rows_per_warp;
  if (gemm_blocks) *gemm_blocks = G->ls.gemm_blocks;
  return GREST_OK;
}

void grest_group_destroy(grest_group* G) {
  if (!G) return;
  cudaSetDevice(G->dev);
  if (G->stream) cudaStreamSynchronize(G->stream);
  free_group(G);
}
