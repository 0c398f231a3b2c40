// libgrest: context, the G-REST step orchestration (Alg. 2), and the C ABI
// declared in include/grest.h.
//
// One update, FP64 path (all on the context's stream):
//   A1  validate + apply Delta to the slack CSR           graph.cu
//   A2  X_bar = [X; 0] (Alg. 2 pad)                       copy / zero
//   A3  Y1 = M X_bar                                      spmm.cu
//   A4  C = X_bar^T Y1, W = P_perp Y1 (two passes)        dense.cu
//   A5  new-node block: B = P_perp Delta_2 (S <= L+P) or
//       the RSVD basis R of steps S.1-S.4 (Sec. 3.5)      rsvd.cu, spmm.cu, dense.cu, eig.cu
//   A6  Q = orth(P_perp [W, B]) by CholQR2 with pivoting  dense.cu
//   A7  MQ = M Q                                          spmm.cu
//   A8  H = Z^T (M Z), Z = [X_bar, Q] (Eq. main2)         dense.cu
//   A9  leading K eigenpairs of H (Alg. 1)                eig.cu
//   A10 X = Z F_K, sign normalization                     dense.cu
// Rank decisions (kept columns) are read back to the host at three points
// so that later launches use the exact widths.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <thread>
#include <vector>

#include "common.cuh"

using namespace grest;

namespace {

inline int64_t round_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

}  // namespace

namespace grest {
std::mutex& smem_attr_mutex() {
  static std::mutex mu;
  return mu;
}

size_t* smem_reserved_slot(const void* kernel, int dev) {  // caller holds smem_attr_mutex()
  struct Slot {
    const void* k;
    int dev;
    size_t bytes;
  };
  static Slot table[256];
  static int used = 0;
  for (int i = 0; i < used; ++i)
    if (table[i].k == kernel && table[i].dev == dev) return &table[i].bytes;
  if (used == 256) return nullptr;
  table[used] = Slot{kernel, dev, 0};
  return &table[used++].bytes;
}
}  // namespace grest

struct grest_ctx {
  grest_config cfg{};
  int dev = 0;
  cudaStream_t stream = nullptr;
  Csr g;
  GraphWork gw;
  int K = 0, q = 0, Lr = 0, cmax = 0, mmax = 0;
  int64_t ldu = 0, ldz = 0, ldq = 0, ldv = 0;
  int64_t step = 0;
  int Ku = 0;            // columns of X currently valid (K unless nodes were removed)
  double* U = nullptr;   // n_cap x ldu
  double* Un = nullptr;  // next U
  double* theta = nullptr;
  // N x w blocks in the step's storage type (double for FP64, float for MIXED)
  size_t esz = 8;
  void* Zv = nullptr;    // n_cap x ldz : [X_bar | W | B/R] -> [X_bar | Q]
  void* MZv = nullptr;   // n_cap x ldz : [Y1 | MQ]
  void* V2v = nullptr;   // n_cap x ldv : CholQR staging
  void* Yrv = nullptr;   // n_cap x ldq : RSVD sketch / basis
  void* Yr2v = nullptr;  // n_cap x ldq
  void* Omv = nullptr;   // S_cap x ldq
  void* EtMv = nullptr;  // S_cap x ldq : rows N.. of M M_rs, then B_s^T
  int64_t S_cap = 0;
  void* Idv = nullptr;   // q x q identity (exact new-node block)
  float* U32 = nullptr;  // mixed path: Ritz vectors before the FP64 refinement (n_cap x ldu)
  double* Rres = nullptr;  // residual vectors for GREST_FLAG_CHECK (n_cap x ldu)
  double *Cm = nullptr, *Cv = nullptr, *G = nullptr, *T = nullptr, *H = nullptr, *F = nullptr, *XtM = nullptr,
         *Gs = nullptr, *Uh = nullptr, *ritz = nullptr, *th_new = nullptr, *tmpk = nullptr;
  double* info = nullptr;  // device diagnostics [64]
  double* resn = nullptr;  // residual norms [64]
  double* part = nullptr;
  int64_t part_cap = 0;
  int64_t* ipart = nullptr;
  int* piv = nullptr;    // pivot order of the pivoted Cholesky (cmax + K ints)
  double* dmax_old = nullptr;   // d_max before the update (DELTA / LOWRANK modes)
  double* XZ = nullptr;         // X_bar^T Z (LOWRANK mode), 64 x mmax
  uint8_t* gemm_img = nullptr;  // tensor-core GEMM: B^T operand images
  size_t gemm_img_cap = 0;
  // second lane of the step (large graphs with an RSVD new-node block): a
  // high-priority stream and its own Gram / GEMM scratch, so that the RSVD
  // sketch (A5, S.1) runs beside A3 and A4 (see step_t)
  cudaStream_t s2 = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  double* part2 = nullptr;
  uint8_t* gemm_img2 = nullptr;
  double* Cv2 = nullptr;
  // grest_get_embedding_async: copy stream, its events, and whether a copy
  // of U may still be reading the pairs
  cudaStream_t cstream = nullptr;
  cudaEvent_t ev_ready = nullptr, ev_copied = nullptr;
  bool copy_pending = false;
  double* eigwork = nullptr;
  int32_t* err = nullptr;
  // grest_centrality scratch (allocated on first use)
  void* cent_work = nullptr;
  size_t cent_work_cap = 0;
  double* cent_buf = nullptr;   // n_cap
  int32_t* top_id_buf = nullptr;
  double* top_val_buf = nullptr;
  // batch staging
  int32_t *b_iu = nullptr, *b_iv = nullptr, *b_du = nullptr, *b_dv = nullptr, *b_dn = nullptr;
  double* b_w = nullptr;
  int64_t b_cap = 0, b_dn_cap = 0;
  // host mirrors
  double* h_info = nullptr;  // pinned [64]
  int32_t* h_err = nullptr;  // pinned
  int64_t* h_scal = nullptr; // pinned [8]
  grest_stats stats{};
  std::vector<double> last_ritz;
  int last_m = 0;
  int64_t nnz = 0;        // directed nonzeros (exact, read back after each graph update)
  int64_t batch_new_edges = 0;  // inserted edges of the current batch (upper bound for the new-node block)
  int64_t launches = 0;         // kernels enqueued during the current step
  size_t dev_bytes = 0;         // device bytes allocated for this context (cumulative)
  cudaEvent_t ev[10];
  // GREST_FLAG_PROFILE: event pairs around every launch group of the step
  static constexpr int kProfEvents = 512;
  cudaEvent_t pev[kProfEvents];
  int prof_n = 0;
  int prof_cls[kProfEvents / 2];
  int prof_kind[kProfEvents / 2];  // GREST_KIND_*, or -1
  double prof_work[kProfEvents / 2];
  double prof_bytes[kProfEvents / 2];
  bool profiling() const { return (cfg.flags & GREST_FLAG_PROFILE) != 0; }
};

namespace {

grest_status from_cuda(cudaError_t e) {
  if (e == cudaSuccess) return GREST_OK;
  if (e == cudaErrorMemoryAllocation) return GREST_ERR_OOM;
  return GREST_ERR_CUDA;
}

#define CK(x)                                  \
  do {                                         \
    cudaError_t e_ = (x);                      \
    if (e_ != cudaSuccess) return from_cuda(e_); \
  } while (0)

// device bytes allocated by this host thread (context sizes for admission)
thread_local size_t t_dev_bytes = 0;

cudaError_t dmalloc(void** p, size_t bytes) {
  const cudaError_t e = cudaMalloc(p, bytes);
  if (e == cudaSuccess) t_dev_bytes += bytes;
  return e;
}

template <typename T>
cudaError_t dalloc(T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  return dmalloc((void**)p, sizeof(T) * count);
}

// release a buffer of `bytes` that dmalloc / dalloc counted
void dfree(void* p, size_t bytes) {
  if (!p) return;
  cudaFree(p);
  t_dev_bytes -= bytes;
}

// wait (host) until an embedding copy started by grest_get_embedding_async
// has finished reading the device pairs
grest_status settle_copy(grest_ctx* c) {
  if (!c->copy_pending) return GREST_OK;
  const cudaError_t e = cudaEventSynchronize(c->ev_copied);
  c->copy_pending = false;
  return e == cudaSuccess ? GREST_OK : GREST_ERR_CUDA;
}

grest_status map_dev_err(int32_t e) {
  switch (e) {
    case DERR_NONE: return GREST_OK;
    case DERR_CAPACITY: return GREST_ERR_CAPACITY;
    case DERR_ARENA: return GREST_ERR_CAPACITY;
    case DERR_NUMERIC: return GREST_ERR_NUMERIC;
    case DERR_TIMEOUT: return GREST_ERR_TIMEOUT;
    default: return GREST_ERR_INVALID_UPDATE;
  }
}

void free_ctx(grest_ctx* c) {
  if (!c) return;
  void* ptrs[] = {c->g.row_off, c->g.row_len, c->g.row_cap, c->g.col, c->g.val, c->g.live, c->g.deg, c->g.dis,
                  c->g.arena_top, c->g.dmax, c->gw.cnt, c->gw.seg, c->gw.cursor, c->gw.delflag, c->gw.rowflag,
                  c->gw.touched, c->gw.tmp_off, c->gw.need, c->gw.new_len, c->gw.ekey, c->gw.erow, c->gw.ew,
                  c->gw.eins, c->gw.tmp_col, c->gw.tmp_val, c->gw.long_rows, c->gw.scalars, c->gw.scan_tmp,
                  c->U, c->Un, c->theta, c->Zv, c->MZv, c->V2v, c->Yrv, c->Yr2v, c->Omv, c->EtMv, c->Idv, c->U32,
                  c->Rres, c->Cm, c->Cv,
                  c->G, c->T, c->H, c->F, c->XtM, c->Gs, c->Uh, c->ritz, c->th_new, c->tmpk, c->info, c->part,
                  c->ipart, c->piv, c->gemm_img, c->part2, c->gemm_img2, c->Cv2, c->dmax_old, c->XZ, c->gw.edel, c->eigwork, c->err, c->resn, c->cent_work, c->cent_buf, c->top_id_buf, c->top_val_buf, c->b_iu, c->b_iv, c->b_du, c->b_dv, c->b_dn, c->b_w};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (c->h_info) cudaFreeHost(c->h_info);
  if (c->h_err) cudaFreeHost(c->h_err);
  if (c->h_scal) cudaFreeHost(c->h_scal);
  for (auto& e : c->ev)
    if (e) cudaEventDestroy(e);
  for (auto& e : c->pev)
    if (e) cudaEventDestroy(e);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  if (c->s2) cudaStreamDestroy(c->s2);
  if (c->ev_ready) cudaEventDestroy(c->ev_ready);
  if (c->ev_copied) cudaEventDestroy(c->ev_copied);
  if (c->cstream) cudaStreamDestroy(c->cstream);
  delete c;
}

grest_status ensure_batch(grest_ctx* c, int64_t n_edges, int64_t n_dn) {
  if (n_edges > c->b_cap) {
    int64_t cap = std::max<int64_t>(n_edges, 2 * c->b_cap);
    if (c->b_iu) {
      const size_t o = (size_t)std::max<int64_t>(c->b_cap, 1);
      dfree(c->b_iu, 4 * o); dfree(c->b_iv, 4 * o); dfree(c->b_du, 4 * o); dfree(c->b_dv, 4 * o); dfree(c->b_w, 8 * o);
    }
    c->b_iu = c->b_iv = c->b_du = c->b_dv = nullptr;
    c->b_w = nullptr;
    c->b_cap = 0;
    CK(dalloc(&c->b_iu, cap)); CK(dalloc(&c->b_iv, cap)); CK(dalloc(&c->b_du, cap)); CK(dalloc(&c->b_dv, cap));
    CK(dalloc(&c->b_w, cap));
    c->b_cap = cap;
  }
  if (n_dn > c->b_dn_cap) {
    int64_t cap = std::max<int64_t>(n_dn, 2 * c->b_dn_cap);
    if (c->b_dn) dfree(c->b_dn, 4 * (size_t)std::max<int64_t>(c->b_dn_cap, 1));
    c->b_dn = nullptr;
    c->b_dn_cap = 0;
    CK(dalloc(&c->b_dn, cap));
    c->b_dn_cap = cap;
  }
  return GREST_OK;
}

grest_status ensure_graph_work(grest_ctx* c, int64_t entries) {
  GraphWork& w = c->gw;
  if (entries > w.ent_cap) {
    int64_t cap = std::max<int64_t>(entries, 2 * w.ent_cap);
    const size_t old = (size_t)std::max<int64_t>(w.ent_cap, 1);
    if (w.ekey) {
      dfree(w.ekey, sizeof(uint64_t) * old); dfree(w.ew, sizeof(double) * old);
      dfree(w.eins, sizeof(int32_t) * old); dfree(w.edel, sizeof(double) * old);
    }
    w.ekey = nullptr; w.ew = nullptr; w.eins = nullptr; w.edel = nullptr;
    w.ent_cap = 0;
    CK(dalloc(&w.ekey, cap)); CK(dalloc(&w.ew, cap)); CK(dalloc(&w.eins, cap)); CK(dalloc(&w.edel, cap));
    w.ent_cap = cap;
  }
  int64_t tneed = c->g.nnz_cap + w.ent_cap;
  if (tneed > w.tmp_cap) {
    const size_t old = (size_t)std::max<int64_t>(w.tmp_cap, 1);
    if (w.tmp_col) dfree(w.tmp_col, sizeof(int32_t) * old);
    if (w.tmp_val) dfree(w.tmp_val, sizeof(double) * old);
    w.tmp_col = nullptr; w.tmp_val = nullptr;
    w.tmp_cap = 0;
    CK(dalloc(&w.tmp_col, tneed));
    if (c->g.val) CK(dalloc(&w.tmp_val, tneed));
    w.tmp_cap = tneed;
  }
  return GREST_OK;
}

// Per-node arrays for `cap` ids.  Alg. 2 appends S ids per step, so a context
// that keeps receiving batches outgrows any fixed capacity; grow_nodes moves
// every array listed here to a larger capacity.  keep: state that carries
// over between steps (its first n rows are copied); the rest is per-step
// scratch.
struct NodeArray {
  void** slot;
  size_t per_node, extra;
  bool keep;
};

std::vector<NodeArray> node_arrays(grest_ctx* c) {
  Csr& g = c->g;
  GraphWork& w = c->gw;
  std::vector<NodeArray> a = {
      {(void**)&g.row_off, 8, 0, true},  {(void**)&g.row_len, 4, 0, true},   {(void**)&g.row_cap, 4, 0, true},
      {(void**)&g.live, 1, 0, true},     {(void**)&g.deg, 8, 0, true},       {(void**)&g.dis, 8, 0, true},
      {(void**)&w.long_rows, 4, 0, true},{(void**)&c->U, 8 * (size_t)c->ldu, 0, true},
      {(void**)&w.cnt, 4, 4, false},     {(void**)&w.seg, 8, 8, false},      {(void**)&w.cursor, 4, 0, false},
      {(void**)&w.delflag, 1, 0, false}, {(void**)&w.rowflag, 8, 8, false},  {(void**)&w.touched, 4, 0, false},
      {(void**)&w.tmp_off, 8, 8, false}, {(void**)&w.need, 8, 8, false},     {(void**)&w.new_len, 4, 0, false},
      {(void**)&c->Un, 8 * (size_t)c->ldu, 0, false},
      {&c->Zv, c->esz * (size_t)c->ldz, 0, false}, {&c->MZv, c->esz * (size_t)c->ldz, 0, false},
      {&c->V2v, c->esz * (size_t)c->ldv, 0, false},
      {&c->Yrv, c->esz * (size_t)c->ldq, 0, false}, {&c->Yr2v, c->esz * (size_t)c->ldq, 0, false}};
  if (c->U32) a.push_back({(void**)&c->U32, 4 * (size_t)c->ldu, 0, false});
  if (c->Rres) a.push_back({(void**)&c->Rres, 8 * (size_t)c->ldu, 0, false});
  return a;
}

// Grow the node capacity to at least `need` ids (1.5x steps).  Every new
// buffer is allocated before an old one is released, so a failed
// allocation returns GREST_ERR_OOM with the context unchanged.
grest_status grow_nodes(grest_ctx* c, int64_t need) {
  {
    const grest_status st = settle_copy(c);  // U moves to a new buffer
    if (st != GREST_OK) return st;
  }
  const int64_t old_cap = c->g.n_cap, n = c->g.n;
  int64_t cap = std::max<int64_t>(need, old_cap + old_cap / 2);
  cap = std::min<int64_t>(round_up(cap, 1024), (int64_t)INT32_MAX);
  if (cap < need) return GREST_ERR_CAPACITY;
  std::vector<NodeArray> arrs = node_arrays(c);
  std::vector<void*> fresh(arrs.size() + 1, nullptr);
  auto release = [&]() {
    for (size_t i = 0; i < arrs.size(); ++i) dfree(fresh[i], arrs[i].per_node * cap + arrs[i].extra);
    dfree(fresh.back(), scan_temp_bytes(cap + 1));
  };
  for (size_t i = 0; i < arrs.size(); ++i) {
    if (dmalloc(&fresh[i], arrs[i].per_node * cap + arrs[i].extra) != cudaSuccess) {
      cudaGetLastError();
      fresh[i] = nullptr;
      release();
      return GREST_ERR_OOM;
    }
  }
  if (dmalloc(&fresh.back(), scan_temp_bytes(cap + 1)) != cudaSuccess) {
    cudaGetLastError();
    fresh.back() = nullptr;
    release();
    return GREST_ERR_OOM;
  }
  cudaStream_t s = c->stream;
  for (size_t i = 0; i < arrs.size(); ++i)
    if (arrs[i].keep && n > 0)
      CK(cudaMemcpyAsync(fresh[i], *arrs[i].slot, arrs[i].per_node * n, cudaMemcpyDeviceToDevice, s));
  for (size_t i = 0; i < arrs.size(); ++i)  // live: ids >= n are not in use
    if (arrs[i].slot == (void**)&c->g.live) CK(cudaMemsetAsync(static_cast<uint8_t*>(fresh[i]) + n, 0, cap - n, s));
  CK(cudaStreamSynchronize(s));
  for (size_t i = 0; i < arrs.size(); ++i) {
    dfree(*arrs[i].slot, arrs[i].per_node * old_cap + arrs[i].extra);
    *arrs[i].slot = fresh[i];
  }
  dfree(c->gw.scan_tmp, scan_temp_bytes(old_cap + 1));
  c->gw.scan_tmp = fresh.back();
  if (c->cent_buf) {  // centrality scratch: allocated again at the next call
    cudaFree(c->cent_buf);
    c->cent_buf = nullptr;
  }
  c->g.n_cap = cap;
  c->cfg.node_capacity = cap;
  return GREST_OK;
}

// Grow the edge arena: every row is copied, compacted, into an arena of
// max(1.5 nnz_cap, 2 compacted + extra + 2^20) entries (the holes left by
// rows that moved are reclaimed).  The row order inside each row is kept, so
// later products sum in the same order.  On OOM the context is unchanged.
grest_status grow_arena(grest_ctx* c, int64_t n, int64_t extra) {
  Csr& g = c->g;
  cudaStream_t s = c->stream;
  c->launches += graph_compact_plan(g, c->gw, n, s);
  CK(cudaMemcpyAsync(c->h_scal + 6, c->gw.rowflag + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  const int64_t total = c->h_scal[6];
  const int64_t cap = std::max<int64_t>(g.nnz_cap + g.nnz_cap / 2, 2 * total + extra + (1 << 20));
  int32_t* ncol = nullptr;
  double* nval = nullptr;
  if (dalloc(&ncol, cap) != cudaSuccess) {
    cudaGetLastError();
    return GREST_ERR_OOM;
  }
  if (g.val && dalloc(&nval, cap) != cudaSuccess) {
    cudaGetLastError();
    dfree(ncol, sizeof(int32_t) * cap);
    return GREST_ERR_OOM;
  }
  c->launches += graph_compact_copy(g, c->gw, n, ncol, nval, s);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s));
  dfree(g.col, sizeof(int32_t) * g.nnz_cap);
  if (g.val) dfree(g.val, sizeof(double) * g.nnz_cap);
  g.col = ncol;
  g.val = nval;
  g.nnz_cap = cap;
  c->cfg.nnz_capacity = cap;
  return ensure_graph_work(c, c->gw.ent_cap);  // merge staging is sized by the arena
}

grest_status ensure_S(grest_ctx* c, int64_t S) {
  if (S <= c->S_cap) return GREST_OK;
  int64_t cap = std::max<int64_t>(S, 2 * c->S_cap);
  if (c->Omv) {
    dfree(c->Omv, c->esz * c->S_cap * c->ldq);
    dfree(c->EtMv, c->esz * c->S_cap * c->ldq);
  }
  c->Omv = c->EtMv = nullptr;
  c->S_cap = 0;
  CK(dmalloc((void**)&c->Omv, c->esz * cap * c->ldq));
  CK(dmalloc((void**)&c->EtMv, c->esz * cap * c->ldq));
  c->S_cap = cap;
  return GREST_OK;
}

grest_status read_back(grest_ctx* c, int n_info) {
  CK(cudaMemcpyAsync(c->h_err, c->err, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
  if (n_info > 0) CK(cudaMemcpyAsync(c->h_info, c->info, sizeof(double) * n_info, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return GREST_OK;
}

int prof_begin(grest_ctx* c) {
  if (!c->profiling() || c->prof_n + 2 > grest_ctx::kProfEvents) return -1;
  int i = c->prof_n;
  cudaEventRecord(c->pev[i], c->stream);
  c->prof_n += 2;
  return i;
}

void prof_end(grest_ctx* c, int i, int cls, double work, double bytes = 0.0, int kind = -1) {
  if (i < 0) return;
  cudaEventRecord(c->pev[i + 1], c->stream);
  c->prof_cls[i / 2] = cls;
  c->prof_kind[i / 2] = kind >= 0 ? kind : (cls == 3 ? GREST_KIND_SMALL : cls == 4 ? GREST_KIND_GRAPH : -1);
  c->prof_work[i / 2] = work;
  c->prof_bytes[i / 2] = bytes;
}

void prof_collect(grest_ctx* c, grest_stats& st) {
  for (int k = 0; k < 5; ++k) {
    st.prof_ms[k] = 0.0;
    st.prof_work[k] = 0.0;
    st.prof_bytes[k] = 0.0;
    st.prof_launches[k] = 0;
  }
  for (int k = 0; k < GREST_KIND_COUNT; ++k) {
    st.prof_kind_ms[k] = 0.0;
    st.prof_kind_work[k] = 0.0;
    st.prof_kind_bytes[k] = 0.0;
    st.prof_kind_launches[k] = 0;
  }
  for (int i = 0; i + 1 < c->prof_n; i += 2) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c->pev[i], c->pev[i + 1]);
    int k = c->prof_cls[i / 2];
    st.prof_ms[k] += ms;
    st.prof_work[k] += c->prof_work[i / 2];
    st.prof_bytes[k] += c->prof_bytes[i / 2];
    st.prof_launches[k] += 1;
    const int kd = c->prof_kind[i / 2];
    if (kd >= 0 && kd < GREST_KIND_COUNT) {
      st.prof_kind_ms[kd] += ms;
      st.prof_kind_work[kd] += c->prof_work[i / 2];
      st.prof_kind_bytes[kd] += c->prof_bytes[i / 2];
      st.prof_kind_launches[kd] += 1;
    }
  }
  c->prof_n = 0;
}

OpParams op_params(const grest_ctx* c) {
  OpParams p;
  p.op = c->cfg.op;
  p.deg = c->g.deg;
  p.dis = c->g.dis;
  p.dmax = c->g.dmax;
  p.live = c->g.live;
  return p;
}

// ---------------------------------------------------------------- typed launch wrappers
// nnz_proc: entries of the processed rows that take part (all of them, or the
// new-node block); x_rows: rows of X read at least once
void prof_spmm(grest_ctx* c, int p, int w, int64_t r0, int64_t r1, int64_t col_lo, int64_t nnz_proc, int64_t x_rows,
               double xbytes, double ybytes, int kind) {
  if (r1 > r0 && w > 0) c->launches += col_lo == 0 ? 2 : 1;
  if (nnz_proc < 0) nnz_proc = c->nnz;
  if (x_rows < 0) x_rows = r1 - r0;
  const double eb = c->g.val ? 12.0 : 4.0;
  const double by = 12.0 * (r1 - r0) + eb * nnz_proc + w * (ybytes * (r1 - r0) + xbytes * x_rows);
  prof_end(c, p, 0, 2.0 * nnz_proc * w, by, kind);  // work: a multiply-add per nonzero and column
}

void spmm(grest_ctx* c, const double* X, int64_t ldx, double* Y, int64_t ldy, int w, int64_t r0, int64_t r1,
          int64_t col_lo, int64_t nnz_proc = -1, int64_t x_rows = -1) {
  int p = prof_begin(c);
  spmm_f64(c->g, op_params(c), c->gw.long_rows, c->gw.scalars + 1, X, ldx, Y, ldy, w, r0, r1, col_lo, c->stream);
  prof_spmm(c, p, w, r0, r1, col_lo, nnz_proc, x_rows, 8.0, 8.0, GREST_KIND_SPMM_F64);
}

void spmm(grest_ctx* c, const float* X, int64_t ldx, float* Y, int64_t ldy, int w, int64_t r0, int64_t r1,
          int64_t col_lo, int64_t nnz_proc = -1, int64_t x_rows = -1) {
  int p = prof_begin(c);
  spmm_f32(c->g, op_params(c), c->gw.long_rows, c->gw.scalars + 1, X, ldx, Y, ldy, w, r0, r1, col_lo, c->stream);
  prof_spmm(c, p, w, r0, r1, col_lo, nnz_proc, x_rows, 4.0, 4.0, GREST_KIND_SPMM_F32);
}

void spmm(grest_ctx* c, const float* X, int64_t ldx, double* Y, int64_t ldy, int w, int64_t r0, int64_t r1,
          int64_t col_lo, int64_t nnz_proc = -1, int64_t x_rows = -1) {
  int p = prof_begin(c);
  spmm_f32_f64(c->g, op_params(c), c->gw.long_rows, c->gw.scalars + 1, X, ldx, Y, ldy, w, r0, r1, col_lo, c->stream);
  prof_spmm(c, p, w, r0, r1, col_lo, nnz_proc, x_rows, 4.0, 8.0, GREST_KIND_SPMM_F32);
}

// Y = Delta X (Sec. 3.3 block, Eq. main3) for the batch just applied
template <typename T>
void delta(grest_ctx* c, const T* X, int64_t ldx, T* Y, int64_t ldy, int w, int64_t N, int64_t N2) {
  int p = prof_begin(c);
  c->launches += delta_apply(c->g, c->gw, c->cfg.op, X, ldx, Y, ldy, w, N, N2, c->dmax_old, c->stream);
  const double by = (double)sizeof(T) * N2 * w * 2.0;
  prof_end(c, p, 0, by, by);
}

void gram(grest_ctx* c, const double* X, int64_t ldx, int a, const double* Y, int64_t ldy, int b, int64_t n,
          double* C, int64_t ldc, bool sym) {
  int p = prof_begin(c);
  gram_f64(X, ldx, a, Y, ldy, b, n, C, ldc, c->part, sym, c->stream);
  if (a > 0 && b > 0 && n > 0) c->launches += 2;
  prof_end(c, p, 1, 2.0 * n * a * b, 8.0 * n * (X == Y && a == b ? a : a + b), GREST_KIND_GRAM_CUDA);
}

// FP32 Gram of the mixed path: a narrow side (the projections X_bar^T Y, K
// columns) on the CUDA cores, wider products on the tensor cores; false when
// neither kernel takes the shape or alignment
int gram_f32_fast(const float* X, int64_t ldx, int a, const float* Y, int64_t ldy, int b, int64_t n, double* C,
                  int64_t ldc, double* part, int64_t part_cap, int32_t* err, cudaStream_t s) {
  if (n <= 0) return -1;
  if (std::min(a, b) <= 32 && gram_f32_narrow(X, ldx, a, Y, ldy, b, n, C, ldc, part, part_cap, err, s) == 0)
    return GREST_KIND_GRAM_NARROW;
  if (gram_tc_supported(X, ldx, a, Y, ldy, b) && gram_f32_tc(X, ldx, a, Y, ldy, b, n, C, ldc, part, part_cap, err, s) == 0)
    return GREST_KIND_GRAM_TC;
  return -1;
}

void gram(grest_ctx* c, const float* X, int64_t ldx, int a, const float* Y, int64_t ldy, int b, int64_t n, double* C,
          int64_t ldc, bool sym) {
  int p = prof_begin(c);
  int kind = gram_f32_fast(X, ldx, a, Y, ldy, b, n, C, ldc, c->part, c->part_cap, c->err, c->stream);
  if (kind < 0) {
    gram_f32(X, ldx, a, Y, ldy, b, n, C, ldc, c->part, sym, c->stream);
    kind = GREST_KIND_GRAM_CUDA;
  }
  if (a > 0 && b > 0 && n > 0) c->launches += 2;
  prof_end(c, p, 1, 2.0 * n * a * b, 4.0 * n * (X == Y && a == b ? a : a + b), kind);
}

void gemm(grest_ctx* c, int64_t n, int a, int cc, double alpha, const double* X, int64_t ldx, const double* B,
          int64_t ldb, double beta, const double* Cin, int64_t ldc, double* Out, int64_t ldo) {
  int p = prof_begin(c);
  gemm_nn_f64(n, a, cc, alpha, X, ldx, B, ldb, beta, Cin, ldc, Out, ldo, c->stream);
  if (n > 0 && cc > 0) c->launches += 1;
  prof_end(c, p, 2, 2.0 * n * a * cc, 8.0 * n * (a + cc * (beta != 0.0 ? 2 : 1)), GREST_KIND_GEMM_CUDA);
}

void gemm(grest_ctx* c, int64_t n, int a, int cc, double alpha, const float* X, int64_t ldx, const double* B,
          int64_t ldb, double beta, const float* Cin, int64_t ldc, float* Out, int64_t ldo) {
  int p = prof_begin(c);
  int kind = GREST_KIND_GEMM_CUDA;
  if (n > 0 && cc > 0 && gemm_f32_tc(n, a, cc, alpha, X, ldx, B, ldb, beta, Cin, ldc, Out, ldo, c->gemm_img,
                                     c->gemm_img_cap, c->err, c->stream) == 0) {
    c->launches += 2;
    kind = GREST_KIND_GEMM_TC;
  } else {
    gemm_nn_f32(n, a, cc, alpha, X, ldx, B, ldb, beta, Cin, ldc, Out, ldo, c->stream);
    if (n > 0 && cc > 0) c->launches += 1;
  }
  prof_end(c, p, 2, 2.0 * n * a * cc, 4.0 * n * (a + cc * (beta != 0.0 ? 2 : 1)), kind);
}

// f32: the projected problem's entries come from FP32 blocks (mixed path), so
// it is solved in FP32 arithmetic; the refinement's K x K problem uses FP64
void eig(grest_ctx* c, double* H, int64_t ld, int m, int k, int op, double* theta, double* F, int64_t ldf,
         double* ritz, double* info, bool f32) {
  int p = prof_begin(c);
  // FP64 problems of at most 64 columns: cyclic Jacobi in one CTA (group_dense.cu)
  int nl = f32 ? -1 : eig_small_f64(H, (int)ld, m, k, op, theta, F, (int)ldf, ritz, info, c->stream);
  if (nl < 0) nl = sym_eig_select(H, ld, m, k, op, theta, F, ldf, ritz, info, c->eigwork, f32, c->stream);
  c->launches += nl;
  prof_end(c, p, 3, 4.0 * m * m * m / 3.0 + 2.0 * m * m * k);
}

// Arithmetic of the projected problems (pivoted Cholesky, m x m and q x q
// eigensolves): FP32 only in GREST_MIXED_FAST, whose Grams are FP32-accurate
// (reading R15); FP64 in GREST_MIXED and GREST_FP64.
template <typename T>
bool small_f32(const grest_ctx* c) {
  return sizeof(T) == sizeof(float) && c->cfg.precision == GREST_MIXED_FAST;
}

template <typename T>
T* Zp(grest_ctx* c) { return static_cast<T*>(c->Zv); }
template <typename T>
T* MZp(grest_ctx* c) { return static_cast<T*>(c->MZv); }
template <typename T>
T* V2p(grest_ctx* c) { return static_cast<T*>(c->V2v); }
template <typename T>
T* Yrp(grest_ctx* c) { return static_cast<T*>(c->Yrv); }
template <typename T>
T* Yr2p(grest_ctx* c) { return static_cast<T*>(c->Yr2v); }
template <typename T>
T* Omp(grest_ctx* c) { return static_cast<T*>(c->Omv); }
template <typename T>
T* EtMp(grest_ctx* c) { return static_cast<T*>(c->EtMv); }
template <typename T>
T* Idp(grest_ctx* c) { return static_cast<T*>(c->Idv); }

// X (n x w) <- P_perp X = X - U (U^T X), U = first Ku columns of Z
template <typename T>
void project_out(grest_ctx* c, T* X, int64_t ldx, int w, int64_t n) {
  if (c->Ku == 0 || w == 0) return;
  gram(c, Zp<T>(c), c->ldz, c->Ku, X, ldx, w, n, c->Cv, w, false);
  gemm(c, n, c->Ku, w, -1.0, Zp<T>(c), c->ldz, c->Cv, w, 1.0, X, ldx, X, ldx);
}

// With GREST_FLAG_TWO_STREAMS, graphs of at least this many nodes at
// grest_init get the step's second lane.
constexpr int64_t kOverlapRows = 1 << 17;

// While alive, the step's launch wrappers enqueue on the second lane: its
// stream and its own Gram partials, GEMM operand images and projection
// coefficients (the wrappers read these from the context).
struct Lane2 {
  grest_ctx* c;
  explicit Lane2(grest_ctx* ctx) : c(ctx) { flip(); }
  ~Lane2() { flip(); }
  void flip() {
    std::swap(c->stream, c->s2);
    std::swap(c->part, c->part2);
    std::swap(c->gemm_img, c->gemm_img2);
    std::swap(c->Cv, c->Cv2);
  }
};

// CholQR with pivoting: Out (n x rank) = X (n x w) T; returns rank via info slot
template <typename T>
grest_status cholqr_pass(grest_ctx* c, const T* X, int64_t ldx, int w, int64_t n, double tol, double abs_ref,
                         const double* abs_ref_ptr, T* Out, int64_t ldo, int info_slot, bool read_rank,
                         int* rank_out) {
  gram(c, X, ldx, w, X, ldx, w, n, c->G, w, true);
  int p = prof_begin(c);
  // FP64 problems of at most 64 columns: one CTA (group_dense.cu); else the cluster kernels
  int nl = small_f32<T>(c) ? -1
                           : pchol_small_f64(c->G, w, w, tol, abs_ref, abs_ref_ptr, c->T, w, c->info + info_slot,
                                             c->stream);
  if (nl < 0)
    nl = pchol_inverse(c->G, w, w, tol, abs_ref, abs_ref_ptr, c->T, w, c->piv, c->info + info_slot, small_f32<T>(c),
                       c->stream);
  c->launches += nl;
  prof_end(c, p, 3, (double)w * w * w / 3.0 + (double)w * w * w / 3.0);
  int rank = w;
  if (read_rank) {
    grest_status st = read_back(c, info_slot + 4);
    if (st != GREST_OK) return st;
    if (*c->h_err) return map_dev_err(*c->h_err);
    rank = (int)c->h_info[info_slot];
  }
  if (rank > 0) gemm(c, n, w, rank, 1.0, X, ldx, c->T, w, 0.0, static_cast<const T*>(nullptr), 0, Out, ldo);
  if (rank_out) *rank_out = rank;
  return GREST_OK;
}

template <typename T>
__global__ void k_fill_identity(T* I, int64_t ld, int q) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e < (int64_t)q * q) I[(e / q) * ld + (e % q)] = (e / q == e % q) ? (T)1 : (T)0;
}

template <typename T>
__global__ void k_pad_copy(const double* U, int64_t ldu, T* Z, int64_t ldz, int64_t N, int64_t N2, int K) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < N2 * K; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t r = e / K;
    int c = (int)(e % K);
    Z[r * ldz + c] = r < N ? (T)U[r * ldu + c] : (T)0;
  }
}

__global__ void k_sum_removed_degree(const int32_t* dn, int64_t n_dn, const int64_t N, const int32_t* row_len,
                                     int64_t* out) {
  int64_t s = 0;
  for (int64_t i = threadIdx.x; i < n_dn; i += blockDim.x) {
    int32_t d = dn[i];
    if (d >= 0 && d < N) s += row_len[d];
  }
  __shared__ int64_t red[256];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

__global__ void k_orth_err(const double* G, int64_t ld, int k, double* out) {
  double m = 0.0;
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
    int i = e / k, j = e % k;
    m = fmax(m, fabs(G[(int64_t)i * ld + j] - (i == j ? 1.0 : 0.0)));
  }
  __shared__ double red[256];
  red[threadIdx.x] = m;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

__global__ void k_resid_vecs(const double* MU, const double* U, int64_t ld, int k, const double* theta, int64_t n,
                             double* R, int64_t ldr) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * k; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t r = e / k;
    int c = (int)(e % k);
    R[r * ldr + c] = MU[r * ld + c] - theta[c] * U[r * ld + c];
  }
}

__global__ void k_maxabs(const double* A, int64_t ld, int rows, int cols, double* out) {
  double m = 0.0;
  for (int e = threadIdx.x; e < rows * cols; e += blockDim.x) m = fmax(m, fabs(A[(int64_t)(e / cols) * ld + e % cols]));
  __shared__ double red[256];
  red[threadIdx.x] = m;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

// Small k x k products for the refinement: Hs = T^T H T, and F' = T F.
__global__ void k_small_tht(const double* T, const double* H, int k, double* HT, double* out) {
  // HT = H T, then out = T^T HT (one block, k <= 64)
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
    int i = e / k, j = e % k;
    double s = 0.0;
    for (int l = 0; l < k; ++l) s = fma(H[i * k + l], T[l * k + j], s);
    HT[i * k + j] = s;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
    int i = e / k, j = e % k;
    double s = 0.0;
    for (int l = 0; l < k; ++l) s = fma(T[l * k + i], HT[l * k + j], s);
    out[i * k + j] = s;
  }
}

__global__ void k_small_mm(const double* A, const double* B, int k, double* out) {
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
    int i = e / k, j = e % k;
    double s = 0.0;
    for (int l = 0; l < k; ++l) s = fma(A[i * k + l], B[l * k + j], s);
    out[i * k + j] = s;
  }
}

// Eq. main3: H += (X_bar^T Z)^T Lambda (X_bar^T Z); XZ is ku x m (ld m)
__global__ void k_lowrank_add(const double* XZ, int m, int ku, const double* lam, double* H, int64_t ldh) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)m * m) return;
  const int i = (int)(e / m), j = (int)(e % m);
  double s = 0.0;
  for (int k = 0; k < ku; ++k) s = fma(XZ[(int64_t)k * m + i] * lam[k], XZ[(int64_t)k * m + j], s);
  H[(int64_t)i * ldh + j] += s;
}

float ev_ms(cudaEvent_t a, cudaEvent_t b) {
  float ms = 0.f;
  cudaEventElapsedTime(&ms, a, b);
  return ms;
}

// Mixed path, A11: FP64 Rayleigh-Ritz in span(U32).  With G = U^T U, the
// pivoted Cholesky gives T with (U T)^T (U T) = I; the K x K problem
// T^T (U^T M U) T F'' = F'' Theta is solved in FP64 and X = U (T F'').  The
// N x K products read U's exact FP32 values and are carried in double-float
// (FP32 hi + lo, about 48 bits; refine.cu), which on this GPU runs on the
// FP32 pipes at many times the FP64 rate; their K x K results are FP64.
grest_status refine_mixed(grest_ctx* c, int64_t N2) {
  cudaStream_t s = c->stream;
  const int K = c->K;
  float* MUh = reinterpret_cast<float*>(c->Un);  // Un (n_cap x ldu doubles) holds M U as hi / lo floats
  float* MUl = MUh + (size_t)c->g.n_cap * c->ldu;
  int p = prof_begin(c);
  c->launches += gram_df(c->U32, c->ldu, c->U32, nullptr, c->ldu, K, N2, c->G, K, c->part, c->part_cap, s);
  prof_end(c, p, 1, 2.0 * N2 * K * K, 4.0 * N2 * K, GREST_KIND_DOUBLE_FLOAT);
  p = prof_begin(c);
  c->launches += spmm_df(c->g, op_params(c), c->gw.long_rows, c->gw.scalars + 1, c->U32, c->ldu, MUh, MUl, c->ldu,
                         K, N2, s);
  {
    const double by = 12.0 * N2 + (c->g.val ? 12.0 : 4.0) * c->nnz + K * (8.0 * N2 + 4.0 * N2);
    prof_end(c, p, 0, by, by, GREST_KIND_DOUBLE_FLOAT);
  }
  p = prof_begin(c);
  c->launches += gram_df(c->U32, c->ldu, MUh, MUl, c->ldu, K, N2, c->H, K, c->part, c->part_cap, s);
  prof_end(c, p, 1, 2.0 * N2 * K * K, 12.0 * N2 * K, GREST_KIND_DOUBLE_FLOAT);
  p = prof_begin(c);
  {  // the K x K problems of the refinement fit one CTA (K <= 64)
    int nl = pchol_small_f64(c->G, K, K, 1e-14, 0.0, nullptr, c->T, K, c->info + 44, s);
    if (nl < 0) nl = pchol_inverse(c->G, K, K, 1e-14, 0.0, nullptr, c->T, K, c->piv, c->info + 44, false, s);
    c->launches += nl;
  }
  k_small_tht<<<1, 256, 0, s>>>(c->T, c->H, K, c->Gs, c->Uh);
  symmetrize(c->Uh, K, K, s);
  c->launches += 2;
  prof_end(c, p, 3, 4.0 * K * K * K);
  {
    p = prof_begin(c);
    const int ne = eig_small_f64(c->Uh, K, K, K, c->cfg.op, c->th_new, c->F, K, c->tmpk, c->info + 48, s);
    prof_end(c, p, 3, 4.0 * K * K * K);
    if (ne < 0) eig(c, c->Uh, K, K, K, c->cfg.op, c->th_new, c->F, K, c->tmpk, c->info + 48, false);
    else c->launches += ne;
  }
  k_small_mm<<<1, 256, 0, s>>>(c->T, c->F, K, c->Gs);
  c->launches += 1;
  p = prof_begin(c);
  c->launches += lift_df(c->U32, c->ldu, c->Gs, K, N2, c->U, c->ldu, s);
  c->launches += sign_normalize_fast(c->U, c->ldu, K, N2, c->part, c->ipart, s);
  prof_end(c, p, 2, 2.0 * N2 * K * K, 4.0 * N2 * K + 8.0 * N2 * K * 3, GREST_KIND_DOUBLE_FLOAT);
  CK(cudaMemcpyAsync(c->theta, c->th_new, sizeof(double) * K, cudaMemcpyDeviceToDevice, s));
  return GREST_OK;
}

// Mixed path, A11 in FP64 arithmetic (GREST_MIXED): X64 = U32 widened
// exactly, MU = M X64 with FP64 products and sums, G = X64^T X64 and
// H' = X64^T MU as FP64 Grams (upper triangles only: both are symmetric,
// H' because M is); then the same K x K Rayleigh-Ritz problem as
// refine_mixed (FP64), and X = X64 (T F'') as an FP64 GEMM.  The previous
// pairs in U are no longer read at this point of the step, so U holds MU
// until the lift overwrites it.
grest_status refine_mixed_f64(grest_ctx* c, int64_t N2) {
  cudaStream_t s = c->stream;
  const int K = c->K;
  const int64_t ldu = c->ldu;
  double* X64 = c->Un;
  double* MU = c->U;
  int p = prof_begin(c);
  convert_f32_to_f64(c->U32, ldu, X64, ldu, N2, K, s);
  c->launches += 1;
  prof_end(c, p, 2, 0.0, 12.0 * N2 * K);
  spmm(c, X64, ldu, MU, ldu, K, 0, N2, 0);
  p = prof_begin(c);
  const int nl = gram_pair_sym_f64(X64, MU, ldu, K, N2, c->G, c->H, c->part, c->part_cap, s);
  if (nl < 0) return GREST_ERR_CAPACITY;
  c->launches += nl;
  prof_end(c, p, 1, 2.0 * N2 * K * (K + 1), 16.0 * N2 * K, GREST_KIND_GRAM_CUDA);
  p = prof_begin(c);
  {  // the K x K problems of the refinement fit one CTA (K <= 64)
    int nl = pchol_small_f64(c->G, K, K, 1e-14, 0.0, nullptr, c->T, K, c->info + 44, s);
    if (nl < 0) nl = pchol_inverse(c->G, K, K, 1e-14, 0.0, nullptr, c->T, K, c->piv, c->info + 44, false, s);
    c->launches += nl;
  }
  k_small_tht<<<1, 256, 0, s>>>(c->T, c->H, K, c->Gs, c->Uh);
  symmetrize(c->Uh, K, K, s);
  c->launches += 2;
  prof_end(c, p, 3, 4.0 * K * K * K);
  {
    p = prof_begin(c);
    const int ne = eig_small_f64(c->Uh, K, K, K, c->cfg.op, c->th_new, c->F, K, c->tmpk, c->info + 48, s);
    prof_end(c, p, 3, 4.0 * K * K * K);
    if (ne < 0) eig(c, c->Uh, K, K, K, c->cfg.op, c->th_new, c->F, K, c->tmpk, c->info + 48, false);
    else c->launches += ne;
  }
  k_small_mm<<<1, 256, 0, s>>>(c->T, c->F, K, c->Gs);
  c->launches += 1;
  gemm(c, N2, K, K, 1.0, X64, ldu, c->Gs, K, 0.0, static_cast<const double*>(nullptr), 0, c->U, ldu);
  p = prof_begin(c);
  c->launches += sign_normalize_fast(c->U, ldu, K, N2, c->part, c->ipart, s);
  prof_end(c, p, 2, 0.0, 16.0 * N2 * K);
  CK(cudaMemcpyAsync(c->theta, c->th_new, sizeof(double) * K, cudaMemcpyDeviceToDevice, s));
  return GREST_OK;
}

// A5 with an RSVD block (Sec. 3.5), the part that needs X_bar but not
// M X_bar: S.1 Y = P_perp Delta_2 Omega and its CholQR2 with pivoting (basis
// in Yr, rank rY), then Delta_2^T Yr (rows N.. of M Yr into EtM) and
// X_bar^T Yr for S.2.
template <typename T>
grest_status rsvd_sketch(grest_ctx* c, int64_t N, int64_t N2, int64_t S, int* rY_out) {
  const int q = c->q, Ku = c->Ku;
  const int64_t ldq = c->ldq, ldz = c->ldz;
  T* Z = Zp<T>(c);
  T* Yr = Yrp<T>(c);
  T* Yr2 = Yr2p<T>(c);
  T* Om = Omp<T>(c);
  T* EtM = EtMp<T>(c);
  // S.1: Y = P_perp Delta_2 Omega, one projection as in S.1: the basis only
  // enters S.2 through Delta_2^T P_perp M (the formula below applies P_perp
  // itself) and A6 projects the block R = M U_hat again, so rounding left
  // along X_bar here does not reach the result
  gaussian_omega(Om, ldq, S, q, c->cfg.seed, (uint64_t)c->step, c->stream);
  c->launches += 1;
  spmm(c, Om, ldq, Yr, ldq, q, 0, N2, N, c->batch_new_edges + S, S);
  project_out(c, Yr, ldq, q, N2);
  // M = orth(Y): CholQR2 with pivoting
  int rY = 0;
  grest_status st = cholqr_pass(c, Yr, ldq, q, N2, c->cfg.drop_tol, 0.0, c->theta, Yr2, ldq, 8, true, &rY);
  if (st != GREST_OK) return st;
  int rY2 = 0;
  st = cholqr_pass(c, Yr2, ldq, rY, N2, 1e-14, 0.0, nullptr, Yr, ldq, 12, false, &rY2);
  if (st != GREST_OK) return st;
  c->stats.rank_y = rY;
  if (rY > 0) {
    // S.2, first products: Delta_2^T M (rows N.. of M Yr) and X_bar^T M
    spmm(c, Yr, ldq, EtM, ldq, rY, N, N2, 0, c->batch_new_edges + S, N2);
    gram(c, Z, ldz, Ku, Yr, ldq, rY, N2, c->XtM, rY, false);
  }
  *rY_out = rY;
  return GREST_OK;
}

template <typename T>
grest_status step_t(grest_ctx* c, int64_t N, int64_t S, bool removed) {
  const int64_t N2 = N + S;
  cudaStream_t s = c->stream;
  const int K = c->K;
  Csr& g = c->g;
  T* Z = Zp<T>(c);
  T* MZ = MZp<T>(c);
  T* V2 = V2p<T>(c);
  const int64_t ldz = c->ldz, ldv = c->ldv, ldq = c->ldq;
  CK(cudaEventRecord(c->ev[1], s));
  // A2: X_bar = [X; 0]; removed nodes: zero their rows and re-orthonormalize (reading of node removal)
  k_pad_copy<T><<<1024, 256, 0, s>>>(c->U, c->ldu, Z, ldz, N, N2, c->Ku);
  c->launches += 1;
  if (removed) {
    zero_dead_rows(Z, ldz, c->Ku, g.live, N2, s);
    c->launches += 1;
    int r1 = 0;
    grest_status st = cholqr_pass(c, Z, ldz, c->Ku, N2, c->cfg.drop_tol, 1.0, nullptr, V2, ldv, 0, true, &r1);
    if (st != GREST_OK) return st;
    int r2 = 0;
    st = cholqr_pass(c, V2, ldv, r1, N2, 1e-14, 0.0, nullptr, Z, ldz, 4, false, &r2);
    if (st != GREST_OK) return st;
    c->Ku = r1;
  }
  const int Ku = c->Ku;
  // A5 with an RSVD block: its sketch (S.1 and the products of S.2 that need
  // X_bar only) is independent of A3 and A4; with a second lane
  // (GREST_FLAG_TWO_STREAMS) it runs there, beside them (its pivoted
  // Cholesky and eigen kernels hold few SMs, and A3 / A4 fill the rest),
  // joined before S.2's use of M X_bar.  The same kernels see the same
  // inputs either way, so the results do not change.
  const bool rsvd_block = S > 0 && c->cfg.subspace != GREST_SUB_GREST2 &&
                          (c->cfg.subspace == GREST_SUB_RSVD || (c->cfg.subspace == GREST_SUB_AUTO && S > c->q));
  const bool overlap = rsvd_block && c->s2 != nullptr;
  if (rsvd_block) {
    grest_status st = ensure_S(c, S);
    if (st != GREST_OK) return st;
  }
  if (overlap) CK(cudaEventRecord(c->ev_fork, s));
  const bool lowrank = c->cfg.projection == GREST_PROJ_LOWRANK;
  const bool delta_w = c->cfg.w_block == GREST_WB_DELTA;
  // A3: MZ[:, 0:Ku] = M X_bar (EXACT projection) or Delta X_bar (LOWRANK,
  // Eq. main3); the W block is projected from M X_bar (RESID) or Delta X_bar
  // (DELTA, Sec. 3.3); when that is the other product it goes to V2
  const T* src = MZ;
  int64_t lds = ldz;
  if (!lowrank) {
    spmm(c, Z, ldz, MZ, ldz, Ku, 0, N2, 0);
    if (delta_w) {
      delta(c, (const T*)Z, ldz, V2, ldv, Ku, N, N2);
      src = V2;
      lds = ldv;
    }
  } else {
    delta(c, (const T*)Z, ldz, MZ, ldz, Ku, N, N2);
    if (!delta_w) {
      spmm(c, Z, ldz, V2, ldv, Ku, 0, N2, 0);
      src = V2;
      lds = ldv;
    }
  }
  CK(cudaEventRecord(c->ev[2], s));
  // A4: C = X_bar^T src; W = src - X_bar C, re-projected once
  T* W = Z + Ku;
  gram(c, Z, ldz, Ku, src, lds, Ku, N2, c->Cm, Ku, false);
  gemm(c, N2, Ku, Ku, -1.0, Z, ldz, c->Cm, Ku, 1.0, src, lds, W, ldz);
  project_out(c, W, ldz, Ku, N2);
  int rY = 0;
  if (overlap) {
    grest_status st2;
    {
      Lane2 lane(c);
      CK(cudaStreamWaitEvent(c->stream, c->ev_fork, 0));
      st2 = rsvd_sketch<T>(c, N, N2, S, &rY);
      CK(cudaEventRecord(c->ev_join, c->stream));
    }
    CK(cudaStreamWaitEvent(s, c->ev_join, 0));
    if (st2 != GREST_OK) return st2;
  }
  // A5: new-node block
  int cb = 0;
  int mode = 2;
  T* B = Z + 2 * Ku;
  const int q = c->q;
  if (S > 0 && c->cfg.subspace != GREST_SUB_GREST2) {
    bool rsvd = c->cfg.subspace == GREST_SUB_RSVD || (c->cfg.subspace == GREST_SUB_AUTO && S > q);
    if (!rsvd) {
      if (S > q) return GREST_ERR_UNSUPPORTED;  // exact block wider than the basis buffers
      mode = 3;
      // E = M_new[:, N:N2] = M_new * [0; I_S] (restricted SpMM against the identity)
      spmm(c, Idp<T>(c), ldq, B, ldz, (int)S, 0, N2, N, c->batch_new_edges + S, S);
      project_out(c, B, ldz, (int)S, N2);
      cb = (int)S;
    } else {
      mode = 4;
      if (!overlap) {
        grest_status st = rsvd_sketch<T>(c, N, N2, S, &rY);
        if (st != GREST_OK) return st;
      }
      T* Yr = Yrp<T>(c);
      T* EtM = EtMp<T>(c);
      if (rY > 0) {
        // S.2 (cont.): B_s^T = Delta_2^T M - (Delta_2^T X_bar)(X_bar^T M), Delta_2^T X_bar = Y1[N:N2]
        gemm(c, S, Ku, rY, -1.0, MZ + N * ldz, ldz, c->XtM, rY, 1.0, EtM, ldq, EtM, ldq);
        // left singular vectors of B_s via eig(B_s B_s^T), L leading
        gram(c, EtM, ldq, rY, EtM, ldq, rY, S, c->Gs, rY, true);
        const int Lp = std::min(c->Lr, rY);
        eig(c, c->Gs, rY, rY, Lp, GREST_OP_LAP, c->tmpk, c->Uh, Lp, c->ritz, c->info + 16, small_f32<T>(c));
        // S.4: R = M U_hat
        gemm(c, N2, rY, Lp, 1.0, Yr, ldq, c->Uh, Lp, 0.0, static_cast<const T*>(nullptr), 0, B, ldz);
        cb = Lp;
      }
    }
  }
  CK(cudaEventRecord(c->ev[3], s));
  // A6: Q = orth(P_perp [W, B]) by CholQR2 with pivoting (partial orthogonality: X_bar is fixed)
  int cw = Ku + cb;
  T* V = Z + Ku;
  project_out(c, V, ldz, cw, N2);
  int r = 0;
  grest_status st = cholqr_pass(c, V, ldz, cw, N2, c->cfg.drop_tol, 0.0, c->theta, V2, ldv, 20, true, &r);
  if (st != GREST_OK) return st;
  c->stats.pivot_kept_min = c->h_info[21];
  c->stats.pivot_dropped_max = c->h_info[22];
  if (r > 0) {
    project_out(c, V2, ldv, r, N2);
    int r2 = 0;
    st = cholqr_pass(c, V2, ldv, r, N2, 1e-14, 0.0, nullptr, V, ldz, 24, false, &r2);
    if (st != GREST_OK) return st;
  }
  const int m = Ku + r;
  if (m < K) return GREST_ERR_NUMERIC;
  // A7: MQ = M Q (EXACT) or Delta Q (LOWRANK)
  if (r > 0) {
    if (!lowrank)
      spmm(c, V, ldz, MZ + Ku, ldz, r, 0, N2, 0);
    else
      delta(c, (const T*)V, ldz, MZ + Ku, ldz, r, N, N2);
  }
  CK(cudaEventRecord(c->ev[4], s));
  // A8: H = Z^T (M Z) (Eq. main2), or Z^T (Delta Z) + (X_bar^T Z)^T Lambda
  // (X_bar^T Z) (Eq. main3); symmetrized
  gram(c, Z, ldz, m, MZ, ldz, m, N2, c->H, m, false);
  if (lowrank) {
    gram(c, Z, ldz, Ku, Z, ldz, m, N2, c->XZ, m, false);
    k_lowrank_add<<<(unsigned)(((int64_t)m * m + 255) / 256), 256, 0, s>>>(c->XZ, m, Ku, c->theta, c->H, m);
    c->launches += 1;
  }
  symmetrize(c->H, m, m, s);
  c->launches += 1;
  CK(cudaEventRecord(c->ev[5], s));
  // A9: leading K eigenpairs of H (Alg. 1)
  eig(c, c->H, m, m, K, c->cfg.op, c->th_new, c->F, K, c->ritz, c->info + 28, small_f32<T>(c));
  CK(cudaEventRecord(c->ev[6], s));
  // the lift is the step's first write to the buffers of the previous pairs:
  // a copy of them started by grest_get_embedding_async finishes first
  if (c->copy_pending) CK(cudaStreamWaitEvent(s, c->ev_copied, 0));
  // A10: X = Z F_K, sign normalization
  if constexpr (sizeof(T) == sizeof(double)) {
    gemm(c, N2, m, K, 1.0, Z, ldz, c->F, K, 0.0, static_cast<const T*>(nullptr), 0, c->Un, c->ldu);
    c->launches += sign_normalize_fast(c->Un, c->ldu, K, N2, c->part, c->ipart, s);
    CK(cudaMemcpyAsync(c->theta, c->th_new, sizeof(double) * K, cudaMemcpyDeviceToDevice, s));
    std::swap(c->U, c->Un);
    CK(cudaEventRecord(c->ev[7], s));
    CK(cudaEventRecord(c->ev[8], s));
  } else {
    gemm(c, N2, m, K, 1.0, Z, ldz, c->F, K, 0.0, static_cast<const T*>(nullptr), 0, c->U32, c->ldu);
    CK(cudaEventRecord(c->ev[7], s));
    // A11: FP64-accurate refinement (FP64 products, or double-float ones in GREST_MIXED_FAST)
    grest_status st2 = c->cfg.precision == GREST_MIXED_FAST ? refine_mixed(c, N2) : refine_mixed_f64(c, N2);
    if (st2 != GREST_OK) return st2;
    CK(cudaEventRecord(c->ev[8], s));
  }
  c->Ku = K;
  c->stats.m = m;
  c->stats.k_u = Ku;
  c->stats.rank_q = r;
  c->stats.mode = mode;
  c->last_m = m;
  return GREST_OK;
}

// Ynew = a MY + b Y + g Yold over n x w (shared ld; Yold may be Ynew): one
// step of the scaled Chebyshev recurrence
__global__ void k_cheb_step(const double* __restrict__ MY, const double* __restrict__ Y, const double* Yold,
                            double* Ynew, int64_t ld, int w, int64_t n, double a, double b, double g) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * w; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t o = (e / w) * ld + (e % w);
    Ynew[o] = fma(a, MY[o], fma(b, Y[o], Yold ? g * Yold[o] : 0.0));
  }
}

// H[r0 + i][c0 + j] = A[i][j] (+ B[i][j]) for an a x w block (ld w)
__global__ void k_put_block(double* __restrict__ H, int64_t ldh, int64_t c0, const double* __restrict__ A,
                            const double* __restrict__ B, int a, int w) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)a * w) return;
  const int64_t i = e / w, j = e % w;
  H[i * ldh + c0 + j] = B ? A[e] + B[e] : A[e];
}

// H (m x m): the strict lower triangle from the upper one
__global__ void k_mirror_upper(double* __restrict__ H, int64_t ld, int m) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)m * m) return;
  const int64_t r = e / m, cc = e % m;
  if (r > cc) H[r * ld + cc] = H[cc * ld + r];
}

// Alg. 2's initial pairs on the device: the K leading pairs of M^(0) (FP64).
// Two kinds of round, each ending in Rayleigh-Ritz for b = K + max(8, K/2)
// vectors X and the residuals of the K tracked ones:
//  * block Krylov: the basis V = [V_0 .. V_s] (n x m, m = (s+1) b <= 512,
//    V_0 = X) grows by V_{j+1} = orth(M V_j), two classical Gram-Schmidt
//    passes against all of V and CholQR2; H = V^T M V is assembled from the
//    Gram-Schmidt coefficients (block column j of H is V^T M V_j).  A block
//    Gram-Schmidt leaves rank deficient (converged pairs, an invariant
//    subspace) has the missing columns replaced by Gaussian ones.
//  * Chebyshev-filtered subspace iteration (Zhou and Saad, J. Comput. Phys.
//    2007, scaled three-term recurrence): once the block is within 1e-3 of
//    converging, the leading pairs that already meet the tolerance are
//    locked, and the other columns are multiplied by a Chebyshev polynomial
//    that damps [lower bound, cut] (ADJ: a polynomial in M^2 on
//    [0, theta_b^2], as both ends of the spectrum are wanted; LAP / NLAP: in
//    M on [0, theta_b]) with the locked vectors projected out after every
//    product, then re-orthonormalized.  Its cost is mostly SpMMs, which on
//    this hardware are far cheaper than the FP64 Gram-Schmidt of a Krylov
//    round; a round that does not halve the residual goes back to Krylov.
// Stops when every tracked residual ||M x - theta x|| is at most
// tol |theta_1|.  Graphs of at most 288 nodes take the dense route: H = M.
grest_status initial_pairs_device(grest_ctx* c, int max_rounds, double tol) {
  cudaStream_t s = c->stream;
  const int K = c->K, op = c->cfg.op;
  const int64_t n = c->g.n;
  if (n < K) return GREST_ERR_INVALID_ARG;
  const bool dense = n <= 288;
  int b = std::min<int64_t>(K + std::max(8, K / 2), std::min<int64_t>(c->cmax, n));
  int sdeg = dense ? 0 : (int)std::min<int64_t>(16, std::min<int64_t>(512 / b - 1, n / b - 1));
  if (!dense && sdeg < 1) return GREST_ERR_INVALID_ARG;
  const int m = dense ? (int)n : (sdeg + 1) * b;
  double *V = nullptr, *W = nullptr, *MX = nullptr, *Hc = nullptr, *C1 = nullptr, *C2 = nullptr, *F = nullptr,
         *rz = nullptr, *th = nullptr, *ew = nullptr;
  CK(dalloc(&V, n * (int64_t)m)); CK(dalloc(&W, n * (int64_t)b)); CK(dalloc(&MX, n * (int64_t)b));
  CK(dalloc(&Hc, (int64_t)m * m)); CK(dalloc(&C1, (int64_t)m * b)); CK(dalloc(&C2, (int64_t)m * b));
  CK(dalloc(&F, (int64_t)m * b)); CK(dalloc(&rz, m)); CK(dalloc(&th, b)); CK(dalloc(&ew, eig_work_doubles(m)));
  struct Free {
    double** p[10];
    ~Free() { for (auto q : p) { cudaFree(*q); *q = nullptr; } }
  } fr{{&V, &W, &MX, &Hc, &C1, &C2, &F, &rz, &th, &ew}};
  auto sym_eig = [&](int mm, int k) {
    int p = prof_begin(c);
    c->launches += sym_eig_select(Hc, mm, mm, k, op, th, F, k, rz, c->info + 56, ew, false, s);
    prof_end(c, p, 3, 4.0 * mm * mm * mm / 3.0 + 2.0 * mm * mm * k);
  };
  auto finish = [&](const double* X, int64_t ldx) -> grest_status {
    CK(cudaMemcpy2DAsync(c->U, sizeof(double) * c->ldu, X, sizeof(double) * ldx, sizeof(double) * K, n,
                         cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(c->theta, th, sizeof(double) * K, cudaMemcpyDeviceToDevice, s));
    c->launches += sign_normalize_fast(c->U, c->ldu, K, n, c->part, c->ipart, s);
    CK(cudaGetLastError());
    {
      const grest_status rb = read_back(c, 0);
      if (rb != GREST_OK) return rb;
    }
    return *c->h_err ? map_dev_err(*c->h_err) : GREST_OK;
  };
  if (dense) {
    // H = M I, all n pairs of the dense operator; the K leading ones are X
    k_fill_identity<double><<<(unsigned)((n * n + 255) / 256), 256, 0, s>>>(V, n, (int)n);
    spmm(c, (const double*)V, n, Hc, n, (int)n, 0, n, 0);
    symmetrize(Hc, n, (int)n, s);
    c->launches += 2;
    b = std::min<int>(b, (int)n);
    sym_eig((int)n, K);
    return finish(F, K);
  }
  // |M| <= ub: Gershgorin (ADJ: d_max; LAP: alpha = 2 d_max; NLAP: 2), the
  // reference for the rank test of a new block
  CK(cudaMemcpyAsync(c->h_info, c->g.dmax, sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  const double dmax = c->h_info[0];
  const double ub = std::max(op == GREST_OP_NLAP ? 2.0 : (op == GREST_OP_LAP ? 2.0 * dmax : dmax), 1e-300);
  uint64_t draws = 0;  // Philox stream index of the Gaussian blocks
  // columns [col0, col0 + w) of V: orthonormal Gaussian columns orthogonal to V's columns before col0
  auto random_cols = [&](int col0, int w) -> grest_status {
    for (int attempt = 0; attempt < 4; ++attempt) {
      gaussian_omega(W, b, n, w, c->cfg.seed ^ 0x494e495449414cull, draws++, s);
      c->launches += 1;
      for (int pass = 0; pass < 2 && col0 > 0; ++pass) {
        gram(c, (const double*)V, m, col0, (const double*)W, b, w, n, C1, w, false);
        gemm(c, n, col0, w, -1.0, (const double*)V, m, C1, w, 1.0, (const double*)W, b, W, b);
      }
      int r = 0;
      grest_status st = cholqr_pass(c, (const double*)W, b, w, n, 1e-10, 0.0, nullptr, V + col0, m, 0, true, &r);
      if (st != GREST_OK) return st;
      if (r < w) continue;
      st = cholqr_pass(c, (const double*)(V + col0), m, w, n, 1e-14, 0.0, nullptr, W, b, 4, false, &r);
      if (st != GREST_OK) return st;
      copy_cols_f64(W, b, V + col0, m, n, w, s);
      c->launches += 1;
      return GREST_OK;
    }
    return GREST_ERR_NUMERIC;
  };
  grest_status st = random_cols(0, b);
  if (st != GREST_OK) return st;
  bool have_mx = false;  // MX = M V_0 from the previous round's residual check
  bool krylov = true;
  double prev = HUGE_VAL;
  int nc = 0;            // locked leading pairs (Chebyshev rounds)
  std::vector<double> hres(K), hth(b);
  // Chebyshev rounds work in V_0 with V_1 .. V_4 as scratch (needs s >= 4)
  const bool cheb_ok = sdeg >= 4;
  const unsigned gbk = (unsigned)std::min<int64_t>((n * b + 255) / 256, 152 * 32);
  auto deflate = [&](double* Y, int w) {  // Y -= X_L (X_L^T Y), X_L = V_0[:, :nc]
    if (nc == 0) return;
    gram(c, (const double*)V, m, nc, (const double*)Y, m, w, n, C1, w, false);
    gemm(c, n, nc, w, -1.0, (const double*)V, m, C1, w, 1.0, (const double*)Y, m, Y, m);
  };
  for (int round = 0; round < max_rounds; ++round) {
    if (krylov) {
      for (int j = 0; j <= sdeg; ++j) {
        double* Vj = V + (int64_t)j * b;
        const int a = (j + 1) * b;  // columns of V so far
        if (j == 0 && have_mx) {
          copy_cols_f64(MX, b, W, b, n, b, s);
          c->launches += 1;
        } else {
          spmm(c, (const double*)Vj, m, W, b, b, 0, n, 0);
        }
        // block column j of H = V^T M V_j: first Gram-Schmidt pass
        gram(c, (const double*)V, m, a, (const double*)W, b, b, n, C1, b, false);
        if (j == sdeg) {
          k_put_block<<<(unsigned)((a * b + 255) / 256), 256, 0, s>>>(Hc, m, (int64_t)j * b, C1, nullptr, a, b);
          c->launches += 1;
          break;
        }
        gemm(c, n, a, b, -1.0, (const double*)V, m, C1, b, 1.0, (const double*)W, b, W, b);
        gram(c, (const double*)V, m, a, (const double*)W, b, b, n, C2, b, false);
        gemm(c, n, a, b, -1.0, (const double*)V, m, C2, b, 1.0, (const double*)W, b, W, b);
        k_put_block<<<(unsigned)((a * b + 255) / 256), 256, 0, s>>>(Hc, m, (int64_t)j * b, C1, C2, a, b);
        c->launches += 1;
        // V_{j+1} = CholQR2(W).  Directions left at the rounding level of |M|
        // (pairs that have converged, or an invariant subspace reached) are
        // replaced by Gaussian columns orthogonal to everything before them.
        int r = 0;
        double* Vn = Vj + b;
        st = cholqr_pass(c, (const double*)W, b, b, n, 1e-13, ub, nullptr, Vn, m, 0, true, &r);
        if (st != GREST_OK) return st;
        if (r > 0) {
          st = cholqr_pass(c, (const double*)Vn, m, r, n, 1e-14, 0.0, nullptr, W, b, 4, false, &r);
          if (st != GREST_OK) return st;
          copy_cols_f64(W, b, Vn, m, n, r, s);
          c->launches += 1;
        }
        if (r < b) {
          st = random_cols((j + 1) * b + r, b - r);
          if (st != GREST_OK) return st;
        }
      }
      // Rayleigh-Ritz in span(V): the b leading pairs, X = V F
      k_mirror_upper<<<(unsigned)(((int64_t)m * m + 255) / 256), 256, 0, s>>>(Hc, m, m);
      c->launches += 1;
      sym_eig(m, b);
      gemm(c, n, m, b, 1.0, (const double*)V, m, F, b, 0.0, (const double*)nullptr, 0, W, b);
    } else {
      // filter the active columns V_0[:, nc:] in place (t = M^2 for ADJ, M otherwise)
      const int a = b - nc;
      double* Xa = V + nc;
      const double cut = op == GREST_OP_ADJ ? std::fabs(hth[b - 1]) : hth[b - 1];
      const double a0 = 0.0;  // M^2 >= 0; T = alpha I - L >= 0; T_n >= 0
      const double tb = op == GREST_OP_ADJ ? ub * ub : ub;
      double a1 = op == GREST_OP_ADJ ? cut * cut : cut;
      // a cut at the spectral bound (a multiple top eigenvalue) leaves no room above it
      if (!(tb - a1 > 1e-3 * (tb - a0))) a1 = a0 + 0.5 * (tb - a0);
      if (!(a1 > a0) || !(tb > a1)) return GREST_ERR_NUMERIC;
      const double c0 = 0.5 * (a0 + a1), e0 = 0.5 * (a1 - a0);
      const double sigma1 = e0 / (tb - c0);
      // degree: the largest active pair gains at most 1e6 over the cut, so the
      // filtered block keeps a condition number CholQR2 orthonormalizes to O(u)
      const double t1 = op == GREST_OP_ADJ ? hth[nc] * hth[nc] : hth[nc];
      const double z1 = std::max((t1 - c0) / e0, 1.0);
      int degree = 1;
      for (double tm = 1.0, tk = z1; degree < 32;) {
        const double tn = 2.0 * z1 * tk - tm;
        if (!(tn <= 1e6)) break;
        tm = tk;
        tk = tn;
        ++degree;
      }
      double* P0 = V + 1 * (int64_t)b;  // Y_{k-1}
      double* P1 = V + 2 * (int64_t)b;  // Y_k
      double* Tb = V + 3 * (int64_t)b;  // T Y_k
      double* T2 = V + 4 * (int64_t)b;  // M Y_k (ADJ)
      auto apply_t = [&](const double* in, double* out) {
        if (op == GREST_OP_ADJ) {
          spmm(c, in, m, T2, m, a, 0, n, 0);
          deflate(T2, a);
          spmm(c, (const double*)T2, m, out, m, a, 0, n, 0);
        } else {
          spmm(c, in, m, out, m, a, 0, n, 0);
        }
        deflate(out, a);
      };
      copy_cols_f64(Xa, m, P0, m, n, a, s);
      apply_t(P0, Tb);
      k_cheb_step<<<gbk, 256, 0, s>>>(Tb, P0, nullptr, P1, m, a, n, sigma1 / e0, -c0 * sigma1 / e0, 0.0);
      c->launches += 2;
      double sigma = sigma1;
      for (int k = 2; k <= degree; ++k) {
        const double sigma_new = 1.0 / (2.0 / sigma1 - sigma);
        apply_t(P1, Tb);
        k_cheb_step<<<gbk, 256, 0, s>>>(Tb, P1, P0, P0, m, a, n, 2.0 * sigma_new / e0, -2.0 * sigma_new * c0 / e0,
                                        -sigma * sigma_new);
        c->launches += 1;
        std::swap(P0, P1);
        sigma = sigma_new;
      }
      // P1 = filtered block: project out X_L twice, CholQR2 into V_0[:, nc:]
      deflate(P1, a);
      deflate(P1, a);
      int r = 0;
      st = cholqr_pass(c, (const double*)P1, m, a, n, 1e-14, 0.0, nullptr, Xa, m, 0, true, &r);
      if (st != GREST_OK) return st;
      if (r < a) {  // the filter collapsed some columns: Gaussian ones take their place
        st = random_cols(nc + r, a - r);
        if (st != GREST_OK) return st;
      }
      st = cholqr_pass(c, (const double*)Xa, m, a, n, 1e-14, 0.0, nullptr, P0, m, 4, false, &r);
      if (st != GREST_OK) return st;
      copy_cols_f64(P0, m, Xa, m, n, a, s);
      // Rayleigh-Ritz in span(V_0)
      spmm(c, (const double*)V, m, MX, b, b, 0, n, 0);
      gram(c, (const double*)V, m, b, (const double*)MX, b, b, n, Hc, b, false);
      symmetrize(Hc, b, b, s);
      c->launches += 2;
      sym_eig(b, b);
      gemm(c, n, b, b, 1.0, (const double*)V, m, F, b, 0.0, (const double*)nullptr, 0, W, b);
    }
    spmm(c, (const double*)W, b, MX, b, b, 0, n, 0);
    residual_norms(MX, W, b, K, th, n, c->part, c->resn, s);
    c->launches += 1;
    CK(cudaMemcpyAsync(hres.data(), c->resn, sizeof(double) * K, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(hth.data(), th, sizeof(double) * b, cudaMemcpyDeviceToHost, s));
    {
      const grest_status rb = read_back(c, 0);
      if (rb != GREST_OK) return rb;
    }
    if (*c->h_err) return map_dev_err(*c->h_err);
    const double scale = std::max(std::fabs(hth[0]), 1e-300);
    double rmax = 0.0;
    for (int j = 0; j < K; ++j) rmax = std::max(rmax, hres[j]);
    if (!(rmax == rmax)) return GREST_ERR_NUMERIC;
    if (rmax <= tol * scale) return finish(W, b);
    // next round starts from V_0 = X (orthonormal: V and F are), M V_0 = MX
    copy_cols_f64(W, b, V, m, n, b, s);
    c->launches += 1;
    have_mx = true;
    krylov = !cheb_ok || rmax > 1e-3 * scale || rmax > 0.5 * prev;
    prev = rmax;
    nc = 0;
    if (!krylov)
      while (nc < K && hres[nc] <= tol * scale) ++nc;
  }
  return GREST_ERR_NUMERIC;
}

grest_status run_checks(grest_ctx* c, int64_t n) {
  // M U, residual norms, orthonormality and Galerkin residual, in FP64
  cudaStream_t s = c->stream;
  const int K = c->K;
  double* MU = c->Un;  // free after the step; same leading dimension as U
  spmm(c, c->U, c->ldu, MU, c->ldu, K, 0, n, 0);
  residual_norms(MU, c->U, c->ldu, K, c->theta, n, c->part, c->resn, s);
  gram(c, c->U, c->ldu, K, c->U, c->ldu, K, n, c->Cm, K, true);
  k_orth_err<<<1, 256, 0, s>>>(c->Cm, K, K, c->info + 36);
  c->launches += 3;  // residual_norms (2) + k_orth_err
  // R = MU - U theta, Galerkin residual: Z^T R for the FP64 path (Z = [X_bar, Q]),
  // U^T R for the mixed path (its last Rayleigh-Ritz runs in span(U))
  double* R = c->Rres;
  k_resid_vecs<<<1024, 256, 0, s>>>(MU, c->U, c->ldu, K, c->theta, n, R, c->ldu);
  if (c->cfg.precision == GREST_FP64) {
    gram(c, Zp<double>(c), c->ldz, c->last_m, R, c->ldu, K, n, c->H, K, false);
    k_maxabs<<<1, 256, 0, s>>>(c->H, K, c->last_m, K, c->info + 37);
  } else {
    gram(c, c->U, c->ldu, K, R, c->ldu, K, n, c->H, K, false);
    k_maxabs<<<1, 256, 0, s>>>(c->H, K, K, K, c->info + 37);
  }
  c->launches += 2;  // k_resid_vecs + k_maxabs
  return GREST_OK;
}

}  // namespace

extern "C" {

grest_status grest_config_default(grest_config* cfg, int32_t k) {
  if (!cfg) return GREST_ERR_INVALID_ARG;
  memset(cfg, 0, sizeof(*cfg));
  cfg->op = GREST_OP_ADJ;
  cfg->k = k;
  cfg->subspace = GREST_SUB_AUTO;
  cfg->L = 100;
  cfg->P = 100;
  cfg->precision = GREST_FP64;
  cfg->projection = GREST_PROJ_EXACT;
  cfg->w_block = GREST_WB_RESID;
  cfg->seed = 0;
  cfg->drop_tol = 1e-7;
  return GREST_OK;
}

const char* grest_status_str(grest_status s) {
  switch (s) {
    case GREST_OK: return "ok";
    case GREST_ERR_INVALID_ARG: return "invalid argument";
    case GREST_ERR_INVALID_UPDATE: return "invalid update batch";
    case GREST_ERR_OOM: return "device out of memory";
    case GREST_ERR_CAPACITY: return "capacity exceeded";
    case GREST_ERR_NUMERIC: return "numerical breakdown";
    case GREST_ERR_CUDA: return "CUDA error";
    case GREST_ERR_TIMEOUT: return "device wait timed out";
    case GREST_ERR_UNSUPPORTED: return "unsupported option";
  }
  return "unknown status";
}

grest_status grest_init(const grest_config* cfg, int64_t n, const int64_t* rowptr, const int32_t* col,
                        const double* val, const double* U0, const double* theta0, void* cuda_stream,
                        grest_ctx** out) {
  if (!cfg || !out || n < 1 || !rowptr || (!col && rowptr[n] > 0)) return GREST_ERR_INVALID_ARG;
  const size_t bytes0 = t_dev_bytes;
  *out = nullptr;
  if (cfg->k < 1 || cfg->k > 64 || cfg->op < 0 || cfg->op > 2 || cfg->L < 1 || cfg->P < 0 || cfg->L + cfg->P > 256 ||
      cfg->subspace < 0 || cfg->subspace > 3 || !(cfg->drop_tol > 0.0) || cfg->k > n)
    return GREST_ERR_INVALID_ARG;
  if ((cfg->precision != GREST_FP64 && cfg->precision != GREST_MIXED && cfg->precision != GREST_MIXED_FAST) ||
      (cfg->projection != GREST_PROJ_EXACT && cfg->projection != GREST_PROJ_LOWRANK) ||
      (cfg->w_block != GREST_WB_RESID && cfg->w_block != GREST_WB_DELTA))
    return GREST_ERR_INVALID_ARG;
  // the explicit Delta of the paper's block and of Eq. main3 is formed for the
  // adjacency and the shifted Laplacian; the low-rank surrogate has no FP64
  // refinement in the mixed path
  if ((cfg->projection == GREST_PROJ_LOWRANK || cfg->w_block == GREST_WB_DELTA) && cfg->op == GREST_OP_NLAP)
    return GREST_ERR_UNSUPPORTED;
  if (cfg->projection == GREST_PROJ_LOWRANK && cfg->precision != GREST_FP64) return GREST_ERR_UNSUPPORTED;
  if ((U0 == nullptr) != (theta0 == nullptr)) return GREST_ERR_INVALID_ARG;
  const int64_t nnz = rowptr[n];
  for (int64_t i = 0; i < n; ++i)
    if (rowptr[i + 1] < rowptr[i]) return GREST_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return GREST_ERR_CUDA;
  grest_ctx* c = new grest_ctx();
  for (auto& e : c->ev) e = nullptr;
  for (auto& e : c->pev) e = nullptr;
  c->cfg = *cfg;
  c->dev = dev;
  c->stream = (cudaStream_t)cuda_stream;
  c->K = cfg->k;
  c->Ku = cfg->k;
  c->q = cfg->L + cfg->P;
  c->Lr = cfg->L;
  c->cmax = cfg->k + std::max(c->q, cfg->L);
  c->mmax = cfg->k + c->cmax;
  c->ldu = round_up(c->K, 8);
  c->ldz = round_up(c->mmax, 8);
  c->ldq = round_up(c->q, 8);
  c->ldv = round_up(std::max(c->cmax, c->K), 8);
  Csr& g = c->g;
  g.n = n;
  g.n_cap = cfg->node_capacity > 0 ? cfg->node_capacity : (n + n / 4 + 1024);
  if (g.n_cap < n) { free_ctx(c); return GREST_ERR_INVALID_ARG; }
  // host layout with slack: cap = len + len/4 + 4, rows sorted
  std::vector<int64_t> off(n);
  std::vector<int32_t> len(n), cap(n);
  int64_t total = 0;
  for (int64_t i = 0; i < n; ++i) {
    len[i] = (int32_t)(rowptr[i + 1] - rowptr[i]);
    cap[i] = len[i] + len[i] / 4 + 4;
    off[i] = total;
    total += cap[i];
  }
  g.nnz_cap = cfg->nnz_capacity > 0 ? cfg->nnz_capacity : (2 * total + (1 << 20));
  if (g.nnz_cap < total) { free_ctx(c); return GREST_ERR_INVALID_ARG; }
  std::vector<int32_t> hcol(total, 0);
  std::vector<double> hval(val ? total : 0, 0.0), hdeg(n, 0.0);
  for (int64_t i = 0; i < n; ++i) {
    std::vector<std::pair<int32_t, double>> row;
    row.reserve(len[i]);
    for (int64_t j = rowptr[i]; j < rowptr[i + 1]; ++j) {
      int32_t cj = col[j];
      if (cj < 0 || cj >= n || cj == i) { free_ctx(c); return GREST_ERR_INVALID_ARG; }
      double w = val ? val[j] : 1.0;
      if (!(w > 0.0) || w != w) { free_ctx(c); return GREST_ERR_INVALID_ARG; }
      row.push_back({cj, w});
    }
    std::sort(row.begin(), row.end());
    for (size_t j = 0; j < row.size(); ++j) {
      if (j > 0 && row[j].first == row[j - 1].first) { free_ctx(c); return GREST_ERR_INVALID_ARG; }
      hcol[off[i] + j] = row[j].first;
      if (val) hval[off[i] + j] = row[j].second;
      hdeg[i] += row[j].second;
    }
  }
  (void)nnz;
#define IK(x)                            \
  do {                                   \
    cudaError_t e_ = (x);                \
    if (e_ != cudaSuccess) {             \
      free_ctx(c);                       \
      return from_cuda(e_);              \
    }                                    \
  } while (0)
  const int64_t nc = g.n_cap;
  IK(dalloc(&g.row_off, nc)); IK(dalloc(&g.row_len, nc)); IK(dalloc(&g.row_cap, nc));
  IK(dalloc(&g.col, g.nnz_cap));
  if (val) IK(dalloc(&g.val, g.nnz_cap));
  IK(dalloc(&g.live, nc)); IK(dalloc(&g.deg, nc)); IK(dalloc(&g.dis, nc));
  IK(dalloc(&g.arena_top, 1)); IK(dalloc(&g.dmax, 1));
  GraphWork& w = c->gw;
  IK(dalloc(&w.cnt, nc + 1)); IK(dalloc(&w.seg, nc + 1)); IK(dalloc(&w.cursor, nc)); IK(dalloc(&w.delflag, nc));
  IK(dalloc(&w.rowflag, nc + 1)); IK(dalloc(&w.touched, nc)); IK(dalloc(&w.tmp_off, nc + 1));
  IK(dalloc(&w.need, nc + 1)); IK(dalloc(&w.new_len, nc)); IK(dalloc(&w.long_rows, nc));
  IK(dalloc(&w.scalars, 8));
  IK(dmalloc((void**)&w.scan_tmp, scan_temp_bytes(nc + 1)));
  {
    int64_t mb = cfg->max_batch_edges > 0 ? cfg->max_batch_edges : (1 << 20);
    if (ensure_graph_work(c, 2 * mb) != GREST_OK) { free_ctx(c); return GREST_ERR_OOM; }
    if (ensure_batch(c, mb, 1024) != GREST_OK) { free_ctx(c); return GREST_ERR_OOM; }
  }
  IK(dalloc(&c->U, nc * c->ldu)); IK(dalloc(&c->Un, nc * c->ldu)); IK(dalloc(&c->theta, 64));
  c->esz = cfg->precision != GREST_FP64 ? sizeof(float) : sizeof(double);
  IK(dmalloc((void**)&c->Zv, c->esz * nc * c->ldz)); IK(dmalloc((void**)&c->MZv, c->esz * nc * c->ldz));
  IK(dmalloc((void**)&c->V2v, c->esz * nc * c->ldv));
  IK(dmalloc((void**)&c->Yrv, c->esz * nc * c->ldq)); IK(dmalloc((void**)&c->Yr2v, c->esz * nc * c->ldq));
  IK(dmalloc((void**)&c->Idv, c->esz * (int64_t)c->q * c->ldq));
  if (cfg->precision != GREST_FP64) IK(dalloc(&c->U32, nc * c->ldu));
  if (cfg->flags & GREST_FLAG_CHECK) IK(dalloc(&c->Rres, nc * c->ldu));
  const int cm = c->cmax, mm = c->mmax;
  IK(dalloc(&c->Cm, 64 * 64)); IK(dalloc(&c->Cv, (int64_t)64 * (cm + 64))); IK(dalloc(&c->G, (int64_t)cm * cm));
  IK(dalloc(&c->T, (int64_t)cm * cm)); IK(dalloc(&c->H, (int64_t)mm * mm)); IK(dalloc(&c->F, (int64_t)mm * 64));
  // Gs, Uh: the RSVD's q x q problem and the refinement's K x K products
  const int64_t qk = std::max(c->q, c->K);
  IK(dalloc(&c->XtM, (int64_t)64 * c->ldq)); IK(dalloc(&c->Gs, qk * qk));
  IK(dalloc(&c->Uh, qk * qk)); IK(dalloc(&c->ritz, mm)); IK(dalloc(&c->th_new, 64));
  IK(dalloc(&c->tmpk, 256)); IK(dalloc(&c->info, 64)); IK(dalloc(&c->resn, 64));
  c->part_cap = 8'000'000;  // FP64 partial sums of the split-K Gram kernels (64 MB)
  IK(dalloc(&c->part, c->part_cap)); IK(dalloc(&c->ipart, 304 * 64));
  IK(dalloc(&c->eigwork, eig_work_doubles(std::max(mm, c->q))));
  IK(dalloc(&c->piv, std::max(mm, c->q) + 8));
  IK(dalloc(&c->dmax_old, 1));
  IK(dalloc(&c->XZ, (int64_t)64 * mm));
  c->gemm_img_cap = gemm_tc_img_bytes(512, 256);
  IK(dalloc(&c->gemm_img, c->gemm_img_cap));
  if (n >= kOverlapRows && (cfg->flags & GREST_FLAG_TWO_STREAMS) &&
      (cfg->subspace == GREST_SUB_AUTO || cfg->subspace == GREST_SUB_RSVD)) {
    int lo = 0, hi = 0;
    IK(cudaDeviceGetStreamPriorityRange(&lo, &hi));
    IK(cudaStreamCreateWithPriority(&c->s2, cudaStreamNonBlocking, hi));
    IK(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
    IK(cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming));
    IK(dalloc(&c->part2, c->part_cap));
    IK(dmalloc((void**)&c->gemm_img2, c->gemm_img_cap));
    IK(dalloc(&c->Cv2, (int64_t)64 * (cm + 64)));
  }
  IK(dalloc(&c->err, 1));
  IK(cudaMallocHost((void**)&c->h_info, sizeof(double) * 64));
  IK(cudaMallocHost((void**)&c->h_err, sizeof(int32_t)));
  IK(cudaMallocHost((void**)&c->h_scal, sizeof(int64_t) * 8));
  for (auto& e : c->ev) IK(cudaEventCreate(&e));
  for (auto& e : c->pev) IK(cudaEventCreate(&e));
  cudaStream_t s = c->stream;
  // graph upload
  IK(cudaMemcpyAsync(g.row_off, off.data(), sizeof(int64_t) * n, cudaMemcpyHostToDevice, s));
  IK(cudaMemcpyAsync(g.row_len, len.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, s));
  IK(cudaMemcpyAsync(g.row_cap, cap.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, s));
  IK(cudaMemcpyAsync(g.col, hcol.data(), sizeof(int32_t) * total, cudaMemcpyHostToDevice, s));
  if (val) IK(cudaMemcpyAsync(g.val, hval.data(), sizeof(double) * total, cudaMemcpyHostToDevice, s));
  IK(cudaMemcpyAsync(g.deg, hdeg.data(), sizeof(double) * n, cudaMemcpyHostToDevice, s));
  IK(cudaMemsetAsync(g.live, 0, nc, s));
  IK(cudaMemsetAsync(g.live, 1, n, s));
  IK(cudaMemcpyAsync(g.arena_top, &total, sizeof(int64_t), cudaMemcpyHostToDevice, s));
  IK(cudaMemsetAsync(c->err, 0, sizeof(int32_t), s));
  // initial pairs given by the caller (else computed on the device below)
  if (U0) {
    std::vector<double> hu((size_t)n * c->ldu, 0.0);
    for (int64_t i = 0; i < n; ++i)
      for (int j = 0; j < c->K; ++j) hu[(size_t)i * c->ldu + j] = U0[(size_t)i * c->K + j];
    IK(cudaMemcpyAsync(c->U, hu.data(), sizeof(double) * hu.size(), cudaMemcpyHostToDevice, s));
    IK(cudaMemcpyAsync(c->theta, theta0, sizeof(double) * c->K, cudaMemcpyHostToDevice, s));
    IK(cudaStreamSynchronize(s));
  }
  if (c->esz == sizeof(double))
    k_fill_identity<double><<<(unsigned)((c->q * c->q + 255) / 256), 256, 0, s>>>(static_cast<double*>(c->Idv), c->ldq, c->q);
  else
    k_fill_identity<float><<<(unsigned)((c->q * c->q + 255) / 256), 256, 0, s>>>(static_cast<float*>(c->Idv), c->ldq, c->q);
  (void)graph_refresh_derived(g, w, n, s);
  IK(cudaGetLastError());
  IK(cudaStreamSynchronize(s));
#undef IK
  c->stats.n_nodes = n;
  c->stats.nnz = nnz;
  c->nnz = nnz;
  c->dev_bytes = t_dev_bytes - bytes0;  // the solver's temporaries below are released before returning
  if (!U0) {
    const grest_status ist = initial_pairs_device(c, 100, 1e-11);
    if (ist != GREST_OK) {
      free_ctx(c);
      return ist;
    }
  }
  *out = c;
  return GREST_OK;
}

grest_status grest_get_device_bytes(grest_ctx* c, int64_t* bytes) {
  if (!c || !bytes) return GREST_ERR_INVALID_ARG;
  *bytes = (int64_t)c->dev_bytes;
  return GREST_OK;
}

static grest_status apply_update_impl(grest_ctx* c, const grest_update* u, grest_stats* stats) {
  if (!c || !u) return GREST_ERR_INVALID_ARG;
  if (u->n_new_nodes < 0 || u->n_ins < 0 || u->n_del < 0 || u->n_del_nodes < 0) return GREST_ERR_INVALID_ARG;
  if ((u->n_ins > 0 && (!u->ins_u || !u->ins_v)) || (u->n_del > 0 && (!u->del_u || !u->del_v)) ||
      (u->n_del_nodes > 0 && !u->del_nodes))
    return GREST_ERR_INVALID_ARG;
  if (u->ins_w && !c->g.val) return GREST_ERR_INVALID_ARG;
  const bool delta_modes = c->cfg.projection == GREST_PROJ_LOWRANK || c->cfg.w_block == GREST_WB_DELTA;
  if (delta_modes && u->n_del_nodes > 0) return GREST_ERR_UNSUPPORTED;  // Delta of a removed row is not kept
  if (cudaSetDevice(c->dev) != cudaSuccess) return GREST_ERR_CUDA;
  cudaStream_t s = c->stream;
  const int64_t N = c->g.n, S = u->n_new_nodes;
  if (N + S > INT32_MAX) return GREST_ERR_CAPACITY;
  c->prof_n = 0;
  c->launches = 0;
  grest_status st = GREST_OK;
  if (N + S > c->g.n_cap) {
    st = grow_nodes(c, N + S);
    if (st != GREST_OK) return st;
  }
  st = ensure_batch(c, std::max(u->n_ins, u->n_del), u->n_del_nodes);
  if (st != GREST_OK) return st;
  CK(cudaEventRecord(c->ev[0], s));
  const cudaMemcpyKind kind = u->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if (u->n_ins > 0) {
    CK(cudaMemcpyAsync(c->b_iu, u->ins_u, sizeof(int32_t) * u->n_ins, kind, s));
    CK(cudaMemcpyAsync(c->b_iv, u->ins_v, sizeof(int32_t) * u->n_ins, kind, s));
    if (u->ins_w) CK(cudaMemcpyAsync(c->b_w, u->ins_w, sizeof(double) * u->n_ins, kind, s));
  }
  if (u->n_del > 0) {
    CK(cudaMemcpyAsync(c->b_du, u->del_u, sizeof(int32_t) * u->n_del, kind, s));
    CK(cudaMemcpyAsync(c->b_dv, u->del_v, sizeof(int32_t) * u->n_del, kind, s));
  }
  if (u->n_del_nodes > 0) CK(cudaMemcpyAsync(c->b_dn, u->del_nodes, sizeof(int32_t) * u->n_del_nodes, kind, s));
  // entry buffers: both directions of every edit plus the edges of removed nodes
  int64_t entries = 2 * (u->n_ins + u->n_del);
  if (u->n_del_nodes > 0) {
    k_sum_removed_degree<<<1, 256, 0, s>>>(c->b_dn, u->n_del_nodes, N, c->g.row_len, c->gw.scalars + 4);
    c->launches += 1;
    CK(cudaMemcpyAsync(c->h_scal + 4, c->gw.scalars + 4, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    entries += c->h_scal[4];
  }
  st = ensure_graph_work(c, entries + 1);
  if (st != GREST_OK) return st;
  BatchDev bd;
  bd.S = S;
  bd.n_ins = u->n_ins;
  bd.n_del = u->n_del;
  bd.n_dn = u->n_del_nodes;
  bd.ins_u = c->b_iu;
  bd.ins_v = c->b_iv;
  bd.ins_w = u->ins_w ? c->b_w : nullptr;
  bd.del_u = c->b_du;
  bd.del_v = c->b_dv;
  bd.dn = c->b_dn;
  c->batch_new_edges = u->n_ins;
  if (delta_modes) CK(cudaMemcpyAsync(c->dmax_old, c->g.dmax, sizeof(double), cudaMemcpyDeviceToDevice, s));
  // A batch that does not fit the edge arena changes nothing (the commit is
  // skipped); the arena is then compacted into a larger one and the batch
  // applied again.
  for (int attempt = 0;; ++attempt) {
    CK(cudaMemsetAsync(c->err, 0, sizeof(int32_t), s));
    {
      int p = prof_begin(c);
      c->launches += graph_apply_batch(c->g, c->gw, bd, c->err, s);
      prof_end(c, p, 4, 0.0);
    }
    c->launches += graph_count_nnz(c->g, N + S, c->gw.scalars + 5, s);
    CK(cudaMemcpyAsync(c->h_scal + 5, c->gw.scalars + 5, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(c->h_scal + 7, c->gw.tmp_off + (N + S), sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    CK(cudaGetLastError());
    st = read_back(c, 0);
    if (st != GREST_OK) return st;
    if (*c->h_err == DERR_ARENA && attempt == 0) {
      // the merged rows of this batch need at most 1.5x their staged length plus a rounding slot each
      const int64_t staged = c->h_scal[7];
      st = grow_arena(c, N, staged + staged / 2 + 24 * (N + S));
      if (st != GREST_OK) return st;
      continue;
    }
    if (*c->h_err) {
      c->prof_n = 0;
      return map_dev_err(*c->h_err);
    }
    break;
  }
  c->nnz = c->h_scal[5];
  // committed: the graph now has N + S ids; until the step's pairs replace
  // them, the tracked pairs are the padded previous ones [X; 0]
  c->g.n = N + S;
  if (S > 0) CK(cudaMemset2DAsync(c->U + N * c->ldu, sizeof(double) * c->ldu, 0, sizeof(double) * c->K, S, s));
  c->launches += graph_refresh_derived(c->g, c->gw, N + S, s);
  c->stats.rank_y = 0;
  st = c->cfg.precision != GREST_FP64 ? step_t<float>(c, N, S, u->n_del_nodes > 0)
                                       : step_t<double>(c, N, S, u->n_del_nodes > 0);
  CK(cudaGetLastError());
  if (st != GREST_OK) return st;
  ++c->step;
  if (c->cfg.flags & GREST_FLAG_CHECK) run_checks(c, N + S);
  CK(cudaMemcpyAsync(c->h_info, c->info, sizeof(double) * 64, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(c->h_err, c->err, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(c->h_scal, c->g.arena_top, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  c->last_ritz.resize(c->last_m);
  CK(cudaMemcpyAsync(c->last_ritz.data(), c->ritz, sizeof(double) * c->last_m, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  CK(cudaGetLastError());
  if (*c->h_err) return map_dev_err(*c->h_err);
  grest_stats& S_ = c->stats;
  S_.step = c->step;
  S_.n_nodes = c->g.n;
  S_.nnz = c->nnz;
  prof_collect(c, S_);
  S_.kernel_launches = c->launches;
  S_.boundary_gap = c->h_info[28];
  if (c->h_info[24] < c->stats.rank_q) return GREST_ERR_NUMERIC;
  if (c->cfg.flags & GREST_FLAG_CHECK) {
    double th[64], rn[64];
    CK(cudaMemcpy(th, c->theta, sizeof(double) * c->K, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(rn, c->resn, sizeof(double) * c->K, cudaMemcpyDeviceToHost));
    double th1 = 0.0, mr = 0.0;
    for (int j = 0; j < c->K; ++j) {
      th1 = std::max(th1, std::fabs(th[j]));
      mr = std::max(mr, rn[j]);
    }
    S_.orth_err = c->h_info[36];
    S_.max_residual = th1 > 0 ? mr / th1 : mr;
    S_.galerkin = th1 > 0 ? c->h_info[37] / th1 : c->h_info[37];
  }
  S_.ms_total = ev_ms(c->ev[0], c->ev[8]);
  S_.ms_graph = ev_ms(c->ev[0], c->ev[1]);
  S_.ms_spmm = ev_ms(c->ev[1], c->ev[2]);
  S_.ms_basis = ev_ms(c->ev[2], c->ev[4]);
  S_.ms_project = ev_ms(c->ev[4], c->ev[5]);
  S_.ms_eig = ev_ms(c->ev[5], c->ev[6]);
  S_.ms_lift = ev_ms(c->ev[6], c->ev[7]);
  S_.ms_refine = ev_ms(c->ev[7], c->ev[8]);
  if (stats) *stats = S_;
  return GREST_OK;
}

grest_status grest_apply_update(grest_ctx* c, const grest_update* u, grest_stats* stats) {
  const size_t b0 = t_dev_bytes;
  const grest_status st = apply_update_impl(c, u, stats);
  if (c) c->dev_bytes += t_dev_bytes - b0;  // buffers grown for this batch
  return st;
}

grest_status grest_sync(grest_ctx* c) {
  if (!c) return GREST_ERR_INVALID_ARG;
  if (cudaSetDevice(c->dev) != cudaSuccess) return GREST_ERR_CUDA;
  return from_cuda(cudaStreamSynchronize(c->stream));
}

grest_status grest_get_embedding(grest_ctx* c, double* U, double* theta, uint8_t* live, int64_t* n_out,
                                 int32_t on_device) {
  if (!c || !n_out) return GREST_ERR_INVALID_ARG;
  if (cudaSetDevice(c->dev) != cudaSuccess) return GREST_ERR_CUDA;
  const int64_t n = c->g.n;
  *n_out = n;
  cudaStream_t s = c->stream;
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  // rows of U are contiguous when ldu = K: one linear copy (a pitched copy
  // of n rows of 8 K bytes runs far below the host link's bandwidth)
  if (U && c->ldu == c->K) CK(cudaMemcpyAsync(U, c->U, sizeof(double) * c->K * n, kind, s));
  else if (U) CK(cudaMemcpy2DAsync(U, sizeof(double) * c->K, c->U, sizeof(double) * c->ldu, sizeof(double) * c->K, n, kind, s));
  if (theta) CK(cudaMemcpyAsync(theta, c->theta, sizeof(double) * c->K, kind, s));
  if (live) CK(cudaMemcpyAsync(live, c->g.live, n, kind, s));
  return from_cuda(cudaStreamSynchronize(s));
}

}  // extern "C"

namespace grest {
// (X_K, Lambda_K) -> host memory mapped into the device's address space,
// written by the SMs over the host link: the GPU's copy engines stay free for
// the small reads the next update makes (a copy-engine transfer of U would
// hold them, and each such read would wait behind it).  16-byte stores when
// both sides allow them.
__global__ void k_pairs_to_host(const double* __restrict__ U, int64_t ldu, int K, int64_t n,
                                const double* __restrict__ theta, double* __restrict__ outU,
                                double* __restrict__ outT) {
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, nth = (int64_t)gridDim.x * blockDim.x;
  if (outT && tid < K) outT[tid] = theta[tid];
  if (!outU) return;
  const int64_t total = n * K;
  if (ldu == K && ((reinterpret_cast<uintptr_t>(U) | reinterpret_cast<uintptr_t>(outU)) & 15) == 0) {
    const double2* src = reinterpret_cast<const double2*>(U);
    double2* dst = reinterpret_cast<double2*>(outU);
    const int64_t m = total / 2;
    int64_t e = tid;
    // four 16-byte loads in flight per thread before their stores
    for (; e + 3 * nth < m; e += 4 * nth) {
      const double2 a = src[e], b = src[e + nth], c = src[e + 2 * nth], d = src[e + 3 * nth];
      dst[e] = a;
      dst[e + nth] = b;
      dst[e + 2 * nth] = c;
      dst[e + 3 * nth] = d;
    }
    for (; e < m; e += nth) dst[e] = src[e];
    if ((total & 1) && tid == 0) outU[total - 1] = U[total - 1];
  } else {
    for (int64_t e = tid; e < total; e += nth) outU[e] = U[(e / K) * ldu + (e % K)];
  }
}
}  // namespace grest

extern "C" {

grest_status grest_get_embedding_async(grest_ctx* c, double* U, double* theta, int64_t* n_out) {
  if (!c || !n_out) return GREST_ERR_INVALID_ARG;
  if (cudaSetDevice(c->dev) != cudaSuccess) return GREST_ERR_CUDA;
  if (!c->cstream) {
    CK(cudaStreamCreateWithFlags(&c->cstream, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&c->ev_ready, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&c->ev_copied, cudaEventDisableTiming));
  }
  const int64_t n = c->g.n;
  *n_out = n;
  cudaStream_t cs = c->cstream;
  CK(cudaEventRecord(c->ev_ready, c->stream));
  CK(cudaStreamWaitEvent(cs, c->ev_ready, 0));
  // pinned (mapped) host outputs: written by a kernel; anything else (device
  // memory, pageable host memory): cudaMemcpyAsync on the copy stream
  double *dU = nullptr, *dT = nullptr;
  const bool mapped = (!U || cudaHostGetDevicePointer((void**)&dU, U, 0) == cudaSuccess) &&
                      (!theta || cudaHostGetDevicePointer((void**)&dT, theta, 0) == cudaSuccess);
  cudaGetLastError();  // a failed lookup only selects the copy path
  if (mapped) {
    // few blocks: the copy overlaps the next update and should take little of it
    grest::k_pairs_to_host<<<64, 256, 0, cs>>>(c->U, c->ldu, c->K, n, c->theta, dU, dT);
    CK(cudaGetLastError());
  } else {
    if (U && c->ldu == c->K) CK(cudaMemcpyAsync(U, c->U, sizeof(double) * c->K * n, cudaMemcpyDefault, cs));
    else if (U) CK(cudaMemcpy2DAsync(U, sizeof(double) * c->K, c->U, sizeof(double) * c->ldu, sizeof(double) * c->K,
                                     n, cudaMemcpyDefault, cs));
    if (theta) CK(cudaMemcpyAsync(theta, c->theta, sizeof(double) * c->K, cudaMemcpyDefault, cs));
  }
  CK(cudaEventRecord(c->ev_copied, cs));
  c->copy_pending = true;
  return GREST_OK;
}

grest_status grest_wait_embedding(grest_ctx* c) {
  if (!c) return GREST_ERR_INVALID_ARG;
  if (cudaSetDevice(c->dev) != cudaSuccess) return GREST_ERR_CUDA;
  return settle_copy(c);
}

grest_status grest_set_embedding(grest_ctx* c, const double* U, const double* theta, int32_t on_device) {
  if (!c || !U || !theta) return GREST_ERR_INVALID_ARG;
  if (cudaSetDevice(c->dev) != cudaSuccess) return GREST_ERR_CUDA;
  {
    const grest_status st = settle_copy(c);
    if (st != GREST_OK) return st;
  }
  cudaStream_t s = c->stream;
  const int64_t n = c->g.n;
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  CK(cudaMemcpy2DAsync(c->U, sizeof(double) * c->ldu, U, sizeof(double) * c->K, sizeof(double) * c->K, n, kind, s));
  CK(cudaMemcpyAsync(c->theta, theta, sizeof(double) * c->K, kind, s));
  zero_dead_rows(c->U, c->ldu, c->K, c->g.live, n, s);
  c->Ku = c->K;
  CK(cudaGetLastError());
  return from_cuda(cudaStreamSynchronize(s));
}

// ------------------------------------------------------------------ checkpoints
// A checkpoint is one host byte array: a header, then the graph as a compact
// CSR (rows sorted, as the context keeps them), the weighted degrees as
// maintained by the updates, the tracked pairs and the live mask.  Restoring
// it gives a context whose next steps are bit-identical to the original's:
// the per-row neighbour order, the degrees, (X_K, Lambda_K) and the step
// counter (which seeds the RSVD test matrix) are all carried over.
namespace {

constexpr char kCkptMagic[8] = {'G', 'R', 'E', 'S', 'T', 'C', 'K', '1'};

struct CkptHeader {
  char magic[8];
  int32_t version, K;
  int64_t n, nnz, step, has_val;
  grest_config cfg;
};

struct CkptLayout {
  size_t rowptr, col, val, deg, U, theta, live, total;
};

inline size_t up8(size_t x) { return (x + 7) & ~(size_t)7; }

CkptLayout ckpt_layout(int64_t n, int64_t nnz, int K, bool has_val) {
  CkptLayout L;
  size_t o = up8(sizeof(CkptHeader));
  L.rowptr = o;
  o += sizeof(int64_t) * (size_t)(n + 1);
  L.col = o;
  o = up8(o + sizeof(int32_t) * (size_t)nnz);
  L.val = o;
  if (has_val) o += sizeof(double) * (size_t)nnz;
  L.deg = o;
  o += sizeof(double) * (size_t)n;
  L.U = o;
  o += sizeof(double) * (size_t)n * K;
  L.theta = o;
  o += sizeof(double) * (size_t)K;
  L.live = o;
  L.total = up8(o + (size_t)n);
  return L;
}

// Header and size checks of a checkpoint (host only); rowptr is checked too.
bool ckpt_parse(const void* buf, int64_t bytes, CkptHeader* h, CkptLayout* L) {
  if (!buf || bytes < (int64_t)sizeof(CkptHeader)) return false;
  memcpy(h, buf, sizeof(CkptHeader));
  if (memcmp(h->magic, kCkptMagic, 8) != 0 || h->version != 1) return false;
  if (h->n < 1 || h->n > INT32_MAX || h->nnz < 0 || h->nnz > ((int64_t)1 << 40) || h->K < 1 || h->K > 64 ||
      h->K > h->n || h->cfg.k != h->K || (h->has_val != 0 && h->has_val != 1) || h->step < 0)
    return false;
  *L = ckpt_layout(h->n, h->nnz, h->K, h->has_val != 0);
  if ((int64_t)L->total != bytes) return false;
  const int64_t* rp = reinterpret_cast<const int64_t*>(static_cast<const uint8_t*>(buf) + L->rowptr);
  if (rp[0] != 0 || rp[h->n] != h->nnz) return false;
  for (int64_t i = 0; i < h->n; ++i)
    if (rp[i + 1] < rp[i]) return false;
  return true;
}

}  // namespace

}  // extern "C"

namespace grest {
bool ckpt_view(const void* buf, int64_t bytes, CkptView* v) {
  CkptHeader h;
  CkptLayout L;
  if (!v || !ckpt_parse(buf, bytes, &h, &L)) return false;
  const uint8_t* b = static_cast<const uint8_t*>(buf);
  v->n = h.n;
  v->nnz = h.nnz;
  v->step = h.step;
  v->K = h.K;
  v->has_val = h.has_val != 0;
  v->cfg = h.cfg;
  v->rowptr = reinterpret_cast<const int64_t*>(b + L.rowptr);
  v->col = reinterpret_cast<const int32_t*>(b + L.col);
  v->val = v->has_val ? reinterpret_cast<const double*>(b + L.val) : nullptr;
  v->deg = reinterpret_cast<const double*>(b + L.deg);
  v->U = reinterpret_cast<const double*>(b + L.U);
  v->theta = reinterpret_cast<const double*>(b + L.theta);
  v->live = b + L.live;
  return true;
}
}  // namespace grest

extern "C" {

grest_status grest_checkpoint(grest_ctx* c, void* buf, int64_t* bytes) {
  if (!c || !bytes) return GREST_ERR_INVALID_ARG;
  if (cudaSetDevice(c->dev) != cudaSuccess) return GREST_ERR_CUDA;
  cudaStream_t s = c->stream;
  CK(cudaStreamSynchronize(s));
  const Csr& g = c->g;
  const int64_t n = g.n, nnz = c->nnz;
  const int K = c->K;
  const bool has_val = g.val != nullptr;
  const CkptLayout L = ckpt_layout(n, nnz, K, has_val);
  if (!buf) {
    *bytes = (int64_t)L.total;
    return GREST_OK;
  }
  if (*bytes < (int64_t)L.total) {
    *bytes = (int64_t)L.total;
    return GREST_ERR_CAPACITY;
  }
  int64_t top = 0;
  CK(cudaMemcpy(&top, g.arena_top, sizeof(int64_t), cudaMemcpyDeviceToHost));
  std::vector<int64_t> off(n);
  std::vector<int32_t> len(n), arena(top);
  std::vector<double> varena(has_val ? top : 0);
  CK(cudaMemcpyAsync(off.data(), g.row_off, sizeof(int64_t) * n, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(len.data(), g.row_len, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s));
  if (top > 0) CK(cudaMemcpyAsync(arena.data(), g.col, sizeof(int32_t) * top, cudaMemcpyDeviceToHost, s));
  if (has_val && top > 0) CK(cudaMemcpyAsync(varena.data(), g.val, sizeof(double) * top, cudaMemcpyDeviceToHost, s));
  uint8_t* b = static_cast<uint8_t*>(buf);
  memset(b, 0, L.total);  // padding bytes too: equal states give equal checkpoints
  CK(cudaMemcpyAsync(b + L.deg, g.deg, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpy2DAsync(b + L.U, sizeof(double) * K, c->U, sizeof(double) * c->ldu, sizeof(double) * K, n,
                       cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(b + L.theta, c->theta, sizeof(double) * K, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(b + L.live, g.live, n, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  int64_t* rp = reinterpret_cast<int64_t*>(b + L.rowptr);
  int32_t* col = reinterpret_cast<int32_t*>(b + L.col);
  double* val = reinterpret_cast<double*>(b + L.val);
  rp[0] = 0;
  for (int64_t i = 0; i < n; ++i) {
    if (len[i] < 0 || off[i] < 0 || off[i] + len[i] > top || rp[i] + len[i] > nnz) return GREST_ERR_CUDA;
    memcpy(col + rp[i], arena.data() + off[i], sizeof(int32_t) * len[i]);
    if (has_val) memcpy(val + rp[i], varena.data() + off[i], sizeof(double) * len[i]);
    rp[i + 1] = rp[i] + len[i];
  }
  if (rp[n] != nnz) return GREST_ERR_CUDA;
  CkptHeader h;
  memset(&h, 0, sizeof(h));
  memcpy(h.magic, kCkptMagic, 8);
  h.version = 1;
  h.K = K;
  h.n = n;
  h.nnz = nnz;
  h.step = c->step;
  h.has_val = has_val ? 1 : 0;
  h.cfg = c->cfg;
  memcpy(b, &h, sizeof(h));
  *bytes = (int64_t)L.total;
  return GREST_OK;
}

grest_status grest_checkpoint_embedding(const void* buf, int64_t bytes, double* U, double* theta, uint8_t* live,
                                        int64_t* n_out, int32_t* k_out) {
  CkptHeader h;
  CkptLayout L;
  if (!n_out || !ckpt_parse(buf, bytes, &h, &L)) return GREST_ERR_INVALID_ARG;
  const uint8_t* b = static_cast<const uint8_t*>(buf);
  *n_out = h.n;
  if (k_out) *k_out = h.K;
  if (U) memcpy(U, b + L.U, sizeof(double) * (size_t)h.n * h.K);
  if (theta) memcpy(theta, b + L.theta, sizeof(double) * h.K);
  if (live) memcpy(live, b + L.live, (size_t)h.n);
  return GREST_OK;
}

grest_status grest_restore(const void* buf, int64_t bytes, void* cuda_stream, grest_ctx** out) {
  if (!out) return GREST_ERR_INVALID_ARG;
  *out = nullptr;
  CkptHeader h;
  CkptLayout L;
  if (!ckpt_parse(buf, bytes, &h, &L)) return GREST_ERR_INVALID_ARG;
  const uint8_t* b = static_cast<const uint8_t*>(buf);
  const int64_t* rp = reinterpret_cast<const int64_t*>(b + L.rowptr);
  const int32_t* col = reinterpret_cast<const int32_t*>(b + L.col);
  const double* val = h.has_val ? reinterpret_cast<const double*>(b + L.val) : nullptr;
  const uint8_t* live = b + L.live;
  // the slack layout of grest_init must fit the saved capacities
  grest_config cfg = h.cfg;
  if (cfg.node_capacity > 0 && cfg.node_capacity < h.n) cfg.node_capacity = 0;
  if (cfg.nnz_capacity > 0) {
    int64_t need = 0;
    for (int64_t i = 0; i < h.n; ++i) {
      const int64_t l = rp[i + 1] - rp[i];
      need += l + l / 4 + 4;
    }
    if (cfg.nnz_capacity < need) cfg.nnz_capacity = 0;
  }
  grest_ctx* c = nullptr;
  grest_status st = grest_init(&cfg, h.n, rp, col, val, reinterpret_cast<const double*>(b + L.U),
                               reinterpret_cast<const double*>(b + L.theta), cuda_stream, &c);
  if (st != GREST_OK) return st;
  c->cfg = h.cfg;
  c->cfg.node_capacity = cfg.node_capacity;
  c->cfg.nnz_capacity = cfg.nnz_capacity;
  cudaStream_t s = c->stream;
  Csr& g = c->g;
  bool ok = cudaMemcpyAsync(g.deg, b + L.deg, sizeof(double) * h.n, cudaMemcpyHostToDevice, s) == cudaSuccess &&
            cudaMemcpyAsync(g.live, live, h.n, cudaMemcpyHostToDevice, s) == cudaSuccess;
  if (ok) {
    graph_refresh_derived(g, c->gw, h.n, s);
    zero_dead_rows(c->U, c->ldu, c->K, g.live, h.n, s);
    ok = cudaGetLastError() == cudaSuccess && cudaStreamSynchronize(s) == cudaSuccess;
  }
  if (!ok) {
    grest_destroy(c);
    return GREST_ERR_CUDA;
  }
  c->step = h.step;
  c->stats.step = h.step;
  *out = c;
  return GREST_OK;
}

grest_status grest_get_ritz_values(grest_ctx* c, double* ritz, int32_t* m_out) {
  if (!c || !m_out) return GREST_ERR_INVALID_ARG;
  *m_out = c->last_m;
  if (ritz) memcpy(ritz, c->last_ritz.data(), sizeof(double) * c->last_m);
  return GREST_OK;
}

grest_status grest_get_stats(grest_ctx* c, grest_stats* st) {
  if (!c || !st) return GREST_ERR_INVALID_ARG;
  *st = c->stats;
  return GREST_OK;
}

grest_status grest_apply_operator(grest_ctx* c, const double* X, int64_t ldx, double* Y, int64_t ldy, int32_t w) {
  if (!c || !X || !Y || w < 1 || w > 288 || ldx < w || ldy < w) return GREST_ERR_INVALID_ARG;
  if (cudaSetDevice(c->dev) != cudaSuccess) return GREST_ERR_CUDA;
  spmm(c, X, ldx, Y, ldy, w, 0, c->g.n, 0);
  CK(cudaGetLastError());
  return from_cuda(cudaStreamSynchronize(c->stream));
}

grest_status grest_centrality(grest_ctx* c, int32_t J, double* cent, int32_t* top_ids, double* top_vals,
                              int32_t on_device) {
  if (!c || J < 0 || J > central_max_j() || c->K > 64) return GREST_ERR_INVALID_ARG;
  if (cudaSetDevice(c->dev) != cudaSuccess) return GREST_ERR_CUDA;
  cudaStream_t s = c->stream;
  const int64_t n = c->g.n;
  const size_t need = central_work_bytes(c->g.n_cap);
  if (need > c->cent_work_cap) {
    cudaFree(c->cent_work);
    c->cent_work = nullptr;
    c->cent_work_cap = 0;
    CK(dmalloc((void**)&c->cent_work, need));
    c->cent_work_cap = need;
  }
  if (!c->cent_buf) CK(dalloc(&c->cent_buf, c->g.n_cap));
  if (!c->top_id_buf) CK(dalloc(&c->top_id_buf, central_max_j()));
  if (!c->top_val_buf) CK(dalloc(&c->top_val_buf, central_max_j()));
  double* cdev = (on_device && cent) ? cent : c->cent_buf;
  CK(cudaMemsetAsync(c->err, 0, sizeof(int32_t), s));
  central_values(c->U, c->ldu, c->K, c->theta, c->g.live, n, cdev, c->cent_work, c->h_scal, c->err, s);
  CK(cudaMemcpyAsync(c->h_err, c->err, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s));
  if (*c->h_err) return map_dev_err(*c->h_err);
  if ((int64_t)J > c->h_scal[0]) return GREST_ERR_INVALID_ARG;
  if (cent && !on_device) CK(cudaMemcpyAsync(cent, cdev, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
  if (J > 0 && (top_ids || top_vals)) {
    int32_t* ids = on_device && top_ids ? top_ids : c->top_id_buf;
    double* vals = on_device && top_vals ? top_vals : c->top_val_buf;
    central_top(n, J, ids, vals, c->cent_work, s);
    CK(cudaGetLastError());
    if (!on_device) {
      if (top_ids) CK(cudaMemcpyAsync(top_ids, ids, sizeof(int32_t) * J, cudaMemcpyDeviceToHost, s));
      if (top_vals) CK(cudaMemcpyAsync(top_vals, vals, sizeof(double) * J, cudaMemcpyDeviceToHost, s));
    }
  }
  return from_cuda(cudaStreamSynchronize(s));
}

grest_status grest_gram(grest_ctx* c, const double* X, int64_t ldx, int32_t a, const double* Y, int64_t ldy,
                        int32_t b, int64_t n, double* C, int64_t ldc) {
  if (!c || !X || !Y || !C || a < 1 || b < 1 || a > 256 || b > 256 || n < 0 || ldx < a || ldy < b || ldc < b)
    return GREST_ERR_INVALID_ARG;
  if (cudaSetDevice(c->dev) != cudaSuccess) return GREST_ERR_CUDA;
  if (gram_parts(n, a, b) * (int64_t)a * b > c->part_cap) return GREST_ERR_CAPACITY;
  gram_f64(X, ldx, a, Y, ldy, b, n, C, ldc, c->part, false, c->stream);
  CK(cudaGetLastError());
  return from_cuda(cudaStreamSynchronize(c->stream));
}

grest_status grest_gram_f32(grest_ctx* c, const float* X, int64_t ldx, int32_t a, const float* Y, int64_t ldy,
                            int32_t b, int64_t n, double* C, int64_t ldc) {
  if (!c || !X || !Y || !C || a < 1 || b < 1 || a > 256 || b > 256 || n < 0 || ldx < a || ldy < b || ldc < b)
    return GREST_ERR_INVALID_ARG;
  if (cudaSetDevice(c->dev) != cudaSuccess) return GREST_ERR_CUDA;
  CK(cudaMemsetAsync(c->err, 0, sizeof(int32_t), c->stream));
  const bool done = gram_f32_fast(X, ldx, a, Y, ldy, b, n, C, ldc, c->part, c->part_cap, c->err, c->stream) >= 0;
  if (!done) {
    if (gram_parts(n, a, b) * (int64_t)a * b > c->part_cap) return GREST_ERR_CAPACITY;
    gram_f32(X, ldx, a, Y, ldy, b, n, C, ldc, c->part, false, c->stream);
  }
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(c->h_err, c->err, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return *c->h_err ? map_dev_err(*c->h_err) : GREST_OK;
}

grest_status grest_gemm_f32(grest_ctx* c, int64_t n, int32_t a, int32_t cc, double alpha, const float* X, int64_t ldx,
                            const double* B, int64_t ldb, double beta, const float* Cin, int64_t ldc, float* Out,
                            int64_t ldo) {
  if (!c || !X || !B || !Out || a < 1 || cc < 1 || n < 0 || ldx < a || ldb < cc || ldo < cc ||
      (beta != 0.0 && (!Cin || ldc < cc)))
    return GREST_ERR_INVALID_ARG;
  if (n == 0) return GREST_OK;
  if (cudaSetDevice(c->dev) != cudaSuccess) return GREST_ERR_CUDA;
  CK(cudaMemsetAsync(c->err, 0, sizeof(int32_t), c->stream));
  if (gemm_f32_tc(n, a, cc, alpha, X, ldx, B, ldb, beta, beta != 0.0 ? Cin : nullptr, ldc, Out, ldo, c->gemm_img,
                  c->gemm_img_cap, c->err, c->stream) != 0)
    gemm_nn_f32(n, a, cc, alpha, X, ldx, B, ldb, beta, beta != 0.0 ? Cin : nullptr, ldc, Out, ldo, c->stream);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(c->h_err, c->err, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return *c->h_err ? map_dev_err(*c->h_err) : GREST_OK;
}

void grest_destroy(grest_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->dev);
  cudaStreamSynchronize(c->stream);
  if (c->cstream) cudaStreamSynchronize(c->cstream);
  free_ctx(c);
}

// ---------------------------------------------------------------- batches of contexts
struct grest_batch {
  std::vector<grest_ctx*> ctx;
  int threads = 1;
};

grest_status grest_batch_create(int32_t n_graphs, grest_ctx* const* ctxs, int32_t n_threads, grest_batch** out) {
  if (!out || !ctxs || n_graphs < 1 || n_threads < 1) return GREST_ERR_INVALID_ARG;
  *out = nullptr;
  std::vector<grest_ctx*> v(ctxs, ctxs + n_graphs);
  for (grest_ctx* c : v)
    if (!c) return GREST_ERR_INVALID_ARG;
  std::vector<grest_ctx*> sorted = v;
  std::sort(sorted.begin(), sorted.end());
  if (std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end()) return GREST_ERR_INVALID_ARG;
  grest_batch* b = new grest_batch;
  b->ctx = std::move(v);
  b->threads = std::min<int>(n_threads, n_graphs);
  *out = b;
  return GREST_OK;
}

grest_status grest_batch_apply_updates(grest_batch* b, const grest_update* updates, grest_status* status,
                                       grest_stats* stats) {
  if (!b || !updates) return GREST_ERR_INVALID_ARG;
  const int n = (int)b->ctx.size();
  std::vector<grest_status> st(n, GREST_OK);
  std::atomic<int> next{0};
  auto worker = [&]() {
    for (int i = next.fetch_add(1); i < n; i = next.fetch_add(1))
      st[i] = grest_apply_update(b->ctx[i], &updates[i], stats ? &stats[i] : nullptr);
  };
  std::vector<std::thread> pool;
  for (int t = 1; t < b->threads; ++t) pool.emplace_back(worker);
  worker();
  for (auto& t : pool) t.join();
  grest_status first = GREST_OK;
  for (int i = 0; i < n; ++i) {
    if (status) status[i] = st[i];
    if (first == GREST_OK && st[i] != GREST_OK) first = st[i];
  }
  return first;
}

void grest_batch_destroy(grest_batch* b) { delete b; }

}  // extern "C"
