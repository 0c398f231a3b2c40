// Internal declarations shared by the libgrest translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "../../include/grest.h"

namespace grest {

constexpr int kWarp = 32;

// Error word written by device-side validation; kernels that change state
// return early once it is non-zero, so a failed step leaves no trace.
enum DevErr : int32_t {
  DERR_NONE = 0,
  DERR_RANGE = 1,        // node id out of range
  DERR_SELF = 2,         // self loop
  DERR_DEAD = 3,         // edge touches a tombstoned or removed node
  DERR_DUP = 4,          // the same edge twice in a batch
  DERR_EXISTS = 5,       // inserted edge already present
  DERR_MISSING = 6,      // deleted edge absent
  DERR_NODE = 7,         // bad removed-node id (range, duplicate, dead)
  DERR_WEIGHT = 8,       // weight not positive and finite
  DERR_CAPACITY = 9,     // edge arena exhausted
  DERR_NUMERIC = 10,     // Cholesky breakdown / rank below K
  DERR_TIMEOUT = 11,     // a bounded device-side wait expired
  DERR_ARENA = 12,       // edge arena too small for this batch (the host grows it and retries)
};

__device__ __forceinline__ void set_err(int32_t* err, int32_t code) { atomicCAS(err, 0, code); }

// 1 / a in FP64 for the serial scalar chains of the small factorizations
// (pivots, reflector coefficients, tridiagonal LU, Jacobi rotations), where
// an IEEE division costs several hundred clocks of latency on this part's
// FP64 pipe: the hardware's reduced-precision reciprocal (rcp.approx.ftz.f64)
// refined by two Newton-Raphson steps x <- x + x (1 - a x), each of which
// squares the relative error, so the result is within a couple of units in
// the last place of 1 / a.  Zero, subnormal, huge (|a| >= 2^1022, whose
// reciprocal is subnormal), infinite and NaN inputs take the IEEE division
// instead (an integer test of the exponent field).
__device__ __forceinline__ double rcp_newton(double a) {
  const int ex = (__double2hiint(a) >> 20) & 0x7ff;
  if (ex < 2 || ex > 2044) return 1.0 / a;
  double x;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(x) : "d"(a));
  double e = fma(-a, x, 1.0);
  x = fma(x, e, x);
  e = fma(-a, x, 1.0);
  return fma(x, e, x);
}

// Largest dynamic shared memory a launch of `kernel` may request on the
// current device (opt-in limit minus the kernel's static shared memory), and
// raise the kernel's limit to `bytes` when that fits.  Returns false (and
// changes nothing) when it does not fit.
// The kernel attribute is process-wide and contexts may launch from several
// host threads at once, so it only ever grows (under one lock): a launch with
// fewer bytes stays valid whatever another thread reserves meanwhile.
std::mutex& smem_attr_mutex();
// Bytes already reserved for (kernel, device), read and written under
// smem_attr_mutex(); nullptr when the table is full (then every call asks the
// driver).
size_t* smem_reserved_slot(const void* kernel, int dev);

template <typename K>
inline bool reserve_dynamic_smem(K kernel, size_t bytes) {
  const void* k = reinterpret_cast<const void*>(kernel);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  std::lock_guard<std::mutex> lock(smem_attr_mutex());
  size_t* slot = smem_reserved_slot(k, dev);
  if (slot && bytes <= *slot) return true;  // reserved before: no driver call
  int optin = 0;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return false;
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, k) != cudaSuccess) return false;
  if (bytes + fa.sharedSizeBytes > (size_t)optin) return false;
  if (bytes > (size_t)fa.maxDynamicSharedSizeBytes &&
      cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (slot) {
    const size_t now = bytes > (size_t)fa.maxDynamicSharedSizeBytes ? bytes : (size_t)fa.maxDynamicSharedSizeBytes;
    if (now > *slot) *slot = now;
  }
  return true;
}

// ---------------------------------------------------------------- CSR state
// Slack CSR: row r occupies col[row_off[r] .. row_off[r] + row_len[r]) sorted
// by column, inside a slot of row_cap[r] entries.  Rows that outgrow their slot
// move to fresh space at the top of the arena (arena_top).
struct Csr {
  int64_t n = 0;          // node ids in use
  int64_t n_cap = 0;      // capacity of the per-node arrays
  int64_t nnz_cap = 0;    // arena entries
  int64_t* row_off = nullptr;
  int32_t* row_len = nullptr;
  int32_t* row_cap = nullptr;
  int32_t* col = nullptr;
  double* val = nullptr;  // nullptr for an unweighted graph
  uint8_t* live = nullptr;
  double* deg = nullptr;     // weighted degree
  double* dis = nullptr;     // d^-1/2 (0 for isolated or dead nodes)
  int64_t* arena_top = nullptr;  // device scalar
  double* dmax = nullptr;        // device scalar, max degree over live nodes
};

// Operator description for the SpMM epilogue (Sec. 4.2).
struct OpParams {
  int op;                  // GREST_OP_*
  const double* deg;       // degree (LAP)
  const double* dis;       // d^-1/2 (NLAP)
  const double* dmax;      // device scalar (LAP: alpha = 2 dmax)
  const uint8_t* live;
};

// ------------------------------------------------------------ small problems in one CTA (group_dense.cu)
// Pivoted Cholesky of G (c x c, upper triangle read, c <= 64) with the drop
// rule of pchol_inverse (reference |abs_ref_ptr[0]| when given, else
// abs_ref); T (c x c, ldt) = P R^-1 on the kept pivots, zero elsewhere;
// info[0..3] = rank, kept_min, dropped_max, 0.  Returns the number of
// kernels launched, -1 when the size is not taken.
int pchol_small_f64(const double* G, int ldg, int c, double tol, double abs_ref, const double* abs_ref_ptr, double* T,
                    int ldt, double* info, cudaStream_t s);
// Leading k eigenpairs (tracking order of op) of the symmetric m x m A
// (m <= 64) by cyclic Jacobi: theta (k), F (m x k, ldf), ritz (m, nullable),
// info[0] = the relative K / K+1 gap (nullable).  Returns launches, or -1.
int eig_small_f64(const double* A, int lda, int m, int k, int op, double* theta, double* F, int ldf, double* ritz,
                  double* info, cudaStream_t s);

// ------------------------------------------------------------ checkpoints
// A checkpoint written by grest_checkpoint, read in place (host pointers into
// the buffer): the compact CSR, the maintained degrees, the pairs and the
// configuration.  ckpt_view returns false for a buffer that is not one.
struct CkptView {
  int64_t n, nnz, step;
  int32_t K;
  bool has_val;
  grest_config cfg;
  const int64_t* rowptr;
  const int32_t* col;
  const double* val;
  const double* deg;
  const double* U;      // n x K row-major
  const double* theta;  // K
  const uint8_t* live;  // n
};
bool ckpt_view(const void* buf, int64_t bytes, CkptView* v);

// ------------------------------------------------------------ launchers
// scan.cu
size_t scan_temp_bytes(int64_t n);
// exclusive prefix sum of n int64 values; out may alias in; writes the total
// to out[n] (out must hold n+1 values).
// returns the number of kernels launched
int exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, void* temp, cudaStream_t s);

// graph.cu
struct BatchDev {
  int64_t S = 0, n_ins = 0, n_del = 0, n_dn = 0;
  const int32_t *ins_u = nullptr, *ins_v = nullptr, *del_u = nullptr, *del_v = nullptr, *dn = nullptr;
  const double* ins_w = nullptr;
};
struct GraphWork {
  int64_t ent_cap = 0;       // capacity of the entry arrays
  int64_t tmp_cap = 0;       // merged-row staging entries
  int32_t* cnt = nullptr;    // per row [n_cap+1]
  int64_t* seg = nullptr;    // segment offsets [n_cap+1]
  int32_t* cursor = nullptr; // [n_cap]
  uint8_t* delflag = nullptr;// [n_cap]
  int64_t* rowflag = nullptr;// [n_cap+1] scan scratch
  int32_t* touched = nullptr;// [n_cap]
  int64_t* tmp_off = nullptr;// [n_cap+1]
  int64_t* need = nullptr;   // [n_cap+1]
  int32_t* new_len = nullptr;// [n_cap]
  uint64_t* ekey = nullptr;  // [ent_cap] entry keys
  int32_t* erow = nullptr;   // [ent_cap]
  double* ew = nullptr;      // [ent_cap] weight (inserts)
  int32_t* eins = nullptr;   // [ent_cap] inserts before entry (prefix)
  double* edel = nullptr;    // [ent_cap] old weight of a deleted edge, by sorted position
  int32_t* tmp_col = nullptr;// [tmp_cap]
  double* tmp_val = nullptr; // [tmp_cap]
  int64_t* dn_pref = nullptr;// [max removed nodes + 1]
  int64_t dn_cap = 0;
  int32_t* long_rows = nullptr; // rows with len > kLongRow [n_cap]
  int64_t* scalars = nullptr;   // device scalars: [0] n_touched [1] n_long [2] total entries [3] tmp total [4] need total
  void* scan_tmp = nullptr;
};
constexpr int kLongRow = 512;
// Validate and apply a batch.  Returns after enqueueing; errors land in *err.
// These launchers return the number of kernels they enqueued.
int graph_apply_batch(Csr& g, GraphWork& w, const BatchDev& b, int32_t* err, cudaStream_t s);
int graph_refresh_derived(Csr& g, GraphWork& w, int64_t n_rows, cudaStream_t s);
// Y = (M_new - M_old) X for the batch just applied (ADJ or LAP; M_old padded
// with zero rows / columns for new nodes; no node removal): Y over all N2 rows.
// dmax_old: device copy of d_max before the update.  Returns launches.
int delta_apply(const Csr& g, const GraphWork& w, int op, const double* X, int64_t ldx, double* Y, int64_t ldy, int wd,
                int64_t N, int64_t N2, const double* dmax_old, cudaStream_t s);
int delta_apply(const Csr& g, const GraphWork& w, int op, const float* X, int64_t ldx, float* Y, int64_t ldy, int wd,
                int64_t N, int64_t N2, const double* dmax_old, cudaStream_t s);
// total row length over rows [0, n) into *out (device int64)
int graph_count_nnz(const Csr& g, int64_t n, int64_t* out, cudaStream_t s);
// Arena compaction, in two parts.  graph_compact_plan writes the compacted
// row offsets (slot of len + len/4 + 4 entries per row, rows in id order) to
// w.rowflag[0..n] (total at [n]).  graph_compact_copy copies rows [0, n) into
// new_col / new_val (at least that total) and rewrites row_off, row_cap and
// arena_top; the caller then replaces g.col / g.val.  Each returns launches.
int graph_compact_plan(const Csr& g, GraphWork& w, int64_t n, cudaStream_t s);
int graph_compact_copy(Csr& g, const GraphWork& w, int64_t n, int32_t* new_col, double* new_val, cudaStream_t s);

// spmm.cu
// Y[r0:r1) = (M X)[r0:r1) for rows r0..r1, w columns; when col_lo > 0 only
// neighbours with id >= col_lo contribute, X is indexed by (id - col_lo), and
// the diagonal term applies only to rows >= col_lo (the new-node block E).
void spmm_f64(const Csr& g, const OpParams& op, const int32_t* long_rows, const int64_t* n_long_dev,
              const double* X, int64_t ldx, double* Y, int64_t ldy, int w, int64_t r0, int64_t r1, int64_t col_lo,
              cudaStream_t s);
void spmm_f32(const Csr& g, const OpParams& op, const int32_t* long_rows, const int64_t* n_long_dev,
              const float* X, int64_t ldx, float* Y, int64_t ldy, int w, int64_t r0, int64_t r1, int64_t col_lo,
              cudaStream_t s);
// FP32 X, FP64 accumulation and output (the refinement pass of the mixed path)
void spmm_f32_f64(const Csr& g, const OpParams& op, const int32_t* long_rows, const int64_t* n_long_dev,
                  const float* X, int64_t ldx, double* Y, int64_t ldy, int w, int64_t r0, int64_t r1, int64_t col_lo,
                  cudaStream_t s);

// dense.cu
// C (a x b, row-major, ldc) = X^T Y over rows [0,n) with X (n x a, ldx), Y (n x b, ldy).
// part must hold parts(n,a,b) * a * b doubles.
int64_t gram_parts(int64_t n, int a, int b);
void gram_f64(const double* X, int64_t ldx, int a, const double* Y, int64_t ldy, int b, int64_t n,
              double* C, int64_t ldc, double* part, bool symmetric, cudaStream_t s);
// As gram_f64 (non-symmetric), with the row-chunk count capped so that the
// partials fit in part_cap doubles; returns -1 when even one chunk does not fit.
int gram_f64_capped(const double* X, int64_t ldx, int a, const double* Y, int64_t ldy, int b, int64_t n, double* C,
                    int64_t ldc, double* part, int64_t part_cap, cudaStream_t s);
// G = X^T X and H = X^T Y for n x k FP64 blocks X, Y (shared ld, k <= 64),
// computing only the upper triangles (H is taken as symmetric: X^T M X for a
// symmetric M) and writing both in full (k x k, ld k).  part must hold
// 2 k^2 doubles per row chunk (at most part_cap in all).  Returns the number
// of kernels launched, -1 when nothing fits.
int gram_pair_sym_f64(const double* X, const double* Y, int64_t ld, int k, int64_t n, double* G, double* H,
                      double* part, int64_t part_cap, cudaStream_t s);
// Out (n x c, ldo) = beta * Cin (n x c, ldc) + alpha * X (n x a, ldx) * B (a x c, row-major ldb).
void gemm_nn_f64(int64_t n, int a, int c, double alpha, const double* X, int64_t ldx, const double* B,
                 int64_t ldb, double beta, const double* Cin, int64_t ldc, double* Out, int64_t ldo,
                 cudaStream_t s);
// Pivoted Cholesky with drop tolerance on G (c x c, row-major, ldg; overwritten).
// Produces T (c x c row-major, ldt; columns >= rank zero) with V T orthonormal,
// rank and pivot statistics in info[0..3] (rank, kept_min, dropped_max, status).
// piv: device scratch of c ints.  f32: factor in FP32 arithmetic (storage
// stays FP64).  Returns the number of kernels launched.
int pchol_inverse(double* G, int64_t ldg, int c, double drop_tol, double abs_ref, const double* abs_ref_ptr,
                  double* T, int64_t ldt, int* piv, double* info, bool f32, cudaStream_t s);
void symmetrize(double* H, int64_t ld, int m, cudaStream_t s);
void fill_f64(double* p, double v, int64_t n, cudaStream_t s);
void copy_cols_f64(const double* src, int64_t lds, double* dst, int64_t ldd, int64_t n, int w, cudaStream_t s);
void zero_dead_rows(double* X, int64_t ldx, int w, const uint8_t* live, int64_t n, cudaStream_t s);
void zero_dead_rows(float* X, int64_t ldx, int w, const uint8_t* live, int64_t n, cudaStream_t s);
void sign_normalize(double* X, int64_t ldx, int w, int64_t n, double* part, int64_t* ipart, cudaStream_t s);
void sign_normalize(float* X, int64_t ldx, int w, int64_t n, double* part, int64_t* ipart, cudaStream_t s);
// mixed precision: FP32 blocks, FP64 small matrices
void gram_f32(const float* X, int64_t ldx, int a, const float* Y, int64_t ldy, int b, int64_t n, double* C,
              int64_t ldc, double* part, bool symmetric, cudaStream_t s);
void gemm_nn_f32(int64_t n, int a, int c, double alpha, const float* X, int64_t ldx, const double* B, int64_t ldb,
                 double beta, const float* Cin, int64_t ldc, float* Out, int64_t ldo, cudaStream_t s);
// sum of per-chunk partials into C: part[chunk][a][b], or part[chunk][b][a] when transposed
void gram_reduce_launch(const double* part, int64_t chunks, int a, int b, double* C, int64_t ldc, cudaStream_t s,
                        bool transposed = false);

// tc_gram.cu: tensor-core (tcgen05, 3xTF32) Gram C = X^T Y of FP32 blocks, FP64 output.
bool gram_tc_supported(const float* X, int64_t ldx, int a, const float* Y, int64_t ldy, int b);
// CUDA-core FP32 Gram for a narrow side (min(a, b) <= 64, max(a, b) <= 256,
// 16-byte aligned blocks); returns -1 when the shape or alignment is not taken
bool gram_narrow_supported(const float* X, int64_t ldx, int a, const float* Y, int64_t ldy, int b);
int gram_f32_narrow(const float* X, int64_t ldx, int a, const float* Y, int64_t ldy, int b, int64_t n, double* C,
                    int64_t ldc, double* part, int64_t part_cap, int32_t* err, cudaStream_t s);
// returns 0 when launched, -1 when the shapes or the partial buffer do not allow it
int gram_f32_tc(const float* X, int64_t ldx, int a, const float* Y, int64_t ldy, int b, int64_t n, double* C,
                int64_t ldc, double* part, int64_t part_cap, int32_t* err, cudaStream_t s);
void convert_f32_to_f64(const float* src, int64_t lds, double* dst, int64_t ldd, int64_t n, int w, cudaStream_t s);
void convert_f64_to_f32(const double* src, int64_t lds, float* dst, int64_t ldd, int64_t n, int w, cudaStream_t s);
void residual_norms(const double* MX, const double* X, int64_t ld, int w, const double* theta, int64_t n,
                    double* part, double* out, cudaStream_t s);

// tc_gemm.cu: tensor-core (3xTF32) Out = beta Cin + alpha X B, X n x a FP32
// row-major, B a x c FP64 row-major (c <= 256).  img: device scratch of at
// least gemm_tc_img_bytes(a, c) bytes.  Returns 0 when enqueued (two kernels),
// -1 when the shape or alignment is not supported (nothing enqueued).
size_t gemm_tc_img_bytes(int a, int c);
int gemm_f32_tc(int64_t n, int a, int c, double alpha, const float* X, int64_t ldx, const double* B, int64_t ldb,
                double beta, const float* Cin, int64_t ldc, float* Out, int64_t ldo, uint8_t* img, size_t img_cap,
                int32_t* err, cudaStream_t s);

// refine.cu: double-float (FP32 hi + lo) products of the mixed refinement.
// spmm_df: (Yh + Yl) = M X for FP32 X (n x w, w <= 64), all rows.
// gram_df: C (k x k) = X^T (Yh + Yl) (Yl may be null), k <= 64.
// lift_df: Out (FP64) = X S, S k x k FP64 row-major (ld k).
// sign_normalize_fast: FP64 X, columns flipped so that the entry of largest
// magnitude (lowest row on ties) is positive.  Each returns its launch count.
int spmm_df(const Csr& g, const OpParams& op, const int32_t* long_rows, const int64_t* n_long_dev, const float* X,
            int64_t ldx, float* Yh, float* Yl, int64_t ldy, int w, int64_t n, cudaStream_t s);
int gram_df(const float* X, int64_t ldx, const float* Yh, const float* Yl, int64_t ldy, int k, int64_t n, double* C,
            int64_t ldc, double* part, int64_t part_cap, cudaStream_t s);
int lift_df(const float* X, int64_t ldx, const double* S, int k, int64_t n, double* Out, int64_t ldo, cudaStream_t s);
int sign_normalize_fast(double* X, int64_t ldx, int w, int64_t n, double* part, int64_t* ipart, cudaStream_t s);

// central.cu (Sec. 5 downstream task): c = exp(-theta_max) X_K exp(Lambda_K) X_K^T 1
// over the live rows (0 for removed nodes) into cent[n]; the live count goes
// to *n_live_host (pinned) once the stream reaches it.  central_top then
// writes the J most central ids / values (c descending, id ascending) from
// the keys central_values left in `work`.  Each returns its launch count.
int central_max_j();
size_t central_work_bytes(int64_t n);
int central_values(const double* X, int64_t ldx, int K, const double* theta, const uint8_t* live, int64_t n,
                   double* cent, void* work, int64_t* n_live_host, int32_t* err, cudaStream_t s);
int central_top(int64_t n, int J, int32_t* top_ids, double* top_vals, void* work, cudaStream_t s);

// eig.cu
// Symmetric eigensolver for H (m x m row-major, ld; overwritten).  Writes the
// k leading pairs in tracking order: theta[k], F (m x k row-major, ldf), all m
// eigenvalues in tracking order to ritz[m], boundary gap to info[0].  f32:
// solve in FP32 arithmetic (storage stays FP64).  Returns the number of
// kernels launched.
int sym_eig_select(double* H, int64_t ld, int m, int k, int op_order, double* theta, double* F, int64_t ldf,
                   double* ritz, double* info, double* work, bool f32, cudaStream_t s);
size_t eig_work_doubles(int mmax);

// rsvd.cu
// Omega (S x q, row-major ld) from Philox4x64-10 + Box-Muller at step t.
void gaussian_omega(double* Om, int64_t ld, int64_t S, int q, uint64_t seed, uint64_t step, cudaStream_t s);
void gaussian_omega(float* Om, int64_t ld, int64_t S, int q, uint64_t seed, uint64_t step, cudaStream_t s);

}  // namespace grest
