/*
 * grest.h -- C ABI of libgrest: GPU tracking of the leading eigenpairs of an
 * evolving graph with the G-REST update (Graph Rayleigh-Ritz Eigenspace
 * Tracking) of "Subspace Projection Methods for Fast Spectral Embeddings of
 * Evolving Graphs" (arXiv 2603.19439).
 *
 * The calls follow the paper's Problem 1 (Sec. 2.1): given the K leading
 * eigenpairs {(lambda_j, x_j)} of an N x N matrix and an (N+S) x (N+S)
 * perturbation Delta (Eq. adj_update, Sec. 2), estimate the K leading
 * eigenpairs of the updated matrix.  Alg. 2 applies that update once per
 * received Delta: grest_init takes Alg. 2's input and initial pairs,
 * grest_apply_update is one pass of the loop (receive Delta, pad X, build an
 * orthonormal basis Z, solve the projected eigenproblem, lift X = Z F_K), and
 * grest_get_embedding returns (X_K, Lambda_K).
 *
 * Conventions common to every call:
 *  - Status codes only; no C++ exception crosses this boundary.
 *  - Node ids are 0-based.  The S new nodes of an update take the ids
 *    N .. N+S-1, N being the number of ids before the update (Sec. 2).
 *  - Dense N x K blocks are row-major (row i holds node i's K coordinates).
 *  - Every input array is owned by the caller and is only read during the
 *    call (its contents are copied); the context owns all device memory it
 *    allocates; output arrays are allocated by the caller.
 *  - A context is bound to the CUDA device that was current in grest_init
 *    and to one CUDA stream; it must not be used by two threads at once.
 *  - All computation runs in CUDA kernels of this library on that device.
 *    There is no CPU fallback: without a usable GPU every call returns
 *    GREST_ERR_CUDA.
 */
#ifndef GREST_H
#define GREST_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct grest_ctx grest_ctx; /* opaque; owns every device buffer */

typedef enum {
  GREST_OK = 0,
  GREST_ERR_INVALID_ARG = 1,     /* bad pointer, size or configuration field */
  GREST_ERR_INVALID_UPDATE = 2,  /* batch violates Sec. 2's definition of Delta */
  GREST_ERR_OOM = 3,             /* device allocation failed */
  GREST_ERR_CAPACITY = 4,        /* a fixed limit exceeded (2^31 - 1 node ids, a caller buffer) */
  GREST_ERR_NUMERIC = 5,         /* fewer than K Ritz pairs, or a Cholesky broke down */
  GREST_ERR_CUDA = 6,            /* CUDA runtime error (no device, launch failure) */
  GREST_ERR_TIMEOUT = 7,         /* a bounded device-side wait expired */
  GREST_ERR_UNSUPPORTED = 8      /* option or combination not implemented   */
} grest_status;

/* Operator whose leading eigenpairs are tracked (Sec. 2 and Sec. 4.2). */
enum {
  GREST_OP_ADJ = 0,  /* adjacency A; pairs ordered by |lambda| descending (Sec. 2) */
  GREST_OP_LAP = 1,  /* T = alpha I - (D - A), alpha = 2 d_max of the current graph */
  GREST_OP_NLAP = 2  /* T_n = 2I - L_n = I + D^-1/2 A D^-1/2 (isolated node: identity row) */
};

/* Projection subspace (Table 1 and Sec. 5): */
enum {
  GREST_SUB_GREST2 = 0, /* Ran[X_bar, P_perp W]            (residual-mode subspace)  */
  GREST_SUB_GREST3 = 1, /* Ran[X_bar, P_perp [W, Delta_2]]  exact new-node block      */
  GREST_SUB_RSVD = 2,   /* as GREST3 with Delta_2 replaced by its RSVD basis (Sec. 3.5) */
  GREST_SUB_AUTO = 3    /* GREST3 when S <= L+P, RSVD otherwise (default)              */
};

/* Arithmetic of the step.
 * GREST_FP64: every block and product in FP64.
 * GREST_MIXED: N x w blocks stored in FP32; SpMM in FP32; the Grams and
 *   block updates on the tensor cores (3xTF32, FP32 accumulation, FP64
 *   partial sums); the pivoted Cholesky, the m x m and RSVD eigensolves in
 *   FP64; then one Rayleigh-Ritz refinement in span(U) with FP64 products
 *   (M U, U^T U, U^T M U and the lift), so the result is orthonormal and
 *   Galerkin-consistent to FP64 accuracy.
 * GREST_MIXED_FAST: as GREST_MIXED, but the projected problems are solved in
 *   FP32 arithmetic (their entries come from FP32 blocks) and the
 *   refinement's N x K products run in double-float arithmetic (FP32 hi + lo
 *   pairs, about 48 significant bits) on the FP32 pipes. */
enum { GREST_FP64 = 0, GREST_MIXED = 1, GREST_MIXED_FAST = 2 };
/* Projected operator: EXACT forms H = Z^T M_new Z (Eq. main2); LOWRANK forms
 * the paper's surrogate H = (X_bar^T Z)^T Lambda (X_bar^T Z) + Z^T Delta Z
 * (Eq. main3, Alg. 2 as printed), where Delta = M_new - M_old (M_old padded
 * with zero rows and columns for new nodes) and Lambda the previous Ritz
 * values; it needs no product with the whole graph.
 * W block: RESID uses P_perp (M_new X_bar); DELTA the paper's P_perp (Delta X_bar)
 * (Sec. 3.3).  LOWRANK and DELTA are available for GREST_OP_ADJ and
 * GREST_OP_LAP, for batches without node removal (GREST_ERR_UNSUPPORTED
 * otherwise); LOWRANK runs in GREST_FP64 only. */
enum { GREST_PROJ_EXACT = 0, GREST_PROJ_LOWRANK = 1 };
enum { GREST_WB_RESID = 0, GREST_WB_DELTA = 1 };

/* grest_config.flags */
#define GREST_FLAG_CHECK 1u   /* after each step compute residual diagnostics into grest_stats */
#define GREST_FLAG_PROFILE 2u /* time every kernel class with CUDA events (grest_stats.prof_*) */
/* GREST_FLAG_TWO_STREAMS: a context whose graph has at least 131,072 nodes
 * at grest_init (and whose subspace setting allows the RSVD new-node block)
 * also creates a second, high-priority CUDA stream of its own, with its own
 * Gram and GEMM scratch (about 70 MB).  In a step with an RSVD block, the
 * sketch of Sec. 3.5 (S.1, its CholQR2 and the first products of S.2) then
 * runs there beside the projection of the previous pairs (Alg. 2,
 * Y1 = M X_bar and W), and the caller's stream waits for it before S.2
 * continues, so the step's work is still complete when the caller's stream
 * is.  The results are the same bits either way.  Off by default: the gain
 * is about 2% of a step at n = 1M, and the kernels of the two streams slow
 * each other, so GREST_FLAG_PROFILE's per-class times no longer describe
 * the kernels alone. */
#define GREST_FLAG_TWO_STREAMS 4u

typedef struct {
  int32_t op;          /* GREST_OP_*                                                   */
  int32_t k;           /* K, number of tracked pairs, 1 <= k <= 64                      */
  int32_t subspace;    /* GREST_SUB_*                                                  */
  int32_t L, P;        /* RSVD rank and oversampling (Sec. 3.5); L+P <= 256             */
  int32_t precision;   /* GREST_FP64 | GREST_MIXED | GREST_MIXED_FAST                   */
  int32_t projection;  /* GREST_PROJ_*                                                 */
  int32_t w_block;     /* GREST_WB_*                                                   */
  uint32_t flags;      /* GREST_FLAG_*                                                 */
  uint64_t seed;       /* key of the counter-based generator that draws Omega          */
  double drop_tol;     /* a basis direction is dropped when its pivot R_kk is at most   *
                        * drop_tol * max(R_00, |theta_1|) (|theta_1| ~ ||M||_2)         */
  int64_t node_capacity;   /* initial node-id capacity; 0 = 1.25 x initial + 1024;     *
                            * grows by 1.5x when a batch needs more (see below)         */
  int64_t nnz_capacity;    /* initial directed-edge arena; 0 = 2 x initial + 2^20;     *
                            * compacted into a larger arena when a batch needs more    */
  int64_t max_batch_edges; /* largest n_ins + n_del per update; 0 = 2^20 (grows on demand) */
} grest_config;

/*
 * One update Delta (Eq. adj_update, Sec. 2).
 *  ins_u/ins_v (n_ins): edges to add.  An edge between two old nodes is a +1
 *      entry of K and must not exist yet; an edge touching a new node is an
 *      entry of G or C.  Each undirected edge is listed once, u != v.
 *  ins_w: weights of the inserted edges for a weighted context (positive,
 *      finite); NULL means 1.  Must be NULL for an unweighted context.
 *  del_u/del_v (n_del): existing edges among old nodes to remove (-1 entries of K).
 *  del_nodes (n_del_nodes): old live nodes to remove.  The paper leaves node
 *      removal to future work (Sec. 6); this library reads it as: every
 *      incident edge is removed, the id is tombstoned (never reused), the
 *      operator becomes the principal submatrix on live nodes, and the
 *      tombstoned rows of X are zeroed before X is re-orthonormalized.
 *      No edge of the same batch may touch a removed node.
 *  on_device: 0 = the arrays are host memory, 1 = device memory of the
 *      context's device.
 * The whole batch is validated before any state changes; on any error the
 * context is left exactly as it was (GREST_ERR_INVALID_UPDATE).
 */
typedef struct {
  int64_t n_new_nodes;
  int64_t n_ins;
  const int32_t *ins_u, *ins_v;
  const double *ins_w;
  int64_t n_del;
  const int32_t *del_u, *del_v;
  int64_t n_del_nodes;
  const int32_t *del_nodes;
  int32_t on_device;
} grest_update;

/* Kernel kinds of GREST_FLAG_PROFILE (grest_stats.prof_kind_*): each timed
 * launch group of a step is one of these. */
enum {
  GREST_KIND_SPMM_F32 = 0,     /* k_spmm_rows / k_spmm_long on FP32 blocks (mixed path)        */
  GREST_KIND_SPMM_F64 = 1,     /* the same on FP64 blocks (FP64 path, mixed refinement)         */
  GREST_KIND_GRAM_TC = 2,      /* k_gram_tc (+ its reduce): tcgen05 3xTF32 Gram                  */
  GREST_KIND_GRAM_NARROW = 3,  /* k_gram_narrow (+ reduce): FP32 Gram with a side <= 32         */
  GREST_KIND_GRAM_CUDA = 4,    /* CUDA-core Grams: FP64 split-K, the refinement's pair Gram   */
  GREST_KIND_GEMM_TC = 5,      /* k_gemm_tc (+ k_gemm_prep): tcgen05 3xTF32 block update        */
  GREST_KIND_GEMM_CUDA = 6,    /* CUDA-core block updates (FP64, FP32 fallback)                 */
  GREST_KIND_DOUBLE_FLOAT = 7, /* GREST_MIXED_FAST refinement kernels (double-float)           */
  GREST_KIND_SMALL = 8,        /* small dense: pivoted Cholesky, eigensolver (several kernels) */
  GREST_KIND_GRAPH = 9,        /* graph update (several kernels)                              */
  GREST_KIND_COUNT = 10
};

/* Per-step diagnostics (filled by grest_apply_update / grest_get_stats). */
typedef struct {
  int64_t step;            /* updates applied so far                                   */
  int64_t n_nodes;         /* node ids after the step (live + tombstoned)               */
  int64_t nnz;             /* directed nonzeros of the adjacency after the step        */
  int32_t m;               /* dimension of Z                                           */
  int32_t k_u;             /* columns of X_bar kept (< k only after node removal)      */
  int32_t rank_q;          /* columns added to X_bar (W and new-node block, after drop) */
  int32_t rank_y;          /* rank of the RSVD sketch Y (0 when not used)              */
  int32_t mode;            /* 2 = GREST2, 3 = GREST3, 4 = RSVD                          */
  int32_t pad0;
  double pivot_kept_min;   /* smallest kept pivot / largest pivot                      */
  double pivot_dropped_max;/* largest dropped pivot / largest pivot (0 if none)        */
  double boundary_gap;     /* |theta_K - theta_{K+1}| / |theta_1| in the ordering      */
  double orth_err;         /* max |X^T X - I|           (GREST_FLAG_CHECK)             */
  double max_residual;     /* max_j ||M x_j - theta_j x_j|| / |theta_1| (CHECK)         */
  double galerkin;         /* max |Z^T (M x_j - theta_j x_j)| / |theta_1| (CHECK)       */
  float ms_total, ms_graph, ms_spmm, ms_basis, ms_project, ms_eig, ms_lift, ms_refine;
  /* GREST_FLAG_PROFILE: summed device time and algorithmic work per kernel class
   * (index 0 SpMM, 1 Gram X^T Y, 2 tall-skinny GEMM X B, 3 small dense: Cholesky,
   * eigensolver; 4 graph update).  Work is flops: 2 per nonzero and column
   * for SpMM, the products' flops for the dense classes. */
  double prof_ms[5];
  double prof_work[5];
  int64_t prof_launches[5];
  int64_t kernel_launches; /* kernels this library enqueued during the step       */
  /* GREST_FLAG_PROFILE: compulsory HBM bytes per class (each operand block read
   * once, each output written once; SpMM: row pointers, column indices,
   * one read of X and one write of Y). */
  double prof_bytes[5];
  /* GREST_FLAG_PROFILE: the same figures per kernel kind (GREST_KIND_*), so
   * that the classes that mix kernels (the Gram class holds the tensor-core,
   * the narrow and the CUDA-core Grams) can be told apart. */
  double prof_kind_ms[GREST_KIND_COUNT];
  double prof_kind_work[GREST_KIND_COUNT];
  double prof_kind_bytes[GREST_KIND_COUNT];
  int64_t prof_kind_launches[GREST_KIND_COUNT];
} grest_stats;

/* Fill *cfg with defaults for k tracked pairs: ADJ, AUTO, L = P = 100
 * (the paper's setting, Sec. 5), FP64, EXACT, RESID, drop_tol 1e-7. */
grest_status grest_config_default(grest_config *cfg, int32_t k);

/*
 * Create a context (Alg. 2 input).  The graph is given as a symmetric CSR on
 * the host: rowptr[n+1] (int64), col[rowptr[n]] (int32, no self loops, each
 * undirected edge present in both rows), val (nullable; positive weights,
 * symmetric).  U0 (n x k row-major, orthonormal columns) and theta0 (k) are
 * Alg. 2's initial leading pairs from any eigensolver.  When both are NULL
 * the library computes them on the device in FP64: block Krylov rounds
 * (blocks of k + max(8, k/2) columns, full reorthogonalization,
 * Rayleigh-Ritz) until the block is close, then Chebyshev-filtered subspace
 * iteration with the converged pairs locked (Zhou and Saad's scaled
 * recurrence), until every tracked residual ||M x - theta x|| is at most
 * 1e-11 |theta_1| (GREST_ERR_NUMERIC if 100 rounds do not get there);
 * graphs of at most 288 nodes are solved densely.  Device memory for this
 * is taken and released inside grest_init (about n * 600 doubles).  One NULL
 * and one not -> GREST_ERR_INVALID_ARG.
 * cuda_stream is a cudaStream_t (NULL = the legacy default stream).
 * Errors: GREST_ERR_INVALID_ARG (null pointers, sizes, configuration fields,
 * a malformed CSR: decreasing row pointers, out-of-range or duplicate
 * columns, self loops, non-positive weights), GREST_ERR_UNSUPPORTED (mode
 * combinations listed with GREST_PROJ_* above), GREST_ERR_OOM, GREST_ERR_CUDA;
 * *out is NULL on any error.
 */
grest_status grest_init(const grest_config *cfg, int64_t n, const int64_t *rowptr,
                        const int32_t *col, const double *val, const double *U0,
                        const double *theta0, void *cuda_stream, grest_ctx **out);

/*
 * Apply one update (one iteration of Alg. 2's loop): validate and apply
 * Delta to the device CSR, pad X, build Z = [X_bar, Q] with
 * Q = orth(P_perp [W, B]) (Sec. 3.3-3.5), form H = Z^T M Z (Eq. main2) or the
 * rank-K surrogate (Eq. main3), solve H F = F Theta, set X = Z F_K,
 * Lambda = Theta_K.  Returns when the step has finished on the device.
 * stats may be NULL.
 * Errors: GREST_ERR_INVALID_ARG (null context or update, negative counts,
 * null arrays for nonzero counts, weights for an unweighted context);
 * GREST_ERR_INVALID_UPDATE (the batch breaks Sec. 2's definition of Delta:
 * an existing edge inserted, a missing edge deleted, a duplicate, a self
 * loop, an id out of range or removed) with the context unchanged;
 * GREST_ERR_CAPACITY (more than 2^31 - 1 node ids) with the context
 * unchanged; GREST_ERR_UNSUPPORTED (node removal in the DELTA / LOWRANK
 * modes; an exact new-node block wider than L + P); GREST_ERR_NUMERIC: the
 * graph is updated, and either the basis had fewer than k directions (the
 * tracked pairs are then the previous ones, padded with zero rows for the
 * new nodes) or the second CholQR pass lost rank (the pairs are updated from
 * the smaller basis); GREST_ERR_TIMEOUT (a bounded device-side wait gave
 * up); GREST_ERR_OOM, GREST_ERR_CUDA.
 * Growth: Alg. 2 appends S ids per step, so the context grows instead of
 * failing.  A batch whose N + S exceeds the node capacity first moves every
 * per-node array (the CSR row arrays, X and the N x w blocks) to
 * max(N + S, 1.5 x capacity) ids; a batch whose merged rows do not fit the
 * edge arena is applied again after the arena is compacted into one of
 * max(1.5 x size, 2 x compacted + the batch's need + 2^20) entries.  Both
 * allocate before they release, so an allocation failure returns
 * GREST_ERR_OOM with the context unchanged; both make the call synchronize
 * the device (cudaFree).  Results do not depend on the capacities.
 */
grest_status grest_apply_update(grest_ctx *ctx, const grest_update *upd, grest_stats *stats);

/* Wait for all work of the context's stream. */
grest_status grest_sync(grest_ctx *ctx);

/*
 * Copy out (X_K, Lambda_K).  n_out (required) receives the number of node
 * ids.  U (nullable) receives n_out x k row-major values (tombstoned rows are
 * zero), theta (nullable) k values in tracking order, live_mask (nullable)
 * n_out bytes (1 = live).  Columns are sign-normalized: the entry of largest
 * magnitude (lowest index on ties) is positive.  on_device selects host (0)
 * or device (1) destination pointers.  Call with all outputs NULL to query n.
 */
grest_status grest_get_embedding(grest_ctx *ctx, double *U, double *theta, uint8_t *live_mask,
                                 int64_t *n_out, int32_t on_device);

/*
 * The same read of (X_K, Lambda_K) as grest_get_embedding (U and theta; no
 * live mask), started without waiting, so that the copy to the host overlaps
 * the next grest_apply_update (the pairs are the step's result, Alg. 2; the
 * paper has no counterpart for the transfer).  The copies run on a copy
 * stream of the context after the work enqueued so far on its stream; U
 * (n_out x k, row-major) and theta (k) are caller-owned host or device
 * memory.  Pinned host memory mapped into the device's address space
 * (cudaHostAlloc, or cudaHostRegister with cudaHostRegisterMapped) is
 * written by a kernel over the host link, leaving the copy engines to the
 * next update's own small reads; other memory is copied with
 * cudaMemcpyAsync (pageable host memory makes that copy wait on the host).  n_out (required) receives the number
 * of node ids now.  The outputs are complete after grest_wait_embedding (or
 * grest_destroy); until then the caller must not read or reuse them.  The
 * next update keeps the pairs being copied until the copy is done: its lift
 * (the first write to them) waits for the copy on the device, and a
 * capacity growth or grest_set_embedding waits on the host.  Several reads
 * may be outstanding; they complete in order.
 */
grest_status grest_get_embedding_async(grest_ctx *ctx, double *U, double *theta, int64_t *n_out);

/* Wait (host) until every read started by grest_get_embedding_async is complete. */
grest_status grest_wait_embedding(grest_ctx *ctx);

/*
 * Replace (X_K, Lambda_K) for the current graph, e.g. to resume from a saved
 * embedding or to start from pairs computed after grest_init.  U: n x k
 * row-major with orthonormal columns (rows of tombstoned ids are ignored and
 * stored as zero), theta: k values in tracking order; host (on_device = 0) or
 * device (1) pointers of the context's device.
 */
grest_status grest_set_embedding(grest_ctx *ctx, const double *U, const double *theta, int32_t on_device);

/*
 * Checkpoint and restore of a context (the tracked state of Alg. 2 between
 * two updates: the graph G^(t), (X_K, Lambda_K) and the step counter).
 *
 * grest_checkpoint writes the context's state into the caller's host buffer
 * buf of *bytes bytes.  buf == NULL: *bytes receives the size needed and
 * nothing is written.  A buffer smaller than that size: GREST_ERR_CAPACITY
 * with the size needed in *bytes.  On success *bytes is the size written.
 * The call waits for the context's stream; the context is not modified.
 * The buffer holds: a header (format tag, version, the grest_config, node
 * and nonzero counts, the step counter), the graph as a compact CSR (int64
 * row pointers, int32 columns sorted within each row, FP64 weights when the
 * graph is weighted), the FP64 weighted degrees, U (n x k row-major), theta
 * (k) and the live mask (n bytes).  It is a plain byte array (host byte
 * order) that the caller may store and reload.
 *
 * grest_restore builds a new context from such a buffer (read only; the
 * caller keeps ownership), with its work on cuda_stream.  Its next updates
 * give bit-identical results to those of the checkpointed context: the
 * neighbour order of every row, the degrees, the pairs and the step counter
 * (which seeds the RSVD test matrix of Sec. 3.5) are restored.  Slack
 * capacities are laid out afresh (node_capacity / nnz_capacity of the saved
 * configuration are kept when the restored graph fits them, else the
 * defaults are used).  A buffer that is not a checkpoint of this format
 * (tag, version, sizes, row pointers): GREST_ERR_INVALID_ARG before any
 * device work; grest_init's errors otherwise.
 *
 * grest_checkpoint_embedding reads (X_K, Lambda_K) and the live mask out of a
 * checkpoint buffer on the host (no device needed), with the conventions of
 * grest_get_embedding: n_out (required) receives n, k_out (nullable) k;
 * U (n x k), theta (k) and live (n) are nullable host outputs.
 */
grest_status grest_checkpoint(grest_ctx *ctx, void *buf, int64_t *bytes);
grest_status grest_restore(const void *buf, int64_t bytes, void *cuda_stream, grest_ctx **out);
grest_status grest_checkpoint_embedding(const void *buf, int64_t bytes, double *U, double *theta,
                                        uint8_t *live, int64_t *n_out, int32_t *k_out);

/* All m Ritz values of the last step in tracking order (Alg. 1); *m_out receives m.
 * ritz may be NULL to query m; it must hold at least m values otherwise. */
grest_status grest_get_ritz_values(grest_ctx *ctx, double *ritz, int32_t *m_out);

/* Diagnostics of the last completed step. */
grest_status grest_get_stats(grest_ctx *ctx, grest_stats *stats);

/*
 * Sec. 5 downstream task: subgraph centrality approximated from the tracked
 * pairs, exp(M) 1 ~= X_K exp(Lambda_K) X_K^T 1, returned scaled by
 * exp(-theta_max) (theta_max the largest tracked value) so that it cannot
 * overflow; the scaling leaves the ranking unchanged.  For the adjacency
 * operator this is the paper's measure; for LAP / NLAP it is the same formula
 * on the tracked (shifted) operator.
 *   cent:     n_nodes values (NULL: not returned); removed nodes get 0.
 *   top_ids:  the J most central live node ids (NULL: not returned), ordered by
 *             value descending, equal values by id ascending (a unique order).
 *   top_vals: their values (NULL: not returned).
 * 0 <= J <= min(4096, live nodes), K <= 64, else GREST_ERR_INVALID_ARG.
 * on_device: 1 = the output pointers are device memory, 0 = host memory.
 * GREST_ERR_NUMERIC if a value is NaN.  Synchronous; the caller owns every
 * buffer; the tracked state is not modified.
 */
grest_status grest_centrality(grest_ctx *ctx, int32_t J, double *cent, int32_t *top_ids,
                              double *top_vals, int32_t on_device);

/*
 * Y = M X for the context's current operator M (Sec. 4.2 kinds, principal
 * submatrix on live nodes).  X and Y are device arrays of n_nodes rows,
 * row-major with leading dimensions ldx, ldy (>= w), w <= 288 columns.  This
 * is the library's CSR SpMM, exposed for residual checks and measurement.
 */
grest_status grest_apply_operator(grest_ctx *ctx, const double *X, int64_t ldx, double *Y,
                                  int64_t ldy, int32_t w);

/*
 * C = X^T Y for device blocks X (n x a, row-major, leading dimension ldx) and
 * Y (n x b, ldy), a, b <= 256, written to the device array C (a x b,
 * row-major, ldc).  This is the split-K Gram kernel of the projection steps
 * (X_bar^T Y1, Gram matrices of CholQR2, H = Z^T (M Z) of Alg. 1); it runs on
 * the context's stream and uses the context's scratch, so calls on one
 * context must not overlap.  Useful for checks such as X^T X - I.
 */
grest_status grest_gram(grest_ctx *ctx, const double *X, int64_t ldx, int32_t a, const double *Y, int64_t ldy,
                        int32_t b, int64_t n, double *C, int64_t ldc);

/*
 * C = X^T Y for FP32 device blocks (X n x a, Y n x b, row-major, ldx, ldy),
 * FP64 result C (a x b, ldc), a, b <= 256: the Gram kernels of the
 * mixed-precision step.  When min(a, b) <= 32 (the projections X_bar^T Y) a
 * CUDA-core kernel computes it (exact FP32 products inside the FMA, FP32 sums
 * over at most 256 rows added into double-float, FP64 partial sums); wider
 * products run on the tensor cores (tcgen05 kind::tf32, each value split into
 * two TF32 parts, three products, FP32 accumulation over at most 256 rows,
 * FP64 partial sums).  Blocks whose base address or leading dimension is not
 * 16-byte aligned use a generic CUDA-core kernel with the same accumulation
 * rule.  Runs on the context's stream and uses its scratch; returns when C
 * is complete; GREST_ERR_TIMEOUT if a device-side wait gave up.
 */
grest_status grest_gram_f32(grest_ctx *ctx, const float *X, int64_t ldx, int32_t a, const float *Y, int64_t ldy,
                            int32_t b, int64_t n, double *C, int64_t ldc);

/*
 * Out = beta Cin + alpha X B for FP32 device blocks: X (n x a, ldx), Cin and
 * Out (n x c, ldc, ldo), row-major; B (a x c, ldb) FP64 on the device, c <=
 * 256 for the tensor-core path.  This is the block update of the
 * mixed-precision step (the projections X - U (U^T X), the CholQR products
 * V T, the lift Z F_K of Alg. 2).  On sm_100-class GPUs it runs on the tensor
 * cores (tcgen05 kind::tf32 with X and B each split into two TF32 parts,
 * three products, FP32 accumulation over the a columns); shapes or
 * alignments the tensor-core kernel does not take (X not 16-byte aligned, ldx
 * not a multiple of 4, c > 256, a > 512) use a CUDA-core FP32 kernel.  Cin
 * may equal Out (in-place update); X must not overlap Out.  Cin is not read
 * when beta == 0.  Runs on the context's stream and uses its scratch;
 * returns when Out is complete.  Errors: GREST_ERR_INVALID_ARG for null
 * pointers or leading dimensions smaller than the widths,
 * GREST_ERR_TIMEOUT if a device-side wait of the tensor-core kernel gave up.
 */
grest_status grest_gemm_f32(grest_ctx *ctx, int64_t n, int32_t a, int32_t c, double alpha, const float *X,
                            int64_t ldx, const double *B, int64_t ldb, double beta, const float *Cin, int64_t ldc,
                            float *Out, int64_t ldo);

/*
 * grest_gram_noalloc -- the same product as grest_gram, C = X^T Y, for
 * callers that cannot allocate device memory: a host application that hands
 * all of the GPU's memory to its own pool (a cudaMalloc would fail or break
 * the pool's accounting), or a latency-critical loop that must not pay the
 * device-wide synchronization a cudaMalloc/cudaFree can cause.  It needs no
 * context and allocates nothing: it calls no cudaMalloc, cudaFree or other
 * allocating routine.  (The paper has no counterpart; this is a library
 * service.)
 *
 * X (n x a, ldx), Y (n x b, ldy) and C (a x b, ldc) are row-major device
 * arrays owned by the caller; 1 <= a, b <= 256 (larger widths return
 * GREST_ERR_CAPACITY), n >= 1.  The split-K partial sums live in one
 * fixed 4 MiB array of device memory inside the library (a file-scope
 * __device__ array that every GPU loading the library holds until the
 * process exits).  Every call on a device shares that array and the array
 * keeps the last call's contents, so calls that overlap on the GPU (two
 * streams, or two host threads) race and must be serialized by the caller;
 * every partial a call reads is written earlier in the same call, so nothing
 * needs clearing.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress) with that device current; make that first
 * call before any stream capture.  With CUDA's lazy module loading (the
 * default since CUDA 12.2) the array is brought onto a device by that first
 * call, not when the library is loaded, so the first call can fail
 * (GREST_ERR_CUDA) if the caller's pool has already taken all device
 * memory: make one call on each device before the pool reserves memory.
 * The work is enqueued on cuda_stream (NULL = legacy default stream) and C
 * is complete when that stream's work is; the call itself does not
 * synchronize.  A CUDA error already pending on the calling host thread is
 * returned as GREST_ERR_CUDA before anything is enqueued.
 */
grest_status grest_gram_noalloc(const double *X, int64_t ldx, int32_t a, const double *Y, int64_t ldy, int32_t b,
                                int64_t n, double *C, int64_t ldc, void *cuda_stream);

/*
 * grest_check_bounded_wait -- a check of the library's failure detection
 * (the paper has no counterpart).  Every wait of the library's kernels on a
 * device-side barrier is bounded: after about a second without progress the
 * kernel records a timeout, waits (bounded) for its own copies, releases its
 * tensor memory and returns, and the call reports GREST_ERR_TIMEOUT with the
 * device still usable.  This entry point runs that path on purpose: one
 * thread waits on a barrier that nothing arrives on.  It returns
 * GREST_ERR_TIMEOUT (the expected result) after about a second, or
 * GREST_ERR_OOM / GREST_ERR_CUDA.  Work on cuda_stream (NULL = legacy
 * default stream); synchronous.
 */
grest_status grest_check_bounded_wait(void *cuda_stream);

/*
 * grest_check_fast_recip -- a check of the FP64 reciprocal that the small
 * factorizations use in their serial scalar chains (pivots of the pivoted
 * Cholesky, Householder coefficients, the tridiagonal LU of inverse
 * iteration, Jacobi rotations; Alg. 1 and the CholQR of Alg. 2): the
 * hardware's reduced-precision reciprocal refined by two Newton-Raphson
 * steps, within a few units in the last place of 1 / x for normal x with
 * normal 1 / x (other inputs take the IEEE division).  The paper has no
 * counterpart; this is a test hook.
 * x and out are device arrays of n doubles owned by the caller; out[i] =
 * that reciprocal of x[i].  Work on cuda_stream (NULL = legacy default
 * stream); synchronous.  Returns GREST_ERR_INVALID_ARG for n < 0 or a null
 * array with n > 0, GREST_ERR_CUDA on a CUDA error (including one already
 * pending on the calling thread).
 */
grest_status grest_check_fast_recip(const double *x, int64_t n, double *out, void *cuda_stream);

/* Release every device buffer of the context. NULL is ignored. */
void grest_destroy(grest_ctx *ctx);

/*
 * Groups: one update of many small graphs at once, Alg. 2 per graph, with
 * every stage of the step (graph update, SpMM, Grams, block updates, the
 * pivoted Cholesky factorizations, the eigensolves) run as ONE grouped launch
 * for all graphs of the group.  Each graph's shapes (node count, new-node
 * block mode, CholQR ranks, basis width m) stay in device memory, so an
 * update of the whole group needs no host synchronization inside it: the
 * launch sequence is captured once as a CUDA graph and replayed for every
 * later update.  After the first successful update an autotuner times the
 * launch shapes of the SpMM and GEMM stages that compute every row the same
 * way (grid size, rows per warp) and keeps the fastest for the group's shape
 * bucket, so tuning never changes a result.  Each graph's result depends only
 * on its own data: updating it in any group, or alone in a group of one,
 * gives bit-identical pairs.
 *
 * grest_group_create loads n_graphs graphs from checkpoints written by
 * grest_checkpoint (host buffers, read only, not kept).  All must share k,
 * op, L, P, subspace and drop_tol; the group computes in FP64 whatever the
 * checkpoints' precision.  Supported: unweighted graphs without removed
 * nodes, the EXACT projection and the RESID block, and 2k + L + P <= 64
 * columns (k + max(L+P, L) + k <= 64); else GREST_ERR_UNSUPPORTED.  Each
 * graph gets capacity_factor (1 .. 64) times its node ids and edge slots,
 * fixed for the life of the group; a batch of a graph may carry up to a
 * quarter of its nonzeros in edits.  Errors: GREST_ERR_INVALID_ARG (a buffer
 * that is not a checkpoint, mismatched configurations), GREST_ERR_OOM,
 * GREST_ERR_CUDA.
 *
 * grest_group_apply_updates applies updates[i] (host arrays; no node
 * removal, no weights: else GREST_ERR_UNSUPPORTED) to graph i of the group.
 * status (nullable, n_graphs entries) gets each graph's result; stats
 * (nullable) each graph's step diagnostics (no timings).  A graph whose batch
 * is invalid (Sec. 2's definition of Delta) or does not fit its capacity is
 * left unchanged with GREST_ERR_INVALID_UPDATE / GREST_ERR_CAPACITY; the
 * others are updated.  Returns GREST_OK, or the first failing graph's status.
 * Returns when the update has finished on the device.
 *
 * grest_group_get_embedding copies graph i's (X_K, Lambda_K) to host memory
 * (U: n x k row-major, or NULL; theta: k, or NULL); *n_out = its node count.
 * grest_group_get_ritz_values: graph i's m Ritz values of the last update in
 * tracking order (ritz may be NULL to query m).  grest_group_info reports
 * whether the update is captured as a CUDA graph, the kernel launches of one
 * update of the whole group, whether the autotuner has run, and the chosen
 * SpMM grid, rows per warp and GEMM grid (each pointer nullable).
 * grest_group_destroy releases the group (NULL is ignored).
 */
typedef struct grest_group grest_group;
grest_status grest_group_create(int32_t n_graphs, const void *const *ckpts, const int64_t *ckpt_bytes,
                                double capacity_factor, grest_group **out);
grest_status grest_group_apply_updates(grest_group *group, const grest_update *updates, grest_status *status,
                                       grest_stats *stats);
grest_status grest_group_get_embedding(grest_group *group, int32_t i, double *U, double *theta, int64_t *n_out);
grest_status grest_group_get_ritz_values(grest_group *group, int32_t i, double *ritz, int32_t *m);
grest_status grest_group_info(grest_group *group, int32_t *captured, int32_t *launches_per_update, int32_t *tuned,
                              int32_t *spmm_blocks, int32_t *spmm_rows_per_warp, int32_t *gemm_blocks);
void grest_group_destroy(grest_group *group);

/*
 * Batches: many independent graphs, one update each per call.  A batch
 * refers to existing contexts (it owns none of them; destroy them after the
 * batch); each context should have its own non-blocking CUDA stream so that
 * their work overlaps on the device.  grest_batch_apply_updates applies
 * updates[i] to context i as grest_apply_update would, with n_threads host
 * threads taking contexts in turn; each context's result is the same as when
 * it is updated alone (its kernels and their order are unchanged).
 *   n_graphs >= 1, n_threads >= 1, no context twice -> else GREST_ERR_INVALID_ARG.
 *   status (nullable): n_graphs per-context results; stats (nullable):
 *   n_graphs step diagnostics.  Returns GREST_OK, or the first (lowest index)
 *   failing context's status; a failed context keeps its previous state as
 *   with grest_apply_update, the others are updated.
 * The caller must not use the batch's contexts from other threads while a
 * call is running.
 */
typedef struct grest_batch grest_batch;
grest_status grest_batch_create(int32_t n_graphs, grest_ctx *const *ctxs, int32_t n_threads, grest_batch **out);
grest_status grest_batch_apply_updates(grest_batch *batch, const grest_update *updates, grest_status *status,
                                       grest_stats *stats);
void grest_batch_destroy(grest_batch *batch);

/* Device bytes the library allocated for the context (buffers grown by later
 * batches included); used for admission by a memory budget. */
grest_status grest_get_device_bytes(grest_ctx *ctx, int64_t *bytes);

/*
 * Serving many resident graphs.  A server owns n_workers host threads and a
 * device-memory budget.  Graphs are registered with their host CSR (and
 * optional initial pairs; NULL = computed on the device as in grest_init);
 * the server copies them.  A graph becomes resident (its context and its own
 * non-blocking stream are created) when it first has a request and its
 * context fits in the budget beside the resident graphs, or when nothing else
 * is resident; otherwise its requests wait until removals free memory.
 * Requests (one update each, host arrays, copied at submission) of one graph
 * run in submission order; different graphs run concurrently, and a request
 * starts as soon as a worker is free (continuous batching).  Each result is
 * the same as the update applied alone.
 *   grest_server_submit returns a ticket; grest_server_wait blocks until the
 *   ticket's update ran and returns its status, step diagnostics, the time it
 *   waited after submission and the time it ran (ms; any output may be NULL).
 *   grest_server_poll sets *done to 1 once the ticket has run (0 before).
 *   grest_server_remove_graph releases the graph's device memory once its
 *   pending requests have run; no further submissions are accepted for it.
 *   grest_server_get_embedding waits until the graph is idle and copies its
 *   (X_K, Lambda_K, live) to host memory (GREST_ERR_INVALID_ARG when the
 *   graph was never admitted or was removed).
 *   grest_server_resident reports the resident bytes and graph count.
 * The budget is checked at admission against the context's size then; a
 * resident graph whose buffers grow for a larger batch keeps its place (its
 * new size counts toward later admissions).
 *   grest_server_set_eviction(on = 1): when the oldest waiting request
 *   belongs to a graph that does not fit, the least recently used idle
 *   resident graph (no request queued or running) is checkpointed to host
 *   memory (grest_checkpoint) and its context freed, one graph at a time
 *   until the waiting graph fits; an evicted graph is restored from its
 *   checkpoint (grest_restore) at its next admission, so its results are
 *   unchanged by the eviction.  grest_server_get_embedding of an evicted
 *   graph reads the checkpoint.  Off (0, the default): a graph that does
 *   not fit waits until removals free memory.  Other values:
 *   GREST_ERR_INVALID_ARG.
 *   grest_server_counters reports admissions (restores included),
 *   evictions and restores so far (each output nullable).
 * grest_server_destroy stops the workers after their current requests and
 * releases every context; no other call may be in progress or follow.
 */
typedef struct grest_server grest_server;
grest_status grest_server_create(int32_t n_workers, int64_t hbm_budget_bytes, grest_server **out);
grest_status grest_server_add_graph(grest_server *server, const grest_config *cfg, int64_t n, const int64_t *rowptr,
                                    const int32_t *col, const double *val, const double *U0, const double *theta0,
                                    int32_t *graph_id);
grest_status grest_server_submit(grest_server *server, int32_t graph_id, const grest_update *update,
                                 int64_t *ticket);
grest_status grest_server_wait(grest_server *server, int64_t ticket, grest_status *result, grest_stats *stats,
                               double *wait_ms, double *run_ms);
grest_status grest_server_poll(grest_server *server, int64_t ticket, int32_t *done);
grest_status grest_server_remove_graph(grest_server *server, int32_t graph_id);
grest_status grest_server_get_embedding(grest_server *server, int32_t graph_id, double *U, double *theta,
                                        uint8_t *live, int64_t *n_out);
grest_status grest_server_resident(grest_server *server, int64_t *bytes, int32_t *n_resident);
grest_status grest_server_set_eviction(grest_server *server, int32_t on);
grest_status grest_server_counters(grest_server *server, int64_t *admissions, int64_t *evictions,
                                   int64_t *restores);
void grest_server_destroy(grest_server *server);

/* Static string naming a status code. */
const char *grest_status_str(grest_status s);

#ifdef __cplusplus
}
#endif
#endif /* GREST_H */
