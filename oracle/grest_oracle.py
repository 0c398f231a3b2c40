"""Plain FP64 CPU oracle of the G-REST eigenpair update.

TEST INFRASTRUCTURE.  This module exists to check the CUDA library; it is not
part of the product path.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU legs of ``bench.py`` (``cpu_baseline`` and ``--impl reference``) may import
it.  It shares no code with the CUDA path: its only inputs are plain arrays and
batches produced by the seeded generators.

What it computes (paper: "Subspace Projection Methods for Fast Spectral
Embeddings of Evolving Graphs", arXiv 2603.19439), step by step in the paper's
order and notation, in float64 with NumPy/SciPy library primitives
(sparse products, LAPACK QR and symmetric eigensolver):

  Sec. 2, Eq. (adj_update)    A_hat = pad(A) + Delta, Delta = [[K, G], [G^T, C]]
  Sec. 4.2                    operator M: adjacency A, shifted Laplacian
                              T = alpha I - (D - A) with alpha = 2 d_max, or
                              shifted normalized Laplacian T_n = I + D^-1/2 A D^-1/2
  Alg. 2 (pad)                X_bar = [X; 0]
  Sec. 3.3, Eq. for Z, Tab. 1 Z = Ran([X_bar, P_perp [Delta X_bar, Delta_2]])
  Sec. 3.5, steps S.1-S.4     randomized range basis R of P_perp Delta_2
  Sec. 4 (orthogonalization)  only P_perp [Delta X_bar, R] is orthonormalized
  Eq. (main2) / Eq. (main3)   H = Z^T M_new Z (exact) or its rank-K surrogate
  Alg. 1                      leading eigenpairs of H -> Ritz pairs (theta, Z f)
  Sec. 5 (downstream task)    subgraph centrality X_K exp(Lambda_K) X_K^T 1, top-J
                              sets and their overlap

Readings where the paper is silent, ambiguous or garbled:
  R1  EXACT projection (Eq. main2) is the default; LOWRANK (Eq. main3) is a mode.
  R2  default W block is P_perp(M_new X_bar) = P_perp(Delta X_bar) + P_perp(A_bar X_bar);
      it equals the paper's P_perp(Delta X_bar) when X holds exact eigenvectors.
      w_block=DELTA uses the paper's block literally.
  R3  ordering: adjacency by |theta| descending (Sec. 2), ties to the larger
      algebraic value then the lower index; Laplacian kinds algebraic descending.
  R4  sign: each output column is flipped so its largest-|.| entry (lowest
      index among equal magnitudes) is positive.
  R5  rank deficiency: column-pivoted QR, columns whose |R_ii| falls below
      drop_tol * max(|R_00|, |theta_1|) are dropped (Sec. 3.4 notes the low
      rank of Delta_2); |theta_1| of the previous step is about ||M||_2, so a
      block that is pure rounding noise (W when X is exact and Delta = 0) is
      dropped instead of spanning random directions.
  R6  Omega: Philox4x64-10 + Box-Muller, see oracle/philox.py.
  R7  the SVD of the (L+P) x S matrix in S.2 is taken through the eigenpairs
      of B B^T; exact basis when S <= L+P, RSVD otherwise (AUTO).
  R9  Laplacian shift alpha = 2 d_max of the new graph for the exact projection.
  R10 isolated node in T_n: d^-1/2 = 0, so its row of T_n is the identity row.
  R11 node removal (future work in Sec. 6): incident edges removed, the id is
      tombstoned, M is the principal submatrix on live nodes, the tombstoned
      rows of X_bar are zeroed and X_bar is re-orthonormalized.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from .philox import gaussian_matrix

OP_ADJ, OP_LAP, OP_NLAP = 0, 1, 2
SUB_GREST2, SUB_GREST3, SUB_RSVD, SUB_AUTO = 0, 1, 2, 3
WB_RESID, WB_DELTA = 0, 1
PROJ_EXACT, PROJ_LOWRANK = 0, 1


class InvalidUpdate(ValueError):
    """The batch violates Sec. 2's definition of Delta (see validate_batch)."""


class NumericFailure(RuntimeError):
    """Fewer than K Ritz pairs are available (subspace dimension below K)."""


@dataclass
class Config:
    k: int
    op: int = OP_ADJ
    subspace: int = SUB_AUTO
    L: int = 100
    P: int = 100
    w_block: int = WB_RESID
    projection: int = PROJ_EXACT
    seed: int = 0
    drop_tol: float = 1e-7


@dataclass
class State:
    """Graph A^(t) (symmetric CSR over all ids, zero rows at tombstones),
    live mask, the K tracked pairs (X, Lambda) and the step counter t."""
    A: sp.csr_matrix
    live: np.ndarray
    X: np.ndarray
    lam: np.ndarray
    step: int = 0

    @property
    def n(self):
        return self.A.shape[0]


@dataclass
class StepInfo:
    m: int = 0
    K_u: int = 0
    rank_w: int = 0
    rank_b: int = 0
    mode: str = ""
    ritz_all: np.ndarray = field(default_factory=lambda: np.zeros(0))
    pivots_kept_min: float = 0.0
    pivots_dropped_max: float = 0.0
    boundary_gap: float = np.inf
    Z: np.ndarray | None = None
    H: np.ndarray | None = None
    M: object = None


# --------------------------------------------------------------- graph (Sec. 2)

def csr_from_arrays(n, rowptr, col, val=None):
    data = np.ones(col.size) if val is None else np.asarray(val, np.float64)
    return sp.csr_matrix((data, np.asarray(col, np.int64), np.asarray(rowptr, np.int64)), shape=(n, n))


def validate_batch(A, live, b, weighted=False):
    """Check the batch against Sec. 2: K has +1 only for previously unconnected
    and -1 only for previously connected old pairs; G and C connect new nodes;
    edges join distinct nodes (no self loops).  Additionally (node removal
    reading) deleted nodes must be live old nodes and no edge edit may touch
    them.  Raises InvalidUpdate."""
    n = A.shape[0]
    S = int(b.n_new)
    if S < 0:
        raise InvalidUpdate("negative new-node count")
    n2 = n + S
    iu = np.asarray(b.ins_u, np.int64)
    iv = np.asarray(b.ins_v, np.int64)
    du = np.asarray(b.del_u, np.int64)
    dv = np.asarray(b.del_v, np.int64)
    dn = np.asarray(b.del_nodes, np.int64)
    live2 = np.concatenate([live, np.ones(S, bool)])
    if iu.size != iv.size or du.size != dv.size:
        raise InvalidUpdate("edge arrays differ in length")
    for u, v in ((iu, iv), (du, dv)):
        if u.size and (u.min() < 0 or v.min() < 0 or u.max() >= n2 or v.max() >= n2):
            raise InvalidUpdate("node id out of range")
        if np.any(u == v):
            raise InvalidUpdate("self loop")
    if du.size and (du.max() >= n or dv.max() >= n):
        raise InvalidUpdate("deleted edge touches a new node")
    if weighted and b.ins_w is not None:
        w = np.asarray(b.ins_w, np.float64)
        if w.size != iu.size or np.any(~np.isfinite(w)) or np.any(w <= 0):
            raise InvalidUpdate("weights must be positive and finite")
    if dn.size:
        if dn.min() < 0 or dn.max() >= n:
            raise InvalidUpdate("deleted node id out of range")
        if np.unique(dn).size != dn.size:
            raise InvalidUpdate("duplicate deleted node")
        if not np.all(live[dn]):
            raise InvalidUpdate("deleted node already tombstoned")
    dead = ~live2
    dead[dn] = True
    for u, v in ((iu, iv), (du, dv)):
        if u.size and np.any(dead[u] | dead[v]):
            raise InvalidUpdate("edge touches a tombstoned or deleted node")
    allk = np.concatenate([np.minimum(iu, iv) * n2 + np.maximum(iu, iv),
                           np.minimum(du, dv) * n2 + np.maximum(du, dv)])
    if np.unique(allk).size != allk.size:
        raise InvalidUpdate("edge listed twice in the batch")
    old = (iu < n) & (iv < n)
    if np.any(old):
        ex = np.asarray(A[iu[old], iv[old]]).ravel()
        if np.any(ex != 0):
            raise InvalidUpdate("inserted edge already present")
    if du.size:
        ex = np.asarray(A[du, dv]).ravel()
        if np.any(ex == 0):
            raise InvalidUpdate("deleted edge not present")


def apply_batch(A, live, b):
    """A^(t+1) = pad(A^(t)) + Delta (Eq. adj_update), then node tombstones."""
    n = A.shape[0]
    S = int(b.n_new)
    n2 = n + S
    Ab = sp.csr_matrix((A.data, A.indices, np.concatenate([A.indptr, np.full(S, A.indptr[-1])])), shape=(n2, n2))
    iu = np.asarray(b.ins_u, np.int64)
    iv = np.asarray(b.ins_v, np.int64)
    du = np.asarray(b.del_u, np.int64)
    dv = np.asarray(b.del_v, np.int64)
    w = np.ones(iu.size) if b.ins_w is None else np.asarray(b.ins_w, np.float64)
    dw = np.asarray(A[du, dv]).ravel() if du.size else np.zeros(0)
    rows = np.concatenate([iu, iv, du, dv])
    cols = np.concatenate([iv, iu, dv, du])
    vals = np.concatenate([w, w, -dw, -dw])
    Delta = sp.csr_matrix((vals, (rows, cols)), shape=(n2, n2))
    live2 = np.concatenate([live, np.ones(S, bool)])
    dn = np.asarray(b.del_nodes, np.int64)
    if dn.size:
        # removing every edge incident to a deleted node is part of Delta too
        Adn = (Ab + Delta).tocsr()
        mask = np.zeros(n2)
        mask[dn] = 1.0
        Dm = sp.diags(mask)
        inc = (Dm @ Adn + Adn @ Dm - Dm @ Adn @ Dm)
        Delta = Delta - inc
        live2[dn] = False
    Anew = (Ab + Delta).tocsr()
    Anew.eliminate_zeros()
    Delta = Delta.tocsr()
    Delta.eliminate_zeros()
    return Anew, live2, Delta


# ------------------------------------------------------------ operator (Sec 4.3)

def operator_matrix(A, live, op):
    """M for the operator kind on the live principal submatrix (zero elsewhere).
    Returns (M, alpha): alpha = 2 d_max for the shifted Laplacian, else 0."""
    n = A.shape[0]
    d = np.asarray(A.sum(axis=1)).ravel()
    lv = live.astype(np.float64)
    if op == OP_ADJ:
        return A.tocsr(), 0.0
    if op == OP_LAP:
        alpha = 2.0 * (d[live].max() if np.any(live) else 0.0)
        M = sp.diags(lv * (alpha - d)) + A
        return M.tocsr(), alpha
    if op == OP_NLAP:
        dis = np.zeros(n)
        pos = (d > 0) & live
        dis[pos] = 1.0 / np.sqrt(d[pos])
        Dh = sp.diags(dis)
        M = sp.diags(lv) + Dh @ A @ Dh
        return M.tocsr(), 0.0
    raise ValueError("unknown operator kind")


def dense_operator(A, live, op):
    M, _ = operator_matrix(A, live, op)
    return M.toarray()


# ----------------------------------------------------------- linear algebra

def project_out(X, V):
    """P_perp V = (I - X X^T) V."""
    return V - X @ (X.T @ V)


def orth_pivoted(V, drop_tol, abs_ref=0.0):
    """Orthonormal basis of Ran(V) by Householder QR with column pivoting;
    columns with |R_ii| <= drop_tol * max(|R_00|, abs_ref) are dropped
    (reading R5: abs_ref is a magnitude of the operator, so a block made only
    of rounding noise is dropped whole).
    Returns (Q, kept_min_ratio, dropped_max_ratio)."""
    if V.shape[1] == 0:
        return np.zeros((V.shape[0], 0)), np.inf, 0.0
    Q, R, _ = sla.qr(V, mode="economic", pivoting=True)
    dg = np.abs(np.diag(R))
    if dg.size == 0 or max(dg[0], abs_ref) == 0.0:
        return np.zeros((V.shape[0], 0)), np.inf, 0.0
    ratio = dg / max(dg[0], abs_ref)
    keep = ratio > drop_tol
    r = int(np.argmin(keep)) if not np.all(keep) else keep.size
    kmin = float(ratio[r - 1]) if r else np.inf
    dmax = float(ratio[r]) if r < ratio.size else 0.0
    return Q[:, :r], kmin, dmax


def orth_against(X, V, drop_tol, abs_ref=0.0):
    """Q = orth(P_perp V), re-projected once against X (two projection passes)."""
    V1 = project_out(X, V)
    Q1, kmin, dmax = orth_pivoted(V1, drop_tol, abs_ref)
    if Q1.shape[1] == 0:
        return Q1, kmin, dmax
    V2 = project_out(X, Q1)
    Q2, _ = np.linalg.qr(V2)
    return Q2, kmin, dmax


def select_order(theta, op):
    """Indices of all Ritz values in tracking order (reading R3)."""
    idx = np.arange(theta.size)
    if op == OP_ADJ:
        return np.array(sorted(idx, key=lambda i: (-abs(theta[i]), -theta[i], i)), dtype=np.int64)
    return np.array(sorted(idx, key=lambda i: (-theta[i], i)), dtype=np.int64)


def normalize_signs(X):
    """Flip each column so its largest-magnitude entry is positive (reading R4)."""
    X = X.copy()
    for j in range(X.shape[1]):
        col = X[:, j]
        if col.size == 0:
            continue
        i = int(np.argmax(np.abs(col)))
        if col[i] < 0:
            X[:, j] = -col
    return X


# --------------------------------------------------------- RSVD (Sec. 3.5)

def rsvd_range_basis(E, Xb, Omega, L, drop_tol, abs_ref=0.0):
    """Steps S.1-S.4: Y = P_perp Delta_2 Omega, M = orth(Y), SVD of M^T P_perp Delta_2
    (through its Gram, reading R7), R = M U_hat_L.  Returns (R, rank of M)."""
    Y = project_out(Xb, E @ Omega)                              # S.1
    Mb, _, _ = orth_pivoted(Y, drop_tol, abs_ref)               # M = orth(Ran(Y))
    if Mb.shape[1] == 0:
        return np.zeros((E.shape[0], 0)), 0
    # S.2: M^T P_perp Delta_2 = M^T Delta_2 - (M^T X_bar)(X_bar^T Delta_2), E kept sparse
    MtE = np.asarray((E.T @ Mb).T)
    XtE = np.asarray((E.T @ Xb).T)
    Bs = MtE - (Mb.T @ Xb) @ XtE
    ev, Uh = np.linalg.eigh(Bs @ Bs.T)                           # left singular vectors
    order = np.argsort(-ev, kind="stable")
    Lp = min(L, Mb.shape[1])
    Uh = Uh[:, order[:Lp]]
    return Mb @ Uh, Mb.shape[1]                                  # S.4: R = M U_hat


# ------------------------------------------------------------- the step (Alg 2)

def grest_step(state: State, b, cfg: Config, weighted=False, keep=False):
    """One iteration of Alg. 2 (G-REST).  Returns (new State, StepInfo);
    keep=True also returns the basis Z, the projected H and the operator M."""
    validate_batch(state.A, state.live, b, weighted)
    n, S, K = state.n, int(b.n_new), cfg.k
    Aold, live_old = state.A, state.live
    Anew, live, Delta = apply_batch(Aold, live_old, b)
    n2 = n + S
    M, alpha = operator_matrix(Anew, live, cfg.op)
    info = StepInfo()

    # Alg. 2: X_bar = [X; 0]; reading R11 zeroes tombstoned rows and re-orthonormalizes
    Xb = np.zeros((n2, state.X.shape[1]))
    Xb[:n] = state.X
    if np.asarray(b.del_nodes).size:
        Xb[~live] = 0.0
        Xb, _, _ = orth_pivoted(Xb, cfg.drop_tol, 1.0)
    Ku = Xb.shape[1]
    info.K_u = Ku
    scale = abs(state.lam[0]) if state.lam.size else 0.0   # |theta_1| ~ ||M||_2 (reading R5)

    # Delta of the operator (used by the paper's W block and by Eq. main3)
    def delta_op():
        Mold, _ = operator_matrix(Aold, live_old, cfg.op)
        Mold_p = sp.csr_matrix((Mold.data, Mold.indices, np.concatenate([Mold.indptr, np.full(S, Mold.indptr[-1])])), shape=(n2, n2))
        return (M - Mold_p).tocsr()

    # perturbation-derived block (Sec. 3.3): W = P_perp (M_new X_bar) or P_perp (Delta X_bar)
    Y1 = M @ Xb
    if cfg.w_block == WB_RESID:
        W = project_out(Xb, Y1)
    else:
        W = project_out(Xb, delta_op() @ Xb)
    W = project_out(Xb, W)

    # new-node block Delta_2 = trailing S columns of Delta (Prop. 3), = M_new[:, N:]
    use_rsvd = False
    Bblk = np.zeros((n2, 0))
    if S > 0 and cfg.subspace != SUB_GREST2:
        E = M[:, n:n2]
        q = cfg.L + cfg.P
        use_rsvd = cfg.subspace == SUB_RSVD or (cfg.subspace == SUB_AUTO and S > q)
        if use_rsvd:
            Omega = gaussian_matrix(cfg.seed, state.step, S, q)
            Bblk, _ = rsvd_range_basis(E, Xb, Omega, cfg.L, cfg.drop_tol, scale)
        else:
            Bblk = project_out(Xb, E.toarray())
    info.mode = "GREST2" if (S == 0 or cfg.subspace == SUB_GREST2) else ("RSVD" if use_rsvd else "GREST3")

    # orthonormalize only P_perp [W, B] (partial-orthogonality remark, Sec. 4)
    V = np.hstack([W, Bblk])
    Q, kmin, dmax = orth_against(Xb, V, cfg.drop_tol, scale)
    info.pivots_kept_min, info.pivots_dropped_max = kmin, dmax
    Z = np.hstack([Xb, Q])
    m = Z.shape[1]
    info.m = m
    info.rank_w = min(Q.shape[1], W.shape[1])
    info.rank_b = Q.shape[1] - info.rank_w
    if m < K:
        raise NumericFailure("subspace dimension below K")

    # Rayleigh-Ritz matrix: Eq. (main2) or Eq. (main3)
    if cfg.projection == PROJ_EXACT:
        H = Z.T @ (M @ Z)
    else:
        XZ = Xb.T @ Z
        lam = state.lam
        H = XZ.T @ (lam[:Ku, None] * XZ) + Z.T @ (delta_op() @ Z)
    H = 0.5 * (H + H.T)

    # Alg. 1: leading eigenpairs of H, Ritz vectors Z f
    theta, F = np.linalg.eigh(H)
    order = select_order(theta, cfg.op)
    info.ritz_all = theta[order]
    sel = order[:K]
    if m > K:
        a, bb = abs(theta[order[K - 1]]), abs(theta[order[K]])
        if cfg.op != OP_ADJ:
            a, bb = theta[order[K - 1]], theta[order[K]]
        info.boundary_gap = abs(a - bb) / max(abs(theta[order[0]]), 1e-300)
    Xnew = normalize_signs(Z @ F[:, sel])
    if keep:
        info.Z, info.H, info.M = Z, H, M
    return State(A=Anew, live=live, X=Xnew, lam=theta[sel].copy(), step=state.step + 1), info


# ------------------------------------------------------------ Sec. 5 downstream task

def subgraph_centrality(X, lam, live):
    """Sec. 5: exp(A) 1 approximated from the K tracked pairs as
    X_K exp(Lambda_K) X_K^T 1, multiplied by exp(-max(lam)) (a positive common
    factor, so the ranking is unchanged and nothing overflows).  Removed nodes
    (live false) take no part in X^T 1 and get the value 0."""
    X = np.where(live[:, None], X, 0.0)
    s = X.T @ np.ones(X.shape[0])
    c = X @ (np.exp(lam - lam.max()) * s)
    return np.where(live, c, 0.0)


def top_central(c, live, J):
    """Sec. 5: the J most central live nodes, by value descending; equal values
    go to the lower node id, so the set and its order are unique."""
    ids = np.flatnonzero(live)
    order = np.lexsort((ids, -c[ids]))
    return ids[order[:J]]


def central_overlap(found, ref):
    """Sec. 5 accuracy measure: |I_hat intersect I| / J for two top-J id sets."""
    return len(np.intersect1d(found, ref)) / max(len(ref), 1)


# ------------------------------------------------------------ helpers for tests

def init_state(n, rowptr, col, val, K, op, X0=None, lam0=None, dense_limit=4000):
    """Initial pairs of Alg. 2 by a direct eigendecomposition: dense eigh
    for small graphs, scipy eigsh otherwise; the same X0 is given to both sides."""
    A = csr_from_arrays(n, rowptr, col, val)
    live = np.ones(n, bool)
    if X0 is None:
        X0, lam0 = leading_pairs(A, live, K, op, dense_limit)
    return State(A=A, live=live, X=np.array(X0, np.float64), lam=np.array(lam0, np.float64), step=0)


def leading_pairs(A, live, K, op, dense_limit=4000):
    M, _ = operator_matrix(A, live, op)
    n = M.shape[0]
    if n <= dense_limit:
        ev, V = np.linalg.eigh(M.toarray())
    else:
        import scipy.sparse.linalg as sla_sp
        which = "LM" if op == OP_ADJ else "LA"
        ev, V = sla_sp.eigsh(M, k=min(K + 8, n - 1), which=which, tol=1e-12)
    order = select_order(ev, op)[:K]
    return normalize_signs(V[:, order]), ev[order]
