"""Pins for the FP64 CPU oracle: facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: the worked
example of Fig. 1, closed-form spectra, brute-force dense eigendecompositions,
Cauchy interlacing, the Rayleigh-Ritz optimality of Thm. 1, the Galerkin
condition, Props. 1, 3 and 4, RSVD exactness for low-rank Delta_2 (Sec. 3.5),
basis independence of the orthonormalization (pivoted QR against CholQR2),
and an independent Philox implementation (numpy's).
"""
import json
import os

import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
from oracle.philox import gaussian_matrix, philox4x64_10
from paper_2603_19439_gb300 import workloads as wl

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def state_from_edges(n, edges, K, op, weights=None, dense=True):
    keys = wl.keys_of(np.array([e[0] for e in edges], np.int64), np.array([e[1] for e in edges], np.int64)) if edges else np.zeros(0, np.int64)
    g = wl.EdgeSetGraph(n, keys, weights)
    rp, col, val = g.csr()
    return O.init_state(n, rp, col, val, K, op), g


def batch(n_new=0, ins=(), dels=(), del_nodes=(), ins_w=None):
    ins = np.array(ins, np.int32).reshape(-1, 2)
    dels = np.array(dels, np.int32).reshape(-1, 2)
    return wl.Batch(n_new=n_new, ins_u=ins[:, 0].copy(), ins_v=ins[:, 1].copy(), del_u=dels[:, 0].copy(),
                    del_v=dels[:, 1].copy(), del_nodes=np.array(del_nodes, np.int32),
                    ins_w=None if ins_w is None else np.array(ins_w, np.float64))


def sin_angle(U, V):
    """sin of the largest principal angle between Ran(U) and Ran(V) (orthonormal)."""
    P = V - U @ (U.T @ V)
    return np.linalg.norm(P, 2)


# ------------------------------------------------------------------ Philox

def test_philox_matches_independent_numpy_philox():
    # numpy's Philox (4x64, 10 rounds) increments its counter before each block
    for key, ctr in (([0, 0], [0, 0, 0, 0]), ([123456789, 987654321], [5, 7, 9, 11]),
                     ([2**64 - 1, 2**63 + 5], [2**64 - 3, 1, 2, 3])):
        bg = np.random.Philox(counter=np.array(ctr, dtype=np.uint64), key=np.array(key, dtype=np.uint64))
        ref = [int(x) for x in bg.random_raw(8)]
        c0 = (ctr[0] + 1) % 2**64
        mine = list(philox4x64_10((c0, *ctr[1:]), key)) + list(philox4x64_10(((ctr[0] + 2) % 2**64, *ctr[1:]), key))
        assert mine == ref


def test_gaussian_matrix_is_standard_normal():
    from scipy import stats
    Om = gaussian_matrix(7, 3, 200, 100)
    z = Om.ravel()
    assert abs(z.mean()) < 0.02 and abs(z.var() - 1) < 0.03
    assert stats.kstest(z, "norm").pvalue > 1e-3
    # different step or seed gives a different (uncorrelated) matrix
    Om2 = gaussian_matrix(7, 4, 200, 100)
    assert abs(np.corrcoef(Om.ravel(), Om2.ravel())[0, 1]) < 0.03
    # deterministic
    assert np.array_equal(Om, gaussian_matrix(7, 3, 200, 100))


# ------------------------------------------------------------ Fig. 1 example

def fig1():
    with open(os.path.join(GOLD, "fig1_example.json")) as f:
        return json.load(f)


def test_fig1_delta_blocks_match_caption():
    d = fig1()
    n = d["n_before"]
    edges = [(a - 1, b - 1) for a, b in d["edges_before"]]
    st, _ = state_from_edges(n, edges, 2, O.OP_ADJ)
    ins = [(a - 1, b - 1) for a, b in d["added_edges_old"] + d["added_edges_new"]]
    dels = [(a - 1, b - 1) for a, b in d["deleted_edges"]]
    b = batch(n_new=d["n_new"], ins=ins, dels=dels)
    O.validate_batch(st.A, st.live, b)
    Anew, live, Delta = O.apply_batch(st.A, st.live, b)
    D = Delta.toarray()
    Kc = np.zeros((n, n))
    for i, j, v in d["caption_K"]:
        Kc[i - 1, j - 1] = v
    Gc = np.zeros((n, d["n_new"]))
    for i, j, v in d["caption_G"]:
        Gc[i - 1, j - 1] = v
    assert np.array_equal(D[:n, :n], Kc)
    assert np.array_equal(D[:n, n:], Gc)
    assert np.array_equal(D[n:, :n], Gc.T)
    assert np.array_equal(D[n:, n:], np.zeros((2, 2)))   # no edge among 7 and 8
    # A_hat = pad(A) + Delta (Eq. adj_update), and the drawn G^(t+1)
    Ab = np.zeros((8, 8))
    Ab[:6, :6] = st.A.toarray()
    assert np.array_equal(Anew.toarray(), Ab + D)
    assert Anew.nnz == 2 * (7 - 1 + 2 + 4)


def test_fig1_brute_force_exact():
    """K=3 on Fig. 1: Z spans R^8 (m = 3 + 3 + 2), so G-REST equals dense eigh."""
    d = fig1()
    edges = [(a - 1, b - 1) for a, b in d["edges_before"]]
    ins = [(a - 1, b - 1) for a, b in d["added_edges_old"] + d["added_edges_new"]]
    dels = [(a - 1, b - 1) for a, b in d["deleted_edges"]]
    for op in (O.OP_ADJ, O.OP_LAP, O.OP_NLAP):
        st, _ = state_from_edges(6, edges, 3, op)
        cfg = O.Config(k=3, op=op, subspace=O.SUB_GREST3)
        st2, info = O.grest_step(st, batch(2, ins, dels), cfg, keep=True)
        Md = O.dense_operator(st2.A, st2.live, op)
        ev, V = np.linalg.eigh(Md)
        o = O.select_order(ev, op)
        if info.m == 8:
            assert np.allclose(st2.lam, ev[o[:3]], rtol=0, atol=1e-12)
            gap = abs(abs(ev[o[2]]) - abs(ev[o[3]]))
            if gap > 1e-8:
                assert sin_angle(V[:, o[:3]], st2.X) < 1e-10


# ---------------------------------------------------- operators: closed forms

def complete(n):
    return [(i, j) for i in range(n) for j in range(i + 1, n)]


def cycle(n):
    return [(i, (i + 1) % n) for i in range(n)]


def path(n):
    return [(i, i + 1) for i in range(n - 1)]


def star(n):
    return [(0, i) for i in range(1, n)]


def kab(a, b):
    return [(i, a + j) for i in range(a) for j in range(b)]


def spectrum(n, edges, op):
    st, _ = state_from_edges(n, edges, 1, op)
    return np.sort(np.linalg.eigvalsh(O.dense_operator(st.A, st.live, op)))


def test_closed_form_adjacency_spectra():
    n = 9
    assert np.allclose(spectrum(n, complete(n), O.OP_ADJ), np.sort([n - 1] + [-1] * (n - 1)))
    assert np.allclose(spectrum(n, cycle(n), O.OP_ADJ), np.sort(2 * np.cos(2 * np.pi * np.arange(n) / n)))
    assert np.allclose(spectrum(n, path(n), O.OP_ADJ), np.sort(2 * np.cos(np.pi * np.arange(1, n + 1) / (n + 1))))
    assert np.allclose(spectrum(n, star(n), O.OP_ADJ), np.sort([np.sqrt(n - 1), -np.sqrt(n - 1)] + [0] * (n - 2)))
    a, b = 3, 5
    assert np.allclose(spectrum(a + b, kab(a, b), O.OP_ADJ), np.sort([np.sqrt(a * b), -np.sqrt(a * b)] + [0] * (a + b - 2)))


def test_closed_form_shifted_laplacians():
    n = 8
    # T = alpha I - L, alpha = 2 d_max (Sec. 4.2); L(K_n) = {0, n x (n-1)}
    al = 2 * (n - 1)
    assert np.allclose(spectrum(n, complete(n), O.OP_LAP), np.sort([al] + [al - n] * (n - 1)))
    # cycle: L eigenvalues 2 - 2cos(2 pi j/n), d_max = 2, alpha = 4
    assert np.allclose(spectrum(n, cycle(n), O.OP_LAP), np.sort(4 - (2 - 2 * np.cos(2 * np.pi * np.arange(n) / n))))
    # T_n = 2I - L_n with L_n(K_n) = {0, n/(n-1) x (n-1)}
    assert np.allclose(spectrum(n, complete(n), O.OP_NLAP), np.sort([2.0] + [2 - n / (n - 1)] * (n - 1)))
    # Gershgorin bounds of Sec. 4.2: T in [0, 2 d_max], T_n in [0, 2]
    g, _ = wl.sbm_graph(60, 3, 0.3, 0.05, 5)
    rp, col, _ = g.csr()
    A = O.csr_from_arrays(60, rp, col)
    live = np.ones(60, bool)
    ev = np.linalg.eigvalsh(O.dense_operator(A, live, O.OP_LAP))
    dmax = np.asarray(A.sum(1)).max()
    assert ev.min() > -1e-9 and ev.max() < 2 * dmax + 1e-9
    ev = np.linalg.eigvalsh(O.dense_operator(A, live, O.OP_NLAP))
    assert ev.min() > -1e-9 and ev.max() < 2 + 1e-9


def test_isolated_node_nlap_identity_row():
    st, _ = state_from_edges(4, [(0, 1), (1, 2)], 1, O.OP_NLAP)
    M = O.dense_operator(st.A, st.live, O.OP_NLAP)
    assert np.array_equal(M[3], [0, 0, 0, 1.0])


# ------------------------------------------------------------- exactness (§4)

def random_graph(n, p, seed):
    g, _ = wl.sbm_graph(n, 2, p, p / 4, seed)
    return g


@pytest.mark.parametrize("op", [O.OP_ADJ, O.OP_LAP, O.OP_NLAP])
def test_exact_when_subspace_is_whole_space(op):
    """With K = 7, N = 14 and S = 4, the basis [X_bar, W, B] has up to
    2K + S = 18 = N' columns; when it spans the whole space, H = Z^T M Z is
    similar to M, so every Ritz value is an eigenvalue of the dense operator
    and the tracked pairs are the exact leading ones."""
    rng = np.random.default_rng(1)
    hits = 0
    for trial in range(4):
        g = random_graph(14, 0.35, 10 + trial)
        K = 7
        rp, col, _ = g.csr()
        st = O.init_state(g.n, rp, col, None, K, op)
        b = wl.random_churn_batch(g, 4, 3, 3, rng)
        st2, info = O.grest_step(st, b, O.Config(k=K, op=op, subspace=O.SUB_GREST3), keep=True)
        Md = O.dense_operator(st2.A, st2.live, op)
        ev, V = np.linalg.eigh(Md)
        o = O.select_order(ev, op)
        assert np.linalg.matrix_rank(info.Z) == info.m
        if info.m == Md.shape[0]:
            hits += 1
            assert np.allclose(np.sort(info.ritz_all), np.sort(ev), atol=1e-11)
            assert np.allclose(st2.lam, ev[o[:K]], atol=1e-11)
            # the tracked subspace is the exact one where the K / K+1 boundary is separated
            key = np.abs(ev[o]) if op == O.OP_ADJ else ev[o]
            if abs(key[K - 1] - key[K]) > 1e-6:
                assert sin_angle(V[:, o[:K]], st2.X) < 1e-9
    assert hits >= 3, f"the whole-space case was reached in {hits} of 4 trials"


@pytest.mark.parametrize("op", [O.OP_ADJ, O.OP_LAP, O.OP_NLAP])
def test_noop_update_keeps_exact_pairs(op):
    g = random_graph(40, 0.2, 3)
    rp, col, _ = g.csr()
    K = 4
    st = O.init_state(g.n, rp, col, None, K, op)
    st2, info = O.grest_step(st, batch(), O.Config(k=K, op=op))
    assert info.m == K   # W = P_perp(A X) is pure rounding noise when X is exact: dropped
    assert np.allclose(st2.lam, st.lam, atol=1e-12)
    assert sin_angle(st.X, st2.X) < 1e-10


def test_disjoint_component_append_is_exact():
    """G = 0 and C a new component: Ran(Z) contains an invariant subspace
    holding the leading pairs of A_hat (Sec. 4 exactness construction)."""
    g = random_graph(30, 0.25, 4)
    rp, col, _ = g.csr()
    K = 3
    st = O.init_state(g.n, rp, col, None, K, O.OP_ADJ)
    # new component: a dense clique on 6 new nodes (eigenvalue 5 may enter the top 3)
    ins = [(30 + i, 30 + j) for i in range(6) for j in range(i + 1, 6)]
    st2, info = O.grest_step(st, batch(6, ins), O.Config(k=K, op=O.OP_ADJ, subspace=O.SUB_GREST3))
    ev = np.linalg.eigvalsh(O.dense_operator(st2.A, st2.live, O.OP_ADJ))
    o = O.select_order(ev, O.OP_ADJ)
    assert np.allclose(st2.lam, ev[o[:K]], atol=1e-11)


# ---------------------------------------------------- RR theory (Alg. 1, Thm 1)

def stream_step(op=O.OP_ADJ, K=6, n=120, S=8, seed=11, subspace=O.SUB_GREST3):
    rng = np.random.default_rng(seed)
    g = random_graph(n, 0.08, seed)
    rp, col, _ = g.csr()
    st = O.init_state(g.n, rp, col, None, K, op)
    b = wl.random_churn_batch(g, S, 10, 6, rng)
    st2, info = O.grest_step(st, b, O.Config(k=K, op=op, subspace=subspace), keep=True)
    return st, st2, info


@pytest.mark.parametrize("op", [O.OP_ADJ, O.OP_LAP, O.OP_NLAP])
def test_cauchy_interlacing(op):
    _, st2, info = stream_step(op)
    lam = np.sort(np.linalg.eigvalsh(O.dense_operator(st2.A, st2.live, op)))[::-1]
    th = np.sort(info.ritz_all)[::-1]
    m = th.size
    assert np.all(th <= lam[:m] + 1e-10)
    assert np.all(th[::-1] >= lam[::-1][:m] - 1e-10)


def test_thm1_rr_optimality_and_galerkin():
    _, st2, info = stream_step()
    Z, M = info.Z, info.M
    MZ = M @ Z
    S0 = Z.T @ MZ
    r0 = np.linalg.norm(MZ - Z @ S0, 2)
    # equals ||Z_perp^T M Z||_2
    Qf, _ = np.linalg.qr(np.hstack([Z, np.random.default_rng(0).standard_normal((Z.shape[0], Z.shape[0] - Z.shape[1]))]))
    Zp = Qf[:, Z.shape[1]:]
    assert abs(r0 - np.linalg.norm(Zp.T @ MZ, 2)) < 1e-9
    rng = np.random.default_rng(1)
    for _ in range(20):
        E = rng.standard_normal(S0.shape) * 1e-3
        assert np.linalg.norm(MZ - Z @ (S0 + E), 2) >= r0 - 1e-12
    # Galerkin condition Z^T (M u - theta u) = 0 for every output pair
    R = M @ st2.X - st2.X * st2.lam
    assert np.abs(Z.T @ R).max() < 1e-10 * max(1, abs(st2.lam).max())
    # orthonormality of Z and of the output
    assert np.abs(Z.T @ Z - np.eye(Z.shape[1])).max() < 1e-13
    assert np.abs(st2.X.T @ st2.X - np.eye(st2.X.shape[1])).max() < 1e-13


def test_ritz_vectors_beat_other_bases_of_the_subspace():
    """Thm 1, second part: Z F minimizes ||M P - P D|| over bases P of Ran(Z)."""
    _, st2, info = stream_step()
    Z, M = info.Z, info.M
    th, F = np.linalg.eigh(Z.T @ (M @ Z))
    P = Z @ F
    best = np.linalg.norm(M @ P - P * th, 2)
    rng = np.random.default_rng(3)
    for _ in range(10):
        Qr, _ = np.linalg.qr(F + 1e-2 * rng.standard_normal(F.shape))
        P2 = Z @ Qr
        D = np.diag(np.diag(P2.T @ M @ P2))
        assert np.linalg.norm(M @ P2 - P2 @ D, 2) >= best - 1e-12


def test_orth_against_matches_cholqr2_basis():
    """Basis independence (the device path orthonormalizes by CholQR2, the
    oracle by pivoted QR): Q = orth_against(X, V) spans the same space as a
    Cholesky-based basis of (I - X X^T) V built here from its definition,
    is orthonormal and orthogonal to X, and both bases give the same Ritz
    values of M on [X, Q]."""
    _, st2, info = stream_step()
    M = info.M
    rng = np.random.default_rng(5)
    n = M.shape[0]
    X = np.linalg.qr(rng.standard_normal((n, 6)))[0]
    V = rng.standard_normal((n, 9))
    Q, _, _ = O.orth_against(X, V, 1e-10)
    assert Q.shape[1] == 9
    W = V - X @ (X.T @ V)
    W = W - X @ (X.T @ W)
    for _ in range(2):  # CholQR2: W <- W R^-1 with R^T R = W^T W
        R = np.linalg.cholesky(W.T @ W).T
        W = np.linalg.solve(R.T, W.T).T
    assert np.abs(Q.T @ Q - np.eye(9)).max() < 1e-13
    assert np.abs(X.T @ Q).max() < 1e-13
    assert np.abs(Q @ Q.T - W @ W.T).max() < 1e-12
    ritz = lambda B: np.linalg.eigvalsh(B.T @ (M @ B))
    ra, rb = ritz(np.hstack([X, Q])), ritz(np.hstack([X, W]))
    assert np.abs(ra - rb).max() <= 1e-12 * np.abs(ra).max()


# ------------------------------------------------------------ Props 1, 3, 4

def test_prop1_corollary_no_K_block():
    """With K = 0 (only new nodes), x_bar_i^T Delta x_bar_j = 0 (Corollary to Prop. 1)."""
    g = random_graph(50, 0.15, 8)
    rp, col, _ = g.csr()
    st = O.init_state(g.n, rp, col, None, 4, O.OP_ADJ)
    ins = [(50, 3), (50, 7), (51, 9), (51, 50), (52, 1)]
    _, _, Delta = O.apply_batch(st.A, st.live, batch(3, ins))
    Xb = np.vstack([st.X, np.zeros((3, 4))])
    assert np.abs(Xb.T @ (Delta @ Xb)).max() == 0.0


def test_prop3_range_of_delta_xbar():
    rng = np.random.default_rng(5)
    g = random_graph(60, 0.1, 9)
    rp, col, _ = g.csr()
    st = O.init_state(g.n, rp, col, None, 5, O.OP_ADJ)
    b = wl.random_churn_batch(g, 6, 8, 5, rng)
    _, _, Delta = O.apply_batch(st.A, st.live, b)
    D = Delta.toarray()
    Xb = np.vstack([st.X, np.zeros((6, 5))])
    D1 = D[:, :60]
    assert np.allclose(D @ Xb, D1 @ st.X, atol=1e-14)
    r1 = np.linalg.matrix_rank(D1)
    assert np.linalg.matrix_rank(np.hstack([D1, D @ Xb])) == r1


def test_prop4_rank_bound_of_delta2():
    rng = np.random.default_rng(6)
    for seed in range(5):
        g = random_graph(80, 0.08, 20 + seed)
        rp, col, _ = g.csr()
        st = O.init_state(g.n, rp, col, None, 4, O.OP_ADJ)
        S = 12
        # new nodes attach to only 3 old nodes: J = 3
        hubs = rng.choice(80, size=3, replace=False)
        ins = [(80 + s, int(hubs[s % 3])) for s in range(S)] + [(80 + s, int(hubs[(s + 1) % 3])) for s in range(0, S, 2)]
        _, _, Delta = O.apply_batch(st.A, st.live, batch(S, ins))
        D2 = Delta.toarray()[:, 80:]
        J = np.unique([e[1] for e in ins]).size
        Q = np.unique([e[0] for e in ins]).size
        assert np.linalg.matrix_rank(D2) <= min(J, Q)


# ------------------------------------------------------- modes and readings

def _alpha(A, live, op):
    return O.operator_matrix(A, live, op)[1]


@pytest.mark.parametrize("op", [O.OP_ADJ, O.OP_LAP])
def test_resid_block_equals_delta_block_at_exact_eigvecs(op):
    """Reading R2: P_perp(M_new X_bar) = P_perp(Delta X_bar) + P_perp(M_old X_bar)
    with M_old padded by zero rows, and M_old X_bar = X_bar Lambda when X is
    exact, so both blocks give one Z.  For the shifted Laplacian (Sec. 4.2)
    the batch raises d_max, so Delta carries the change of alpha = 2 d_max on
    every old diagonal entry besides the degree changes (reading R9)."""
    rng = np.random.default_rng(7)
    g = random_graph(70, 0.12, 31)
    rp, col, _ = g.csr()
    K = 5
    st = O.init_state(g.n, rp, col, None, K, op)  # exact (dense eigh)
    b = wl.random_churn_batch(g, 5, 6, 4, rng)
    if op == O.OP_LAP:  # three new edges at the node of largest degree: d_max and alpha grow
        hub = int(np.argmax(np.diff(rp)))
        others = [v for v in range(g.n) if v != hub and not g.has(wl.keys_of(np.array([hub]), np.array([v])))[0]]
        extra = np.array(others[:3], np.int32)
        b = wl.Batch(b.n_new, np.concatenate([b.ins_u, np.full(3, hub, np.int32)]),
                     np.concatenate([b.ins_v, extra]), b.del_u, b.del_v, b.del_nodes)
    s1, i1 = O.grest_step(st, b, O.Config(k=K, op=op, w_block=O.WB_RESID, subspace=O.SUB_GREST3), keep=True)
    s2, i2 = O.grest_step(st, b, O.Config(k=K, op=op, w_block=O.WB_DELTA, subspace=O.SUB_GREST3), keep=True)
    if op == O.OP_LAP:
        assert _alpha(s1.A, s1.live, op) > _alpha(st.A, st.live, op)
    assert i1.m == i2.m
    assert np.allclose(s1.lam, s2.lam, rtol=1e-10, atol=1e-12)
    assert sin_angle(i1.Z, i2.Z) < 1e-8


def test_rsvd_equals_exact_when_delta2_low_rank():
    """Sec. 3.5: if rank(Delta_2) < L+P the sketch recovers Ran(P_perp Delta_2)
    with probability one, so G-REST_RSVD reproduces G-REST_3."""
    rng = np.random.default_rng(8)
    g = random_graph(150, 0.06, 41)
    rp, col, _ = g.csr()
    K = 4
    st = O.init_state(g.n, rp, col, None, K, O.OP_ADJ)
    S = 40
    hubs = rng.choice(150, size=5, replace=False)
    ins = []
    for s in range(S):
        for h in rng.choice(hubs, size=2, replace=False):
            ins.append((150 + s, int(h)))
    b = batch(S, ins)
    ex, ie = O.grest_step(st, b, O.Config(k=K, subspace=O.SUB_GREST3, seed=3))
    rs, ir = O.grest_step(st, b, O.Config(k=K, subspace=O.SUB_RSVD, L=10, P=6, seed=3))
    assert ie.m == ir.m
    assert np.allclose(ex.lam, rs.lam, rtol=1e-10, atol=1e-12)
    assert sin_angle(ex.X, rs.X) < 1e-8


@pytest.mark.parametrize("op", [O.OP_ADJ, O.OP_LAP])
def test_lowrank_equals_exact_when_all_pairs_tracked(op):
    """Eq. (main3) replaces M_old by X_bar Lambda X_bar^T; with K = N that is
    exact, so H = (X_bar^T Z)^T Lambda (X_bar^T Z) + Z^T Delta Z equals
    Z^T M_new Z.  For the shifted Laplacian this fixes Delta's diagonal:
    alpha_new - alpha_old minus the degree change on old rows, and
    alpha_new - d on the rows of new nodes (reading R9); the batch adds
    nodes and raises d_max so both are exercised."""
    rng = np.random.default_rng(9)
    g = random_graph(12, 0.4, 51)
    rp, col, _ = g.csr()
    K = 12
    st = O.init_state(g.n, rp, col, None, K, op)
    b = wl.random_churn_batch(g, 2, 2, 2, rng)
    if op == O.OP_LAP:
        hub = int(np.argmax(np.diff(rp)))
        free = [v for v in range(g.n) if v != hub and not g.has(wl.keys_of(np.array([hub]), np.array([v])))[0]
                and not any({hub, v} == {int(a), int(c)} for a, c in zip(b.ins_u, b.ins_v))]
        b = wl.Batch(b.n_new, np.concatenate([b.ins_u, np.array([hub, hub], np.int32)]),
                     np.concatenate([b.ins_v, np.array([12, free[0]], np.int32)]), b.del_u, b.del_v, b.del_nodes)
    e1, i1 = O.grest_step(st, b, O.Config(k=K, op=op, projection=O.PROJ_EXACT, subspace=O.SUB_GREST3))
    e2, i2 = O.grest_step(st, b, O.Config(k=K, op=op, projection=O.PROJ_LOWRANK, subspace=O.SUB_GREST3))
    if op == O.OP_LAP:
        assert _alpha(e1.A, e1.live, op) > _alpha(st.A, st.live, op)
    assert b.n_new == 2
    assert np.allclose(i1.ritz_all, i2.ritz_all, atol=1e-11)
    assert np.allclose(e1.lam, e2.lam, atol=1e-11)


def test_grest2_subspace_ignores_new_node_block():
    """G-REST_2 uses Ran[X_bar, P_perp Delta X_bar] only (Sec. 5): dimension <= 2K."""
    _, st2, info = stream_step(subspace=O.SUB_GREST2)
    assert info.m <= 2 * 6


@pytest.mark.parametrize("op", [O.OP_ADJ, O.OP_LAP, O.OP_NLAP])
def test_node_deletion_reading(op):
    """Reading R11 on a step that removes nodes: removed ids have zero rows
    in X and M; the Ritz values interlace the spectrum of the live principal
    submatrix (Cauchy: Z restricted to the live rows is orthonormal); the
    Galerkin condition holds; and the output is orthonormal."""
    rng = np.random.default_rng(10)
    g = random_graph(40, 0.2, 61)
    rp, col, _ = g.csr()
    K = 5
    st = O.init_state(g.n, rp, col, None, K, op)
    b = wl.random_churn_batch(g, 3, 4, 3, rng, n_del_nodes=3)
    st2, info = O.grest_step(st, b, O.Config(k=K, op=op, subspace=O.SUB_GREST3), keep=True)
    dead = np.asarray(b.del_nodes)
    assert dead.size == 3
    assert np.all(st2.X[dead] == 0) and not st2.live[dead].any()
    Md = O.dense_operator(st2.A, st2.live, op)
    assert np.all(Md[dead] == 0) and np.all(Md[:, dead] == 0)
    livei = np.flatnonzero(st2.live)
    Z = info.Z
    assert np.all(Z[dead] == 0)
    assert np.abs(Z.T @ Z - np.eye(Z.shape[1])).max() < 1e-13
    lam = np.sort(np.linalg.eigvalsh(Md[np.ix_(livei, livei)]))[::-1]
    th = np.sort(info.ritz_all)[::-1]
    m = th.size
    assert np.all(th <= lam[:m] + 1e-10) and np.all(th[::-1] >= lam[::-1][:m] - 1e-10)
    R = Md @ st2.X - st2.X * st2.lam
    assert np.abs(Z.T @ R).max() < 1e-10 * max(1.0, abs(st2.lam).max())
    assert np.abs(st2.X.T @ st2.X - np.eye(K)).max() < 1e-13


@pytest.mark.parametrize("op", [O.OP_ADJ, O.OP_LAP, O.OP_NLAP])
def test_node_deletion_exact_on_whole_live_space(op):
    """Reading R11 with exactness: N = 10, two nodes removed and S = 2 added,
    K = 4, so [X_bar, W, B] (at most 2K + S = 10 columns) can span all 10 live
    ids; then the tracked pairs are exactly the leading pairs of the live
    principal submatrix, which only holds if the masked X_bar was
    re-orthonormalized correctly."""
    hits = 0
    for trial in range(4):
        rng = np.random.default_rng(100 + trial)
        g = random_graph(10, 0.5, 70 + trial)
        rp, col, _ = g.csr()
        K = 4
        st = O.init_state(g.n, rp, col, None, K, op)
        b = wl.random_churn_batch(g, 2, 2, 1, rng, n_del_nodes=2)
        st2, info = O.grest_step(st, b, O.Config(k=K, op=op, subspace=O.SUB_GREST3), keep=True)
        livei = np.flatnonzero(st2.live)
        assert livei.size == 10
        if info.m != livei.size:
            continue
        hits += 1
        Md = O.dense_operator(st2.A, st2.live, op)
        ev = np.linalg.eigvalsh(Md[np.ix_(livei, livei)])
        o = O.select_order(ev, op)
        assert np.allclose(np.sort(info.ritz_all), np.sort(ev), atol=1e-11)
        assert np.allclose(st2.lam, ev[o[:K]], atol=1e-11)
    assert hits >= 2, f"the whole-live-space case was reached in {hits} of 4 trials"


def test_ordering_and_signs():
    th = np.array([1.0, -3.0, 3.0, 0.5, -0.5, 2.0])
    assert list(O.select_order(th, O.OP_ADJ)) == [2, 1, 5, 0, 3, 4]
    assert list(O.select_order(th, O.OP_LAP)) == [2, 5, 0, 3, 4, 1]
    X = np.array([[0.1, -0.2], [-0.9, 0.2], [0.3, 0.1]])
    Y = O.normalize_signs(X)
    assert Y[1, 0] > 0 and Y[0, 1] > 0 and Y[1, 1] < 0  # tie |-0.2|=|0.2| -> lowest index


def test_invalid_batches_rejected():
    st, _ = state_from_edges(5, [(0, 1), (1, 2), (2, 3)], 2, O.OP_ADJ)
    bad = [batch(0, [(0, 1)]), batch(0, [], [(0, 4)]), batch(0, [(2, 2)]), batch(0, [(0, 9)]),
           batch(1, [(5, 1), (1, 5)]), batch(0, [(0, 3)], [(0, 3)]), batch(0, [], [(0, 1)], [0]),
           batch(0, [], [], [1, 1]), batch(1, [], [(5, 0)])]
    for b in bad:
        with pytest.raises(O.InvalidUpdate):
            O.validate_batch(st.A, st.live, b)
    O.validate_batch(st.A, st.live, batch(1, [(0, 3), (5, 4)], [(0, 1)]))


def test_weighted_graph_matches_dense_definition():
    st, _ = state_from_edges(4, [(0, 1), (1, 2), (2, 3)], 2, O.OP_LAP, weights=[2.0, 0.5, 1.5])
    M = O.dense_operator(st.A, st.live, O.OP_LAP)
    A = np.zeros((4, 4))
    for (i, j), w in zip([(0, 1), (1, 2), (2, 3)], [2.0, 0.5, 1.5]):
        A[i, j] = A[j, i] = w
    d = A.sum(1)
    assert np.allclose(M, 2 * d.max() * np.eye(4) - (np.diag(d) - A))


def test_sbm_trajectory_tracks_dense_truth():
    """SBM stream (n=400 -> 440, K=8): G-REST_3 stays near the true leading pair,
    and on every step the larger subspace of G-REST_3 (Ran Z_2 in Ran Z_3) gives a
    top Ritz value at least the G-REST_2 one and at most lambda_1 (min-max)."""
    g0, batches = wl.sbm_stream(n0=400, steps=4, n_new=10, n_rand=40)
    rp, col, _ = g0.csr()
    K = 8
    st = O.init_state(g0.n, rp, col, None, K, O.OP_ADJ)
    for b in batches:
        s2, _ = O.grest_step(st, b, O.Config(k=K, subspace=O.SUB_GREST2))
        st, info = O.grest_step(st, b, O.Config(k=K, seed=1))
        ev = np.linalg.eigvalsh(O.dense_operator(st.A, st.live, O.OP_ADJ))
        assert s2.lam[0] <= st.lam[0] + 1e-12 <= ev.max() + 2e-12
    ev, V = np.linalg.eigh(O.dense_operator(st.A, st.live, O.OP_ADJ))
    o = O.select_order(ev, O.OP_ADJ)
    psi1 = np.arccos(min(1.0, abs(V[:, o[0]] @ st.X[:, 0])))
    assert psi1 < 0.1
    assert abs(st.lam[0] - ev[o[0]]) / ev[o[0]] < 1e-2


def test_rsvd_steps_give_top_left_singular_vectors():
    """When L < rank(P_perp Delta_2) < L+P, Ran(Y) = Ran(P_perp Delta_2) and
    S.2-S.4 must return exactly its top-L left singular subspace (checked
    against a dense LAPACK SVD)."""
    rng = np.random.default_rng(12)
    n, S, K = 90, 30, 4
    X, _ = np.linalg.qr(rng.standard_normal((n + S, K)))
    X[n:] = 0
    X, _ = np.linalg.qr(X)
    # Delta_2 of rank 8: rows on 8 "hub" nodes only, random weights
    E = np.zeros((n + S, S))
    hubs = rng.choice(n, size=8, replace=False)
    E[hubs] = rng.standard_normal((8, S))
    Om = gaussian_matrix(5, 0, S, 11)
    R, r = O.rsvd_range_basis(sp.csr_matrix(E), X, Om, 5, 1e-9)
    assert r == 8 and R.shape[1] == 5
    PE = E - X @ (X.T @ E)
    Usv, sv, _ = np.linalg.svd(PE, full_matrices=False)
    assert sv[4] - sv[5] > 1e-3 * sv[0]
    assert sin_angle(Usv[:, :5], R) < 1e-10
    assert np.abs(R.T @ R - np.eye(5)).max() < 1e-13


# ------------------------------------------------------------------ Sec. 5 subgraph centrality

def test_centrality_with_all_pairs_equals_matrix_exponential():
    """K = N: X exp(Lambda) X^T 1 is exp(A) 1 exactly (scipy's expm, Pade)."""
    import scipy.linalg as sla
    g = wl.chung_lu_graph(40, 2.3, 4, 5)
    rp, col, val = g.csr()
    A = O.csr_from_arrays(g.n, rp, col, val).toarray()
    lam, V = np.linalg.eigh(A)
    live = np.ones(g.n, bool)
    c = O.subgraph_centrality(V, lam, live)
    ref = sla.expm(A) @ np.ones(g.n) * np.exp(-lam.max())
    assert np.abs(c - ref).max() <= 1e-12 * np.abs(ref).max()
    # a removed node: the principal submatrix on the live nodes, 0 for the removed one
    live[7] = False
    Al = A[np.ix_(live, live)]
    lam2, V2 = np.linalg.eigh(Al)
    X = np.zeros((g.n, g.n - 1))
    X[live] = V2
    c2 = O.subgraph_centrality(X, lam2, live)
    ref2 = sla.expm(Al) @ np.ones(g.n - 1) * np.exp(-lam2.max())
    assert c2[7] == 0.0
    assert np.abs(c2[live] - ref2).max() <= 1e-12 * np.abs(ref2).max()


def test_centrality_closed_forms():
    """Complete graph K_n: 1 is the eigenvector of n - 1, so exp(A) 1 = e^(n-1) 1
    from the top pair alone.  Star with m leaves: 1 lies in the span of the
    +-sqrt(m) pairs, and exp(A) 1 = cosh(r) 1 + sinh(r) / r * A 1, r = sqrt(m):
    hub cosh r + r sinh r, leaves cosh r + sinh(r) / r."""
    n = 9
    X = np.full((n, 1), 1 / np.sqrt(n))
    c = O.subgraph_centrality(X, np.array([n - 1.0]), np.ones(n, bool))
    assert np.allclose(c, 1.0, rtol=0, atol=1e-14)
    m = 16
    r = np.sqrt(m)
    st, _ = state_from_edges(m + 1, [(0, j) for j in range(1, m + 1)], 2, O.OP_ADJ)
    assert np.allclose(np.sort(st.lam), [-r, r], atol=1e-12)
    c = O.subgraph_centrality(st.X, st.lam, np.ones(m + 1, bool)) * np.exp(r)
    assert abs(c[0] - (np.cosh(r) + r * np.sinh(r))) <= 1e-12 * c[0]
    assert np.abs(c[1:] - (np.cosh(r) + np.sinh(r) / r)).max() <= 1e-12 * c[0]


def test_top_central_order_ties_and_removed_nodes():
    c = np.array([3.0, 5.0, 5.0, 1.0, 5.0, 0.0, 7.0, -2.0])
    live = np.array([1, 1, 1, 1, 0, 1, 1, 1], bool)
    assert O.top_central(c, live, 3).tolist() == [6, 1, 2]
    assert O.top_central(c, live, 4).tolist() == [6, 1, 2, 0]
    assert O.top_central(c, live, 7).tolist() == [6, 1, 2, 0, 3, 5, 7]
    assert O.central_overlap(np.array([6, 1, 2]), np.array([2, 6, 0])) == pytest.approx(2 / 3)
