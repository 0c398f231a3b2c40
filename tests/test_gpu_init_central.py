"""GPU parity of the two entry points around the tracking loop: the on-device
initial eigensolver (grest_init without U0 / theta0) against the oracle's
direct eigendecomposition, and grest_centrality (Sec. 5's subgraph
centrality and top-J sets) against the oracle's formula."""
import numpy as np
import pytest

import oracle as O
from paper_2603_19439_gb300 import grest as G
from paper_2603_19439_gb300 import workloads as wl
from tests import gpu_util as U

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_19439_gb300.build import build
    build()
    torch.cuda.set_device(0)
    return torch


def full_spectrum(g, op):
    rp, col, val = g.csr()
    A = O.csr_from_arrays(g.n, rp, col, val)
    M, _ = O.operator_matrix(A, np.ones(g.n, bool), op)
    ev, V = np.linalg.eigh(M.toarray())
    order = O.select_order(ev, op)
    return M, ev[order], V[:, order]


def check_initial_pairs(tr, M, ev, V, op, k):
    Ug, thg, _ = tr.embedding()
    scale = abs(ev[0])
    assert np.max(np.abs(thg - ev[:k])) <= U.THETA_TOL * scale, np.max(np.abs(thg - ev[:k])) / scale
    j = U.cluster_cut(ev, op, k)
    ang = U.sin_angle(V[:, :j], Ug[:, :j])
    assert ang <= U.ANGLE_TOL, (ang, j)
    assert np.abs(Ug.T @ Ug - np.eye(k)).max() < 1e-12
    res = np.linalg.norm(M @ Ug - Ug * thg, axis=0).max()
    assert res <= 1e-11 * scale, res / scale
    # R4 signs: the largest-magnitude entry of every column is positive
    idx = np.argmax(np.abs(Ug), axis=0)
    assert np.all(Ug[idx, np.arange(k)] > 0)


@pytest.mark.parametrize("op", [O.OP_ADJ, O.OP_LAP, O.OP_NLAP])
@pytest.mark.parametrize("weighted", [False, True])
def test_device_initial_pairs_match_dense_eigh(op, weighted):
    g = wl.chung_lu_graph(2500, 2.3, 8, 11 + op)
    if weighted:
        g = wl.EdgeSetGraph(g.n, g.keys, np.random.default_rng(4).uniform(0.5, 2.0, size=g.keys.size))
    M, ev, V = full_spectrum(g, op)
    k = 16
    rp, col, val = g.csr()
    tr = G.Tracker(g.n, rp, col, val, None, None, k, op=op)
    check_initial_pairs(tr, M, ev, V, op, k)
    tr.close()


@pytest.mark.parametrize("k", [1, 8, 32])
def test_device_initial_pairs_sbm(k):
    """Equal-size communities: degenerate clusters inside the tracked block."""
    g, _ = wl.sbm_graph(1500, 6, 0.04, 0.002, 3)
    op = O.OP_ADJ
    M, ev, V = full_spectrum(g, op)
    rp, col, val = g.csr()
    tr = G.Tracker(g.n, rp, col, val, None, None, k, op=op)
    check_initial_pairs(tr, M, ev, V, op, k)
    tr.close()


def test_device_initial_pairs_rejects_half_given():
    g = wl.chung_lu_graph(300, 2.3, 6, 1)
    rp, col, val = g.csr()
    with pytest.raises(G.GrestError):
        G.Tracker(g.n, rp, col, val, np.eye(g.n, 4), None, 4)


def test_device_initial_pairs_chung_lu_200k():
    """A larger member of the benchmark family against ARPACK (tol 1e-12)."""
    g = wl.chung_lu_graph(200_000, 2.3, 8, 21)
    rp, col, val = g.csr()
    op, k = O.OP_ADJ, 32
    A = O.csr_from_arrays(g.n, rp, col, val)
    M, _ = O.operator_matrix(A, np.ones(g.n, bool), op)
    import scipy.sparse.linalg as ssl
    ev, V = ssl.eigsh(M, k=k + 8, which="LM", tol=1e-13)
    order = O.select_order(ev, op)
    ev, V = ev[order], V[:, order]
    tr = G.Tracker(g.n, rp, col, val, None, None, k, op=op)
    Ug, thg, _ = tr.embedding()
    scale = abs(ev[0])
    assert np.max(np.abs(thg - ev[:k])) <= U.THETA_TOL * scale
    j = U.cluster_cut(ev, op, k)
    assert U.sin_angle(V[:, :j], Ug[:, :j]) <= U.ANGLE_TOL
    res = np.linalg.norm(M @ Ug - Ug * thg, axis=0).max()
    assert res <= 1e-11 * scale
    tr.close()


# ------------------------------------------------------------------ centrality

def check_top_valid(c, live, ids, vals, J):
    """The GPU's top-J list is the unique one its own values define: live ids,
    values descending, equal values by id ascending, nothing outside it ranks
    higher."""
    assert len(ids) == J and len(set(ids.tolist())) == J
    assert np.all(live[ids])
    assert np.array_equal(vals, c[ids])
    for a in range(J - 1):
        assert vals[a] > vals[a + 1] or (vals[a] == vals[a + 1] and ids[a] < ids[a + 1])
    rest = np.setdiff1d(np.flatnonzero(live), ids)
    if J and rest.size:
        lo_v, lo_i = vals[-1], ids[-1]
        assert np.all((c[rest] < lo_v) | ((c[rest] == lo_v) & (rest > lo_i)))


def compare_sets(ids, ref_ids, c_ref, tol):
    """Equal top-J sets up to near-ties at the threshold of the oracle's values."""
    if len(ref_ids) == 0:
        return
    thr = c_ref[ref_ids[-1]]
    for i in np.setxor1d(ids, ref_ids):
        assert abs(c_ref[i] - thr) <= tol, (i, c_ref[i], thr)


@pytest.mark.parametrize("op", [O.OP_ADJ, O.OP_NLAP])
def test_centrality_after_tracking_matches_oracle(op):
    g = wl.chung_lu_graph(4000, 2.3, 8, 31)
    k = 16
    tr, st, cfg = U.make_pair(g, k, op)
    rng = np.random.default_rng(2)
    gb = g.copy()
    for t in range(3):
        b = wl.random_churn_batch(gb, 20, 60, 40, rng, n_del_nodes=2)
        gb.apply(b)
        tr.update(b)
        st, _ = O.grest_step(st, b, cfg)
    c_ref = O.subgraph_centrality(st.X, st.lam, st.live)
    J = 100
    ref_ids = O.top_central(c_ref, st.live, J)
    c, ids, vals = tr.centrality(J)
    scale = np.abs(c_ref).max()
    assert np.abs(c - c_ref).max() <= 1e-7 * scale
    _, _, live = tr.embedding()
    check_top_valid(c, live, ids, vals, J)
    compare_sets(ids, ref_ids, c_ref, 2e-7 * scale)
    tr.close()


def test_centrality_values_from_set_state_bitwise_ties_and_limits(cuda):
    """The kernel's arithmetic on a given state: c within rounding of the
    oracle's, many exact ties (rows drawn from 40 patterns, identical rows give
    identical values on the device), removed nodes, and every J limit."""
    torch = cuda
    rng = np.random.default_rng(8)
    g = wl.chung_lu_graph(50_000, 2.3, 6, 9)
    rp, col, val = g.csr()
    k = 24
    X0 = np.linalg.qr(rng.standard_normal((g.n, k)))[0]
    tr = G.Tracker(g.n, rp, col, val, X0, np.linspace(5, 1, k), k)
    # remove a few nodes through an update so that live is not all-true
    dead = np.array([3, 17, 4000, 49_999], np.int32)
    b = wl.Batch(n_new=0, ins_u=np.zeros(0, np.int32), ins_v=np.zeros(0, np.int32), del_u=np.zeros(0, np.int32),
                 del_v=np.zeros(0, np.int32), del_nodes=dead)
    tr.update(b)
    pat = rng.standard_normal((40, k))
    X = pat[rng.integers(0, 40, size=g.n)]
    lam = np.sort(rng.uniform(-3.0, 6.0, size=k))[::-1].copy()
    tr.set_embedding(X, lam)
    _, _, live = tr.embedding()
    assert live.sum() == g.n - dead.size
    c_ref = O.subgraph_centrality(X, lam, live)
    scale = np.abs(c_ref).max()
    for J in (0, 1, 7, 100, 1000, 4096):
        c, ids, vals = tr.centrality(J)
        assert np.abs(c - c_ref).max() <= 1e-13 * scale
        assert np.all(c[~live] == 0.0)
        check_top_valid(c, live, ids, vals, J)
        compare_sets(ids, O.top_central(c_ref, live, J), c_ref, 1e-13 * scale)
    # device outputs
    cd = torch.empty(g.n, dtype=torch.float64, device="cuda")
    idd = torch.empty(500, dtype=torch.int32, device="cuda")
    vd = torch.empty(500, dtype=torch.float64, device="cuda")
    tr.centrality_device(500, cd, idd, vd)
    c, ids, vals = tr.centrality(500)
    assert np.array_equal(cd.cpu().numpy(), c)
    assert np.array_equal(idd.cpu().numpy(), ids) and np.array_equal(vd.cpu().numpy(), vals)
    for bad in (-1, 4097):
        with pytest.raises(G.GrestError):
            tr.centrality(bad)
    tr.close()


def test_centrality_small_graph_all_nodes():
    """J equal to the live count, n below one CTA, and J above it rejected."""
    g = wl.chung_lu_graph(60, 2.3, 4, 2)
    M, ev, V = full_spectrum(g, O.OP_ADJ)
    rp, col, val = g.csr()
    k = 5
    tr = G.Tracker(g.n, rp, col, val, V[:, :k], ev[:k], k)
    c_ref = O.subgraph_centrality(V[:, :k], ev[:k], np.ones(g.n, bool))
    c, ids, vals = tr.centrality(g.n)
    assert np.abs(c - c_ref).max() <= 1e-13 * np.abs(c_ref).max()
    check_top_valid(c, np.ones(g.n, bool), ids, vals, g.n)
    with pytest.raises(G.GrestError):
        tr.centrality(g.n + 1)
    tr.close()


@pytest.mark.parametrize("op", [O.OP_ADJ, O.OP_LAP, O.OP_NLAP])
def test_device_initial_pairs_dense_route_small_graph(op):
    """n <= 288: the device solver takes H = M densely (no Krylov rounds)."""
    g = wl.chung_lu_graph(250, 2.3, 6, 40 + op)
    M, ev, V = full_spectrum(g, op)
    k = 12
    rp, col, val = g.csr()
    tr = G.Tracker(g.n, rp, col, val, None, None, k, op=op)
    check_initial_pairs(tr, M, ev, V, op, k)
    tr.close()


@pytest.mark.parametrize("op", [O.OP_ADJ, O.OP_NLAP])
def test_tracking_from_device_initial_pairs(op):
    """Device start, then update steps: the oracle starts from its own dense
    eigendecomposition of the same graph (the two starts agree to ~1e-12), and
    the tracked pairs stay within the FP64 tolerances step by step."""
    g = wl.chung_lu_graph(3000, 2.3, 8, 51 + op)
    k = 16
    rp, col, val = g.csr()
    tr = G.Tracker(g.n, rp, col, val, None, None, k, op=op)
    st = O.init_state(g.n, rp, col, val, k, op)
    cfg = O.Config(k=k, op=op, subspace=G.SUB_AUTO, L=100, P=100, seed=0, drop_tol=1e-7)
    rng = np.random.default_rng(5)
    gb = g.copy()
    for t in range(3):
        b = wl.random_churn_batch(gb, 15, 50, 30, rng)
        gb.apply(b)
        tr.update(b)
        st, info = O.grest_step(st, b, cfg)
        U.compare(tr, st, info, op, k, f"step {t}")
    tr.close()
