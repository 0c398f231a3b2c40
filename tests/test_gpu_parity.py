"""GPU parity: the CUDA library (through its C ABI) against the FP64 CPU oracle
on the same seeded inputs.  Every step of the CUDA path runs in libgrest's
kernels; the oracle never sees a value the GPU produced."""
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


def hub_graph(n, seed, weighted=False):
    """Power-law graph plus one star hub with more neighbours than the long-row cut."""
    g = wl.chung_lu_graph(n, 2.3, 8, seed)
    keys = np.union1d(g.keys, wl.keys_of(np.zeros(n - 1, np.int64), np.arange(1, n)))
    w = None
    if weighted:
        w = np.random.default_rng(seed).uniform(0.5, 2.0, size=keys.size)
    return wl.EdgeSetGraph(n, keys, w)


@pytest.mark.parametrize("op", [O.OP_ADJ, O.OP_LAP, O.OP_NLAP])
@pytest.mark.parametrize("weighted", [False, True])
def test_spmm_matches_oracle_operator(cuda, op, weighted):
    torch = cuda
    g = hub_graph(3000, 7 + op, weighted)
    rp, col, val = g.csr()
    k = 4
    X0 = np.linalg.qr(np.random.default_rng(1).standard_normal((g.n, k)))[0]
    tr = G.Tracker(g.n, rp, col, val, X0, np.ones(k), k, op=op)
    M, _ = O.operator_matrix(O.csr_from_arrays(g.n, rp, col, val), np.ones(g.n, bool), op)
    rng = np.random.default_rng(3)
    for w in (1, 8, 33, 130, 288):
        Xh = rng.standard_normal((g.n, w))
        X = torch.tensor(Xh, dtype=torch.float64, device="cuda")
        Y = torch.empty_like(X)
        tr.apply_operator(X, Y)
        ref = M @ Xh
        err = np.abs(Y.cpu().numpy() - ref).max() / np.abs(ref).max()
        assert err < 1e-13, (w, err)
    tr.close()


@pytest.mark.parametrize("op", [O.OP_ADJ, O.OP_LAP, O.OP_NLAP])
def test_fig1_example(cuda, op):
    import json, os
    d = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "fig1_example.json")))
    edges = [(a - 1, b - 1) for a, b in d["edges_before"]]
    g = wl.EdgeSetGraph(6, wl.keys_of([e[0] for e in edges], [e[1] for e in edges]))
    tr, st, ocfg = U.make_pair(g, 3, op, subspace=G.SUB_GREST3)
    ins = np.array([(a - 1, b - 1) for a, b in d["added_edges_old"] + d["added_edges_new"]], np.int32)
    dels = np.array([(a - 1, b - 1) for a, b in d["deleted_edges"]], np.int32)
    b = wl.Batch(2, ins[:, 0].copy(), ins[:, 1].copy(), dels[:, 0].copy(), dels[:, 1].copy())
    st2, info = O.grest_step(st, b, ocfg)
    tr.update(b)
    U.compare(tr, st2, info, op, 3, "fig1")
    # brute force: the whole space is spanned, so the pairs are the exact ones
    ev = np.linalg.eigvalsh(O.dense_operator(st2.A, st2.live, op))
    o = O.select_order(ev, op)
    _, th, _ = tr.embedding()
    if info.m == 8:
        assert np.allclose(th, ev[o[:3]], atol=1e-12)
    tr.close()


def test_sbm_stream_config(cuda):
    """SBM n=2,000, 4 communities, p_in=0.05, p_out=0.005, K=8, 10 steps of
    +50 nodes and +200 random edges (exact new-node block, m <= 66)."""
    g0, batches = wl.sbm_stream()
    tr, st, ocfg = U.make_pair(g0, 8, O.OP_ADJ)
    for t, b in enumerate(batches):
        st, info = O.grest_step(st, b, ocfg)
        s = tr.update(b)
        assert s["m"] == info.m and s["mode"] == 3
        U.compare(tr, st, info, O.OP_ADJ, 8, f"sbm step {t}")
    tr.close()


def test_rsvd_stream_nlap(cuda):
    """Chung-Lu (gamma 2.5), normalized Laplacian, S > L+P so the RSVD basis
    (steps S.1-S.4) is used; Omega comes from the shared Philox definition."""
    g0, batches = wl.chung_lu_stream(4000, 2.5, 12, 4, 0.02, 6, 0.002, seed=11, lcc=True)
    tr, st, ocfg = U.make_pair(g0, 8, O.OP_NLAP, L=20, P=12, seed=5)
    for t, b in enumerate(batches):
        st, info = O.grest_step(st, b, ocfg)
        s = tr.update(b)
        assert info.mode == "RSVD" and s["mode"] == 4
        assert s["m"] == info.m
        U.compare(tr, st, info, O.OP_NLAP, 8, f"rsvd step {t}")
    tr.close()


def test_laplacian_with_node_removal(cuda):
    rng = np.random.default_rng(21)
    g, _ = wl.sbm_graph(600, 3, 0.06, 0.01, 21)
    gb = g.copy()
    tr, st, ocfg = U.make_pair(g, 6, O.OP_LAP)
    for t in range(4):
        b = wl.random_churn_batch(gb, 12, 30, 20, rng, n_del_nodes=3 if t % 2 == 0 else 0)
        gb.apply(b)
        st, info = O.grest_step(st, b, ocfg)
        tr.update(b)
        U.compare(tr, st, info, O.OP_LAP, 6, f"lap step {t}")
    _, _, live = tr.embedding()
    assert live.sum() == st.live.sum() and (~live).sum() == 6
    tr.close()


def test_weighted_adjacency(cuda):
    rng = np.random.default_rng(31)
    g = hub_graph(900, 31, weighted=True)
    gb = g.copy()
    tr, st, ocfg = U.make_pair(g, 5, O.OP_ADJ, subspace=G.SUB_GREST3)
    for t in range(3):
        b = wl.random_churn_batch(gb, 8, 25, 15, rng)
        b.ins_w = rng.uniform(0.5, 2.0, size=b.n_ins)
        gb.apply(b)
        st, info = O.grest_step(st, b, ocfg, weighted=True)
        tr.update(b)
        U.compare(tr, st, info, O.OP_ADJ, 5, f"weighted step {t}")
    tr.close()


def test_invalid_batches_leave_state_unchanged(cuda):
    rng = np.random.default_rng(41)
    g, _ = wl.sbm_graph(300, 2, 0.1, 0.02, 41)
    tr, st, ocfg = U.make_pair(g, 4, O.OP_ADJ)
    U0, th0, live0 = tr.embedding()
    u, v = wl.split_keys(g.keys[:3])
    absent = np.array([0, 1], np.int32)
    while g.has(wl.keys_of([absent[0]], [absent[1]]))[0]:
        absent[1] += 1
    bad = [
        wl.Batch(0, u[:1], v[:1], np.zeros(0, np.int32), np.zeros(0, np.int32)),           # insert existing
        wl.Batch(0, np.zeros(0, np.int32), np.zeros(0, np.int32), absent[:1], absent[1:]),  # delete missing
        wl.Batch(0, np.array([5], np.int32), np.array([5], np.int32), np.zeros(0, np.int32), np.zeros(0, np.int32)),
        wl.Batch(1, np.array([300, 3], np.int32), np.array([3, 300], np.int32), np.zeros(0, np.int32), np.zeros(0, np.int32)),
        wl.Batch(0, np.array([0], np.int32), np.array([999], np.int32), np.zeros(0, np.int32), np.zeros(0, np.int32)),
        wl.Batch(0, np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0, np.int32),
                 del_nodes=np.array([7, 7], np.int32)),
        wl.Batch(0, np.array([7], np.int32), np.array([absent[1]], np.int32), np.zeros(0, np.int32),
                 np.zeros(0, np.int32), del_nodes=np.array([7], np.int32)),
    ]
    for i, b in enumerate(bad):
        with pytest.raises(G.GrestError) as e:
            tr.update(b)
        assert e.value.code == 2, i
        U1, th1, live1 = tr.embedding()
        assert np.array_equal(U0, U1) and np.array_equal(th0, th1) and np.array_equal(live0, live1)
    # the context still works and matches the oracle
    b = wl.random_churn_batch(g, 5, 10, 10, rng)
    st, info = O.grest_step(st, b, ocfg)
    tr.update(b)
    U.compare(tr, st, info, O.OP_ADJ, 4, "after invalid")
    tr.close()


def test_degenerate_batches(cuda):
    rng = np.random.default_rng(51)
    g, _ = wl.sbm_graph(400, 2, 0.08, 0.02, 51)
    gb = g.copy()
    tr, st, ocfg = U.make_pair(g, 5, O.OP_ADJ)
    e0 = np.zeros(0, np.int32)
    # empty batch: exact pairs stay exact
    b = wl.Batch(0, e0, e0, e0, e0)
    st, info = O.grest_step(st, b, ocfg)
    tr.update(b)
    U.compare(tr, st, info, O.OP_ADJ, 5, "empty")
    # only deletions
    du, dv = wl.split_keys(rng.choice(gb.keys, 20, replace=False))
    b = wl.Batch(0, e0, e0, du, dv)
    gb.apply(b)
    st, info = O.grest_step(st, b, ocfg)
    tr.update(b)
    U.compare(tr, st, info, O.OP_ADJ, 5, "deletions only")
    # isolated new nodes next to connected ones
    b = wl.Batch(4, np.array([400, 401], np.int32), np.array([3, 400], np.int32), e0, e0)
    gb.apply(b)
    st, info = O.grest_step(st, b, ocfg)
    tr.update(b)
    U.compare(tr, st, info, O.OP_ADJ, 5, "isolated new nodes")
    tr.close()


def test_chung_lu_200k_nlap_steps(cuda):
    """Full-size normalized-Laplacian workload (n = 200,000, gamma 2.5, mean
    degree 16, K = 16, +0.5% nodes by preferential attachment, -0.1% edges):
    three consecutive RSVD steps, each against the oracle."""
    g0, batches = wl.chung_lu_stream(200_000, 2.5, 16, 3, 0.005, 8, 0.001, seed=20260305, lcc=True)
    tr, st, ocfg = U.make_pair(g0, 16, O.OP_NLAP, dense_limit=0)
    for t, b in enumerate(batches):
        st, info = O.grest_step(st, b, ocfg)
        s = tr.update(b)
        assert s["mode"] == 4 and s["m"] == info.m, t
        U.compare(tr, st, info, O.OP_NLAP, 16, f"cl200k step {t}")
    tr.close()


def test_gram_entry_point(cuda):
    """grest_gram: C = X^T Y against a plain float64 product, several tile
    shapes, row counts that leave a ragged final chunk."""
    torch = cuda
    g, _ = wl.sbm_graph(200, 2, 0.1, 0.02, 61)
    rp, col, _ = g.csr()
    tr = G.Tracker(g.n, rp, col, None, np.linalg.qr(np.random.default_rng(0).standard_normal((200, 4)))[0],
                   np.ones(4), 4)
    rng = np.random.default_rng(62)
    for n, a, b in ((1, 1, 1), (1000, 7, 9), (100_003, 64, 65), (50_001, 200, 132), (3000, 256, 256)):
        X = rng.standard_normal((n, a))
        Y = rng.standard_normal((n, b))
        Xd = torch.tensor(X, device="cuda")
        Yd = torch.tensor(Y, device="cuda")
        Cd = torch.empty((a, b), dtype=torch.float64, device="cuda")
        tr.gram(Xd, Yd, Cd)
        ref = X.T @ Y
        assert np.abs(Cd.cpu().numpy() - ref).max() <= 1e-12 * max(1.0, np.abs(X).max() * np.abs(Y).max() * n)
    tr.close()


def test_gram_f32_tensor_core_entry_point(cuda):
    """grest_gram_f32 against a float64 product of the same FP32 inputs; the
    bound is relative to |X|^T |Y| (the scale of the accumulated terms).
    Products with a side of at most 32 columns take the narrow CUDA-core
    kernel (FP32 FMAs, 256-row FP32 spans into double-float, FP64 partials;
    a right-narrow product computed transposed), the others the tensor-core
    kernel (tcgen05, 3xTF32, FP32 accumulation over <= 256 rows, FP64
    partial sums).  Includes ragged row counts, widths 1..256 and a
    misaligned view that must fall back to the generic CUDA-core kernel."""
    torch = cuda
    g, _ = wl.sbm_graph(200, 2, 0.1, 0.02, 71)
    rp, col, _ = g.csr()
    tr = G.Tracker(g.n, rp, col, None, np.linalg.qr(np.random.default_rng(0).standard_normal((200, 4)))[0],
                   np.ones(4), 4)
    rng = np.random.default_rng(72)
    cases = [(1, 1, 1), (33, 7, 9), (100_003, 32, 200), (250_001, 232, 232), (70_000, 200, 32), (4097, 256, 256),
             (65_536, 132, 164), (1000, 129, 17), (300_001, 32, 256), (50_017, 20, 37), (80_000, 232, 31),
             (40_000, 32, 32), (257, 3, 250)]
    for n, a, b in cases:
        X = torch.tensor(rng.standard_normal((n, a)), dtype=torch.float32, device="cuda")
        Y = torch.tensor(rng.standard_normal((n, b)), dtype=torch.float32, device="cuda")
        C = torch.empty((a, b), dtype=torch.float64, device="cuda")
        tr.gram_f32(X, Y, C)
        Xh, Yh = X.double().cpu().numpy(), Y.double().cpu().numpy()
        ref = Xh.T @ Yh
        bound = np.abs(Xh).T @ np.abs(Yh)
        err = np.abs(C.cpu().numpy() - ref)
        assert np.all(err <= 2e-6 * bound + 1e-30), (n, a, b, float((err / np.maximum(bound, 1e-30)).max()))
    # X = Y (the CholQR Grams): only the upper tiles are computed and mirrored.
    # The diagonal sums have terms of one sign, so the FP32 accumulation over a
    # 256-row span reaches its worst-case bound 256 * 2^-24 ~ 1.5e-5 of the sum
    # of magnitudes (independent random signs above stay within 2e-6)
    for n, a in ((100_003, 200), (70_001, 100), (4097, 256), (33, 40)):
        X = torch.tensor(rng.standard_normal((n, a)), dtype=torch.float32, device="cuda")
        C = torch.empty((a, a), dtype=torch.float64, device="cuda")
        tr.gram_f32(X, X, C)
        Xh = X.double().cpu().numpy()
        err = np.abs(C.cpu().numpy() - Xh.T @ Xh)
        bound = np.abs(Xh).T @ np.abs(Xh)
        assert np.all(err <= (256 * 2.0 ** -24 + 2e-7) * bound + 1e-30), (n, a)
        off = ~np.eye(a, dtype=bool)
        assert np.all(err[off] <= 2e-6 * bound[off] + 1e-30), (n, a)
    # misaligned base pointer (column offset 1): CUDA-core fallback, same rule
    Z = torch.tensor(rng.standard_normal((5000, 40)), dtype=torch.float32, device="cuda")
    X, Y = Z[:, 1:33], Z[:, 3:40]
    C = torch.empty((32, 37), dtype=torch.float64, device="cuda")
    tr.gram_f32(X, Y, C)
    Xh, Yh = X.double().cpu().numpy(), Y.double().cpu().numpy()
    err = np.abs(C.cpu().numpy() - Xh.T @ Yh)
    assert np.all(err <= 2e-6 * (np.abs(Xh).T @ np.abs(Yh)))
    tr.close()


def test_gemm_f32_tensor_core_entry_point(cuda):
    """grest_gemm_f32 (tcgen05, 3xTF32, FP32 accumulation over the a columns)
    against a float64 product of the same FP32 inputs: |Out - ref| <=
    4e-6 (|X| |alpha B|) + 2^-23 |beta Cin| elementwise.  Covers resident
    (a <= 64) and streamed B^T images, ragged row tails, a < 32, c up to 256,
    beta 0 and not, in-place updates (Cin = Out), and a misaligned view that
    must fall back to the CUDA-core kernel."""
    torch = cuda
    g, _ = wl.sbm_graph(200, 2, 0.1, 0.02, 71)
    rp, col, _ = g.csr()
    tr = G.Tracker(g.n, rp, col, None, np.linalg.qr(np.random.default_rng(0).standard_normal((200, 4)))[0],
                   np.ones(4), 4)
    rng = np.random.default_rng(73)
    cases = [(1, 1, 1, 1.0, 0.0), (129, 7, 9, -1.0, 1.0), (100_003, 32, 200, -1.0, 1.0), (250_001, 200, 200, 1.0, 0.0),
             (70_000, 200, 100, 1.0, 0.0), (4097, 256, 256, 0.5, 0.0), (65_536, 132, 132, 1.0, 0.0),
             (77_777, 164, 32, 1.0, 0.0), (1000, 33, 129, 2.0, -0.5), (40_000, 384, 64, 1.0, 0.0),
             (250_000, 32, 256, 1.0, 0.0), (60_001, 32, 32, -1.0, 1.0), (9_999, 20, 37, 0.5, 2.0), (513, 3, 255, 1.0, 1.0)]
    for n, a, c, alpha, beta in cases:
        X = torch.tensor(rng.standard_normal((n, a)), dtype=torch.float32, device="cuda")
        B = torch.tensor(rng.standard_normal((a, c)), dtype=torch.float64, device="cuda")
        Cin = torch.tensor(rng.standard_normal((n, c)), dtype=torch.float32, device="cuda") if beta else None
        Out = torch.empty((n, c), dtype=torch.float32, device="cuda")
        tr.gemm_f32(X, B, Out, alpha, beta, Cin)
        Xh, Bh = X.double().cpu().numpy(), B.cpu().numpy()
        ref = alpha * (Xh @ Bh)
        bound = 4e-6 * (np.abs(Xh) @ np.abs(alpha * Bh))
        if beta:
            Ch = Cin.double().cpu().numpy()
            ref += beta * Ch
            bound += 2.0 ** -23 * np.abs(beta * Ch)
        err = np.abs(Out.double().cpu().numpy() - ref)
        assert np.all(err <= bound + 1e-30), (n, a, c, float((err / np.maximum(bound, 1e-30)).max()))
    # in place: Out = Out - X B (narrow and tensor-core kernels)
    for n, a, c in ((30_001, 32, 132), (20_011, 48, 200)):
        X = torch.tensor(rng.standard_normal((n, a)), dtype=torch.float32, device="cuda")
        B = torch.tensor(rng.standard_normal((a, c)), dtype=torch.float64, device="cuda")
        W = torch.tensor(rng.standard_normal((n, c)), dtype=torch.float32, device="cuda")
        W0 = W.double().cpu().numpy()
        tr.gemm_f32(X, B, W, -1.0, 1.0, W)
        Xh, Bh = X.double().cpu().numpy(), B.cpu().numpy()
        err = np.abs(W.double().cpu().numpy() - (W0 - Xh @ Bh))
        assert np.all(err <= 4e-6 * (np.abs(Xh) @ np.abs(Bh)) + 2.0 ** -23 * np.abs(W0)), (n, a, c)
    # misaligned X (column offset 1): CUDA-core fallback, same bound
    Z = torch.tensor(rng.standard_normal((5000, 40)), dtype=torch.float32, device="cuda")
    X = Z[:, 1:33]
    B = torch.tensor(rng.standard_normal((32, 20)), dtype=torch.float64, device="cuda")
    Out = torch.empty((5000, 20), dtype=torch.float32, device="cuda")
    tr.gemm_f32(X, B, Out)
    Xh, Bh = X.double().cpu().numpy(), B.cpu().numpy()
    err = np.abs(Out.double().cpu().numpy() - Xh @ Bh)
    assert np.all(err <= 4e-6 * (np.abs(Xh) @ np.abs(Bh)))
    tr.close()
