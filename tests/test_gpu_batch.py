"""GPU tests of batched updates (grest_batch_apply_updates): many independent
graphs, one update each per call, their contexts stepped concurrently by the
library's host threads on their own streams.  Each graph's result must be
bit-identical to updating it alone, match the oracle, and a failing member
must not disturb the others."""
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


def small_graphs(count, seed):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(np.exp(rng.uniform(np.log(600), np.log(5000))))
        if i % 2 == 0:
            R = int(rng.integers(2, 7))
            g, _ = wl.sbm_graph(n, R, min(0.5, 12.0 * R / n), min(0.5, 1.2 / n), seed + i)
        else:
            g = wl.chung_lu_graph(n, 2.3, 8, seed + i)
        out.append(g)
    return out


def make_trackers(graphs, states, k, torch, streams):
    trs = []
    for g, st, s in zip(graphs, states, streams):
        rp, col, val = g.csr()
        trs.append(G.Tracker(g.n, rp, col, val, st.X, st.lam, k, stream=s.cuda_stream))
    return trs


def test_batch_equals_alone_and_oracle(cuda):
    torch = cuda
    k = 8
    graphs = small_graphs(10, 300)
    states = [O.init_state(g.n, *g.csr(), k, O.OP_ADJ) for g in graphs]
    cfg = O.Config(k=k, op=O.OP_ADJ, subspace=G.SUB_AUTO, L=100, P=100, seed=0, drop_tol=1e-7)
    streams_a = [torch.cuda.Stream() for _ in graphs]
    streams_b = [torch.cuda.Stream() for _ in graphs]
    alone = make_trackers(graphs, states, k, torch, streams_a)
    mixed = make_trackers(graphs, states, k, torch, streams_b)
    batch = G.Batch(mixed, n_threads=4)
    rng = np.random.default_rng(9)
    gbs = [g.copy() for g in graphs]
    for t in range(3):
        ups = []
        for gb in gbs:
            b = wl.random_churn_batch(gb, max(1, gb.n // 100), 40, 30, rng)
            gb.apply(b)
            ups.append(b)
        for tr, b in zip(alone, ups):
            tr.update(b)
        codes, stats = batch.update(ups)
        assert codes == [0] * len(graphs)
        for i, (ta, tb) in enumerate(zip(alone, mixed)):
            Ua, tha, la = ta.embedding()
            Ub, thb, lb = tb.embedding()
            assert np.array_equal(Ua, Ub) and np.array_equal(tha, thb) and np.array_equal(la, lb), (t, i)
        # two members against the oracle
        for i in (0, 1):
            states[i], info = O.grest_step(states[i], ups[i], cfg)
            U.compare(mixed[i], states[i], info, O.OP_ADJ, k, f"graph {i} step {t}")
        for i in range(2, len(graphs)):
            states[i], _ = O.grest_step(states[i], ups[i], cfg)
    batch.close()
    for tr in alone + mixed:
        tr.close()


def test_batch_failing_member_leaves_others_updated(cuda):
    torch = cuda
    k = 8
    graphs = small_graphs(6, 400)
    states = [O.init_state(g.n, *g.csr(), k, O.OP_ADJ) for g in graphs]
    streams = [torch.cuda.Stream() for _ in graphs]
    trs = make_trackers(graphs, states, k, torch, streams)
    ref = make_trackers(graphs, states, k, torch, [torch.cuda.Stream() for _ in graphs])
    batch = G.Batch(trs, n_threads=3)
    rng = np.random.default_rng(11)
    ups = [wl.random_churn_batch(g, 5, 20, 10, rng) for g in graphs]
    # member 2 inserts an edge that already exists: an invalid update
    g2 = graphs[2]
    u0, v0 = wl.split_keys(g2.keys[:1])
    bad = ups[2]
    bad.ins_u = np.concatenate([bad.ins_u, u0.astype(np.int32)])
    bad.ins_v = np.concatenate([bad.ins_v, v0.astype(np.int32)])
    U2_before, th2_before, _ = trs[2].embedding()
    with pytest.raises(G.GrestError):
        batch.update(ups)
    # the valid members were updated: each equals the same update applied alone
    for i, (tr, rf) in enumerate(zip(trs, ref)):
        if i == 2:
            U2, th2, _ = tr.embedding()
            assert np.array_equal(U2, U2_before) and np.array_equal(th2, th2_before)
            continue
        rf.update(ups[i])
        Ua, tha, _ = rf.embedding()
        Ub, thb, _ = tr.embedding()
        assert np.array_equal(Ua, Ub) and np.array_equal(tha, thb), i
    batch.close()
    for tr in trs + ref:
        tr.close()


def test_batch_mixed_precision_equals_alone(cuda):
    """Mixed-precision contexts of different sizes stepped concurrently (their
    tensor-core kernels reserve different amounts of shared memory from
    several host threads at once): each result equals the update alone."""
    torch = cuda
    k = 8
    graphs = small_graphs(12, 700)
    states = [O.init_state(g.n, *g.csr(), k, O.OP_ADJ) for g in graphs]
    kw = dict(precision=G.MIXED, drop_tol=1e-3, L=20, P=20)
    alone, mixed = [], []
    for g, st in zip(graphs, states):
        rp, col, val = g.csr()
        alone.append(G.Tracker(g.n, rp, col, val, st.X, st.lam, k, stream=torch.cuda.Stream().cuda_stream, **kw))
        mixed.append(G.Tracker(g.n, rp, col, val, st.X, st.lam, k, stream=torch.cuda.Stream().cuda_stream, **kw))
    batch = G.Batch(mixed, n_threads=12)
    rng = np.random.default_rng(13)
    gbs = [g.copy() for g in graphs]
    for t in range(2):
        ups = []
        for gb in gbs:
            b = wl.random_churn_batch(gb, max(1, gb.n // 50), 60, 40, rng)
            gb.apply(b)
            ups.append(b)
        for tr, b in zip(alone, ups):
            tr.update(b)
        codes, _ = batch.update(ups)
        assert codes == [0] * len(graphs)
        for i, (ta, tb) in enumerate(zip(alone, mixed)):
            Ua, tha, _ = ta.embedding()
            Ub, thb, _ = tb.embedding()
            assert np.array_equal(Ua, Ub) and np.array_equal(tha, thb), (t, i)
    batch.close()
    for tr in alone + mixed:
        tr.close()
