"""GPU tests of the grouped update (grest_group_*): many small graphs updated
by one launch per stage, the update captured as a CUDA graph and its launch
shapes autotuned.

  * every graph matches the FP64 CPU oracle (Alg. 2) after every round, with
    exact new-node blocks (S <= L + P) and RSVD blocks (S > L + P) in the
    same group, at the FP64 tolerances of the single-graph tests;
  * a graph's result does not depend on the group: the same updates applied
    to each graph alone in a group of one give bit-identical pairs, and the
    autotuned launch shapes change nothing either;
  * the update is captured as a CUDA graph (after the first update, which
    also runs the autotuner) and later updates replay it;
  * an invalid batch fails alone and leaves its graph unchanged."""
import numpy as np
import pytest

import oracle as O
from paper_2603_19439_gb300 import grest as G
from paper_2603_19439_gb300 import workloads as wl
from tests import gpu_util as U

pytestmark = pytest.mark.gpu

K, L, P = 6, 8, 4


@pytest.fixture(scope="module", autouse=True)
def cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_19439_gb300.build import build
    build()
    torch.cuda.set_device(0)
    return torch


def make_graphs(count, seed, op=O.OP_ADJ):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(rng.integers(300, 2500))
        if i % 2:
            g = wl.chung_lu_graph(n, 2.4, 10, seed + i)
        else:
            g = wl.sbm_graph(n, int(rng.integers(2, 5)), 20.0 / n, 2.0 / n, seed + i)[0]
        out.append(g)
    return out


def streams(graphs, rounds, seed):
    """Per graph: batches of new nodes (some graphs fewer than L + P = 12 new
    nodes per round, so the exact block; others more, so RSVD), insertions
    and deletions."""
    rng = np.random.default_rng(seed)
    copies = [g.copy() for g in graphs]
    out = [[] for _ in graphs]
    for t in range(rounds):
        for i, gb in enumerate(copies):
            S = 5 if i % 3 == 0 else 20
            b = wl.random_churn_batch(gb, S, 25, 15, rng)
            gb.apply(b)
            out[i].append(b)
    return out


def checkpoints(graphs, op):
    states, blobs = [], []
    for g in graphs:
        rp, col, val = g.csr()
        st = O.init_state(g.n, rp, col, val, K, op)
        tr = G.Tracker(g.n, rp, col, val, st.X, st.lam, K, op=op, L=L, P=P, seed=11)
        blobs.append(tr.checkpoint())
        tr.close()
        states.append(st)
    return states, blobs


def oracle_compare(grp, i, st, info, op, where):
    Ug, thg = grp.embedding(i)
    ritz = grp.ritz_values(i)
    scale = abs(st.lam[0])
    assert ritz.size == info.m, f"{where}: m {ritz.size} vs {info.m}"
    assert np.max(np.abs(ritz - info.ritz_all)) <= 1e-10 * scale, f"{where}: ritz"
    assert np.max(np.abs(thg - st.lam)) <= 1e-10 * scale, f"{where}: theta"
    j = U.cluster_cut(info.ritz_all, op, K)
    assert U.sin_angle(st.X[:, :j], Ug[:, :j]) <= 1e-8, f"{where}: angle"
    assert np.abs(Ug.T @ Ug - np.eye(K)).max() < 1e-12, where


@pytest.mark.parametrize("op", [O.OP_ADJ, O.OP_NLAP])
def test_group_matches_oracle_every_round(op):
    graphs = make_graphs(6, 900 + op, op)
    sts, blobs = checkpoints(graphs, op)
    grp = G.Group(blobs)
    batches = streams(graphs, 3, 5)
    cfg = O.Config(k=K, op=op, L=L, P=P, seed=11)
    modes = set()
    for t in range(3):
        codes, stats = grp.update([batches[i][t] for i in range(len(graphs))])
        assert codes == [0] * len(graphs), codes
        for i in range(len(graphs)):
            sts[i], info = O.grest_step(sts[i], batches[i][t], cfg)
            assert stats[i]["m"] == info.m
            modes.add(stats[i]["mode"])
            oracle_compare(grp, i, sts[i], info, op, f"graph {i} round {t}")
    assert modes == {3, 4}  # both new-node blocks ran in one group
    grp.close()


def test_group_result_does_not_depend_on_the_group():
    graphs = make_graphs(5, 950)
    _, blobs = checkpoints(graphs, O.OP_ADJ)
    batches = streams(graphs, 3, 6)
    big = G.Group(blobs)
    alone = [G.Group([b]) for b in blobs]
    for t in range(3):
        codes, stats = big.update([batches[i][t] for i in range(len(graphs))])
        assert codes == [0] * len(graphs)
        info = big.info()
        if t == 0:
            assert info["tuned"] == 1 and info["launches_per_update"] > 40
        else:
            assert info["captured"] == 1  # the update replays a CUDA graph
        for i, a in enumerate(alone):
            c, _ = a.update([batches[i][t]])
            assert c == [0]
    for i, a in enumerate(alone):
        U1, th1 = big.embedding(i)
        U2, th2 = a.embedding(0)
        assert np.array_equal(U1, U2) and np.array_equal(th1, th2), i
        a.close()
    big.close()


def test_group_invalid_batch_fails_alone():
    graphs = make_graphs(4, 970)
    sts, blobs = checkpoints(graphs, O.OP_ADJ)
    grp = G.Group(blobs)
    batches = [s[0] for s in streams(graphs, 1, 7)]
    bad = batches[2]
    u0, v0 = wl.split_keys(graphs[2].keys[:1])  # insert an edge that exists
    bad.ins_u = np.concatenate([bad.ins_u, u0.astype(np.int32)])
    bad.ins_v = np.concatenate([bad.ins_v, v0.astype(np.int32)])
    U_before, th_before = grp.embedding(2)
    codes, _ = grp.update(batches)
    assert codes[2] == 2 and all(codes[i] == 0 for i in (0, 1, 3))
    U_after, th_after = grp.embedding(2)
    assert np.array_equal(U_before, U_after) and np.array_equal(th_before, th_after)
    cfg = O.Config(k=K, L=L, P=P, seed=11)
    for i in (0, 1, 3):
        st, info = O.grest_step(sts[i], batches[i], cfg)
        oracle_compare(grp, i, st, info, O.OP_ADJ, f"graph {i}")
    grp.close()
