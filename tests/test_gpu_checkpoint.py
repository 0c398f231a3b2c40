"""GPU tests of checkpoint / restore (grest_checkpoint, grest_restore) and of
the serving loop's eviction of idle graphs to host memory.  A restored
context must continue bit-identically: the same later updates give the same
(X_K, Lambda_K, live) as on the original context, including RSVD steps
(whose test matrix is seeded by the step counter), node removal (live mask)
and weighted Laplacians (degrees kept by the updates)."""
import numpy as np
import pytest

import oracle as O
from paper_2603_19439_gb300 import grest as G
from paper_2603_19439_gb300 import workloads as wl

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


def first_diff(a, b):
    if len(a) != len(b):
        return f"lengths {len(a)} and {len(b)}"
    d = np.flatnonzero(np.frombuffer(a, np.uint8) != np.frombuffer(b, np.uint8))
    return f"{d.size} bytes differ, the first at offset {d[0]} of {len(a)}" if d.size else "equal"


def same(tr_a, tr_b, where):
    Ua, tha, la = tr_a.embedding()
    Ub, thb, lb = tr_b.embedding()
    assert np.array_equal(Ua, Ub) and np.array_equal(tha, thb) and np.array_equal(la, lb), where


def stream_batches(g, steps, rng, weighted=False):
    out = []
    gb = g.copy()
    for t in range(steps):
        # alternate an RSVD-sized growth step (S > L + P) and a churn step with node removal
        if t % 2 == 0:
            b = wl.random_churn_batch(gb, 90, 60, 40, rng)
        else:
            b = wl.random_churn_batch(gb, 5, 40, 30, rng, n_del_nodes=3)
        if weighted:
            b.ins_w = rng.uniform(0.5, 2.0, size=b.n_ins)
        gb.apply(b)
        out.append(b)
    return out


@pytest.mark.parametrize("precision,op,weighted", [(G.FP64, O.OP_ADJ, False), (G.MIXED, O.OP_LAP, True),
                                                   (G.FP64, O.OP_NLAP, False)])
def test_restore_continues_bit_identically(cuda, precision, op, weighted):
    torch = cuda
    rng = np.random.default_rng(41)
    g = wl.chung_lu_graph(6000, 2.4, 10, 17)
    if weighted:
        g.w = rng.uniform(0.5, 2.0, size=g.n_edges)
    k = 8
    rp, col, val = g.csr()
    st = O.init_state(g.n, rp, col, val, k, op)
    kw = dict(op=op, L=30, P=30, seed=5)
    if precision == G.MIXED:
        kw.update(precision=G.MIXED, drop_tol=1e-3)
    s_a = torch.cuda.Stream()
    tr = G.Tracker(g.n, rp, col, val, st.X, st.lam, k, stream=s_a.cuda_stream, **kw)
    batches = stream_batches(g, 6, rng, weighted)
    for b in batches[:3]:
        tr.update(b)
    blob = tr.checkpoint()
    # the host reader sees what the context holds
    U0, th0, live0 = tr.embedding()
    Uc, thc, livec = G.checkpoint_embedding(blob)
    assert np.array_equal(U0, Uc) and np.array_equal(th0, thc) and np.array_equal(live0, livec)
    assert not livec.all()  # a removal step ran
    s_b = torch.cuda.Stream()
    tr2 = G.Tracker.restore(blob, stream=s_b.cuda_stream)
    same(tr, tr2, "right after restore")
    # the checkpoint is a function of the state: taken again, and taken from
    # the restored context (whose slack layout differs), it is the same bytes
    again = tr.checkpoint()
    assert again == blob, first_diff(again, blob)
    restored = tr2.checkpoint()
    assert restored == blob, first_diff(restored, blob)
    assert tr2.stats()["step"] == 3
    for t, b in enumerate(batches[3:]):
        sa = tr.update(b)
        sb = tr2.update(b)
        assert sa["step"] == sb["step"] == 4 + t
        assert sa["mode"] == sb["mode"] and sa["m"] == sb["m"]
        same(tr, tr2, f"step {4 + t}")
    # a truncated checkpoint is refused
    with pytest.raises(G.GrestError):
        G.Tracker.restore(blob[:-8])
    tr.close()
    tr2.close()


def test_checkpoint_size_query_and_small_buffer(cuda):
    import ctypes
    g = wl.sbm_graph(1500, 3, 0.03, 0.002, 9)[0]
    k = 6
    rp, col, val = g.csr()
    st = O.init_state(g.n, rp, col, val, k, O.OP_ADJ)
    tr = G.Tracker(g.n, rp, col, val, st.X, st.lam, k)
    nb = ctypes.c_int64()
    assert tr.lib.grest_checkpoint(tr.h, None, ctypes.byref(nb)) == 0
    need = nb.value
    # header + rowptr + col + degrees + U + theta + live, at least
    assert need >= 8 * (g.n + 1) + 4 * rp[-1] + 8 * g.n + 8 * g.n * k + 8 * k + g.n
    buf = (ctypes.c_uint8 * need)()
    nb.value = need - 1
    assert tr.lib.grest_checkpoint(tr.h, buf, ctypes.byref(nb)) == 4  # GREST_ERR_CAPACITY
    assert nb.value == need
    tr.close()


def test_server_eviction_keeps_results(cuda):
    """Budget for about two of four graphs, eviction on: requests for all
    four run (idle graphs are checkpointed to host memory and restored), and
    every graph's result equals its updates applied alone in order."""
    k = 8
    rng = np.random.default_rng(23)
    items = []
    for i in range(4):
        g = wl.chung_lu_graph(int(rng.integers(2500, 4000)), 2.3, 8, 300 + i)
        items.append((g, O.init_state(g.n, *g.csr(), k, O.OP_ADJ)))
    probe = G.Tracker(items[0][0].n, *items[0][0].csr(), items[0][1].X, items[0][1].lam, k)
    nbytes = probe.device_bytes()
    probe.close()
    rounds = []
    copies = [g.copy() for g, _ in items]
    for _ in range(3):
        r = []
        for gb in copies:
            b = wl.random_churn_batch(gb, 6, 25, 15, rng)
            gb.apply(b)
            r.append(b)
        rounds.append(r)
    sv = G.Server(n_workers=3, hbm_budget=int(2.2 * nbytes))
    sv.set_eviction(True)
    gids = [sv.add_graph(g.n, *g.csr(), k, U0=st.X, theta0=st.lam) for g, st in items]
    for t in range(3):
        tickets = [sv.submit(gid, rounds[t][i]) for i, gid in enumerate(gids)]
        for tk in tickets:
            code, _, _, _ = sv.wait(tk)
            assert code == 0
        used, nres = sv.resident()
        assert nres <= 3
    adm, ev, rs = sv.counters()
    assert ev >= 1 and rs >= 1 and adm >= 4
    for i, (g, st) in enumerate(items):
        tr = G.Tracker(g.n, *g.csr(), st.X, st.lam, k)
        for t in range(3):
            tr.update(rounds[t][i])
        Ua, tha, la = tr.embedding()
        Ub, thb, lb = sv.embedding(gids[i])  # from the context, or from the checkpoint when evicted
        assert np.array_equal(Ua, Ub) and np.array_equal(tha, thb) and np.array_equal(la, lb), i
        tr.close()
    sv.close()
