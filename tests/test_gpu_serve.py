"""GPU tests of the serving loop (grest_server_*): requests for many resident
graphs arrive together and run concurrently on the library's workers; each
graph's result equals its updates applied alone in order; graphs are
admitted by a device-memory budget and memory returns on removal; an invalid
request fails alone."""
import time

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


def graphs_and_pairs(count, seed, k):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(rng.integers(800, 4000))
        g = wl.chung_lu_graph(n, 2.3, 8, seed + i) if i % 2 else wl.sbm_graph(n, 3, 24.0 / n, 1.0 / n, seed + i)[0]
        st = O.init_state(g.n, *g.csr(), k, O.OP_ADJ)
        out.append((g, st))
    return out


def test_server_results_equal_updates_alone():
    k = 8
    items = graphs_and_pairs(8, 500, k)
    rng = np.random.default_rng(3)
    rounds = []
    copies = [g.copy() for g, _ in items]
    for _ in range(3):
        r = []
        for gb in copies:
            b = wl.random_churn_batch(gb, 8, 30, 20, rng)
            gb.apply(b)
            r.append(b)
        rounds.append(r)
    sv = G.Server(n_workers=4)
    gids = [sv.add_graph(g.n, *g.csr(), k, U0=st.X, theta0=st.lam) for g, st in items]
    tickets = [[sv.submit(gid, rounds[t][i]) for i, gid in enumerate(gids)] for t in range(3)]
    for row in tickets:
        for tk in row:
            code, stats, wait_ms, run_ms = sv.wait(tk)
            assert code == 0 and run_ms > 0 and wait_ms >= 0
    for i, (g, st) in enumerate(items):
        tr = G.Tracker(g.n, *g.csr(), st.X, st.lam, k)
        for t in range(3):
            tr.update(rounds[t][i])
        Ua, tha, la = tr.embedding()
        Ub, thb, lb = sv.embedding(gids[i])
        assert np.array_equal(Ua, Ub) and np.array_equal(tha, thb) and np.array_equal(la, lb), i
        tr.close()
        # and every served result matches the FP64 oracle run on the same requests (Alg. 2 per request)
        so = st
        for t in range(3):
            so, info = O.grest_step(so, rounds[t][i], O.Config(k=k))
        oracle_close(Ub, thb, lb, so, info, k, f"graph {i}")
    sv.close()


def oracle_close(U, th, live, st, info, k, where, theta_tol=1e-10, angle_tol=1e-8):
    """FP64 parity of a served result with the oracle: tracked values within
    theta_tol |theta_1|, the tracked subspace (cut at separated clusters)
    within a sin angle of angle_tol."""
    from tests import gpu_util as U_
    scale = abs(st.lam[0])
    assert np.array_equal(live, st.live), where
    assert np.max(np.abs(th - st.lam)) <= theta_tol * scale, f"{where}: {np.max(np.abs(th - st.lam)) / scale:.2e}"
    j = U_.cluster_cut(info.ritz_all, O.OP_ADJ, k)
    ang = U_.sin_angle(st.X[:, :j], U[:, :j])
    assert ang <= angle_tol, f"{where}: sin angle {ang:.2e}"


def test_mixed_server_matches_oracle_under_admission():
    """The mixed-precision path served under a budget that holds two of four
    graphs at once (admission and eviction to host memory exercised): every
    request succeeds, each graph's result equals its updates applied alone,
    and matches the FP64 oracle within the mixed path's tolerances."""
    k = 8
    items = graphs_and_pairs(4, 700, k)
    rng = np.random.default_rng(11)
    copies = [g.copy() for g, _ in items]
    reqs = []
    for t in range(4):
        for i, gb in enumerate(copies):
            b = wl.random_churn_batch(gb, 6, 24, 12, rng)
            gb.apply(b)
            reqs.append((i, b))
    kw = dict(precision=G.MIXED, drop_tol=1e-3)
    probe = max(items, key=lambda it: it[0].n)
    pt = G.Tracker(probe[0].n, *probe[0].csr(), probe[1].X, probe[1].lam, k, **kw)
    nbytes = pt.device_bytes()
    pt.close()
    sv = G.Server(n_workers=3, hbm_budget=int(2.2 * nbytes))
    sv.set_eviction(True)
    gids = [sv.add_graph(g.n, *g.csr(), k, U0=st.X, theta0=st.lam, **kw) for g, st in items]
    # three rounds at once (two graphs fit; the others are admitted as graphs
    # go idle and are evicted), then a fourth round after all of them: it
    # restores the graphs evicted meanwhile
    first = [sv.submit(gids[i], b) for i, b in reqs[:12]]
    assert all(sv.wait(t)[0] == 0 for t in first)
    last = [sv.submit(gids[i], b) for i, b in reqs[12:]]
    assert all(sv.wait(t)[0] == 0 for t in last)
    adm, evc, rst = sv.counters()
    assert evc >= 2 and rst >= 1
    for i, (g, st) in enumerate(items):
        Ub, thb, lb = sv.embedding(gids[i])
        tr = G.Tracker(g.n, *g.csr(), st.X, st.lam, k, **kw)
        so = st
        ocfg = O.Config(k=k, drop_tol=1e-3)
        for j, b in reqs:
            if j == i:
                tr.update(b)
                so, info = O.grest_step(so, b, ocfg)
        Ua, tha, _ = tr.embedding()
        tr.close()
        assert np.array_equal(Ua, Ub) and np.array_equal(tha, thb), i
        scale = abs(so.lam[0])
        assert np.max(np.abs(thb - so.lam)) <= 1e-6 * scale, i
        M, _ = O.operator_matrix(so.A, so.live, O.OP_ADJ)
        rg = np.linalg.norm(M @ Ub - Ub * thb, axis=0)
        ro = np.linalg.norm(M @ so.X - so.X * so.lam, axis=0)
        assert np.max(np.abs(rg - ro)) <= 1e-6 * scale, i
    sv.close()


def test_server_admission_by_budget_and_removal():
    k = 8
    g = wl.chung_lu_graph(3000, 2.3, 8, 77)
    st = O.init_state(g.n, *g.csr(), k, O.OP_ADJ)
    probe = G.Tracker(g.n, *g.csr(), st.X, st.lam, k)
    nbytes = probe.device_bytes()
    probe.close()
    assert nbytes > 0
    sv = G.Server(n_workers=3, hbm_budget=int(2.5 * nbytes))
    gids = [sv.add_graph(g.n, *g.csr(), k, U0=st.X, theta0=st.lam) for _ in range(3)]
    rng = np.random.default_rng(5)
    b = wl.random_churn_batch(g, 5, 20, 10, rng)
    t = [sv.submit(gid, b) for gid in gids]
    # two graphs fit (which two is up to the workers); the third waits for memory
    deadline = time.time() + 60
    while sum(sv.done(x) for x in t) < 2 and time.time() < deadline:
        time.sleep(0.05)
    time.sleep(0.5)
    done = [sv.done(x) for x in t]
    assert sum(done) == 2
    waiting = done.index(False)
    first = done.index(True)
    other = 3 - waiting - first
    used, nres = sv.resident()
    assert nres == 2 and used <= int(2.5 * nbytes)
    sv.remove_graph(gids[first])
    code, _, wait_ms, _ = sv.wait(t[waiting])
    assert code == 0 and wait_ms >= 400
    used, nres = sv.resident()
    assert nres == 2 and used <= int(2.5 * nbytes)
    # all three saw the same update from the same start: identical results
    Ua, tha, _ = sv.embedding(gids[other])
    Ub, thb, _ = sv.embedding(gids[waiting])
    assert np.array_equal(Ua, Ub) and np.array_equal(tha, thb)
    with pytest.raises(G.GrestError):
        sv.submit(gids[first], b)  # removed
    sv.close()


def test_server_invalid_request_fails_alone():
    k = 8
    items = graphs_and_pairs(3, 600, k)
    sv = G.Server(n_workers=2)
    gids = [sv.add_graph(g.n, *g.csr(), k, U0=st.X, theta0=st.lam) for g, st in items]
    rng = np.random.default_rng(7)
    ups = [wl.random_churn_batch(g, 4, 12, 8, rng) for g, _ in items]
    bad = ups[1]
    u0, v0 = wl.split_keys(items[1][0].keys[:1])
    bad.ins_u = np.concatenate([bad.ins_u, u0.astype(np.int32)])
    bad.ins_v = np.concatenate([bad.ins_v, v0.astype(np.int32)])
    t = [sv.submit(gid, u) for gid, u in zip(gids, ups)]
    codes = [sv.wait(x)[0] for x in t]
    assert codes[0] == 0 and codes[2] == 0 and codes[1] != 0
    U1, th1, _ = sv.embedding(gids[1])
    assert np.array_equal(U1, items[1][1].X) and np.array_equal(th1, items[1][1].lam)
    sv.close()
