"""GPU parity of the paper's own formulations against the FP64 oracle: the W
block P_perp (Delta X_bar) of Sec. 3.3 (w_block = DELTA) and the low-rank
projection of Eq. main3 (projection = LOWRANK, Alg. 2 as printed), with
Delta = M_new - M_old for the adjacency and the shifted Laplacian.  Same
tolerances as the EXACT parity tests (tests/gpu_util.py)."""
import numpy as np
import pytest

import oracle as O
from paper_2603_19439_gb300 import grest as G
from paper_2603_19439_gb300 import workloads as wl
from tests import gpu_util as U
from tests.test_gpu_parity import hub_graph

pytestmark = pytest.mark.gpu

MODES = [(G.PROJ_EXACT, G.WB_DELTA), (G.PROJ_LOWRANK, G.WB_RESID), (G.PROJ_LOWRANK, G.WB_DELTA)]


@pytest.fixture(scope="module", autouse=True)
def cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_19439_gb300.build import build
    build()
    torch.cuda.set_device(0)
    return torch


@pytest.mark.parametrize("op", [O.OP_ADJ, O.OP_LAP])
@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("weighted", [False, True])
def test_modes_churn_stream(cuda, op, mode, weighted):
    """New nodes, inserts and deletions (old weights of deleted edges enter
    Delta), a hub row longer than the long-row cut, three steps."""
    proj, wb = mode
    rng = np.random.default_rng(51 + op)
    g = hub_graph(900, 51, weighted)
    gb = g.copy()
    tr, st, ocfg = U.make_pair(g, 5, op, subspace=G.SUB_GREST3, projection=proj, w_block=wb)
    ocfg.projection, ocfg.w_block = proj, wb
    for t in range(3):
        b = wl.random_churn_batch(gb, 8, 25, 15, rng)
        if weighted:
            b.ins_w = rng.uniform(0.5, 2.0, size=b.n_ins)
        gb.apply(b)
        st, info = O.grest_step(st, b, ocfg, weighted=weighted)
        tr.update(b)
        U.compare(tr, st, info, op, 5, f"op {op} mode {mode} weighted {weighted} step {t}")
    tr.close()


def test_lowrank_delta_rsvd_stream(cuda):
    """Eq. main3 with the RSVD new-node basis (S > L + P); the sketch reads the
    new rows of Delta X_bar, which equal those of M_new X_bar."""
    g0, batches = wl.chung_lu_stream(3000, 2.5, 10, 3, 0.02, 5, 0.002, seed=13, lcc=True)
    tr, st, ocfg = U.make_pair(g0, 6, O.OP_ADJ, L=20, P=12, seed=9, projection=G.PROJ_LOWRANK,
                               w_block=G.WB_DELTA)
    ocfg.projection, ocfg.w_block = G.PROJ_LOWRANK, G.WB_DELTA
    for t, b in enumerate(batches):
        st, info = O.grest_step(st, b, ocfg)
        s = tr.update(b)
        assert s["mode"] == 4 and s["m"] == info.m
        U.compare(tr, st, info, O.OP_ADJ, 6, f"lowrank rsvd step {t}")
    tr.close()


def test_mixed_delta_block(cuda):
    """Mixed precision with the paper's W block (the FP64 refinement uses M_new)."""
    from tests.test_gpu_mixed import compare_mixed
    g0, batches = wl.sbm_stream(n0=800, steps=3, n_new=20, n_rand=80)
    tr, st, ocfg = U.make_pair(g0, 6, O.OP_ADJ, precision=G.MIXED, drop_tol=1e-3, w_block=G.WB_DELTA)
    ocfg.drop_tol, ocfg.w_block = 1e-3, G.WB_DELTA
    for t, b in enumerate(batches):
        st, info = O.grest_step(st, b, ocfg)
        s = tr.update(b)
        assert s["m"] == info.m
        compare_mixed(tr, st, info, O.OP_ADJ, 6, f"mixed delta step {t}")
    tr.close()


def test_node_removal_unsupported_in_delta_modes(cuda):
    rng = np.random.default_rng(61)
    g, _ = wl.sbm_graph(400, 2, 0.08, 0.02, 61)
    tr, st, ocfg = U.make_pair(g, 4, O.OP_ADJ, projection=G.PROJ_LOWRANK)
    U0, th0, _ = tr.embedding()
    b = wl.random_churn_batch(g.copy(), 0, 5, 5, rng, n_del_nodes=2)
    with pytest.raises(G.GrestError) as e:
        tr.update(b)
    assert e.value.code == 8
    U1, th1, _ = tr.embedding()
    assert np.array_equal(U0, U1) and np.array_equal(th0, th1)
    tr.close()
