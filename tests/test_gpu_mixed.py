"""GPU parity of the mixed-precision paths against the FP64 CPU oracle on the
same seeded inputs: GREST_MIXED (FP32 blocks and tensor-core products, FP64
projected problems, FP64 refinement) and GREST_MIXED_FAST (the same with FP32
projected problems and a double-float refinement); every test runs both.

Tolerances (reading of the precision targets): tracked values within
1e-6 * |theta_1| of the oracle's; per pair, the residual ||M u - theta u||
of the mixed result differs from the oracle's by at most 1e-6 * ||M||
(||M|| ~ |theta_1|); tracked subspaces (split at clusters) within a sin angle
of 1e-4; the output is orthonormal to FP64 accuracy (1e-12) because the last
Rayleigh-Ritz pass runs in FP64; on the exactness fixture (the whole space is
spanned) the absolute residual is at most 1e-6 * ||M||."""
import numpy as np
import pytest

import oracle as O
from paper_2603_19439_gb300 import grest as G
from paper_2603_19439_gb300 import workloads as wl
from tests import gpu_util as U

pytestmark = pytest.mark.gpu
PRECISIONS = pytest.mark.parametrize("prec", [G.MIXED, G.MIXED_FAST], ids=["mixed", "mixed_fast"])

THETA_TOL = 1e-6
RES_TOL = 1e-6
ANGLE_TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_19439_gb300.build import build
    build()
    torch.cuda.set_device(0)
    return torch


def residuals(M, X, th):
    return np.linalg.norm(M @ X - X * th, axis=0)


def compare_mixed(tr, st, info, op, k, where):
    Ug, thg, live = tr.embedding()
    scale = abs(st.lam[0])
    assert np.array_equal(live, st.live), where
    assert np.max(np.abs(thg - st.lam)) <= THETA_TOL * scale, \
        f"{where}: theta err {np.max(np.abs(thg - st.lam)) / scale:.2e}"
    M, _ = O.operator_matrix(st.A, st.live, op)
    rg = residuals(M, Ug, thg)
    ro = residuals(M, st.X, st.lam)
    assert np.max(np.abs(rg - ro)) <= RES_TOL * scale, f"{where}: residual diff {np.max(np.abs(rg - ro)) / scale:.2e}"
    j = U.cluster_cut(info.ritz_all, op, k)
    ang = U.sin_angle(st.X[:, :j], Ug[:, :j])
    assert ang <= ANGLE_TOL, f"{where}: sin angle {ang:.2e}"
    assert np.abs(Ug.T @ Ug - np.eye(k)).max() < 1e-12, where
    return np.max(np.abs(rg - ro)) / scale


@PRECISIONS
def test_mixed_fig1_exact(cuda, prec):
    import json, os
    d = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "fig1_example.json")))
    edges = [(a - 1, b - 1) for a, b in d["edges_before"]]
    g = wl.EdgeSetGraph(6, wl.keys_of([e[0] for e in edges], [e[1] for e in edges]))
    for op in (O.OP_ADJ, O.OP_LAP, O.OP_NLAP):
        tr, st, ocfg = U.make_pair(g, 3, op, subspace=G.SUB_GREST3, precision=prec, drop_tol=1e-3)
        ocfg.drop_tol = 1e-3
        ins = np.array([(a - 1, b - 1) for a, b in d["added_edges_old"] + d["added_edges_new"]], np.int32)
        dels = np.array([(a - 1, b - 1) for a, b in d["deleted_edges"]], np.int32)
        b = wl.Batch(2, ins[:, 0].copy(), ins[:, 1].copy(), dels[:, 0].copy(), dels[:, 1].copy())
        st2, info = O.grest_step(st, b, ocfg)
        tr.update(b)
        compare_mixed(tr, st2, info, op, 3, f"fig1 op {op}")
        Ug, thg, _ = tr.embedding()
        M = O.dense_operator(st2.A, st2.live, op)
        if info.m == 8:  # exactness: absolute residual
            assert residuals(M, Ug, thg).max() <= RES_TOL * abs(thg[0])
        tr.close()


@PRECISIONS
def test_mixed_sbm_stream(cuda, prec):
    g0, batches = wl.sbm_stream()
    tr, st, ocfg = U.make_pair(g0, 8, O.OP_ADJ, precision=prec, drop_tol=1e-3)
    ocfg.drop_tol = 1e-3
    worst = 0.0
    for t, b in enumerate(batches):
        st, info = O.grest_step(st, b, ocfg)
        s = tr.update(b)
        assert s["m"] == info.m
        worst = max(worst, compare_mixed(tr, st, info, O.OP_ADJ, 8, f"mixed sbm step {t}"))
    tr.close()


@PRECISIONS
def test_mixed_rsvd_nlap_stream(cuda, prec):
    g0, batches = wl.chung_lu_stream(4000, 2.5, 12, 3, 0.02, 6, 0.002, seed=11, lcc=True)
    tr, st, ocfg = U.make_pair(g0, 8, O.OP_NLAP, L=20, P=12, seed=5, precision=prec, drop_tol=1e-3)
    ocfg.drop_tol = 1e-3
    for t, b in enumerate(batches):
        st, info = O.grest_step(st, b, ocfg)
        s = tr.update(b)
        assert s["mode"] == 4 and s["m"] == info.m
        compare_mixed(tr, st, info, O.OP_NLAP, 8, f"mixed rsvd step {t}")
    tr.close()


@PRECISIONS
def test_mixed_check_flag_reports_fp64_residuals(cuda, prec):
    """GREST_FLAG_CHECK: orthonormality and Galerkin residual of the refined
    pairs are at FP64 level; the max residual matches the one computed here."""
    g0, batches = wl.sbm_stream(n0=600, steps=2, n_new=20, n_rand=60)
    tr, st, ocfg = U.make_pair(g0, 6, O.OP_ADJ, precision=prec, drop_tol=1e-3, flags=G.FLAG_CHECK)
    ocfg.drop_tol = 1e-3
    for b in batches:
        st, info = O.grest_step(st, b, ocfg)
        s = tr.update(b)
    assert s["orth_err"] < 1e-12 and s["galerkin"] < 1e-12
    Ug, thg, _ = tr.embedding()
    M, _ = O.operator_matrix(st.A, st.live, O.OP_ADJ)
    r = residuals(M, Ug, thg).max() / abs(thg[0])
    assert abs(s["max_residual"] - r) <= 1e-9
    tr.close()


@PRECISIONS
def test_mixed_more_than_32_pairs(cuda, prec):
    """K = 40 tracked pairs with L + P = 32 < K: the refinement's K x K
    products and double-float kernels in their two-columns-per-lane forms,
    the projections on the tensor-core Gram, on a power-law stream with the
    RSVD new-node block (normalized Laplacian: algebraic ordering, so no
    +-theta near-ties at the K boundary)."""
    g0, batches = wl.chung_lu_stream(3000, 2.4, 14, 2, 0.02, 6, 0.002, seed=21, lcc=True)
    tr, st, ocfg = U.make_pair(g0, 40, O.OP_NLAP, L=20, P=12, seed=3, precision=prec, drop_tol=1e-3)
    ocfg.drop_tol = 1e-3
    for t, b in enumerate(batches):
        st, info = O.grest_step(st, b, ocfg)
        s = tr.update(b)
        assert s["mode"] == 4 and s["m"] == info.m
        compare_mixed(tr, st, info, O.OP_NLAP, 40, f"mixed K=40 step {t}")
    tr.close()
