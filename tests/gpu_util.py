"""Helpers shared by the GPU parity tests: run the oracle and the CUDA library on
the same seeded inputs and compare them under the stated tolerances.

Tolerances (FP64 path): every Ritz value within 1e-10 * |theta_1| of the
oracle's, and the sin of the largest principal angle between the tracked
subspaces at most 1e-8.  Where consecutive tracked values are closer than
1e-6 * |theta_1| (degenerate clusters, e.g. the equal communities of an SBM)
the individual vectors are not unique, so subspaces are compared only up to
the last index that ends a cluster (reading of Sec. 5.1's psi metric).
"""
import numpy as np

import oracle as O
from paper_2603_19439_gb300 import grest as G
from paper_2603_19439_gb300 import workloads as wl

THETA_TOL = 1e-10
ANGLE_TOL = 1e-8
GAP_SPLIT = 1e-6


def sin_angle(U, V):
    if U.shape[1] == 0:
        return 0.0
    Qu, _ = np.linalg.qr(U)
    Qv, _ = np.linalg.qr(V)
    return float(np.linalg.norm(Qv - Qu @ (Qu.T @ Qv), 2))


def cluster_cut(theta, op, upto):
    """Largest j <= upto such that the tracked values j-1 and j are separated."""
    scale = max(abs(theta[0]), 1e-300)
    key = np.abs(theta) if op == O.OP_ADJ else theta
    for j in range(upto, 0, -1):
        if j == len(theta) or abs(key[j - 1] - key[j]) > GAP_SPLIT * scale:
            return j
    return 0


def compare(tr: "G.Tracker", st: "O.State", info: "O.StepInfo", op, k, where=""):
    Ug, thg, liveg = tr.embedding()
    ritz_g = tr.ritz_values()
    scale = abs(st.lam[0])
    assert Ug.shape == st.X.shape, where
    assert np.array_equal(liveg, st.live), where
    assert ritz_g.size == info.m, f"{where}: m {ritz_g.size} vs {info.m}"
    assert np.max(np.abs(ritz_g - info.ritz_all)) <= THETA_TOL * scale, \
        f"{where}: ritz err {np.max(np.abs(ritz_g - info.ritz_all)) / scale:.3e}"
    assert np.max(np.abs(thg - st.lam)) <= THETA_TOL * scale, where
    # the boundary K / K+1 may itself sit inside a cluster
    j = cluster_cut(info.ritz_all, op, k)
    ang = sin_angle(st.X[:, :j], Ug[:, :j])
    assert ang <= ANGLE_TOL, f"{where}: sin angle {ang:.3e} over {j} vectors"
    # orthonormality of the GPU result
    assert np.abs(Ug.T @ Ug - np.eye(k)).max() < 1e-12, where
    return ang


def make_pair(g: "wl.EdgeSetGraph", k, op, dense_limit=4000, **cfg):
    rp, col, val = g.csr()
    st = O.init_state(g.n, rp, col, val, k, op, dense_limit=dense_limit)
    tr = G.Tracker(g.n, rp, col, val, st.X, st.lam, k, op=op, **cfg)
    ocfg = O.Config(k=k, op=op, subspace=cfg.get("subspace", G.SUB_AUTO), L=cfg.get("L", 100),
                    P=cfg.get("P", 100), seed=cfg.get("seed", 0), drop_tol=cfg.get("drop_tol", 1e-7))
    return tr, st, ocfg
