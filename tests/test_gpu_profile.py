"""GREST_FLAG_PROFILE per kernel kind: every timed launch group of a step is
counted under one kind (grest_stats.prof_kind_*) and one class (prof_*), so
the kinds of each class add up to the class, and each path uses the kinds
it should: the mixed path's tensor-core and narrow Grams and tensor-core
GEMMs with its FP64 refinement (CUDA-core Gram and GEMM, FP64 SpMM); the
FP64 path only CUDA-core kinds.  The mixed path's GEMM class also times
two elementwise passes of the refinement (the widening of U to FP64 and the
sign normalization), which have no kind."""
import numpy as np
import pytest

import oracle as O
from paper_2603_19439_gb300 import grest as G
from paper_2603_19439_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

KIND = {k: i for i, k in enumerate(G.PROF_KINDS)}
CLASS_OF = {"spmm_f32": 0, "spmm_f64": 0, "gram_tc": 1, "gram_narrow": 1, "gram_cuda": 1, "gemm_tc": 2,
            "gemm_cuda": 2, "small": 3, "graph": 4}


@pytest.fixture(scope="module", autouse=True)
def cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_19439_gb300.build import build
    build()
    torch.cuda.set_device(0)
    return torch


def step_stats(prec):
    g0, batches = wl.power_law_workload(30_000, 2.3, 16, 2, 0.01, 8, 0.001, 77)
    rp, col, _ = wl.csr_fast(g0)
    st = O.init_state(g0.n, rp, col, None, 16, O.OP_ADJ)
    tr = G.Tracker(g0.n, rp, col, None, st.X, st.lam, 16, precision=prec, L=40, P=40, seed=5,
                   drop_tol=1e-3 if prec != G.FP64 else 1e-7, flags=G.FLAG_PROFILE,
                   node_capacity=g0.n + 2000)
    out = [tr.update(b) for b in batches]
    tr.close()
    return out


@pytest.mark.parametrize("prec", [G.FP64, G.MIXED], ids=["fp64", "mixed"])
def test_kinds_add_up_to_classes(prec):
    for d in step_stats(prec):
        assert d["mode"] == 4  # an RSVD step: every stage runs
        kl = np.array(d["prof_kind_launches"])
        cl = np.array(d["prof_launches"])
        kms = np.array(d["prof_kind_ms"])
        cms = np.array(d["prof_ms"])
        elementwise = {G.FP64: 0, G.MIXED: 2}[prec]
        for c in range(5):
            ks = [KIND[k] for k, cc in CLASS_OF.items() if cc == c]
            assert kl[ks].sum() == cl[c] - (elementwise if c == 2 else 0), (c, kl, cl)
            if c != 2:
                assert abs(kms[ks].sum() - cms[c]) <= 1e-3 * max(cms[c], 1e-3), (c, kms, cms)
            else:
                assert kms[ks].sum() <= cms[c] * (1 + 1e-3) + 1e-3
        used = {k for k in G.PROF_KINDS if kl[KIND[k]] > 0}
        if prec == G.FP64:
            assert used <= {"spmm_f64", "gram_cuda", "gemm_cuda", "small", "graph"}, used
        else:
            assert {"spmm_f32", "gram_tc", "gram_narrow", "gemm_tc", "spmm_f64", "gram_cuda", "gemm_cuda"} <= used
