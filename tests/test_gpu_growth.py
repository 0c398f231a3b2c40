"""A context outgrows its initial capacities (Alg. 2 appends S ids every step,
Eq. adj_update): the per-node arrays move to a larger node capacity and the
edge arena is compacted into a larger one while a stream runs.  Each step must
match the FP64 CPU oracle as any other, and the results must be bit-identical
to those of a context created with room for the whole stream (capacities are
storage, not arithmetic)."""
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


def tight_arena(rp):
    """The smallest edge arena grest_init accepts: one slot of len + len/4 + 4 per row."""
    ln = np.diff(rp)
    return int(np.sum(ln + ln // 4 + 4))


@pytest.mark.parametrize("precision", [G.FP64, G.MIXED])
def test_context_grows_and_matches_oracle(cuda, precision):
    g0, batches = wl.sbm_stream(n0=600, steps=6, n_new=40, n_rand=150, seed=77)
    rp, col, _ = g0.csr()
    K = 6
    tol = 1e-7 if precision == G.FP64 else 1e-3
    st = O.init_state(g0.n, rp, col, None, K, O.OP_ADJ)
    kw = dict(precision=precision, drop_tol=tol)
    tight = G.Tracker(g0.n, rp, col, None, st.X, st.lam, K, node_capacity=g0.n + 8,
                      nnz_capacity=tight_arena(rp) + 16, **kw)
    roomy = G.Tracker(g0.n, rp, col, None, st.X, st.lam, K, node_capacity=4 * g0.n,
                      nnz_capacity=8 * int(rp[-1]) + (1 << 20), **kw)
    ocfg = O.Config(k=K, drop_tol=tol)
    bytes0 = tight.device_bytes()
    for t, b in enumerate(batches):
        st, info = O.grest_step(st, b, ocfg)
        s1 = tight.update(b)
        s2 = roomy.update(b)
        assert s1["n_nodes"] == s2["n_nodes"] == st.A.shape[0]
        assert s1["nnz"] == s2["nnz"] == st.A.nnz
        U1, th1, live1 = tight.embedding()
        U2, th2, live2 = roomy.embedding()
        assert np.array_equal(U1, U2) and np.array_equal(th1, th2) and np.array_equal(live1, live2), f"step {t}"
        if precision == G.FP64:
            U.compare(tight, st, info, O.OP_ADJ, K, f"growth step {t}")
        else:
            scale = abs(st.lam[0])
            assert np.max(np.abs(th1 - st.lam)) <= 1e-6 * scale, f"growth step {t}"
    # both kinds of growth happened: 600 + 6 x 40 ids against a capacity of 608,
    # and an arena with 16 spare entries against 150 + 40 x (about 24) new edges per step
    assert tight.device_bytes() > bytes0
    tight.close()
    roomy.close()


def test_growth_keeps_checkpoints_equal(cuda):
    """A grown context checkpoints to the same bytes as a roomy one (the
    compacted arena keeps every row's neighbour order)."""
    g0, batches = wl.sbm_stream(n0=400, steps=3, n_new=30, n_rand=80, seed=78)
    rp, col, _ = g0.csr()
    K = 4
    st = O.init_state(g0.n, rp, col, None, K, O.OP_ADJ)
    tight = G.Tracker(g0.n, rp, col, None, st.X, st.lam, K, node_capacity=g0.n + 1,
                      nnz_capacity=tight_arena(rp))
    roomy = G.Tracker(g0.n, rp, col, None, st.X, st.lam, K, node_capacity=2 * g0.n)
    for b in batches:
        tight.update(b)
        roomy.update(b)
    c1, c2 = tight.checkpoint(), roomy.checkpoint()
    # the headers carry the configured capacities, which differ by design; the graph and pairs do not
    import ctypes
    hdr = (8 + 8 + 8 * 4 + ctypes.sizeof(G.Config) + 7) // 8 * 8  # magic, version + K, 4 int64, config
    assert len(c1) == len(c2)
    assert c1[hdr:] == c2[hdr:]
    tight.close()
    roomy.close()
