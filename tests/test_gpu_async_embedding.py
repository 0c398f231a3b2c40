"""grest_get_embedding_async: reading each step's pairs (X_K, Lambda_K) into
pinned host memory while the next update runs gives, bit for bit, what the
synchronous grest_get_embedding gives after that step, in the FP64 and the
mixed path, including a step that grows the node capacity while a copy is
still outstanding (the growth moves U, so it must wait for the copy); pinned
buffers take the kernel path, pageable ones the cudaMemcpyAsync path."""
import numpy as np
import pytest

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


@pytest.mark.parametrize("prec,pinned", [(G.FP64, True), (G.MIXED, True), (G.MIXED, False)],
                         ids=["fp64-pinned", "mixed-pinned", "mixed-pageable"])
def test_async_reads_equal_sync_reads(cuda, prec, pinned):
    torch = cuda
    K, steps = 6, 4
    g0, batches = wl.sbm_stream(n0=3000, steps=steps, n_new=150, n_rand=200)
    rp, col, _ = g0.csr()
    import oracle as O
    s0 = O.init_state(g0.n, rp, col, None, K, O.OP_ADJ)
    kw = dict(precision=prec, drop_tol=1e-3 if prec != G.FP64 else 1e-12, L=8, P=4, seed=3,
              node_capacity=g0.n + 200)  # the second batch already needs more ids
    sync_tr = G.Tracker(g0.n, rp, col, None, s0.X, s0.lam, K, **kw)
    async_tr = G.Tracker(g0.n, rp, col, None, s0.X, s0.lam, K, **kw)
    want = []
    for b in batches:
        sync_tr.update(b)
        U, th, _ = sync_tr.embedding()
        want.append((U, th))
    n_max = g0.n + sum(b.n_new for b in batches)
    def host(*shape):
        t = torch.empty(shape, dtype=torch.float64)
        return t.pin_memory() if pinned else t  # pinned: written by a kernel; pageable: cudaMemcpyAsync
    bufs = [(host(n_max, K), host(K)) for _ in batches]
    rows = []
    for b, (Ub, tb) in zip(batches, bufs):
        async_tr.update(b)  # the previous read may still be in flight
        rows.append(async_tr.embedding_async(Ub, tb))
    async_tr.wait_embedding()
    for t, ((U, th), (Ub, tb), n) in enumerate(zip(want, bufs, rows)):
        assert n == U.shape[0]
        assert np.array_equal(Ub.numpy()[:n], U), f"step {t}"
        assert np.array_equal(tb.numpy(), th), f"step {t}"
    sync_tr.close()
    async_tr.close()
