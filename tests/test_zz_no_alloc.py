"""grest_gram_noalloc, the Gram entry point for callers that cannot allocate
device memory: its result must equal the context-based grest_gram on the same
inputs, on two calls in a row (the second call reuses the library's fixed
scratch array and must not see the first call's partial sums).

This file's name sorts last so that a run that stops at the first failure has
already run every other test; it also passes alone in a fresh process."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_19439_gb300.build import build
    build()
    torch.cuda.set_device(0)
    return torch


def test_noalloc_gram_matches_context_gram_twice(torch_cuda):
    torch = torch_cuda
    from paper_2603_19439_gb300 import grest as G
    from paper_2603_19439_gb300 import workloads as wl

    g, _ = wl.sbm_graph(100, 2, 0.2, 0.05, 3)
    rp, col, _ = g.csr()
    U0 = np.linalg.qr(np.random.default_rng(0).standard_normal((g.n, 3)))[0]
    tr = G.Tracker(g.n, rp, col, None, U0, np.ones(3), 3)
    rng = np.random.default_rng(7)
    # two calls in a row with different shapes; the second has fewer rows per
    # chunk and narrower blocks, so stale partials of the first would show
    for n, a, b in ((200_003, 200, 132), (40_001, 33, 64)):
        X = torch.tensor(rng.standard_normal((n, a)), device="cuda")
        Y = torch.tensor(rng.standard_normal((n, b)), device="cuda")
        C_ref = torch.empty((a, b), dtype=torch.float64, device="cuda")
        C_new = torch.full((a, b), np.nan, dtype=torch.float64, device="cuda")
        tr.gram(X, Y, C_ref)
        G.gram_noalloc(X, Y, C_new)
        torch.cuda.synchronize()
        ref = C_ref.cpu().numpy()
        new = C_new.cpu().numpy()
        scale = np.abs(ref).max()
        assert np.isfinite(new).all()
        assert np.abs(new - ref).max() <= 1e-12 * scale
        # and both agree with a plain float64 product
        plain = X.cpu().numpy().T @ Y.cpu().numpy()
        assert np.abs(new - plain).max() <= 1e-12 * scale
    # widths beyond the fixed scratch are rejected with a clear status
    X = torch.zeros((10, 257), dtype=torch.float64, device="cuda")
    C = torch.zeros((257, 257), dtype=torch.float64, device="cuda")
    with pytest.raises(G.GrestError) as e:
        G.gram_noalloc(X, X, C)
    assert e.value.code == 4
    tr.close()
