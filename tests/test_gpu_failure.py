"""Failure detection on the GPU without a fault: every wait of the library's
kernels on a device-side barrier is bounded, and an expired wait becomes
GREST_ERR_TIMEOUT with the device still usable.  grest_check_bounded_wait
makes one wait run out (a barrier that nothing arrives on); the test checks
the status and then runs a normal update in the same process."""
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


def test_expired_wait_reports_timeout_and_device_stays_usable(cuda):
    torch = cuda
    lib = G.load_library()
    st = lib.grest_check_bounded_wait(torch.cuda.current_stream().cuda_stream)
    assert st == 7, G.STATUS.get(st)
    # the same process keeps working: a small mixed update matches the oracle
    g0, batches = wl.sbm_stream(n0=300, steps=1, n_new=10, n_rand=20)
    rp, col, _ = g0.csr()
    s0 = O.init_state(g0.n, rp, col, None, 4, O.OP_ADJ)
    tr = G.Tracker(g0.n, rp, col, None, s0.X, s0.lam, 4, precision=G.MIXED, drop_tol=1e-3)
    tr.update(batches[0])
    s1, _ = O.grest_step(s0, batches[0], O.Config(k=4, drop_tol=1e-3))
    _, th, _ = tr.embedding()
    assert np.max(np.abs(th - s1.lam)) <= 1e-6 * abs(s1.lam[0])
    tr.close()
