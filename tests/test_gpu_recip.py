"""The FP64 reciprocal of the small factorizations' scalar chains (two
Newton-Raphson steps from the hardware's reduced-precision reciprocal) held
to its error bound: within 2 units in the last place of the correctly
rounded 1 / x (numpy's IEEE division) over normal inputs of every binade
from 2^-1000 to 2^1000, both signs, and exact on powers of two; zero,
subnormal, huge, infinite and NaN inputs give what IEEE division gives."""
import numpy as np
import pytest

from paper_2603_19439_gb300 import grest as G

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


def recip_on_device(torch, x):
    lib = G.load_library()
    xd = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()
    out = torch.empty_like(xd)
    st = lib.grest_check_fast_recip(xd.data_ptr(), x.size, out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert st == 0, G.STATUS.get(st)
    return out.cpu().numpy()


def ulp_distance(a, b):
    """Distance in units in the last place between non-negative finite doubles."""
    return np.abs(a.view(np.int64) - b.view(np.int64))


def test_newton_reciprocal_within_two_ulp(cuda):
    rng = np.random.default_rng(5)
    mant = rng.uniform(1.0, 2.0, 200_000)
    expo = rng.integers(-1000, 1001, mant.size)
    x = np.ldexp(mant, expo) * np.where(rng.random(mant.size) < 0.5, -1.0, 1.0)
    x = np.concatenate([x, np.nextafter(1.0, 2.0) * np.arange(1, 1000), -np.ldexp(1.0, np.arange(-1000, 1001, 7))])
    got = recip_on_device(cuda, x)
    want = 1.0 / x
    assert np.all(np.signbit(got) == np.signbit(want))
    d = ulp_distance(np.abs(got), np.abs(want))
    assert d.max() <= 2, d.max()
    p2 = np.ldexp(1.0, np.arange(-1000, 1001))
    assert np.array_equal(recip_on_device(cuda, p2), 1.0 / p2)


def test_newton_reciprocal_special_inputs(cuda):
    x = np.array([0.0, -0.0, 5e-324, -1e-310, 2.0 ** -1022, 2.0 ** 1022, 1.5 * 2.0 ** 1023, np.inf, -np.inf, np.nan])
    got = recip_on_device(cuda, x)
    with np.errstate(divide="ignore", over="ignore"):
        want = 1.0 / x
    both_nan = np.isnan(got) & np.isnan(want)
    assert np.all(both_nan | (got == want)), (got, want)
    assert np.array_equal(np.signbit(got[~both_nan]), np.signbit(want[~both_nan]))
