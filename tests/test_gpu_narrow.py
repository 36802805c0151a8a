"""The double -> float narrowing the adjoint uses on the integer pipe, against IEEE-754
round-to-nearest-even as numpy's float64 -> float32 conversion implements it: bit for bit
over random doubles across the normal float range, exact ties (even and odd), values
rounding up into the next binade and into overflow, and the special values; results
below the smallest normal float become a signed zero (documented)."""
import numpy as np
import pytest

from paper_1204_5434_gb300 import pft

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1204_5434_gb300 import build
    build.build()


def _narrow(x):
    torch = pytest.importorskip("torch")
    xd = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()
    yd = torch.empty(xd.shape, dtype=torch.float32, device="cuda")
    pft.pft_debug_narrow_rn(xd, yd)
    torch.cuda.synchronize()
    return yd.cpu().numpy()


def test_matches_ieee_round_to_nearest_even():
    rng = np.random.default_rng(0)
    mant = rng.uniform(1.0, 2.0, 200000)
    expo = rng.integers(-125, 127, 200000)
    x = np.ldexp(mant, expo) * rng.choice([-1.0, 1.0], 200000)
    # exact ties between neighbouring floats, even and odd last bits
    f = rng.uniform(1.0, 2.0, 20000).astype(np.float32)
    up = np.nextafter(f, np.float32(3.0))
    ties = (f.astype(np.float64) + up.astype(np.float64)) / 2.0
    # just below and above a tie
    near = np.concatenate([np.nextafter(ties, 0.0), np.nextafter(ties, 4.0)])
    fmax = float(np.finfo(np.float32).max)
    fmin = float(np.finfo(np.float32).tiny)
    edge = np.array([0.0, -0.0, 1.0, -1.0, fmax, -fmax, fmin, -fmin, np.inf, -np.inf,
                     np.nextafter(2.0, 0.0),                      # rounds up into the next binade
                     fmax * (1 + 2.0 ** -25), fmax * (1 + 2.0 ** -23)])  # below / above the overflow tie
    allx = np.concatenate([x, ties, near, edge])
    got = _narrow(allx)
    with np.errstate(over="ignore"):
        ref = allx.astype(np.float32)
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))


def test_nan_and_below_the_normal_range():
    got = _narrow(np.array([np.nan, 1e-39, -1e-39, 1e-300, -5e-45]))
    assert np.isnan(got[0])
    assert np.array_equal(got[1:].view(np.uint32), np.array([0.0, -0.0, 0.0, -0.0], np.float32).view(np.uint32))
