"""The float-float split of FP64 values (the mixed solve's residual and Born
term, Sec. 4.1 precision), done with integer operations on the device (an
FP64-pipe conversion per value was the splitting kernels' limit): hi and lo
must be exactly IEEE 754 round-to-nearest-even, as numpy's float64 -> float32
cast gives them, wherever the result is a normal float; a part below the
float normal range (2^-126) is zero."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TINY = 2.0**-126


@pytest.fixture(scope="module")
def W():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1508_07441_gb300 import build, wpcd

    build.build()
    return wpcd


def _values(seed):
    rng = np.random.default_rng(seed)
    n = 1 << 18
    # every binade of the float normal range, both signs
    x = rng.uniform(1.0, 2.0, n) * np.exp2(rng.integers(-125, 127, n).astype(np.float64))
    x *= np.where(rng.random(n) < 0.5, -1.0, 1.0)
    # exact ties between two floats: the 29 bits dropped are 1 followed by 0s,
    # with the float's last kept bit both even and odd
    b = rng.integers(0, 1 << 52, 4096, dtype=np.uint64) & ~np.uint64((1 << 29) - 1)
    b |= np.uint64(1 << 28)
    b |= (rng.integers(900, 1140, 4096).astype(np.uint64) << np.uint64(52))
    ties = b.view(np.float64)
    specials = np.array([0.0, -0.0, 1.0, -1.0, np.finfo(np.float32).max, np.finfo(np.float32).tiny,
                         2.0**-126 * 1.5, 3.4e38, 1e-30, 123456789.123456789, np.pi, -np.e])
    return np.concatenate([x, ties, specials])


@pytest.mark.parametrize("seed", [1, 2])
def test_split_matches_ieee_rounding(W, seed):
    import torch

    x = _values(seed)
    xd = torch.from_numpy(x).cuda()
    hi = torch.full(x.shape, float("nan"), dtype=torch.float32, device="cuda")
    lo = torch.full_like(hi, float("nan"))
    W.wpcd_split_f64(xd, hi, lo)
    torch.cuda.synchronize()
    h, l = hi.cpu().numpy(), lo.cpu().numpy()
    with np.errstate(over="ignore"):
        h_ref = x.astype(np.float32)
        l_ref = (x - h_ref.astype(np.float64)).astype(np.float32)
    assert np.array_equal(h.view(np.uint32), h_ref.view(np.uint32))
    normal = (np.abs(l_ref) >= TINY) | (l_ref == 0)
    assert normal.sum() > 0.8 * len(x)
    assert np.array_equal(l[normal].view(np.uint32), l_ref[normal].view(np.uint32))
    assert np.all(l[~normal] == 0)
    # the pair carries x to the float-float precision where lo, about 2^-24 x,
    # is itself a normal float
    hl = h.astype(np.float64) + l.astype(np.float64)
    fin = np.isfinite(h) & (np.abs(x) >= 2.0**-90)
    assert np.max(np.abs(hl[fin] - x[fin]) / np.abs(x[fin])) <= 2.0**-47


def test_split_below_float_range_is_zero(W):
    import torch

    x = np.array([1e-39, -1e-40, 2.0**-127, 1e-300, -5e-324])
    xd = torch.from_numpy(x).cuda()
    hi = torch.full(x.shape, float("nan"), dtype=torch.float32, device="cuda")
    lo = torch.full_like(hi, float("nan"))
    W.wpcd_split_f64(xd, hi, lo)
    assert np.all(hi.cpu().numpy() == 0) and np.all(lo.cpu().numpy() == 0)
    assert np.array_equal(np.signbit(hi.cpu().numpy()), np.signbit(x))
