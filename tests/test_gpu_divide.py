"""The library's correctly rounded FP64 division (the edge weights c_ij of
the matching, Sec. 3.1, depend on one division per edge and must match the
oracle's IEEE division bit for bit): through amg_div_check, every quotient
equals numpy's IEEE binary64 quotient (round to nearest even), on random
operands across and beyond the fast path's exponent range, on all-ones and
power-of-two mantissas, and on quotients placed next to rounding midpoints;
the fast path accepts nearly every in-range quotient."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2511_21268_gb300 import amg as A  # noqa: E402


def _check(a, b):
    q, fast = A.amg_div_check(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda())
    torch.cuda.synchronize()
    want = a / b
    got = q.cpu().numpy()
    # bit for bit; NaN against NaN whatever its payload
    bad = np.nonzero((got.view(np.uint64) != want.view(np.uint64)) & ~(np.isnan(got) & np.isnan(want)))[0]
    assert len(bad) == 0, (a[bad[:5]], b[bad[:5]], got[bad[:5]], want[bad[:5]])
    return int(fast.item())


def _random(rng, n, emin, emax):
    m = rng.uniform(1.0, 2.0, n)
    e = rng.integers(emin, emax + 1, n)
    s = rng.choice([-1.0, 1.0], n)
    return s * np.ldexp(m, e)


def test_random_operands_in_range_take_the_fast_path():
    rng = np.random.default_rng(11)
    n = 4_000_000
    a = _random(rng, n, -480, 480)
    b = _random(rng, n, -480, 480)
    fast = _check(a, b)
    assert fast >= 0.999 * n, fast


def test_operands_beyond_the_range_and_special_values():
    rng = np.random.default_rng(12)
    a = _random(rng, 200_000, -1020, 1020)
    b = _random(rng, 200_000, -1020, 1020)
    sub = np.array([5e-324, 1e-310, -2.5e-320, 0.0, -0.0, np.inf, -np.inf, 1.0, 3.0, 7.0])
    A2, B2 = np.meshgrid(np.concatenate([sub, [np.nan]]), np.concatenate([sub, [np.nan, 1e300]]))
    with np.errstate(all="ignore"):
        _check(np.concatenate([a, A2.ravel()]), np.concatenate([b, B2.ravel()]))


def test_hard_mantissas_and_near_midpoint_quotients():
    rng = np.random.default_rng(13)
    n = 1_000_000
    ones = np.nextafter(2.0, 0.0)  # mantissa of all ones
    b = np.concatenate([np.ldexp(ones, rng.integers(-300, 300, n // 4)),
                        np.ldexp(1.0, rng.integers(-300, 300, n // 4)),
                        rng.choice([3.0, 5.0, 7.0, 11.0, 13.0, 1.5, 0.75], n // 2) *
                        np.ldexp(1.0, rng.integers(-40, 40, n // 2))])
    q = _random(rng, n, -200, 200)
    # a = b (q + u/2) rounded: the quotient sits within an ulp's fraction of
    # the midpoint between q and its upper neighbour
    u = np.spacing(np.abs(q))
    a = b * q + b * (np.sign(q) * u * 0.5)  # the second product is exact
    a2 = b * q  # products, mostly inexact
    a3 = np.ldexp(rng.integers(1, 1 << 53, n).astype(np.float64), rng.integers(-60, 60, n))
    fast = _check(np.concatenate([a, a2, a3]), np.concatenate([b, b, b]))
    assert fast >= 0.99 * 3 * n, fast
