"""The FP64 step's division routine (lr_arith_check) against IEEE 754
division (numpy on the host): correctly rounded but for rare one-ulp cases
near rounding midpoints, exact IEEE results where it hands over to the
division instruction sequence (divisor zero, subnormal, infinite, NaN or of
magnitude >= 2^1020)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _gpu_div(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    from paper_2208_13409_gb300 import lr
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ta = torch.from_numpy(a).cuda()
    tb = torch.from_numpy(b).cuda()
    out = torch.empty_like(ta)
    lr.arith_check(lr.ARITH_DIV, ta, tb, out, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _ulps(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Distance in units in the last place between same-sign finite doubles."""
    ix = x.view(np.int64).astype(np.float64)
    iy = y.view(np.int64).astype(np.float64)
    return np.abs(ix - iy)


def _random(rng, n, lo, hi):
    mant = rng.uniform(1.0, 2.0, n)
    ex = rng.integers(lo, hi, n)
    sign = np.where(rng.random(n) < 0.5, -1.0, 1.0)
    return sign * np.ldexp(mant, ex)


def test_quotients_correctly_rounded_but_rarely():
    rng = np.random.default_rng(20813409)
    n = 1 << 21
    a = _random(rng, n, -480, 480)
    b = _random(rng, n, -480, 480)
    # physically scaled operands too: velocity differences, widths, masses
    a[: n // 4] = rng.normal(0.0, 1.0, n // 4) * 10.0 ** rng.integers(-12, 4, n // 4)
    b[: n // 4] = rng.uniform(1e-4, 1e3, n // 4) * np.where(rng.random(n // 4) < 0.5, -1.0, 1.0)
    ref = a / b
    got = _gpu_div(a, b)
    assert np.all(np.isfinite(got))
    assert np.all(np.sign(got) == np.sign(ref))
    d = _ulps(got, ref)
    assert d.max() <= 1.0, d.max()
    exact = np.mean(d == 0)
    assert exact >= 0.9999, exact


def test_divisor_edge_exponents_and_handover():
    big = np.ldexp(1.0, 1019)
    cases_b = np.array([
        np.ldexp(1.0, -1022), np.ldexp(1.5, -1022), -np.ldexp(1.25, -1021),       # smallest normal exponents
        np.ldexp(1.999, 1019), -big, np.ldexp(1.0, 1020), np.ldexp(1.7, 1023),   # around 2^1020
        5e-324, -1e-310, 0.0, -0.0, np.inf, -np.inf, np.nan,                     # handed over
        1.0, -1.0, 3.0, 0.1, 7.0 / 3.0,
    ])
    cases_a = np.array([1.0, -3.0, 2.5, 1e-300, 0.5, 1e300, 1.0, 1e-300, 1.0, 1.0, 1.0, 2.0, 2.0, 1.0,
                        1.0, 1.0, 1.0, 1.0, 1.0])
    assert cases_a.shape == cases_b.shape
    with np.errstate(all="ignore"):
        ref = cases_a / cases_b
    got = _gpu_div(cases_a, cases_b)
    ed = (cases_b.view(np.uint64) >> np.uint64(52)) & np.uint64(0x7FF)
    handled = (ed >= 1) & (ed <= 2043)
    # handed over to IEEE division: identical bits (NaN stays NaN)
    hb = ~handled
    assert np.array_equal(np.isnan(got[hb]), np.isnan(ref[hb]))
    fin = hb & ~np.isnan(ref)
    assert np.array_equal(got[fin].view(np.int64), ref[fin].view(np.int64))
    # handled divisors with a normal quotient: within one ulp
    normal = handled & np.isfinite(ref) & (np.abs(ref) >= np.ldexp(1.0, -1022))
    assert normal.sum() >= 10
    assert _ulps(got[normal], ref[normal]).max() <= 1.0


def test_zero_numerator_and_quotients_near_underflow():
    b = np.array([1.0, -2.0, 1e-200, 3.0e250, 0.3])
    a = np.zeros_like(b)
    got = _gpu_div(a, b)
    assert np.all(got == 0.0)
    # quotients below the normal range: absolute error of a few subnormal steps
    a2 = np.array([1e-300, -3e-305, 2.5e-310])
    b2 = np.array([1e20, 7e3, 3.0])
    with np.errstate(all="ignore"):
        ref = a2 / b2
    got2 = _gpu_div(a2, b2)
    assert np.all(np.abs(got2 - ref) <= 4 * 5e-324)


def _gpu_sqrt(a: np.ndarray) -> np.ndarray:
    from paper_2208_13409_gb300 import lr
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ta = torch.from_numpy(a).cuda()
    out = torch.empty_like(ta)
    lr.arith_check(lr.ARITH_SQRT, ta, ta, out, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_square_roots_correctly_rounded_but_rarely():
    rng = np.random.default_rng(1340913)
    n = 1 << 21
    x = np.abs(_random(rng, n, -1020, 1020))
    x[: n // 4] = rng.uniform(0.0, 1.0, n // 4) * 10.0 ** rng.integers(-8, 12, n // 4)  # c^2, |u|^2 scales
    x[n // 4: n // 4 + 1000] = np.arange(1, 1001, dtype=np.float64) ** 2                 # perfect squares
    ref = np.sqrt(x)
    got = _gpu_sqrt(x)
    d = _ulps(got, ref)
    assert d.max() <= 1.0, d.max()
    assert np.mean(d == 0) >= 0.9999
    assert np.array_equal(got[n // 4: n // 4 + 1000], np.arange(1, 1001, dtype=np.float64))


def test_square_root_handover_cases():
    x = np.array([0.0, -0.0, 5e-324, 1e-310, -1.0, np.inf, np.nan, np.ldexp(1.5, 1023),
                  np.ldexp(1.0, -1022), np.ldexp(1.0, 1022), 2.0, 0.25])
    with np.errstate(all="ignore"):
        ref = np.sqrt(x)
    got = _gpu_sqrt(x)
    ex = (x.view(np.uint64) >> np.uint64(52)).astype(np.int64)  # sign bit included
    handled = (ex >= 1) & (ex <= 2045)
    hb = ~handled
    assert np.array_equal(np.isnan(got[hb]), np.isnan(ref[hb]))
    fin = hb & ~np.isnan(ref)
    assert np.array_equal(got[fin].view(np.int64), ref[fin].view(np.int64))
    assert _ulps(got[handled], ref[handled]).max() <= 1.0
    # even powers of two have exact roots
    assert got[8] == np.ldexp(1.0, -511) and got[9] == np.ldexp(1.0, 511) and got[11] == 0.5
