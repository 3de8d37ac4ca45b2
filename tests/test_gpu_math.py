"""Accuracy of the stage kernels' reciprocal and root routines (hardware
approximation + one Newton-Raphson step) against exact values: the library
uses them in place of correctly rounded division and square roots, so their
error bound is what keeps the FP64 path within 1e-12 of the oracle."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _ph():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2202_12309_gb300 as ph
    return ph, torch


def _inputs(n=1 << 20, lo=-60, hi=60, seed=5, positive=False, extremes=True):
    rng = np.random.default_rng(seed)
    x = np.exp2(rng.uniform(lo, hi, n))
    # values at and next to powers of two, where a reciprocal's mantissa wraps
    p2 = np.exp2(np.arange(lo, hi + 1, dtype=np.float64))
    x = np.concatenate([x, p2, np.nextafter(p2, 0), np.nextafter(p2, np.inf)])
    if extremes:  # just inside the range the refined path takes
        x = np.concatenate([x, [2.0 ** -999.5, 2.0 ** 999.5]])
    if not positive:
        x[rng.random(x.size) < 0.5] *= -1.0
    return x


def _ulp_err(y, exact, dtype):
    """|y - exact| in units of the last place of exact in `dtype`."""
    exact_d = exact.astype(dtype)
    ulp = np.spacing(np.abs(exact_d).astype(dtype)).astype(np.longdouble)
    return np.abs(y.astype(np.longdouble) - exact) / ulp


def _run(ph, torch, fn, x, dtype=np.float64):
    xt = torch.from_numpy(x.astype(dtype)).cuda()
    y = ph.debug_math(fn, xt)
    torch.cuda.synchronize()
    return y.cpu().numpy()


def test_fp64_reciprocal_within_one_ulp():
    ph, torch = _ph()
    x = _inputs()
    y = _run(ph, torch, "rcp", x)
    err = _ulp_err(y, 1 / x.astype(np.longdouble), np.float64)
    assert err.max() <= 1.0, err.max()
    # most results are the correctly rounded ones
    assert np.mean(y == 1.0 / x) > 0.95


def test_fp64_rsqrt_and_sqrt_within_bounds():
    ph, torch = _ph()
    x = _inputs(positive=True)
    xl = x.astype(np.longdouble)
    r = _run(ph, torch, "rsqrt", x)
    s = _run(ph, torch, "sqrt", x)
    er = _ulp_err(r, 1 / np.sqrt(xl), np.float64)
    es = _ulp_err(s, np.sqrt(xl), np.float64)
    assert er.max() <= 1.0, er.max()
    assert es.max() <= 2.0, es.max()  # x * rsqrt(x): two roundings


def test_fp64_hardware_approximations_good_to_2_pow_minus_19():
    """The one-step refinement assumes the start value has relative error
    well below 2^-18 (the truncation error is then below 2^-53)."""
    ph, torch = _ph()
    x = _inputs(positive=True)
    xl = x.astype(np.longdouble)
    a = _run(ph, torch, "rcp_approx", x).astype(np.longdouble)
    b = _run(ph, torch, "rsqrt_approx", x).astype(np.longdouble)
    ea = np.abs(a * xl - 1).max()
    eb = np.abs(b * np.sqrt(xl) - 1).max()
    assert ea <= 2.0 ** -19, float(ea)
    assert eb <= 2.0 ** -19, float(eb)


def test_fp64_special_arguments_take_the_correctly_rounded_path():
    ph, torch = _ph()
    tiny = np.nextafter(0.0, 1.0)
    x = np.array([0.0, -0.0, tiny, 1e-310, 2.0 ** -1001, 2.0 ** 1001, 1e308, np.inf, -np.inf, np.nan,
                  -1.0, -1e-310])
    with np.errstate(all="ignore"):
        ref = {"rcp": 1.0 / x, "sqrt": np.sqrt(x), "rsqrt": 1.0 / np.sqrt(x)}
    for fn in ("rcp", "sqrt", "rsqrt"):
        y = _run(ph, torch, fn, x)
        same = (y == ref[fn]) | (np.isnan(y) & np.isnan(ref[fn]))
        if fn == "rsqrt":  # CUDA's rsqrt is not correctly rounded: compare to 1 ulp
            fin = np.isfinite(ref[fn]) & (ref[fn] != 0)
            same[fin] = _ulp_err(y[fin], 1 / np.sqrt(x[fin].astype(np.longdouble)), np.float64) <= 1
        assert same.all(), (fn, x[~same], y[~same], ref[fn][~same])


def test_fp32_routines_within_bounds():
    """FP32: the hardware approximations alone (one special-function
    instruction each).  The kernels call them on normal positive numbers
    well inside the float range only (reciprocals also on negative sums of
    slopes)."""
    ph, torch = _ph()
    x = _inputs(n=1 << 18, lo=-40, hi=40, extremes=False).astype(np.float32)
    xp = np.abs(x)
    xl = xp.astype(np.longdouble)
    y = _run(ph, torch, "rcp", x, np.float32)
    err = _ulp_err(y, 1 / x.astype(np.longdouble), np.float32)
    assert err.max() <= 1.0, err.max()
    r = _run(ph, torch, "rsqrt", xp, np.float32)
    er = _ulp_err(r, 1 / np.sqrt(xl), np.float32)
    assert er.max() <= 2.0, er.max()
    s = _run(ph, torch, "sqrt", xp, np.float32)
    es = _ulp_err(s, np.sqrt(xl), np.float32)
    assert es.max() <= 2.0, es.max()
    # sqrt(0) = 0 (the Roe sound speed of a vanishing a^2)
    z = _run(ph, torch, "sqrt", np.zeros(4, dtype=np.float32), np.float32)
    assert np.all(z == 0.0)
