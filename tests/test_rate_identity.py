"""The two identities the signal-rate code relies on, checked on the host in
IEEE arithmetic (numpy rounds every operation as the device does):

* cubic cells: max_d round(round(|v_d| + c) * idx) equals
  round(round(max_d |v_d| + c) * idx) bit for bit, because rounding is
  monotone (the device then takes two adds and two multiplies fewer);
* the running max on unsigned bit patterns (rate_max): for non-negative
  numbers it is the numeric max, and a NaN of either sign, once in, stays on
  top whatever finite rates follow (an FP `not (r <= m)` test does not)."""
import numpy as np


def test_cubic_cell_rate_is_the_max_speed_plus_c():
    rng = np.random.default_rng(7)
    for dtype in (np.float64, np.float32):
        n = 200000
        v = np.abs(rng.standard_normal((n, 3)) * 10.0 ** rng.integers(-8, 8, (n, 1))).astype(dtype)
        v[::7, 1] = v[::7, 0]                                     # ties
        v[::11, 2] = 0
        c = (rng.random(n) * 10.0 ** rng.integers(-6, 6, n)).astype(dtype)
        idx = (rng.random(n) * 10.0 ** rng.integers(-3, 4, n)).astype(dtype)
        per_dir = ((v + c[:, None]).astype(dtype) * idx[:, None]).astype(dtype)
        a = per_dir.max(axis=1)
        b = ((v.max(axis=1) + c).astype(dtype) * idx).astype(dtype)
        assert np.array_equal(a.view(np.uint64 if dtype == np.float64 else np.uint32),
                              b.view(np.uint64 if dtype == np.float64 else np.uint32))


def _rate_max_bits(seq, dtype):
    u = np.uint64 if dtype == np.float64 else np.uint32
    m = np.array([0], dtype=dtype).view(u)[0]
    for r in seq:
        m = max(m, np.array([r], dtype=dtype).view(u)[0])
    return np.array([m], dtype=u).view(dtype)[0]


def _rate_max_fp(seq):
    m = 0.0
    for r in seq:
        if not (r <= m):
            m = r
    return m


def test_bit_pattern_max_keeps_nan():
    rng = np.random.default_rng(3)
    for dtype in (np.float64, np.float32):
        for _ in range(200):
            seq = list((rng.random(9) * 100).astype(dtype))
            assert _rate_max_bits(seq, dtype) == max(seq)           # numeric max without NaN
            neg_nan = -np.array([np.nan], dtype=dtype)[0]           # sign bit set
            for nan in (dtype(np.nan), neg_nan):
                k = int(rng.integers(0, 8))
                s2 = seq[:k] + [nan] + seq[k:]
                assert np.isnan(_rate_max_bits(s2, dtype))
        # the FP test loses a NaN that is followed by a finite rate
        assert not np.isnan(_rate_max_fp([1.0, float("nan"), 2.0]))
