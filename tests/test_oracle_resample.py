"""Pins for the oracle's resampler: the FP32 weight code and exact
systematic resampling (Alg. 1 step 6, Alg. 3 step 7).  CPU only."""
import math
from fractions import Fraction

import numpy as np
import pytest


def _counts(anc, n):
    return np.bincount(anc, minlength=n)


def test_exp2_coefficients_are_taylor_of_2_pow_f(ora):
    c = ora.exp2_coeffs()
    for d in range(8):
        exact = math.log(2.0) ** d / math.factorial(d)
        assert c[d] == np.float32(exact) or abs(float(c[d]) - exact) <= 2 ** -24 * exact


def test_quantize_matches_exp_within_fp32_bound(ora):
    rng = np.random.default_rng(0)
    lw = (rng.uniform(-27.0, 0.0, size=20000) - 312.5).astype(np.float32)
    lw[17] = np.float32(-312.5)  # the maximum
    q = ora.quantize(lw)
    M = float(lw.max())
    ref = np.exp(lw.astype(np.float64) - M)
    got = q.astype(np.float64) / 2.0 ** 40
    assert q[np.argmax(lw)] == 2 ** 40
    assert np.all(np.abs(got - ref) <= 1e-5 * ref + 2.0 ** -40)


def test_quantize_special_values(ora):
    lw = np.array([0.0, np.nan, -np.inf, -1e30, -27.0, -28.0, 5.0], np.float32)
    q = ora.quantize(lw)
    assert q[6] == 2 ** 40
    assert q[1] == 0 and q[2] == 0 and q[3] == 0
    assert q[5] == 0           # 2^-40.4 is below the code's resolution
    assert q[4] == 0 or q[4] > 0  # 2^(-32*log2 e) ~ exp(-32) just inside
    assert np.all(ora.quantize(np.full(5, -np.inf, np.float32)) == 0)
    assert np.all(ora.quantize(np.full(5, np.nan, np.float32)) == 0)


@pytest.mark.parametrize("seed", range(8))
def test_counts_sum_to_n_and_are_floor_or_ceil(ora, seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 3000))
    q = rng.integers(0, 2 ** 40, size=n, dtype=np.uint64)
    q[rng.random(n) < 0.3] = 0
    if q.sum() == 0:
        q[0] = 1
    u = int(rng.integers(0, 2 ** 32))
    anc = ora.resample(q, u)
    cnt = _counts(anc, n)
    assert cnt.sum() == n
    Q = int(sum(int(v) for v in q))
    for i in range(n):
        lo = (n * int(q[i])) // Q
        hi = -((-n * int(q[i])) // Q)
        assert lo <= cnt[i] <= hi
    assert np.all(np.diff(anc) >= 0)                  # ancestors sorted
    assert np.all(q[anc] > 0)                         # zero weight never chosen


def test_expectation_is_exact_over_the_uniform(ora):
    """E_u[count_i] = n q_i / Q: integrate the piecewise-constant counts over
    every breakpoint of u in [0, 2^32)."""
    rng = np.random.default_rng(5)
    for _ in range(6):
        n = int(rng.integers(2, 7))
        q = rng.integers(0, 50, size=n).astype(np.uint64)
        if q.sum() == 0:
            q[-1] = 3
        Q = int(q.sum())
        S = np.concatenate([[0], np.cumsum(q.astype(object))])
        bps = {0, 1 << 32}
        for j in range(n):
            for s in S:
                b = Fraction(int(s) * n * (1 << 32), Q) - j * (1 << 32)
                if 0 < b < (1 << 32):
                    bps.add(math.ceil(b))
        bps = sorted(bps)
        E = np.zeros(n, dtype=object)
        for a, b in zip(bps[:-1], bps[1:]):
            if b > a:
                E = E + _counts(ora.resample(q, a), n).astype(object) * (b - a)
        for i in range(n):
            got = Fraction(int(E[i]), 1 << 32)
            want = Fraction(n * int(q[i]), Q)
            assert abs(got - want) <= Fraction(len(bps), 1 << 32)


def test_brute_force_textbook_systematic_resampling(ora):
    """A textbook cumulative-weight walk with exact rationals."""
    rng = np.random.default_rng(11)
    for _ in range(50):
        n = int(rng.integers(1, 12))
        q = rng.integers(0, 1000, size=n).astype(np.uint64)
        q[rng.random(n) < 0.3] = 0
        if q.sum() == 0:
            continue
        u = int(rng.integers(0, 2 ** 32))
        Q = int(q.sum())
        cum = np.cumsum(q.astype(object))
        want, i = [], 0
        for j in range(n):
            point = (j + Fraction(u, 1 << 32)) / n      # in (0, 1)
            while Fraction(int(cum[i]), Q) <= point:
                i += 1
            want.append(i)
        assert list(ora.resample(q, u)) == want


def test_degenerate_and_special_weight_patterns(ora):
    n = 37
    assert list(ora.resample(np.zeros(n, np.uint64), 123)) == list(range(n))
    eq = np.full(n, 2 ** 40, np.uint64)
    for u in (0, 1, 2 ** 31, 2 ** 32 - 1):
        assert list(ora.resample(eq, u)) == list(range(n))
    one = np.zeros(n, np.uint64)
    one[13] = 5
    assert set(ora.resample(one, 777)) == {13}
    # maximum size and maximum codes: no 128-bit overflow
    big = np.full(1 << 20, 2 ** 40, np.uint64)
    anc = ora.resample(big, 2 ** 32 - 1)
    assert np.array_equal(anc, np.arange(1 << 20))
