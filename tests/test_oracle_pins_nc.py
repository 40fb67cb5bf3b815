"""Pins of the FP64 oracle of NC-LS (the domain-transform normalised convolution embedded in
place of the BLF, Section III-D) against closed forms, scipy and a brute-force loop (no GPU)."""
import math

import numpy as np
import pytest
import scipy.ndimage as ndi

import oracle


def _rng(seed):
    return np.random.default_rng(seed)


def test_schedule_variances_sum_to_sigma_s_squared_and_halve():
    rs = oracle.nc_schedule(6.0, 3)
    sig = [r / math.sqrt(3.0) for r in rs]
    assert abs(sum(s * s for s in sig) - 36.0) < 1e-12
    assert abs(sig[0] / sig[1] - 2.0) < 1e-12 and abs(sig[1] / sig[2] - 2.0) < 1e-12


def test_domain_transform_by_hand():
    s = np.array([[0.0, 0.5, 0.5, 0.25]])
    ct, T = oracle.domain_transform(s, 2.0, axis=1)
    # increments 1 + 2 |ds|: 2.0, 1.0, 1.5; wrap increment 1 + 2 |0 - 0.25| = 1.5 (all exact)
    np.testing.assert_array_equal(ct, [[0.0, 2.0, 3.0, 4.5]])
    np.testing.assert_array_equal(T, [6.0])
    np.testing.assert_array_equal(oracle.increments(s, 2.0, axis=1), [[1.5, 2.0, 1.0, 1.5]])


def test_transform_distances_are_exact_sums_of_the_increments():
    """The distance a pass compares with r, against exact rational arithmetic: every margin
    |ct(i + d) - ct(i)| - r equals the exact sum of 1 + a |s[j] - s[j-1]| over the steps between
    i and i + d (periodic, several periods for a short line) minus r, to FP64 rounding."""
    from fractions import Fraction
    s = _rng(4).normal(scale=0.4, size=(2, 9))
    ss, sr = 3.0, 0.25
    a = float(np.float32(ss)) / float(np.float32(sr))
    r1 = oracle.nc_schedule(float(np.float32(ss)), 1)[0]
    seen = 0
    for k, axis, d, m in oracle.nc_margins(s, ss, sr, n_iter=1):
        if axis != 1:
            continue
        for row in range(2):
            for i in range(9):
                acc = Fraction(0)
                lo, hi = (i, i + d) if d > 0 else (i + d, i)
                for j in range(lo + 1, hi + 1):
                    acc += 1 + Fraction(a) * abs(Fraction(s[row, j % 9]) - Fraction(s[row, (j - 1) % 9]))
                assert abs(Fraction(m[row, i]) - (acc - Fraction(r1))) <= Fraction(1, 2 ** 40)
                seen += 1
    assert seen == 2 * 9 * 2 * int(math.floor(r1))


def _nc_pass_brute(v, ct, T, r):
    """Every sample of the previous, current and next period, scanned one by one (the inclusion
    test written out on the FP64 running sum and period)."""
    n = v.size
    out = np.empty(n)
    for i in range(n):
        acc = cnt = 0.0
        for k in (-1, 0, 1):
            for j in range(n):
                if abs(ct[j] + k * T - ct[i]) <= r:
                    acc += v[j]
                    cnt += 1
        out[i] = acc / cnt
    return out


@pytest.mark.parametrize("r", [0.7, 2.5, 4.0])
def test_nc_pass_matches_a_brute_force_scan(r):
    s = _rng(1).normal(scale=0.3, size=(1, 13))
    ct, T = oracle.domain_transform(s, 1.5, axis=1)
    got = oracle.nc_pass(s, oracle.increments(s, 1.5, axis=1), r, axis=1)
    np.testing.assert_allclose(got[0], _nc_pass_brute(s[0], ct[0], T[0], r), rtol=0, atol=1e-14)


def test_a_flipped_decision_is_the_decision_at_a_slightly_other_radius():
    """With r equal to one pair's transform distance, that pair is inside (<=) from both ends;
    reversing those two decisions equals the pass at a radius a hair smaller, where only that
    pair leaves."""
    s = _rng(5).normal(scale=0.3, size=(1, 15))
    inc = oracle.increments(s, 2.0, axis=1)
    i0, d0 = 6, 2
    r = float(inc[0, i0 + 1] + inc[0, i0 + 2])          # distance from 6 to 8
    flip = {d0: np.zeros_like(s, dtype=bool), -d0: np.zeros_like(s, dtype=bool)}
    flip[d0][0, i0] = True                               # 6 -> 8
    flip[-d0][0, i0 + d0] = True                         # 8 -> 6
    got = oracle.nc_pass(s, inc, r, axis=1, flip=flip)
    want = oracle.nc_pass(s, inc, r * (1 - 1e-12), axis=1)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-15)
    assert np.max(np.abs(got - oracle.nc_pass(s, inc, r, axis=1))) > 1e-3


def test_infinite_sigma_r_is_a_cascade_of_periodic_box_means():
    g = _rng(2).normal(size=(17, 23))
    want = g.copy()
    for r in oracle.nc_schedule(4.0, 3):
        size = 2 * int(math.floor(r)) + 1
        want = ndi.uniform_filter1d(want, size, axis=1, mode="wrap")
        want = ndi.uniform_filter1d(want, size, axis=0, mode="wrap")
    np.testing.assert_allclose(oracle.nc_filter(g, 4.0, math.inf), want, rtol=0, atol=1e-13)


def test_constant_field_and_separated_regions():
    np.testing.assert_allclose(oracle.nc_filter(np.full((9, 11), 0.3), 3.0, 0.1), 0.3, atol=1e-15)
    # a jump of 1 with a = sigma_s / sigma_r = 300 puts the two sides 300 apart in the transformed
    # domain, far beyond every radius: no averaging across the edge
    g = np.zeros((12, 20))
    g[:, 10:] = 1.0
    np.testing.assert_allclose(oracle.nc_filter(g, 3.0, 0.01), g, rtol=0, atol=1e-15)


def test_ncls_special_cases():
    f = _rng(3).uniform(size=(2, 16, 18))
    np.testing.assert_allclose(oracle.ncls(f, 0.0, 3.0, 0.1), f, rtol=0, atol=1e-14)
    c = np.full((10, 12), 0.7)
    np.testing.assert_allclose(oracle.ncls(c, 30.0, 3.0, 0.1), c, rtol=0, atol=1e-13)
    u = oracle.ncls(f, 20.0, 3.0, 0.1)
    np.testing.assert_allclose(u.sum(axis=(1, 2)), f.sum(axis=(1, 2)), rtol=1e-12)
    np.testing.assert_array_equal(oracle.ncls(f, 20.0, 3.0, 0.1, iters=2),
                                  oracle.ncls(u, 20.0, 3.0, 0.1))
