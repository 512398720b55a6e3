"""Pins for the oracle's step 6: the nearest-rank 99th percentile of the
voxel-averaged |E| per tissue and over the whole body (Sec. II-A step 6,
Sec. III-E).

The nearest-rank value v of n numbers at level p is fixed by two counts,
checked here in exact rational arithmetic: at least p*n of the numbers are
<= v and fewer than p*n are < v.  Besides that defining property the oracle
is checked against closed forms (a permutation of 1..n), numpy's
inverted-CDF quantile where p*n is far from an integer, and the edge cases
(p = 1 is the maximum, tiny p the minimum, empty groups, air voxels and
out-of-range labels).
"""

import math
from fractions import Fraction

import numpy as np
import pytest


def _check_nearest_rank(values, v, p):
    """v is the nearest-rank p-quantile of values (exact arithmetic)."""
    n = len(values)
    need = Fraction(p) * n
    assert sum(1 for x in values if x <= v) >= need
    assert sum(1 for x in values if x < v) < need
    assert v in values


def test_nearest_rank_exact(oracle_mod):
    for p in (0.99, 0.5, 0.25, 1.0, 0.1, 0.999, 1e-300, 0.3):
        for n in (1, 2, 3, 4, 7, 10, 99, 100, 101, 1000, 12345, 8954036, 2**40 + 3):
            k = oracle_mod.nearest_rank(p, n)
            assert k == max(1, math.ceil(Fraction(p) * n)), (p, n, k)
    # the binary value of 0.99 lies just below 0.99, so 0.99 * 100 ranks 99
    assert oracle_mod.nearest_rank(0.99, 100) == 99
    assert oracle_mod.nearest_rank(0.5, 4) == 2
    assert oracle_mod.nearest_rank(0.99, 0) == 0


def test_percentile_defining_property(oracle_mod):
    rng = np.random.default_rng(99)
    shape = (6, 7, 9)
    sigma = np.where(rng.random(shape) < 0.25, 0.0, rng.uniform(0.1, 1.0, shape))
    # few distinct values: many ties, the hard case for a rank rule
    E = rng.integers(0, 12, shape).astype(np.float64) * 0.125
    lab = rng.integers(-1, 5, shape).astype(np.int32)
    for p in (0.99, 0.5, 0.9, 0.01, 1.0):
        out, cnt = oracle_mod.percentile(sigma, E, lab, 4, p)
        cond = sigma > 0
        for t in range(5):
            sel = cond & (lab == t) if t < 4 else cond
            vals = list(E[sel])
            assert cnt[t] == len(vals)
            if vals:
                _check_nearest_rank(vals, out[t], p)
            else:
                assert math.isnan(out[t])


def test_percentile_permutation_closed_form(oracle_mod):
    rng = np.random.default_rng(7)
    n = 1000
    E = rng.permutation(np.arange(1, n + 1, dtype=np.float64)).reshape(10, 10, 10)
    sigma = np.ones_like(E)
    lab = np.zeros(E.shape, dtype=np.int32)
    out, cnt = oracle_mod.percentile(sigma, E, lab, 1, 0.99)
    assert out[0] == 990.0 and out[1] == 990.0 and cnt[0] == n
    out, _ = oracle_mod.percentile(sigma, E, lab, 1, 1.0)
    assert out[0] == n
    out, _ = oracle_mod.percentile(sigma, E, lab, 1, 1e-9)
    assert out[0] == 1.0


def test_percentile_matches_numpy_inverted_cdf(oracle_mod):
    rng = np.random.default_rng(2010)
    shape = (16, 12, 20)
    sigma = rng.uniform(0.02, 2.0, shape)
    E = rng.lognormal(-3.0, 1.0, shape)
    lab = rng.integers(0, 6, shape).astype(np.int32)
    p = 0.99
    out, cnt = oracle_mod.percentile(sigma, E, lab, 6, p)
    for t in range(7):
        vals = E[lab == t] if t < 6 else E.reshape(-1)
        frac = p * vals.size - math.floor(p * vals.size)
        if 0.01 < frac < 0.99:   # far from an integer: numpy's rounding agrees
            assert out[t] == np.percentile(vals, 100 * p, method="inverted_cdf")
        _check_nearest_rank(list(vals), out[t], p)


def test_percentile_air_and_labels(oracle_mod):
    E = np.array([[[5.0, 1.0, 2.0, 3.0]]])
    sigma = np.array([[[0.0, 1.0, 1.0, 1.0]]])    # the 5.0 voxel is air
    lab = np.array([[[0, 0, 7, -1]]], dtype=np.int32)  # 7 and -1: body only
    out, cnt = oracle_mod.percentile(sigma, E, lab, 2, 1.0)
    assert out[0] == 1.0 and cnt[0] == 1
    assert math.isnan(out[1]) and cnt[1] == 0
    assert out[2] == 3.0 and cnt[2] == 3
