"""Pin of the oracle's compensated sum on arrays above 2^20 elements (the
branch every reference norm at N >= 21 and every BEGIN MEASUREMENT reference
at N >= 22 goes through): a Neumaier sum down 1024 rows, then the exactly
rounded sum of the column totals.  Checked against math.fsum (the correctly
rounded sum) on arrays built to defeat a plain or a half-compensated sum:
values spread over 16 orders of magnitude, cancelling pairs planted far
apart, and a ragged tail that is not a multiple of the row count."""
import math

import numpy as np
import pytest

from oracle import statevec as sv

U = 2.0 ** -53


def adversarial(n, seed):
    g = np.random.default_rng(seed)
    x = g.standard_normal(n) * 10.0 ** g.uniform(-8, 8, n)
    # planted cancellation: +big at one place, -big at a far one, so the
    # running sums swing by 1e16 while the total stays small
    idx = g.choice(n, 2 * 64, replace=False)
    big = 10.0 ** g.uniform(14, 16, 64)
    x[idx[:64]] = big
    x[idx[64:]] = -big
    return x


def neumaier_bound(x, total):
    # a Neumaier sum of n_rows terms per column leaves s + c within
    # n_rows u^2 sum|partial sums| <= n_rows^2 u^2 sum|x| of the column's exact
    # total; the exactly rounded sum of every s and c adds one rounding
    return 2 * U * abs(total) + 2 * 1024 * 1024 * U * U * float(np.sum(np.abs(x)))


@pytest.mark.parametrize("n,seed", [((1 << 21) + 37, 1), (1 << 22, 2), ((1 << 22) + 1023, 3)])
def test_csum_large_against_fsum(n, seed):
    x = adversarial(n, seed)
    exact = math.fsum(x.tolist())
    got = sv.csum(x)
    assert abs(got - exact) <= neumaier_bound(x, exact)
    # the same data in another order: the bound holds again
    y = x[np.random.default_rng(seed + 10).permutation(n)]
    assert abs(sv.csum(y) - exact) <= neumaier_bound(y, exact)
    # a plain float64 sum misses by far more than the bound (the pin can fail)
    plain = float(np.cumsum(x)[-1])
    assert abs(plain - exact) > 10 * neumaier_bound(x, exact)


def test_csum_large_exact_cases():
    # sums that are exact in binary: ones, alternating +-2^k, and a tail
    n = (1 << 21) + 5
    assert sv.csum(np.ones(n)) == float(n)
    x = np.where(np.arange(n) % 2 == 0, 2.0 ** 40, -(2.0 ** 40))
    x[-1] = 3.0
    assert sv.csum(x) == math.fsum(x.tolist())
    # tiny values under a huge one that later cancels: only compensation keeps them
    y = np.full(1 << 21, 1e-3)
    y[0] = 1e17
    y[-1] = -1e17
    assert abs(sv.csum(y) - 1e-3 * ((1 << 21) - 2)) <= 1e-9
