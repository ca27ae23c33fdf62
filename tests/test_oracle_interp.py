"""Pins for the oracle's Newton (Eq. newton) and Thiele (Eq. thiele)
interpolation (CPU only)."""
import random

import numpy as np
import pytest

from tests import pyref
from tests.pyref import P63


def _distinct(rnd, n):
    s = []
    while len(s) < n:
        x = rnd.randrange(P63)
        if x not in s:
            s.append(x)
    return s


def test_newton_two_points_closed_form(orc):
    rnd = random.Random(20)
    for _ in range(20):
        x0, x1 = _distinct(rnd, 2)
        f0, f1 = rnd.randrange(P63), rnd.randrange(P63)
        c = [int(v) for v in orc.newton([x0, x1], [f0, f1])]
        slope = (f1 - f0) * pyref.inv(x1 - x0) % P63
        assert c == [(f0 - slope * x0) % P63, slope]


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8])
def test_newton_matches_lagrange(orc, n):
    rnd = random.Random(21 + n)
    xs = _distinct(rnd, n)
    fs = [rnd.randrange(P63) for _ in range(n)]
    assert [int(v) for v in orc.newton(xs, fs)] == pyref.lagrange_coeffs(xs, fs)


def test_newton_evaluate_back_and_truth(orc):
    rnd = random.Random(22)
    n = 21
    xs = _distinct(rnd, n)
    g = [rnd.randrange(P63) for _ in range(n)]
    fs = [pyref.poly_eval(g, x) for x in xs]
    c = [int(v) for v in orc.newton(xs, fs)]
    assert c == g
    for x, f in zip(xs, fs):
        assert pyref.poly_eval(c, x) == f


def test_newton_batched_columns(orc):
    rnd = random.Random(23)
    n, nt = 6, 9
    xs = _distinct(rnd, n)
    vals = np.array([[rnd.randrange(P63) for _ in range(nt)] for _ in range(n)], dtype=np.uint64)
    out = orc.newton_batched(xs, vals)
    for j in range(nt):
        assert [int(v) for v in out[:, j]] == pyref.lagrange_coeffs(xs, [int(v) for v in vals[:, j]])


def test_newton_duplicate_nodes(orc):
    with pytest.raises(orc.OracleError) as e:
        orc.newton([4, 9, 4], [1, 2, 3])
    assert e.value.status == orc.SINGULAR


def _ratfun(rnd, dn, dd):
    N = [rnd.randrange(P63) for _ in range(dn + 1)]
    D = [rnd.randrange(P63) for _ in range(dd + 1)]
    N[-1] = N[-1] or 1
    D[-1] = D[-1] or 1
    return N, D


@pytest.mark.parametrize("dn,dd", [(0, 0), (1, 0), (0, 1), (3, 0), (0, 3), (2, 2), (5, 3), (3, 5), (15, 15), (7, 12)])
def test_thiele_recovers_rational_function(orc, dn, dd):
    rnd = random.Random(1000 + 31 * dn + dd)
    N, D = _ratfun(rnd, dn, dd)
    n = 2 * max(dn, dd) + 2
    xs = _distinct(rnd, n)
    fs = [pyref.poly_eval(N, x) * pyref.inv(pyref.poly_eval(D, x)) % P63 for x in xs]
    num, den = orc.thiele(xs, fs, dn, dd)
    num, den = [int(v) for v in num], [int(v) for v in den]
    # same function: num * D == N * den, exact degrees, den(x_0) = 1
    assert pyref.poly_trim(pyref.poly_mul(num, D)) == pyref.poly_trim(pyref.poly_mul(N, den))
    assert len(num) - 1 == dn and len(den) - 1 == dd
    assert pyref.poly_eval(den, xs[0]) == 1
    # and the unique such pair: N, D scaled by 1 / D(x_0)
    s = pyref.inv(pyref.poly_eval(D, xs[0]))
    assert num == [c * s % P63 for c in N]
    assert den == [c * s % P63 for c in D]


def test_thiele_constant(orc):
    num, den = orc.thiele([3, 5, 8], [7, 7, 7], 2, 2)
    assert [int(v) for v in num] == [7] and [int(v) for v in den] == [1]


def test_thiele_too_few_points(orc):
    rnd = random.Random(40)
    N, D = _ratfun(rnd, 4, 4)
    xs = _distinct(rnd, 8)    # 2*4+2 = 10 needed
    fs = [pyref.poly_eval(N, x) * pyref.inv(pyref.poly_eval(D, x)) % P63 for x in xs]
    with pytest.raises(orc.OracleError) as e:
        orc.thiele(xs, fs, 4, 4)
    assert e.value.status == orc.DEGREE


def test_thiele_degree_bound(orc):
    rnd = random.Random(41)
    N, D = _ratfun(rnd, 3, 2)
    xs = _distinct(rnd, 10)
    fs = [pyref.poly_eval(N, x) * pyref.inv(pyref.poly_eval(D, x)) % P63 for x in xs]
    with pytest.raises(orc.OracleError) as e:
        orc.thiele(xs, fs, 2, 2)   # numerator bound too small
    assert e.value.status == orc.DEGREE
