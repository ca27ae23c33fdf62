"""Pins for the oracle's master polynomial, synthetic division and transposed
Vandermonde solve (CPU only).

Each pin is fixed by something other than the oracle itself: elementary
symmetric polynomials, polynomial identities checked with Python integers,
closed forms at T = 1 and T = 2, Gaussian elimination, and multiply-back.
"""
import itertools
import random

import numpy as np
import pytest

from tests import pyref
from tests.pyref import P63


def _nodes(rnd, T):
    s = set()
    while len(s) < T:
        s.add(rnd.randrange(1, P63))
    return list(s)


def test_master_poly_elementary_symmetric(orc):
    rnd = random.Random(10)
    for T in range(1, 5):
        v = _nodes(rnd, T)
        m = [int(x) for x in orc.master_poly(v)]
        assert m[T] == 1
        for l in range(T):
            # coefficient of z^l is (-1)^(T-l) e_{T-l}(v)
            d = T - l
            e = sum(np.prod([x for x in c], dtype=object) for c in itertools.combinations(v, d)) % P63
            assert m[l] == (-1) ** d * e % P63


def test_master_poly_roots_and_product(orc):
    rnd = random.Random(11)
    v = _nodes(rnd, 40)
    m = [int(x) for x in orc.master_poly(v)]
    for x in v:
        assert pyref.poly_eval(m, x) == 0
    ref = [1]
    for x in v:
        ref = pyref.poly_mul(ref, [(-x) % P63, 1])
    assert m == ref


def test_synthetic_division_identity(orc):
    rnd = random.Random(12)
    v = _nodes(rnd, 30)
    m = [int(x) for x in orc.master_poly(v)]
    for j in [0, 7, 29]:
        q = [int(x) for x in orc.synthetic_division(m, v[j])]
        assert len(q) == 30
        assert pyref.poly_mul([(-v[j]) % P63, 1], q) == m
        # q_j(v_j) = prod_{l != j} (v_j - v_l)
        den = 1
        for l, x in enumerate(v):
            if l != j:
                den = den * (v[j] - x) % P63
        assert pyref.poly_eval(q, v[j]) == den


def test_solve_T1_closed_form(orc):
    rnd = random.Random(13)
    for _ in range(20):
        v0, b0 = rnd.randrange(1, P63), rnd.randrange(P63)
        assert int(orc.tvandermonde_solve([v0], [[b0]], offset=0)[0, 0]) == b0
        assert int(orc.tvandermonde_solve([v0], [[b0]], offset=1)[0, 0]) == b0 * pyref.inv(v0) % P63


def test_solve_T2_closed_form(orc):
    rnd = random.Random(14)
    for _ in range(20):
        v0, v1 = _nodes(rnd, 2)
        b0, b1 = rnd.randrange(P63), rnd.randrange(P63)
        c = orc.tvandermonde_solve([v0, v1], [[b0, b1]], offset=0)[0]
        d = pyref.inv(v0 - v1)
        assert int(c[0]) == (b1 - v1 * b0) * d % P63
        assert int(c[1]) == (v0 * b0 - b1) * d % P63


@pytest.mark.parametrize("offset", [0, 1])
@pytest.mark.parametrize("T", [1, 3, 8, 17])
def test_solve_matches_gaussian_elimination(orc, T, offset):
    rnd = random.Random(100 + T + 1000 * offset)
    v = _nodes(rnd, T)
    S = 3
    b = [[rnd.randrange(P63) for _ in range(T)] for _ in range(S)]
    c = orc.tvandermonde_solve(v, b, offset=offset)
    A = [[pow(v[j], k + offset, P63) for j in range(T)] for k in range(T)]
    ref = pyref.solve_linear(A, [[b[s][k] for s in range(S)] for k in range(T)])
    for s in range(S):
        assert [int(x) for x in c[s]] == [ref[j][s] for j in range(T)]


def test_solve_multiply_back(orc):
    rnd = random.Random(15)
    T = 300
    v = _nodes(rnd, T)
    b = [[rnd.randrange(P63) for _ in range(T)] for _ in range(2)]
    c = orc.tvandermonde_solve(v, b, offset=0, nthreads=4)
    cj = [int(x) for x in c[1]]
    for k in range(0, T, 7):
        assert sum(cj[j] * pow(v[j], k, P63) for j in range(T)) % P63 == b[1][k]


def test_solve_generator_truth(orc):
    """b_k = sum_j a_j v_j^k with known a: the solve returns a."""
    rnd = random.Random(16)
    T = 120
    v = _nodes(rnd, T)
    a = [rnd.randrange(P63) for _ in range(T)]
    b = [sum(a[j] * pow(v[j], k, P63) for j in range(T)) % P63 for k in range(T)]
    assert [int(x) for x in orc.tvandermonde_solve(v, [b])[0]] == a


def test_solve_roots_subset(orc):
    rnd = random.Random(17)
    T = 200
    v = _nodes(rnd, T)
    b = np.array([[rnd.randrange(P63) for _ in range(T)] for _ in range(3)], dtype=np.uint64)
    full = orc.tvandermonde_solve(v, b)
    m = orc.master_poly(v)
    roots = [0, 5, 199, 77]
    sub = orc.tvandermonde_solve_roots(v, m, b, roots)
    assert np.array_equal(sub, full[:, roots])


def test_solve_singular(orc):
    assert orc.check_nodes([5, 7, 5]) == orc.SINGULAR
    assert orc.check_nodes([0, 7, 5], offset=1) == orc.SINGULAR
    assert orc.check_nodes([0, 7, 5], offset=0) == orc.OK
    with pytest.raises(orc.OracleError) as e:
        orc.tvandermonde_solve([3, 9, 3], [[1, 2, 3]])
    assert e.value.status == orc.SINGULAR


def test_anchor_values_definition(orc):
    rnd = random.Random(18)
    exps = np.array([[rnd.randrange(21) for _ in range(4)] for _ in range(50)], dtype=np.uint8)
    y = [rnd.randrange(1, P63) for _ in range(4)]
    v = orc.anchor_values(exps, 3, y)
    for j in range(50):
        assert int(v[j]) == pyref.monomial_value(exps[j, :3], y[:3])
