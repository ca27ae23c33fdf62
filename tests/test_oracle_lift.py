"""Pins of the oracle's lift to rational numbers (no GPU): the Chinese
remainder result against brute force and its defining congruences; rational
reconstruction against an exhaustive table on a small modulus, against
fractions it must recover, and against the uniqueness bound."""
import math
import random

import pytest

from oracle import lift
from oracle import is_prime


def test_crt_brute_force_small():
    primes = [3, 5, 7]
    P = 105
    for r in [(0, 0, 0), (1, 2, 3), (2, 4, 6), (1, 0, 0)]:
        want = [x for x in range(P) if all(x % p == ri for p, ri in zip(primes, r))]
        assert want == [lift.crt(r, primes)]


def test_crt_congruences_large():
    rnd = random.Random(1)
    primes = [p for p in range(2**63 - 1, 2**63 - 2000, -2) if is_prime(p)][:6]
    assert len(primes) == 6
    for L in range(1, 7):
        ps = primes[:L]
        P = math.prod(ps)
        for _ in range(20):
            r = [rnd.randrange(p) for p in ps]
            x = lift.crt(r, ps)
            assert 0 <= x < P and all(x % p == ri for p, ri in zip(ps, r))


def test_rational_reconstruct_exhaustive_small():
    """Every x mod P = 101 * 103: the oracle returns the unique fraction in
    the bound when there is one, and None exactly when there is none."""
    P = 101 * 103
    N = lift.bound(P)
    assert 2 * N * N < P <= 2 * (N + 1) ** 2 + 1
    table = {}
    for d in range(1, N + 1):
        for n in range(-N, N + 1):
            if math.gcd(abs(n), d) == 1:
                x = n * pow(d, -1, P) % P
                assert x not in table          # uniqueness
                table[x] = (n, d)
    for x in range(P):
        assert lift.rational_reconstruct(x, P) == table.get(x)


def test_rational_reconstruct_recovers_fractions():
    rnd = random.Random(2)
    primes = [p for p in range(2**63 - 1, 2**63 - 4000, -2) if is_prime(p)][:8]
    for L in (1, 2, 3, 5, 8):
        ps = primes[:L]
        P = math.prod(ps)
        N = lift.bound(P)
        for _ in range(30):
            d = rnd.randrange(1, N + 1)
            n = rnd.randrange(-N, N + 1)
            g = math.gcd(abs(n), d)
            n, d = n // g, d // g
            res = [[n * pow(d, -1, p) % p] for p in ps]
            assert lift.rational_lift(res, ps) == [(n, d)]
        # just past the bound: another fraction or none, never the true one
        n, d = N + 1, 1
        got = lift.rational_reconstruct(n % P, P)
        assert got != (n, d)


@pytest.mark.parametrize("x,want", [(0, (0, 1)), (1, (1, 1))])
def test_rational_reconstruct_special(x, want):
    P = (2**63 - 25) * (2**63 - 165)
    assert lift.rational_reconstruct(x, P) == want
    assert lift.rational_reconstruct(P - 1, P) == (-1, 1)
