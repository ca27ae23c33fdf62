"""Pins for the oracle's modular arithmetic and random streams (CPU only).

The oracle's routines are compared with Python's exact integers, which share
nothing with the oracle's C code, and with published test vectors.
"""
import random

import pytest

from tests.pyref import P63

EDGE = [0, 1, 2, P63 - 1, P63 - 2, 2**32 - 1, 2**32, 2**32 + 1, 2**62, 2**62 + 12345, 25, P63 // 2]


def test_p63_is_prime(orc):
    assert orc.is_prime(P63)
    sympy = pytest.importorskip("sympy")
    assert sympy.isprime(P63)


def test_is_prime_matches_sympy(orc):
    sympy = pytest.importorskip("sympy")
    rnd = random.Random(5)
    nums = [rnd.getrandbits(63) | 1 for _ in range(300)] + [2**61 - 1, 2**64 - 59, 3215031751, 341550071728321]
    for n in nums:
        assert orc.is_prime(n) == sympy.isprime(n), n


def test_mulmod_edges_and_random(orc):
    rnd = random.Random(1)
    vals = EDGE + [rnd.randrange(P63) for _ in range(200)]
    for a in vals:
        for b in EDGE:
            assert orc.mulmod(a, b) == a * b % P63
    for _ in range(5000):
        a, b = rnd.randrange(P63), rnd.randrange(P63)
        assert orc.mulmod(a, b) == a * b % P63


def test_add_sub_mod(orc):
    rnd = random.Random(2)
    for _ in range(2000):
        a, b = rnd.randrange(P63), rnd.randrange(P63)
        assert orc.addmod(a, b) == (a + b) % P63
        assert orc.submod(a, b) == (a - b) % P63
    for a in EDGE:
        for b in EDGE:
            assert orc.addmod(a, b) == (a + b) % P63
            assert orc.submod(a, b) == (a - b) % P63


def test_powmod_and_fermat(orc):
    rnd = random.Random(3)
    for _ in range(300):
        a, e = rnd.randrange(P63), rnd.getrandbits(64)
        assert orc.powmod(a, e) == pow(a, e, P63)
    for a in [1, 2, 3, P63 - 1] + [rnd.randrange(1, P63) for _ in range(20)]:
        assert orc.powmod(a, P63 - 1) == 1


def test_invmod(orc):
    rnd = random.Random(4)
    for a in [1, 2, P63 - 1, 2**32] + [rnd.randrange(1, P63) for _ in range(2000)]:
        i = orc.invmod(a)
        assert a * i % P63 == 1
    assert orc.invmod(0) == 0
    # a small composite modulus: not invertible -> 0
    assert orc.invmod(6, 9) == 0
    assert orc.invmod(2, 9) == 5


def test_splitmix_published_vectors(orc):
    # splitmix64 seeded with 0: the first three outputs of the published
    # reference sequence (Steele, Lea, Flood 2014; Vigna's splitmix64.c)
    want = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    assert [orc.splitmix_at(0, n) for n in range(3)] == want
    from paper_2505_24256_gb300 import workloads as W
    assert [W.splitmix_at(0, n) for n in range(3)] == want
    rnd = random.Random(6)
    for _ in range(50):
        k, n = rnd.getrandbits(64), rnd.randrange(1 << 40)
        assert W.splitmix_at(k, n) == orc.splitmix_at(k, n)


def test_workload_residues_in_range():
    from paper_2505_24256_gb300 import workloads as W
    st = W.Stream(7, 1)
    r = st.residues(10000)
    assert r.min() >= 1 and int(r.max()) < P63
    d = W.Stream(7, 2).distinct_residues(500)
    assert len(set(int(x) for x in d)) == 500
