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


# ---- the elementwise batch used by the device-arithmetic parity test --------

def _edge_pairs():
    rnd = random.Random(21)
    vals = EDGE + [rnd.randrange(P63) for _ in range(40)]
    return [(a, b) for a in vals for b in vals]


def test_arith_batch_products_and_sums(orc):
    import numpy as np
    pairs = _edge_pairs()
    a = np.array([x for x, _ in pairs], dtype=np.uint64)
    b = np.array([y for _, y in pairs], dtype=np.uint64)
    got = {op: orc.arith_batch(op, a, b) for op in ("mulmod", "add", "sub")}
    for i, (x, y) in enumerate(pairs):
        assert int(got["mulmod"][i]) == x * y % P63
        assert int(got["add"][i]) == (x + y) % P63
        assert int(got["sub"][i]) == (x - y) % P63


def test_arith_batch_reduce_and_shoup(orc):
    """reduce: (a 2^64 + b) mod p; shoup_pre: the floor of w 2^64 / p, pinned by
    its defining inequality; shoup_lazy: congruent to x w, in [0, 2p), and the
    exact value of Shoup's formula in Python integers."""
    import numpy as np
    rnd = random.Random(22)
    his = EDGE + [rnd.randrange(P63) for _ in range(300)]
    los = [0, 1, 2**64 - 1, 2**63, P63, 2 * P63] + [rnd.getrandbits(64) for _ in range(300)]
    hi = np.array(his[:len(los)] + his[:len(los)], dtype=np.uint64)[:len(los)]
    lo = np.array(los, dtype=np.uint64)
    red = orc.arith_batch("reduce", hi, lo)
    for h, l_, r in zip(hi.tolist(), lo.tolist(), red.tolist()):
        assert r == ((h << 64) + l_) % P63
    w = np.array(his, dtype=np.uint64)
    pre = orc.arith_batch("shoup_pre", w)
    for wi, q in zip(w.tolist(), pre.tolist()):
        assert q * P63 <= wi << 64 < (q + 1) * P63
    xs = np.array([0, 1, 2**64 - 1, 2**63, 2 * P63 - 1] + [rnd.getrandbits(64) for _ in range(len(his) - 5)],
                  dtype=np.uint64)
    lazy = orc.arith_batch("shoup_lazy", xs, w)
    for x, wi, q, r in zip(xs.tolist(), w.tolist(), pre.tolist(), lazy.tolist()):
        assert r % P63 == x * wi % P63 and r < 2 * P63
        assert r == (x * wi - ((x * q) >> 64) * P63) % 2**64


def test_arith_batch_pow_inv_dot(orc):
    import numpy as np
    rnd = random.Random(23)
    a = np.array([1, 2, P63 - 1, 2**32 + 1] + [rnd.randrange(1, P63) for _ in range(200)], dtype=np.uint64)
    e = np.array([P63 - 1] * a.size, dtype=np.uint64)
    assert (orc.arith_batch("pow", a, e) == 1).all()                    # Fermat
    e2 = np.array([rnd.getrandbits(64) for _ in range(a.size)], dtype=np.uint64)
    for x, y, r in zip(a.tolist(), e2.tolist(), orc.arith_batch("pow", a, e2).tolist()):
        assert r == pow(x, y, P63)
    for op in ("inv", "batch_inv"):
        inv = orc.arith_batch(op, a)
        for x, r in zip(a.tolist(), inv.tolist()):
            assert x * r % P63 == 1
        assert int(orc.arith_batch(op, np.zeros(1, dtype=np.uint64))[0]) == 0
    # dot: (p-1)^2 = 1 mod p, so 2^16 products of (p-1)(p-1) sum to 2^16
    n = 1 << 16
    full = np.full(n, P63 - 1, dtype=np.uint64)
    assert int(orc.arith_batch("dot", full, full, length=n)[0]) == n
    g = 7
    x = np.array([rnd.randrange(P63) for _ in range(g * 50)], dtype=np.uint64)
    y = np.array([rnd.randrange(P63) for _ in range(g * 50)], dtype=np.uint64)
    d = orc.arith_batch("dot", x, y, length=50)
    for i in range(g):
        assert int(d[i]) == sum(int(x[i * 50 + t]) * int(y[i * 50 + t]) for t in range(50)) % P63
