"""GPU parity: the lift of modular images to rational numbers
(zr_rational_lift) against the oracle's Chinese remaindering and rational
reconstruction, value by value, and end to end: rational-coefficient
functions reconstructed modulo several primes, then lifted."""
import math
import random

import numpy as np
import pytest

from paper_2505_24256_gb300 import workloads as W
from tests.gpuutil import d64, h64
from tests.pyref import P63

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def zr():
    import torch

    import __graft_entry__ as ge
    from paper_2505_24256_gb300 import zr as zrmod

    ge.build()
    assert torch.cuda.is_available()
    return zrmod


@pytest.fixture(scope="module")
def ctx(zr):
    c = zr.Context(P63)
    yield c
    c.close()


@pytest.fixture(scope="module")
def primes():
    from oracle import is_prime
    ps = [p for p in range(2**63 - 25, 2**63 - 6000, -2) if is_prime(p)][:8]
    assert len(ps) == 8
    return ps


def gpu_lift(zr, ctx, ps, res_rows):
    import torch
    L, n = len(ps), len(res_rows[0])
    words = zr.lift_words(L) + 1      # one word more than needed: extension checked too
    res = d64(np.array(res_rows, dtype=np.uint64).reshape(L, n))
    num = torch.zeros((n, words), dtype=torch.int64, device="cuda")
    den = torch.zeros((n, words), dtype=torch.int64, device="cuda")
    ok = torch.zeros(n, dtype=torch.int32, device="cuda")
    ctx.rational_lift(ps, res, n, words, num, den, ok)
    hn, hd, hok = h64(num), h64(den), ok.cpu().numpy()
    out = []
    for j in range(n):
        if hok[j]:
            out.append((zr.words_to_int(hn[j], True), zr.words_to_int(hd[j], False)))
        else:
            assert not hn[j].any() and not hd[j].any()
            out.append(None)
    return out


def cases(rnd, ps, n):
    """Recoverable fractions of every size up to the bound, values at and
    past the bound, zero, +-1, and uniform residues."""
    P = math.prod(ps)
    N = math.isqrt((P - 1) // 2)
    vals = []
    for j in range(n):
        kind = j % 6
        if kind == 0:
            vals.append(rnd.randrange(P))
            continue
        if kind == 1:
            bits = rnd.randrange(1, N.bit_length() + 1)
            nn, dd = rnd.randrange(-(1 << bits), 1 << bits), rnd.randrange(1, 1 << bits)
        elif kind == 2:
            nn, dd = rnd.choice([0, 1, -1, N, -N, N + 1, -(N + 1)]), rnd.choice([1, 1, N, N + 1, 2])
        elif kind == 3:
            nn, dd = rnd.randrange(-N, N + 1), rnd.randrange(1, N + 1)
        elif kind == 4:
            nn, dd = rnd.randrange(-2**30, 2**30), rnd.randrange(1, 2**30)
        else:
            nn, dd = rnd.randrange(-N, N + 1) * 6, rnd.randrange(1, N + 1) * 6   # common factor
        if math.gcd(dd, P) != 1:
            dd += 1
        vals.append(nn * pow(dd, -1, P) % P)
    return [[v % p for v in vals] for p in ps]


@pytest.mark.parametrize("L", [1, 2, 3, 4, 5, 8])
def test_lift_matches_oracle(zr, ctx, primes, L):
    from oracle import lift
    rnd = random.Random(100 + L)
    ps = primes[:L]
    rows = cases(rnd, ps, 3000)
    got = gpu_lift(zr, ctx, ps, rows)
    want = lift.rational_lift(rows, ps)
    assert got == want
    assert sum(g is not None for g in got) > 1000


def test_lift_rejects_bad_moduli(zr, ctx, primes):
    import torch
    res = torch.zeros((2, 4), dtype=torch.int64, device="cuda")
    out = torch.zeros((4, 8), dtype=torch.int64, device="cuda")
    ok = torch.zeros(4, dtype=torch.int32, device="cuda")
    for bad in ([primes[0], primes[0]], [primes[0], 2**63 - 27], [primes[0], 97]):
        with pytest.raises(zr.ZrError) as ei:
            ctx.rational_lift(bad, res, 4, 8, out, out, ok)
        assert ei.value.status == zr.INVALID_ARG


def _images(frac, p):
    return [a * pow(b, -1, p) % p for a, b in frac]


def test_rational_coefficients_end_to_end(zr, primes):
    """A polynomial and a rational function with rational coefficients:
    reconstructed modulo three primes (one context each), then lifted."""
    rnd = random.Random(7)
    wl = W.poly_simplex_workload(901, 4, 7, 90)
    frac = []
    for _ in range(wl.exps.shape[0]):
        a, b = rnd.randrange(-2**40, 2**40), rnd.randrange(1, 2**40)
        a = a or 1
        g = math.gcd(abs(a), b)
        frac.append((a // g, b // g))
    rw = W.rational_simplex_workload(902, 3, 6, 30, 20)
    nfr = [(rnd.randrange(-10**9, 10**9) or 1, rnd.randrange(1, 10**9)) for _ in range(rw.Nexps.shape[0])]
    dfr = [(1, 1)] + [(rnd.randrange(-10**9, 10**9) or 1, rnd.randrange(1, 10**9)) for _ in range(rw.Dexps.shape[0] - 1)]
    nfr = [(a // math.gcd(abs(a), b), b // math.gcd(abs(a), b)) for a, b in nfr]
    dfr = [(a // math.gcd(abs(a), b), b // math.gcd(abs(a), b)) for a, b in dfr]
    ps = primes[:3]
    prow, nrow, drow = [], [], []
    for p in ps:
        c = zr.Context(p)
        try:
            (e, co), _, _ = c.reconstruct(4, wl.deg, wl.seed, wl.exps, np.array(_images(frac, p), dtype=np.uint64))
            assert np.array_equal(e, wl.exps)
            prow.append([int(x) for x in co])
            (Ne, Nc), (De, Dc), _ = c.reconstruct(3, rw.degN, rw.seed, rw.Nexps,
                                                  np.array(_images(nfr, p), dtype=np.uint64), rw.Dexps,
                                                  np.array(_images(dfr, p), dtype=np.uint64), degD=rw.degD)
            assert np.array_equal(Ne, rw.Nexps) and np.array_equal(De, rw.Dexps)
            nrow.append([int(x) for x in Nc])
            drow.append([int(x) for x in Dc])
        finally:
            c.close()
    ctx = zr.Context(P63)
    try:
        assert gpu_lift(zr, ctx, ps, prow) == frac
        assert gpu_lift(zr, ctx, ps, nrow) == nfr
        assert gpu_lift(zr, ctx, ps, drow) == dfr
        # one prime is too few for 80-bit fractions: rejected or different, never silently equal
        one = gpu_lift(zr, ctx, ps[:1], prow[:1])
        assert one != frac
    finally:
        ctx.close()
