"""Device modular arithmetic against the oracle, operand by operand.

zr_check_arith applies the step kernels' own primitives (zr_arith.cuh:
the Moller-Granlund reduction, Shoup's precomputed-quotient product, the
160-bit deferred multiply-accumulate, Fermat inversion, Montgomery's batch
inversion) to operand arrays; the oracle's zro_arith_batch is the plain
128-bit definition (Sec. 2.1; Sec. 2.2 for the once-reduced dot product).
Bit-exact on edges, on ten million random operands, on lazy inputs in
[p, 2^64) and on sums of up to 2^24 products of (p-1)^2.

The reduction has two correction steps.  For p = 2^63 - 25 the normalised
divisor is d = 2p = 2^64 - 50 and the precomputed reciprocal is v = 50, so
with X = 50 n1 + n0 the first quotient estimate is n1 + floor(X / 2^64) + 1
while the true quotient is n1 + floor(X / (2^64 - 50)): the estimate is one
too large (the first correction runs, almost always) or exact, and when it
is exact the remainder is below 50 k while the estimate's low word is above
2^64 - 50 k, so the second correction can never run for this prime.  The
smallest prime above 2^32 reaches it on about 8% of random operands; the
tests count both corrections on both primes.
"""
import numpy as np
import pytest

from tests.gpuutil import d64, h64
from tests.pyref import P63

pytestmark = pytest.mark.gpu

P_SMALL = 4294967311          # the smallest prime above 2^32


@pytest.fixture(scope="module")
def env():
    import torch

    import __graft_entry__ as ge
    from paper_2505_24256_gb300 import zr

    ge.build()
    assert torch.cuda.is_available()
    ctxs = {P63: zr.Context(P63), P_SMALL: zr.Context(P_SMALL)}
    yield zr, ctxs
    for c in ctxs.values():
        c.close()


def edges(p):
    e = [0, 1, 2, 3, 25, p - 1, p - 2, p - 3, p // 2, p // 2 + 1, 2**32 - 1, 2**32, 2**32 + 1, 2**31, 2**33 - 1]
    if p > 2**62 + 2:
        e += [2**62 - 1, 2**62, 2**62 + 1]
    return sorted({x % p for x in e})


def uniform(rng, n, p):
    return (rng.integers(0, 2**63, size=n, dtype=np.uint64) * np.uint64(2) +
            rng.integers(0, 2, size=n, dtype=np.uint64)) % np.uint64(p)


def run(env, p, op, a, b=None, length=1, count=False):
    import torch
    zr, ctxs = env
    ctx = ctxs[p]
    a = np.ascontiguousarray(a, dtype=np.uint64)
    n = a.size // length if op == "dot" else a.size
    da = d64(a)
    db = d64(b) if b is not None else None
    out = torch.zeros(max(n, 1), dtype=torch.int64, device=da.device)
    hits = torch.zeros(4, dtype=torch.int32, device=da.device) if count else None
    ctx.check_arith(op, n, da, db, out, hits, length=length)
    got = h64(out)[:n]
    return (got, hits.cpu().numpy().astype(np.int64)) if count else got


def oracle_of(orc, op, a, b=None, p=P63, length=1):
    return orc.arith_batch(op, a, b, p=p, length=length)


@pytest.mark.parametrize("p", [P63, P_SMALL])
def test_products_sums_and_reductions(env, orc, p):
    rng = np.random.default_rng(31)
    E = np.array(edges(p), dtype=np.uint64)
    ea, eb = np.meshgrid(E, E)
    n = 10_000_000 if p == P63 else 2_000_000
    a = np.concatenate([ea.ravel(), uniform(rng, n, p)])
    b = np.concatenate([eb.ravel(), uniform(rng, n, p)])
    for op in ("mulmod", "add", "sub"):
        got = run(env, p, op, a, b)
        assert np.array_equal(got, oracle_of(orc, op, a, b, p)), op
    # reduce: high word < p, any low word; remainders near 0 and near p
    hi = np.concatenate([uniform(rng, n // 4, p), E, E])
    lo = np.concatenate([rng.integers(0, 2**63, size=n // 4, dtype=np.uint64) * np.uint64(2) + np.uint64(1),
                         np.full(E.size, 2**64 - 1, dtype=np.uint64), np.zeros(E.size, dtype=np.uint64)])
    got, hits = run(env, p, "reduce", hi, lo, count=True)
    assert np.array_equal(got, oracle_of(orc, "reduce", hi, lo, p))
    assert hits[0] > 0
    if p == P63:
        assert hits[1] == 0          # unreachable for this prime (module docstring)
    else:
        assert hits[1] > 0           # the second correction ran and gave the exact remainder


def test_shoup_forms(env, orc):
    rng = np.random.default_rng(32)
    p = P63
    E = np.array(edges(p), dtype=np.uint64)
    w = np.concatenate([E, uniform(rng, 1_000_000, p)])
    got, hits = run(env, p, "shoup_pre", w, count=True)
    assert np.array_equal(got, oracle_of(orc, "shoup_pre", w, None, p))
    assert hits[2] > 0
    # lazy products: x anywhere in [0, 2^64), including [p, 2p) and 2^64 - 1
    m = w.size
    x = rng.integers(0, 2**63, size=m, dtype=np.uint64) * np.uint64(2) + rng.integers(0, 2, size=m, dtype=np.uint64)
    x[: E.size] = E
    x[E.size: 2 * E.size] = E + np.uint64(p)
    x[-1] = np.uint64(2**64 - 1)
    x[-2] = np.uint64(2 * p - 1)
    got = run(env, p, "shoup_lazy", x, w)
    want = oracle_of(orc, "shoup_lazy", x, w, p)
    assert np.array_equal(got, want)
    assert (got < np.uint64(2 * p)).all()


@pytest.mark.parametrize("p", [P63, P_SMALL])
def test_pow_and_inverses(env, orc, p):
    rng = np.random.default_rng(33)
    E = np.array(edges(p), dtype=np.uint64)
    a = np.concatenate([E, uniform(rng, 200_000, p)])
    e = rng.integers(0, 2**63, size=a.size, dtype=np.uint64) * np.uint64(2) + np.uint64(1)
    e[:4] = [0, 1, p - 1, p - 2]
    assert np.array_equal(run(env, p, "pow", a, e), oracle_of(orc, "pow", a, e, p))
    for op in ("inv", "batch_inv"):
        x = a.copy()
        x[::97] = 0                      # zeros map to 0 and leave their warp's other inverses exact
        x = x[: x.size - 13]             # a ragged last warp
        got = run(env, p, op, x)
        assert np.array_equal(got, oracle_of(orc, op, x, None, p)), op


def test_long_dot_products(env, orc):
    p = P63
    rng = np.random.default_rng(34)
    # 2^24 products of (p-1)^2 = 1 (mod p) in one 160-bit accumulator
    n = 1 << 24
    full = np.full(n, p - 1, dtype=np.uint64)
    got, hits = run(env, p, "dot", full, full, length=n, count=True)
    assert int(got[0]) == n % p
    # 2^20 products of the largest residue with the largest 64-bit-range partner
    n2 = 1 << 20
    a = np.full(n2, p - 1, dtype=np.uint64)
    b = np.full(n2, p - 2, dtype=np.uint64)
    assert int(run(env, p, "dot", a, b, length=n2)[0]) == int(oracle_of(orc, "dot", a, b, p, length=n2)[0])
    # 4096 random groups of 997 terms, and groups of one term
    g, L = 4096, 997
    a = uniform(rng, g * L, p)
    b = uniform(rng, g * L, p)
    assert np.array_equal(run(env, p, "dot", a, b, length=L), oracle_of(orc, "dot", a, b, p, length=L))
    assert np.array_equal(run(env, p, "dot", a[:5000], b[:5000], length=1),
                          oracle_of(orc, "dot", a[:5000], b[:5000], p, length=1))


def test_invalid_arguments(env):
    zr, ctxs = env
    ctx = ctxs[P63]
    with pytest.raises(zr.ZrError):
        ctx.check_arith("dot", 1, None, None, None)
    st = ctx.L.zr_check_arith(ctx.handle, 42, 1, 1, None, None, None, None, None)
    assert st == zr.INVALID_ARG
