"""The O(T log^2 T) transposed Vandermonde solve (subproduct tree, scaled
remainder tree, power sums) against the oracle.

The solution is unique, so the fast path must give the oracle's values bit
for bit: element by element for T up to 2^14 + 5 (every transform size from
2^8 to 2^16, the column passes of transforms above 2^13, ragged last blocks,
both offsets, each way of computing the power sums: the direct T^2 kernel
up to 12288 including T = 2^13 + 1, the cluster's Newton iteration and
division step from 12289 to 2^14, Newton's inverse and a product above),
through full Zippel steps at T = 10^4 and T = 2^20 against generator truth,
in batches mixing both methods, and in reconstructions.
"""
import random

import numpy as np
import pytest

from paper_2505_24256_gb300 import workloads as W
from tests.gpuutil import d8, d64, h64, rand_nodes, rand_res, zeros8, zeros64
from tests.pyref import P63

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch

    import __graft_entry__ as ge
    from paper_2505_24256_gb300 import zr

    ge.build()
    assert torch.cuda.is_available()
    c = zr.Context(P63)
    yield c
    c.close()


def solve(ctx, v, b, offset, method):
    S, T = b.shape
    c = zeros64(S, T)
    ctx.solve_method(method)
    try:
        ctx.vandermonde_solve([dict(T=T, S=S, offset=offset, v=d64(v), b=d64(b), ldb=T, c=c, ldc=T)])
    finally:
        ctx.solve_method(0)
    return h64(c)


@pytest.mark.parametrize("T,S,offset", [(1, 1, 0), (2, 3, 1), (3, 2, 0), (127, 2, 0), (128, 3, 1), (129, 1, 0),
                                        (1000, 5, 0), (4097, 3, 1), (8193, 1, 0), (12288, 1, 0), (12289, 2, 1),
                                        (9000, 2, 0), (16384, 2, 1), (16389, 2, 1)])
def test_fast_solve_matches_oracle(ctx, orc, T, S, offset):
    rnd = random.Random(T * 7 + S)
    v = rand_nodes(rnd, T, P63)
    b = rand_res(rnd, (S, T), P63)
    want = orc.tvandermonde_solve(v, b, offset=offset)
    assert np.array_equal(solve(ctx, v, b, offset, ctx.SOLVE_FAST), want)


def test_fast_solve_edge_nodes(ctx, orc):
    """Nodes at the ends of the residue range, small consecutive nodes, and
    right-hand sides of zeros and of p - 1."""
    T = 700
    rnd = random.Random(5)
    base = [1, 2, 3, P63 - 1, P63 - 2, 2**32, 2**32 + 1, 2**62]
    v = np.array(base + [x for x in rand_nodes(rnd, T + 20, P63).tolist() if x not in base][:T - len(base)],
                 dtype=np.uint64)
    b = np.stack([np.zeros(T, dtype=np.uint64), np.full(T, P63 - 1, dtype=np.uint64), rand_res(rnd, (T,), P63)])
    for off in (0, 1):
        assert np.array_equal(solve(ctx, v, b, off, ctx.SOLVE_FAST), orc.tvandermonde_solve(v, b, offset=off))


def test_fast_solve_singular(ctx):
    from paper_2505_24256_gb300 import zr
    rnd = random.Random(6)
    v = rand_nodes(rnd, 600, P63)
    v[17] = v[400]
    b = rand_res(rnd, (2, 600), P63)
    with pytest.raises(zr.ZrError) as ei:
        solve(ctx, v, b, 0, ctx.SOLVE_FAST)
    assert ei.value.status == zr.SINGULAR


def test_both_methods_in_one_batch(ctx, orc):
    """Systems below and above the crossover in one call: each takes its
    method, and every result equals the oracle's."""
    rnd = random.Random(8)
    shapes = [(50, 3, 0), (3000, 2, 1), (700, 1, 0), (5000, 4, 0)]
    systems, want = [], []
    for T, S, off in shapes:
        v, b = rand_nodes(rnd, T, P63), rand_res(rnd, (S, T), P63)
        c = zeros64(S, T)
        systems.append(dict(T=T, S=S, offset=off, v=d64(v), b=d64(b), ldb=T, c=c, ldc=T))
        want.append(orc.tvandermonde_solve(v, b, offset=off))
    ctx.solve_method(0, 1000)
    try:
        ctx.vandermonde_solve(systems)
    finally:
        ctx.solve_method(0)
    for s, w in zip(systems, want):
        assert np.array_equal(h64(s["c"]), w)


def test_many_fast_entries_in_one_batch(ctx, orc):
    """Six systems above the crossover and one below in one call: the fast
    ones run on four streams of their own, two of them twice, each with its
    workspace slot; every result equals the oracle's."""
    rnd = random.Random(9)
    shapes = [(1100, 2, 0), (2048, 3, 1), (1500, 1, 0), (4100, 2, 0), (1200, 4, 1), (3333, 1, 0), (300, 2, 0)]
    systems, want = [], []
    for T, S, off in shapes:
        v, b = rand_nodes(rnd, T, P63), rand_res(rnd, (S, T), P63)
        c = zeros64(S, T)
        systems.append(dict(T=T, S=S, offset=off, v=d64(v), b=d64(b), ldb=T, c=c, ldc=T))
        want.append(orc.tvandermonde_solve(v, b, offset=off))
    ctx.solve_method(0, 1000)
    try:
        ctx.vandermonde_solve(systems)
    finally:
        ctx.solve_method(0)
    for sy, w in zip(systems, want):
        assert np.array_equal(h64(sy["c"]), w)


def step(ctx, wl, method):
    import torch
    fe, fc = d8(wl.exps), d64(wl.coef)
    f = ctx.poly(wl.nv, wl.exps.shape[0], fe, fc)
    y, cs, z = d64(wl.y), d64(wl.cs), d64(wl.z)
    b = zeros64(wl.S, wl.T)
    ctx.zippel_probes(f, wl.k, y, wl.S, cs, z, wl.T, 0, b, wl.T)
    del fe, fc
    ske = d8(wl.skel)
    cap = wl.T * wl.S
    oe, oc = zeros8(cap, wl.nv), zeros64(cap)
    ctx.solve_method(method)
    try:
        n = ctx.zippel_step(ctx.poly(wl.nv, wl.T, ske), wl.k, y, wl.S, cs, b, wl.T, 0, oe, oc, cap)
    finally:
        ctx.solve_method(0)
    torch.cuda.synchronize()
    return oe[:n].cpu().numpy(), h64(oc[:n])


def test_fast_step_workload_1e4(ctx):
    """The T = 10^4, S = 21 step through the fast path: generator truth."""
    wl = W.batched_step_1e4()
    e, c = step(ctx, wl, ctx.SOLVE_FAST)
    assert np.array_equal(e, wl.exps) and np.array_equal(c, wl.coef)


def test_fast_step_workload_2p20(ctx):
    """The T = 2^20, S = 9 step through the fast path: generator truth in full."""
    wl = W.large_step_2p20()
    e, c = step(ctx, wl, ctx.SOLVE_FAST)
    assert np.array_equal(e, wl.exps) and np.array_equal(c, wl.coef)


def test_fast_reconstruction(ctx, orc):
    """A rational reconstruction whose steps take the fast path equals the oracle's."""
    wl = W.rational_simplex_workload(4321, 4, 8, 400, 250)
    ctx.solve_method(ctx.SOLVE_FAST)
    try:
        (Ne, Nc), (De, Dc), _ = ctx.reconstruct(wl.nv, wl.degN, wl.seed, wl.Nexps, wl.Ncoef, wl.Dexps, wl.Dcoef,
                                                degD=wl.degD)
    finally:
        ctx.solve_method(0)
    assert np.array_equal(Ne, wl.Nexps) and np.array_equal(Nc, wl.Ncoef)
    assert np.array_equal(De, wl.Dexps) and np.array_equal(Dc, wl.Dcoef)


def test_solve_method_arguments(ctx):
    from paper_2505_24256_gb300 import zr
    for bad in ((3, 0), (-1, 0), (0, -5)):
        with pytest.raises(zr.ZrError):
            ctx.solve_method(*bad)


@pytest.mark.parametrize("seed,T,k,maxe,S,off", [(61, 1, 2, 5, 3, 0), (62, 37, 2, 9, 5, 1), (63, 300, 3, 6, 9, 0),
                                                 (64, 2000, 4, 12, 21, 1), (65, 9000, 5, 20, 4, 0)])
def test_fast_probes_match_oracle(ctx, orc, seed, T, k, maxe, S, off):
    """Probes by the transposed tree (weighted power sums rev(N)/rev(M)) equal
    the oracle's and the matrix-vector evaluator's element by element."""
    wl = W.step_workload(seed, T, k, maxe, S)
    fe, fc = d8(wl.exps), d64(wl.coef)
    f = ctx.poly(wl.nv, wl.exps.shape[0], fe, fc)
    y, cs, z = d64(wl.y), d64(wl.cs), d64(wl.z)
    got = {}
    for method in (ctx.SOLVE_FAST, ctx.SOLVE_QUADRATIC):
        b = zeros64(S, T + 3)
        ctx.solve_method(method)
        try:
            ctx.zippel_probes(f, wl.k, y, S, cs, z, T, off, b, T + 3)
        finally:
            ctx.solve_method(0)
        got[method] = h64(b)[:, :T]
    want = orc.zippel_probes(wl.exps, wl.coef, wl.k, wl.y, wl.cs, wl.z, T, offset=off)
    assert np.array_equal(got[ctx.SOLVE_FAST], want)
    assert np.array_equal(got[ctx.SOLVE_QUADRATIC], want)


def test_fast_probes_few_groups(ctx, orc):
    """Many terms sharing few anchor monomials (G much smaller than T and Tf)."""
    wl = W.step_workload(66, 3, 2, 1, 7)     # 3 skeleton terms, 7 samples: G = 3 groups of 7 terms
    fe, fc = d8(wl.exps), d64(wl.coef)
    f = ctx.poly(wl.nv, wl.exps.shape[0], fe, fc)
    y, cs, z = d64(wl.y), d64(wl.cs), d64(wl.z)
    T = 5000
    b = zeros64(wl.S, T)
    ctx.solve_method(ctx.SOLVE_FAST)
    try:
        ctx.zippel_probes(f, wl.k, y, wl.S, cs, z, T, 0, b, T)
    finally:
        ctx.solve_method(0)
    assert np.array_equal(h64(b), orc.zippel_probes(wl.exps, wl.coef, wl.k, wl.y, wl.cs, wl.z, T))


def test_fast_probes_fall_back_above_64_samples(ctx, orc):
    """With the fast method forced, 65 samples exceed the transposed tree's
    column limit: the matrix-vector evaluator runs instead, and the probes
    still equal the oracle's."""
    wl = W.step_workload(67, 600, 3, 12, 65)
    fe, fc = d8(wl.exps), d64(wl.coef)
    f = ctx.poly(wl.nv, wl.exps.shape[0], fe, fc)
    y, cs, z = d64(wl.y), d64(wl.cs), d64(wl.z)
    b = zeros64(wl.S, wl.T)
    ctx.solve_method(ctx.SOLVE_FAST)
    try:
        ctx.profile(True)
        ctx.zippel_probes(f, wl.k, y, wl.S, cs, z, wl.T, 0, b, wl.T)
        ntt_launches = ctx.profile_query("ntt")[1]
        ctx.profile(False)
    finally:
        ctx.solve_method(0)
    assert ntt_launches == 0
    assert np.array_equal(h64(b), orc.zippel_probes(wl.exps, wl.coef, wl.k, wl.y, wl.cs, wl.z, wl.T))


@pytest.mark.parametrize("T,levels", [(1000, (8, 9, 10)), (1100, (8, 9, 10, 11))])
def test_profiler_counts_the_descent_butterflies(ctx, orc, T, levels):
    """The profiler's work count for the descent's cluster levels is the
    formula the bench's roofline uses: for each level of transform size
    n = 2^l, the nodes with roots in both children x (S + 1) rows x 5 primes
    x 3 transforms x (n / 2) log2 n butterflies.  At T = 1000 every level's
    nodes qualify (ceil(T / n) of them); at T = 1100 the last node of the
    levels 2^8 .. 2^10 has its 76 roots in its left child and is copied
    without a transform, and the solution is still the oracle's."""
    S = 2
    rnd = random.Random(21)
    v, b = rand_nodes(rnd, T, P63), rand_res(rnd, (S, T), P63)
    c = zeros64(S, T)
    ctx.solve_method(ctx.SOLVE_FAST)
    try:
        ctx.profile(True)
        ctx.vandermonde_solve([dict(T=T, S=S, offset=0, v=d64(v), b=d64(b), ldb=T, c=c, ldc=T)])
        work = ctx.profile_work("desc")
        launches = ctx.profile_query("desc")[1]
        ps_launches, ps_work = ctx.profile_query("psum")[1], ctx.profile_work("psum")
        ctx.profile(False)
    finally:
        ctx.solve_method(0)

    def transformed(l):
        n = 1 << l
        nodes = -(-T // n)
        return nodes - (1 if T - (nodes - 1) * n <= n // 2 else 0)

    want = sum(transformed(l) * (S + 1) * 5 * 3 * (1 << (l - 1)) * l for l in levels)
    assert launches == len(levels)         # one launch a level, all S + 1 rows in one descent (direct power sums)
    assert work == want
    assert ps_launches == 1 and ps_work == T * T   # the direct power sums: T^2 Shoup steps
    assert np.array_equal(h64(c), orc.tvandermonde_solve(v, b, offset=0))
