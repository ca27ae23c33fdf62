"""GPU parity: transposed Vandermonde solve, Newton, anchor values and the
evaluator through the C ABI, element by element against the oracle."""
import random

import numpy as np
import pytest

from tests.gpuutil import d8, d64, h64, rand_nodes, rand_res, zeros64
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
    # these tests cover the O(T^2) kernels (the paper's method) at every size;
    # tests/test_gpu_fast.py covers the O(T log^2 T) path
    c.solve_method(c.SOLVE_QUADRATIC)
    yield c
    c.close()


def _solve(ctx, v, b, offset, plain=False):
    S, T = b.shape
    dv, db = d64(v), d64(b)
    dc = zeros64(S, T)
    ctx.vandermonde_solve([dict(T=T, S=S, offset=offset, v=dv, b=db, ldb=T, c=dc, ldc=T)], plain=plain)
    return h64(dc)


@pytest.mark.parametrize("T,S,offset", [(1, 1, 0), (1, 3, 1), (2, 2, 0), (3, 1, 1), (17, 5, 0), (100, 21, 0),
                                        (257, 9, 1), (1000, 4, 0), (1031, 24, 0), (1500, 25, 1), (3000, 13, 0)])
def test_solve_matches_oracle(ctx, orc, T, S, offset):
    rnd = random.Random(T * 7 + S)
    v = rand_nodes(rnd, T, P63)
    b = rand_res(rnd, (S, T), P63)
    got = _solve(ctx, v, b, offset)
    want = orc.tvandermonde_solve(v, b, offset=offset)
    assert np.array_equal(got, want)


def test_solve_kblocked_sampled_roots(ctx, orc):
    """T large enough for the k-blocked chain (several k-blocks)."""
    rnd = random.Random(99)
    T, S = 20000, 3
    v = rand_nodes(rnd, T, P63)
    b = rand_res(rnd, (S, T), P63)
    got = _solve(ctx, v, b, 0)
    m = orc.master_poly(v)
    roots = sorted(rnd.sample(range(T), 40)) + [0, T - 1]
    want = orc.tvandermonde_solve_roots(v, m, b, roots)
    assert np.array_equal(got[:, roots], want)


def test_solve_leading_dimensions(ctx, orc):
    rnd = random.Random(5)
    T, S = 333, 4
    v = rand_nodes(rnd, T, P63)
    b = rand_res(rnd, (S, T + 7), P63)
    dv, db = d64(v), d64(b)
    dc = zeros64(S, T + 3)
    ctx.vandermonde_solve([dict(T=T, S=S, offset=0, v=dv, b=db, ldb=T + 7, c=dc, ldc=T + 3)])
    want = orc.tvandermonde_solve(v, np.ascontiguousarray(b[:, :T]))
    assert np.array_equal(h64(dc)[:, :T], want)


def test_solve_several_systems(ctx, orc):
    rnd = random.Random(6)
    systems, keep, wants = [], [], []
    for T, S, off in [(50, 3, 0), (700, 9, 1), (1, 1, 0), (2049, 5, 0)]:
        v = rand_nodes(rnd, T, P63)
        b = rand_res(rnd, (S, T), P63)
        dv, db, dc = d64(v), d64(b), zeros64(S, T)
        keep.append(dc)
        systems.append(dict(T=T, S=S, offset=off, v=dv, b=db, ldb=T, c=dc, ldc=T, _keep=(dv, db)))
        wants.append(orc.tvandermonde_solve(v, b, offset=off))
    ctx.vandermonde_solve(systems)
    for dc, want in zip(keep, wants):
        assert np.array_equal(h64(dc), want)


def test_solve_singular(ctx):
    from paper_2505_24256_gb300 import zr
    v = np.array([5, 9, 5, 11], dtype=np.uint64)
    b = np.ones((2, 4), dtype=np.uint64)
    with pytest.raises(zr.ZrError) as e:
        _solve(ctx, v, b, 0)
    assert e.value.status == zr.SINGULAR
    v = np.array([0, 9, 7], dtype=np.uint64)
    with pytest.raises(zr.ZrError) as e:
        _solve(ctx, v, np.ones((1, 3), dtype=np.uint64), 1)
    assert e.value.status == zr.SINGULAR


def test_solve_empty(ctx):
    ctx.vandermonde_solve([])
    _solve(ctx, np.zeros(0, np.uint64), np.zeros((2, 0), np.uint64), 0)


@pytest.mark.parametrize("npts,nterms", [(1, 5), (2, 33), (5, 100), (9, 1000), (21, 777), (33, 64), (64, 40)])
def test_newton_matches_oracle(ctx, orc, npts, nterms):
    rnd = random.Random(npts * 1000 + nterms)
    x = rand_nodes(rnd, npts, P63)
    vals = rand_res(rnd, (npts, nterms), P63)
    dx, dvals, dcoef = d64(x), d64(vals), zeros64(npts, nterms)
    ctx.newton_batched(nterms, npts, dx, dvals, nterms, dcoef)
    assert np.array_equal(h64(dcoef), orc.newton_batched(x, vals))


def test_newton_duplicate_nodes(ctx):
    from paper_2505_24256_gb300 import zr
    x = np.array([3, 8, 3], dtype=np.uint64)
    with pytest.raises(zr.ZrError) as e:
        ctx.newton_batched(2, 3, d64(x), zeros64(3, 2), 2, zeros64(3, 2))
    assert e.value.status == zr.SINGULAR


@pytest.mark.parametrize("T,nv,k", [(1, 3, 2), (1000, 6, 5), (4097, 8, 3)])
def test_anchor_values(ctx, orc, T, nv, k):
    rnd = random.Random(T + nv)
    exps = np.array([[rnd.randrange(21) for _ in range(nv)] for _ in range(T)], dtype=np.uint8)
    # make the rows distinct in their first k columns
    exps[:, 0] = np.arange(T) % 251
    exps[:, 1] = (np.arange(T) // 251) % 251
    y = rand_res(rnd, (k,), P63)
    dv = zeros64(T)
    ctx.anchor_values(T, nv, d8(exps), k, d64(y), 0, dv)
    assert np.array_equal(h64(dv), orc.anchor_values(exps, k, y))


def test_eval_points(ctx, orc):
    rnd = random.Random(11)
    nv, Tf, npts = 4, 300, 17
    exps = np.array([[rnd.randrange(30) for _ in range(nv)] for _ in range(Tf)], dtype=np.uint8)
    coef = rand_res(rnd, (Tf,), P63)
    pts = rand_res(rnd, (npts, nv), P63)
    out = zeros64(npts)
    f = ctx.poly(nv, Tf, de := d8(exps), dc := d64(coef))
    ctx.eval_points(f, npts, d64(pts), out)
    assert np.array_equal(h64(out), orc.eval_points(exps, coef, pts))
