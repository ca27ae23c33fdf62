"""GPU parity: the probe evaluator and the Zippel step through the C ABI,
against the oracle (element by element) and against generator truth."""
import os
import random

import numpy as np
import pytest

from paper_2505_24256_gb300 import workloads as W
from tests.gpuutil import d8, d64, h64, zeros8, zeros64
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


class Dev:
    """Device copies of a step workload (kept alive with the object)."""

    def __init__(self, ctx, wl):
        self.wl = wl
        self.fe, self.fc = d8(wl.exps), d64(wl.coef)
        self.f = ctx.poly(wl.nv, wl.exps.shape[0], self.fe, self.fc)
        self.y, self.cs, self.z = d64(wl.y if len(wl.y) else [0]), d64(wl.cs), d64(wl.z)
        self.ske = d8(wl.skel)
        self.skel = ctx.poly(wl.nv, wl.T, self.ske)

    def probes(self, ctx, offset=0):
        wl = self.wl
        b = zeros64(wl.S, max(wl.T, 1))
        ctx.zippel_probes(self.f, wl.k, self.y, wl.S, self.cs, self.z, wl.T, offset, b, max(wl.T, 1))
        return b

    def step(self, ctx, b, offset=0):
        wl = self.wl
        cap = max(wl.T * wl.S, 1)
        oe, oc = zeros8(cap, wl.nv), zeros64(cap)
        n = ctx.zippel_step(self.skel, wl.k, self.y, wl.S, self.cs, b, max(wl.T, 1), offset, oe, oc, cap)
        return oe[:n].cpu().numpy(), h64(oc[:n])


@pytest.mark.parametrize("T,k,maxe,S,offset", [(1, 1, 3, 1, 0), (2, 2, 3, 2, 0), (150, 3, 6, 5, 0),
                                               (150, 3, 6, 5, 1), (1000, 4, 9, 9, 0), (2500, 5, 20, 21, 1),
                                               (777, 2, 40, 33, 0), (300, 6, 4, 64, 0)])
def test_probes_and_step_match_oracle(ctx, orc, T, k, maxe, S, offset):
    wl = W.step_workload(500 + T + S, T, k, maxe, S)
    D = Dev(ctx, wl)
    b = D.probes(ctx, offset)
    want_b = orc.zippel_probes(wl.exps, wl.coef, wl.k, wl.y, wl.cs, wl.z, wl.T, offset=offset)
    assert np.array_equal(h64(b)[:, :T], want_b)
    ge_, gc_ = D.step(ctx, b, offset)
    we, wc = orc.zippel_step(wl.skel, wl.k, wl.y, wl.cs, want_b, offset=offset)
    assert np.array_equal(ge_, we) and np.array_equal(gc_, wc)
    # generator truth: the step recovers the hidden terms
    assert np.array_equal(ge_, wl.exps) and np.array_equal(gc_, wl.coef)


def test_step_zero_coefficients_dropped(ctx, orc):
    wl = W.step_workload(78, 600, 2, 40, 7)
    G = wl.G.copy()
    G[3, :] = 0
    G[10, 2] = 0
    G[599, 6] = 0
    wl = W.StepWorkload(wl.name, wl.p, wl.nv, wl.k, wl.T, wl.S, wl.skel, G, wl.y, wl.cs, wl.z)
    D = Dev(ctx, wl)
    b = D.probes(ctx)
    ge_, gc_ = D.step(ctx, b)
    keep = wl.coef != 0
    assert np.array_equal(ge_, wl.exps[keep]) and np.array_equal(gc_, wl.coef[keep])


def test_step_singular_anchor(ctx):
    from paper_2505_24256_gb300 import zr
    wl = W.step_workload(79, 20, 2, 5, 3)
    D = Dev(ctx, wl)
    D.y = d64([1, 1])
    b = zeros64(3, 20)
    with pytest.raises(zr.ZrError) as e:
        D.step(ctx, b)
    assert e.value.status == zr.SINGULAR


def test_step_duplicate_samples(ctx):
    from paper_2505_24256_gb300 import zr
    wl = W.step_workload(80, 20, 2, 5, 3)
    D = Dev(ctx, wl)
    D.cs = d64([7, 9, 7])
    b = zeros64(3, 20)
    with pytest.raises(zr.ZrError) as e:
        D.step(ctx, b)
    assert e.value.status == zr.SINGULAR


def test_step_empty_skeleton(ctx):
    wl = W.step_workload(81, 0, 2, 5, 3)
    D = Dev(ctx, wl)
    e, c = D.step(ctx, zeros64(3, 1))
    assert e.shape[0] == 0


def test_step_capacity(ctx):
    from paper_2505_24256_gb300 import zr
    wl = W.step_workload(82, 40, 2, 9, 3)
    D = Dev(ctx, wl)
    b = D.probes(ctx)
    oe, oc = zeros8(10, wl.nv), zeros64(10)
    with pytest.raises(zr.ZrError) as e:
        ctx.zippel_step(D.skel, wl.k, D.y, wl.S, D.cs, b, wl.T, 0, oe, oc, 10)
    assert e.value.status == zr.CAPACITY


def test_step_host_buffers(ctx, orc):
    wl = W.step_workload(83, 900, 4, 12, 8)
    b = orc.zippel_probes(wl.exps, wl.coef, wl.k, wl.y, wl.cs, wl.z, wl.T)
    skel = ctx.poly(wl.nv, wl.T, wl.skel)
    cap = wl.T * wl.S
    oe = np.zeros((cap, wl.nv), dtype=np.uint8)
    oc = np.zeros(cap, dtype=np.uint64)
    n = ctx.zippel_step_host(skel, wl.k, np.ascontiguousarray(wl.y), wl.S, np.ascontiguousarray(wl.cs),
                             np.ascontiguousarray(b), wl.T, 0, oe, oc, cap)
    assert n == wl.exps.shape[0]
    assert np.array_equal(oe[:n], wl.exps) and np.array_equal(oc[:n], wl.coef)
    # buffers of n terms and a sentinel: the one transfer out copies
    # min(T S, out_cap) terms, so nothing is written past out_cap
    oe2 = np.zeros((n + 1, wl.nv), dtype=np.uint8)
    oc2 = np.zeros(n + 1, dtype=np.uint64)
    oe2[n] = 77
    oc2[n] = 12345
    n2 = ctx.zippel_step_host(skel, wl.k, np.ascontiguousarray(wl.y), wl.S, np.ascontiguousarray(wl.cs),
                              np.ascontiguousarray(b), wl.T, 0, oe2, oc2, n)
    assert n2 == n
    assert np.array_equal(oe2[:n], wl.exps) and np.array_equal(oc2[:n], wl.coef)
    assert (oe2[n] == 77).all() and oc2[n] == 12345


def probes_at_points(orc, wl, sidx, iidx, offset=0):
    """The probes (s, i) by the oracle's plain point-by-point evaluation at the
    explicit points (y^(i+offset), c_s, z), one point per host thread."""
    from concurrent.futures import ThreadPoolExecutor
    k = wl.k
    pts = [[pow(int(wl.y[m]), i + offset, wl.p) for m in range(k)] + [int(wl.cs[s])] +
           [int(x) for x in wl.z[k + 1:]] for s, i in zip(sidx, iidx)]
    with ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        vals = list(ex.map(lambda pt: int(orc.eval_points(wl.exps, wl.coef, [pt])[0]), pts))
    return np.array(vals, dtype=np.uint64)


def test_batched_step_workload_full(ctx, orc):
    """The T = 10^4, S = 21 step in full: probes and new skeleton against the
    oracle element by element, and against generator truth; 64 sampled probes
    also against the plain evaluation at their explicit points."""
    wl = W.batched_step_1e4()
    D = Dev(ctx, wl)
    b = D.probes(ctx)
    want_b = orc.zippel_probes(wl.exps, wl.coef, wl.k, wl.y, wl.cs, wl.z, wl.T)
    assert np.array_equal(h64(b), want_b)
    rnd = random.Random(4)
    sidx = [rnd.randrange(wl.S) for _ in range(62)] + [0, wl.S - 1]
    iidx = [rnd.randrange(wl.T) for _ in range(62)] + [wl.T - 1, 0]
    assert np.array_equal(h64(b)[sidx, iidx], probes_at_points(orc, wl, sidx, iidx))
    ge_, gc_ = D.step(ctx, b)
    assert np.array_equal(ge_, wl.exps) and np.array_equal(gc_, wl.coef)
    we, wc = orc.zippel_step(wl.skel, wl.k, wl.y, wl.cs, want_b)
    assert np.array_equal(ge_, we) and np.array_equal(gc_, wc)


def test_large_step_workload(ctx, orc):
    """The T = 2^20, S = 9 step: 64 sampled probes against the oracle and
    against the plain evaluation at their explicit points, the new skeleton
    against generator truth in full."""
    wl = W.large_step_2p20()
    D = Dev(ctx, wl)
    b = D.probes(ctx)
    hb = h64(b)
    rnd = random.Random(3)
    sidx = [rnd.randrange(wl.S) for _ in range(62)] + [0, wl.S - 1]
    iidx = [rnd.randrange(wl.T) for _ in range(62)] + [0, wl.T - 1]
    want = orc.zippel_probes_sampled(wl.exps, wl.coef, wl.k, wl.y, wl.cs, wl.z, sidx, iidx)
    assert np.array_equal(hb[sidx, iidx], want)
    # all 64 also by the plain point-by-point evaluation of the hidden function
    assert np.array_equal(hb[sidx, iidx], probes_at_points(orc, wl, sidx, iidx))
    ge_, gc_ = D.step(ctx, b)
    assert np.array_equal(ge_, wl.exps) and np.array_equal(gc_, wl.coef)


def test_batched_steps_match_single_steps(ctx, orc):
    """Uneven steps (different T, S, k, nv, offset) in one batched call give
    exactly the results of the single-step calls and of the oracle."""
    import torch
    shapes = [(700, 3, 9, 5, 0), (1, 2, 4, 3, 0), (2500, 5, 20, 21, 1), (64, 2, 9, 9, 0), (0, 2, 5, 4, 0),
              (4100, 4, 12, 9, 0)]
    devs, wls, steps, outs = [], [], [], []
    for n, (T, k, maxe, S, off) in enumerate(shapes):
        wl = W.step_workload(3000 + n, T, k, maxe, S)
        D = Dev(ctx, wl)
        b = D.probes(ctx, off) if T else zeros64(S, 1)
        cap = max(T * S, 1)
        oe, oc, cnt = zeros8(cap, wl.nv), zeros64(cap), zeros64(1)
        steps.append(dict(skel=D.skel, newvar=wl.k, S=S, offset=off, y=D.y, samples=D.cs, probes=b,
                          ldb=max(T, 1), out_exps=oe, out_coef=oc, out_cap=cap, out_count=cnt))
        devs.append((D, b))
        wls.append((wl, off))
        outs.append((oe, oc, cnt))
    ctx.zippel_step_batched(steps)
    torch.cuda.synchronize()
    for (wl, off), (D, b), (oe, oc, cnt) in zip(wls, devs, outs):
        n = int(cnt.cpu().item())
        ge_, gc_ = oe[:n].cpu().numpy(), h64(oc[:n])
        assert np.array_equal(ge_, wl.exps) and np.array_equal(gc_, wl.coef)
        if wl.T:
            se, sc = D.step(ctx, b, off)
            assert np.array_equal(ge_, se) and np.array_equal(gc_, sc)
            if wl.T <= 2500:
                we, wc = orc.zippel_step(wl.skel, wl.k, wl.y, wl.cs, h64(b)[:, :wl.T], offset=off)
                assert np.array_equal(ge_, we) and np.array_equal(gc_, wc)


def test_batched_solve_equals_plain(ctx, orc):
    """zr_vandermonde_solve_batched (shared launches) against the plain form."""
    rnd = random.Random(12)
    systems, plain_out, batch_out, keep = [], [], [], []
    from tests.gpuutil import rand_nodes, rand_res
    for T, S, off in [(10, 3, 0), (3000, 21, 0), (1, 1, 1), (257, 9, 1), (5000, 4, 0)]:
        v = rand_nodes(rnd, T, P63)
        bb = rand_res(rnd, (S, T), P63)
        dv, db = d64(v), d64(bb)
        c1, c2 = zeros64(S, T), zeros64(S, T)
        keep.append((dv, db))
        systems.append((dict(T=T, S=S, offset=off, v=dv, b=db, ldb=T, c=c1, ldc=T),
                        dict(T=T, S=S, offset=off, v=dv, b=db, ldb=T, c=c2, ldc=T)))
        plain_out.append(c1)
        batch_out.append(c2)
    ctx.vandermonde_solve([s[0] for s in systems], plain=True)
    ctx.vandermonde_solve([s[1] for s in systems], plain=False)
    for c1, c2 in zip(plain_out, batch_out):
        assert np.array_equal(h64(c1), h64(c2))


def test_autotuned_plan_gives_the_same_skeleton(ctx):
    """The autotuner only changes the schedule: after tuning a shape the
    step's output is unchanged, and the stored plan is one the solve is
    built for."""
    wl = W.step_workload(701, 3000, 4, 12, 9)
    D = Dev(ctx, wl)
    b = D.probes(ctx)
    before = D.step(ctx, b)
    ctx.autotune_step(wl.T, wl.S, 8)
    tile, nb = ctx.step_plan(wl.T, wl.S)
    assert tile in (2, 3, 4, 6, 8) and 1 <= nb <= wl.T // 32 + 1
    after = D.step(ctx, b)
    assert np.array_equal(before[0], after[0]) and np.array_equal(before[1], after[1])
    assert np.array_equal(after[0], wl.exps) and np.array_equal(after[1], wl.coef)


@pytest.mark.parametrize("S,T,k,offset", [(80, 300, 2, 0), (130, 97, 3, 1), (7, 5000, 1, 0)])
def test_probes_general_function(ctx, orc, S, T, k, offset):
    """Probes of a hidden function without the step's structure (groups of
    uneven size), with sample sets wider than one column block of the
    evaluator, and split group ranges."""
    rnd = random.Random(S * 1000 + T)
    nv = 5
    wl = W.poly_simplex_workload(600 + S, nv, 8, 400)
    y = [rnd.randrange(1, P63) for _ in range(k)]
    cs = [rnd.randrange(1, P63) for _ in range(S)]
    z = [rnd.randrange(1, P63) for _ in range(nv)]
    fe, fc = d8(wl.exps), d64(wl.coef)
    f = ctx.poly(nv, wl.exps.shape[0], fe, fc)
    b = zeros64(S, T)
    ctx.zippel_probes(f, k, d64(y), S, d64(cs), d64(z), T, offset, b, T)
    want = orc.zippel_probes(wl.exps, wl.coef, k, y, cs, z, T, offset=offset)
    assert np.array_equal(h64(b), want)
