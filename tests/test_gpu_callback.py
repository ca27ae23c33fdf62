"""GPU: black boxes given as functions (zr_bb_kind CALL_*).

The callback reconstructions must be identical to the same reconstructions of
the built-in sparse black box (the library draws the same points from the
same seed and asks the function for the same values) and to the hidden
function; zr_probe_points must lay out the Zippel probe points exactly; a
function that reports a pole must lead to a redraw (rational) or a clean
ZR_ERR_POLE (polynomial)."""
import random

import numpy as np
import pytest

from paper_2505_24256_gb300 import workloads as W
from tests.gpuutil import d8, d64, h64, zeros64
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
def evctx(zr):
    """A second context that plays the caller's evaluator."""
    c = zr.Context(P63)
    yield c
    c.close()


class DeviceFn:
    """A sparse polynomial held on the device, evaluated by zr_eval_points."""

    def __init__(self, zr, evctx, exps, coef):
        self.zr, self.evctx = zr, evctx
        self.exps, self.coef = d8(exps), d64(coef)
        self.f = zr.zr_poly(exps.shape[1], exps.shape[0], self.exps.data_ptr(), self.coef.data_ptr())

    def __call__(self, npts, nv, pts, out, stream):
        self.evctx.eval_points(self.f, npts, pts, out, stream=stream)
        return 0


def test_probe_points_layout(ctx):
    rnd = random.Random(5)
    nv, k, S, T, offset = 5, 2, 3, 7, 1
    y = [rnd.randrange(1, P63) for _ in range(k)]
    cs = [rnd.randrange(1, P63) for _ in range(S)]
    z = [rnd.randrange(1, P63) for _ in range(nv)]
    pts = zeros64(S * T * nv)
    ctx.probe_points(nv, k, d64(y), S, d64(cs), d64(z), T, offset, pts)
    got = h64(pts).reshape(S, T, nv)
    for s in range(S):
        for i in range(T):
            want = [pow(y[m], i + offset, P63) for m in range(k)] + [cs[s]] + z[k + 1:]
            assert [int(x) for x in got[s, i]] == want


@pytest.mark.parametrize("nv,deg,T,seed,offset", [(1, 5, 4, 1, 0), (3, 4, 30, 2, 0), (4, 5, 80, 3, 1),
                                                  (6, 5, 200, 4, 0)])
def test_callback_poly_matches_builtin(zr, ctx, evctx, nv, deg, T, seed, offset):
    wl = W.poly_simplex_workload(500 + seed, nv, deg, T)
    fn = DeviceFn(zr, evctx, wl.exps, wl.coef)
    (e, c), D, info = ctx.reconstruct_callback(nv, wl.deg, wl.seed, fn, TN_hint=T, offset=offset)
    assert D is None
    assert np.array_equal(e, wl.exps) and np.array_equal(c, wl.coef)
    (be, bc), _, binfo = ctx.reconstruct(nv, wl.deg, wl.seed, wl.exps, wl.coef, offset=offset)
    assert np.array_equal(e, be) and np.array_equal(c, bc)
    assert info["steps"] == binfo["steps"] and info["redraws"] == binfo["redraws"]


class RationalFn:
    """N / D from two device polynomials; a zero denominator is a pole."""

    def __init__(self, zr, evctx, wl, poles=0):
        self.N = DeviceFn(zr, evctx, wl.Nexps, wl.Ncoef)
        self.D = DeviceFn(zr, evctx, wl.Dexps, wl.Dcoef)
        self.zr = zr
        self.poles = poles   # report this many calls as poles first
        self.calls = 0

    def __call__(self, npts, nv, pts, out, stream):
        import torch

        self.calls += 1
        if self.calls <= self.poles:
            return 1
        # no zero fill: it would run on another stream than the evaluation
        nval = torch.empty(npts, dtype=torch.int64, device="cuda")
        dval = torch.empty(npts, dtype=torch.int64, device="cuda")
        self.N(npts, nv, pts, nval.data_ptr(), stream)
        self.D(npts, nv, pts, dval.data_ptr(), stream)
        n, d = h64(nval), h64(dval)
        if np.any(d == 0):
            return 1
        q = np.array([int(a) * pow(int(b), P63 - 2, P63) % P63 for a, b in zip(n, d)], dtype=np.uint64)
        self.zr.device_array(out, npts).copy_(d64(q))
        torch.cuda.synchronize()
        return 0


@pytest.mark.parametrize("nv,deg,TN,TD,seed", [(2, 3, 5, 4, 1), (3, 4, 12, 8, 2), (4, 5, 40, 25, 3)])
def test_callback_rational_matches_builtin(zr, ctx, evctx, nv, deg, TN, TD, seed):
    wl = W.rational_simplex_workload(300 + seed, nv, deg, TN, TD)
    fn = RationalFn(zr, evctx, wl)
    (Ne, Nc), (De, Dc), info = ctx.reconstruct_callback(nv, wl.degN, wl.seed, fn, rational=True, degD=wl.degD,
                                                        TN_hint=TN, TD_hint=TD)
    assert np.array_equal(Ne, wl.Nexps) and np.array_equal(Nc, wl.Ncoef)
    assert np.array_equal(De, wl.Dexps) and np.array_equal(Dc, wl.Dcoef)
    (bNe, bNc), (bDe, bDc), binfo = ctx.reconstruct(nv, wl.degN, wl.seed, wl.Nexps, wl.Ncoef, wl.Dexps, wl.Dcoef,
                                                    degD=wl.degD)
    assert np.array_equal(Ne, bNe) and np.array_equal(Nc, bNc)
    assert np.array_equal(De, bDe) and np.array_equal(Dc, bDc)


def test_callback_rational_pole_redraws(zr, ctx, evctx):
    """Poles reported by the function cost a redraw each, not the result."""
    wl = W.rational_simplex_workload(311, 3, 4, 12, 8)
    fn = RationalFn(zr, evctx, wl, poles=2)
    (Ne, Nc), (De, Dc), info = ctx.reconstruct_callback(3, wl.degN, wl.seed, fn, rational=True, degD=wl.degD)
    assert np.array_equal(Ne, wl.Nexps) and np.array_equal(Nc, wl.Ncoef)
    assert np.array_equal(De, wl.Dexps) and np.array_equal(Dc, wl.Dcoef)
    assert info["redraws"] >= 2


def test_callback_failures(zr, ctx, evctx):
    wl = W.poly_simplex_workload(77, 3, 4, 20)
    with pytest.raises(zr.ZrError) as ei:
        ctx.reconstruct_callback(3, wl.deg, wl.seed, lambda *a: 1)
    assert ei.value.status == zr.POLE

    def boom(*a):
        raise ValueError("evaluator failed")

    with pytest.raises(ValueError, match="evaluator failed"):
        ctx.reconstruct_callback(3, wl.deg, wl.seed, boom)
    # the context stays usable
    fn = DeviceFn(zr, evctx, wl.exps, wl.coef)
    (e, c), _, _ = ctx.reconstruct_callback(3, wl.deg, wl.seed, fn)
    assert np.array_equal(e, wl.exps) and np.array_equal(c, wl.coef)


def test_callback_requests_served(zr, evctx):
    """Callback requests share the serving loop with built-in boxes."""
    ctx = zr.Context(P63)
    try:
        srv = zr.Server(ctx, 1 << 30, 8)
        wls = [W.poly_simplex_workload(900 + i, 3 + i % 3, 5, 20 + 10 * i) for i in range(4)]
        rw = W.rational_simplex_workload(950, 3, 4, 12, 8)
        keep, tickets = [], []
        for i, wl in enumerate(wls):
            if i % 2:
                req, k = zr.make_callback_request(wl.nv, wl.deg, wl.seed, DeviceFn(zr, evctx, wl.exps, wl.coef),
                                                  TN_hint=wl.exps.shape[0])
            else:
                req, k = zr.make_request(wl.nv, wl.deg, wl.seed, wl.exps, wl.coef)
            keep.append(k)
            tickets.append(srv.submit(req))
        req, k = zr.make_callback_request(3, rw.degN, rw.seed, RationalFn(zr, evctx, rw), rational=True,
                                          degD=rw.degD, TN_hint=12, TD_hint=8)
        keep.append(k)
        tickets.append(srv.submit(req))
        for t, wl in zip(tickets[:4], wls):
            (e, c), D, _ = srv.wait(t)
            assert D is None and np.array_equal(e, wl.exps) and np.array_equal(c, wl.coef)
        (Ne, Nc), (De, Dc), _ = srv.wait(tickets[4])
        assert np.array_equal(Ne, rw.Nexps) and np.array_equal(Nc, rw.Ncoef)
        assert np.array_equal(De, rw.Dexps) and np.array_equal(Dc, rw.Dcoef)
        assert not any(k[-1] for k in keep if isinstance(k[-1], list))
        srv.close()
    finally:
        ctx.close()
