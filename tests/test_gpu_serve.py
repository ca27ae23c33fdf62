"""GPU: the serving loop (zr_serve_*).  Each request's result must equal the
hidden function and be identical to the same request reconstructed alone by
zr_reconstruct; the scheduler must overlap requests (several active at once)
and report consistent statistics."""
import time

import numpy as np
import pytest

from paper_2505_24256_gb300 import workloads as W
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


def _mix(n, seed, tmax):
    reqs = W.serve_requests(n, seed=seed, tmax=tmax)
    # degenerate shapes alongside the generated mix: one variable, one term
    reqs.append(dict(id=n, rational=False, nv=1, T=7, seed=seed * 7 + 1))
    reqs.append(dict(id=n + 1, rational=False, nv=4, T=1, seed=seed * 7 + 2))
    reqs.append(dict(id=n + 2, rational=True, nv=3, T=2, seed=seed * 7 + 3))
    return reqs, [W.serve_blackbox(r) for r in reqs]


def _request(zr, wl):
    if isinstance(wl, W.RationalWorkload):
        return zr.make_request(wl.nv, wl.degN, wl.seed, wl.Nexps, wl.Ncoef, wl.Dexps, wl.Dcoef, degD=wl.degD)
    return zr.make_request(wl.nv, wl.deg, wl.seed, wl.exps, wl.coef)


def _alone(ctx, wl):
    if isinstance(wl, W.RationalWorkload):
        return ctx.reconstruct(wl.nv, wl.degN, wl.seed, wl.Nexps, wl.Ncoef, wl.Dexps, wl.Dcoef, degD=wl.degD)
    return ctx.reconstruct(wl.nv, wl.deg, wl.seed, wl.exps, wl.coef)


def _check_truth(wl, res):
    (Ne, Nc), D, _ = res
    if isinstance(wl, W.RationalWorkload):
        assert np.array_equal(Ne, wl.Nexps) and np.array_equal(Nc, wl.Ncoef), wl.name
        assert D is not None and np.array_equal(D[0], wl.Dexps) and np.array_equal(D[1], wl.Dcoef), wl.name
    else:
        assert D is None
        assert np.array_equal(Ne, wl.exps) and np.array_equal(Nc, wl.coef), wl.name


def _same(a, b):
    (ae, ac), aD, ai = a
    (be, bc), bD, bi = b
    assert np.array_equal(ae, be) and np.array_equal(ac, bc)
    assert (aD is None) == (bD is None)
    if aD is not None:
        assert np.array_equal(aD[0], bD[0]) and np.array_equal(aD[1], bD[1])
    assert ai["steps"] == bi["steps"] and ai["redraws"] == bi["redraws"]


def _serve(zr, wls, budget, slots, mean_gap_s, seed):
    ctx = zr.Context(P63)
    srv = zr.Server(ctx, budget, slots)
    rng = np.random.default_rng(seed)
    tickets = []
    try:
        for wl in wls:                       # Poisson arrivals
            req, keep = _request(zr, wl)
            tickets.append(srv.submit(req))
            del keep
            if mean_gap_s > 0:
                time.sleep(rng.exponential(mean_gap_s))
        out = [srv.wait(t, timeout_s=300) for t in tickets]
        stats = srv.stats()
    finally:
        srv.close()
        ctx.close()
    return out, stats


def test_serve_mix_equals_alone(zr, orc):
    reqs, wls = _mix(40, 77, 3000)
    ctx = zr.Context(P63)
    try:
        alone = [_alone(ctx, wl) for wl in wls]
    finally:
        ctx.close()
    served, stats = _serve(zr, wls, 4 << 30, 16, 0.0005, 3)
    for wl, a, s in zip(wls, alone, served):
        _check_truth(wl, a)
        _check_truth(wl, s)
        _same(a, s)
    assert stats["completed"] == len(wls) and stats["failed"] == 0
    assert stats["submitted"] == len(wls)
    assert stats["max_active"] > 1, "requests never overlapped"
    assert stats["batch_entries"] >= stats["ticks"] > 0
    assert 0 < stats["p50_ms"] <= stats["p99_ms"]
    assert stats["terms"] == sum(int(np.asarray(s[0][1]).shape[0]) + (0 if s[1] is None else s[1][1].shape[0])
                                 for s in served)
    # the oracle on a few of the small requests
    small = [i for i, r in enumerate(reqs) if r["T"] <= 200][:6]
    for i in small:
        wl, s = wls[i], served[i]
        if isinstance(wl, W.RationalWorkload):
            (oNe, oNc), (oDe, oDc) = orc.reconstruct_rational(wl.Nexps, wl.Ncoef, wl.Dexps, wl.Dcoef, wl.degN,
                                                              wl.degD, seed=wl.seed)
            assert np.array_equal(s[0][0], oNe) and np.array_equal(s[0][1], oNc)
            assert np.array_equal(s[1][0], oDe) and np.array_equal(s[1][1], oDc)
        else:
            oe, oc = orc.reconstruct_poly(wl.exps, wl.coef, wl.deg, seed=wl.seed)
            assert np.array_equal(s[0][0], oe) and np.array_equal(s[0][1], oc)


def test_serve_tiny_budget_runs_one_at_a_time(zr):
    """A budget below every request's estimate admits one request at a time;
    results are unchanged."""
    _, wls = _mix(8, 91, 800)
    served, stats = _serve(zr, wls, 1, 8, 0.0, 4)
    for wl, s in zip(wls, served):
        _check_truth(wl, s)
    assert stats["max_active"] == 1 and stats["completed"] == len(wls)


def test_serve_poll_and_errors(zr):
    wl = W.serve_blackbox(dict(id=0, rational=False, nv=3, T=300, seed=5))
    ctx = zr.Context(P63)
    srv = zr.Server(ctx, 1 << 30, 4)
    try:
        req, keep = _request(zr, wl)
        t = srv.submit(req)
        with pytest.raises(zr.ZrError):
            srv.poll(t + 100)                # never issued
        res = None
        for _ in range(20000):
            res = srv.poll(t)
            if res is not None:
                break
            time.sleep(0.001)
        assert res is not None
        _check_truth(wl, res)
        with pytest.raises(zr.ZrError):      # a result is handed out once
            srv.poll(t)
        # invalid request: zero variables
        bad, keep2 = zr.make_request(0, np.zeros(0, np.int32), 1, np.zeros((1, 0), np.uint8),
                                     np.ones(1, np.uint64))
        with pytest.raises(zr.ZrError):
            srv.submit(bad)
        # requests left uncollected are completed and freed by destroy
        for s in range(3):
            req, keep = _request(zr, W.serve_blackbox(dict(id=s, rational=bool(s & 1), nv=4, T=100, seed=40 + s)))
            srv.submit(req)
    finally:
        srv.close()
        ctx.close()
