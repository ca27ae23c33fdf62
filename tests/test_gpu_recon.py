"""GPU parity: full reconstructions (zr_reconstruct) and the balanced step
(zr_zippel_step_balanced) against the oracle and generator truth."""
import itertools
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
    yield c
    c.close()


@pytest.mark.parametrize("offset", [0, 1])
def test_reconstruct_plain_poly_workload(ctx, orc, offset):
    wl = W.plain_poly_3var()
    (e, c), D, info = ctx.reconstruct(wl.nv, wl.deg, wl.seed, wl.exps, wl.coef, offset=offset)
    assert D is None
    assert np.array_equal(e, wl.exps) and np.array_equal(c, wl.coef)
    oe, oc = orc.reconstruct_poly(wl.exps, wl.coef, wl.deg, seed=wl.seed, offset=offset)
    assert np.array_equal(e, oe) and np.array_equal(c, oc)
    assert info["steps"] >= wl.nv - 1


@pytest.mark.parametrize("nv,deg,T,seed", [(1, 5, 4, 1), (2, 3, 6, 2), (3, 3, 12, 3), (4, 4, 40, 4), (6, 5, 120, 5)])
def test_reconstruct_poly_small(ctx, orc, nv, deg, T, seed):
    rnd = random.Random(seed)
    box = list(itertools.product(range(deg + 1), repeat=nv)) if (deg + 1) ** nv <= 20000 else None
    if box is not None:
        chosen = sorted(rnd.sample(box, T))
    else:
        chosen = sorted({tuple(rnd.randrange(deg + 1) for _ in range(nv)) for _ in range(T)})
    exps = np.array(chosen, dtype=np.uint8).reshape(-1, nv)
    coef = np.array([rnd.randrange(1, P63) for _ in range(exps.shape[0])], dtype=np.uint64)
    degs = [deg] * nv
    (e, c), _, _ = ctx.reconstruct(nv, degs, 900 + seed, exps, coef)
    oe, oc = orc.reconstruct_poly(exps, coef, degs, seed=900 + seed)
    assert np.array_equal(e, oe) and np.array_equal(c, oc)
    assert np.array_equal(e, exps) and np.array_equal(c, coef)


@pytest.mark.parametrize("nv,deg,TN,TD,seed", [(2, 3, 5, 4, 1), (3, 4, 12, 8, 2), (3, 6, 25, 15, 3), (4, 5, 60, 40, 4)])
def test_reconstruct_rational_small(ctx, orc, nv, deg, TN, TD, seed):
    wl = W.rational_simplex_workload(200 + seed, nv, deg, TN, TD)
    (Ne, Nc), (De, Dc), info = ctx.reconstruct(nv, wl.degN, wl.seed, wl.Nexps, wl.Ncoef, wl.Dexps, wl.Dcoef,
                                               degD=wl.degD)
    assert np.array_equal(Ne, wl.Nexps) and np.array_equal(Nc, wl.Ncoef)
    assert np.array_equal(De, wl.Dexps) and np.array_equal(Dc, wl.Dcoef)
    (oNe, oNc), (oDe, oDc) = orc.reconstruct_rational(wl.Nexps, wl.Ncoef, wl.Dexps, wl.Dcoef, wl.degN, wl.degD,
                                                      seed=wl.seed)
    assert np.array_equal(Ne, oNe) and np.array_equal(Nc, oNc)
    assert np.array_equal(De, oDe) and np.array_equal(Dc, oDc)


def test_balanced_step_matches_oracle(ctx, orc):
    """One balanced step through the C ABI against the oracle's balancing and steps."""
    rnd = random.Random(31)
    nv, k = 4, 3
    wl = W.rational_simplex_workload(77, nv, 6, 40, 25)
    dN = dD = 6
    Sf = 2 * 6 + 2
    z = [int(x) for x in W.Stream(5, 1).residues(nv)]
    y = [rnd.randrange(1, P63) for _ in range(k)]
    cs = [z[k]] + [int(x) for x in W.Stream(5, 2).distinct_residues(Sf - 1, avoid=[z[k]])]
    # skeletons of N and D at x_k = c_0 with the later variables at z: evaluate the hidden terms
    def skeleton(exps, coef):
        rows = {}
        for e, c in zip(exps, coef):
            key = tuple(int(v) for v in e[:k])
            val = int(c)
            for m in range(k, nv):
                val = val * pow(z[m] if m > k else cs[0], int(e[m]), P63) % P63
            rows[key] = (rows.get(key, 0) + val) % P63
        keys = sorted(kk for kk, v in rows.items() if v)
        ex = np.zeros((len(keys), nv), dtype=np.uint8)
        ex[:, :k] = np.array(keys, dtype=np.uint8).reshape(-1, k)
        return ex, np.array([rows[kk] for kk in keys], dtype=np.uint64)
    sNe, sNc = skeleton(wl.Nexps, wl.Ncoef)
    sDe, sDc = skeleton(wl.Dexps, wl.Dcoef)
    TN, TD = sNe.shape[0], sDe.shape[0]
    Tmax = max(TN, TD)
    Nv = orc.zippel_probes(wl.Nexps, wl.Ncoef, k, y, cs, z, Tmax)
    Dv = orc.zippel_probes(wl.Dexps, wl.Dcoef, k, y, cs, z, Tmax)
    f = np.array([[int(Nv[s, i]) * pow(int(Dv[s, i]), P63 - 2, P63) % P63 for i in range(Tmax)] for s in range(Sf)],
                 dtype=np.uint64)
    # oracle: D'(y^i) from the skeleton, balancing, two steps
    dprev = orc.zippel_probes(sDe, sDc, k, y, [1], [1] * nv, Tmax)[0]
    bN, bD = orc.balance_probes(cs, f, dprev, dN, dD, TN, TD)
    wNe, wNc = orc.zippel_step(sNe, k, y, cs[: dN + 1], bN)
    wDe, wDc = orc.zippel_step(sDe, k, y, cs[: dD + 1], bD)
    # GPU
    keep = [d8(sNe), d8(sDe), d64(sDc), d64(y), d64(cs), d64(f)]
    pN = ctx.poly(nv, TN, keep[0])
    pD = ctx.poly(nv, TD, keep[1], keep[2])
    capN, capD = TN * (dN + 1), TD * (dD + 1)
    oNe, oNc, oDe, oDc = zeros8(capN, nv), zeros64(capN), zeros8(capD, nv), zeros64(capD)
    nN, nD = ctx.zippel_step_balanced(pN, pD, k, keep[3], dN, dD, keep[4], keep[5], Tmax, 0, oNe, oNc, capN, oDe, oDc,
                                      capD)
    assert np.array_equal(oNe[:nN].cpu().numpy(), wNe) and np.array_equal(h64(oNc[:nN]), wNc)
    assert np.array_equal(oDe[:nD].cpu().numpy(), wDe) and np.array_equal(h64(oDc[:nD]), wDc)


def test_reconstruct_balanced_workload(ctx, orc):
    """N: 5000 and D: 3000 terms in 5 variables, total degree <= 15: exact
    recovery (generator truth) and agreement with the oracle."""
    wl = W.balanced_5var()
    (Ne, Nc), (De, Dc), info = ctx.reconstruct(wl.nv, wl.degN, wl.seed, wl.Nexps, wl.Ncoef, wl.Dexps, wl.Dcoef,
                                               degD=wl.degD)
    assert np.array_equal(Ne, wl.Nexps) and np.array_equal(Nc, wl.Ncoef)
    assert np.array_equal(De, wl.Dexps) and np.array_equal(Dc, wl.Dcoef)
    (oNe, oNc), (oDe, oDc) = orc.reconstruct_rational(wl.Nexps, wl.Ncoef, wl.Dexps, wl.Dcoef, wl.degN, wl.degD,
                                                      seed=wl.seed)
    assert np.array_equal(Ne, oNe) and np.array_equal(Nc, oNc)
    assert np.array_equal(De, oDe) and np.array_equal(Dc, oDc)


# ---- verification at a fresh point and unknown degrees -----------------------

@pytest.mark.parametrize("nv,deg,T,seed", [(3, 4, 20, 11), (5, 6, 150, 12)])
def test_verify_changes_nothing_when_lucky(ctx, nv, deg, T, seed):
    """A verified run takes the same probes as an unverified one (its points
    come from streams of their own) and returns the same result."""
    wl = W.poly_simplex_workload(700 + seed, nv, deg, T)
    (e0, c0), _, i0 = ctx.reconstruct(nv, wl.deg, wl.seed, wl.exps, wl.coef)
    (e1, c1), _, i1 = ctx.reconstruct(nv, wl.deg, wl.seed, wl.exps, wl.coef, verify=True)
    assert np.array_equal(e0, e1) and np.array_equal(c0, c1)
    assert np.array_equal(e1, wl.exps) and np.array_equal(c1, wl.coef)
    assert i0["steps"] == i1["steps"] and i1["redraws"] == 0
    rw = W.rational_simplex_workload(710 + seed, nv, deg, T, T // 2 + 1)
    a = (nv, rw.degN, rw.seed, rw.Nexps, rw.Ncoef, rw.Dexps, rw.Dcoef)
    (N0, D0, j0), (N1, D1, j1) = ctx.reconstruct(*a, degD=rw.degD), ctx.reconstruct(*a, degD=rw.degD, verify=True)
    for x, y in zip(N0 + D0, N1 + D1):
        assert np.array_equal(x, y)
    assert np.array_equal(N1[0], rw.Nexps) and np.array_equal(N1[1], rw.Ncoef)
    assert np.array_equal(D1[0], rw.Dexps) and np.array_equal(D1[1], rw.Dcoef)
    assert j0["steps"] == j1["steps"]


@pytest.mark.parametrize("nv,deg,T,seed,known", [(1, 9, 8, 1, []), (3, 5, 30, 2, [1]), (4, 12, 60, 3, []),
                                                 (6, 5, 120, 4, [0, 5])])
def test_unknown_degrees_poly(ctx, orc, nv, deg, T, seed, known):
    """Negative bounds: detected by growing the bound after each mismatch;
    the result is the hidden polynomial, the same as the oracle's with the
    true bounds."""
    wl = W.poly_simplex_workload(720 + seed, nv, deg, T)
    true_deg = [int(wl.exps[:, m].max()) for m in range(nv)]
    bounds = [true_deg[m] if m in known else -1 for m in range(nv)]
    (e, c), _, info = ctx.reconstruct(nv, bounds, wl.seed, wl.exps, wl.coef)
    assert np.array_equal(e, wl.exps) and np.array_equal(c, wl.coef)
    oe, oc = orc.reconstruct_poly(wl.exps, wl.coef, true_deg, seed=wl.seed)
    assert np.array_equal(e, oe) and np.array_equal(c, oc)
    if max(true_deg[m] for m in range(nv) if m not in known) > 3:
        assert info["redraws"] >= 1


def test_unknown_degrees_rational(ctx):
    wl = W.rational_simplex_workload(731, 3, 9, 30, 20)
    (Ne, Nc), (De, Dc), info = ctx.reconstruct(3, [-1] * 3, wl.seed, wl.Nexps, wl.Ncoef, wl.Dexps, wl.Dcoef,
                                               degD=[-1] * 3)
    assert np.array_equal(Ne, wl.Nexps) and np.array_equal(Nc, wl.Ncoef)
    assert np.array_equal(De, wl.Dexps) and np.array_equal(Dc, wl.Dcoef)
    assert info["redraws"] >= 1


def test_degree_beyond_detection(ctx):
    """x_0^70 needs 71 samples; detection stops at 64 with ZR_ERR_DEGREE."""
    from paper_2505_24256_gb300 import zr
    exps = np.array([[0, 0], [0, 1], [70, 0]], dtype=np.uint8)
    coef = np.array([5, 7, 11], dtype=np.uint64)
    with pytest.raises(zr.ZrError) as ei:
        ctx.reconstruct(2, [-1, 1], 3, exps, coef)
    assert ei.value.status == zr.DEGREE


def test_verify_catches_a_low_bound(ctx):
    """A known bound below the true degree: unverified, the result is wrong;
    verified, every attempt mismatches and the call fails with ZR_ERR_UNLUCKY."""
    from paper_2505_24256_gb300 import zr
    wl = W.poly_simplex_workload(741, 3, 6, 25)
    low = [6, 6, 2]
    assert int(wl.exps[:, 2].max()) > 2
    (e, c), _, _ = ctx.reconstruct(3, low, wl.seed, wl.exps, wl.coef)
    assert not (e.shape == wl.exps.shape and np.array_equal(e, wl.exps) and np.array_equal(c, wl.coef))
    with pytest.raises(zr.ZrError) as ei:
        ctx.reconstruct(3, low, wl.seed, wl.exps, wl.coef, verify=True)
    assert ei.value.status == zr.UNLUCKY


def test_unknown_degrees_served(ctx):
    from paper_2505_24256_gb300 import zr
    c2 = zr.Context(P63)
    try:
        srv = zr.Server(c2, 1 << 30, 4)
        wl = W.poly_simplex_workload(751, 4, 8, 70)
        rw = W.rational_simplex_workload(752, 3, 6, 20, 12)
        r1, k1 = zr.make_request(4, [-1] * 4, wl.seed, wl.exps, wl.coef)
        r2, k2 = zr.make_request(3, [-1] * 3, rw.seed, rw.Nexps, rw.Ncoef, rw.Dexps, rw.Dcoef, degD=[-1] * 3)
        t1, t2 = srv.submit(r1), srv.submit(r2)
        (e, c), _, _ = srv.wait(t1)
        assert np.array_equal(e, wl.exps) and np.array_equal(c, wl.coef)
        (Ne, Nc), (De, Dc), _ = srv.wait(t2)
        assert np.array_equal(Ne, rw.Nexps) and np.array_equal(Nc, rw.Ncoef)
        assert np.array_equal(De, rw.Dexps) and np.array_equal(Dc, rw.Dcoef)
        srv.close()
    finally:
        c2.close()


def test_reconstruct_most_variables(ctx, orc):
    """64 variables (the limit): 63 Zippel steps over a sparse polynomial,
    against the oracle and the hidden terms; 65 variables are rejected."""
    from paper_2505_24256_gb300 import zr
    nv = 64
    rnd = random.Random(64)
    rows = set()
    while len(rows) < 24:
        rows.add(tuple(rnd.randrange(3) if rnd.random() < 0.15 else 0 for _ in range(nv)))
    exps = np.array(sorted(rows), dtype=np.uint8)
    coef = np.array([rnd.randrange(1, P63) for _ in range(exps.shape[0])], dtype=np.uint64)
    degs = [2] * nv
    (e, c), _, info = ctx.reconstruct(nv, degs, 6400, exps, coef)
    assert np.array_equal(e, exps) and np.array_equal(c, coef)
    oe, oc = orc.reconstruct_poly(exps, coef, degs, seed=6400)
    assert np.array_equal(e, oe) and np.array_equal(c, oc)
    assert info["steps"] >= nv - 1
    wide = np.zeros((1, 65), dtype=np.uint8)
    with pytest.raises(zr.ZrError) as ei:
        ctx.reconstruct(65, [1] * 65, 1, wide, np.array([1], dtype=np.uint64))
    assert ei.value.status == zr.INVALID_ARG
