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
