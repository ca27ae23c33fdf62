"""Pins for the oracle's probe evaluator, Zippel step, balancing and full
reconstructions (CPU only).

Fixed by: the plain definition of the black box evaluated point by point in
Python, generator truth (the hidden terms are known), brute-force dense
interpolation over the full monomial box on tiny inputs, and N - f D = 0 at
fresh random points.
"""
import itertools
import random

import numpy as np
import pytest

from paper_2505_24256_gb300 import workloads as W
from tests import pyref
from tests.pyref import P63


def test_probes_match_plain_definition(orc):
    rnd = random.Random(50)
    nv, k = 4, 2
    Tf = 40
    exps = np.array([[rnd.randrange(5) for _ in range(nv)] for _ in range(Tf)], dtype=np.uint8)
    exps[5] = exps[3]; exps[5, 3] = (exps[3, 3] + 1) % 5      # shared prefixes
    exps[6, :k] = exps[3, :k]
    coef = np.array([rnd.randrange(P63) for _ in range(Tf)], dtype=np.uint64)
    y = [rnd.randrange(1, P63) for _ in range(k)]
    cs = [rnd.randrange(P63) for _ in range(3)]
    z = [rnd.randrange(P63) for _ in range(nv)]
    T = 9
    for offset in (0, 1):
        b = orc.zippel_probes(exps, coef, k, y, cs, z, T, offset=offset)
        for s in range(3):
            for i in range(T):
                pt = [pow(y[m], i + offset, P63) for m in range(k)] + [cs[s]] + z[k + 1:]
                assert int(b[s, i]) == pyref.eval_sparse(exps, coef, pt)
        samp = orc.zippel_probes_sampled(exps, coef, k, y, cs, z, [0, 2, 1], [8, 0, 4], offset=offset)
        assert [int(x) for x in samp] == [int(b[0, 8]), int(b[2, 0]), int(b[1, 4])]


def test_probes_match_plain_definition_heavy_sharing(orc):
    """2000 hidden terms whose x_0, x_1 exponents come from only 12 prefixes
    (groups of ~170 terms merged by the regrouped sum), against the plain
    point-by-point definition in Python integers."""
    rnd = random.Random(52)
    nv, k, Tf, T, S = 4, 2, 2000, 30, 3
    prefixes = [(rnd.randrange(9), rnd.randrange(9)) for _ in range(12)]
    rows = set()
    while len(rows) < Tf:
        a, b = prefixes[rnd.randrange(12)]
        rows.add((a, b, rnd.randrange(15), rnd.randrange(15)))
    exps = np.array(sorted(rows, key=lambda r: rnd.random()), dtype=np.uint8)
    coef = np.array([rnd.randrange(P63) for _ in range(Tf)], dtype=np.uint64)
    y = [rnd.randrange(1, P63) for _ in range(k)]
    cs = [rnd.randrange(P63) for _ in range(S)]
    z = [rnd.randrange(P63) for _ in range(nv)]
    for offset in (0, 1):
        b = orc.zippel_probes(exps, coef, k, y, cs, z, T, offset=offset)
        for s in range(S):
            for i in range(T):
                pt = [pow(y[m], i + offset, P63) for m in range(k)] + [cs[s]] + z[k + 1:]
                assert int(b[s, i]) == pyref.eval_sparse(exps, coef, pt)


def test_eval_points_definition(orc):
    rnd = random.Random(51)
    exps = np.array([[rnd.randrange(7) for _ in range(3)] for _ in range(25)], dtype=np.uint8)
    coef = [rnd.randrange(P63) for _ in range(25)]
    pts = [[rnd.randrange(P63) for _ in range(3)] for _ in range(6)]
    out = orc.eval_points(exps, coef, pts)
    assert [int(x) for x in out] == [pyref.eval_sparse(exps, coef, pt) for pt in pts]


@pytest.mark.parametrize("offset", [0, 1])
def test_zippel_step_generator_truth(orc, offset):
    wl = W.step_workload(77, 150, 3, 6, 5)
    b = orc.zippel_probes(wl.exps, wl.coef, wl.k, wl.y, wl.cs, wl.z, wl.T, offset=offset)
    e, c, cmat = orc.zippel_step(wl.skel, wl.k, wl.y, wl.cs, b, offset=offset, want_c=True)
    assert np.array_equal(e, wl.exps) and np.array_equal(c, wl.coef)
    # c[s][j] = g_j(c_s)
    for j in [0, 17, 149]:
        for s in range(wl.S):
            assert int(cmat[s, j]) == pyref.poly_eval([int(x) for x in wl.G[j]], int(wl.cs[s]))


def test_zippel_step_drops_zero_coefficients(orc):
    wl = W.step_workload(78, 60, 2, 9, 4)
    G = wl.G.copy()
    G[3, :] = 0          # a term that vanishes entirely
    G[10, 2] = 0         # one missing power
    wl2 = W.StepWorkload(wl.name, wl.p, wl.nv, wl.k, wl.T, wl.S, wl.skel, G, wl.y, wl.cs, wl.z)
    b = orc.zippel_probes(wl2.exps, wl2.coef, wl2.k, wl2.y, wl2.cs, wl2.z, wl2.T)
    e, c = orc.zippel_step(wl2.skel, wl2.k, wl2.y, wl2.cs, b)
    keep = wl2.coef != 0
    assert np.array_equal(e, wl2.exps[keep]) and np.array_equal(c, wl2.coef[keep])


def test_zippel_step_singular_anchor(orc):
    wl = W.step_workload(79, 20, 2, 5, 3)
    y = [1, 1]            # every monomial evaluates to 1
    b = np.zeros((3, 20), dtype=np.uint64)
    with pytest.raises(orc.OracleError) as e:
        orc.zippel_step(wl.skel, wl.k, y, wl.cs, b)
    assert e.value.status == orc.SINGULAR


def _dense_interpolate(f_exps, f_coef, nv, deg, rnd):
    """Brute force: solve for all coefficients of the full box [0..deg]^nv."""
    box = list(itertools.product(range(deg + 1), repeat=nv))
    pts = [[rnd.randrange(P63) for _ in range(nv)] for _ in range(len(box))]
    A = [[pyref.monomial_value(e, pt) for e in box] for pt in pts]
    b = [[pyref.eval_sparse(f_exps, f_coef, pt)] for pt in pts]
    sol = pyref.solve_linear(A, b)
    return {e: sol[i][0] for i, e in enumerate(box) if sol[i][0]}


@pytest.mark.parametrize("nv,deg,T,seed", [(2, 3, 6, 1), (3, 2, 9, 2), (3, 3, 12, 3), (1, 3, 3, 4)])
def test_reconstruct_poly_matches_dense_interpolation(orc, nv, deg, T, seed):
    rnd = random.Random(seed)
    box = list(itertools.product(range(deg + 1), repeat=nv))
    chosen = sorted(rnd.sample(box, T))
    exps = np.array(chosen, dtype=np.uint8).reshape(T, nv)
    coef = np.array([rnd.randrange(1, P63) for _ in range(T)], dtype=np.uint64)
    e, c = orc.reconstruct_poly(exps, coef, [deg] * nv, seed=seed)
    got = {tuple(int(x) for x in row): int(v) for row, v in zip(e, c)}
    assert got == _dense_interpolate(exps, coef, nv, deg, rnd)


@pytest.mark.parametrize("offset", [0, 1])
def test_reconstruct_plain_poly_workload(orc, offset):
    wl = W.plain_poly_3var()
    e, c = orc.reconstruct_poly(wl.exps, wl.coef, wl.deg, seed=wl.seed, offset=offset)
    assert np.array_equal(e, wl.exps) and np.array_equal(c, wl.coef)


def test_balance_probes_identity(orc):
    """With D' = D(., c_0) (scale C = 1) the balanced values are exactly
    N(y^i, c_s) and D(y^i, c_s)."""
    rnd = random.Random(60)
    nv, k = 3, 2
    wl = W.rational_simplex_workload(61, nv, 4, 10, 6)
    y = [rnd.randrange(1, P63) for _ in range(k)]
    dn = dd = 4
    Sf = 2 * 4 + 2
    cs = [rnd.randrange(P63) for _ in range(Sf)]
    z = [0] * nv
    Tmax = 12
    Nv = orc.zippel_probes(wl.Nexps, wl.Ncoef, k, y, cs, z, Tmax)
    Dv = orc.zippel_probes(wl.Dexps, wl.Dcoef, k, y, cs, z, Tmax)
    f = np.array([[int(Nv[s, i]) * pyref.inv(int(Dv[s, i])) % P63 for i in range(Tmax)] for s in range(Sf)],
                 dtype=np.uint64)
    dprev = Dv[0].copy()      # D(y^i, c_0): C = 1
    bN, bD = orc.balance_probes(cs, f, dprev, dn, dd, 9, 12)
    assert np.array_equal(bN, Nv[: dn + 1, :9])
    assert np.array_equal(bD, Dv[: dd + 1, :12])


@pytest.mark.parametrize("nv,deg,TN,TD,seed", [(2, 3, 5, 4, 1), (3, 4, 12, 8, 2), (3, 6, 25, 15, 3)])
def test_reconstruct_rational_exact(orc, nv, deg, TN, TD, seed):
    wl = W.rational_simplex_workload(200 + seed, nv, deg, TN, TD)
    (Ne, Nc), (De, Dc) = orc.reconstruct_rational(wl.Nexps, wl.Ncoef, wl.Dexps, wl.Dcoef, wl.degN, wl.degD,
                                                  seed=wl.seed)
    assert np.array_equal(Ne, wl.Nexps) and np.array_equal(Nc, wl.Ncoef)
    assert np.array_equal(De, wl.Dexps) and np.array_equal(Dc, wl.Dcoef)
    # N - f D = 0 at fresh points
    rnd = random.Random(seed)
    for _ in range(20):
        pt = [rnd.randrange(P63) for _ in range(nv)]
        dv = pyref.eval_sparse(wl.Dexps, wl.Dcoef, pt)
        if dv == 0:
            continue
        f = pyref.eval_sparse(wl.Nexps, wl.Ncoef, pt) * pyref.inv(dv) % P63
        assert (pyref.eval_sparse(Ne, Nc, pt) - f * pyref.eval_sparse(De, Dc, pt)) % P63 == 0


def test_oracle_recovers_serving_requests(orc):
    """The serving mix's hidden functions (box exponents <= 20, rational ones
    in lowest terms) are recovered exactly by the oracle."""
    from paper_2505_24256_gb300 import workloads as W

    reqs = W.serve_requests(12, seed=33, tmax=300)
    reqs.append(dict(id=99, rational=True, nv=3, T=2, seed=5))    # D a single monomial
    for r in reqs:
        wl = W.serve_blackbox(r)
        if isinstance(wl, W.RationalWorkload):
            (Ne, Nc), (De, Dc) = orc.reconstruct_rational(wl.Nexps, wl.Ncoef, wl.Dexps, wl.Dcoef, wl.degN, wl.degD,
                                                          seed=wl.seed)
            assert np.array_equal(Ne, wl.Nexps) and np.array_equal(Nc, wl.Ncoef), wl.name
            assert np.array_equal(De, wl.Dexps) and np.array_equal(Dc, wl.Dcoef), wl.name
        else:
            e, c = orc.reconstruct_poly(wl.exps, wl.coef, wl.deg, seed=wl.seed)
            assert np.array_equal(e, wl.exps) and np.array_equal(c, wl.coef), wl.name
