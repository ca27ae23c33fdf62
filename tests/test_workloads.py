"""The seeded synthetic workloads follow their stated recipes (no GPU): sizes,
value ranges, distinctness, ordering and the serving mix's distribution.
The generators hold no method arithmetic; these checks pin what the
benchmarks and the parity tests are run on."""
import math

import numpy as np
import pytest

from paper_2505_24256_gb300 import workloads as W

P63 = 2**63 - 25


def _distinct_rows(e):
    return np.unique(e, axis=0).shape[0] == e.shape[0]


def _lex_ordered(e):
    return all(tuple(a) < tuple(b) for a, b in zip(e[:-1], e[1:]))


def test_stream_residues_are_canonical_and_reproducible():
    a = W.Stream(7, 3).residues(20000)
    b = W.Stream(7, 3).residues(20000)
    assert np.array_equal(a, b)
    assert a.min() >= 1 and int(a.max()) < P63
    assert not np.array_equal(a, W.Stream(7, 4).residues(20000))
    d = W.Stream(9, 1).distinct_residues(5000, avoid=[int(a[0])])
    assert np.unique(d).size == 5000 and int(a[0]) not in set(int(x) for x in d)


def test_plain_poly_recipe():
    wl = W.plain_poly_3var()
    assert wl.exps.shape == (200, 3) and _distinct_rows(wl.exps) and _lex_ordered(wl.exps)
    assert int(wl.exps.sum(axis=1).max()) <= 10
    assert wl.coef.min() >= 1 and int(wl.coef.max()) < P63
    assert list(wl.deg) == [10, 10, 10]


def test_batched_step_recipe():
    wl = W.batched_step_1e4()
    assert (wl.T, wl.S, wl.nv, wl.k) == (10000, 21, 6, 5)
    assert _distinct_rows(wl.skel) and not wl.skel[:, 5].any() and int(wl.skel.max()) <= 20
    assert np.unique(wl.cs).size == 21
    # the hidden function: every skeleton term times a dense degree-20 polynomial in x_5
    assert wl.exps.shape == (210000, 6) and wl.coef.shape == (210000,)
    assert np.array_equal(wl.exps[:21, 5], np.arange(21)) and (wl.coef >= 1).all()


def test_balanced_recipe():
    wl = W.balanced_5var()
    assert wl.Nexps.shape == (5000, 5) and wl.Dexps.shape == (3000, 5)
    for e in (wl.Nexps, wl.Dexps):
        assert _distinct_rows(e) and _lex_ordered(e) and int(e.sum(axis=1).max()) <= 15
    assert int(wl.Dcoef[0]) == 1   # the lexicographically smallest denominator term
    # no common monomial factor of N and D
    assert np.minimum(wl.Nexps.min(axis=0), wl.Dexps.min(axis=0)).max() == 0


def test_serving_mix_recipe():
    reqs = W.serve_requests(4096)
    assert len(reqs) == 4096
    rational = sum(r["rational"] for r in reqs)
    assert 0.45 < rational / 4096 < 0.55
    nvs = [r["nv"] for r in reqs]
    assert min(nvs) == 2 and max(nvs) == 8
    Ts = np.array([r["T"] for r in reqs])
    assert Ts.min() >= 16 and Ts.max() <= 1 << 17
    assert all(r["T"] <= 21 ** r["nv"] // 2 for r in reqs)
    # log-uniform on [16, 2^17]: the median near the geometric mean (~1450) where the cap is far
    big = Ts[[r["nv"] >= 5 for r in reqs]]
    assert 900 < np.median(big) < 2400
    assert len({r["seed"] for r in reqs}) == 4096


@pytest.mark.parametrize("i", [0, 1, 2, 3, 5, 8])
def test_serving_black_boxes(i):
    req = W.serve_requests(16)[i]
    wl = W.serve_blackbox(req)
    if isinstance(wl, W.RationalWorkload):
        TN, TD = wl.Ncoef.shape[0], wl.Dcoef.shape[0]
        assert TN + TD == max(req["T"], 2) or TN + TD == req["T"]
        assert TN == max(1, (req["T"] * 3 + 4) // 5)
        assert int(wl.Dcoef[0]) == 1 and _lex_ordered(wl.Dexps)
        assert int(max(wl.Nexps.max(), wl.Dexps.max())) <= 20
    else:
        assert wl.exps.shape == (req["T"], req["nv"]) and _distinct_rows(wl.exps) and _lex_ordered(wl.exps)
        assert int(wl.exps.max()) <= 20 and (wl.coef >= 1).all()


def test_large_step_recipe_sampled():
    """The 2^20-term skeleton: distinct rows, 7 variables, exponents <= 12
    (checked in full; the hidden coefficients are drawn the same way as the
    T = 10^4 workload's)."""
    wl = W.large_step_2p20()
    assert (wl.T, wl.S, wl.nv, wl.k) == (1 << 20, 9, 8, 7)
    assert wl.skel.shape == (1 << 20, 8) and not wl.skel[:, 7].any() and int(wl.skel.max()) <= 12
    keys = np.zeros(wl.T, dtype=np.int64)
    for m in range(7):
        keys = keys * 13 + wl.skel[:, m].astype(np.int64)
    assert np.unique(keys).size == wl.T
    assert math.isclose(float(np.mean(wl.skel[:, :7])), 6.0, abs_tol=0.05)
