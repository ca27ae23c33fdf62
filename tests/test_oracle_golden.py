"""The oracle against tiny examples worked by hand (tests/golden/hand_worked.json)."""
import json
import os

import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_worked.json")


@pytest.fixture(scope="module")
def gold():
    with open(GOLDEN) as f:
        return json.load(f)


def test_golden_vandermonde(orc, gold):
    for case in gold["vandermonde"]:
        c = orc.tvandermonde_solve(case["v"], [case["b"]], offset=case["offset"], p=gold["p"])
        assert [int(x) for x in c[0]] == case["c"], case["source"]


def test_golden_master_poly(orc, gold):
    for case in gold["master_poly"]:
        assert [int(x) for x in orc.master_poly(case["v"], p=gold["p"])] == case["m"], case["source"]


def test_golden_newton(orc, gold):
    for case in gold["newton"]:
        assert [int(x) for x in orc.newton(case["x"], case["f"], p=gold["p"])] == case["coef"], case["source"]


def test_golden_thiele(orc, gold):
    p = gold["p"]
    for case in gold["thiele"]:
        f = [a * pow(b, p - 2, p) % p for a, b in zip(case["f_num"], case["f_den"])]
        num, den = orc.thiele(case["x"], f, case["maxdn"], case["maxdd"], p=p)
        assert [int(x) for x in num] == case["num"], case["source"]
        assert [int(x) for x in den] == case["den"], case["source"]
