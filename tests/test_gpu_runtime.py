"""GPU: runtime facilities around the step -- the bounded device waits give
up and report instead of hanging, the context stays usable afterwards, and
the measured ceilings are consistent with one another."""
import numpy as np
import pytest

from paper_2505_24256_gb300 import workloads as W
from tests.gpuutil import d8, d64, h64, zeros64, zeros8
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


def _small_step(ctx):
    wl = W.step_workload(601, 500, 3, 9, 7)
    fe, fc = d8(wl.exps), d64(wl.coef)
    f = ctx.poly(wl.nv, wl.exps.shape[0], fe, fc)
    y, cs, z = d64(wl.y), d64(wl.cs), d64(wl.z)
    ske = d8(wl.skel)
    b = zeros64(wl.S, wl.T)
    ctx.zippel_probes(f, wl.k, y, wl.S, cs, z, wl.T, 0, b, wl.T)
    cap = wl.T * wl.S
    oe, oc = zeros8(cap, wl.nv), zeros64(cap)
    n = ctx.zippel_step(ctx.poly(wl.nv, wl.T, ske), wl.k, y, wl.S, cs, b, wl.T, 0, oe, oc, cap)
    return np.array_equal(oe[:n].cpu().numpy(), wl.exps) and np.array_equal(h64(oc[:n]), wl.coef)


def test_bounded_wait_times_out_and_context_survives(ctx):
    from paper_2505_24256_gb300 import zr

    assert ctx.check_bounded_wait(4096) == zr.TIMEOUT
    assert ctx.check_bounded_wait(1) == zr.TIMEOUT
    assert _small_step(ctx)                 # the context (and the GPU) still work


def test_measured_ceilings_are_consistent(ctx):
    p = ctx.measure_peaks()
    assert p["sms"] > 0
    for k in ("mac_per_s", "chain_per_s", "imad_lo_per_s", "imad_hi_per_s", "butterfly_per_s"):
        assert p[k] > 1e9, (k, p[k])
    # a butterfly takes one mad.hi (x w') and two 32-bit products
    assert p["butterfly_per_s"] <= p["imad_hi_per_s"] * 1.05
    # a 64x64 multiply-accumulate needs four mad.lo and four mad.hi
    assert p["mac_per_s"] <= p["imad_lo_per_s"] / 4 * 1.05
    assert p["mac_per_s"] <= p["imad_hi_per_s"] / 4 * 1.05 * 2
    assert p["chain_per_s"] < p["mac_per_s"]          # a Shoup step costs more than one product
