"""GPU: Zippel steps captured into CUDA graphs (zr_step_graph_*) give the
same results as the direct calls, re-run on the current contents of their
buffers, and report device-detected conditions."""
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


class Step:
    """Device buffers of one step workload plus its descriptor."""

    def __init__(self, ctx, wl, offset=0):
        import torch

        self.wl = wl
        self.f_e, self.f_c = d8(wl.exps), d64(wl.coef)
        self.f = ctx.poly(wl.nv, wl.exps.shape[0], self.f_e, self.f_c)
        self.y, self.cs, self.z = d64(wl.y), d64(wl.cs), d64(wl.z)
        self.ske = d8(wl.skel)
        self.skel = ctx.poly(wl.nv, wl.T, self.ske)
        self.b = zeros64(wl.S, wl.T)
        ctx.zippel_probes(self.f, wl.k, self.y, wl.S, self.cs, self.z, wl.T, offset, self.b, wl.T)
        self.cap = wl.T * wl.S
        self.oe, self.oc = zeros8(self.cap, wl.nv), zeros64(self.cap)
        self.cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
        self.desc = dict(skel=self.skel, newvar=wl.k, S=wl.S, offset=offset, y=self.y, samples=self.cs,
                         probes=self.b, ldb=wl.T, out_exps=self.oe, out_coef=self.oc, out_cap=self.cap,
                         out_count=self.cnt)

    def result(self):
        n = int(self.cnt.item())
        return self.oe[:n].cpu().numpy(), h64(self.oc[:n])


def test_graph_step_matches_direct_and_reruns_on_new_probes(ctx, orc):
    from paper_2505_24256_gb300 import zr

    wl = W.step_workload(501, 3000, 4, 12, 9)
    st = Step(ctx, wl)
    g = ctx.step_graph([st.desc])
    try:
        e, c = st.result()
        assert np.array_equal(e, wl.exps) and np.array_equal(c, wl.coef)
        assert g.kernels > 0
        # new hidden coefficients on the same skeleton: new probes in the same buffer
        G2 = (wl.G + np.uint64(12345)) % np.uint64(P63)
        G2[G2 == 0] = 1
        wl2 = W.StepWorkload(wl.name, wl.p, wl.nv, wl.k, wl.T, wl.S, wl.skel, G2, wl.y, wl.cs, wl.z)
        f2e, f2c = d8(wl2.exps), d64(wl2.coef)
        f2 = ctx.poly(wl2.nv, wl2.exps.shape[0], f2e, f2c)
        ctx.zippel_probes(f2, wl.k, st.y, wl.S, st.cs, st.z, wl.T, 0, st.b, wl.T)
        st.oc.zero_()
        n0 = zr.launch_count()
        g.launch()
        g.status()
        assert zr.launch_count() - n0 == g.kernels
        e2, c2 = st.result()
        assert np.array_equal(e2, wl2.exps) and np.array_equal(c2, wl2.coef)
        # the direct call on the same probes gives the same skeleton
        oe, oc = zeros8(st.cap, wl.nv), zeros64(st.cap)
        n = ctx.zippel_step(st.skel, wl.k, st.y, wl.S, st.cs, st.b, wl.T, 0, oe, oc, st.cap)
        assert np.array_equal(oe[:n].cpu().numpy(), e2) and np.array_equal(h64(oc[:n]), c2)
        want_e, want_c = orc.zippel_step(wl.skel, wl.k, wl.y, wl.cs, h64(st.b))
        assert np.array_equal(e2, want_e) and np.array_equal(c2, want_c)
    finally:
        g.close()


def test_graph_uneven_batch(ctx):
    wls = [W.step_workload(511, 700, 3, 10, 11), W.step_workload(512, 2500, 5, 9, 21),
           W.step_workload(513, 41, 2, 8, 3)]
    steps = [Step(ctx, wl, offset=i % 2) for i, wl in enumerate(wls)]
    g = ctx.step_graph([s.desc for s in steps])
    try:
        for s in steps:
            s.oc.zero_()
            s.cnt.zero_()
        for _ in range(3):
            g.launch()
        g.status()
        for s, wl in zip(steps, wls):
            e, c = s.result()
            assert np.array_equal(e, wl.exps) and np.array_equal(c, wl.coef)
    finally:
        g.close()


def test_graph_reports_duplicate_samples(ctx):
    from paper_2505_24256_gb300 import zr

    wl = W.step_workload(521, 200, 3, 8, 5)
    st = Step(ctx, wl)
    cs = wl.cs.copy()
    cs[3] = cs[1]
    st.cs.copy_(d64(cs))
    with pytest.raises(zr.ZrError) as ei:
        ctx.step_graph([st.desc])
    assert ei.value.status == zr.SINGULAR


def test_graph_fast_steps(ctx):
    """Steps that take the O(T log^2 T) solve captured in one graph: a lone
    fast step (its power sums on the auxiliary stream) and an uneven batch
    with two fast entries beside an O(T^2) one (the fast entries on streams
    of their own); replayed three times, each result equals generator truth
    and the direct call's."""
    ctx.solve_method(0, 1500)
    try:
        lone = Step(ctx, W.step_workload(531, 2600, 4, 12, 9))
        g = ctx.step_graph([lone.desc])
        try:
            for _ in range(3):
                lone.oc.zero_()
                lone.cnt.zero_()
                g.launch()
            g.status()
            e, c = lone.result()
            assert np.array_equal(e, lone.wl.exps) and np.array_equal(c, lone.wl.coef)
        finally:
            g.close()
        wls = [W.step_workload(532, 1800, 4, 10, 11), W.step_workload(533, 400, 5, 9, 21),
               W.step_workload(534, 3100, 3, 16, 5)]
        steps = [Step(ctx, wl, offset=i % 2) for i, wl in enumerate(wls)]
        g = ctx.step_graph([s.desc for s in steps])
        try:
            for _ in range(3):
                for s in steps:
                    s.oc.zero_()
                    s.cnt.zero_()
                g.launch()
            g.status()
            for s, wl in zip(steps, wls):
                e, c = s.result()
                assert np.array_equal(e, wl.exps) and np.array_equal(c, wl.coef)
        finally:
            g.close()
    finally:
        ctx.solve_method(0)
