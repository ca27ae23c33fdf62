"""The allocation-free Newton entry point (zr_newton_batched_noalloc).

It exists for callers that cannot allocate device memory and so cannot create
a context.  Its results must equal those of zr_newton_batched bit for bit
(the tolerance of every parity test here is zero), call after call, because
the two share the kernels and differ only in where the scratch table lives.
This file is collected last so that a stop at the first failure has already
run every other test.
"""
import random

import numpy as np
import pytest

from tests.gpuutil import d64, h64, rand_nodes, rand_res, zeros64
from tests.pyref import P63

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def zrmod():
    import torch

    import __graft_entry__ as ge
    from paper_2505_24256_gb300 import zr

    ge.build()
    assert torch.cuda.is_available()
    return zr


def test_noalloc_matches_context_version_on_consecutive_calls(zrmod):
    zr = zrmod
    ctx = zr.Context(P63)
    try:
        # two calls in a row with different sizes: the second must not see the first's table
        for npts, nterms, seed in [(21, 1000, 1), (9, 4097, 2), (64, 300, 3)]:
            rnd = random.Random(seed)
            x = d64(rand_nodes(rnd, npts, P63))
            vals = d64(rand_res(rnd, (npts, nterms), P63))
            want = zeros64(npts, nterms)
            ctx.newton_batched(nterms, npts, x, vals, nterms, want)
            got = zeros64(npts, nterms)
            assert zr.newton_batched_noalloc(P63, nterms, npts, x, vals, nterms, got) == zr.OK
            assert np.array_equal(h64(got), h64(want))
    finally:
        ctx.close()


def test_noalloc_limits_and_status_reset(zrmod):
    zr = zrmod
    x = d64(np.arange(1, 66, dtype=np.uint64))
    vals = zeros64(65, 4)
    out = zeros64(65, 4)
    assert zr.newton_batched_noalloc(P63, 4, 65, x, vals, 4, out) == zr.INVALID_ARG      # above the maximum
    assert zr.newton_batched_noalloc(2**63 + 1, 4, 3, x, vals, 4, out) == zr.INVALID_ARG  # not a valid prime
    dup = d64([5, 9, 5])
    assert zr.newton_batched_noalloc(P63, 4, 3, dup, vals, 4, out) == zr.SINGULAR
    # the next call starts from a cleared status word
    rnd = random.Random(7)
    xs = rand_nodes(rnd, 5, P63)
    v = rand_res(rnd, (5, 10), P63)
    got = zeros64(5, 10)
    assert zr.newton_batched_noalloc(P63, 10, 5, d64(xs), d64(v), 10, got) == zr.OK
    import oracle
    assert np.array_equal(h64(got), oracle.newton_batched(xs, v))
