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


def test_noalloc_allocates_no_device_memory(zrmod):
    """The defining property: after a warm-up call (which looks the scratch
    array up), calls of different sizes leave the device's free memory
    unchanged.  Every input and output is allocated before the first reading."""
    import torch

    zr = zrmod
    rnd = random.Random(11)
    cases = []
    for npts, nterms in [(3, 10), (21, 5000), (64, 2048), (40, 1)]:
        x = d64(rand_nodes(rnd, npts, P63))
        vals = d64(rand_res(rnd, (npts, nterms), P63))
        cases.append((npts, nterms, x, vals, zeros64(npts, nterms)))
    npts, nterms, x, vals, out = cases[0]
    assert zr.newton_batched_noalloc(P63, nterms, npts, x, vals, nterms, out) == zr.OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(2):
        for npts, nterms, x, vals, out in cases:
            assert zr.newton_batched_noalloc(P63, nterms, npts, x, vals, nterms, out) == zr.OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_on_a_second_device(zrmod):
    """The scratch address and the kernels' shared-memory limits are set up per
    device: npts = 64 (above the default shared-memory limit) on device 1 after
    device 0 gives the context version's result."""
    import torch

    zr = zrmod
    if torch.cuda.device_count() < 2:
        pytest.skip("needs two visible GPUs")
    rnd = random.Random(12)
    xs, v = rand_nodes(rnd, 64, P63), rand_res(rnd, (64, 300), P63)
    for d in (0, 1):
        with torch.cuda.device(d):
            x = torch.from_numpy(xs.view(np.int64)).to(f"cuda:{d}")
            vals = torch.from_numpy(v.view(np.int64)).to(f"cuda:{d}")
            got = torch.zeros((64, 300), dtype=torch.int64, device=f"cuda:{d}")
            assert zr.newton_batched_noalloc(P63, 300, 64, x, vals, 300, got) == zr.OK
            ctx = zr.Context(P63)
            try:
                want = torch.zeros_like(got)
                ctx.newton_batched(300, 64, x, vals, 300, want)
            finally:
                ctx.close()
            assert np.array_equal(h64(got), h64(want))
