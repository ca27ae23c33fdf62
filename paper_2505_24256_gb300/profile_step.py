"""Runs Zippel steps of a named workload on cuda:0 for profiling.

    python -m paper_2505_24256_gb300.profile_step [--workload batched|large]
        [--steps N] [--plan TILE,NB] [--probe-sets M] [--T N]
        [--method auto|quadratic|fast]

The probes are generated M times (default 1) by the GPU evaluator, each
timed with CUDA events; then N steps run back to back (the first is a
warm-up when N > 1) with the given solve plan (else the planner's model),
and the per-phase device times of the context profiler are printed.  Under
ncu, select the solve kernel with -k regex:k_solve (or the evaluator's
product with -k regex:k_eval_ring) and skip the warm-up launch with -s 1.
--method picks the solve: the library's choice by size, always the O(T^2)
kernels, or the O(T log^2 T) path (phase "fast").
"""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="batched", choices=["batched", "large"])
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--plan", default=None, help="solve plan TILE,NB (default: the planner's model)")
    ap.add_argument("--probe-sets", type=int, default=1, help="probe generations, each timed")
    ap.add_argument("--T", type=int, default=0,
                    help="the large workload's recipe at this many terms (a smaller case for counters)")
    ap.add_argument("--method", default="auto", choices=["auto", "quadratic", "fast"])
    args = ap.parse_args()
    if args.plan:
        os.environ["ZR_SOLVE_PLAN"] = args.plan
    import numpy as np
    import torch

    from paper_2505_24256_gb300 import build, workloads as W, zr

    build.build()
    if args.workload == "batched":
        wl = W.batched_step_1e4()
    elif args.T:
        wl = W.step_workload(1003, args.T, 7, 12, 9, name=f"step_T{args.T}_S9")
    else:
        wl = W.large_step_2p20()
    dev = torch.device("cuda:0")

    def d64(a):
        return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint64).view(np.int64)).to(dev)

    ctx = zr.Context(wl.p)
    ctx.solve_method({"auto": 0, "quadratic": 1, "fast": 2}[args.method])
    fe, fc = torch.from_numpy(wl.exps).to(dev), d64(wl.coef)     # kept alive: zr_poly holds raw pointers
    f = ctx.poly(wl.nv, wl.exps.shape[0], fe, fc)
    y, cs, z = d64(wl.y), d64(wl.cs), d64(wl.z)
    ske = torch.from_numpy(wl.skel).to(dev)
    skel = ctx.poly(wl.nv, wl.T, ske)
    b = torch.empty((wl.S, wl.T), dtype=torch.int64, device=dev)
    probe_ms = []
    for _ in range(max(1, args.probe_sets)):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ctx.zippel_probes(f, wl.k, y, wl.S, cs, z, wl.T, 0, b, wl.T)
        e1.record()
        torch.cuda.synchronize()
        probe_ms.append(e0.elapsed_time(e1))
    cap = wl.T * wl.S
    oe = torch.zeros((cap, wl.nv), dtype=torch.uint8, device=dev)
    oc = torch.zeros(cap, dtype=torch.int64, device=dev)
    ctx.profile(True)
    n = 0
    for _ in range(args.steps):
        n = ctx.zippel_step(skel, wl.k, y, wl.S, cs, b, wl.T, 0, oe, oc, cap)
    torch.cuda.synchronize()
    got = oc[:n].cpu().numpy().view(np.uint64)
    ok = n == wl.exps.shape[0] and np.array_equal(got, wl.coef)
    phases = {ph: ctx.profile_query(ph)[0] / args.steps for ph in zr.Context.PHASES[:7] + ("fast", "ntt", "desc", "psum")}
    ntt_ms, ntt_n = ctx.profile_query("ntt")
    line = {"workload": wl.name, "steps": args.steps, "method": args.method, "plan": ctx.step_plan(wl.T, wl.S),
            "phase_ms": phases,
            "ntt": {"launches": ntt_n, "ms": ntt_ms, "butterflies": ctx.profile_work("ntt")},
            "desc": {"launches": ctx.profile_query("desc")[1], "ms": ctx.profile_query("desc")[0],
                     "butterflies": ctx.profile_work("desc")},
            "psum": {"launches": ctx.profile_query("psum")[1], "ms": ctx.profile_query("psum")[0],
                     "shoup_steps": ctx.profile_work("psum")},
            "probe_ms": probe_ms, "check": "generator truth" if ok else "MISMATCH"}
    if not ok:
        line["terms"] = [int(n), int(wl.exps.shape[0])]
        if n == wl.exps.shape[0]:
            bad = np.nonzero(got != wl.coef)[0]
            line["bad_terms"] = int(bad.size)
            line["bad_roots"] = int(np.unique(bad // wl.S).size)
            line["first_bad"] = [[int(i // wl.S), int(i % wl.S)] for i in bad[:6]]
    print(json.dumps(line), flush=True)
    ctx.close()
    return 0 if ok else 1


if __name__ == "__main__":
    rc = main()
    sys.stdout.flush()
    os._exit(rc)
