"""Thin ctypes binding of libzr.so (include/zr.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Device arrays are torch tensors on the current CUDA device (uint64
data held in int64 tensors, exponent rows in uint8 tensors); streams are
``torch.cuda.Stream`` objects or raw handles.  There is no CPU fallback:
loading fails loudly when the library is missing.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "libzr.so")

OK, INVALID_ARG, SINGULAR, POLE, OOM, TIMEOUT, CUDA, UNLUCKY, BUSY, CAPACITY, DEGREE = range(11)
P63 = 2**63 - 25


class ZrError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"zr status {status}: {msg}")
        self.status = status


class zr_vsys(ctypes.Structure):
    _fields_ = [("T", ctypes.c_int64), ("S", ctypes.c_int32), ("offset", ctypes.c_int32),
                ("v", ctypes.c_void_p), ("b", ctypes.c_void_p), ("ldb", ctypes.c_int64),
                ("c", ctypes.c_void_p), ("ldc", ctypes.c_int64)]


class zr_poly(ctypes.Structure):
    _fields_ = [("nv", ctypes.c_int32), ("T", ctypes.c_int64), ("exps", ctypes.c_void_p),
                ("coef", ctypes.c_void_p)]


class zr_step_desc(ctypes.Structure):
    _fields_ = [("skel", zr_poly), ("newvar", ctypes.c_int32), ("S", ctypes.c_int32), ("offset", ctypes.c_int32),
                ("pad", ctypes.c_int32), ("y", ctypes.c_void_p), ("samples", ctypes.c_void_p),
                ("probes", ctypes.c_void_p), ("ldb", ctypes.c_int64), ("out_exps", ctypes.c_void_p),
                ("out_coef", ctypes.c_void_p), ("out_cap", ctypes.c_int64), ("out_count", ctypes.c_void_p)]


BB_POLY, BB_RATIONAL, BB_CALL_POLY, BB_CALL_RATIONAL = range(4)

# zr_eval_fn(user, npts, nv, pts, out, stream) -> 0, or nonzero at a pole
zr_eval_fn = ctypes.CFUNCTYPE(ctypes.c_int32, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p,
                              ctypes.c_void_p, ctypes.c_void_p)


class zr_blackbox(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("nv", ctypes.c_int32),
                ("TN", ctypes.c_int64), ("N_exps", ctypes.c_void_p), ("N_coef", ctypes.c_void_p),
                ("TD", ctypes.c_int64), ("D_exps", ctypes.c_void_p), ("D_coef", ctypes.c_void_p),
                ("eval", zr_eval_fn), ("user", ctypes.c_void_p)]


class zr_recon_params(ctypes.Structure):
    _fields_ = [("nv", ctypes.c_int32), ("offset", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("degN", ctypes.c_void_p), ("degD", ctypes.c_void_p), ("verify", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class zr_result(ctypes.Structure):
    _fields_ = [("nv", ctypes.c_int32), ("rational", ctypes.c_int32),
                ("TN", ctypes.c_int64), ("N_exps", ctypes.POINTER(ctypes.c_uint8)),
                ("N_coef", ctypes.POINTER(ctypes.c_uint64)),
                ("TD", ctypes.c_int64), ("D_exps", ctypes.POINTER(ctypes.c_uint8)),
                ("D_coef", ctypes.POINTER(ctypes.c_uint64)),
                ("steps", ctypes.c_int32), ("redraws", ctypes.c_int32), ("device_ms", ctypes.c_double)]


class zr_peaks(ctypes.Structure):
    _fields_ = [("mac_per_s", ctypes.c_double), ("chain_per_s", ctypes.c_double),
                ("imad_lo_per_s", ctypes.c_double), ("imad_hi_per_s", ctypes.c_double),
                ("butterfly_per_s", ctypes.c_double), ("sms", ctypes.c_int32), ("pad", ctypes.c_int32)]


class zr_request(ctypes.Structure):
    _fields_ = [("bb", zr_blackbox), ("prm", zr_recon_params)]


class zr_serve_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("failed", ctypes.c_int64),
                ("terms", ctypes.c_int64), ("ticks", ctypes.c_int64), ("batch_entries", ctypes.c_int64),
                ("max_active", ctypes.c_int32), ("pad", ctypes.c_int32), ("p50_ms", ctypes.c_double),
                ("p99_ms", ctypes.c_double), ("mean_ms", ctypes.c_double), ("wall_s", ctypes.c_double),
                ("terms_per_s", ctypes.c_double)]


_V, _I32, _I64, _U64, _P = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_void_p
_ST = ctypes.c_int

# exported symbol -> (restype, argtypes); the list mirrors include/zr.h
SIGNATURES = {
    "zr_create": (_ST, [_U64, ctypes.POINTER(_V)]),
    "zr_destroy": (None, [_V]),
    "zr_last_error": (ctypes.c_char_p, [_V]),
    "zr_status_string": (ctypes.c_char_p, [_ST]),
    "zr_prime": (_U64, [_V]),
    "zr_workspace_bytes": (ctypes.c_size_t, [_V]),
    "zr_launch_count": (_U64, []),
    "zr_profile_enable": (_ST, [_V, _I32]),
    "zr_profile_query": (_ST, [_V, _I32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_I64)]),
    "zr_profile_work": (_ST, [_V, _I32, ctypes.POINTER(ctypes.c_double)]),
    "zr_autotune_step": (_ST, [_V, _I64, _I32, _I32, _V]),
    "zr_step_plan": (_ST, [_V, _I64, _I32, ctypes.POINTER(_I32), ctypes.POINTER(_I32)]),
    "zr_solve_method": (_ST, [_V, _I32, _I64]),
    "zr_vandermonde_solve_batched": (_ST, [_V, _I32, _P, _V]),
    "zr_vandermonde_solve_plain": (_ST, [_V, _I32, _P, _V]),
    "zr_newton_batched": (_ST, [_V, _I64, _I32, _P, _P, _I64, _P, _V]),
    "zr_anchor_values": (_ST, [_V, _I64, _I32, _P, _I32, _P, _I32, _P, _V]),
    "zr_newton_batched_noalloc": (_ST, [_U64, _I64, _I32, _P, _P, _I64, _P, _V]),
    "zr_zippel_step": (_ST, [_V, _P, _I32, _P, _I32, _P, _P, _I64, _I32, _P, _P, _I64, _P, _V]),
    "zr_zippel_step_async": (_ST, [_V, _P, _I32, _P, _I32, _P, _P, _I64, _I32, _P, _P, _I64, _P, _V]),
    "zr_stream_status": (_ST, [_V, _V]),
    "zr_zippel_step_batched": (_ST, [_V, _I32, _P, _V]),
    "zr_zippel_step_host": (_ST, [_V, _P, _I32, _P, _I32, _P, _P, _I64, _I32, _P, _P, _I64, _P, _V]),
    "zr_zippel_probes": (_ST, [_V, _P, _I32, _P, _I32, _P, _P, _I64, _I32, _P, _I64, _V]),
    "zr_eval_points": (_ST, [_V, _P, _I64, _P, _P, _V]),
    "zr_probe_points": (_ST, [_V, _I32, _I32, _P, _I32, _P, _P, _I64, _I32, _P, _V]),
    "zr_lift_words": (_I32, [_I32]),
    "zr_rational_lift": (_ST, [_V, _I32, _P, _I64, _P, _I64, _I32, _P, _P, _P, _V]),
    "zr_zippel_step_balanced": (_ST, [_V, _P, _P, _I32, _P, _I32, _I32, _P, _P, _I64, _I32, _P, _P, _I64, _P,
                                      _P, _P, _I64, _P, _V]),
    "zr_reconstruct": (_ST, [_V, _P, _P, ctypes.POINTER(ctypes.POINTER(zr_result)), _V]),
    "zr_result_free": (None, [ctypes.POINTER(zr_result)]),
    "zr_measure_peaks": (_ST, [_V, _P, _V]),
    "zr_check_bounded_wait": (_ST, [_V, ctypes.c_uint32, _V]),
    "zr_check_arith": (_ST, [_V, _I32, _I64, _I64, _P, _P, _P, _P, _V]),
    "zr_step_graph_create": (_ST, [_V, _I32, _P, _V, ctypes.POINTER(_V)]),
    "zr_step_graph_launch": (_ST, [_V, _V]),
    "zr_step_graph_status": (_ST, [_V, _V]),
    "zr_step_graph_kernels": (_U64, [_V]),
    "zr_step_graph_destroy": (None, [_V]),
    "zr_serve_create": (_ST, [_V, ctypes.c_size_t, _I32, ctypes.POINTER(_V)]),
    "zr_serve_submit": (_ST, [_V, _P, ctypes.POINTER(_U64)]),
    "zr_serve_poll": (_ST, [_V, _U64, ctypes.POINTER(ctypes.POINTER(zr_result))]),
    "zr_serve_wait": (_ST, [_V, _U64, _I64, ctypes.POINTER(ctypes.POINTER(zr_result))]),
    "zr_serve_stats_get": (_ST, [_V, ctypes.POINTER(zr_serve_stats)]),
    "zr_serve_destroy": (None, [_V]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Loads libzr.so; raises when it has not been built (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libzr.so not found at {path}: build it with paper_2505_24256_gb300.build.build() "
                           "(there is no CPU fallback)")
    L = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(L, name, None)
        if fn is None:
            continue
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class Context:
    """A zr_ctx bound to the current CUDA device."""

    def __init__(self, prime: int = P63):
        L = load()
        h = ctypes.c_void_p()
        st = L.zr_create(prime, ctypes.byref(h))
        if st != OK:
            raise ZrError(st, f"zr_create({prime}) failed: {L.zr_status_string(st).decode()}")
        self._h = h
        self.L = L
        self.p = prime

    def close(self):
        if getattr(self, "_h", None):
            self.L.zr_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def check(self, st: int, what: str):
        if st != OK:
            msg = self.L.zr_last_error(self._h).decode(errors="replace")
            raise ZrError(st, f"{what}: {msg}")

    def check_bounded_wait(self, tries=4096, stream=None) -> int:
        """Status of a device wait that nothing completes (TIMEOUT when it gives up as designed)."""
        return int(self.L.zr_check_bounded_wait(self._h, tries, _stream(stream)))

    ARITH_OPS = {"mulmod": 0, "reduce": 1, "shoup_pre": 2, "shoup_lazy": 3, "pow": 4, "inv": 5, "dot": 6, "add": 7,
                 "sub": 8, "batch_inv": 9}

    def check_arith(self, op, n, a, b, out, hits=None, length=1, stream=None):
        """zr_check_arith: device primitive `op` on device arrays (see the header)."""
        self.check(self.L.zr_check_arith(self._h, self.ARITH_OPS[op], n, length, _ptr(a), _ptr(b), _ptr(out),
                                         _ptr(hits), _stream(stream)), "zr_check_arith")

    def measure_peaks(self, stream=None) -> dict:
        """Measured MAC / chain-step / IMAD / transform-butterfly rates (operations per second)."""
        p = zr_peaks()
        self.check(self.L.zr_measure_peaks(self._h, ctypes.byref(p), _stream(stream)), "zr_measure_peaks")
        return {f: getattr(p, f) for f, _ in zr_peaks._fields_ if f != "pad"}

    def workspace_bytes(self) -> int:
        return int(self.L.zr_workspace_bytes(self._h))

    PHASES = ("anchor", "master", "expand", "carry", "solve", "newton", "compact", "eval", "fast", "ntt", "desc", "psum")
    SOLVE_AUTO, SOLVE_QUADRATIC, SOLVE_FAST = 0, 1, 2

    def solve_method(self, method, crossover=0):
        """zr_solve_method: 0 by size (fast from `crossover` terms), 1 always O(T^2), 2 fast where supported."""
        self.check(self.L.zr_solve_method(self._h, method, crossover), "zr_solve_method")

    def profile(self, on: bool = True):
        self.check(self.L.zr_profile_enable(self._h, 1 if on else 0), "zr_profile_enable")

    def autotune_step(self, T, S, budget=12, stream=None):
        self.check(self.L.zr_autotune_step(self._h, T, S, budget, _stream(stream)), "zr_autotune_step")

    def step_plan(self, T, S):
        tile, nb = ctypes.c_int32(), ctypes.c_int32()
        self.check(self.L.zr_step_plan(self._h, T, S, ctypes.byref(tile), ctypes.byref(nb)), "zr_step_plan")
        return tile.value, nb.value

    def profile_query(self, phase):
        idx = self.PHASES.index(phase) if isinstance(phase, str) else int(phase)
        ms = ctypes.c_double()
        n = ctypes.c_int64()
        self.check(self.L.zr_profile_query(self._h, idx, ctypes.byref(ms), ctypes.byref(n)), "zr_profile_query")
        return ms.value, n.value

    def profile_work(self, phase):
        """zr_profile_work: the algorithmic work recorded with a phase (butterflies for "ntt" and "desc")."""
        idx = self.PHASES.index(phase) if isinstance(phase, str) else int(phase)
        u = ctypes.c_double()
        self.check(self.L.zr_profile_work(self._h, idx, ctypes.byref(u)), "zr_profile_work")
        return u.value


    # ------------------------------------------------------------------ calls
    def vandermonde_solve(self, systems, stream=None, plain=False):
        """systems: list of dicts with T, S, offset, v, b, ldb, c, ldc (tensors)."""
        arr = (zr_vsys * max(len(systems), 1))()
        for i, s in enumerate(systems):
            arr[i] = zr_vsys(s["T"], s["S"], s.get("offset", 0), _ptr(s["v"]), _ptr(s["b"]), s["ldb"],
                             _ptr(s["c"]), s["ldc"])
        fn = self.L.zr_vandermonde_solve_plain if plain else self.L.zr_vandermonde_solve_batched
        self.check(fn(self._h, len(systems), ctypes.cast(arr, ctypes.c_void_p), _stream(stream)),
                   "zr_vandermonde_solve")

    def newton_batched(self, nterms, npts, x, vals, ld, coef, stream=None):
        self.check(self.L.zr_newton_batched(self._h, nterms, npts, _ptr(x), _ptr(vals), ld, _ptr(coef),
                                            _stream(stream)), "zr_newton_batched")

    def anchor_values(self, T, nv, exps, k, y, offset, v, stream=None):
        self.check(self.L.zr_anchor_values(self._h, T, nv, _ptr(exps), k, _ptr(y), offset, _ptr(v),
                                           _stream(stream)), "zr_anchor_values")

    @staticmethod
    def poly(nv, T, exps, coef=None):
        return zr_poly(nv, T, _ptr(exps), _ptr(coef))

    def zippel_step(self, skel: zr_poly, newvar, y, S, samples, probes, ldb, offset, out_exps, out_coef,
                    out_cap, stream=None):
        n = ctypes.c_int64()
        st = self.L.zr_zippel_step(self._h, ctypes.byref(skel), newvar, _ptr(y), S, _ptr(samples), _ptr(probes),
                                   ldb, offset, _ptr(out_exps), _ptr(out_coef), out_cap, ctypes.byref(n),
                                   _stream(stream))
        self.check(st, "zr_zippel_step")
        return n.value

    def zippel_step_async(self, skel: zr_poly, newvar, y, S, samples, probes, ldb, offset, out_exps, out_coef,
                          out_cap, d_count, stream=None):
        st = self.L.zr_zippel_step_async(self._h, ctypes.byref(skel), newvar, _ptr(y), S, _ptr(samples),
                                         _ptr(probes), ldb, offset, _ptr(out_exps), _ptr(out_coef), out_cap,
                                         _ptr(d_count), _stream(stream))
        self.check(st, "zr_zippel_step_async")

    def zippel_step_batched(self, steps, stream=None):
        """steps: list of dicts with skel (zr_poly), newvar, S, offset, y, samples, probes, ldb, out_exps,
        out_coef, out_cap, out_count (device int64 tensor of one element)."""
        arr = (zr_step_desc * max(len(steps), 1))()
        for i, d in enumerate(steps):
            arr[i] = zr_step_desc(d["skel"], d["newvar"], d["S"], d.get("offset", 0), 0, _ptr(d["y"]),
                                  _ptr(d["samples"]), _ptr(d["probes"]), d["ldb"], _ptr(d["out_exps"]),
                                  _ptr(d["out_coef"]), d["out_cap"], _ptr(d["out_count"]))
        self.check(self.L.zr_zippel_step_batched(self._h, len(steps), ctypes.cast(arr, ctypes.c_void_p),
                                                 _stream(stream)), "zr_zippel_step_batched")

    def step_graph(self, steps, stream=None):
        """A StepGraph for the given step descriptors (same dicts as zippel_step_batched)."""
        arr = (zr_step_desc * len(steps))()
        for i, d in enumerate(steps):
            arr[i] = zr_step_desc(d["skel"], d["newvar"], d["S"], d.get("offset", 0), 0, _ptr(d["y"]),
                                  _ptr(d["samples"]), _ptr(d["probes"]), d["ldb"], _ptr(d["out_exps"]),
                                  _ptr(d["out_coef"]), d["out_cap"], _ptr(d["out_count"]))
        h = ctypes.c_void_p()
        st = self.L.zr_step_graph_create(self._h, len(steps), ctypes.cast(arr, ctypes.c_void_p), _stream(stream),
                                         ctypes.byref(h))
        if st != OK and h.value:
            self.L.zr_step_graph_destroy(h)
        self.check(st, "zr_step_graph_create")
        return StepGraph(self, h)

    def stream_status(self, stream=None):
        self.check(self.L.zr_stream_status(self._h, _stream(stream)), "zr_stream_status")

    def zippel_step_host(self, skel: zr_poly, newvar, y, S, samples, probes, ldb, offset, out_exps, out_coef,
                         out_cap, stream=None):
        n = ctypes.c_int64()
        st = self.L.zr_zippel_step_host(self._h, ctypes.byref(skel), newvar, _ptr(y), S, _ptr(samples),
                                        _ptr(probes), ldb, offset, _ptr(out_exps), _ptr(out_coef), out_cap,
                                        ctypes.byref(n), _stream(stream))
        self.check(st, "zr_zippel_step_host")
        return n.value

    def zippel_probes(self, f: zr_poly, k, y, S, samples, z, T, offset, out, ldo, stream=None):
        self.check(self.L.zr_zippel_probes(self._h, ctypes.byref(f), k, _ptr(y), S, _ptr(samples), _ptr(z), T,
                                           offset, _ptr(out), ldo, _stream(stream)), "zr_zippel_probes")

    def eval_points(self, f: zr_poly, npts, pts, out, stream=None):
        self.check(self.L.zr_eval_points(self._h, ctypes.byref(f), npts, _ptr(pts), _ptr(out), _stream(stream)),
                   "zr_eval_points")

    def probe_points(self, nv, k, y, S, samples, z, T, offset, pts, stream=None):
        self.check(self.L.zr_probe_points(self._h, nv, k, _ptr(y), S, _ptr(samples), _ptr(z), T, offset, _ptr(pts),
                                          _stream(stream)), "zr_probe_points")

    def zippel_step_balanced(self, skelN: zr_poly, skelD: zr_poly, newvar, y, dN, dD, samples, fvals, ldf, offset,
                             outN_exps, outN_coef, outN_cap, outD_exps, outD_coef, outD_cap, stream=None):
        nN = ctypes.c_int64()
        nD = ctypes.c_int64()
        st = self.L.zr_zippel_step_balanced(self._h, ctypes.byref(skelN), ctypes.byref(skelD), newvar, _ptr(y),
                                            dN, dD, _ptr(samples), _ptr(fvals), ldf, offset, _ptr(outN_exps),
                                            _ptr(outN_coef), outN_cap, ctypes.byref(nN), _ptr(outD_exps),
                                            _ptr(outD_coef), outD_cap, ctypes.byref(nD), _stream(stream))
        self.check(st, "zr_zippel_step_balanced")
        return nN.value, nD.value

    def reconstruct(self, nv, degN, seed, N_exps, N_coef, D_exps=None, D_coef=None, degD=None, offset=0,
                    stream=None, verify=False):
        """Full reconstruction of a built-in sparse black box given by host
        (numpy) arrays (a negative degree bound: unknown, detected; verify:
        check every step at a fresh point).
        Returns ((N_exps, N_coef), (D_exps, D_coef) or None, info)."""
        rational = D_exps is not None
        N_exps = np.ascontiguousarray(N_exps, dtype=np.uint8)
        N_coef = np.ascontiguousarray(N_coef, dtype=np.uint64)
        bb = zr_blackbox(1 if rational else 0, nv, N_exps.shape[0], N_exps.ctypes.data, N_coef.ctypes.data, 0,
                         None, None)
        if rational:
            D_exps = np.ascontiguousarray(D_exps, dtype=np.uint8)
            D_coef = np.ascontiguousarray(D_coef, dtype=np.uint64)
            bb.TD, bb.D_exps, bb.D_coef = D_exps.shape[0], D_exps.ctypes.data, D_coef.ctypes.data
        dN = np.ascontiguousarray(degN, dtype=np.int32)
        dD = np.ascontiguousarray(degD if degD is not None else degN, dtype=np.int32)
        prm = zr_recon_params(nv, offset, seed, dN.ctypes.data, dD.ctypes.data, 1 if verify else 0, 0)
        res = ctypes.POINTER(zr_result)()
        st = self.L.zr_reconstruct(self._h, ctypes.byref(bb), ctypes.byref(prm), ctypes.byref(res), _stream(stream))
        self.check(st, "zr_reconstruct")
        return _take_result(self.L, res)


    def rational_lift(self, primes, res, ld, words, num, den, ok, stream=None):
        """zr_rational_lift over n = res's columns (device tensors; primes a host list)."""
        pr = np.ascontiguousarray(np.asarray(primes, dtype=np.uint64))
        n = int(ok.shape[0])
        self.check(self.L.zr_rational_lift(self._h, len(pr), pr.ctypes.data, n, _ptr(res), ld, words, _ptr(num),
                                           _ptr(den), _ptr(ok), _stream(stream)), "zr_rational_lift")

    def reconstruct_callback(self, nv, degN, seed, fn, rational=False, degD=None, TN_hint=0, TD_hint=0, offset=0,
                             stream=None, verify=False):
        """Full reconstruction of a black box given as a function
        fn(npts, nv, pts, out, stream) -> int over raw device pointers (pts:
        npts x nv residues, out: npts residues; nonzero return: a pole).
        Returns ((N_exps, N_coef), (D_exps, D_coef) or None, info)."""
        raised = []
        cb = _callback(fn, raised)
        bb = zr_blackbox(BB_CALL_RATIONAL if rational else BB_CALL_POLY, nv, TN_hint, None, None, TD_hint, None,
                         None, cb, None)
        dN = np.ascontiguousarray(degN, dtype=np.int32)
        dD = np.ascontiguousarray(degD if degD is not None else degN, dtype=np.int32)
        prm = zr_recon_params(nv, offset, seed, dN.ctypes.data, dD.ctypes.data, 1 if verify else 0, 0)
        res = ctypes.POINTER(zr_result)()
        st = self.L.zr_reconstruct(self._h, ctypes.byref(bb), ctypes.byref(prm), ctypes.byref(res), _stream(stream))
        if raised:
            if st == OK:
                self.L.zr_result_free(res)
            raise raised[0]
        self.check(st, "zr_reconstruct")
        return _take_result(self.L, res)


def lift_words(nprimes: int) -> int:
    return int(load().zr_lift_words(nprimes))


def words_to_int(words, signed: bool) -> int:
    """A little-endian uint64 word row as a Python integer."""
    v = 0
    for i, w in enumerate(np.asarray(words, dtype=np.uint64).tolist()):
        v |= int(w) << (64 * i)
    if signed and words.size and (int(words[-1]) >> 63):
        v -= 1 << (64 * words.size)
    return v


def launch_count() -> int:
    """Kernels launched by libzr in this process so far."""
    return int(load().zr_launch_count())


def newton_batched_noalloc(prime, nterms, npts, x, vals, ld, coef, stream=None) -> int:
    """zr_newton_batched_noalloc: the batched Newton interpolation without a
    context and without any allocation, for callers that cannot allocate
    device memory.  Returns the zr status code (0 on success)."""
    return int(load().zr_newton_batched_noalloc(prime, nterms, npts, _ptr(x), _ptr(vals), ld, _ptr(coef),
                                                 _stream(stream)))


class StepGraph:
    """zr_step_graph_*: captured steps re-run by one graph launch."""

    def __init__(self, ctx, h):
        self.ctx, self.L, self._h = ctx, ctx.L, h

    def launch(self, stream=None):
        self.ctx.check(self.L.zr_step_graph_launch(self._h, _stream(stream)), "zr_step_graph_launch")

    def status(self, stream=None):
        self.ctx.check(self.L.zr_step_graph_status(self._h, _stream(stream)), "zr_step_graph_status")

    @property
    def kernels(self) -> int:
        return int(self.L.zr_step_graph_kernels(self._h))

    def close(self):
        if getattr(self, "_h", None):
            self.L.zr_step_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _take_result(L, res):
    """Copies a zr_result into numpy arrays and frees it."""
    try:
        r = res.contents
        nv = r.nv
        Ne = np.ctypeslib.as_array(r.N_exps, shape=(r.TN * nv,)).reshape(r.TN, nv).copy() if r.TN else \
            np.zeros((0, nv), np.uint8)
        Nc = np.ctypeslib.as_array(r.N_coef, shape=(r.TN,)).copy() if r.TN else np.zeros(0, np.uint64)
        D = None
        if r.rational:
            De = np.ctypeslib.as_array(r.D_exps, shape=(r.TD * nv,)).reshape(r.TD, nv).copy() if r.TD else \
                np.zeros((0, nv), np.uint8)
            Dc = np.ctypeslib.as_array(r.D_coef, shape=(r.TD,)).copy() if r.TD else np.zeros(0, np.uint64)
            D = (De, Dc)
        info = dict(steps=r.steps, redraws=r.redraws, device_ms=r.device_ms)
        return (Ne, Nc), D, info
    finally:
        L.zr_result_free(res)


def make_request(nv, degN, seed, N_exps, N_coef, D_exps=None, D_coef=None, degD=None, offset=0, verify=False):
    """A zr_request plus the numpy arrays it points to (keep both alive until submitted)."""
    rational = D_exps is not None
    keep = [np.ascontiguousarray(N_exps, dtype=np.uint8), np.ascontiguousarray(N_coef, dtype=np.uint64),
            np.ascontiguousarray(degN, dtype=np.int32)]
    bb = zr_blackbox(1 if rational else 0, nv, keep[0].shape[0], keep[0].ctypes.data, keep[1].ctypes.data, 0, None,
                     None)
    if rational:
        keep += [np.ascontiguousarray(D_exps, dtype=np.uint8), np.ascontiguousarray(D_coef, dtype=np.uint64),
                 np.ascontiguousarray(degD if degD is not None else degN, dtype=np.int32)]
        bb.TD, bb.D_exps, bb.D_coef = keep[3].shape[0], keep[3].ctypes.data, keep[4].ctypes.data
        degd_ptr = keep[5].ctypes.data
    else:
        degd_ptr = keep[2].ctypes.data
    prm = zr_recon_params(nv, offset, seed, keep[2].ctypes.data, degd_ptr, 1 if verify else 0, 0)
    return zr_request(bb, prm), keep


def _callback(fn, raised):
    def call(user, npts, nv, pts, out, st):
        try:
            return int(fn(npts, nv, pts, out, st))
        except BaseException as e:  # the library sees a failed evaluation; the caller re-raises
            raised.append(e)
            return 1
    return zr_eval_fn(call)


def make_callback_request(nv, degN, seed, fn, rational=False, degD=None, TN_hint=0, TD_hint=0, offset=0,
                          verify=False):
    """A zr_request whose black box is fn(npts, nv, pts, out, stream) -> int
    over raw device pointers (see Context.reconstruct_callback), plus what it
    points to.  keep[-1] collects exceptions raised inside fn."""
    raised = []
    cb = _callback(fn, raised)
    dN = np.ascontiguousarray(degN, dtype=np.int32)
    dD = np.ascontiguousarray(degD if degD is not None else degN, dtype=np.int32)
    bb = zr_blackbox(BB_CALL_RATIONAL if rational else BB_CALL_POLY, nv, TN_hint, None, None, TD_hint, None, None,
                     cb, None)
    prm = zr_recon_params(nv, offset, seed, dN.ctypes.data, dD.ctypes.data, 1 if verify else 0, 0)
    return zr_request(bb, prm), [cb, dN, dD, raised]


def device_array(ptr: int, n: int):
    """A torch int64 view of n residues at a raw device address (no copy),
    for black-box functions that receive device pointers."""
    import torch

    class _Dev:
        __cuda_array_interface__ = dict(shape=(n,), typestr="<i8", data=(ptr, False), version=3)

    return torch.as_tensor(_Dev(), device="cuda")


class Server:
    """zr_serve_*: continuous batching of reconstructions on one context."""

    def __init__(self, ctx: Context, mem_budget: int, max_slots: int):
        self.ctx = ctx
        self.L = ctx.L
        h = ctypes.c_void_p()
        st = self.L.zr_serve_create(ctx.handle, mem_budget, max_slots, ctypes.byref(h))
        if st != OK:
            raise ZrError(st, "zr_serve_create")
        self._h = h

    def submit(self, req) -> int:
        t = ctypes.c_uint64()
        st = self.L.zr_serve_submit(self._h, ctypes.byref(req), ctypes.byref(t))
        if st != OK:
            raise ZrError(st, "zr_serve_submit")
        return t.value

    def poll(self, ticket):
        res = ctypes.POINTER(zr_result)()
        st = self.L.zr_serve_poll(self._h, ticket, ctypes.byref(res))
        if st == BUSY:
            return None
        if st != OK:
            raise ZrError(st, f"request {ticket}")
        return _take_result(self.L, res)

    def wait(self, ticket, timeout_s=600.0):
        res = ctypes.POINTER(zr_result)()
        st = self.L.zr_serve_wait(self._h, ticket, int(timeout_s * 1e6), ctypes.byref(res))
        if st != OK:
            raise ZrError(st, f"request {ticket}")
        return _take_result(self.L, res)

    def stats(self) -> dict:
        s = zr_serve_stats()
        st = self.L.zr_serve_stats_get(self._h, ctypes.byref(s))
        if st != OK:
            raise ZrError(st, "zr_serve_stats_get")
        return {f: getattr(s, f) for f, _ in zr_serve_stats._fields_ if f != "pad"}

    def close(self):
        if getattr(self, "_h", None):
            self.L.zr_serve_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
