"""Plain CPU oracle for the Zippel step -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline /
reference leg may import this package.  The product path (the CUDA library in
``paper_2505_24256_gb300``) never imports it, and this package imports nothing
from the product path: the two share no code.  The only module both sides use
is the seeded input generator (``paper_2505_24256_gb300.workloads``), which
holds random-number generation and sampling only.

The arithmetic lives in ``zr_oracle.c`` (compiled to ``_build/libzroracle.so``
by :func:`build`); this module only marshals numpy arrays through ctypes.
Every routine is the plain definition the paper states (see the C file's
header): 128-bit products reduced with ``%``, sums reduced at every step,
inverses by the extended Euclidean algorithm, the transposed Vandermonde solve
through the master polynomial and synthetic division (Sec. 1, Sec. 2.2),
Newton (Eq. newton) and Thiele (Eq. thiele) interpolation, and the balanced
scaling of Sec. 2.2.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "zr_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libzroracle.so")

OK, INVALID_ARG, SINGULAR, POLE, OOM, UNLUCKY, CAPACITY, DEGREE = 0, 1, 2, 3, 4, 7, 9, 10

P63 = 2**63 - 25


class OracleError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: oracle status {status}")
        self.status = status


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C11, pthreads)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-std=gnu11", "-Wall", "-shared", "-fPIC", "-pthread",
                        "-o", tmp, _SRC], check=True)
        os.replace(tmp, _LIB)
    return _LIB


_lib = None

_u64p = ctypes.POINTER(ctypes.c_uint64)
_i64p = ctypes.POINTER(ctypes.c_int64)
_i32p = ctypes.POINTER(ctypes.c_int32)
_u8p = ctypes.POINTER(ctypes.c_uint8)
_u64, _i64, _i32 = ctypes.c_uint64, ctypes.c_int64, ctypes.c_int32

_SIGS = {
    "zro_mulmod": (_u64, [_u64, _u64, _u64]),
    "zro_addmod": (_u64, [_u64, _u64, _u64]),
    "zro_submod": (_u64, [_u64, _u64, _u64]),
    "zro_powmod": (_u64, [_u64, _u64, _u64]),
    "zro_invmod": (_u64, [_u64, _u64]),
    "zro_arith_batch": (ctypes.c_int, [_i32, _i64, _i64, _u64p, _u64p, _u64, _u64p]),
    "zro_is_prime": (ctypes.c_int, [_u64]),
    "zro_default_threads": (ctypes.c_int, []),
    "zro_splitmix_at": (_u64, [_u64, _u64]),
    "zro_anchor_values": (None, [_i64, _i32, _u8p, _i32, _u64p, _u64, _u64p]),
    "zro_check_nodes": (ctypes.c_int, [_i64, _u64p, _i32]),
    "zro_master_poly": (None, [_i64, _u64p, _u64, _u64p]),
    "zro_synthetic_division": (None, [_i64, _u64p, _u64, _u64, _u64p]),
    "zro_tvandermonde_solve": (ctypes.c_int, [_i64, _i32, _i32, _u64p, _u64p, _i64, _u64, _u64p, _i64, _i32]),
    "zro_tvandermonde_solve_roots": (ctypes.c_int, [_i64, _i32, _i32, _u64p, _u64p, _u64p, _i64, _i64, _i64p,
                                                    _u64, _u64p, _i64, _i32]),
    "zro_newton": (ctypes.c_int, [_i32, _u64p, _u64p, _u64, _u64p]),
    "zro_newton_batched": (ctypes.c_int, [_i64, _i32, _u64p, _u64p, _i64, _u64, _u64p]),
    "zro_eval_points": (None, [_i64, _i32, _u8p, _u64p, _i64, _u64p, _u64, _u64p]),
    "zro_zippel_probes": (ctypes.c_int, [_i64, _i32, _u8p, _u64p, _i32, _u64p, _i32, _u64p, _u64p, _i64, _i32,
                                         _u64, _i32, _u64p, _i64]),
    "zro_zippel_probes_sampled": (ctypes.c_int, [_i64, _i32, _u8p, _u64p, _i32, _u64p, _i32, _u64p, _u64p, _i32,
                                                 _i64, _i32p, _i64p, _u64, _i32, _u64p]),
    "zro_zippel_step": (ctypes.c_int, [_i64, _i32, _u8p, _i32, _u64p, _i32, _u64p, _u64p, _i64, _i32, _u64, _i32,
                                       _i64, _i64p, _u8p, _u64p, _u64p]),
    "zro_thiele": (ctypes.c_int, [_i32, _u64p, _u64p, _u64, _i32, _i32, _i32p, _i32p, _u64p, _u64p]),
    "zro_balance_probes": (ctypes.c_int, [_i32, _u64p, _u64p, _i64, _i64, _u64p, _i32, _i32, _i64, _i64, _u64,
                                          _i32, _u64p, _i64, _u64p, _i64]),
    "zro_reconstruct_poly": (ctypes.c_int, [_i64, _i32, _u8p, _u64p, _i32p, _u64, _i32, _u64, _i32, _i64, _i64p,
                                            _u8p, _u64p, _i64p]),
    "zro_reconstruct_rational": (ctypes.c_int, [_i64, _u8p, _u64p, _i64, _u8p, _u64p, _i32, _i32p, _i32p, _u64,
                                                _i32, _u64, _i32, _i64, _i64, _i64p, _u8p, _u64p, _i64p, _u8p,
                                                _u64p]),
}


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _p(a, ct=_u64p):
    return a.ctypes.data_as(ct) if a is not None else None


def _u64arr(x, n=None):
    a = np.ascontiguousarray(np.asarray(x, dtype=np.uint64))
    if n is not None and a.size < n:
        raise ValueError("array too short")
    return a


def _u8arr(x):
    return np.ascontiguousarray(np.asarray(x, dtype=np.uint8))


def _check(st, what):
    if st != OK:
        raise OracleError(st, what)


# ---------------------------------------------------------------- scalars

def mulmod(a, b, p=P63):
    return int(lib().zro_mulmod(a, b, p))


def addmod(a, b, p=P63):
    return int(lib().zro_addmod(a, b, p))


def submod(a, b, p=P63):
    return int(lib().zro_submod(a, b, p))


def powmod(a, e, p=P63):
    return int(lib().zro_powmod(a, e, p))


def invmod(a, p=P63):
    return int(lib().zro_invmod(a, p))


def is_prime(n):
    return bool(lib().zro_is_prime(n))


ARITH_OPS = {"mulmod": 0, "reduce": 1, "shoup_pre": 2, "shoup_lazy": 3, "pow": 4, "inv": 5, "dot": 6, "add": 7,
             "sub": 8, "batch_inv": 9}


def arith_batch(op, a, b=None, p=P63, length=1):
    """Elementwise modular primitive `op` (see zro_arith_batch) on uint64
    arrays; for "dot" the operands hold len(out) groups of `length` terms."""
    a = np.ascontiguousarray(a, dtype=np.uint64)
    b = np.ascontiguousarray(np.zeros_like(a) if b is None else b, dtype=np.uint64)
    n = a.size // length if op == "dot" else a.size
    out = np.zeros(n, dtype=np.uint64)
    r = lib().zro_arith_batch(ARITH_OPS[op], n, length, _p(a), _p(b), p, _p(out))
    if r:
        raise OracleError(r, f"arith_batch({op})")
    return out


def default_threads():
    return int(lib().zro_default_threads())


def splitmix_at(key, n):
    return int(lib().zro_splitmix_at(key, n))


# ---------------------------------------------------------------- step pieces

def anchor_values(exps, k, y, p=P63):
    exps = _u8arr(exps)
    T, nv = exps.shape
    y = _u64arr(y)
    v = np.zeros(T, dtype=np.uint64)
    lib().zro_anchor_values(T, nv, _p(exps, _u8p), k, _p(y), p, _p(v))
    return v


def check_nodes(v, offset=0):
    v = _u64arr(v)
    return int(lib().zro_check_nodes(v.size, _p(v), offset))


def master_poly(v, p=P63):
    v = _u64arr(v)
    m = np.zeros(v.size + 1, dtype=np.uint64)
    lib().zro_master_poly(v.size, _p(v), p, _p(m))
    return m


def synthetic_division(m, vj, p=P63):
    m = _u64arr(m)
    T = m.size - 1
    q = np.zeros(max(T, 1), dtype=np.uint64)
    lib().zro_synthetic_division(T, _p(m), vj, p, _p(q))
    return q[:T]


def tvandermonde_solve(v, b, offset=0, p=P63, nthreads=0):
    """Solve sum_j c_j v_j^(k+offset) = b[s][k] for every row s of b."""
    v = _u64arr(v)
    b = np.ascontiguousarray(np.atleast_2d(np.asarray(b, dtype=np.uint64)))
    S, T = b.shape
    if T != v.size:
        raise ValueError("b must have T columns")
    c = np.zeros((S, T), dtype=np.uint64)
    _check(lib().zro_tvandermonde_solve(T, S, offset, _p(v), _p(b), T, p, _p(c), T, nthreads), "tvandermonde_solve")
    return c


def tvandermonde_solve_roots(v, m, b, roots, offset=0, p=P63, nthreads=0):
    v, m = _u64arr(v), _u64arr(m)
    b = np.ascontiguousarray(np.atleast_2d(np.asarray(b, dtype=np.uint64)))
    roots = np.ascontiguousarray(np.asarray(roots, dtype=np.int64))
    S, T = b.shape
    c = np.zeros((S, roots.size), dtype=np.uint64)
    _check(lib().zro_tvandermonde_solve_roots(T, S, offset, _p(v), _p(m), _p(b), T, roots.size, _p(roots, _i64p),
                                              p, _p(c), roots.size, nthreads), "tvandermonde_solve_roots")
    return c


def newton(x, f, p=P63):
    x, f = _u64arr(x), _u64arr(f)
    coef = np.zeros(x.size, dtype=np.uint64)
    _check(lib().zro_newton(x.size, _p(x), _p(f), p, _p(coef)), "newton")
    return coef


def newton_batched(x, vals, p=P63):
    """vals is npts x nterms; returns npts x nterms monomial coefficients."""
    x = _u64arr(x)
    vals = np.ascontiguousarray(np.asarray(vals, dtype=np.uint64))
    npts, nterms = vals.shape
    coef = np.zeros_like(vals)
    _check(lib().zro_newton_batched(nterms, npts, _p(x), _p(vals), nterms, p, _p(coef)), "newton_batched")
    return coef


# ---------------------------------------------------------------- black box

def eval_points(exps, coef, pts, p=P63):
    exps, coef = _u8arr(exps), _u64arr(coef)
    pts = np.ascontiguousarray(np.atleast_2d(np.asarray(pts, dtype=np.uint64)))
    Tf, nv = exps.shape
    out = np.zeros(pts.shape[0], dtype=np.uint64)
    lib().zro_eval_points(Tf, nv, _p(exps, _u8p), _p(coef), pts.shape[0], _p(pts), p, _p(out))
    return out


def zippel_probes(exps, coef, k, y, cs, z, T, offset=0, p=P63, nthreads=0):
    exps, coef = _u8arr(exps), _u64arr(coef)
    Tf, nv = exps.shape
    y = _u64arr(y if len(y) else [0])
    cs = _u64arr(cs)
    z = _u64arr(z if z is not None and len(z) else np.zeros(nv, dtype=np.uint64))
    S = cs.size
    b = np.zeros((S, max(T, 1)), dtype=np.uint64)
    _check(lib().zro_zippel_probes(Tf, nv, _p(exps, _u8p), _p(coef), k, _p(y), S, _p(cs), _p(z), T, offset, p,
                                   nthreads, _p(b), max(T, 1)), "zippel_probes")
    return b[:, :T]


def zippel_probes_sampled(exps, coef, k, y, cs, z, sidx, iidx, offset=0, p=P63, nthreads=0):
    exps, coef = _u8arr(exps), _u64arr(coef)
    Tf, nv = exps.shape
    y = _u64arr(y if len(y) else [0])
    cs = _u64arr(cs)
    z = _u64arr(z if z is not None and len(z) else np.zeros(nv, dtype=np.uint64))
    sidx = np.ascontiguousarray(np.asarray(sidx, dtype=np.int32))
    iidx = np.ascontiguousarray(np.asarray(iidx, dtype=np.int64))
    out = np.zeros(sidx.size, dtype=np.uint64)
    _check(lib().zro_zippel_probes_sampled(Tf, nv, _p(exps, _u8p), _p(coef), k, _p(y), cs.size, _p(cs), _p(z),
                                           offset, sidx.size, _p(sidx, _i32p), _p(iidx, _i64p), p, nthreads,
                                           _p(out)), "zippel_probes_sampled")
    return out


# ---------------------------------------------------------------- steps

def zippel_step(exps, k, y, cs, b, offset=0, p=P63, nthreads=0, want_c=False):
    """Returns (new_exps, new_coef[, c]) of the Zippel step for new variable k."""
    exps = _u8arr(exps)
    T, nv = exps.shape
    y = _u64arr(y if len(y) else [0])
    cs = _u64arr(cs)
    S = cs.size
    b = np.ascontiguousarray(np.asarray(b, dtype=np.uint64).reshape(S, T)) if T else np.zeros((S, 1), np.uint64)
    cap = max(T * S, 1)
    oe = np.zeros((cap, nv), dtype=np.uint8)
    oc = np.zeros(cap, dtype=np.uint64)
    n = np.zeros(1, dtype=np.int64)
    c = np.zeros((S, max(T, 1)), dtype=np.uint64) if want_c else None
    _check(lib().zro_zippel_step(T, nv, _p(exps, _u8p), k, _p(y), S, _p(cs), _p(b), max(T, 1), offset, p, nthreads,
                                 cap, _p(n, _i64p), _p(oe, _u8p), _p(oc), _p(c)), "zippel_step")
    n = int(n[0])
    if want_c:
        return oe[:n], oc[:n], c[:, :T]
    return oe[:n], oc[:n]


def thiele(x, f, maxdn, maxdd, p=P63):
    """Returns (num, den) coefficient arrays (trimmed) with den(x_0) = 1."""
    x, f = _u64arr(x), _u64arr(f)
    n = x.size
    num = np.zeros(n, dtype=np.uint64)
    den = np.zeros(n, dtype=np.uint64)
    dn = ctypes.c_int32()
    dd = ctypes.c_int32()
    _check(lib().zro_thiele(n, _p(x), _p(f), p, maxdn, maxdd, ctypes.byref(dn), ctypes.byref(dd), _p(num), _p(den)),
           "thiele")
    return num[: dn.value + 1], den[: dd.value + 1]


def balance_probes(cs, fvals, dprev, dN, dD, TN, TD, p=P63, nthreads=0):
    cs = _u64arr(cs)
    fvals = np.ascontiguousarray(np.asarray(fvals, dtype=np.uint64))
    Sf, Tmax = fvals.shape
    dprev = _u64arr(dprev)
    bN = np.zeros((dN + 1, max(TN, 1)), dtype=np.uint64)
    bD = np.zeros((dD + 1, max(TD, 1)), dtype=np.uint64)
    _check(lib().zro_balance_probes(Sf, _p(cs), _p(fvals), Tmax, Tmax, _p(dprev), dN, dD, TN, TD, p, nthreads,
                                    _p(bN), max(TN, 1), _p(bD), max(TD, 1)), "balance_probes")
    return bN[:, :TN], bD[:, :TD]


def reconstruct_poly(exps, coef, deg, seed, offset=0, p=P63, nthreads=0, cap=None):
    exps, coef = _u8arr(exps), _u64arr(coef)
    Tf, nv = exps.shape
    deg = np.ascontiguousarray(np.asarray(deg, dtype=np.int32))
    cap = cap or max(4 * Tf + 64, 64)
    oe = np.zeros((cap, nv), dtype=np.uint8)
    oc = np.zeros(cap, dtype=np.uint64)
    n = np.zeros(1, dtype=np.int64)
    work = np.zeros(1, dtype=np.int64)
    _check(lib().zro_reconstruct_poly(Tf, nv, _p(exps, _u8p), _p(coef), _p(deg, _i32p), seed, offset, p, nthreads,
                                      cap, _p(n, _i64p), _p(oe, _u8p), _p(oc), _p(work, _i64p)), "reconstruct_poly")
    n = int(n[0])
    return oe[:n], oc[:n]


def reconstruct_rational(Nexps, Ncoef, Dexps, Dcoef, degN, degD, seed, offset=0, p=P63, nthreads=0, cap=None):
    Nexps, Ncoef, Dexps, Dcoef = _u8arr(Nexps), _u64arr(Ncoef), _u8arr(Dexps), _u64arr(Dcoef)
    nv = Nexps.shape[1]
    degN = np.ascontiguousarray(np.asarray(degN, dtype=np.int32))
    degD = np.ascontiguousarray(np.asarray(degD, dtype=np.int32))
    capN = cap or max(4 * Nexps.shape[0] + 64, 64)
    capD = cap or max(4 * Dexps.shape[0] + 64, 64)
    oNe = np.zeros((capN, nv), dtype=np.uint8)
    oNc = np.zeros(capN, dtype=np.uint64)
    oDe = np.zeros((capD, nv), dtype=np.uint8)
    oDc = np.zeros(capD, dtype=np.uint64)
    nN = np.zeros(1, dtype=np.int64)
    nD = np.zeros(1, dtype=np.int64)
    _check(lib().zro_reconstruct_rational(Nexps.shape[0], _p(Nexps, _u8p), _p(Ncoef), Dexps.shape[0], _p(Dexps, _u8p),
                                          _p(Dcoef), nv, _p(degN, _i32p), _p(degD, _i32p), seed, offset, p, nthreads,
                                          capN, capD, _p(nN, _i64p), _p(oNe, _u8p), _p(oNc), _p(nD, _i64p),
                                          _p(oDe, _u8p), _p(oDc)), "reconstruct_rational")
    nN, nD = int(nN[0]), int(nD[0])
    return (oNe[:nN], oNc[:nN]), (oDe[:nD], oDc[:nD])
