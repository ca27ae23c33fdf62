"""Seeded synthetic workloads for the Zippel step.

This module holds random-number generation and sampling only -- none of the
method's arithmetic (no modular products, no evaluation, no solving).  Both
the CUDA path and the CPU oracle take their inputs from here.

Random numbers come from splitmix64 (Steele, Lea, Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) used as a counter-based
generator, vectorised with numpy:

    key(seed, stream) = mix(seed + (stream + 1) * G)
    draw(key, n)      = mix(key + (n + 1) * G),     G = 0x9E3779B97F4A7C15

A residue is ``draw >> 1`` rejected when it is 0 or >= p, so every generated
coefficient, anchor and sample lies in [1, p).

The paper measures on private reduction data (Sec. 3: skeletons of 125k to
4.8m monomials over the sixth variable).  The workloads below stand in for it
with the shapes its Sec. 1 method implies: a skeleton of T distinct monomials
in the already reconstructed variables, a new variable of degree d (S = d + 1
samples), and hidden coefficients uniform in [1, p).
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass, field

import numpy as np

P63 = 2**63 - 25
_G = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def splitmix_at(key: int, n: int) -> int:
    """n-th output (n >= 0) of the splitmix64 sequence started at ``key``."""
    with np.errstate(over="ignore"):
        z = np.array([key], dtype=np.uint64) + np.uint64(n + 1) * _G
    return int(_mix(z)[0])


class Stream:
    """A counter-based splitmix64 stream identified by (seed, stream)."""

    def __init__(self, seed: int, stream: int):
        self.key = np.uint64(splitmix_at(seed, stream))
        self.ctr = 0

    def raw(self, n: int) -> np.ndarray:
        idx = np.arange(self.ctr + 1, self.ctr + n + 1, dtype=np.uint64)
        self.ctr += n
        with np.errstate(over="ignore"):
            return _mix(self.key + idx * _G)

    def residues(self, n: int, p: int = P63) -> np.ndarray:
        """n values uniform in [1, p)."""
        out = np.empty(0, dtype=np.uint64)
        pp = np.uint64(p)
        while out.size < n:
            x = self.raw(n - out.size + 8) >> np.uint64(1)
            x = x[(x != 0) & (x < pp)]
            out = np.concatenate([out, x])
        return out[:n].copy()

    def distinct_residues(self, n: int, p: int = P63, avoid=()) -> np.ndarray:
        """n pairwise distinct values in [1, p), none in ``avoid``."""
        seen = set(int(a) for a in avoid)
        out = []
        while len(out) < n:
            for x in self.residues(n - len(out)):
                xi = int(x)
                if xi not in seen:
                    seen.add(xi)
                    out.append(xi)
        return np.array(out[:n], dtype=np.uint64)

    def below(self, n: int, bound: int) -> np.ndarray:
        """n integers uniform in [0, bound) (modulo bias below 2^-40)."""
        return (self.raw(n) % np.uint64(bound)).astype(np.int64)


# --------------------------------------------------------------------------
# monomial sampling
# --------------------------------------------------------------------------

def distinct_monomials_box(st: Stream, n: int, nv: int, maxexp: int) -> np.ndarray:
    """n distinct exponent vectors with entries uniform in [0, maxexp],
    kept in order of first draw.  Returns n x nv uint8."""
    base = maxexp + 1
    if base ** nv < n:
        raise ValueError("box too small")
    keys: list[int] = []
    seen: set[int] = set()
    rows = []
    while len(rows) < n:
        m = (n - len(rows)) * 2 + 64
        e = st.below(m * nv, base).reshape(m, nv)
        code = np.zeros(m, dtype=np.int64)
        for c in range(nv):
            code = code * base + e[:, c]
        for r in range(m):
            key = int(code[r])
            if key not in seen:
                seen.add(key)
                keys.append(key)
                rows.append(e[r])
                if len(rows) == n:
                    break
    return np.asarray(rows, dtype=np.uint8).reshape(n, nv)


def simplex_monomials(nv: int, deg: int) -> np.ndarray:
    """All exponent vectors with total degree <= deg, lexicographic order."""
    rows = [e for e in itertools.product(range(deg + 1), repeat=nv) if sum(e) <= deg]
    return np.asarray(rows, dtype=np.uint8).reshape(-1, nv)


def choose_distinct(st: Stream, population: int, n: int) -> np.ndarray:
    """n distinct indices of range(population), uniformly (partial Fisher-Yates)."""
    if n > population:
        raise ValueError("n > population")
    perm = np.arange(population, dtype=np.int64)
    draws = st.raw(n)
    for i in range(n):
        j = i + int(draws[i] % np.uint64(population - i))
        perm[i], perm[j] = perm[j], perm[i]
    return perm[:n].copy()


# --------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------

@dataclass
class StepWorkload:
    """One Zippel step for new variable k = nv - 1.

    The hidden function is f = sum_j x'^{e_j} g_j(x_k), x' = (x_0..x_{k-1}),
    g_j of degree S-1 with coefficients G[j, 0..S-1] in [1, p).  The skeleton
    is the support of f at fixed x_k: the T monomials e_j.  ``exps`` / ``coef``
    list the hidden terms ordered by j, then by the power of x_k; that is
    also the order in which the step emits its output.
    """
    name: str
    p: int
    nv: int
    k: int
    T: int
    S: int
    skel: np.ndarray          # T x nv uint8 (column k zero)
    G: np.ndarray             # T x S uint64, hidden coefficients
    y: np.ndarray             # k anchors
    cs: np.ndarray            # S distinct samples of x_k
    z: np.ndarray             # nv rest values (unused here: k is the last variable)
    exps: np.ndarray = field(default=None)   # (T*S) x nv
    coef: np.ndarray = field(default=None)   # T*S

    def __post_init__(self):
        if self.exps is None:
            T, S, nv, k = self.T, self.S, self.nv, self.k
            e = np.repeat(self.skel, S, axis=0)
            e[:, k] = np.tile(np.arange(S, dtype=np.uint8), T)
            self.exps = e
            self.coef = self.G.reshape(-1).copy()


def step_workload(seed: int, T: int, k: int, maxexp: int, S: int, p: int = P63, name: str = "") -> StepWorkload:
    nv = k + 1
    skel = np.zeros((T, nv), dtype=np.uint8)
    if T:
        skel[:, :k] = distinct_monomials_box(Stream(seed, 1), T, k, maxexp)
    G = Stream(seed, 2).residues(T * S, p).reshape(T, S)
    y = Stream(seed, 3).residues(k, p)
    cs = Stream(seed, 4).distinct_residues(S, p)
    z = Stream(seed, 5).residues(nv, p)
    return StepWorkload(name or f"step_T{T}_k{k}_S{S}", p, nv, k, T, S, skel, G, y, cs, z)


@dataclass
class PolyWorkload:
    name: str
    p: int
    nv: int
    exps: np.ndarray   # Tf x nv
    coef: np.ndarray   # Tf
    deg: np.ndarray    # per-variable degree bounds
    seed: int          # seed of the reconstruction's own draws


@dataclass
class RationalWorkload:
    name: str
    p: int
    nv: int
    Nexps: np.ndarray
    Ncoef: np.ndarray
    Dexps: np.ndarray
    Dcoef: np.ndarray
    degN: np.ndarray
    degD: np.ndarray
    seed: int


def poly_simplex_workload(seed: int, nv: int, total_deg: int, T: int, p: int = P63, name: str = "") -> PolyWorkload:
    mons = simplex_monomials(nv, total_deg)
    idx = np.sort(choose_distinct(Stream(seed, 1), mons.shape[0], T))
    exps = mons[idx]
    coef = Stream(seed, 2).residues(T, p)
    deg = np.full(nv, total_deg, dtype=np.int32)
    return PolyWorkload(name or f"poly_n{nv}_d{total_deg}_T{T}", p, nv, exps, coef, deg, seed + 7)


def rational_simplex_workload(seed: int, nv: int, total_deg: int, TN: int, TD: int, p: int = P63,
                              name: str = "") -> RationalWorkload:
    """Hidden N/D with TN and TD distinct terms from the total-degree simplex;
    the lexicographically smallest term of D has coefficient 1."""
    mons = simplex_monomials(nv, total_deg)
    iN = np.sort(choose_distinct(Stream(seed, 1), mons.shape[0], TN))
    iD = np.sort(choose_distinct(Stream(seed, 2), mons.shape[0], TD))
    Ncoef = Stream(seed, 3).residues(TN, p)
    Dcoef = Stream(seed, 4).residues(TD, p)
    Nexps, Dexps = _cancel_monomial_content(mons[iN], mons[iD])
    Dcoef[0] = 1          # rows are in lexicographic order: row 0 is the smallest
    deg = np.full(nv, total_deg, dtype=np.int32)
    return RationalWorkload(name or f"rat_n{nv}_d{total_deg}_N{TN}_D{TD}", p, nv, Nexps, Ncoef, Dexps, Dcoef,
                            deg, deg.copy(), seed + 7)


# The workloads the project is measured on (seed = 1000 + workload number).

def plain_poly_3var() -> PolyWorkload:
    """3 variables, total degree <= 10, 200 distinct terms from the simplex."""
    return poly_simplex_workload(1001, 3, 10, 200, name="plain_poly_n3_d10_T200")


def batched_step_1e4() -> StepWorkload:
    """T = 10^4 monomials in 5 variables (exponents <= 20), new variable of degree 20."""
    return step_workload(1002, 10_000, 5, 20, 21, name="step_T10000_S21")


def large_step_2p20() -> StepWorkload:
    """T = 2^20 monomials in 7 variables (exponents <= 12), new variable of degree 8."""
    return step_workload(1003, 1 << 20, 7, 12, 9, name="step_T1048576_S9")


def balanced_5var() -> RationalWorkload:
    """N: 5000 and D: 3000 terms in 5 variables, total degree <= 15."""
    return rational_simplex_workload(1004, 5, 15, 5000, 3000, name="balanced_n5_d15_N5000_D3000")


def serve_requests(n: int = 4096, seed: int = 1005, p: int = P63, tmax: int = 1 << 17):
    """Request mix for the serving loop: half polynomial, half rational,
    n_vars uniform in 2..8, T log-uniform in [16, tmax], exponents <= 20."""
    st = Stream(seed, 1)
    out = []
    for r in range(n):
        u = st.raw(3)
        rational = bool(u[0] & np.uint64(1))
        nv = 2 + int(u[1] % np.uint64(7))
        frac = float(u[2] >> np.uint64(11)) / float(1 << 53)
        T = int(math.exp(math.log(16) + frac * (math.log(tmax) - math.log(16))))
        T = max(1, min(T, (21 ** nv) // 2))
        out.append(dict(id=r, rational=rational, nv=nv, T=T, seed=seed * 100000 + r))
    return out


def _lex_sorted(e: np.ndarray) -> np.ndarray:
    if e.shape[0] == 0:
        return e
    order = np.lexsort(tuple(e[:, c] for c in range(e.shape[1] - 1, -1, -1)))
    return e[order]


def _cancel_monomial_content(Ne: np.ndarray, De: np.ndarray):
    """Divides N and D by their common monomial factor, so that the hidden N/D
    is in lowest terms (a random sparse pair shares no other factor with
    overwhelming probability); row order is unchanged."""
    m = np.minimum(Ne.min(axis=0), De.min(axis=0)).astype(np.uint8)
    return Ne - m, De - m


def serve_blackbox(req: dict, p: int = P63, maxexp: int = 20):
    """The hidden function of one serving request: exponents uniform in
    [0, maxexp] per variable (distinct, lexicographic rows), coefficients
    uniform mod p, degree bound maxexp in every variable.  A rational request
    splits T 60/40 between N and D, and D's lexicographically smallest term
    has coefficient 1."""
    nv, T, seed = req["nv"], req["T"], req["seed"]
    deg = np.full(nv, maxexp, dtype=np.int32)
    if not req["rational"]:
        exps = _lex_sorted(distinct_monomials_box(Stream(seed, 1), T, nv, maxexp))
        return PolyWorkload(f"serve{req['id']}_poly_n{nv}_T{T}", p, nv, exps, Stream(seed, 2).residues(T, p), deg,
                            seed + 7)
    TN = max(1, (T * 3 + 4) // 5)
    TD = max(1, T - TN)
    Ne = _lex_sorted(distinct_monomials_box(Stream(seed, 1), TN, nv, maxexp))
    De = _lex_sorted(distinct_monomials_box(Stream(seed, 2), TD, nv, maxexp))
    Ne, De = _cancel_monomial_content(Ne, De)
    Nc = Stream(seed, 3).residues(TN, p)
    Dc = Stream(seed, 4).residues(TD, p)
    Dc[0] = 1
    return RationalWorkload(f"serve{req['id']}_rat_n{nv}_N{TN}_D{TD}", p, nv, Ne, Nc, De, Dc, deg, deg.copy(), seed + 7)
