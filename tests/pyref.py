"""Small brute-force references in pure Python integers, used to pin the oracle.

Nothing here shares code with the oracle or the CUDA library: these are the
textbook routines (Gaussian elimination, Lagrange interpolation, polynomial
products) on Python's exact integers, only fast enough for tiny inputs.
"""
from __future__ import annotations

P63 = 2**63 - 25


def inv(a, p=P63):
    a %= p
    if a == 0:
        raise ZeroDivisionError
    return pow(a, p - 2, p)


def poly_mul(a, b, p=P63):
    out = [0] * (len(a) + len(b) - 1)
    for i, x in enumerate(a):
        for j, y in enumerate(b):
            out[i + j] = (out[i + j] + x * y) % p
    return out


def poly_eval(a, x, p=P63):
    return sum(int(c) * pow(int(x), e, p) for e, c in enumerate(a)) % p


def poly_trim(a):
    a = [int(c) for c in a]
    while len(a) > 1 and a[-1] == 0:
        a.pop()
    return a


def solve_linear(A, b, p=P63):
    """Gauss-Jordan elimination mod p; A is n x n, b is n x r (lists)."""
    n = len(A)
    r = len(b[0])
    M = [[int(A[i][j]) % p for j in range(n)] + [int(b[i][c]) % p for c in range(r)] for i in range(n)]
    for col in range(n):
        piv = next((i for i in range(col, n) if M[i][col]), None)
        if piv is None:
            raise ZeroDivisionError("singular")
        M[col], M[piv] = M[piv], M[col]
        iv = inv(M[col][col], p)
        M[col] = [x * iv % p for x in M[col]]
        for i in range(n):
            if i != col and M[i][col]:
                f = M[i][col]
                M[i] = [(x - f * y) % p for x, y in zip(M[i], M[col])]
    return [[M[i][n + c] for c in range(r)] for i in range(n)]


def lagrange_coeffs(xs, fs, p=P63):
    """Monomial coefficients of the interpolant through (xs, fs), by Lagrange."""
    n = len(xs)
    out = [0] * n
    for i in range(n):
        basis = [1]
        den = 1
        for j in range(n):
            if j != i:
                basis = poly_mul(basis, [(-xs[j]) % p, 1], p)
                den = den * (xs[i] - xs[j]) % p
        s = int(fs[i]) * inv(den, p) % p
        for e in range(n):
            out[e] = (out[e] + s * basis[e]) % p
    return out


def monomial_value(e, pt, p=P63):
    v = 1
    for x, k in zip(pt, e):
        v = v * pow(int(x), int(k), p) % p
    return v


def eval_sparse(exps, coef, pt, p=P63):
    return sum(int(c) * monomial_value(e, pt, p) for e, c in zip(exps, coef)) % p
