"""Plain CPU oracle for the lift of modular results to rational numbers --
TEST INFRASTRUCTURE ONLY (see the package header: only tests, the smoke check
and the bench's CPU legs import it).

The reconstruction runs modulo large primes and recovers the rational
numbers as a final step (Sec. 1).  For the images r_i of one value modulo
distinct primes p_i:

* the Chinese remainder theorem gives the unique x in [0, P), P = prod p_i,
  with x = r_i (mod p_i) for every i -- here written out as
  x = sum_i r_i M_i (M_i^-1 mod p_i) mod P, M_i = P / p_i;
* rational reconstruction (Wang's method) finds n / d with n = d x (mod P),
  |n| <= N, 0 < d <= N, N = floor(sqrt((P - 1) / 2)) -- unique when it
  exists, since 2 N^2 < P.  The extended Euclidean algorithm on (P, x) is
  run until the first remainder r <= N; with its cofactor t of x the value
  is sign(t) r / |t|, accepted when 0 < |t| <= N and gcd(r, |t|) = 1.

Python integers throughout; a loop per value, for test sizes.
"""
from __future__ import annotations

import math


def crt(residues, primes):
    """x in [0, prod primes) with x = residues[i] mod primes[i]."""
    P = math.prod(primes)
    x = 0
    for r, p in zip(residues, primes):
        M = P // p
        x += (int(r) % p) * M * pow(M, -1, p)
    return x % P


def bound(P):
    """N = floor(sqrt((P - 1) / 2))."""
    return math.isqrt((P - 1) // 2)


def rational_reconstruct(x, P):
    """(n, d) with n / d = x mod P, |n|, d <= bound(P), or None."""
    N = bound(P)
    r0, r1 = P, x % P
    t0, t1 = 0, 1
    while r1 > N:
        q = r0 // r1
        r0, r1 = r1, r0 - q * r1
        t0, t1 = t1, t0 - q * t1
    if t1 == 0 or abs(t1) > N or math.gcd(r1, abs(t1)) != 1:
        return None
    return (r1 if t1 > 0 else -r1), abs(t1)


def rational_lift(residue_rows, primes):
    """For residue_rows[i][j] = value j mod primes[i]: a list of (n, d) or None."""
    P = math.prod(primes)
    n = len(residue_rows[0]) if residue_rows else 0
    return [rational_reconstruct(crt([row[j] for row in residue_rows], primes), P) for j in range(n)]
