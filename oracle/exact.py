"""Exact rational R-distance for tiny graphs -- TEST INFRASTRUCTURE ONLY.

Used to pin the FP64 oracle: with a rational gain gamma, Y = (I - gamma A)^-1 (Sec. 2,
Y-defined) is a matrix of rationals, and the rounded R-distance of Sec. 4.1
(rounded-distance-function) is decided exactly through its equivalent form (Y-limits):

    ceil(log_gamma Y_ij) = m   iff   gamma^m <= Y_ij < gamma^(m-1),

i.e. m is the smallest integer with gamma^m <= Y_ij (0 < gamma < 1).  No floating point is
involved, so this decode needs no rounding snap.
"""
from __future__ import annotations

from fractions import Fraction

UNREACHABLE = 2**31 - 1


def inverse(A, gamma: Fraction, W=None):
    """Exact (I - X)^-1 by Gauss-Jordan elimination over the rationals.

    X = gamma * A (Sec. 2) or, with integer weights W, X_ij = gamma^W_ij on edges (Sec. 3.2).
    """
    n = len(A)
    g = Fraction(gamma)
    M = []
    for i in range(n):
        row = []
        for j in range(n):
            x = Fraction(0)
            if A[i][j]:
                x = g ** int(W[i][j]) if W is not None else g
            row.append((Fraction(1) if i == j else Fraction(0)) - x)
        row += [Fraction(1) if i == j else Fraction(0) for j in range(n)]
        M.append(row)
    for k in range(n):
        p = next(r for r in range(k, n) if M[r][k] != 0)
        M[k], M[p] = M[p], M[k]
        piv = M[k][k]
        M[k] = [v / piv for v in M[k]]
        for r in range(n):
            if r != k and M[r][k] != 0:
                f = M[r][k]
                M[r] = [a - f * b for a, b in zip(M[r], M[k])]
    return [row[n:] for row in M]


def rounded_log(y: Fraction, gamma: Fraction) -> int:
    """ceil(log_gamma y) for y > 0: the smallest integer m with gamma^m <= y."""
    g = Fraction(gamma)
    m = 0
    if y >= 1:
        while y >= g ** (m - 1):
            m -= 1
        return m
    while y < g ** m:
        m += 1
    return m


def decode(Y, gamma: Fraction):
    """Exact D with D_ii = 0 and the unreachable sentinel for Y_ij <= 0."""
    n = len(Y)
    D = [[0] * n for _ in range(n)]
    for i in range(n):
        for j in range(n):
            if i == j:
                continue
            y = Y[i][j]
            D[i][j] = UNREACHABLE if y <= 0 else rounded_log(y, gamma)
    return D


def walk_counts(A, kmax: int):
    """Integer walk counts N^(k) = A^k for k = 0..kmax (Sec. 3.1, walk-count identity)."""
    n = len(A)
    I = [[1 if i == j else 0 for j in range(n)] for i in range(n)]
    out = [I]
    P = I
    for _ in range(kmax):
        P = [[sum(P[i][t] * (1 if A[t][j] else 0) for t in range(n)) for j in range(n)]
             for i in range(n)]
        out.append(P)
    return out
