"""Exact rational arithmetic used to pin the oracle on tiny integer inputs (no floating point anywhere)."""
from fractions import Fraction


def solve_spd_exact(A, b):
    """Solve A x = b exactly by Gauss-Jordan elimination over the rationals (A nonsingular)."""
    n = len(A)
    M = [[Fraction(v) for v in row] + [Fraction(bv)] for row, bv in zip(A, b)]
    for col in range(n):
        piv = next(r for r in range(col, n) if M[r][col] != 0)
        M[col], M[piv] = M[piv], M[col]
        pv = M[col][col]
        M[col] = [v / pv for v in M[col]]
        for r in range(n):
            if r != col and M[r][col] != 0:
                f = M[r][col]
                M[r] = [a - f * c for a, c in zip(M[r], M[col])]
    return [M[r][n] for r in range(n)]


def normal_equations_exact(rows, rhs):
    """X^T X and X^T b as exact rationals, from explicit integer rows."""
    p = len(rows[0])
    G = [[sum(Fraction(r[j]) * r[k] for r in rows) for k in range(p)] for j in range(p)]
    h = [sum(Fraction(r[j]) * bb for r, bb in zip(rows, rhs)) for j in range(p)]
    return G, h
