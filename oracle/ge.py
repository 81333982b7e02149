"""Dense solution of the PageRank fixed point -- TEST INFRASTRUCTURE ONLY.

Section 2.1 of the paper defines the limit X of the iteration by
``X = dPX + (1-d)V``, i.e. ``(I - dP) X = (1-d) V``, with P_ij the probability
of the move j -> i (column j of P carries 1/outdeg(j) on each child of j).
Section 3.3 leaves dangling columns at zero (P is not completed), which is the
matrix used here.

``I - dP`` is strictly diagonally dominant by columns: column j has diagonal
1 - d P_jj and off-diagonal mass d (sum_i P_ij - P_jj) <= d (1 - P_jj) < 1 - d P_jj.
Gaussian elimination without pivoting is therefore well defined and stable on
it (dominance is preserved by every elimination step), so the routines below
are the textbook algorithm with no pivot search.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np


def transition_matrix(n, row_ptr, col_idx, dtype=np.float64):
    """Dense P with P[j, i] = (number of listed edges i -> j) / outdeg(i); dangling columns zero."""
    P = np.zeros((n, n), dtype=dtype)
    for i in range(n):
        beg, end = int(row_ptr[i]), int(row_ptr[i + 1])
        if end == beg:
            continue
        for e in range(beg, end):
            P[int(col_idx[e]), i] += 1.0 / (end - beg)
    return P


def solve_no_pivot(M, b):
    """Gaussian elimination without pivoting, then back substitution (FP64)."""
    A = np.array(M, dtype=np.float64, copy=True)
    x = np.array(b, dtype=np.float64, copy=True)
    n = A.shape[0]
    for k in range(n - 1):
        f = A[k + 1:, k] / A[k, k]
        A[k + 1:, k:] -= np.outer(f, A[k, k:])
        x[k + 1:] -= f * x[k]
    for k in range(n - 1, -1, -1):
        x[k] = (x[k] - A[k, k + 1:] @ x[k + 1:]) / A[k, k]
    return x


def pagerank_dense(n, row_ptr, col_idx, d, V):
    """X solving (I - dP) X = (1-d) V by elimination (Section 2.1, uncompleted P of Section 3.3)."""
    P = transition_matrix(n, row_ptr, col_idx)
    M = np.eye(n) - d * P
    return solve_no_pivot(M, (1.0 - d) * np.asarray(V, dtype=np.float64))


def solve_exact(n, row_ptr, col_idx, d: Fraction, V):
    """The same elimination in exact rational arithmetic; returns a list of Fractions."""
    d = Fraction(d)
    V = [Fraction(v) for v in V]
    M = [[Fraction(int(r == c)) for c in range(n)] for r in range(n)]
    for i in range(n):
        beg, end = int(row_ptr[i]), int(row_ptr[i + 1])
        for e in range(beg, end):
            M[int(col_idx[e])][i] -= d * Fraction(1, end - beg)
    x = [(1 - d) * v for v in V]
    for k in range(n - 1):
        for r in range(k + 1, n):
            if M[r][k] == 0:
                continue
            f = M[r][k] / M[k][k]
            for c in range(k, n):
                M[r][c] -= f * M[k][c]
            x[r] -= f * x[k]
    for k in range(n - 1, -1, -1):
        s = x[k]
        for c in range(k + 1, n):
            s -= M[k][c] * x[c]
        x[k] = s / M[k][k]
    return x
