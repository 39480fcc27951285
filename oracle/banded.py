"""Oracle for the symmetric band eigenproblem.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper's Section 5 points to the divide and conquer for band matrices.  A symmetric
matrix of bandwidth b (A(i, j) = 0 for |i - j| > b) is stored in the lower band layout
of LAPACK: AB(i - j, j) = A(i, j) for j <= i <= min(n - 1, j + b), AB of (b + 1) x n.
The eigen-decomposition it defines is computed by the plain route: the dense matrix
written out from the band, the Householder reduction, the tridiagonal oracle and the
back-transform (householder.syevd).
"""
from __future__ import annotations

import numpy as np


def dense_from_band(AB):
    """The dense symmetric matrix of lower band storage AB ((b + 1) x n)."""
    AB = np.asarray(AB, dtype=np.float64)
    b1, n = AB.shape
    A = np.zeros((n, n))
    for j in range(n):
        for r in range(b1):
            i = j + r
            if i < n:
                A[i, j] = AB[r, j]
                A[j, i] = AB[r, j]
    return A


def band_from_dense(A, b):
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    AB = np.zeros((b + 1, n))
    for j in range(n):
        for r in range(b + 1):
            if j + r < n:
                AB[r, j] = A[j + r, j]
    return AB


def sbevd(AB):
    """(lam ascending, Q) of the band matrix AB."""
    from .householder import syevd
    lam, Q, _ = syevd(dense_from_band(AB))
    return lam, Q
