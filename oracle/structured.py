"""Oracle for products with Toeplitz and Hankel operands given by their generators.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper names Toeplitz, Hankel, Vandermonde and DFT matrices as further structured
operands of its product (the matrices of O(n) parameters, Section 1; the remarks of
Section 3.1 and Section 5).  An n x n Toeplitz matrix is constant along its diagonals,
B(k, j) = t[k - j + n - 1] with t of length 2n - 1 (t[n - 1 + i] on the i-th
subdiagonal); a Hankel matrix is constant along its anti-diagonals, B(k, j) = t[k + j].
The oracle writes the matrix out from that definition and multiplies with the C
oracle's plain triple loop.
"""
from __future__ import annotations

import numpy as np

TOEPLITZ, HANKEL = 1, 2


def dense(t, n, kind):
    """The n x n matrix of generators t (length 2n - 1), entry by entry."""
    t = np.asarray(t, dtype=np.float64)
    B = np.empty((n, n))
    for k in range(n):
        for j in range(n):
            B[k, j] = t[k - j + n - 1] if kind == TOEPLITZ else t[k + j]
    return B


def product(A, t, kind):
    """C = A B with B the Toeplitz or Hankel matrix of t."""
    from . import gemm
    n = np.asarray(A).shape[1]
    return gemm(np.asarray(A, dtype=np.float64), dense(t, n, kind))
