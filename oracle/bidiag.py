"""Oracle for the bidiagonal SVD through the divide-and-conquer eigensolver.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The SVD of an upper bidiagonal B (diagonal d[n], superdiagonal e[n-1]) follows from the
symmetric tridiagonal Golub-Kahan matrix of order 2n with zero diagonal and off-diagonal
(d_1, e_1, d_2, e_2, ..., e_{n-1}, d_n): its eigenvalues are +-sigma_i, and the
eigenvector of +sigma_i is (v_1, u_1, v_2, u_2, ..., v_n, u_n) / sqrt(2) with
B v = sigma u and B^T u = sigma v (Golub & Kahan 1965; Golub & Van Loan Section 8.6).
The paper's introduction points to the divide and conquer for the bidiagonal SVD; here
the tridiagonal oracle solves the Golub-Kahan matrix and the singular triplets are read
off its positive half.  Singular values come out descending.
"""
from __future__ import annotations

import numpy as np


def golub_kahan(d, e):
    """Diagonal (zeros) and off-diagonal (d_1, e_1, ..., e_{n-1}, d_n) of the order-2n matrix."""
    d = np.asarray(d, dtype=np.float64)
    e = np.asarray(e, dtype=np.float64)
    n = d.size
    off = np.zeros(max(2 * n - 1, 0))
    off[0::2] = d
    off[1::2] = e[: max(n - 1, 0)]
    return np.zeros(2 * n), off


def bdsdc(d, e, leaf=32):
    """(sigma, U, VT) with B = U diag(sigma) VT, sigma descending."""
    from . import eig
    n = len(d)
    if n == 0:
        return np.zeros(0), np.zeros((0, 0)), np.zeros((0, 0))
    td, te = golub_kahan(d, e)
    lam, Z = eig(td, te, leaf=leaf, max_iter=2000)
    pos = np.arange(2 * n - 1, n - 1, -1)  # +sigma_1 >= ... >= +sigma_n
    sigma = lam[pos]
    Zp = Z[:, pos] * np.sqrt(2.0)
    V = Zp[0::2, :]
    U = Zp[1::2, :]
    return sigma, U, V.T


def bidiag(d, e):
    n = len(d)
    return np.diag(np.asarray(d, float)) + np.diag(np.asarray(e, float)[: max(n - 1, 0)], 1)
