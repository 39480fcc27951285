"""Oracle for products with Toeplitz, Hankel, Vandermonde and DFT operands given by their
generators.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper names Toeplitz, Hankel, Vandermonde and DFT matrices as further structured
operands of its product (the matrices of O(n) parameters, Section 1; the remarks of
Section 3.1 and Section 5).  An n x n Toeplitz matrix is constant along its diagonals,
B(k, j) = t[k - j + n - 1] with t of length 2n - 1 (t[n - 1 + i] on the i-th
subdiagonal); a Hankel matrix is constant along its anti-diagonals, B(k, j) = t[k + j].
A Vandermonde matrix of nodes x has B(k, j) = x_k^j; the DFT matrix of order n has
F(k, j) = exp(-2 pi i k j / n), whose real and imaginary parts are cos(2 pi k j / n) and
-sin(2 pi k j / n).  The oracle writes the matrix out from that definition and multiplies
with the C oracle's plain triple loop (the DFT product as its two real parts).
"""
from __future__ import annotations

import numpy as np

TOEPLITZ, HANKEL, VANDERMONDE = 1, 2, 3


def dense(t, n, kind):
    """The n x n matrix of generators t (length 2n - 1; the n nodes for Vandermonde), entry
    by entry."""
    t = np.asarray(t, dtype=np.float64)
    B = np.empty((n, n))
    for k in range(n):
        for j in range(n):
            if kind == TOEPLITZ:
                B[k, j] = t[k - j + n - 1]
            elif kind == HANKEL:
                B[k, j] = t[k + j]
            else:
                B[k, j] = t[k] ** j
    return B


def dft_parts(n):
    """Real and imaginary parts of the DFT matrix F(k, j) = exp(-2 pi i k j / n)."""
    k = np.arange(n)
    # omega^(kj) with omega = exp(-2 pi i / n) depends on kj mod n only; reducing it in
    # integer arithmetic keeps the angle below 2 pi (no rounding of large arguments)
    ang = 2.0 * np.pi * (np.outer(k, k) % n) / n
    return np.cos(ang), -np.sin(ang)


def dft_product(A):
    """(Re, Im) of C = A F, F the DFT matrix of order n = A's column count."""
    from . import gemm
    A = np.asarray(A, dtype=np.float64)
    Fr, Fi = dft_parts(A.shape[1])
    return gemm(A, Fr), gemm(A, Fi)


def product(A, t, kind):
    """C = A B with B the Toeplitz or Hankel matrix of t."""
    from . import gemm
    n = np.asarray(A).shape[1]
    return gemm(np.asarray(A, dtype=np.float64), dense(t, n, kind))
