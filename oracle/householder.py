"""Oracle for the dense symmetric -> tridiagonal reduction and its back-transform.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper's Example 3 runs the divide and conquer on the tridiagonal matrix that a
Householder reduction of a dense symmetric matrix produces (T = Q^T A Q); the
reduction itself is the textbook one (Golub & Van Loan, Matrix Computations,
Algorithm 8.3.1), written out here in plain numpy FP64, column by column, with the
reflector convention of LAPACK's xLARFG:

  for k = 0 .. n-3, x = A(k+1:n, k), alpha = x_0, sigma = ||x(1:)||:
      beta = -sign(alpha) sqrt(alpha^2 + sigma^2)     (beta = alpha, tau = 0 if sigma = 0)
      tau = (beta - alpha) / beta,  v = [1, x(1:) / (alpha - beta)]
      H_k = I - tau v v^T maps x to beta e_1
      p = tau A22 v,  w = p - (tau/2) (p^T v) v,  A22 <- A22 - v w^T - w v^T
      e_k = beta
  d_k = A(k, k) after the updates; e_{n-2} = A(n-1, n-2).

Q = H_0 H_1 ... H_{n-3} (each H_k acting on rows / columns k+1..n-1), so that
Q^T A Q = T and the eigenvectors of A are Q times those of T.
"""
from __future__ import annotations

import numpy as np


def tridiagonalize(A):
    """Householder reduction of the symmetric A (n x n): returns (d, e, V, tau) with
    T = tridiag(d, e) = Q^T A Q; column k of V holds the reflector v_k (v_k[k+1] = 1,
    zeros above), tau[k] its scalar."""
    A = np.array(A, dtype=np.float64, copy=True)
    n = A.shape[0]
    V = np.zeros((n, max(n - 2, 0)))
    tau = np.zeros(max(n - 2, 0))
    e = np.zeros(max(n - 1, 0))
    for k in range(n - 2):
        x = A[k + 1:, k].copy()
        alpha = x[0]
        sigma = np.linalg.norm(x[1:])
        if sigma == 0.0:
            t, beta = 0.0, alpha
            v = np.zeros_like(x)
            v[0] = 1.0
        else:
            beta = -np.copysign(np.hypot(alpha, sigma), alpha)
            t = (beta - alpha) / beta
            v = x / (alpha - beta)
            v[0] = 1.0
        V[k + 1:, k] = v
        tau[k] = t
        e[k] = beta
        A22 = A[k + 1:, k + 1:]
        p = t * (A22 @ v)
        w = p - 0.5 * t * float(p @ v) * v
        A22 -= np.outer(v, w) + np.outer(w, v)
        A[k + 1:, k] = 0.0
        A[k, k + 1:] = 0.0
        A[k + 1, k] = A[k, k + 1] = beta
    if n >= 2:
        e[n - 2] = A[n - 1, n - 2]
    d = np.diag(A).copy()
    return d, e, V, tau


def apply_q(V, tau, C):
    """Q C with Q = H_0 H_1 ... H_{n-3}: the reflectors applied to C's rows, last first."""
    C = np.array(C, dtype=np.float64, copy=True)
    for k in range(V.shape[1] - 1, -1, -1):
        v = V[k + 1:, k]
        C[k + 1:, :] -= tau[k] * np.outer(v, v @ C[k + 1:, :])
    return C


def syevd(A, leaf=32):
    """Eigenvalues (ascending) and eigenvectors of the dense symmetric A: reduction,
    the divide-and-conquer oracle on T, back-transform."""
    from . import eig
    d, e, V, tau = tridiagonalize(A)
    lam, Qt = eig(d, e, leaf=leaf, max_iter=2000)
    return lam, apply_q(V, tau, Qt), (d, e)
