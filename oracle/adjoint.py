"""Oracle for the adjoint (reverse-mode derivative) of the tridiagonal eigensolve.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

For T = Q diag(lam) Q^T with distinct eigenvalues and a loss L(lam, Q) with
cotangents lam_bar = dL/dlam and Q_bar = dL/dQ, the cotangent of the symmetric
matrix T is
    T_bar = Q M Q^T,   M = diag(lam_bar) + F o skew(Q^T Q_bar),
    F_ij = 1/(lam_j - lam_i) (i != j), F_ii = 0,  skew(W) = (W - W^T)/2,
and for the tridiagonal parameters d (diagonal) and e (off-diagonal)
    d_bar_i = T_bar_ii,   e_bar_i = 2 T_bar_{i,i+1}.
F is antisymmetric, so F o skew(W) is the symmetric part of F o W; the form
F o sym(W) would be antisymmetric and contribute nothing to a symmetric T.
Plain numpy FP64, no blocking.
"""
from __future__ import annotations

import numpy as np


def adjoint(lam, Q, lam_bar=None, Q_bar=None):
    lam = np.asarray(lam, dtype=np.float64)
    Q = np.asarray(Q, dtype=np.float64)
    n = lam.size
    M = np.zeros((n, n))
    if Q_bar is not None:
        W = Q.T @ np.asarray(Q_bar, dtype=np.float64)
        S = 0.5 * (W - W.T)
        F = np.zeros((n, n))
        for i in range(n):
            for j in range(n):
                if i != j:
                    F[i, j] = 1.0 / (lam[j] - lam[i])
        M = F * S
    if lam_bar is not None:
        M = M + np.diag(np.asarray(lam_bar, dtype=np.float64))
    Tb = Q @ M @ Q.T
    d_bar = np.diag(Tb).copy()
    e_bar = 2.0 * np.array([Tb[i, i + 1] for i in range(n - 1)])
    return d_bar, e_bar
