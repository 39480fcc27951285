"""Shared checks for the GPU parity tests (verification only, never product code)."""
import numpy as np

EPS = np.finfo(np.float64).eps


def dense(d, e):
    return np.diag(d) + np.diag(e, 1) + np.diag(e, -1)


def norm2_from_lam(lam):
    return float(max(abs(lam[0]), abs(lam[-1]))) if len(lam) else 0.0


def ratios(d, e, lam, Q):
    """(residual ratio ||TQ - Q Lam||_1/(n ||T|| eps), orthogonality ||Q^T Q - I||_1/(n eps))
    with ||T|| = ||T||_2 = max |lam|."""
    n = len(d)
    T = dense(d, e)
    nT = max(norm2_from_lam(lam), np.finfo(float).tiny)
    res = np.abs(T @ Q - Q * lam).sum(axis=0).max() / (n * nT * EPS)
    orth = np.abs(Q.T @ Q - np.eye(n)).sum(axis=0).max() / (n * EPS)
    return res, orth


def clusters(lam, tol):
    """Index ranges [a, b) of eigenvalues closer than tol to a neighbour."""
    out = []
    a = 0
    for i in range(1, len(lam) + 1):
        if i == len(lam) or lam[i] - lam[i - 1] > tol:
            out.append((a, i))
            a = i
    return out


def compare_vectors(Q, Qo, lam, tol_cluster, max_angle):
    """Eigenvectors up to sign for isolated eigenvalues; for clusters compare the
    spanned subspaces through the singular values of Q^T Qo on the cluster."""
    worst = 0.0
    for a, b in clusters(lam, tol_cluster):
        if b - a == 1:
            c = abs(float(np.dot(Q[:, a], Qo[:, a])))
            worst = max(worst, 1.0 - c)
        else:
            s = np.linalg.svd(Q[:, a:b].T @ Qo[:, a:b], compute_uv=False)
            worst = max(worst, 1.0 - float(s.min()))
    assert worst <= max_angle, "eigenvector mismatch %.3e > %.3e" % (worst, max_angle)
    return worst
