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


def check_toeplitz_sampled(lam, Q, n, ns=256, vec_tol=1e-6):
    """tridiag(1,2,1) of order n on the GPU: every eigenvalue against the closed form
    2 + 2 cos(k pi / (n+1)); residual, orthogonality and the sine eigenvectors on
    ns sampled columns.  Returns (residual ratio, orthogonality ratio)."""
    import torch
    dev = Q.device
    k = torch.arange(1, n + 1, dtype=torch.float64, device=dev)
    ref = torch.sort(2.0 + 2.0 * torch.cos(k * np.pi / (n + 1))).values
    assert torch.max(torch.abs(lam - ref)).item() <= 1e-12 * 4
    g = np.random.default_rng(0)
    cols = torch.tensor(np.sort(g.choice(n, ns, replace=False)), device=dev)
    Qs = Q[:, cols]
    Tq = 2.0 * Qs
    Tq[1:] += Qs[:-1]
    Tq[:-1] += Qs[1:]
    res = torch.abs(Tq - Qs * lam[cols]).sum(dim=0).max().item() / (n * 4.0 * EPS)
    G = Qs.t() @ Q
    G[torch.arange(ns, device=dev), cols] -= 1.0
    orth = torch.abs(G).sum(dim=1).max().item() / (n * EPS)
    assert res <= 50 and orth <= 50, (res, orth)
    # eigenvalue lam_k (ascending) belongs to index m = n+1-k of 2+2cos(m pi/(n+1))
    m = (n - cols).to(torch.float64)
    j = torch.arange(1, n + 1, dtype=torch.float64, device=dev)[:, None]
    V = np.sqrt(2.0 / (n + 1)) * torch.sin(j * m[None, :] * np.pi / (n + 1))
    dots = torch.abs(torch.sum(V * Qs, dim=0))
    assert torch.max(torch.abs(dots - 1.0)).item() <= vec_tol
    return res, orth
