"""Pins of the adjoint oracle (oracle/adjoint.py): the Hellmann-Feynman closed
form for eigenvalue cotangents, central finite differences of losses through
the oracle eigensolver, and the reading F o skew (not F o sym)."""
import numpy as np
import pytest

from oracle.adjoint import adjoint
from paper_2008_01990_gb300 import inputs


def separated(n, seed, min_gap=1e-3):
    g = inputs.SplitMix64(seed)
    while True:
        d = g.uniform(n, -1, 1)
        e = g.uniform(n - 1, -1, 1)
        lam = np.linalg.eigvalsh(np.diag(d) + np.diag(e, 1) + np.diag(e, -1))
        if np.min(np.diff(lam)) > min_gap:
            return d, e


def aligned_eig(orc, d, e, Qref):
    lam, Q = orc.eig(d, e, leaf=4)
    sgn = np.sign(np.sum(Q * Qref, axis=0))
    return lam, Q * sgn


def test_hellmann_feynman(orc):
    d, e = separated(12, 1)
    lam, Q = orc.eig(d, e, leaf=4)
    w = inputs.SplitMix64(2).normal(12)
    db, eb = adjoint(lam, Q, lam_bar=w)
    assert np.allclose(db, (Q ** 2) @ w, atol=1e-13)
    assert np.allclose(eb, 2 * (Q[:-1] * Q[1:]) @ w, atol=1e-13)


@pytest.mark.parametrize("n,seed", [(6, 3), (10, 4), (16, 5)])
def test_full_adjoint_vs_central_differences(orc, n, seed):
    d, e = separated(n, seed)
    g = inputs.SplitMix64(100 + seed)
    w = g.normal(n)
    G = g.normal(n * n).reshape(n, n)
    lam, Q = orc.eig(d, e, leaf=4)

    def loss(dd, ee):
        l2, Q2 = aligned_eig(orc, dd, ee, Q)
        return float(np.dot(w, l2) + np.sum(G * Q2))

    db, eb = adjoint(lam, Q, lam_bar=w, Q_bar=G)
    h = 1e-6
    fd_d = np.array([(loss(d + h * np.eye(n)[i], e) - loss(d - h * np.eye(n)[i], e)) / (2 * h) for i in range(n)])
    fd_e = np.array([(loss(d, e + h * np.eye(n - 1)[i]) - loss(d, e - h * np.eye(n - 1)[i])) / (2 * h)
                     for i in range(n - 1)])
    scale = max(1.0, np.abs(fd_d).max(), np.abs(fd_e).max())
    assert np.max(np.abs(db - fd_d)) <= 1e-6 * scale
    assert np.max(np.abs(eb - fd_e)) <= 1e-6 * scale


def test_sym_reading_would_be_wrong(orc):
    # with F o sym(W) the eigenvector part would vanish on the tridiagonal entries
    n = 8
    d, e = separated(n, 7)
    lam, Q = orc.eig(d, e, leaf=4)
    G = inputs.SplitMix64(8).normal(n * n).reshape(n, n)
    W = Q.T @ G
    F = np.array([[0.0 if i == j else 1.0 / (lam[j] - lam[i]) for j in range(n)] for i in range(n)])
    Tsym = Q @ (F * 0.5 * (W + W.T)) @ Q.T
    assert np.max(np.abs(np.diag(Tsym))) < 1e-12
    db, _ = adjoint(lam, Q, Q_bar=G)
    assert np.max(np.abs(db)) > 1e-3
