"""Symmetric band eigenproblems on the GPU (tdc_sbevd: divide and conquer with b rank-one
merges per node) against the oracle (oracle/banded.py): eigenvalues element by element,
eigenvectors by residual and orthogonality, isolated eigenvectors up to sign."""
import numpy as np
import pytest
import torch

from oracle import banded as bo
from paper_2008_01990_gb300 import inputs

from helpers import EPS

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def tdc():
    from paper_2008_01990_gb300 import build, tdc as t
    build.build()
    t.lib()
    return t


@pytest.mark.parametrize("name,n,b", [("uniform", 5, 1), ("uniform", 100, 3), ("uniform", 300, 1),
                                      ("uniform", 600, 4), ("uniform", 1100, 8), ("laplace", 700, 5),
                                      ("graded", 513, 2), ("uniform", 2000, 16), ("uniform", 40, 0),
                                      ("uniform", 1, 0), ("uniform", 257, 8), ("uniform", 1500, 64)])
def test_sbevd_vs_oracle(tdc, orc, name, n, b):
    AB = inputs.band_sym(name, n, b, seed=n + b)
    lam, Q = tdc.sbevd(torch.tensor(AB, device=DEV), check=True)
    lam, Q = lam.cpu().numpy(), Q.cpu().numpy()
    lo, Qo = bo.sbevd(AB)
    A = bo.dense_from_band(AB)
    nA = max(np.abs(lo).max(), np.finfo(float).tiny)
    assert np.all(np.diff(lam) >= 0)
    assert np.max(np.abs(lam - lo)) <= 50 * n * EPS * nA
    res = np.abs(A @ Q - Q * lam).sum(axis=0).max() / (n * nA * EPS)
    orth = np.abs(Q.T @ Q - np.eye(n)).sum(axis=0).max() / (n * EPS)
    assert res <= 50 and orth <= 50, (res, orth)
    gap = np.minimum(np.abs(np.diff(lo, prepend=-np.inf)), np.abs(np.diff(lo, append=np.inf)))
    for i in np.where(gap > 1e-3 * nA)[0][:32]:
        sg = np.sign(Q[:, i] @ Qo[:, i])
        assert np.max(np.abs(sg * Q[:, i] - Qo[:, i])) <= 1e-9


def test_sbevd_clustered_laplace_2500(tdc):
    """The 1-D operator coupled to 8 neighbours at n = 2500 (many close eigenvalues, so many
    type-2 deflations in chains): eigenvalues against LAPACK's banded solver, residual and
    orthogonality ratios <= 50."""
    from scipy.linalg import eig_banded
    n, b = 2500, 8
    AB = inputs.band_sym("laplace", n, b)
    lam, Q = tdc.sbevd(torch.tensor(AB, device=DEV), check=True)
    lam, Q = lam.cpu().numpy(), Q.cpu().numpy()
    ref = eig_banded(AB, lower=True, eigvals_only=True)
    A = bo.dense_from_band(AB)
    nA = np.abs(ref).max()
    assert np.max(np.abs(lam - ref)) <= 50 * n * EPS * nA
    res = np.abs(A @ Q - Q * lam).sum(axis=0).max() / (n * nA * EPS)
    orth = np.abs(Q.T @ Q - np.eye(n)).sum(axis=0).max() / (n * EPS)
    assert res <= 50 and orth <= 50, (res, orth)


@pytest.mark.parametrize("k", [700, -700])
def test_sbevd_extreme_scales_are_solved_exactly_scaled(tdc, k):
    """A band matrix scaled far outside [2^-400, 2^400] is solved as the band matrix with
    its largest entry in [1, 2): the same eigenvectors bit for bit, its eigenvalues times
    2^k exactly."""
    AB = inputs.band_sym("uniform", 1000, 8, seed=3)
    AB0 = np.ldexp(AB, -(np.frexp(np.abs(AB).max())[1] - 1))
    lam0, Q0 = tdc.sbevd(torch.tensor(AB0, device=DEV), check=True)
    lam1, Q1 = tdc.sbevd(torch.tensor(np.ldexp(AB0, k), device=DEV), check=True)
    assert torch.equal(Q0, Q1)
    assert np.array_equal(lam1.cpu().numpy(), np.ldexp(lam0.cpu().numpy(), k))


def test_sbevd_tridiagonal_case_matches_eig(tdc):
    """b = 1 is the tridiagonal problem: the band solver and tdc_eig agree."""
    n = 900
    d, e = inputs.uniform_tridiag(n, 5)
    AB = np.zeros((2, n))
    AB[0] = d
    AB[1, : n - 1] = e
    lam_b, _ = tdc.sbevd(torch.tensor(AB, device=DEV), check=True)
    lam_t, _ = tdc.eig(torch.tensor(d, device=DEV), torch.tensor(e, device=DEV), check=True)
    nT = float(lam_t.abs().max())
    assert float((lam_b - lam_t).abs().max()) <= 50 * n * EPS * nT
