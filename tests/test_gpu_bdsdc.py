"""Bidiagonal SVD on the GPU (tdc_bdsdc: the divide and conquer on the Golub-Kahan
tridiagonal) against the oracle (oracle/bidiag.py): singular values element by element,
the factors by B V = U Sigma, B^T U = V Sigma and orthogonality, singular vectors of
well-separated singular values up to sign."""
import numpy as np
import pytest
import torch

from oracle import bidiag as bd
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


def run(tdc, d, e, opts=None):
    s, U, VT = tdc.bdsdc(torch.tensor(d, device=DEV), torch.tensor(e, device=DEV), opts=opts, check=True)
    return s.cpu().numpy(), U.cpu().numpy(), VT.cpu().numpy()


def check_factors(B, s, U, VT):
    n = B.shape[0]
    nB = max(s[0], np.finfo(float).tiny)
    V = VT.T
    res_r = np.abs(B @ V - U * s).sum(axis=0).max() / (n * nB * EPS)
    res_l = np.abs(B.T @ U - V * s).sum(axis=0).max() / (n * nB * EPS)
    ou = np.abs(U.T @ U - np.eye(n)).sum(axis=0).max() / (n * EPS)
    ov = np.abs(V.T @ V - np.eye(n)).sum(axis=0).max() / (n * EPS)
    return res_r, res_l, ou, ov


@pytest.mark.parametrize("name,n", [("uniform", 1), ("uniform", 2), ("uniform", 3), ("uniform", 100),
                                    ("uniform", 777), ("uniform", 2048), ("graded", 600)])
def test_bdsdc_vs_oracle(tdc, orc, name, n):
    d, e = inputs.bidiag_family(name, n, seed=n)
    s, U, VT = run(tdc, d, e)
    so, Uo, VTo = bd.bdsdc(d, e)
    B = bd.bidiag(d, e)
    nB = so[0]
    assert np.all(np.diff(s) <= 0)
    assert np.max(np.abs(s - so)) <= 50 * n * EPS * nB
    res_r, res_l, ou, ov = check_factors(B, s, U, VT)
    assert res_r <= 50 and res_l <= 50, (res_r, res_l)
    # the Golub-Kahan pair +-sigma_i is 2 sigma_i apart: the vectors hold to about
    # eps ||B|| / sigma_i, so orthogonality is bounded by ||B|| / sigma_min (1 for
    # well-conditioned B)
    kappa = max(1.0, nB / max(so[-1], np.finfo(float).tiny))
    assert ou <= 50 * kappa and ov <= 50 * kappa, (ou, ov, kappa)
    if name == "uniform":
        assert ou <= 50 and ov <= 50
    # vectors of well-separated singular values, up to sign
    gap = np.minimum(np.abs(np.diff(so, prepend=np.inf)), np.abs(np.diff(so, append=-np.inf)))
    sep = np.where(gap > 1e-3 * nB)[0]
    for i in sep[:64]:
        tol = 1e-9 * max(1.0, 1e-3 * nB / so[i])
        sg = np.sign(U[:, i] @ Uo[:, i])
        assert np.max(np.abs(sg * U[:, i] - Uo[:, i])) <= tol
        assert np.max(np.abs(sg * VT[i] - VTo[i])) <= tol


def test_bdsdc_closed_form(tdc):
    n = 1000
    d, e = inputs.bidiag_family("ones", n)
    s, U, VT = run(tdc, d, e)
    k = np.arange(1, n + 1)
    assert np.max(np.abs(s - 2 * np.cos(k * np.pi / (2 * n + 1)))) <= 50 * n * EPS * 2


@pytest.mark.parametrize("mode", ["split", "dense"])
def test_bdsdc_merge_modes(tdc, mode):
    n = 1500
    d, e = inputs.bidiag_family("uniform", n, seed=11)
    md = {"split": tdc.MERGE_SPLIT, "dense": tdc.MERGE_DENSE}[mode]
    s, U, VT = run(tdc, d, e, tdc.default_opts(merge_mode=md, split_min_K=64))
    for r in check_factors(bd.bidiag(d, e), s, U, VT):
        assert r <= 50
