"""Toeplitz and Hankel products on the GPU (tdc_toeplitz_gemm: B generated from its 2n - 1
generators inside the FP64 tiles or the split product's digit images) element by element
against the oracle's product of the written-out matrix (oracle/structured.py)."""
import numpy as np
import pytest
import torch

from oracle import structured as so
from paper_2008_01990_gb300 import inputs

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def tdc():
    from paper_2008_01990_gb300 import build, tdc as t
    build.build()
    t.lib()
    return t


def gens(n, seed, decay=False):
    g = inputs.SplitMix64(seed)
    t = g.uniform(2 * n - 1, -1.0, 1.0)
    if decay:  # generators decaying away from the main diagonal over 30 binades
        t = t * 2.0 ** (-30.0 * np.abs(np.arange(2 * n - 1) - (n - 1)) / max(n, 1))
    return t


@pytest.mark.parametrize("mode", ["dense", "split"])
@pytest.mark.parametrize("kind", [1, 2])
@pytest.mark.parametrize("m,n,decay", [(300, 1024, False), (777, 2048, False), (1, 65, False), (129, 1, False),
                                       (500, 1500, True)])
def test_toeplitz_product_vs_oracle(tdc, orc, mode, kind, m, n, decay):
    t = gens(n, 31 * n + m, decay)
    g = inputs.SplitMix64(n + 7 * m)
    A = g.uniform(m * n, -1.0, 1.0).reshape(m, n)
    B = so.dense(t, n, kind)
    Co = so.product(A, t, kind)
    At = torch.tensor(np.ascontiguousarray(A.T), device=DEV).t()
    md = tdc.MERGE_DENSE if mode == "dense" else tdc.MERGE_SPLIT
    C = tdc.toeplitz_gemm(At, torch.tensor(t, device=DEV), kind, md, check=True).cpu().numpy()
    # error scale of entry (i, j): ||A(i,:)|| ||B(:,j)|| (Cauchy-Schwarz bound of |C_ij|)
    scale = np.linalg.norm(A, axis=1)[:, None] * np.linalg.norm(B, axis=0)[None, :]
    assert np.max(np.abs(C - Co) / np.maximum(scale, np.finfo(float).tiny)) <= 1e-14


def test_toeplitz_identity_and_shift(tdc):
    """Special cases: t = e_{n-1} is the identity (C = A), t = e_n the down-shift
    (C(:, j) = A(:, j+1)); as Hankel, t = e_{n-1} is the exchange matrix (columns reversed).
    Exact in FP64; the split product holds A as 56-bit fixed point of scale 2^eA (eA from
    the largest row norm), so there it is exact to 2^(eA - 56) per entry."""
    n, m = 300, 200
    A = np.random.default_rng(5).uniform(-1, 1, (m, n))
    At = torch.tensor(np.ascontiguousarray(A.T), device=DEV).t()
    eA = int(np.floor(np.log2(np.linalg.norm(A, axis=1).max()))) + 1
    for md in (tdc.MERGE_DENSE, tdc.MERGE_SPLIT):
        tol = 0.0 if md == tdc.MERGE_DENSE else 2.0 ** (eA - 56)
        e = np.zeros(2 * n - 1)
        e[n - 1] = 1.0
        C = tdc.toeplitz_gemm(At, torch.tensor(e, device=DEV), tdc.TOEPLITZ, md, check=True).cpu().numpy()
        assert np.max(np.abs(C - A)) <= tol
        C = tdc.toeplitz_gemm(At, torch.tensor(e, device=DEV), tdc.HANKEL, md, check=True).cpu().numpy()
        assert np.max(np.abs(C - A[:, ::-1])) <= tol
        s = np.zeros(2 * n - 1)
        s[n] = 1.0  # B(k, j) = 1 for k = j + 1
        C = tdc.toeplitz_gemm(At, torch.tensor(s, device=DEV), tdc.TOEPLITZ, md, check=True).cpu().numpy()
        assert np.max(np.abs(C[:, : n - 1] - A[:, 1:])) <= tol and np.all(C[:, n - 1] == 0.0)
