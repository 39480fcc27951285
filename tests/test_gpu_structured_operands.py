"""Products with structured operands on the GPU (tdc_structured_gemm: Toeplitz, Hankel and
Vandermonde B generated from its generators inside the FP64 tiles or the split product's
digit images; tdc_dft_gemm: the DFT matrix's two real parts) element by element against
the oracle's product of the written-out matrix (oracle/structured.py)."""
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
    C = tdc.structured_gemm(At, torch.tensor(t, device=DEV), kind, md, check=True).cpu().numpy()
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
        C = tdc.structured_gemm(At, torch.tensor(e, device=DEV), tdc.TOEPLITZ, md, check=True).cpu().numpy()
        assert np.max(np.abs(C - A)) <= tol
        C = tdc.structured_gemm(At, torch.tensor(e, device=DEV), tdc.HANKEL, md, check=True).cpu().numpy()
        assert np.max(np.abs(C - A[:, ::-1])) <= tol
        s = np.zeros(2 * n - 1)
        s[n] = 1.0  # B(k, j) = 1 for k = j + 1
        C = tdc.structured_gemm(At, torch.tensor(s, device=DEV), tdc.TOEPLITZ, md, check=True).cpu().numpy()
        assert np.max(np.abs(C[:, : n - 1] - A[:, 1:])) <= tol and np.all(C[:, n - 1] == 0.0)


@pytest.mark.parametrize("mode", ["dense", "split"])
@pytest.mark.parametrize("m,n,lo,hi", [(300, 512, -1.0, 1.0), (64, 1000, 0.5, 1.0), (17, 33, -1.3, 1.3)])
def test_vandermonde_product_vs_oracle(tdc, orc, mode, m, n, lo, hi):
    """Nodes in [lo, hi] (|x| up to 1.3: entries up to 1.3^32 at n = 33)."""
    x = inputs.SplitMix64(n + m).uniform(n, lo, hi)
    A = inputs.SplitMix64(3 * n).uniform(m * n, -1.0, 1.0).reshape(m, n)
    B = so.dense(x, n, so.VANDERMONDE)
    Co = so.product(A, x, so.VANDERMONDE)
    At = torch.tensor(np.ascontiguousarray(A.T), device=DEV).t()
    md = tdc.MERGE_DENSE if mode == "dense" else tdc.MERGE_SPLIT
    C = tdc.structured_gemm(At, torch.tensor(x, device=DEV), tdc.VANDERMONDE, md, check=True).cpu().numpy()
    scale = np.linalg.norm(A, axis=1)[:, None] * np.linalg.norm(B, axis=0)[None, :]
    # the powers by repeated squaring carry up to 2 log2(n) roundings against the oracle's
    assert np.max(np.abs(C - Co) / np.maximum(scale, np.finfo(float).tiny)) <= 1e-14 * max(1.0, np.log2(n))


@pytest.mark.parametrize("mode", ["dense", "split"])
@pytest.mark.parametrize("m,n", [(200, 256), (77, 1000), (5, 1)])
def test_dft_product_vs_oracle_and_fft(tdc, orc, mode, m, n):
    A = inputs.SplitMix64(5 * n + m).uniform(m * n, -1.0, 1.0).reshape(m, n)
    At = torch.tensor(np.ascontiguousarray(A.T), device=DEV).t()
    md = tdc.MERGE_DENSE if mode == "dense" else tdc.MERGE_SPLIT
    Cr, Ci = tdc.dft_gemm(At, md, check=True)
    Cr, Ci = Cr.cpu().numpy(), Ci.cpu().numpy()
    Ro, Io = so.dft_product(A)
    scale = np.linalg.norm(A, axis=1)[:, None] * np.sqrt(n)  # ||A_i|| ||F_j||, |F_kj| = 1
    assert np.max(np.abs(Cr - Ro) / scale) <= 1e-14 and np.max(np.abs(Ci - Io) / scale) <= 1e-14
    F = np.fft.fft(A, axis=1)
    assert np.max(np.abs(Cr - F.real) / scale) <= 1e-14 and np.max(np.abs(Ci - F.imag) / scale) <= 1e-14
