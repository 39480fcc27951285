"""Dense symmetric eigenproblems on the GPU (Section 4, Example 3: reduction to tridiagonal
form, the divide and conquer on T, back-transform of its eigenvectors) against the
Householder oracle (oracle/householder.py).

What is unique is compared element by element: T's entries (d, e), and, where the
reflectors are determined by the data rather than by rounding noise, the reflectors and
their scalars.  Q is checked for what makes it valid: orthogonal, and Q^T A Q = T to the
backward-error bound.  The eigensolver is checked by residual and orthogonality ratios,
its eigenvalues against the oracle's.

Tolerances.  The reduction's backward error is of order n eps ||A|| (each reflector
applied with O(n) rounding errors, the split updates exact up to one rounding per
entry); T's entries move by that amount times their condition, which is modest for
these families away from the noise-level off-diagonals.  The element-wise bound used for
d and e is 1e-11 ||A||_2 for n <= 1100, about 40 n eps for n = 1100.  Reflector k
depends on x / ||x|| with ||x|| = |e_k|, so its scalar and vector get the bound
50 n eps ||A||_2 / |e_k|."""
import numpy as np
import pytest
import torch

from oracle import householder as hh
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


def reflectors(R, n):
    """V (n x n-2) of the reduced matrix's lower triangle: unit at k+1, R(k+2:n, k) below."""
    V = np.zeros((n, max(n - 2, 0)))
    for k in range(n - 2):
        V[k + 1, k] = 1.0
        V[k + 2:, k] = R[k + 2:, k]
    return V


def tri(d, e):
    return np.diag(d) + np.diag(e, 1) + np.diag(e, -1)


def gpu_q(tdc, R, tau, n):
    X = torch.eye(n, dtype=torch.float64, device=DEV).t().contiguous().t()
    tdc.ormtr(R, tau, X, check=True)
    return X.cpu().numpy()


@pytest.mark.parametrize("name,n", [("uniform", 3), ("uniform", 5), ("uniform", 130), ("uniform", 300),
                                    ("uniform", 700), ("uniform", 1100), ("zerocol", 257), ("tridiag", 200),
                                    ("lowrank", 600), ("cluster", 520)])
def test_sytrd_vs_oracle(tdc, name, n):
    A = inputs.dense_sym(name, n, seed=n)
    d, e, tau, R = tdc.sytrd(torch.tensor(A, device=DEV), check=True)
    d, e, tau, R = d.cpu().numpy(), e.cpu().numpy(), tau.cpu().numpy(), R.cpu().numpy()
    do, eo, Vo, to = hh.tridiagonalize(A)
    nA = max(np.linalg.norm(A, 2), np.finfo(float).tiny)
    tol = 1e-11 * nA
    assert np.max(np.abs(d - do)) <= tol
    assert np.max(np.abs(e - eo)) <= tol
    assert tau.shape == (max(n - 1, 0),) and (n < 2 or tau[-1] == 0.0)
    if name in ("uniform", "zerocol", "tridiag") and n > 2:
        # reflectors fixed by the data, element-wise.  tau_k = 1 + |alpha| / ||x|| and
        # v_k = x / (alpha - beta) with ||x|| = |e_k|, so a backward perturbation of size
        # n eps ||A|| moves them by about that over |e_k|
        bound = 50 * n * EPS * nA / np.maximum(np.abs(eo[: n - 2]), np.finfo(float).tiny)
        assert np.all(np.abs(tau[: n - 2] - to) <= np.minimum(bound, 2.0))
        dV = np.abs(reflectors(R, n) - Vo).max(axis=0)
        assert np.all(dV <= np.minimum(bound, 2.0))
    if name == "zerocol":
        assert tau[0] == 0.0 and e[0] == 0.0
    if name == "tridiag":
        assert np.all(tau == 0.0)
    # validity of Q and T whatever the noise-level reflectors: Q^T A Q = T, Q orthogonal
    Q = gpu_q(tdc, torch.tensor(R, device=DEV).t().contiguous().t(), torch.tensor(tau, device=DEV), n)
    assert np.abs(Q.T @ Q - np.eye(n)).sum(axis=0).max() / (n * EPS) <= 50
    assert np.abs(Q.T @ A @ Q - tri(d, e)).sum(axis=0).max() / (n * EPS * nA) <= 50


@pytest.mark.parametrize("n,ncols", [(3, 4), (131, 1), (300, 77), (900, 300), (1030, 1030)])
def test_ormtr_vs_oracle(tdc, n, ncols):
    """X <- Q X against the oracle's reflector-by-reflector product with the same reflectors."""
    A = inputs.dense_sym("uniform", n, seed=7 * n)
    _, _, tau, R = tdc.sytrd(torch.tensor(A, device=DEV), check=True)
    g = inputs.SplitMix64(n + ncols)
    X = g.uniform(n * ncols, -1.0, 1.0).reshape(n, ncols)
    Xt = torch.tensor(np.ascontiguousarray(X.T), device=DEV).t()
    tdc.ormtr(R, tau, Xt, check=True)
    got = Xt.cpu().numpy()
    Rn, tn = R.cpu().numpy(), tau.cpu().numpy()
    want = hh.apply_q(reflectors(Rn, n), tn[: max(n - 2, 0)], X)
    col = np.linalg.norm(X, axis=0)
    err = np.abs(got - want).max(axis=0) / np.maximum(col, np.finfo(float).tiny)
    assert err.max() <= 64 * n * EPS


def residual_ratios(A, lam, Z):
    n = A.shape[0]
    nA = max(np.linalg.norm(A, 2), np.finfo(float).tiny)
    res = np.abs(A @ Z - Z * lam).sum(axis=0).max() / (n * nA * EPS)
    orth = np.abs(Z.T @ Z - np.eye(n)).sum(axis=0).max() / (n * EPS)
    # the paper's residual of Example 3: max column norm of A - Z Lam Z^T over ||A||_2
    paper = np.linalg.norm(A - (Z * lam) @ Z.T, axis=0).max() / nA
    return res, orth, paper


@pytest.mark.parametrize("name,n", [("uniform", 1), ("uniform", 2), ("uniform", 3), ("uniform", 129),
                                    ("lowrank", 600), ("cluster", 700), ("zerocol", 513)])
def test_syevd_small_and_degenerate(tdc, orc, name, n):
    A = inputs.dense_sym(name, n, seed=3 * n + 1)
    lam, Z = tdc.syevd(torch.tensor(A, device=DEV), check=True)
    lam, Z = lam.cpu().numpy(), Z.cpu().numpy()
    assert np.all(np.diff(lam) >= 0)
    do, eo, _, _ = hh.tridiagonalize(A)
    lo, _ = orc.eig(do, eo, max_iter=2000) if n > 0 else (np.zeros(0), None)
    nA = max(np.linalg.norm(A, 2), np.finfo(float).tiny)
    assert np.max(np.abs(lam - lo)) <= 50 * max(n, 1) * EPS * nA
    res, orth, paper = residual_ratios(A, lam, Z)
    assert res <= 50 and orth <= 50, (res, orth)
    assert paper <= 50 * max(n, 1) * EPS


def test_syevd_2048_vs_oracle(tdc, orc):
    """The full pipeline at n = 2048 on the uniform family: eigenvalues against the
    oracle's (Householder reduction, then the oracle's divide and conquer), eigenvectors
    by the residual ratio <= 50 and the orthogonality ratio <= 50."""
    n = 2048
    A = inputs.dense_sym("uniform", n, seed=2048)
    lam, Z = tdc.syevd(torch.tensor(A, device=DEV), check=True)
    lam, Z = lam.cpu().numpy(), Z.cpu().numpy()
    do, eo, _, _ = hh.tridiagonalize(A)
    lo, _ = orc.eig(do, eo, max_iter=2000)
    nA = np.linalg.norm(A, 2)
    assert np.max(np.abs(lam - lo)) <= 50 * n * EPS * nA
    res, orth, paper = residual_ratios(A, lam, Z)
    assert res <= 50 and orth <= 50, (res, orth)
    assert paper <= 50 * n * EPS


def test_syevd_split_merge_mode(tdc):
    """The composed solver with the tridiagonal stage forced onto the plain split merge."""
    n = 1500
    A = inputs.dense_sym("uniform", n, seed=15)
    o = tdc.default_opts(merge_mode=tdc.MERGE_SPLIT, split_min_K=64)
    lam, Z = tdc.syevd(torch.tensor(A, device=DEV), opts=o, check=True)
    res, orth, _ = residual_ratios(A, lam.cpu().numpy(), Z.cpu().numpy())
    assert res <= 50 and orth <= 50, (res, orth)


def test_sytrd_subnormal_rows_stay_finite(tdc):
    """Rows and columns scaled down through the subnormal range in quarter binades: the
    split update's per-column scales come from row maxima down to 2^-1074, and each must
    stay a normal power of two (2^+-1024 built from exponent bits is infinite, and one
    infinite scale turns a zero entry into NaN).  T stays finite and Q^T A Q = T."""
    n = 1024
    A = inputs.dense_sym("uniform", n, seed=1024)
    s = np.ones(n)
    s[600:900] = 2.0 ** (-1000.0 - 0.25 * np.arange(300))
    B = np.tril((A * s[:, None]) * s[None, :])
    B = B + np.tril(B, -1).T
    d, e, tau, R = tdc.sytrd(torch.tensor(B, device=DEV), check=True)
    assert bool(torch.isfinite(d).all() and torch.isfinite(e).all() and torch.isfinite(tau).all())
    d, e = d.cpu().numpy(), e.cpu().numpy()
    Q = gpu_q(tdc, R.t().contiguous().t(), tau, n)
    nB = np.linalg.norm(B, 2)
    assert np.abs(Q.T @ Q - np.eye(n)).sum(axis=0).max() / (n * EPS) <= 50
    assert np.abs(Q.T @ B @ Q - tri(d, e)).sum(axis=0).max() / (n * EPS * nB) <= 50


def test_band_matrix_reduction_and_solve(tdc):
    """A band matrix of order 8192, half-bandwidth 8: its reflectors fill in behind a
    front whose entries decay through the whole exponent range, down to subnormals, so
    the split updates see every scale exponent.  T is finite with the eigenvalues of A
    (LAPACK's banded solver as reference); the composed solver's eigenpairs pass the
    residual and orthogonality ratios on sampled columns.  Only T's spectrum is compared,
    not its entries: the reduction of this matrix is backward stable but T itself is
    sensitive (two stable reductions, LAPACK's and the oracle's, part at column 132)."""
    from scipy.linalg import eig_banded, eigvalsh_tridiagonal
    from oracle import banded as bo
    n, b = 8192, 8
    AB = inputs.band_sym("uniform", n, b, seed=1)
    ref = eig_banded(AB, lower=True, eigvals_only=True)
    A = torch.tensor(bo.dense_from_band(AB), device=DEV)
    nA = float(np.max(np.abs(ref)))
    d, e, tau, R = tdc.sytrd(A, check=True)
    assert bool(torch.isfinite(d).all() and torch.isfinite(e).all() and torch.isfinite(tau).all())
    lt = eigvalsh_tridiagonal(d.cpu().numpy(), e.cpu().numpy())
    assert np.max(np.abs(lt - ref)) <= 50 * n * EPS * nA
    lam, Z = tdc.syevd(A, check=True)
    assert np.max(np.abs(lam.cpu().numpy() - ref)) <= 50 * n * EPS * nA
    idx = torch.tensor(np.unique((inputs.SplitMix64(8).uniform01(256) * n).astype(np.int64)), device=DEV)
    Zs = Z[:, idx]
    res = torch.abs(A @ Zs - Zs * lam[idx]).sum(dim=0).max().item() / (n * nA * EPS)
    orth = torch.abs(Z.t() @ Zs - torch.eye(n, dtype=torch.float64, device=DEV)[:, idx]).sum(dim=0).max().item()
    assert res <= 50 and orth / (n * EPS) <= 50, (res, orth / (n * EPS))


@pytest.mark.parametrize("k", [600, -600, 1000, -800])
def test_syevd_extreme_scales_are_solved_exactly_scaled(tdc, k):
    """A dense matrix scaled far outside [2^-400, 2^400] (where the reduction's norms would
    overflow or underflow) is solved as the matrix with its largest entry in [1, 2): the
    same eigenvectors bit for bit, its eigenvalues times 2^k exactly."""
    n = 700
    A = inputs.dense_sym("uniform", n, seed=70)
    A0 = np.ldexp(A, -(np.frexp(np.abs(A).max())[1] - 1))
    lam0, Z0 = tdc.syevd(torch.tensor(A0, device=DEV), check=True)
    lam1, Z1 = tdc.syevd(torch.tensor(np.ldexp(A0, k), device=DEV), check=True)
    assert torch.equal(Z0, Z1)
    assert np.array_equal(lam1.cpu().numpy(), np.ldexp(lam0.cpu().numpy(), k))


def test_sytrd_barrier_timeout_reports_status(tdc):
    """A panel whose grid barriers may poll only once gives up with TDC_ETIMEOUT instead of
    waiting; the context stays usable and the next call succeeds."""
    n = 400
    A = torch.tensor(inputs.dense_sym("uniform", n, seed=4), device=DEV)
    o = tdc.default_opts(spin_budget=1)
    tdc.sytrd(A, opts=o)
    st = tdc.sync_status()
    assert st in (0, tdc.TDC_ETIMEOUT)
    d, e, tau, R = tdc.sytrd(A, check=True)
    do, eo, _, _ = hh.tridiagonalize(A.cpu().numpy())
    assert np.max(np.abs(d.cpu().numpy() - do)) <= 1e-11 * np.linalg.norm(A.cpu().numpy(), 2)
