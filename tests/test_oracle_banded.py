"""Pins of the band eigenproblem oracle (oracle/banded.py): band storage against the
library's banded eigensolver (scipy.linalg.eig_banded, lower form), the decomposition's
residual and orthogonality, the closed form of the one-neighbour Laplacian
(tridiag(-1, 2, -1): 2 - 2 cos(k pi / (n + 1)), sine vectors), and a planted storage
mistake."""
import numpy as np
import pytest

from oracle import banded as bo

EPS = np.finfo(float).eps


def band(n, b, seed):
    g = np.random.default_rng(seed)
    AB = g.uniform(-1, 1, (b + 1, n))
    for r in range(1, b + 1):
        AB[r, n - r:] = 0.0  # entries past the matrix
    return AB


@pytest.mark.parametrize("n,b", [(1, 0), (5, 1), (40, 3), (120, 8)])
def test_against_library_banded_solver(orc, n, b):
    scipy_linalg = pytest.importorskip("scipy.linalg")
    AB = band(n, b, n + b)
    lam, Q = bo.sbevd(AB)
    ref = scipy_linalg.eig_banded(AB, lower=True, eigvals_only=True)
    A = bo.dense_from_band(AB)
    nA = max(np.abs(ref).max(), 1e-300)
    assert np.max(np.abs(lam - ref)) <= 50 * max(n, 1) * EPS * nA
    assert np.abs(A @ Q - Q * lam).max() <= 50 * max(n, 1) * EPS * nA
    assert np.abs(Q.T @ Q - np.eye(n)).max() <= 50 * max(n, 1) * EPS
    assert np.array_equal(bo.band_from_dense(A, b), AB)


def test_laplacian_closed_form(orc):
    """The `laplace` band family at b = 1 is tridiag(-1, 2, -1): eigenvalues
    2 - 2 cos(k pi / (n + 1)) and eigenvectors sin(i k pi / (n + 1)), up to sign."""
    from paper_2008_01990_gb300 import inputs
    n = 200
    lam, Q = bo.sbevd(inputs.band_sym("laplace", n, 1))
    k = np.arange(1, n + 1)
    assert np.max(np.abs(lam - np.sort(2.0 - 2.0 * np.cos(k * np.pi / (n + 1))))) <= 50 * n * EPS * 4
    i = np.arange(1, n + 1)
    for j in (0, 1, n // 2, n - 1):  # the j-th smallest: k = j + 1
        v = np.sin(i * (j + 1) * np.pi / (n + 1))
        v /= np.linalg.norm(v)
        assert abs(abs(v @ Q[:, j]) - 1.0) <= 1e-10


def test_planted_storage_mistake(tmp_path):
    scipy_linalg = pytest.importorskip("scipy.linalg")
    import importlib.util
    import inspect
    src = inspect.getsource(bo)
    old = "A[i, j] = AB[r, j]\n                A[j, i] = AB[r, j]"
    assert old in src
    p = tmp_path / "bo_mut.py"
    p.write_text(src.replace(old, "A[i, j] = AB[r, i]\n                A[j, i] = AB[r, i]"))
    spec = importlib.util.spec_from_file_location("bo_mut", p)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    AB = band(30, 3, 1)
    ev = np.linalg.eigvalsh(mod.dense_from_band(AB))
    ref = scipy_linalg.eig_banded(AB, lower=True, eigvals_only=True)
    assert np.max(np.abs(ev - ref)) > 1e-10
