"""Pins of the Toeplitz / Hankel oracle (oracle/structured.py) against the library's
constructors (scipy.linalg.toeplitz and hankel take the first column and row) and
against a numpy product; planted mistakes in the indexing fail them."""
import numpy as np
import pytest

from oracle import structured as so


def gens(n, seed):
    return np.random.default_rng(seed).uniform(-1, 1, 2 * n - 1)


@pytest.mark.parametrize("n", [1, 2, 5, 33])
def test_matrices_match_library(n):
    scipy_linalg = pytest.importorskip("scipy.linalg")
    t = gens(n, n)
    T = so.dense(t, n, so.TOEPLITZ)
    # first column t[n-1:], first row t[n-1::-1]
    assert np.array_equal(T, scipy_linalg.toeplitz(t[n - 1:], t[n - 1::-1]))
    H = so.dense(t, n, so.HANKEL)
    assert np.array_equal(H, scipy_linalg.hankel(t[:n], t[n - 1:]))


def test_product(orc):
    n, m = 40, 23
    t = gens(n, 7)
    A = np.random.default_rng(8).uniform(-1, 1, (m, n))
    for kind in (so.TOEPLITZ, so.HANKEL):
        C = so.product(A, t, kind)
        assert np.allclose(C, A @ so.dense(t, n, kind), atol=1e-13, rtol=0)


MUTANTS = [("toeplitz sign", "t[k - j + n - 1]", "t[j - k + n - 1]"),
           ("hankel offset", "else t[k + j]", "else t[k + j - 1]")]


@pytest.mark.parametrize("name,old,new", MUTANTS)
def test_planted_mistakes_fail_a_pin(name, old, new, tmp_path):
    scipy_linalg = pytest.importorskip("scipy.linalg")
    import importlib.util
    import inspect
    src = inspect.getsource(so)
    assert old in src
    p = tmp_path / "so_mutant.py"
    p.write_text(src.replace(old, new))
    spec = importlib.util.spec_from_file_location("so_mutant", p)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    n = 6
    t = gens(n, 3)
    ok = (np.array_equal(mod.dense(t, n, 1), scipy_linalg.toeplitz(t[n - 1:], t[n - 1::-1])) and
          np.array_equal(mod.dense(t, n, 2), scipy_linalg.hankel(t[:n], t[n - 1:])))
    assert not ok, name
