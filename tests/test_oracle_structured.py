"""Pins of the structured-operand oracle (oracle/structured.py) against the library's
constructors (scipy.linalg.toeplitz and hankel take the first column and row, numpy's
vander the nodes), against a library FFT for the DFT product, and against a numpy
product; planted mistakes in the indexing fail them."""
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


def test_vandermonde_matches_library():
    x = np.random.default_rng(2).uniform(-1.2, 1.2, 9)
    assert np.allclose(so.dense(x, 9, so.VANDERMONDE), np.vander(x, 9, increasing=True), rtol=1e-15, atol=0)


@pytest.mark.parametrize("n", [48, 1000])
def test_dft_matches_library_fft(orc, n):
    A = np.random.default_rng(4).uniform(-1, 1, (7, n))
    re, im = so.dft_product(A)
    F = np.fft.fft(A, axis=1)  # sum_k A(i, k) exp(-2 pi i k j / n)
    scale = np.linalg.norm(A, axis=1)[:, None] * np.sqrt(n)
    assert np.max(np.abs(re - F.real) / scale) <= 4e-16 * np.log2(n)
    assert np.max(np.abs(im - F.imag) / scale) <= 4e-16 * np.log2(n)


def test_product(orc):
    n, m = 40, 23
    t = gens(n, 7)
    A = np.random.default_rng(8).uniform(-1, 1, (m, n))
    for kind in (so.TOEPLITZ, so.HANKEL):
        C = so.product(A, t, kind)
        assert np.allclose(C, A @ so.dense(t, n, kind), atol=1e-13, rtol=0)


MUTANTS = [("toeplitz sign", "t[k - j + n - 1]", "t[j - k + n - 1]"),
           ("hankel offset", "B[k, j] = t[k + j]", "B[k, j] = t[k + j - 1]"),
           ("vandermonde power", "t[k] ** j", "t[j] ** k"),
           ("dft sign", "return np.cos(ang), -np.sin(ang)", "return np.cos(ang), np.sin(ang)")]


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
    x = t[:n]
    A = np.random.default_rng(4).uniform(-1, 1, (3, n))
    Fr, Fi = mod.dft_parts(n)
    F = np.fft.fft(A, axis=1)
    ok = (np.array_equal(mod.dense(t, n, 1), scipy_linalg.toeplitz(t[n - 1:], t[n - 1::-1])) and
          np.array_equal(mod.dense(t, n, 2), scipy_linalg.hankel(t[:n], t[n - 1:])) and
          np.allclose(mod.dense(x, n, 3), np.vander(x, n, increasing=True), rtol=1e-15, atol=0) and
          np.allclose(A @ Fr, F.real, atol=1e-13) and np.allclose(A @ Fi, F.imag, atol=1e-13))
    assert not ok, name
