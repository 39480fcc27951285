"""Pins of the bidiagonal SVD oracle (oracle/bidiag.py): the closed form of the all-ones
bidiagonal (sigma_k = 2 cos(k pi / (2n + 1))), a library SVD, B V = U Sigma and orthogonal
factors, a diagonal B (singular values |d| sorted), and planted mistakes."""
import numpy as np
import pytest

from oracle import bidiag as bd

EPS = np.finfo(float).eps


def test_all_ones_closed_form(orc):
    n = 200
    s, U, VT = bd.bdsdc(np.ones(n), np.ones(n - 1))
    k = np.arange(1, n + 1)
    assert np.max(np.abs(s - 2 * np.cos(k * np.pi / (2 * n + 1)))) <= 20 * n * EPS


@pytest.mark.parametrize("n,seed", [(1, 1), (2, 2), (7, 3), (150, 4)])
def test_library_svd_and_factors(orc, n, seed):
    g = np.random.default_rng(seed)
    d = g.uniform(0.5, 1.5, n) * g.choice([-1, 1], n)
    e = g.uniform(-1, 1, max(n - 1, 0))
    B = bd.bidiag(d, e)
    s, U, VT = bd.bdsdc(d, e)
    nB = np.linalg.norm(B, 2)
    assert np.max(np.abs(s - np.linalg.svd(B, compute_uv=False))) <= 50 * n * EPS * nB
    assert np.all(np.diff(s) <= 0) and np.all(s >= 0)
    assert np.max(np.abs(U @ np.diag(s) @ VT - B)) <= 50 * n * EPS * nB
    assert np.max(np.abs(U.T @ U - np.eye(n))) <= 50 * n * EPS
    assert np.max(np.abs(VT @ VT.T - np.eye(n))) <= 50 * n * EPS


def test_diagonal_matrix(orc):
    d = np.array([3.0, -1.0, 0.5, 2.0])
    s, U, VT = bd.bdsdc(d, np.zeros(3))
    assert np.allclose(s, [3.0, 2.0, 1.0, 0.5], atol=1e-15)
    assert np.allclose(np.abs(U), np.abs(VT.T), atol=1e-15)


MUTANTS = [
    ("d and e swapped in the Golub-Kahan matrix", "off[0::2] = d\n    off[1::2] = e[: max(n - 1, 0)]",
     "off[1::2] = d[: max(n - 1, 0)]\n    off[0::2] = np.append(e[: max(n - 1, 0)], d[-1])"),
    ("u and v exchanged", "V = Zp[0::2, :]\n    U = Zp[1::2, :]", "U = Zp[0::2, :]\n    V = Zp[1::2, :]"),
    ("no sqrt(2)", "Zp = Z[:, pos] * np.sqrt(2.0)", "Zp = Z[:, pos]"),
    ("negative half", "pos = np.arange(2 * n - 1, n - 1, -1)", "pos = np.arange(0, n)"),
]


@pytest.mark.parametrize("name,old,new", MUTANTS)
def test_planted_mistakes_fail_a_pin(orc, name, old, new, tmp_path):
    import importlib.util
    import inspect
    import sys
    src = inspect.getsource(bd)
    assert old in src
    pkg = tmp_path / "mut_oracle"
    pkg.mkdir()
    (pkg / "__init__.py").write_text("from oracle import eig\n")
    (pkg / "bidiag.py").write_text(src.replace(old, new))
    sys.path.insert(0, str(tmp_path))
    try:
        spec = importlib.util.spec_from_file_location("mut_oracle.bidiag", pkg / "bidiag.py",
                                                      submodule_search_locations=None)
        import mut_oracle  # noqa: F401
        mod = importlib.util.module_from_spec(spec)
        mod.__package__ = "mut_oracle"
        spec.loader.exec_module(mod)
        n = 30
        g = np.random.default_rng(9)
        d = g.uniform(0.5, 1.5, n)
        e = g.uniform(-1, 1, n - 1)
        B = bd.bidiag(d, e)
        s, U, VT = mod.bdsdc(d, e)
        ok = (np.max(np.abs(s - np.linalg.svd(B, compute_uv=False))) <= 1e-12 and
              np.max(np.abs(U @ np.diag(s) @ VT - B)) <= 1e-12)
        assert not ok, name
    finally:
        sys.path.remove(str(tmp_path))
        sys.modules.pop("mut_oracle", None)
        sys.modules.pop("mut_oracle.bidiag", None)
