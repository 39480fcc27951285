"""Pins of the Householder-reduction oracle (oracle/householder.py) against facts fixed
outside it: the eigenvalues of T equal those of A (a library eigenvalue routine), Q is
orthogonal and Q^T A Q is exactly tridiagonal, a matrix that is already tridiagonal
comes back unchanged up to the signs of e, a 3 x 3 case worked by hand, and the
composed eigensolver satisfies A V = V Lam.  Each planted mistake fails one of them."""
import numpy as np
import pytest

from oracle import householder as hh


def sym(n, seed):
    g = np.random.default_rng(seed)
    X = g.uniform(-1, 1, (n, n))
    return (X + X.T) / 2


def q_matrix(V, tau, n):
    return hh.apply_q(V, tau, np.eye(n))


@pytest.mark.parametrize("n,seed", [(2, 1), (3, 2), (7, 3), (64, 4), (200, 5)])
def test_spectrum_orthogonality_and_similarity(n, seed):
    A = sym(n, seed)
    d, e, V, tau = hh.tridiagonalize(A)
    T = np.diag(d) + np.diag(e, 1) + np.diag(e, -1)
    nA = np.linalg.norm(A, 2)
    assert np.max(np.abs(np.linalg.eigvalsh(T) - np.linalg.eigvalsh(A))) <= 50 * n * np.finfo(float).eps * nA
    Q = q_matrix(V, tau, n)
    assert np.max(np.abs(Q.T @ Q - np.eye(n))) <= 20 * n * np.finfo(float).eps
    assert np.max(np.abs(Q.T @ A @ Q - T)) <= 50 * n * np.finfo(float).eps * nA


def test_tridiagonal_input_is_kept_up_to_signs():
    n = 40
    g = np.random.default_rng(6)
    d0, e0 = g.uniform(-1, 1, n), g.uniform(0.1, 1, n - 1)
    A = np.diag(d0) + np.diag(e0, 1) + np.diag(e0, -1)
    d, e, V, tau = hh.tridiagonalize(A)
    assert np.allclose(d, d0, atol=1e-15, rtol=0)
    assert np.allclose(np.abs(e), e0, atol=1e-15, rtol=0)
    assert np.all(tau == 0.0)


def test_three_by_three_by_hand():
    """A = [[4, 1, 2], [1, 3, 0], [2, 0, 1]]: the single reflector maps (1, 2) to
    beta e_1 with beta = -sqrt(5), so e_0 = -sqrt(5); rotating the trailing block by it
    H = [[-1, -2], [-2, 1]] / sqrt(5) (columns h_1, h_2) on diag(3, 1) gives
    d_1 = h_1^T B h_1 = (3 + 4)/5 = 7/5, d_2 = h_2^T B h_2 = (12 + 1)/5 = 13/5 and
    e_1 = h_1^T B h_2 = (6 - 2)/5 = 4/5; the trace 8 is kept."""
    A = np.array([[4.0, 1.0, 2.0], [1.0, 3.0, 0.0], [2.0, 0.0, 1.0]])
    d, e, V, tau = hh.tridiagonalize(A)
    assert np.allclose(d, [4.0, 7.0 / 5.0, 13.0 / 5.0], atol=1e-15)
    assert np.isclose(e[0], -np.sqrt(5.0), atol=1e-15)
    assert np.isclose(abs(e[1]), 4.0 / 5.0, atol=1e-15)


def test_composed_eigensolver(orc):
    n = 150
    A = sym(n, 7)
    lam, Vec, (d, e) = hh.syevd(A)
    eps = np.finfo(float).eps
    nA = np.linalg.norm(A, 2)
    assert np.max(np.abs(lam - np.linalg.eigvalsh(A))) <= 50 * n * eps * nA
    assert np.abs(A @ Vec - Vec * lam).sum(axis=0).max() / (n * nA * eps) <= 50
    assert np.abs(Vec.T @ Vec - np.eye(n)).sum(axis=0).max() / (n * eps) <= 50


MUTANTS = [
    ("beta sign", "beta = -np.copysign(np.hypot(alpha, sigma), alpha)", "beta = np.copysign(np.hypot(alpha, sigma), alpha)"),
    ("tau formula", "t = (beta - alpha) / beta", "t = (alpha - beta) / beta"),
    ("half factor", "w = p - 0.5 * t * float(p @ v) * v", "w = p - t * float(p @ v) * v"),
    ("one-sided update", "A22 -= np.outer(v, w) + np.outer(w, v)", "A22 -= 2 * np.outer(v, w)"),
    ("reflector order", "for k in range(V.shape[1] - 1, -1, -1):", "for k in range(V.shape[1]):"),
]


@pytest.mark.parametrize("name,old,new", MUTANTS)
def test_planted_mistakes_fail_a_pin(name, old, new, tmp_path):
    import importlib.util
    import inspect
    src = inspect.getsource(hh)
    assert old in src
    p = tmp_path / "hh_mutant.py"
    p.write_text(src.replace(old, new))
    spec = importlib.util.spec_from_file_location("hh_mutant", p)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    n = 30
    A = sym(n, 8)
    d, e, V, tau = mod.tridiagonalize(A)
    T = np.diag(d) + np.diag(e, 1) + np.diag(e, -1)
    Q = mod.apply_q(V, tau, np.eye(n))
    ok_spec = np.max(np.abs(np.linalg.eigvalsh(T) - np.linalg.eigvalsh(A))) <= 1e-12
    ok_sim = np.max(np.abs(Q.T @ A @ Q - T)) <= 1e-12
    d3, e3, _, _ = mod.tridiagonalize(np.array([[4.0, 1.0, 2.0], [1.0, 3.0, 0.0], [2.0, 0.0, 1.0]]))
    ok_hand = np.isclose(e3[0], -np.sqrt(5.0), atol=1e-15) and np.allclose(d3, [4.0, 1.4, 2.6], atol=1e-15)
    assert not (ok_spec and ok_sim and ok_hand), name
