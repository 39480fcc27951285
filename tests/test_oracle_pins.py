"""Pins of the FP64 CPU oracle against facts fixed outside it.

Every check here comes from mathematics or a source independent of the oracle:
closed-form spectra (tridiag(1,2,1), Clement/Kac, Hermite), brute-force Jacobi
rotations on tiny matrices, Sturm-sequence inertia counts, the trace and
Frobenius invariants, Cauchy interlacing, dense library eigensolvers on small
arrow/rank-one matrices, and the published SplitMix64 test vector.
"""
import numpy as np
import pytest

from paper_2008_01990_gb300 import inputs

EPS = np.finfo(np.float64).eps


def dense(d, e):
    return np.diag(d) + np.diag(e, 1) + np.diag(e, -1)


def norm1(d, e):
    a = np.abs(np.asarray(d, dtype=float)).copy()
    e = np.abs(np.asarray(e, dtype=float))
    a[:-1] += e
    a[1:] += e
    return float(a.max()) if a.size else 0.0


def jacobi_eig(A, sweeps=60):
    """Cyclic Jacobi rotations on a small dense symmetric matrix (brute force)."""
    A = np.array(A, dtype=float)
    n = A.shape[0]
    V = np.eye(n)
    for _ in range(sweeps):
        off = np.sqrt(np.sum((A - np.diag(np.diag(A))) ** 2))
        if off <= 1e-300:
            break
        for p in range(n - 1):
            for q in range(p + 1, n):
                if A[p, q] == 0.0:
                    continue
                theta = (A[q, q] - A[p, p]) / (2.0 * A[p, q])
                if theta == 0:
                    t = 1.0
                elif abs(theta) > 1e150:
                    t = 0.5 / theta
                else:
                    t = np.sign(theta) / (abs(theta) + np.sqrt(theta * theta + 1.0))
                c = 1.0 / np.sqrt(t * t + 1.0)
                s = t * c
                J = np.eye(n)
                J[p, p] = c
                J[q, q] = c
                J[p, q] = s
                J[q, p] = -s
                A = J.T @ A @ J
                V = V @ J
    w = np.diag(A).copy()
    o = np.argsort(w)
    return w[o], V[:, o]


def sturm_count(d, e, x):
    """Number of eigenvalues of T below each x (LDL^T pivot signs)."""
    x = np.atleast_1d(np.asarray(x, dtype=float))
    cnt = np.zeros(x.shape, dtype=np.int64)
    q = d[0] - x
    tiny = 1e-300
    q = np.where(q == 0, -tiny, q)
    cnt += q < 0
    for i in range(1, len(d)):
        q = (d[i] - x) - e[i - 1] ** 2 / q
        q = np.where(q == 0, -tiny, q)
        cnt += q < 0
    return cnt


def toeplitz_closed_form(n):
    """tridiag(1,2,1): lambda_k = 2 + 2 cos(k pi/(n+1)), q_k(j) = sqrt(2/(n+1)) sin(j k pi/(n+1)),
    returned in ascending eigenvalue order."""
    k = np.arange(1, n + 1)
    lam = 2.0 + 2.0 * np.cos(k * np.pi / (n + 1))
    j = np.arange(1, n + 1)[:, None]
    V = np.sqrt(2.0 / (n + 1)) * np.sin(j * k[None, :] * np.pi / (n + 1))
    o = np.argsort(lam)
    return lam[o], V[:, o]


def ratios(d, e, lam, Q):
    n = len(d)
    T = dense(d, e)
    nT = norm1(d, e)
    res = np.abs(T @ Q - Q * lam).sum(axis=0).max() / (n * nT * EPS)
    orth = np.abs(Q.T @ Q - np.eye(n)).sum(axis=0).max() / (n * EPS)
    return res, orth


def match_vectors_up_to_sign(Q, V, lam, clusters_tol):
    """|<q_j, v_j>| ~ 1 for isolated eigenvalues."""
    n = Q.shape[0]
    gaps = np.full(n, np.inf)
    gaps[1:] = np.minimum(gaps[1:], np.diff(lam))
    gaps[:-1] = np.minimum(gaps[:-1], np.diff(lam))
    iso = gaps > clusters_tol
    dots = np.abs(np.sum(Q * V, axis=0))
    return dots[iso]


# ---------------------------------------------------------------- inputs
def test_splitmix64_published_vector():
    # Published reference outputs of SplitMix64 seeded with 0.
    g = inputs.SplitMix64(0)
    assert [int(v) for v in g.next_u64(3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_tree_depth_definition(orc):
    for n in [1, 2, 31, 32, 33, 64, 65, 1000, 1024, 16384, 32768]:
        for leaf in [1, 8, 32, 64]:
            t = orc.tree_depth(n, leaf)
            assert -(-n // (1 << t)) <= leaf
            if t > 0:
                assert -(-n // (1 << (t - 1))) > leaf


# ---------------------------------------------------------------- leaf solver
@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 13, 16])
def test_leaf_qr_vs_jacobi(orc, n):
    d, e = inputs.uniform_tridiag(n, 100 + n)
    lam, Q, status = orc.leaf_qr(d, e)
    assert status == 0
    w, V = jacobi_eig(dense(d, e))
    nT = norm1(d, e)
    assert np.max(np.abs(lam - w)) <= 1e-13 * nT
    if n > 1:
        dots = match_vectors_up_to_sign(Q, V, w, 1e-6 * nT)
        assert np.all(np.abs(dots - 1.0) < 1e-10)
    res, orth = ratios(d, e, lam, Q)
    assert res < 5 and orth < 5


def test_leaf_qr_toeplitz_closed_form(orc):
    n = 24
    d, e = inputs.toeplitz_tridiag(n)
    lam, Q, status = orc.leaf_qr(d, e)
    lam_ref, V = toeplitz_closed_form(n)
    assert np.max(np.abs(lam - lam_ref)) <= 1e-14 * 4
    assert np.all(np.abs(np.abs(np.sum(Q * V, axis=0)) - 1) < 1e-12)


# ---------------------------------------------------------------- secular / Loewner
def rank_one_case(K, seed, rho=0.7):
    g = inputs.SplitMix64(seed)
    D = np.sort(g.uniform(K, -1.0, 1.0))
    z = g.uniform(K, -1.0, 1.0)
    z /= np.linalg.norm(z)
    return D, z, rho


@pytest.mark.parametrize("K,seed", [(1, 1), (2, 2), (7, 3), (40, 4), (64, 5)])
def test_secular_roots_vs_dense_eig(orc, K, seed):
    D, z, rho = rank_one_case(K, seed)
    org, tau, lam, it = orc.secular(D, z, rho)
    assert it > 0
    ref = np.linalg.eigvalsh(np.diag(D) + rho * np.outer(z, z))
    scale = max(np.abs(D).max(), rho)
    assert np.max(np.abs(lam - ref)) <= 4e-15 * K * scale
    # strict interlacing d_j < lambda_j < d_{j+1}, lambda_K < d_K + rho ||z||^2
    assert np.all(lam > D)
    assert np.all(lam[:-1] < D[1:])
    assert lam[-1] <= D[-1] + rho * np.dot(z, z) * (1 + 1e-15)
    # origin is the closer pole
    for j in range(K):
        assert org[j] in (j, j + 1)
        if org[j] == j:
            assert tau[j] > 0
        else:
            assert tau[j] < 0


def test_secular_value_is_small(orc):
    D, z, rho = rank_one_case(50, 9)
    org, tau, lam, it = orc.secular(D, z, rho)
    for j in range(50):
        delta = (D - D[org[j]]) - tau[j]
        terms = z * z / delta
        f = 1.0 / rho + terms.sum()
        assert abs(f) <= 64 * EPS * (1.0 / rho + np.abs(terms).sum())


@pytest.mark.parametrize("K,seed", [(3, 11), (30, 12), (64, 13)])
def test_lowner_zhat_reproduces_roots(orc, K, seed):
    D, z, rho = rank_one_case(K, seed)
    org, tau, lam, _ = orc.secular(D, z, rho)
    zh = orc.lowner(D, z, rho, org, tau)
    # D + rho zhat zhat^T has exactly the computed roots as eigenvalues
    w = np.linalg.eigvalsh(np.diag(D) + rho * np.outer(zh, zh))
    assert np.max(np.abs(w - lam)) <= 8 * EPS * K * max(1.0, np.abs(D).max())
    assert np.all(np.sign(zh) == np.sign(z))
    assert np.max(np.abs(zh - z)) <= 1e-12
    s = orc.colnorm(D, org, tau, zh)
    U = orc.qhat(D, org, tau, zh, s)
    assert np.abs(U.T @ U - np.eye(K)).max() <= 10 * K * EPS
    M = np.diag(D) + rho * np.outer(zh, zh)
    assert np.abs(M @ U - U * lam).max() <= 10 * K * EPS


def test_qhat_is_cauchy_like(orc):
    # Eq. (Q_Cauchy): the displacement D Qhat - Qhat Lambda has rank one.
    D, z, rho = rank_one_case(32, 21)
    org, tau, lam, _ = orc.secular(D, z, rho)
    zh = orc.lowner(D, z, rho, org, tau)
    s = orc.colnorm(D, org, tau, zh)
    U = orc.qhat(D, org, tau, zh, s)
    Disp = np.diag(D) @ U - U @ np.diag(lam)
    sv = np.linalg.svd(Disp, compute_uv=False)
    assert sv[1] <= 1e-12 * sv[0]
    assert np.allclose(Disp, np.outer(zh, s), atol=1e-12)


# ---------------------------------------------------------------- deflation
def test_deflation_type1_small_z(orc):
    n = 12
    D = np.linspace(-1, 1, n)
    z = np.full(n, 1.0 / np.sqrt(n))
    z[[2, 7]] = 1e-20
    K, kept, defl, D2, z2, Q, t1, t2 = orc.deflate(D, z, 0.5)
    assert (t1, t2, K) == (2, 0, n - 2)
    assert sorted(defl.tolist()) == [2, 7]
    assert np.array_equal(Q, np.eye(n))


def test_deflation_type2_duplicate_poles(orc):
    # three exact duplicates: each pair deflates by one plane rotation
    n = 10
    D = np.array([0.1, 0.5, 0.5, 0.9, 1.3, 1.3, 1.7, 2.0, 2.0, 2.5])
    g = inputs.SplitMix64(5)
    z = g.uniform(n, 0.2, 1.0)
    z /= np.linalg.norm(z)
    rho = 0.8
    K, kept, defl, D2, z2, Q, t1, t2 = orc.deflate(D, z, rho)
    assert (t1, t2, K) == (0, 3, n - 3)
    M = np.diag(D) + rho * np.outer(z, z)
    Mr = Q.T @ M @ Q
    for p in defl:
        row = Mr[p].copy()
        row[p] -= D2[p]
        assert np.abs(row).max() <= 1e-14
    assert np.all(z2[defl] == 0)
    assert np.all(np.diff(D2[kept]) > 0)
    assert np.allclose(Q.T @ Q, np.eye(n), atol=1e-15)


def test_deflation_type2_near_poles_small_weight(orc):
    # Section 3.2: poles 1e-7 apart whose weight ratio is 3e-9 deflate by one rotation
    # (|t c s| ~ 3e-16 is below the tolerance) although neither weight is negligible on its
    # own.  The rotated column must then be an eigenvector of Q^T M Q for the pole left
    # in its place, up to the deflation tolerance, and the kept pole must carry the weight.
    D = np.array([-0.8, -0.2, 0.1, 0.3, 0.3 + 1e-7, 0.6, 0.9])
    z = np.array([0.4, 0.35, 0.3, 1e-9, 0.5, 0.45, 0.42])
    z /= np.linalg.norm(z)
    rho = 1.0
    K, kept, defl, D2, z2, Q, t1, t2 = orc.deflate(D, z, rho)
    assert (t1, t2, K) == (0, 1, 6)
    assert defl.tolist() == [3]
    M = np.diag(D) + rho * np.outer(z, z)
    Mr = Q.T @ M @ Q
    row = Mr[3].copy()
    row[3] -= D2[3]
    assert np.abs(row).max() <= 16 * EPS
    assert abs(D2[3] - 0.3) <= 1e-15 and abs(D2[4] - (0.3 + 1e-7)) <= 1e-15
    assert z2[3] == 0 and abs(z2[4] - np.hypot(z[3], z[4])) <= EPS


def test_deflation_everything_when_rho_zero(orc):
    n = 6
    K, kept, defl, *_ = orc.deflate(np.arange(n, dtype=float), np.ones(n) / np.sqrt(n), 0.0)
    assert K == 0 and len(defl) == n


# ---------------------------------------------------------------- full eigensolve
def test_dc_toeplitz_closed_form(orc):
    n = 1000
    d, e = inputs.toeplitz_tridiag(n)
    lam, Q = orc.eig(d, e, leaf=32)
    ref, V = toeplitz_closed_form(n)
    assert np.max(np.abs(lam - ref)) <= 1e-12 * 4.0
    dots = np.abs(np.sum(Q * V, axis=0))
    assert np.all(np.abs(dots - 1.0) < 1e-6)
    res, orth = ratios(d, e, lam, Q)
    assert res <= 50 and orth <= 50


def test_dc_clement_closed_form(orc):
    n = 101
    d, e = inputs.clement_tridiag(n)
    lam, Q = orc.eig(d, e, leaf=8)
    ref = np.arange(-(n - 1), n, 2, dtype=float)
    nT = norm1(d, e)
    assert np.max(np.abs(lam - ref)) <= 1e-12 * nT


def test_dc_hermite_closed_form(orc):
    n = 120
    d, e = inputs.hermite_tridiag(n)
    lam, Q = orc.eig(d, e, leaf=16)
    ref = np.polynomial.hermite_e.hermegauss(n)[0]
    nT = norm1(d, e)
    assert np.max(np.abs(lam - np.sort(ref))) <= 1e-12 * nT


@pytest.mark.parametrize("n,leaf,seed", [(1, 32, 1), (2, 2, 1), (3, 2, 2), (17, 2, 3), (19, 4, 3), (300, 32, 4), (1024, 32, 1)])
def test_dc_uniform_sturm_and_invariants(orc, n, leaf, seed):
    d, e = inputs.uniform_tridiag(n, seed)
    lam, Q = orc.eig(d, e, leaf=leaf)
    nT = max(norm1(d, e), 1e-300)
    assert np.all(np.diff(lam) >= 0)
    # Sturm counts pin every eigenvalue independently of the solver
    tol = 1e-12 * nT
    below = sturm_count(d, e, lam - tol)
    above = sturm_count(d, e, lam + tol)
    k = np.arange(n)
    assert np.all(below <= k) and np.all(above >= k + 1)
    # trace and Frobenius invariants
    assert abs(lam.sum() - d.sum()) <= 1e-13 * n * nT
    assert abs(np.sum(lam ** 2) - (np.sum(d ** 2) + 2 * np.sum(e ** 2))) <= 1e-13 * n * nT * nT
    if n > 1:
        res, orth = ratios(d, e, lam, Q)
        assert res <= 50 and orth <= 50
        # Cauchy interlacing with the leading (n-1) x (n-1) block
        mu, _ = orc.eig(d[:-1], e[:-2] if n > 2 else e[:0], leaf=leaf)
        assert np.all(lam[:-1] <= mu + tol) and np.all(mu <= lam[1:] + tol)
    # sign convention: the largest-magnitude entry of each column is positive
    im = np.argmax(np.abs(Q), axis=0)
    assert np.all(Q[im, np.arange(n)] > 0)


def test_dc_vs_dense_library(orc):
    n = 256
    d, e = inputs.c4_tridiag(n, 4)
    lam, Q = orc.eig(d, e, leaf=16)
    ref = np.linalg.eigvalsh(dense(d, e))
    assert np.max(np.abs(lam - ref)) <= 1e-12 * norm1(d, e)


@pytest.mark.parametrize("fam,n,leaf", [("sht", 400, 32), ("hermite", 333, 16), ("clement", 257, 8),
                                        ("toeplitz", 300, 64), ("wilkinson", 525, 16)])
def test_dc_families_vs_dense_library(orc, fam, n, leaf):
    # every family the GPU parity tests use: eigenvalues against the dense library
    # solver, residual and orthogonality ratios
    d, e = inputs.family(fam, n, 4)
    lam, Q = orc.eig(d, e, leaf=leaf)
    nT = norm1(d, e)
    assert np.max(np.abs(lam - np.linalg.eigvalsh(dense(d, e)))) <= 1e-12 * nT
    res, orth = ratios(d, e, lam, Q)
    assert res <= 50 and orth <= 50


def test_glued_wilkinson_is_copies_of_w21(orc):
    # with the glue at zero the matrix is 5 decoupled copies of W+_21: every eigenvalue of
    # W+_21 (dense library) five times; with the glue at 1e-10 each moves by at most the glue
    from paper_2008_01990_gb300.inputs import glued_wilkinson
    w = np.linalg.eigvalsh(dense(np.abs(np.arange(21) - 10).astype(float), np.ones(20)))
    for glue in (0.0, 1e-10):
        d, e = glued_wilkinson(105, glue=glue)
        lam, _ = orc.eig(d, e, leaf=16)
        assert np.max(np.abs(lam - np.sort(np.repeat(w, 5)))) <= (1e-13 if glue == 0.0 else 2e-10) * 11


def test_dc_zero_coupling_deflates_everything(orc):
    # e at the top split is 0: the merge is a pure sort of the two halves
    n = 64
    d, e = inputs.uniform_tridiag(n, 77)
    e[n // 2 - 1] = 0.0
    lam, Q, st = orc.eig(d, e, leaf=16, with_stats=True)
    assert st["sum_K"][0] == 0
    ref = np.linalg.eigvalsh(dense(d, e))
    assert np.max(np.abs(lam - ref)) <= 1e-12 * norm1(d, e)


def test_dc_toeplitz_top_merge_deflates_half(orc):
    # the midpoint split of tridiag(1,2,1) gives halves with identical spectra
    n = 512
    d, e = inputs.toeplitz_tridiag(n)
    lam, Q, st = orc.eig(d, e, leaf=32, with_stats=True)
    assert st["sum_K"][0] == n // 2
    assert st["type2"][0] == n // 2


def test_gemm_matches_numpy(orc):
    g = inputs.SplitMix64(3)
    A = g.uniform(35 * 17, -1, 1).reshape(35, 17)
    B = g.uniform(17 * 9, -1, 1).reshape(17, 9)
    assert np.allclose(orc.gemm(A, B), A @ B, atol=1e-14)


def test_secular_iteration_stays_within_its_cap(orc):
    """The safeguarded Newton iteration halves its bracket at least every second step, so
    every root converges within the default cap of 200: on a problem of the batched
    workload that once needed 783 steps (n = 1633, entries uniform(-1,1)), and on a
    rank-one problem with a weight of 1e-14 (just above the deflation tolerance of
    about 8 eps), whose root sits about 1e-28 from its pole: the hardest root the merge
    passes to the secular solver."""
    from paper_2008_01990_gb300 import inputs
    sizes = inputs.batched_sizes(4096, 64, 2048, 3)
    d, e, offs = inputs.batched_uniform(sizes, 3)
    b = 2023
    nb = int(sizes[b])
    assert nb == 1633
    _, _, st = orc.eig(d[offs[b]:offs[b] + nb], e[offs[b]:offs[b] + nb - 1], leaf=32, with_stats=True)
    assert st["secular_noconv"] == 0 and st["secular_iter_max"] <= 200
    K = 64
    D = np.linspace(-1.0, 1.0, K)
    z = np.full(K, 1.0 / np.sqrt(K - 1))
    z[20] = 1e-14
    org, tau, lam, it = orc.secular(D, z, 0.7)
    assert 0 < it <= 200
    # the root next to the tiny weight: d_20 < lam_20 < d_20 + 1e-26
    assert org[20] == 20 and 0.0 < tau[20] < 1e-26
