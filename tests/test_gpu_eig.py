"""GPU parity of the divide-and-conquer eigensolver (tdc_eig / tdc_eig_batched /
tdc_rank_one through the C ABI) against the FP64 CPU oracle.

Tolerances (from the accuracy targets of the method): |lam - lam_oracle| <=
1e-12 ||T||_2, residual ||TQ - Q Lam||_1 / (n ||T|| eps) <= 50, orthogonality
||Q^T Q - I||_1 / (n eps) <= 50, eigenvectors equal up to sign (subspaces for
clusters)."""
import numpy as np
import pytest
import torch

from helpers import EPS, check_toeplitz_sampled, compare_vectors, dense, ratios
from paper_2008_01990_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tdc():
    from paper_2008_01990_gb300 import build, tdc as t
    build.build()
    t.lib()
    return t


DEV = "cuda:0"


def run_gpu(tdc, d, e, **kw):
    o = tdc.default_opts(**kw)
    lam, Q = tdc.eig(torch.tensor(d, device=DEV), torch.tensor(e, device=DEV), o, check=True)
    return lam.cpu().numpy(), Q.cpu().numpy()


def check_vs_oracle(orc, d, e, lam, Q, leaf, vec_tol=1e-9):
    lam_o, Q_o = orc.eig(d, e, leaf=leaf)
    nT = max(abs(lam_o[0]), abs(lam_o[-1]))
    assert np.max(np.abs(lam - lam_o)) <= 1e-12 * nT
    assert np.all(np.diff(lam) >= 0)
    if len(d) > 1:
        res, orth = ratios(d, e, lam, Q)
        assert res <= 50, res
        assert orth <= 50, orth
        compare_vectors(Q, Q_o, lam_o, 1e-8 * nT, vec_tol)
    im = np.argmax(np.abs(Q), axis=0)
    assert np.all(Q[im, np.arange(len(d))] > 0)
    return lam_o, Q_o


def assert_same_deflation(st, sto):
    """Deflation decisions agree level by level: the GPU's parallel tests and chain
    resolution must reproduce the oracle's sequential scan of Section 3.2 exactly
    (both decide in FP64 with the same tolerance): equal non-deflated sizes, equal
    type-1 (small z) and type-2 (rotation) counts."""
    assert st["levels"] == sto["levels"]
    assert st["sum_K"] == sto["sum_K"]
    assert st["type1"] == sto["type1"]
    assert st["type2"] == sto["type2"]


def test_c1_uniform_1024(tdc, orc):
    n = 1024
    d, e = inputs.uniform_tridiag(n, 1)
    lam, Q = run_gpu(tdc, d, e, leaf=32, collect_stats=1)
    check_vs_oracle(orc, d, e, lam, Q, 32)
    st = tdc.get_stats()
    _, _, sto = orc.eig(d, e, leaf=32, with_stats=True)
    assert st["levels"] == sto["levels"] == 5
    assert_same_deflation(st, sto)


@pytest.mark.parametrize("fam,n,leaf", [("c4", 1500, 64), ("toeplitz", 2048, 64), ("uniform", 3000, 16),
                                        ("clement", 2049, 32)])
def test_deflation_counts_equal_the_oracle_scan(tdc, orc, fam, n, leaf):
    d, e = inputs.family(fam, n, 4)
    run_gpu(tdc, d, e, leaf=leaf, collect_stats=1)
    st = tdc.get_stats()
    _, _, sto = orc.eig(d, e, leaf=leaf, with_stats=True)
    assert_same_deflation(st, sto)


@pytest.mark.parametrize("n,leaf", [(2100, 16), (5000, 32)])
def test_glued_wilkinson_clusters(tdc, orc, n, leaf):
    """Copies of W+_21 glued by 1e-10: clusters of nearly equal eigenvalues, whose merges
    deflate long runs of poles by chained rotations.  Eigenvalues against the oracle's;
    residual and orthogonality ratios <= 50 (the clusters' vectors are only fixed as
    subspaces).  The deflation counts are not compared here: many of this family's type-2
    tests fall within rounding of the tolerance, so the GPU's children eigenvalues and the
    oracle's, equally accurate, can decide a few of them differently (at n = 2100, 283
    against 282 non-deflated poles at the top merge)."""
    d, e = inputs.family("wilkinson", n)
    lam, Q = run_gpu(tdc, d, e, leaf=leaf)
    lo, _ = orc.eig(d, e, leaf=leaf)
    nT = np.abs(lo).max()
    assert np.max(np.abs(lam - lo)) <= 1e-12 * nT
    res, orth = ratios(d, e, lam, Q)
    assert res <= 50 and orth <= 50, (res, orth)


@pytest.mark.parametrize("n,leaf", [(1, 32), (2, 2), (3, 2), (5, 2), (9, 2), (31, 32), (33, 32), (64, 64), (65, 64),
                                    (100, 7), (257, 32), (777, 13), (1000, 64)])
def test_ragged_sizes(tdc, orc, n, leaf):
    d, e = inputs.uniform_tridiag(n, 1000 + n)
    lam, Q = run_gpu(tdc, d, e, leaf=leaf)
    check_vs_oracle(orc, d, e, lam, Q, leaf)


@pytest.mark.parametrize("n,leaf,fam", [(3000, 16, "uniform"), (2500, 31, "c4"), (4100, 8, "sht"), (2049, 32, "clement")])
def test_many_small_leaves(tdc, orc, n, leaf, fam):
    """Problems with many leaves of at most 32 rows take the many-leaves-per-block QR."""
    d, e = inputs.family(fam, n, 7)
    lam, Q = run_gpu(tdc, d, e, leaf=leaf)
    check_vs_oracle(orc, d, e, lam, Q, leaf, vec_tol=1e-7)


def test_toeplitz_2048_closed_form_and_deflation(tdc, orc):
    n = 2048
    d, e = inputs.toeplitz_tridiag(n)
    lam, Q = run_gpu(tdc, d, e, leaf=64, collect_stats=1)
    k = np.arange(1, n + 1)
    ref = np.sort(2.0 + 2.0 * np.cos(k * np.pi / (n + 1)))
    assert np.max(np.abs(lam - ref)) <= 1e-12 * 4
    check_vs_oracle(orc, d, e, lam, Q, 64, vec_tol=1e-8)
    st = tdc.get_stats()
    assert st["sum_K"][0] == n // 2
    assert st["type2"][0] == n // 2


@pytest.mark.parametrize("fam,n,leaf", [("clement", 501, 16), ("hermite", 300, 32), ("sht", 700, 32),
                                        ("c4", 1500, 64)])
def test_families(tdc, orc, fam, n, leaf):
    d, e = inputs.family(fam, n, 4)
    lam, Q = run_gpu(tdc, d, e, leaf=leaf)
    check_vs_oracle(orc, d, e, lam, Q, leaf, vec_tol=1e-7)


def test_zero_coupling_deflates_everything(tdc, orc):
    n = 256
    d, e = inputs.uniform_tridiag(n, 77)
    e[n // 2 - 1] = 0.0
    e[n // 4 - 1] = 0.0
    lam, Q = run_gpu(tdc, d, e, leaf=16, collect_stats=1)
    check_vs_oracle(orc, d, e, lam, Q, 16)
    assert tdc.get_stats()["sum_K"][0] == 0


def test_leading_dimension_and_inputs_untouched(tdc, orc):
    n, ld = 300, 311
    d, e = inputs.uniform_tridiag(n, 5)
    dt = torch.tensor(d, device=DEV)
    et = torch.tensor(e, device=DEV)
    store = torch.full((n, ld), 7.0, dtype=torch.float64, device=DEV)  # column-major n x n with ld 311
    Qv = store.t()[:n, :]
    assert Qv.stride(1) == ld
    lam, Q = tdc.eig(dt, et, tdc.default_opts(leaf=32), Q=Qv, check=True)
    assert torch.equal(dt.cpu(), torch.tensor(d)) and torch.equal(et.cpu(), torch.tensor(e))
    assert torch.all(store[:, n:] == 7.0)  # padding rows untouched
    check_vs_oracle(orc, d, e, lam.cpu().numpy(), Q.cpu().numpy(), 32)


def test_batched_uneven_sizes(tdc, orc):
    sizes = np.array([1, 5, 33, 64, 100, 257, 2, 130])
    d, e, offs = inputs.batched_uniform(sizes, 3)
    qoffs = np.concatenate([[0], np.cumsum(sizes.astype(np.int64) ** 2)])
    dt = torch.tensor(d, device=DEV)
    et = torch.tensor(e, device=DEV)
    lam = torch.zeros(int(offs[-1]), dtype=torch.float64, device=DEV)
    Q = torch.zeros(int(qoffs[-1]), dtype=torch.float64, device=DEV)
    tdc.eig_batched(sizes, dt, et, offs[:-1], qoffs[:-1], lam, Q, tdc.default_opts(leaf=16), check=True)
    lam = lam.cpu().numpy()
    Q = Q.cpu().numpy()
    for b, nb in enumerate(sizes):
        lb = lam[offs[b]:offs[b] + nb]
        Qb = Q[qoffs[b]:qoffs[b] + nb * nb].reshape(nb, nb, order="F")
        check_vs_oracle(orc, d[offs[b]:offs[b] + nb], e[offs[b]:offs[b] + nb - 1], lb, Qb, 16)


def test_rank_one_vs_oracle(tdc, orc):
    K = 3000
    g = inputs.SplitMix64(17)
    D = np.sort(g.uniform(K, -1.0, 1.0))
    z = g.uniform(K, -1.0, 1.0)
    z /= np.linalg.norm(z)
    rho = 0.9
    org, tau, zh, s = tdc.rank_one(torch.tensor(D, device=DEV), torch.tensor(z, device=DEV), rho, check=True)
    org = org.cpu().numpy()
    tau = tau.cpu().numpy()
    zh = zh.cpu().numpy()
    s = s.cpu().numpy()
    org_o, tau_o, lam_o, _ = orc.secular(D, z, rho)
    lam = D[org] + tau
    # every root within a few ulps of the pole gap scale; interlacing
    assert np.all(lam > D) and np.all(lam[:-1] < D[1:])
    assert np.max(np.abs(lam - lam_o)) <= 64 * EPS * max(1.0, rho)
    # offsets from the same pole agree to relative accuracy
    same = org == org_o
    assert np.mean(same) > 0.99
    assert np.max(np.abs(tau[same] - tau_o[same]) / np.abs(tau_o[same])) <= 1e-11
    zh_o = orc.lowner(D, z, rho, org_o, tau_o)
    assert np.max(np.abs(zh - zh_o) / np.abs(zh_o)) <= 1e-10
    s_o = orc.colnorm(D, org_o, tau_o, zh_o)
    assert np.max(np.abs(s - s_o) / s_o) <= 1e-10


def test_status_nonconvergence_then_recovery(tdc, orc):
    n = 512
    d, e = inputs.uniform_tridiag(n, 9)
    o = tdc.default_opts(leaf=32, max_iter=1)
    tdc.eig(torch.tensor(d, device=DEV), torch.tensor(e, device=DEV), o)
    assert tdc.sync_status() == tdc.TDC_ENOCONV
    lam, Q = run_gpu(tdc, d, e, leaf=32)  # the next call is clean
    check_vs_oracle(orc, d, e, lam, Q, 32)


@pytest.mark.parametrize("n,where,val", [(100, "d", np.nan), (3000, "e", np.nan), (9000, "d", np.inf),
                                         (9000, "e", -np.inf)])
def test_status_nonfinite_input(tdc, n, where, val):
    """A non-finite d or e entry is read as zero: the call reports TDC_ENONFINITE and
    returns the eigendecomposition of the input with that entry zeroed (finite, so no
    NaN reaches the orderings and ranks the kernels index with, on every merge path the
    default options take up to n = 9000); the next call is clean."""
    from scipy.linalg import eigvalsh_tridiagonal
    d, e = inputs.uniform_tridiag(n, 9)
    (d if where == "d" else e)[n // 3] = val
    lam, Q = tdc.eig(torch.tensor(d, device=DEV), torch.tensor(e, device=DEV), tdc.default_opts(leaf=16))
    assert tdc.sync_status() == tdc.TDC_ENONFINITE
    assert bool(torch.isfinite(lam).all()) and bool(torch.isfinite(Q).all())
    (d if where == "d" else e)[n // 3] = 0.0
    lam, ref = lam.cpu().numpy(), eigvalsh_tridiagonal(d, e)
    assert np.max(np.abs(lam - ref)) <= 50 * n * EPS * np.max(np.abs(ref))
    if n <= 3000:
        res, orth = ratios(d, e, lam, Q.cpu().numpy())
        assert res <= 50 and orth <= 50, (res, orth)
    assert tdc.sync_status() == 0


def _unit_scaled(d, e):
    """d, e times the power of two that puts their largest magnitude in [1, 2)."""
    m = np.frexp(max(np.abs(d).max(), np.abs(e).max()))[1] - 1
    return np.ldexp(d, -m), np.ldexp(e, -m)


@pytest.mark.parametrize("n,k", [(3000, 600), (3000, -600), (3000, 1000), (3000, -900), (9000, 600)])
def test_extreme_scales_are_solved_exactly_scaled(tdc, n, k):
    """Entries far outside [2^-400, 2^400] (where squares and products of entries would
    overflow or underflow): the problem is solved scaled by the power of two that puts its
    largest entry in [1, 2), so its eigenvectors equal, bit for bit, those of that problem
    and its eigenvalues are that problem's times 2^k exactly (n = 9000 takes the
    structured products)."""
    d0, e0 = _unit_scaled(*inputs.uniform_tridiag(n, 7))
    o = tdc.default_opts(leaf=16)
    lam0, Q0 = tdc.eig(torch.tensor(d0, device=DEV), torch.tensor(e0, device=DEV), o, check=True)
    lam1, Q1 = tdc.eig(torch.tensor(np.ldexp(d0, k), device=DEV), torch.tensor(np.ldexp(e0, k), device=DEV), o,
                       check=True)
    assert torch.equal(Q0, Q1)
    assert np.array_equal(lam1.cpu().numpy(), np.ldexp(lam0.cpu().numpy(), k))


def test_c2_toeplitz_16384_sampled(tdc):
    """Full-size tridiag(1,2,1) at n=16384 in the benchmark's configuration (leaf 16,
    default merge): every eigenvalue against the closed form; residual, orthogonality and
    sine vectors on sampled columns."""
    n = 16384
    d, e = inputs.toeplitz_tridiag(n)
    dt = torch.tensor(d, device=DEV)
    et = torch.tensor(e, device=DEV)
    lam, Q = tdc.eig(dt, et, tdc.default_opts(leaf=16), check=True)
    check_toeplitz_sampled(lam, Q, n)


def test_calls_from_two_host_threads_on_two_streams(tdc):
    """Each host thread gets its own internal products stream; two eigensolves issued
    at the same time from two threads on two caller streams give the results of the
    same calls made one after the other."""
    import threading
    cases = [inputs.uniform_tridiag(1500, 11), inputs.c4_tridiag(1800, 12)]
    o = tdc.default_opts(leaf=32)
    ref = []
    for d, e in cases:
        lam, Q = tdc.eig(torch.tensor(d, device=DEV), torch.tensor(e, device=DEV), o, check=True)
        ref.append((lam.cpu().numpy(), Q.cpu().numpy()))
    out = [None, None]
    errors = []

    def work(k):
        try:
            s = torch.cuda.Stream()
            d, e = cases[k]
            with torch.cuda.stream(s):
                dt, et = torch.tensor(d, device=DEV), torch.tensor(e, device=DEV)
                for _ in range(3):
                    lam, Q = tdc.eig(dt, et, o, stream=s)
                s.synchronize()
            out[k] = (lam.cpu().numpy(), Q.cpu().numpy())
        except Exception as exc:  # reported below, on the test's thread
            errors.append(exc)

    threads = [threading.Thread(target=work, args=(k,)) for k in range(2)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
    assert tdc.sync_status() == 0
    for k in range(2):
        assert np.array_equal(out[k][0], ref[k][0])
        assert np.array_equal(out[k][1], ref[k][1])
