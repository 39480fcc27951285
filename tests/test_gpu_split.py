"""Split-precision (tcgen05 BF16 digit) and FP64 eigenvector-update products
against the oracle's plain FP64 product, element by element, and the
eigensolver with the split merge against the oracle."""
import numpy as np
import pytest
import torch

from helpers import EPS, compare_vectors, ratios
from paper_2008_01990_gb300 import inputs

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def tdc():
    from paper_2008_01990_gb300 import build, tdc as t
    build.build()
    t.lib()
    return t


def generators(orc, K, seed):
    g = inputs.SplitMix64(seed)
    D = np.sort(g.uniform(K, -1.0, 1.0))
    z = g.uniform(K, -1.0, 1.0)
    z /= np.linalg.norm(z)
    org, tau, _, _ = orc.secular(D, z, 0.8)
    zh = orc.lowner(D, z, 0.8, org, tau)
    s = orc.colnorm(D, org, tau, zh)
    return D, org, tau, zh, s


def orthogonal_rows(orc, m, K, seed):
    # rows of an orthogonal matrix (the oracle's eigenvectors of a random tridiagonal)
    n = max(m, K)
    d, e = inputs.uniform_tridiag(n, seed)
    _, Q = orc.eig(d, e, leaf=32)
    return np.asfortranarray(Q[:m, :K])


def run_cauchy(tdc, A, D, org, tau, zh, s, mode, **kw):
    t = lambda x: torch.tensor(x, device=DEV)
    At = torch.tensor(np.ascontiguousarray(A.T), device=DEV).t()  # column-major
    C = tdc.cauchy_gemm(At, t(D), torch.tensor(org, dtype=torch.int32, device=DEV), t(tau), t(zh), t(s), mode,
                        tdc.default_opts(**kw), check=True)
    return C.cpu().numpy()


@pytest.mark.parametrize("m,K", [(1, 1), (37, 5), (300, 200), (129, 65), (256, 512)])
def test_cauchy_dense_vs_oracle(tdc, orc, m, K):
    D, org, tau, zh, s = generators(orc, K, 40 + K)
    A = orthogonal_rows(orc, m, K, 7 + m)
    U = orc.qhat(D, org, tau, zh, s)
    Co = orc.gemm(A, U)
    C = run_cauchy(tdc, A, D, org, tau, zh, s, tdc.MERGE_DENSE)
    assert np.max(np.abs(C - Co)) <= 1e-14 * max(1.0, np.sqrt(K))


@pytest.mark.parametrize("m,K", [(1, 1), (37, 5), (300, 200), (129, 65), (256, 512), (700, 1111)])
def test_cauchy_split_vs_oracle(tdc, orc, m, K):
    D, org, tau, zh, s = generators(orc, K, 40 + K)
    A = orthogonal_rows(orc, m, K, 7 + m)
    U = orc.qhat(D, org, tau, zh, s)
    Co = orc.gemm(A, U)
    C = run_cauchy(tdc, A, D, org, tau, zh, s, tdc.MERGE_SPLIT, split_slices=7)
    # 7 digits: truncation and dropped digit levels cost ~2^-56 sqrt(K) per entry
    assert np.max(np.abs(C - Co)) <= 2e-15 * max(1.0, np.sqrt(K))


def test_cauchy_split_error_follows_digit_count(tdc, orc):
    m, K = 256, 384
    D, org, tau, zh, s = generators(orc, K, 99)
    A = orthogonal_rows(orc, m, K, 5)
    Co = orc.gemm(A, orc.qhat(D, org, tau, zh, s))
    errs = {}
    for S in (3, 4, 5, 6, 7):
        C = run_cauchy(tdc, A, D, org, tau, zh, s, tdc.MERGE_SPLIT, split_slices=S)
        errs[S] = float(np.max(np.abs(C - Co)))
    for S in (3, 4, 5, 6):
        # each digit adds 8 bits: the error bound 2^-8S sqrt(K) and a real decrease
        assert errs[S] <= 2.0 ** (-8 * S) * 4 * np.sqrt(K)
        assert errs[S + 1] < errs[S] / 16
    assert errs[3] > 1e-9  # the digits really are the only precision (no FP64 shortcut)


@pytest.mark.parametrize("n,leaf,fam", [(1024, 32, "uniform"), (777, 13, "uniform"), (2048, 64, "toeplitz"),
                                        (1500, 64, "c4"), (501, 16, "clement")])
def test_eig_split_merge_vs_oracle(tdc, orc, n, leaf, fam):
    d, e = inputs.family(fam, n, 1)
    o = tdc.default_opts(leaf=leaf, merge_mode=tdc.MERGE_SPLIT, split_min_K=64)
    lam, Q = tdc.eig(torch.tensor(d, device=DEV), torch.tensor(e, device=DEV), o, check=True)
    lam, Q = lam.cpu().numpy(), Q.cpu().numpy()
    lam_o, Q_o = orc.eig(d, e, leaf=leaf)
    nT = max(abs(lam_o[0]), abs(lam_o[-1]))
    assert np.max(np.abs(lam - lam_o)) <= 1e-12 * nT
    res, orth = ratios(d, e, lam, Q)
    assert res <= 50 and orth <= 50, (res, orth)
    compare_vectors(Q, Q_o, lam_o, 1e-8 * nT, 1e-7)


def sturm_count(d, e, x):
    x = np.atleast_1d(np.asarray(x, dtype=float))
    cnt = np.zeros(x.shape, dtype=np.int64)
    q = d[0] - x
    q = np.where(q == 0, -1e-300, q)
    cnt += q < 0
    for i in range(1, len(d)):
        q = (d[i] - x) - e[i - 1] ** 2 / q
        q = np.where(q == 0, -1e-300, q)
        cnt += q < 0
    return cnt


def test_c4_split_32768_sampled(tdc):
    """n = 32768, d uniform(0,1), e = 1 (seed 4), split merge: sampled eigenvalues
    pinned by Sturm counts, trace invariant, residual and orthogonality on sampled
    columns (the oracle is too slow at this order; these properties hold at any size)."""
    n = 32768
    d, e = inputs.c4_tridiag(n, 4)
    dt, et = torch.tensor(d, device=DEV), torch.tensor(e, device=DEV)
    lam, Q = tdc.eig(dt, et, tdc.default_opts(leaf=64, merge_mode=tdc.MERGE_SPLIT), check=True)
    lh = lam.cpu().numpy()
    nT = max(abs(lh[0]), abs(lh[-1]))
    assert np.all(np.diff(lh) >= 0)
    assert abs(lh.sum() - d.sum()) <= 1e-12 * n * nT
    g = np.random.default_rng(1)
    ks = np.sort(g.choice(n, 64, replace=False))
    tol = 1e-12 * nT
    assert np.all(sturm_count(d, e, lh[ks] - tol) <= ks)
    assert np.all(sturm_count(d, e, lh[ks] + tol) >= ks + 1)
    cols = torch.tensor(np.sort(g.choice(n, 256, replace=False)), device=DEV)
    Qs = Q[:, cols]
    Tq = dt[:, None] * Qs
    Tq[1:] += et[:, None] * Qs[:-1]
    Tq[:-1] += et[:, None] * Qs[1:]
    res = torch.abs(Tq - Qs * lam[cols]).sum(dim=0).max().item() / (n * nT * EPS)
    Gm = Qs.t() @ Q
    Gm[torch.arange(256, device=DEV), cols] -= 1.0
    orth = torch.abs(Gm).sum(dim=1).max().item() / (n * EPS)
    assert res <= 50 and orth <= 50, (res, orth)


def test_bounded_waits_expire_report_a_timeout_and_leave_the_device_usable(tdc, orc):
    """Failure detection without a GPU fault: with a spin budget of one try, the split
    product's epilogue cannot wait out a tile of 512 k-steps (about 0.3 ms), so its
    bounded wait expires.  The CTA then lets its issued copies and MMAs land (their
    own, fixed bound), releases its TMEM and returns; the call reports TDC_ETIMEOUT
    through its status slot.  The next calls, with the default budget, are correct."""
    K = m = 8192
    g = torch.Generator(device=DEV)
    g.manual_seed(11)
    D = torch.sort(torch.rand(K, dtype=torch.float64, device=DEV, generator=g) * 2 - 1).values
    z = torch.rand(K, dtype=torch.float64, device=DEV, generator=g) * 2 - 1
    z /= torch.linalg.norm(z)
    org, tau, zh, s = tdc.rank_one(D, z, 0.9, check=True)
    A = ((torch.rand(K, m, dtype=torch.float64, device=DEV, generator=g) * 2 - 1) / np.sqrt(K)).t()
    o1 = tdc.default_opts(spin_budget=1)
    ws = tdc.workspace(tdc.cauchy_gemm_workspace_size(m, K, tdc.MERGE_SPLIT, o1), DEV)
    tdc.cauchy_gemm(A, D, org, tau, zh, s, tdc.MERGE_SPLIT, o1, ws=ws)
    assert tdc.sync_status() == tdc.TDC_ETIMEOUT
    # the eigensolver's split merges report it the same way
    d, e = inputs.toeplitz_tridiag(8192)
    dt, et = torch.tensor(d, device=DEV), torch.tensor(e, device=DEV)
    oe = tdc.default_opts(leaf=64, merge_mode=tdc.MERGE_SPLIT, spin_budget=1)
    wse = tdc.workspace(tdc.workspace_size(8192, oe), DEV)
    tdc.eig(dt, et, oe, ws=wse)
    assert tdc.sync_status() == tdc.TDC_ETIMEOUT
    # then: clean calls, checked against the oracle
    Kc, mc = 1024, 300
    Dn, on, tn, zn, sn = generators(orc, Kc, 91)
    An = orthogonal_rows(orc, mc, Kc, 92)
    Co = orc.gemm(An, orc.qhat(Dn, on, tn, zn, sn))
    C = run_cauchy(tdc, An, Dn, on, tn, zn, sn, tdc.MERGE_SPLIT)
    assert np.max(np.abs(C - Co)) <= 1e-14 * np.sqrt(Kc)
    d1, e1 = inputs.uniform_tridiag(1024, 93)
    lam, Q = tdc.eig(torch.tensor(d1, device=DEV), torch.tensor(e1, device=DEV), tdc.default_opts(leaf=32), check=True)
    lo, Qo = orc.eig(d1, e1, leaf=32)
    lam, Q = lam.cpu().numpy(), Q.cpu().numpy()
    nT = max(abs(lo[0]), abs(lo[-1]))
    assert np.max(np.abs(lam - lo)) <= 1e-12 * nT
    res, orth = ratios(d1, e1, lam, Q)
    assert res <= 50 and orth <= 50
    compare_vectors(Q, Qo, lo, 1e-8 * nT, 1e-9)


def test_status_slots_of_calls_on_two_streams_stay_apart(tdc):
    """Each stream has its own status slot: a timeout on one stream is not reported for,
    or cleared by, a clean call on another stream, and it outlives the call's workspace."""
    K = 8192
    g = torch.Generator(device=DEV)
    g.manual_seed(12)
    D = torch.sort(torch.rand(K, dtype=torch.float64, device=DEV, generator=g) * 2 - 1).values
    z = torch.rand(K, dtype=torch.float64, device=DEV, generator=g) * 2 - 1
    z /= torch.linalg.norm(z)
    org, tau, zh, s = tdc.rank_one(D, z, 0.9, check=True)
    A = ((torch.rand(K, K, dtype=torch.float64, device=DEV, generator=g) * 2 - 1) / np.sqrt(K)).t()
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    o1 = tdc.default_opts(spin_budget=1)
    ws1 = tdc.workspace(tdc.cauchy_gemm_workspace_size(K, K, tdc.MERGE_SPLIT, o1), DEV)
    d, e = inputs.uniform_tridiag(500, 94)
    dt, et = torch.tensor(d, device=DEV), torch.tensor(e, device=DEV)
    o2 = tdc.default_opts(leaf=32)
    ws2 = tdc.workspace(tdc.workspace_size(500, o2), DEV)
    torch.cuda.synchronize()
    with torch.cuda.stream(s1):
        tdc.cauchy_gemm(A, D, org, tau, zh, s, tdc.MERGE_SPLIT, o1, stream=s1, ws=ws1)
    with torch.cuda.stream(s2):
        tdc.eig(dt, et, o2, ws=ws2, stream=s2)
    torch.cuda.synchronize()
    del ws1, ws2
    torch.cuda.empty_cache()  # the workspaces are gone; the statuses are not
    assert tdc.sync_status(s2) == 0
    assert tdc.sync_status(s1) == tdc.TDC_ETIMEOUT
    assert tdc.sync_status(s1) == 0  # read and cleared
