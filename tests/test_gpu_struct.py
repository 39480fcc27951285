"""Structured (SRRSC low-rank) eigenvector update on the GPU against the oracle's
plain FP64 product, element by element, and the eigensolver with the structured
merge against the oracle."""
import numpy as np
import pytest
import torch

from helpers import check_toeplitz_sampled, compare_vectors, ratios
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


def run(tdc, A, D, org, tau, zh, s, mode, **kw):
    t = lambda x: torch.tensor(x, device=DEV)
    At = torch.tensor(np.ascontiguousarray(A.T), device=DEV).t()
    C = tdc.cauchy_gemm(At, t(D), torch.tensor(org, dtype=torch.int32, device=DEV), t(tau), t(zh), t(s), mode,
                        tdc.default_opts(**kw), check=True)
    return C.cpu().numpy()


@pytest.mark.parametrize("m,K,tile", [(300, 1000, 128), (513, 700, 64), (256, 2048, 256), (1, 640, 64)])
def test_cauchy_structured_vs_oracle(tdc, orc, m, K, tile):
    D, org, tau, zh, s = generators(orc, K, 50 + K)
    g = inputs.SplitMix64(m)
    A = g.uniform(m * K, -1.0, 1.0).reshape(m, K) / np.sqrt(K)
    Co = orc.gemm(A, orc.qhat(D, org, tau, zh, s))
    C = run(tdc, A, D, org, tau, zh, s, tdc.MERGE_STRUCTURED, lr_tile=tile, lr_tol=1e-15)
    assert np.max(np.abs(C - Co)) <= 1e-14 * np.sqrt(K)


def test_cauchy_structured_error_follows_tolerance(tdc, orc):
    m, K = 256, 1536
    D, org, tau, zh, s = generators(orc, K, 77)
    g = inputs.SplitMix64(9)
    A = g.uniform(m * K, -1.0, 1.0).reshape(m, K) / np.sqrt(K)
    Co = orc.gemm(A, orc.qhat(D, org, tau, zh, s))
    e6 = np.max(np.abs(run(tdc, A, D, org, tau, zh, s, tdc.MERGE_STRUCTURED, lr_tile=128, lr_tol=1e-6) - Co))
    e12 = np.max(np.abs(run(tdc, A, D, org, tau, zh, s, tdc.MERGE_STRUCTURED, lr_tile=128, lr_tol=1e-12) - Co))
    assert 1e-12 < e6 <= 1e-5       # the low-rank form is really used
    assert e12 <= 1e-10 and e12 < e6 / 100


def test_cauchy_structured_dense_fallback(tdc, orc):
    # a tolerance no pivot can meet: every far tile exceeds the rank cap and stays dense
    m, K = 200, 1024
    D, org, tau, zh, s = generators(orc, K, 78)
    g = inputs.SplitMix64(10)
    A = g.uniform(m * K, -1.0, 1.0).reshape(m, K) / np.sqrt(K)
    Co = orc.gemm(A, orc.qhat(D, org, tau, zh, s))
    C = run(tdc, A, D, org, tau, zh, s, tdc.MERGE_STRUCTURED, lr_tile=128, lr_tol=1e-300)
    assert np.max(np.abs(C - Co)) <= 1e-14 * np.sqrt(K)


@pytest.mark.parametrize("n,leaf,fam", [(2048, 64, "toeplitz"), (1500, 32, "c4"), (1024, 32, "uniform"),
                                        (901, 16, "clement")])
def test_eig_structured_merge_vs_oracle(tdc, orc, n, leaf, fam):
    d, e = inputs.family(fam, n, 1)
    o = tdc.default_opts(leaf=leaf, merge_mode=tdc.MERGE_STRUCTURED, structured_min_K=256, lr_tile=128)
    lam, Q = tdc.eig(torch.tensor(d, device=DEV), torch.tensor(e, device=DEV), o, check=True)
    lam, Q = lam.cpu().numpy(), Q.cpu().numpy()
    lam_o, Q_o = orc.eig(d, e, leaf=leaf)
    nT = max(abs(lam_o[0]), abs(lam_o[-1]))
    assert np.max(np.abs(lam - lam_o)) <= 1e-12 * nT
    res, orth = ratios(d, e, lam, Q)
    assert res <= 50 and orth <= 50, (res, orth)
    compare_vectors(Q, Q_o, lam_o, 1e-8 * nT, 1e-7)


def test_c2_toeplitz_16384_structured_default_tiles(tdc):
    """The structured merge at full size with the library's defaults (lr_tile 256,
    structured_min_K 4096, rank cap 64, lr_tol 1e-15): the top merge of tridiag(1,2,1)
    at n = 16384 (K = 8192 non-deflated poles) runs on the structured path.  Closed-form
    eigenvalues, sampled residual, orthogonality and sine vectors; every far tile is
    compressed (ranks from the statistics)."""
    n = 16384
    d, e = inputs.toeplitz_tridiag(n)
    o = tdc.default_opts(leaf=64, merge_mode=tdc.MERGE_STRUCTURED, collect_stats=1)
    assert (o.lr_tile, o.structured_min_K) == (256, 4096)
    lam, Q = tdc.eig(torch.tensor(d, device=DEV), torch.tensor(e, device=DEV), o, check=True)
    st = tdc.get_stats()
    assert st["sum_K"][0] == n // 2
    # top merge: 32 x 32 tiles of 256 poles and roots, all but the 94 on or next to the
    # diagonal compressed, in both halves' products (the level below adds its own)
    assert st["lr_tiles"] >= 2 * (32 * 32 - 94)
    assert st["lr_dense_fallbacks"] == 0 and 0 < st["lr_rank_max"] <= 64
    assert st["struct_flops"] > 0
    check_toeplitz_sampled(lam, Q, n)


# --- the structured update with every product on the split tensor-core GEMM ---

@pytest.mark.parametrize("m,K,tile", [(300, 1000, 128), (513, 700, 64), (256, 2048, 256), (1, 640, 64),
                                      (1000, 3000, 512)])
def test_cauchy_structured_split_vs_oracle(tdc, orc, m, K, tile):
    """C = A Qhat with the near-diagonal tiles, the W products and the applications
    W_J R_J on the split path, element by element against the oracle's FP64 product."""
    D, org, tau, zh, s = generators(orc, K, 60 + K)
    g = inputs.SplitMix64(m + 7)
    A = g.uniform(m * K, -1.0, 1.0).reshape(m, K) / np.sqrt(K)
    Co = orc.gemm(A, orc.qhat(D, org, tau, zh, s))
    C = run(tdc, A, D, org, tau, zh, s, tdc.MERGE_STRUCTURED_SPLIT, lr_tile=tile, lr_tol=1e-15)
    assert np.max(np.abs(C - Co)) <= 1e-14 * np.sqrt(K)


@pytest.mark.parametrize("tile", [64, 128])
def test_cauchy_structured_split_dense_fallbacks(tdc, orc, tile):
    """lr_tol = 1e-300 keeps every far tile at full rank: with 128-wide tiles SRRSC passes
    the rank cap (64); with 64-wide tiles every tile keeps rank 64, more low-rank columns
    than the W buffer's budget.  Either way the structured path leaves the part to the
    plain split product, and the product equals the oracle's."""
    m, K = 200, 1500
    D, org, tau, zh, s = generators(orc, K, 61)
    g = inputs.SplitMix64(62)
    A = g.uniform(m * K, -1.0, 1.0).reshape(m, K) / np.sqrt(K)
    Co = orc.gemm(A, orc.qhat(D, org, tau, zh, s))
    C = run(tdc, A, D, org, tau, zh, s, tdc.MERGE_STRUCTURED_SPLIT, lr_tile=tile, lr_tol=1e-300)
    assert np.max(np.abs(C - Co)) <= 1e-14 * np.sqrt(K)


@pytest.mark.parametrize("n,leaf,fam", [(2048, 64, "toeplitz"), (1500, 32, "c4"), (1024, 32, "uniform"),
                                        (901, 16, "clement"), (3000, 64, "sht")])
def test_eig_structured_split_merge_vs_oracle(tdc, orc, n, leaf, fam):
    d, e = inputs.family(fam, n, 1)
    o = tdc.default_opts(leaf=leaf, merge_mode=tdc.MERGE_STRUCTURED_SPLIT, structured_min_K=256, lr_tile=128,
                         collect_stats=1)
    lam, Q = tdc.eig(torch.tensor(d, device=DEV), torch.tensor(e, device=DEV), o, check=True)
    st = tdc.get_stats()
    lam, Q = lam.cpu().numpy(), Q.cpu().numpy()
    lam_o, Q_o = orc.eig(d, e, leaf=leaf)
    nT = max(abs(lam_o[0]), abs(lam_o[-1]))
    assert np.max(np.abs(lam - lam_o)) <= 1e-12 * nT
    res, orth = ratios(d, e, lam, Q)
    assert res <= 50 and orth <= 50, (res, orth)
    compare_vectors(Q, Q_o, lam_o, 1e-8 * nT, 1e-7)
    if st["sum_K"][0] >= 256 + 2 * 128:  # a top merge with far tiles took the structured path
        assert st["lr_tiles"] > 0 and st["split_flops"] > 0 and st["lr_parts_structured"] > 0


def test_c2_toeplitz_16384_structured_split_default_tiles(tdc):
    """The structured merge on the tensor cores at full size with the library's defaults:
    closed-form eigenvalues, sampled residual, orthogonality and sine vectors."""
    n = 16384
    d, e = inputs.toeplitz_tridiag(n)
    o = tdc.default_opts(leaf=64, merge_mode=tdc.MERGE_STRUCTURED_SPLIT, collect_stats=1)
    lam, Q = tdc.eig(torch.tensor(d, device=DEV), torch.tensor(e, device=DEV), o, check=True)
    st = tdc.get_stats()
    assert st["lr_tiles"] >= 2 * (32 * 32 - 94) and st["lr_dense_fallbacks"] == 0
    assert st["lr_parts_split"] == 0 and st["lr_parts_structured"] >= 2
    assert 0 < st["split_level_max"] < 0.5
    check_toeplitz_sampled(lam, Q, n)
