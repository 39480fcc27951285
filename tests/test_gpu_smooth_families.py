"""Accuracy on matrices whose eigenvectors are smooth and deflate little: the
spherical-harmonic matrix of Example 3 at n = 16384 and the Hermite matrix of
Example 2 at n = 8192 (leaf 64), with the library's default merge (the structured
products on the split path for the large merges) and with the plain split product.

On such matrices the rows next to each split are nearly parallel to z, so the
split product's level-3 sums are secular-equation sums whose terms share their
sign over long runs of k.  Summed over a tile's whole reduction they exceed 2^24,
the range the FP32 level accumulators hold exactly (orthogonality ratio about 9e3
at n = 16384).  The default schedule drains the accumulators every 256 terms,
which keeps them far below it; the per-tile schedule (split_chunk_k = 0) is kept
as an option, and on this matrix its hand-offs must raise the TDC_WPRECISION
warning.  Ratios are taken on 256 sampled columns, as in the benchmark."""
import numpy as np
import pytest
import torch

from helpers import EPS, compare_vectors
from paper_2008_01990_gb300 import inputs

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
N = 16384


@pytest.fixture(scope="module")
def tdc():
    from paper_2008_01990_gb300 import build, tdc as t
    build.build()
    t.lib()
    return t


def sampled_ratios(dt, et, lam, Q, ns=256):
    """(||T q - lam q||_1 / (n ||T|| eps), ||Q^T q - e||_1 / (n eps)), max over sampled columns q."""
    n = dt.numel()
    g = np.random.default_rng(0)
    cols = torch.tensor(np.sort(g.choice(n, ns, replace=False)), device=DEV)
    Qs = Q[:, cols]
    Tq = dt[:, None] * Qs
    Tq[1:] += et[:, None] * Qs[:-1]
    Tq[:-1] += et[:, None] * Qs[1:]
    nT = max(abs(lam[0].item()), abs(lam[-1].item()))
    res = torch.abs(Tq - Qs * lam[cols]).sum(dim=0).max().item() / (n * nT * EPS)
    G = Qs.t() @ Q
    G[torch.arange(ns, device=DEV), cols] -= 1.0
    orth = torch.abs(G).sum(dim=1).max().item() / (n * EPS)
    return res, orth


def solve(tdc, mode, d, e, **kw):
    dt = torch.tensor(d, device=DEV)
    et = torch.tensor(e, device=DEV)
    o = tdc.default_opts(leaf=64, merge_mode=mode, collect_stats=1, **kw)
    lam, Q = tdc.eig(dt, et, o)
    st = tdc.sync_status()
    return dt, et, lam, Q, st, tdc.get_stats()


def test_sht_16384_fp64_merge(tdc):
    d, e = inputs.sht_tridiag(N)
    dt, et, lam, Q, st, _ = solve(tdc, tdc.MERGE_DENSE, d, e)
    assert st == 0
    assert torch.all(lam[1:] >= lam[:-1])
    # trace invariant: sum of the eigenvalues equals the trace
    nT = max(abs(lam[0].item()), abs(lam[-1].item()))
    assert abs(lam.sum().item() - dt.sum().item()) <= 1e-12 * N * nT
    res, orth = sampled_ratios(dt, et, lam, Q)
    assert res <= 50 and orth <= 50, (res, orth)


@pytest.mark.parametrize("mode", ["auto", "split"])
def test_sht_16384_split_path_default_schedule(tdc, mode):
    """The library's default merge (the structured products on the split path for the
    large merges) and the plain split product, both with the default drains."""
    d, e = inputs.sht_tridiag(N)
    dt, et, lam, Q, st, stats = solve(tdc, tdc.MERGE_AUTO if mode == "auto" else tdc.MERGE_SPLIT, d, e)
    assert st == 0, tdc.strerror(st)
    # every drained level sum stayed below half of the exact FP32 range
    assert 0 < stats["split_level_max"] < 0.5, stats["split_level_max"]
    res, orth = sampled_ratios(dt, et, lam, Q)
    assert res <= 50 and orth <= 50, (res, orth)


def test_sht_16384_per_tile_schedule_raises_the_precision_warning(tdc):
    """Summed over whole tiles of the plain split product the level sums pass 2^24 on this
    matrix: the guard must report it (the warning is the only sign of the inexact
    product)."""
    d, e = inputs.sht_tridiag(N)
    _, _, _, _, st, stats = solve(tdc, tdc.MERGE_SPLIT, d, e, split_chunk_k=0)
    assert st == tdc.TDC_WPRECISION, st
    assert stats["split_level_max"] >= 0.5


def test_chunked_drains_match_per_tile_schedule_on_random_data(tdc):
    """On random data both schedules are exact, so the products agree to rounding."""
    K = 4096
    g = torch.Generator(device=DEV)
    g.manual_seed(7)
    D = torch.sort(torch.rand(K, dtype=torch.float64, device=DEV, generator=g) * 2 - 1).values
    z = torch.rand(K, dtype=torch.float64, device=DEV, generator=g) * 2 - 1
    z /= torch.linalg.norm(z)
    org, tau, zh, s = tdc.rank_one(D, z, 0.9, check=True)
    A = ((torch.rand(K, K, dtype=torch.float64, device=DEV, generator=g) * 2 - 1) / np.sqrt(K)).t()
    C0 = tdc.cauchy_gemm(A, D, org, tau, zh, s, tdc.MERGE_SPLIT, tdc.default_opts(split_chunk_k=0), check=True)
    C1 = tdc.cauchy_gemm(A, D, org, tau, zh, s, tdc.MERGE_SPLIT, tdc.default_opts(split_chunk_k=256), check=True)
    assert torch.max(torch.abs(C0 - C1)).item() <= 1e-15


def test_hermite_8192_against_the_oracle(tdc, orc):
    """The smallest order at which the per-tile schedule's level sums were seen to pass
    2^24 (the Hermite top merge): the default schedule matches the oracle."""
    import os
    n = 8192
    d, e = inputs.hermite_tridiag(n)
    dt, et, lam, Q, st, _ = solve(tdc, tdc.MERGE_AUTO, d, e)
    assert st == 0, tdc.strerror(st)
    orc.set_threads(os.cpu_count() or 1)
    lam_o, Q_o = orc.eig(d, e, leaf=64)
    lam, Q = lam.cpu().numpy(), Q.cpu().numpy()
    nT = max(abs(lam_o[0]), abs(lam_o[-1]))
    assert np.max(np.abs(lam - lam_o)) <= 1e-12 * nT
    res, orth = sampled_ratios(dt, et, torch.tensor(lam, device=DEV), torch.tensor(Q, device=DEV))
    assert res <= 50 and orth <= 50, (res, orth)
    # eigenvectors up to sign against the oracle's (Hermite eigenvalues are well separated)
    compare_vectors(Q, Q_o, lam_o, 1e-8 * nT, 1e-9)
