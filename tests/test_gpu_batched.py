"""Batched eigensolves (tdc_eig_batched): replay under a CUDA graph, the autotuner,
and the full-size batched workload (4096 tridiagonals of orders uniform in
[64, 2048]) checked problem by problem on a sample against the oracle."""
import numpy as np
import pytest
import torch

from helpers import compare_vectors, ratios
from paper_2008_01990_gb300 import inputs

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def tdc():
    from paper_2008_01990_gb300 import build, tdc as t
    build.build()
    t.lib()
    return t


def batch(sizes, seed):
    d, e, offs = inputs.batched_uniform(sizes, seed)
    qoffs = np.concatenate([[0], np.cumsum(np.asarray(sizes, dtype=np.int64) ** 2)])
    return d, e, offs, qoffs


def test_graph_replay_matches_direct_call(tdc):
    sizes = inputs.batched_sizes(64, 64, 700, 31)
    d, e, offs, qoffs = batch(sizes, 31)
    d2, e2, _, _ = batch(sizes, 32)
    o = tdc.default_opts(leaf=32)
    dt = torch.tensor(d, device=DEV)
    et = torch.tensor(e, device=DEV)
    lam = torch.zeros(int(offs[-1]), dtype=torch.float64, device=DEV)
    Q = torch.zeros(int(qoffs[-1]), dtype=torch.float64, device=DEV)
    ws = tdc.workspace(tdc.batched_workspace_size(sizes, o), DEV)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        tdc.eig_batched(sizes, dt, et, offs[:-1], qoffs[:-1], lam, Q, o, ws=ws, stream=s)  # warm-up
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        tdc.eig_batched(sizes, dt, et, offs[:-1], qoffs[:-1], lam, Q, o, ws=ws, stream=s)
    for dd, ee in ((d, e), (d2, e2)):
        dt.copy_(torch.tensor(dd))
        et.copy_(torch.tensor(ee))
        g.replay()
        torch.cuda.synchronize()
        lam_g, Q_g = lam.cpu().numpy(), Q.cpu().numpy()
        lam_r, Q_r = tdc.eig_batched(sizes, torch.tensor(dd, device=DEV), torch.tensor(ee, device=DEV),
                                     offs[:-1], qoffs[:-1], torch.zeros_like(lam), torch.zeros_like(Q), o,
                                     check=True)
        assert np.array_equal(lam_g, lam_r.cpu().numpy())
        assert np.array_equal(Q_g, Q_r.cpu().numpy())
    assert tdc.sync_status() == 0


def test_nonfinite_problem_leaves_the_others_intact(tdc):
    """One problem of a batch with a NaN off-diagonal: the call reports TDC_ENONFINITE,
    that problem is solved with the entry read as zero, and the others are untouched."""
    from scipy.linalg import eigvalsh_tridiagonal
    sizes = [300, 500, 700]
    d, e, offs, qoffs = batch(sizes, 5)
    e[offs[1] + 123] = np.nan
    o = tdc.default_opts(leaf=16)
    lam = torch.zeros(int(offs[-1]), dtype=torch.float64, device=DEV)
    Q = torch.zeros(int(qoffs[-1]), dtype=torch.float64, device=DEV)
    tdc.eig_batched(sizes, torch.tensor(d, device=DEV), torch.tensor(e, device=DEV), offs[:-1], qoffs[:-1], lam, Q,
                    o)
    assert tdc.sync_status() == tdc.TDC_ENONFINITE
    e[offs[1] + 123] = 0.0
    lam, Q = lam.cpu().numpy(), Q.cpu().numpy()
    for i, n in enumerate(sizes):
        di, ei = d[offs[i]:offs[i] + n], e[offs[i]:offs[i] + n - 1]
        li = lam[offs[i]:offs[i] + n]
        Qi = Q[qoffs[i]:qoffs[i] + n * n].reshape(n, n).T
        ref = eigvalsh_tridiagonal(di, ei)
        assert np.max(np.abs(li - ref)) <= 50 * n * np.finfo(float).eps * np.max(np.abs(ref))
        res, orth = ratios(di, ei, li, Qi)
        assert res <= 50 and orth <= 50, (i, res, orth)
    assert tdc.sync_status() == 0


def test_each_problem_takes_its_own_scale(tdc):
    """A batch whose second problem is scaled by 2^700 and third by 2^-700: each problem
    is solved as the problem with its largest entry in [1, 2), so all three give the
    eigenvectors of those problems bit for bit and the eigenvalues scaled back exactly."""
    sizes = [300, 500, 700]
    d, e, offs, qoffs = batch(sizes, 9)
    for i in range(3):
        a, b = offs[i], offs[i] + sizes[i]
        m = np.frexp(max(np.abs(d[a:b]).max(), np.abs(e[a:b - 1]).max()))[1] - 1
        d[a:b], e[a:b - 1] = np.ldexp(d[a:b], -m), np.ldexp(e[a:b - 1], -m)
    ks = [0, 700, -700]
    ds, es = d.copy(), e.copy()
    for i, k in enumerate(ks):
        a, b = offs[i], offs[i] + sizes[i]
        ds[a:b], es[a:b - 1] = np.ldexp(d[a:b], k), np.ldexp(e[a:b - 1], k)
    o = tdc.default_opts(leaf=16)
    outs = []
    for dd, ee in ((d, e), (ds, es)):
        lam = torch.zeros(int(offs[-1]), dtype=torch.float64, device=DEV)
        Q = torch.zeros(int(qoffs[-1]), dtype=torch.float64, device=DEV)
        outs.append(tdc.eig_batched(sizes, torch.tensor(dd, device=DEV), torch.tensor(ee, device=DEV), offs[:-1],
                                    qoffs[:-1], lam, Q, o, check=True))
    (lam0, Q0), (lam1, Q1) = [(l.cpu().numpy(), q.cpu().numpy()) for l, q in outs]
    assert np.array_equal(Q0, Q1)
    for i, k in enumerate(ks):
        a, b = offs[i], offs[i] + sizes[i]
        assert np.array_equal(lam1[a:b], np.ldexp(lam0[a:b], k))


def test_autotuner_picks_and_caches(tdc, tmp_path):
    from paper_2008_01990_gb300 import autotune
    sizes = inputs.batched_sizes(48, 64, 600, 41)
    d, e, offs, qoffs = batch(sizes, 41)
    cache = str(tmp_path / "tune.json")
    o = autotune.tune_batched(sizes, torch.tensor(d, device=DEV), torch.tensor(e, device=DEV), offs[:-1],
                              sample=16, cache_path=cache)
    assert o.leaf in autotune.LEAVES and o.split_min_K in autotune.SPLIT_MIN_K
    o2 = autotune.tune_batched(sizes, None, None, None, cache_path=cache)  # served from the cache
    assert (o2.leaf, o2.split_min_K) == (o.leaf, o.split_min_K)


def test_single_problem_autotuner(tdc, orc, tmp_path):
    """Leaf size and split threshold timed on one matrix; the chosen options solve it
    to the oracle's accuracy and a second call is served from the cache."""
    from paper_2008_01990_gb300 import autotune
    n = 1500
    d, e = inputs.c4_tridiag(n, 4)
    dt, et = torch.tensor(d, device=DEV), torch.tensor(e, device=DEV)
    cache = str(tmp_path / "tune1.json")
    o = autotune.tune_single(dt, et, cache_path=cache, leaves=(16, 32), split_min_k=(64, 256))
    assert o.leaf in (16, 32) and o.split_min_K in (64, 256)
    o2 = autotune.tune_single(dt, et, cache_path=cache, leaves=(16, 32), split_min_k=(64, 256))
    assert (o2.leaf, o2.split_min_K) == (o.leaf, o.split_min_K)
    lam, Q = tdc.eig(dt, et, o, check=True)
    lo, _ = orc.eig(d, e, leaf=o.leaf)
    assert np.max(np.abs(lam.cpu().numpy() - lo)) <= 1e-12 * max(abs(lo[0]), abs(lo[-1]))


def test_c3_full_batch_sampled(tdc, orc):
    """4096 problems, n_b uniform in [64, 2048] (seed 3), d, e uniform(-1,1) (seed 3+b),
    one call; every eigenvalue sorted and finite, 64 problems spread over the size range
    (evenly spaced ranks of n_b, smallest and largest included) against the oracle."""
    sizes = inputs.batched_sizes(4096, 64, 2048, 3)
    d, e, offs, qoffs = batch(sizes, 3)
    o = tdc.default_opts(leaf=32)
    lam = torch.empty(int(offs[-1]), dtype=torch.float64, device=DEV)
    Q = torch.empty(int(qoffs[-1]), dtype=torch.float64, device=DEV)
    tdc.eig_batched(sizes, torch.tensor(d, device=DEV), torch.tensor(e, device=DEV), offs[:-1], qoffs[:-1],
                    lam, Q, o, check=True)
    lam_h = lam.cpu().numpy()
    assert np.all(np.isfinite(lam_h))
    for b in range(len(sizes)):
        lb = lam_h[offs[b]:offs[b] + sizes[b]]
        assert np.all(np.diff(lb) >= 0)
    import os
    orc.set_threads(os.cpu_count() or 1)
    order = np.argsort(sizes, kind="stable")
    pick = sorted(set(int(order[i]) for i in np.linspace(0, len(sizes) - 1, 64).round().astype(int)))
    assert len(pick) == 64 and sizes[pick].min() == sizes.min() and sizes[pick].max() == sizes.max()
    for b in pick:
        nb = int(sizes[b])
        db, eb = d[offs[b]:offs[b] + nb], e[offs[b]:offs[b] + nb - 1]
        lb = lam_h[offs[b]:offs[b] + nb]
        Qb = Q[int(qoffs[b]):int(qoffs[b]) + nb * nb].cpu().numpy().reshape(nb, nb, order="F")
        # the oracle bisects each root to the rounding level of |tau|, which can take a few
        # hundred halvings when a root lies very close to its pole
        lo, Qo = orc.eig(db, eb, leaf=32, max_iter=2000)
        nT = max(abs(lo[0]), abs(lo[-1]))
        assert np.max(np.abs(lb - lo)) <= 1e-12 * nT
        res, orth = ratios(db, eb, lb, Qb)
        assert res <= 50 and orth <= 50
        compare_vectors(Qb, Qo, lo, 1e-8 * nT, 1e-7)


@pytest.mark.parametrize("leaf,split_min_k", [(8, 16), (16, 32)])
def test_batched_tiny_merges_on_split_path(tdc, orc, leaf, split_min_k):
    """Merges down to K = 16 on the split path (a 128-row tile holding 8 or 16 rows)
    and small leaves: sampled problems against the oracle, test ratios on all of them."""
    sizes = inputs.batched_sizes(160, 64, 700, 53)
    d, e, offs, qoffs = batch(sizes, 53)
    o = tdc.default_opts(leaf=leaf)
    o.split_min_K = split_min_k
    lam = torch.empty(int(offs[-1]), dtype=torch.float64, device=DEV)
    Q = torch.empty(int(qoffs[-1]), dtype=torch.float64, device=DEV)
    tdc.eig_batched(sizes, torch.tensor(d, device=DEV), torch.tensor(e, device=DEV), offs[:-1], qoffs[:-1],
                    lam, Q, o, check=True)
    lam_h, Q_h = lam.cpu().numpy(), Q.cpu().numpy()
    for b in range(len(sizes)):
        nb = int(sizes[b])
        db, eb = d[offs[b]:offs[b] + nb], e[offs[b]:offs[b] + nb - 1]
        lb = lam_h[offs[b]:offs[b] + nb]
        Qb = Q_h[int(qoffs[b]):int(qoffs[b]) + nb * nb].reshape(nb, nb, order="F")
        res, orth = ratios(db, eb, lb, Qb)
        assert res <= 50 and orth <= 50, (b, res, orth)
        if b % 40 == 0:
            lo, Qo = orc.eig(db, eb, leaf=leaf)
            nT = max(abs(lo[0]), abs(lo[-1]))
            assert np.max(np.abs(lb - lo)) <= 1e-12 * nT
            compare_vectors(Qb, Qo, lo, 1e-8 * nT, 1e-7)
