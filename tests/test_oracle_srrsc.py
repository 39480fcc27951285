"""Pins of the SRRSC oracle (oracle/srrsc.py, Section 2.1) against facts fixed
outside it: the explicit Schur complement (Eq. (col-schur), Theorem 1), the
explicit A11^{-1} A12 (Theorem 2 / Eq. (sid)) on well-conditioned cases, SVD
numerical ranks, the reconstruction error at the stopping tolerance, and the
rank pattern of the paper's Table 2 (semi-pinned: the paper gives no tolerance)."""
import os

import numpy as np
import pytest

from oracle.srrsc import Nodes, dense_block, reconstruct, srrsc
from paper_2008_01990_gb300 import inputs

HERE = os.path.dirname(os.path.abspath(__file__))


def qhat_block(orc, K, seed, rows, cols):
    g = inputs.SplitMix64(seed)
    D = np.sort(g.uniform(K, -1, 1))
    z = g.uniform(K, -1, 1)
    z /= np.linalg.norm(z)
    org, tau, _, _ = orc.secular(D, z, 0.8)
    zh = orc.lowner(D, z, 0.8, org, tau)
    s = orc.colnorm(D, org, tau, zh)
    U = orc.qhat(D, org, tau, zh, s)
    nodes = Nodes(D[rows], D[org[cols]], tau[cols])
    return nodes, zh[rows], s[cols], U[np.ix_(rows, cols)]


def test_block_from_generators_is_qhat(orc):
    nodes, u, v, Ub = qhat_block(orc, 400, 1, np.arange(0, 64), np.arange(200, 280))
    assert np.array_equal(dense_block(nodes, u, v), Ub)


def test_schur_complement_generators_theorem1(orc):
    # after r pivots the generators give exactly the explicit Schur complement
    nodes, u, v, A = qhat_block(orc, 300, 2, np.arange(0, 40), np.arange(120, 170))
    r, pr, pc, rest, Z = srrsc(nodes, u, v, tol=1e-13, max_rank=3)
    assert r == 3
    rows_rest = [i for i in range(A.shape[0]) if i not in pr]
    A11 = A[np.ix_(pr, pc)]
    S = A[np.ix_(rows_rest, rest)] - A[np.ix_(rows_rest, pc)] @ np.linalg.solve(A11, A[np.ix_(pr, rest)])
    # rerun the generator recursion to read the Schur complement generators
    u2 = np.array(u, dtype=float)
    v2 = np.array(v, dtype=float)
    for k in range(3):
        pk, qk = pr[k], pc[k]
        for i in range(len(u2)):
            if i not in pr[:k + 1]:
                u2[i] *= nodes.dd(i, pk) / nodes.dw(i, qk)
        for j in range(len(v2)):
            if j not in pc[:k + 1]:
                v2[j] *= nodes.ww(j, qk) / nodes.wd(j, pk)
    Sg = np.array([[u2[i] * v2[j] / nodes.dw(i, j) for j in rest] for i in rows_rest])
    assert np.max(np.abs(Sg - S)) <= 1e-12 * np.max(np.abs(A))


def test_z_equals_a11_inverse_a12_theorem2(orc):
    nodes, u, v, A = qhat_block(orc, 300, 3, np.arange(0, 48), np.arange(150, 200))
    r, pr, pc, rest, Z = srrsc(nodes, u, v, tol=1e-4)
    assert 1 <= r <= 6
    Zs = np.linalg.solve(A[np.ix_(pr, pc)], A[np.ix_(pr, rest)])
    assert np.max(np.abs(Z - Zs)) <= 1e-8 * max(1.0, np.max(np.abs(Zs)))


@pytest.mark.parametrize("tol", [1e-6, 1e-10, 1e-14])
def test_reconstruction_and_rank(orc, tol):
    nodes, u, v, A = qhat_block(orc, 1024, 4, np.arange(0, 128), np.arange(512, 640))
    r, pr, pc, rest, Z = srrsc(nodes, u, v, tol)
    B = reconstruct(A, pc, rest, Z)
    amax = np.max(np.abs(A))
    assert np.max(np.abs(A - B)) <= 20 * tol * amax * np.sqrt(A.shape[0])
    sv = np.linalg.svd(A, compute_uv=False)
    nr = int(np.sum(sv > tol * sv[0]))
    assert abs(r - nr) <= 2


def test_table2_rank_pattern_semi_pinned():
    """Example 1 matrix at n = 2048 in 4 x 4 blocks of 512 (block layout): the ranks of
    B(2,1), B(3,1), B(4,1) fall off with the distance from the diagonal as in the last
    row of Table 2 (34, 11, 9), the adjacent block clearly the largest."""
    rows = [l.split() for l in open(os.path.join(HERE, "golden", "table2_offdiag_ranks.txt"))
            if l.strip() and not l.startswith("#")]
    paper = {int(r[0]): [int(x) for x in r[1:]] for r in rows}
    p21, p31, p41 = paper[4096]
    n, a, b = 2048, 1.0, 9.0
    i = np.arange(1, n + 1)
    d = i * (b - a) / n
    w = d + (b - a) / (2 * n)
    g = inputs.SplitMix64(2020)
    u = g.uniform01(n)
    v = g.uniform01(n)
    m = 512
    ranks = []
    for I in (1, 2, 3):
        rr = np.arange(I * m, (I + 1) * m)
        cc = np.arange(0, m)
        r, *_ = srrsc(Nodes(d[rr], w[cc], np.zeros(m)), u[rr], v[cc], 1e-12)
        ranks.append(r)
    r21, r31, r41 = ranks
    assert p21 > p31 >= p41 and r21 > r31 >= r41
    assert r21 >= 1.5 * r31 and p21 >= 1.5 * p31
    # the cyclic layouts of Table 2 give far higher ranks than the block layout
    assert min(paper[64]) > 10 * max(paper[4096])
