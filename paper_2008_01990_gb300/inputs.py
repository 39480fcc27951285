"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module holds no arithmetic of the eigensolver: it only draws numbers and
writes down the matrix families.  Random numbers come from SplitMix64
(Steele, Lea, Flood 2014): the state advances by 0x9E3779B97F4A7C15 and each
output is the standard 64-bit finaliser of the state; a uniform double in
[0,1) is (x >> 11) * 2^-53.

Matrix families (diagonal d[n], off-diagonal e[n-1]):
  * ``uniform``   d, e i.i.d. uniform(-1, 1)               (random matrices)
  * ``toeplitz``  d = 2, e = 1, tridiag(1,2,1)               (Example 2)
  * ``c4``        d uniform(0, 1), e = 1                     (few deflations)
  * ``clement``   d = 0, e_i = sqrt(i (n - i)), i = 1..n-1  (Example 2, Kac)
  * ``hermite``   d = 0, e_i = sqrt(i)                       (Example 2)
  * ``sht``       spherical-harmonic-transform matrix        (Example 3)

Dense symmetric families (``dense_sym``) for the reduction to tridiagonal form that
precedes the solver in Example 3 (whose SuiteSparse matrices are not available; these
stand in for them).
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


class SplitMix64:
    """Counter-style SplitMix64 stream; ``next_u64(k)`` returns the next k outputs."""

    def __init__(self, seed: int):
        self.state = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)

    def next_u64(self, k: int) -> np.ndarray:
        with np.errstate(over="ignore"):
            steps = np.arange(1, k + 1, dtype=np.uint64)
            x = self.state + steps * _GOLDEN
            self.state = self.state + np.uint64(k) * _GOLDEN
            x = (x ^ (x >> np.uint64(30))) * _M1
            x = (x ^ (x >> np.uint64(27))) * _M2
            x = x ^ (x >> np.uint64(31))
        return x

    def uniform01(self, k: int) -> np.ndarray:
        return (self.next_u64(k) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)

    def uniform(self, k: int, lo: float, hi: float) -> np.ndarray:
        return lo + (hi - lo) * self.uniform01(k)

    def normal(self, k: int) -> np.ndarray:
        """Box-Muller on pairs of uniforms (u1 in (0,1])."""
        m = (k + 1) // 2
        u1 = 1.0 - self.uniform01(m)
        u2 = self.uniform01(m)
        r = np.sqrt(-2.0 * np.log(u1))
        out = np.empty(2 * m)
        out[0::2] = r * np.cos(2.0 * np.pi * u2)
        out[1::2] = r * np.sin(2.0 * np.pi * u2)
        return out[:k]

    def integers(self, k: int, lo: int, hi: int) -> np.ndarray:
        """Uniform integers in [lo, hi] (inclusive) by scaling the 53-bit uniform."""
        span = hi - lo + 1
        return lo + np.minimum((self.uniform01(k) * span).astype(np.int64), span - 1)


def uniform_tridiag(n: int, seed: int):
    g = SplitMix64(seed)
    d = g.uniform(n, -1.0, 1.0)
    e = g.uniform(max(n - 1, 0), -1.0, 1.0)
    return d, e


def toeplitz_tridiag(n: int, diag: float = 2.0, off: float = 1.0):
    return np.full(n, diag), np.full(max(n - 1, 0), off)


def c4_tridiag(n: int, seed: int):
    g = SplitMix64(seed)
    return g.uniform(n, 0.0, 1.0), np.ones(max(n - 1, 0))


def clement_tridiag(n: int):
    i = np.arange(1, n, dtype=np.float64)
    return np.zeros(n), np.sqrt(i * (n - i))


def hermite_tridiag(n: int):
    return np.zeros(n), np.sqrt(np.arange(1, n, dtype=np.float64))


def sht_tridiag(n: int, m: int | None = None):
    """Example 3's spherical-harmonic-transform matrix (rows j = 0..n-1)."""
    if m is None:
        m = n
    def c(l):
        xi = l - m
        return np.sqrt((xi + 1.0) * (xi + 2.0) * (l + m + 1.0) * (l + m + 2.0)
                       / ((2.0 * l + 1.0) * (2.0 * l + 3.0) ** 2 * (2.0 * l + 5.0)))
    def dl(l):
        return (2.0 * l * (l + 1.0) - 2.0 * m * m - 1.0) / ((2.0 * l - 1.0) * (2.0 * l + 3.0))
    j = np.arange(n, dtype=np.float64)
    d = dl(m + 2.0 * j)
    e = c(m + 2.0 * j[:-1])
    return d, e


def batched_sizes(count: int, lo: int, hi: int, seed: int) -> np.ndarray:
    return SplitMix64(seed).integers(count, lo, hi)


def batched_uniform(sizes, seed: int):
    """Problem b draws d, e uniform(-1,1) from seed + b; returns concatenated (d, e)
    with the per-problem offsets (e of problem b has n_b - 1 entries but is stored
    in an n_b slot so that d and e share offsets)."""
    sizes = np.asarray(sizes, dtype=np.int64)
    offs = np.zeros(sizes.size + 1, dtype=np.int64)
    offs[1:] = np.cumsum(sizes)
    d = np.zeros(int(offs[-1]))
    e = np.zeros(int(offs[-1]))
    for b, nb in enumerate(sizes):
        db, eb = uniform_tridiag(int(nb), seed + b)
        d[offs[b]:offs[b] + nb] = db
        e[offs[b]:offs[b] + nb - 1] = eb
    return d, e, offs


def glued_wilkinson(n: int, m: int = 10, glue: float = 1e-10):
    """Copies of the Wilkinson matrix W+ of order 2m + 1 (d_i = |m - i|, e_i = 1) joined by
    off-diagonal entries `glue`, cut to order n: each eigenvalue of W+ appears once per copy
    to within about the glue, so the merges deflate long runs of nearly equal poles (chains
    of type-2 rotations)."""
    k = 2 * m + 1
    c = (n + k - 1) // k
    d = np.tile(np.abs(np.arange(k) - m).astype(np.float64), c)[:n]
    e = np.ones(max(c * k - 1, 0))
    e[k - 1::k] = glue
    return d, e[: max(n - 1, 0)]


def family(name: str, n: int, seed: int = 1):
    if name == "wilkinson":
        return glued_wilkinson(n)
    if name == "uniform":
        return uniform_tridiag(n, seed)
    if name == "toeplitz":
        return toeplitz_tridiag(n)
    if name == "c4":
        return c4_tridiag(n, seed)
    if name == "clement":
        return clement_tridiag(n)
    if name == "hermite":
        return hermite_tridiag(n)
    if name == "sht":
        return sht_tridiag(n)
    raise ValueError("unknown family %r" % name)


def backward_problems(count: int, n: int, seed: int, min_gap_rel: float = 1e-5, max_draws: int = 100000):
    """Problems for the adjoint workload: d, e uniform(-1,1), redrawn until the
    smallest eigenvalue gap is >= min_gap_rel * ||T||_2 (the gap is measured with
    scipy's tridiagonal eigenvalue routine, a library call, not this project's
    solver).  Also draws the loss weights w[n] and G[n, n] from N(0,1)."""
    from scipy.linalg import eigvalsh_tridiagonal

    g = SplitMix64(seed)
    ds, es, ws, Gs, gaps = [], [], [], [], []
    draws = 0
    while len(ds) < count:
        draws += 1
        if draws > max_draws:
            raise RuntimeError("could not draw %d well-separated problems" % count)
        d = g.uniform(n, -1.0, 1.0)
        e = g.uniform(n - 1, -1.0, 1.0)
        lam = eigvalsh_tridiagonal(d, e)
        nrm = max(abs(lam[0]), abs(lam[-1]))
        gap = float(np.min(np.diff(lam)))
        if gap >= min_gap_rel * nrm:
            ds.append(d)
            es.append(e)
            gaps.append(gap / nrm)
    for _ in range(count):
        ws.append(g.normal(n))
        Gs.append(g.normal(n * n).reshape(n, n, order="F"))
    return np.array(ds), np.array(es), np.array(ws), np.array(Gs), np.array(gaps), draws


def example1_cauchy(n: int, seed: int = 2020, a: float = 1.0, b: float = 9.0):
    """Generators of Example 1's Cauchy-like matrix B_ij = u_i v_j / (d_i - w_j):
    d_i = i (b - a) / n, w_j = d_j + (b - a) / (2 n) (i, j = 1..n), u and v uniform(0,1)
    from SplitMix64(seed)."""
    i = np.arange(1, n + 1, dtype=np.float64)
    d = i * (b - a) / n
    w = d + (b - a) / (2 * n)
    g = SplitMix64(seed)
    u = g.uniform01(n)
    v = g.uniform01(n)
    return d, w, u, v


def dense_sym(name: str, n: int, seed: int = 1) -> np.ndarray:
    """Dense symmetric n x n matrices (FP64, both triangles, C order):
      * ``uniform``  (X + X^T) / 2 with X i.i.d. uniform(-1, 1)
      * ``cluster``  I + 1e-8 (X + X^T) / 2          (eigenvalues clustered at 1)
      * ``lowrank``  2 I + u u^T + w w^T, u, w uniform(-1, 1) / sqrt(n)
                     (n - 2 eigenvalues equal to 2: after two reflectors the trailing
                     columns are zero up to rounding)
      * ``zerocol``  ``uniform`` with A(1:n, 0) = A(0, 1:n) = 0 (first reflector trivial)
      * ``tridiag``  the ``uniform`` tridiagonal family written densely (already reduced)"""
    g = SplitMix64(seed)
    if name == "tridiag":
        d, e = uniform_tridiag(n, seed)
        return np.diag(d) + np.diag(e, 1) + np.diag(e, -1)
    if name == "lowrank":
        u = g.uniform(n, -1.0, 1.0) / np.sqrt(max(n, 1))
        w = g.uniform(n, -1.0, 1.0) / np.sqrt(max(n, 1))
        return 2.0 * np.eye(n) + np.outer(u, u) + np.outer(w, w)
    X = g.uniform(n * n, -1.0, 1.0).reshape(n, n)
    A = 0.5 * (X + X.T)
    if name == "uniform":
        return A
    if name == "cluster":
        return np.eye(n) + 1e-8 * A
    if name == "zerocol":
        A[1:, 0] = 0.0
        A[0, 1:] = 0.0
        return A
    raise KeyError(name)


def bidiag_family(name: str, n: int, seed: int = 1):
    """Upper bidiagonal matrices (d[n], e[n-1]) for the SVD:
      * ``uniform``  |d| uniform(0.5, 1.5) with random signs, e uniform(-1, 1)
      * ``ones``     d = e = 1 (sigma_k = 2 cos(k pi / (2n + 1)), k = 1..n)
      * ``graded``   d_i = 2^(-20 i / n) times uniform(0.5, 1.5), e uniform(-1, 1) 2^(-20 i / n)"""
    if name == "ones":
        return np.ones(n), np.ones(max(n - 1, 0))
    g = SplitMix64(seed)
    mag = g.uniform(n, 0.5, 1.5)
    sgn = np.where(g.uniform01(n) < 0.5, -1.0, 1.0)
    e = g.uniform(max(n - 1, 0), -1.0, 1.0)
    if name == "uniform":
        return mag * sgn, e
    if name == "graded":
        s = 2.0 ** (-20.0 * np.arange(n) / max(n, 1))
        return mag * sgn * s, e * s[: max(n - 1, 0)]
    raise KeyError(name)


def band_sym(name: str, n: int, b: int, seed: int = 1) -> np.ndarray:
    """Symmetric band matrices of bandwidth b in lower band storage ((b + 1) x n,
    AB[r, j] = A(j + r, j), zero past the matrix):
      * ``uniform``  entries uniform(-1, 1)
      * ``laplace``  the 1-D operator with coupling to b neighbours: 2 b on the diagonal,
                     -1 on each of the b sub-diagonals (many close eigenvalues)
      * ``graded``   ``uniform`` with column j scaled by 2^(-10 j / n) on both sides"""
    AB = np.zeros((b + 1, n))
    if name == "laplace":
        AB[0, :] = 2.0 * b
        AB[1:, :] = -1.0
    else:
        g = SplitMix64(seed)
        AB[:, :] = g.uniform((b + 1) * n, -1.0, 1.0).reshape(b + 1, n)
        if name == "graded":
            sc = 2.0 ** (-10.0 * np.arange(n) / max(n, 1))
            for r in range(b + 1):
                AB[r, : n - r] *= sc[: n - r] * sc[r:]
        elif name != "uniform":
            raise KeyError(name)
    for r in range(1, b + 1):
        AB[r, max(n - r, 0):] = 0.0
    return AB
