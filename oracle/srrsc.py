"""Oracle for the structured low-rank approximation of Cauchy-like blocks (SRRSC).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Follows Section 2.1 of the paper step by step, in plain numpy FP64:
  * a Cauchy-like block A_ij = u_i v_j / (d_i - w_j) is described by its
    generators (row nodes d, column nodes w, vectors u, v);
  * Eq. (col-schur): the k-th Schur complement A^(k) is again Cauchy-like; its
    generators follow Theorem 1 / Corollary 1:
        u^(k)(i) = u^(k-1)(i) (d_i - d_k) / (d_i - w_k)
        v^(k)(j) = v^(k-1)(j) (w_j - w_k) / (w_j - d_k)
    where (d_k, w_k) are the nodes of the k-th pivot;
  * pivoting: complete pivoting on |A^(k)_ij| computed from the generators
    (ties broken towards the lowest row, then column) -- the paper allows complete
    pivoting and defers its own strategy to another reference;
  * stopping: when max |A^(k)| <= tol * max |A| the remaining Schur complement is
    neglected (the paper's "negligible");
  * Eq. (sid): A P ~= A(:, T) [I  Z], with Z from Theorem 2:
        y(i) = prod_{j != i} (d_j - w_i)/(w_j - w_i) * (d_i - w_i) / v^(0)(i)
        Z_ij = y(i) v^(r)(r+j) / (w_i - w_{r+j})
    (the paper's printed index of Eq. (geneZ) is garbled; this is the form that
    satisfies the displacement equation of Theorem 2).

Node differences are passed in as functions so that callers can form them from
the offset representation of Eq. (d-lambda) (rows are poles d_i, columns are
roots lambda_j = d_org(j) + tau_j).
"""
from __future__ import annotations

import numpy as np


class Nodes:
    """Row nodes (poles) and column nodes (roots as origin pole + offset)."""

    def __init__(self, d_row, d_org_col, tau_col):
        self.d = np.asarray(d_row, dtype=np.float64)
        self.wo = np.asarray(d_org_col, dtype=np.float64)
        self.wt = np.asarray(tau_col, dtype=np.float64)

    def dw(self, i, j):  # d_i - w_j
        return (self.d[i] - self.wo[j]) - self.wt[j]

    def dd(self, i, k):  # d_i - d_k
        return self.d[i] - self.d[k]

    def ww(self, j, k):  # w_j - w_k
        return (self.wo[j] - self.wo[k]) + (self.wt[j] - self.wt[k])

    def wd(self, j, k):  # w_j - d_k
        return (self.wo[j] - self.d[k]) + self.wt[j]


def dense_block(nodes: Nodes, u, v):
    mr, mc = len(u), len(v)
    A = np.empty((mr, mc))
    for i in range(mr):
        for j in range(mc):
            A[i, j] = u[i] * v[j] / nodes.dw(i, j)
    return A


def srrsc(nodes: Nodes, u0, v0, tol: float, max_rank: int | None = None):
    """Returns (r, piv_rows, piv_cols, rest_cols, Z) with
    A[:, piv_cols + rest_cols] ~= A[:, piv_cols] @ [I | Z]."""
    u = np.array(u0, dtype=np.float64)
    v = np.array(v0, dtype=np.float64)
    mr, mc = len(u), len(v)
    rows = list(range(mr))
    cols = list(range(mc))
    amax0 = np.max(np.abs(dense_block(nodes, u, v))) if mr and mc else 0.0
    kmax = min(mr, mc) if max_rank is None else min(mr, mc, max_rank)
    r = 0
    while r < kmax:
        # the r-th Schur complement from its generators; complete pivoting
        best, bi, bj = -1.0, -1, -1
        for a in range(r, mr):
            i = rows[a]
            for b in range(r, mc):
                j = cols[b]
                val = abs(u[i] * v[j] / nodes.dw(i, j))
                if val > best:
                    best, bi, bj = val, a, b
        if best <= tol * amax0:
            break
        rows[r], rows[bi] = rows[bi], rows[r]
        cols[r], cols[bj] = cols[bj], cols[r]
        pk, qk = rows[r], cols[r]
        # Theorem 1: generators of the next Schur complement
        for a in range(r + 1, mr):
            i = rows[a]
            u[i] *= nodes.dd(i, pk) / nodes.dw(i, qk)
        for b in range(r + 1, mc):
            j = cols[b]
            v[j] *= nodes.ww(j, qk) / nodes.wd(j, pk)
        r += 1
    piv_rows, piv_cols, rest = rows[:r], cols[:r], cols[r:]
    # Theorem 2: generators of Z
    y = np.empty(r)
    for a in range(r):
        ci, pi = piv_cols[a], piv_rows[a]
        p = nodes.dw(pi, ci) / v0[ci]
        for b in range(r):
            if b != a:
                p *= nodes.dw(piv_rows[b], ci) / nodes.ww(piv_cols[b], ci)
        y[a] = p
    Z = np.empty((r, len(rest)))
    for a in range(r):
        for b, j in enumerate(rest):
            Z[a, b] = y[a] * v[j] / nodes.ww(piv_cols[a], j)
    return r, piv_rows, piv_cols, rest, Z


def reconstruct(A, piv_cols, rest, Z):
    """A(:, T) [I | Z] put back into the original column order."""
    B = np.empty_like(A)
    B[:, piv_cols] = A[:, piv_cols]
    if len(rest):
        B[:, rest] = A[:, piv_cols] @ Z
    return B
