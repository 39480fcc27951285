"""Plain FP64 CPU oracle for the structured divide-and-conquer eigensolver.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The CUDA product path never imports it and shares no code with it.

The arithmetic lives in ``tdc_oracle.c`` (plain C, optional OpenMP), compiled
by :func:`build` into ``liboracle.so`` next to this file and called through
ctypes with numpy arrays.  ``adjoint.py`` and ``srrsc.py`` hold the numpy
oracles of the adjoint and of the SRRSC low-rank approximation; ``householder.py``
the Householder reduction of a dense symmetric matrix to tridiagonal form and its
back-transform; ``bidiag.py`` the bidiagonal SVD read off the Golub-Kahan tridiagonal;
``structured.py`` products with Toeplitz and Hankel operands written out from their
generators; ``banded.py`` the symmetric band eigenproblem from LAPACK's lower band
storage.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tdc_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

MAX_LEVELS = 48


class Stats(ctypes.Structure):
    _fields_ = [
        ("levels", ctypes.c_int),
        ("n_merges", ctypes.c_int64 * MAX_LEVELS),
        ("sum_n", ctypes.c_int64 * MAX_LEVELS),
        ("sum_K", ctypes.c_int64 * MAX_LEVELS),
        ("max_K", ctypes.c_int64 * MAX_LEVELS),
        ("type1", ctypes.c_int64 * MAX_LEVELS),
        ("type2", ctypes.c_int64 * MAX_LEVELS),
        ("secular_iter_max", ctypes.c_int64),
        ("secular_iter_sum", ctypes.c_int64),
        ("secular_roots", ctypes.c_int64),
        ("secular_noconv", ctypes.c_int64),
        ("leaf_noconv", ctypes.c_int64),
    ]

    def as_dict(self):
        L = self.levels
        return {
            "levels": L,
            "n_merges": list(self.n_merges[:L]),
            "sum_n": list(self.sum_n[:L]),
            "sum_K": list(self.sum_K[:L]),
            "max_K": list(self.max_K[:L]),
            "type1": list(self.type1[:L]),
            "type2": list(self.type2[:L]),
            "secular_iter_max": self.secular_iter_max,
            "secular_iter_mean": self.secular_iter_sum / max(1, self.secular_roots),
            "secular_noconv": self.secular_noconv,
            "leaf_noconv": self.leaf_noconv,
        }


def build(force: bool = False) -> str:
    """Compile the C oracle (gcc, -O2, OpenMP) into ``liboracle.so``."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".%d.tmp" % os.getpid()
        cmd = ["gcc", "-O2", "-fno-fast-math", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
               "-std=c99", "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    _lib = _bind(ctypes.CDLL(_LIB))
    return _lib


def _bind(lib):
    """Declare the C signatures on a loaded copy of the oracle library (the tests
    also bind copies built from the source with a planted mistake)."""
    P = ctypes.c_void_p
    i64 = ctypes.c_int64
    ci = ctypes.c_int
    cd = ctypes.c_double
    lib.orc_set_threads.argtypes = [ci]
    lib.orc_get_threads.restype = ci
    lib.orc_tree_depth.argtypes = [i64, i64]
    lib.orc_tree_depth.restype = ci
    lib.orc_leaf_qr.argtypes = [ci, P, P, P, i64]
    lib.orc_leaf_qr.restype = ci
    lib.orc_secular_root.argtypes = [ci, P, P, cd, ci, ci, P, P]
    lib.orc_secular_root.restype = ci
    lib.orc_secular.argtypes = [ci, P, P, cd, ci, P, P, P]
    lib.orc_secular.restype = ci
    lib.orc_lowner.argtypes = [ci, P, P, cd, P, P, P]
    lib.orc_colnorm.argtypes = [ci, P, P, P, P, P]
    lib.orc_qhat.argtypes = [ci, P, P, P, P, P, P, i64]
    lib.orc_deflate.argtypes = [ci, P, P, P, cd, P, i64, P, P, P, P]
    lib.orc_deflate.restype = ci
    lib.orc_merge.argtypes = [ci, ci, cd, P, P, i64, ci, P, ci]
    lib.orc_merge.restype = ci
    lib.orc_eig.argtypes = [ci, P, P, ci, ci, P, P, i64, P]
    lib.orc_eig.restype = ci
    lib.orc_sign_normalise.argtypes = [ci, P, i64]
    lib.orc_gemm.argtypes = [ci, ci, ci, P, i64, P, i64, P, i64]
    return lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def set_threads(t: int) -> None:
    _load().orc_set_threads(int(t))


def get_threads() -> int:
    return int(_load().orc_get_threads())


def tree_depth(n: int, leaf: int) -> int:
    return int(_load().orc_tree_depth(n, leaf))


def leaf_qr(d, e):
    """Implicit-shift QR on a small tridiagonal: returns (lam ascending, Q, status)."""
    d = _f64(d).copy()
    e = _f64(e).copy()
    n = d.size
    Q = np.zeros((n, n), dtype=np.float64, order="F")
    s = _load().orc_leaf_qr(n, _p(d), _p(e), _p(Q), max(n, 1))
    return d, Q, s


def secular(D, z, rho, max_iter=200):
    """All K roots of 1 + rho sum z_i^2/(d_i - lam): returns (org, tau, lam, max_iter_used)."""
    D = _f64(D)
    z = _f64(z)
    K = D.size
    org = np.zeros(K, dtype=np.int32)
    tau = np.zeros(K, dtype=np.float64)
    isum = ctypes.c_int64(0)
    it = _load().orc_secular(K, _p(D), _p(z), float(rho), max_iter, _p(org), _p(tau), ctypes.byref(isum))
    lam = D[org] + tau
    return org, tau, lam, it


def lowner(D, z, rho, org, tau):
    D = _f64(D)
    z = _f64(z)
    org = np.ascontiguousarray(org, dtype=np.int32)
    tau = _f64(tau)
    K = D.size
    zh = np.zeros(K)
    _load().orc_lowner(K, _p(D), _p(z), float(rho), _p(org), _p(tau), _p(zh))
    return zh


def colnorm(D, org, tau, zhat):
    D = _f64(D)
    org = np.ascontiguousarray(org, dtype=np.int32)
    tau = _f64(tau)
    zhat = _f64(zhat)
    K = D.size
    s = np.zeros(K)
    _load().orc_colnorm(K, _p(D), _p(org), _p(tau), _p(zhat), _p(s))
    return s


def qhat(D, org, tau, zhat, s):
    D = _f64(D)
    org = np.ascontiguousarray(org, dtype=np.int32)
    tau = _f64(tau)
    zhat = _f64(zhat)
    s = _f64(s)
    K = D.size
    U = np.zeros((K, K), order="F")
    _load().orc_qhat(K, _p(D), _p(org), _p(tau), _p(zhat), _p(s), _p(U), max(K, 1))
    return U


def deflate(D, z, rho, Q=None):
    """Deflation scan on (D, z) in merge-column order.  Returns
    (K, kept, defl, D_after, z_after, Q_after, n_type1, n_type2)."""
    D = _f64(D).copy()
    z = _f64(z).copy()
    n = D.size
    perm = np.argsort(D, kind="stable").astype(np.int32)
    if Q is None:
        Q = np.eye(n, order="F")
    Q = np.asfortranarray(Q, dtype=np.float64).copy(order="F")
    kept = np.zeros(n, dtype=np.int32)
    defl = np.zeros(n, dtype=np.int32)
    t1 = ctypes.c_int(0)
    t2 = ctypes.c_int(0)
    K = _load().orc_deflate(n, _p(D), _p(z), _p(perm), float(rho), _p(Q), max(n, 1), _p(kept), _p(defl),
                            ctypes.byref(t1), ctypes.byref(t2))
    return K, kept[:K].copy(), defl[: n - K].copy(), D, z, Q, t1.value, t2.value


def eig(d, e, leaf=32, max_iter=200, with_stats=False):
    """Full divide-and-conquer eigensolve T = Q diag(lam) Q^T (lam ascending)."""
    d = _f64(d)
    e = _f64(e)
    n = d.size
    lam = np.zeros(n)
    Q = np.zeros((n, n), order="F")
    st = Stats()
    status = _load().orc_eig(n, _p(d), _p(e), int(leaf), int(max_iter), _p(lam), _p(Q), max(n, 1),
                             ctypes.byref(st))
    if status != 0:
        raise RuntimeError("oracle eigensolve failed with status %d" % status)
    if with_stats:
        return lam, Q, st.as_dict()
    return lam, Q


def gemm(A, B):
    A = np.asfortranarray(A, dtype=np.float64)
    B = np.asfortranarray(B, dtype=np.float64)
    m, k = A.shape
    k2, n = B.shape
    assert k == k2
    C = np.zeros((m, n), order="F")
    _load().orc_gemm(m, n, k, _p(A), max(m, 1), _p(B), max(k, 1), _p(C), max(m, 1))
    return C
