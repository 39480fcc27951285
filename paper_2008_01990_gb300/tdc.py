"""Thin ctypes binding of ``libtdc.so`` (declared in ``include/tdc.h``).

Argument marshalling only: every step of the eigensolver runs in the CUDA
library.  PyTorch provides device memory and the current stream.  Loading
fails loudly when the library has not been built -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import warnings

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtdc.so")
_lib = None

TDC_OK = 0
TDC_ENOWS = -101
TDC_ENONFINITE = -102
TDC_ENOCONV = -103
TDC_ETIMEOUT = -104
TDC_ECUDA = -105
TDC_EUNSUPPORTED = -106
TDC_ETOOLARGE = -107
TDC_WPRECISION = 1

MERGE_AUTO = 0
MERGE_DENSE = 1
MERGE_STRUCTURED = 2
MERGE_SPLIT = 3
MERGE_STRUCTURED_SPLIT = 4

MAX_LEVELS = 32


class Opts(ctypes.Structure):
    _fields_ = [
        ("leaf", ctypes.c_int32),
        ("merge_mode", ctypes.c_int32),
        ("structured_min_K", ctypes.c_int32),
        ("lr_tile", ctypes.c_int32),
        ("lr_tol", ctypes.c_double),
        ("split_slices", ctypes.c_int32),
        ("split_min_K", ctypes.c_int32),
        ("max_iter", ctypes.c_int32),
        ("sign_normalise", ctypes.c_int32),
        ("collect_stats", ctypes.c_int32),
        ("spin_budget", ctypes.c_int64),
        ("split_chunk_k", ctypes.c_int32),
    ]


class Stats(ctypes.Structure):
    _fields_ = [
        ("levels", ctypes.c_int32),
        ("n_merges", ctypes.c_int64 * MAX_LEVELS),
        ("sum_n", ctypes.c_int64 * MAX_LEVELS),
        ("sum_K", ctypes.c_int64 * MAX_LEVELS),
        ("max_K", ctypes.c_int64 * MAX_LEVELS),
        ("n_rot", ctypes.c_int64 * MAX_LEVELS),
        ("n_type1", ctypes.c_int64 * MAX_LEVELS),
        ("secular_iter_max", ctypes.c_int64),
        ("secular_iter_mean", ctypes.c_double),
        ("phase_ms", ctypes.c_float * 12),
        ("gemm_flops", ctypes.c_double * MAX_LEVELS),
        ("split_flops", ctypes.c_double),
        ("split_bytes", ctypes.c_double),
        ("struct_flops", ctypes.c_double),
        ("launches", ctypes.c_int64),
        ("secular_handoffs", ctypes.c_int64),
        ("split_level_max", ctypes.c_float),
        ("lr_tiles", ctypes.c_int64),
        ("lr_rank_sum", ctypes.c_int64),
        ("lr_dense_fallbacks", ctypes.c_int64),
        ("lr_rank_max", ctypes.c_int64),
        ("lr_parts_structured", ctypes.c_int64),
        ("lr_parts_split", ctypes.c_int64),
    ]

    def as_dict(self):
        L = self.levels
        names = ["leaf", "prepare", "secular", "zhat_norms_order", "gemm_fp64", "split_digits", "split_mma",
                 "copy", "output", "total"]
        return {
            "levels": L,
            "n_merges": list(self.n_merges[:L]),
            "sum_n": list(self.sum_n[:L]),
            "sum_K": list(self.sum_K[:L]),
            "max_K": list(self.max_K[:L]),
            "type2": list(self.n_rot[:L]),
            "type1": list(self.n_type1[:L]),
            "secular_iter_max": self.secular_iter_max,
            "secular_iter_mean": self.secular_iter_mean,
            "phase_ms": dict(zip(names, list(self.phase_ms))),
            "gemm_flops": list(self.gemm_flops[:L]),
            "split_flops": self.split_flops,
            "split_bytes": self.split_bytes,
            "struct_flops": self.struct_flops,
            "launches": self.launches,
            "secular_handoffs": self.secular_handoffs,
            "split_level_max": self.split_level_max,
            "lr_tiles": self.lr_tiles,
            "lr_rank_sum": self.lr_rank_sum,
            "lr_dense_fallbacks": self.lr_dense_fallbacks,
            "lr_rank_max": self.lr_rank_max,
            "lr_parts_structured": self.lr_parts_structured,
            "lr_parts_split": self.lr_parts_split,
        }


class TdcPrecisionWarning(RuntimeWarning):
    """The device status of a call was TDC_WPRECISION: a split-path level sum reached half of
    its exact FP32 range, so the eigenvectors may miss the FP64 accuracy bound."""


class TdcError(RuntimeError):
    def __init__(self, fn, status):
        self.status = status
        msg = lib().tdc_strerror(status).decode() if status != 0 else "ok"
        super().__init__("%s failed: status %d (%s)" % (fn, status, msg))


def lib():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libtdc.so is not built (run __graft_entry__.build() or python -m "
                           "paper_2008_01990_gb300.build); there is no CPU fallback")
    L = ctypes.CDLL(LIB_PATH)
    P = ctypes.c_void_p
    i64, i32, sz = ctypes.c_int64, ctypes.c_int32, ctypes.c_size_t
    L.tdc_default_opts.argtypes = [ctypes.POINTER(Opts)]
    L.tdc_default_opts.restype = None
    L.tdc_workspace_size.argtypes = [i64, ctypes.POINTER(Opts), ctypes.POINTER(sz)]
    L.tdc_eig.argtypes = [i64, P, P, P, P, i64, P, sz, ctypes.POINTER(Opts), P]
    L.tdc_eig_batched_workspace_size.argtypes = [i32, P, ctypes.POINTER(Opts), ctypes.POINTER(sz)]
    L.tdc_eig_batched.argtypes = [i32, P, P, P, P, P, P, P, P, sz, ctypes.POINTER(Opts), P]
    L.tdc_sync_status.argtypes = [P]
    L.tdc_get_stats.argtypes = [ctypes.POINTER(Stats)]
    L.tdc_strerror.argtypes = [ctypes.c_int]
    L.tdc_strerror.restype = ctypes.c_char_p
    if hasattr(L, "tdc_backward_workspace_size"):
        L.tdc_backward_workspace_size.argtypes = [i64, ctypes.POINTER(sz)]
        L.tdc_eig_backward.argtypes = [i64, P, P, i64, P, P, P, P, P, sz, P]
        L.tdc_backward_batched_workspace_size.argtypes = [i32, i64, ctypes.POINTER(sz)]
        L.tdc_eig_backward_batched.argtypes = [i32, i64, P, P, P, P, P, P, P, sz, P]
    if hasattr(L, "tdc_eig_noalloc"):
        L.tdc_eig_noalloc.argtypes = [i64, P, P, P, P, i64, ctypes.POINTER(Opts), P]
    if hasattr(L, "tdc_rank_one"):
        L.tdc_rank_one_workspace_size.argtypes = [i64, ctypes.POINTER(sz)]
        L.tdc_rank_one.argtypes = [i64, P, P, ctypes.c_double, P, P, P, P, i32, P, sz, P]
    if hasattr(L, "tdc_cauchy_like_gemm"):
        L.tdc_cauchy_like_gemm_workspace_size.argtypes = [i64, i64, i32, ctypes.POINTER(Opts), ctypes.POINTER(sz)]
        L.tdc_cauchy_like_gemm.argtypes = [i64, i64, P, i64, P, P, P, P, P, i64, i32, ctypes.POINTER(Opts), P, sz, P]
        L.tdc_cauchy_like_ranks_workspace_size.argtypes = [i64, ctypes.POINTER(Opts), ctypes.POINTER(sz)]
        L.tdc_cauchy_like_ranks.argtypes = [i64, P, P, P, P, ctypes.POINTER(Opts), P, P, sz, P]
    if hasattr(L, "tdc_sytrd"):
        L.tdc_sytrd_workspace_size.argtypes = [i64, ctypes.POINTER(sz)]
        L.tdc_sytrd.argtypes = [i64, P, i64, P, P, P, P, sz, ctypes.POINTER(Opts), P]
        L.tdc_ormtr_workspace_size.argtypes = [i64, i64, ctypes.POINTER(sz)]
        L.tdc_ormtr.argtypes = [i64, i64, P, i64, P, P, i64, P, sz, ctypes.POINTER(Opts), P]
        L.tdc_syevd_workspace_size.argtypes = [i64, ctypes.POINTER(Opts), ctypes.POINTER(sz)]
        L.tdc_syevd.argtypes = [i64, P, i64, P, P, i64, P, sz, ctypes.POINTER(Opts), P]
    if hasattr(L, "tdc_structured_gemm"):
        L.tdc_structured_gemm_workspace_size.argtypes = [i64, i64, i32, ctypes.POINTER(Opts), ctypes.POINTER(sz)]
        L.tdc_structured_gemm.argtypes = [i64, i64, P, i64, i32, P, P, i64, i32, ctypes.POINTER(Opts), P, sz, P]
        L.tdc_dft_gemm_workspace_size.argtypes = [i64, i64, i32, ctypes.POINTER(Opts), ctypes.POINTER(sz)]
        L.tdc_dft_gemm.argtypes = [i64, i64, P, i64, P, P, i64, i32, ctypes.POINTER(Opts), P, sz, P]
    if hasattr(L, "tdc_sbevd"):
        L.tdc_sbevd_workspace_size.argtypes = [i64, i64, ctypes.POINTER(Opts), ctypes.POINTER(sz)]
        L.tdc_sbevd.argtypes = [i64, i64, P, i64, P, P, i64, P, sz, ctypes.POINTER(Opts), P]
    if hasattr(L, "tdc_bdsdc"):
        L.tdc_bdsdc_workspace_size.argtypes = [i64, ctypes.POINTER(Opts), ctypes.POINTER(sz)]
        L.tdc_bdsdc.argtypes = [i64, P, P, P, P, i64, P, i64, P, sz, ctypes.POINTER(Opts), P]
    if hasattr(L, "tdc_cauchy_gemm"):
        L.tdc_cauchy_gemm_workspace_size.argtypes = [i64, i64, i32, ctypes.POINTER(Opts), ctypes.POINTER(sz)]
        L.tdc_cauchy_gemm.argtypes = [i64, i64, P, i64, P, P, P, P, P, P, i64, i32, ctypes.POINTER(Opts), P,
                                      sz, P]
    _lib = L
    return L


def _check(fn, st):
    if st == TDC_WPRECISION:
        warnings.warn("%s: %s" % (fn, lib().tdc_strerror(st).decode()), TdcPrecisionWarning, stacklevel=3)
    elif st != 0:
        raise TdcError(fn, st)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def default_opts(**kw) -> Opts:
    o = Opts()
    lib().tdc_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def workspace_size(n: int, opts: Opts | None = None) -> int:
    b = ctypes.c_size_t(0)
    _check("tdc_workspace_size", lib().tdc_workspace_size(int(n), ctypes.byref(opts) if opts else None,
                                                          ctypes.byref(b)))
    return b.value


def workspace(nbytes: int, device="cuda") -> torch.Tensor:
    return torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=device)


def eig(d: torch.Tensor, e: torch.Tensor, opts: Opts | None = None, ws: torch.Tensor | None = None,
        lam: torch.Tensor | None = None, Q: torch.Tensor | None = None, stream=None, check: bool = False):
    """T = Q diag(lam) Q^T for the tridiagonal (d, e) (device FP64).  Q is
    returned as a column-major n x n matrix (a transposed view of row-major storage)."""
    n = d.numel()
    dev = d.device
    if lam is None:
        lam = torch.empty(n, dtype=torch.float64, device=dev)
    if Q is None:
        Q = torch.empty(n, n, dtype=torch.float64, device=dev).t()  # column-major storage
    if ws is None:
        ws = workspace(workspace_size(n, opts), dev)
    ld = Q.stride(1) if n > 0 else 1
    st = lib().tdc_eig(n, _ptr(d), _ptr(e), _ptr(lam), _ptr(Q), max(ld, 1), _ptr(ws), ws.numel(),
                       ctypes.byref(opts) if opts else None, _stream(stream))
    _check("tdc_eig", st)
    if check:
        _check("tdc_eig (device status)", sync_status(stream))
    return lam, Q


def batched_workspace_size(sizes, opts: Opts | None = None) -> int:
    import numpy as np
    nh = np.ascontiguousarray(sizes, dtype=np.int64)
    b = ctypes.c_size_t(0)
    _check("tdc_eig_batched_workspace_size",
           lib().tdc_eig_batched_workspace_size(len(nh), nh.ctypes.data_as(ctypes.c_void_p),
                                                ctypes.byref(opts) if opts else None, ctypes.byref(b)))
    return b.value


def eig_batched(sizes, d: torch.Tensor, e: torch.Tensor, off_de, off_q, lam: torch.Tensor, Q: torch.Tensor,
                opts: Opts | None = None, ws: torch.Tensor | None = None, stream=None, check: bool = False):
    import numpy as np
    nh = np.ascontiguousarray(sizes, dtype=np.int64)
    od = np.ascontiguousarray(off_de, dtype=np.int64)
    oq = np.ascontiguousarray(off_q, dtype=np.int64)
    if ws is None:
        ws = workspace(batched_workspace_size(nh, opts), d.device)
    st = lib().tdc_eig_batched(len(nh), nh.ctypes.data_as(ctypes.c_void_p), od.ctypes.data_as(ctypes.c_void_p),
                               oq.ctypes.data_as(ctypes.c_void_p), _ptr(d), _ptr(e), _ptr(lam), _ptr(Q), _ptr(ws),
                               ws.numel(), ctypes.byref(opts) if opts else None, _stream(stream))
    _check("tdc_eig_batched", st)
    if check:
        _check("tdc_eig_batched (device status)", sync_status(stream))
    return lam, Q


def rank_one(D: torch.Tensor, z: torch.Tensor, rho: float, max_iter: int = 64, stream=None, check=False):
    """Secular roots, Loewner zhat and column normalisers of D + rho z z^T (device FP64)."""
    K = D.numel()
    dev = D.device
    org = torch.empty(K, dtype=torch.int32, device=dev)
    tau = torch.empty(K, dtype=torch.float64, device=dev)
    zhat = torch.empty(K, dtype=torch.float64, device=dev)
    s = torch.empty(K, dtype=torch.float64, device=dev)
    b = ctypes.c_size_t(0)
    _check("tdc_rank_one_workspace_size", lib().tdc_rank_one_workspace_size(K, ctypes.byref(b)))
    ws = workspace(b.value, dev)
    _check("tdc_rank_one", lib().tdc_rank_one(K, _ptr(D), _ptr(z), float(rho), _ptr(org), _ptr(tau), _ptr(zhat),
                                              _ptr(s), int(max_iter), _ptr(ws), ws.numel(), _stream(stream)))
    if check:
        _check("tdc_rank_one (device status)", sync_status(stream))
    return org, tau, zhat, s


def cauchy_gemm_workspace_size(m: int, K: int, mode: int = MERGE_DENSE, opts: Opts | None = None) -> int:
    b = ctypes.c_size_t(0)
    _check("tdc_cauchy_gemm_workspace_size",
           lib().tdc_cauchy_gemm_workspace_size(m, K, mode, ctypes.byref(opts) if opts else None, ctypes.byref(b)))
    return b.value


def cauchy_gemm(A: torch.Tensor, D: torch.Tensor, org: torch.Tensor, tau: torch.Tensor, zhat: torch.Tensor,
                s: torch.Tensor, mode: int = MERGE_DENSE, opts: Opts | None = None, stream=None, check=False,
                ws: torch.Tensor | None = None):
    """C = A * Qhat with Qhat_ij = zhat_i s_j / ((D_i - D_org_j) - tau_j); A is a column-major m x K view.
    ws: an optional caller-owned workspace of cauchy_gemm_workspace_size bytes."""
    m, K = A.shape
    lda = A.stride(1) if K > 0 else max(m, 1)
    C = torch.empty(K, m, dtype=torch.float64, device=A.device).t()
    if ws is None:
        ws = workspace(cauchy_gemm_workspace_size(m, K, mode, opts), A.device)
    _check("tdc_cauchy_gemm", lib().tdc_cauchy_gemm(m, K, _ptr(A), max(lda, 1), _ptr(D), _ptr(org), _ptr(tau),
                                                    _ptr(zhat), _ptr(s), _ptr(C), max(m, 1), mode,
                                                    ctypes.byref(opts) if opts else None, _ptr(ws), ws.numel(),
                                                    _stream(stream)))
    if check:
        _check("tdc_cauchy_gemm (device status)", sync_status(stream))
    return C


def cauchy_like_gemm(A: torch.Tensor, d: torch.Tensor, w: torch.Tensor, u: torch.Tensor, v: torch.Tensor,
                     mode: int = MERGE_DENSE, opts: Opts | None = None, stream=None, check=False):
    """C = A * B with B_ij = u_i v_j / (d_i - w_j) (Example 1's operand); A a column-major
    m x n view, d and w ascending (device FP64)."""
    m, n = A.shape
    lda = A.stride(1) if n > 0 else max(m, 1)
    C = torch.empty(n, m, dtype=torch.float64, device=A.device).t()
    b = ctypes.c_size_t(0)
    _check("tdc_cauchy_like_gemm_workspace_size",
           lib().tdc_cauchy_like_gemm_workspace_size(m, n, mode, ctypes.byref(opts) if opts else None, ctypes.byref(b)))
    ws = workspace(b.value, A.device)
    _check("tdc_cauchy_like_gemm", lib().tdc_cauchy_like_gemm(m, n, _ptr(A), max(lda, 1), _ptr(d), _ptr(w), _ptr(u),
                                                              _ptr(v), _ptr(C), max(m, 1), mode,
                                                              ctypes.byref(opts) if opts else None, _ptr(ws),
                                                              ws.numel(), _stream(stream)))
    if check:
        _check("tdc_cauchy_like_gemm (device status)", sync_status(stream))
    return C


def cauchy_like_ranks(d: torch.Tensor, w: torch.Tensor, u: torch.Tensor, v: torch.Tensor,
                      opts: Opts | None = None, stream=None) -> torch.Tensor:
    """SRRSC ranks of the off-diagonal tiles of B_ij = u_i v_j / (d_i - w_j): a T x T int32
    tensor (rank of tile (I, J), -1 above the rank cap, 0 on the diagonal)."""
    n = d.numel()
    o = opts if opts else default_opts()
    T = max(1, (n + o.lr_tile - 1) // o.lr_tile)
    ranks = torch.zeros(T, T, dtype=torch.int32, device=d.device)
    b = ctypes.c_size_t(0)
    _check("tdc_cauchy_like_ranks_workspace_size", lib().tdc_cauchy_like_ranks_workspace_size(n, ctypes.byref(o),
                                                                                              ctypes.byref(b)))
    ws = workspace(b.value, d.device)
    _check("tdc_cauchy_like_ranks", lib().tdc_cauchy_like_ranks(n, _ptr(d), _ptr(w), _ptr(u), _ptr(v), ctypes.byref(o),
                                                                _ptr(ranks), _ptr(ws), ws.numel(), _stream(stream)))
    _check("tdc_cauchy_like_ranks (device status)", sync_status(stream))
    return ranks


def _colmajor_copy(A: torch.Tensor) -> torch.Tensor:
    n, m = A.shape
    R = torch.empty(m, n, dtype=torch.float64, device=A.device).t()
    R.copy_(A)
    return R


def sytrd(A: torch.Tensor, opts: Opts | None = None, stream=None, check: bool = False):
    """Householder reduction A = Q T Q^T of the symmetric A (device FP64, n x n, lower
    triangle read; A itself is not modified).  Returns (d, e, tau, R): T's diagonal and
    off-diagonal, the reflector scalars (n - 1, the last 0) and a column-major copy of A
    holding the reflectors below the subdiagonal (the input of ormtr)."""
    n = A.shape[0]
    R = _colmajor_copy(A)
    dev = A.device
    d = torch.empty(max(n, 1), dtype=torch.float64, device=dev)
    e = torch.empty(max(n - 1, 1), dtype=torch.float64, device=dev)
    tau = torch.empty(max(n - 1, 1), dtype=torch.float64, device=dev)
    b = ctypes.c_size_t(0)
    _check("tdc_sytrd_workspace_size", lib().tdc_sytrd_workspace_size(n, ctypes.byref(b)))
    ws = workspace(b.value, dev)
    _check("tdc_sytrd", lib().tdc_sytrd(n, _ptr(R), max(n, 1), _ptr(d), _ptr(e), _ptr(tau), _ptr(ws), ws.numel(),
                                        ctypes.byref(opts) if opts else None, _stream(stream)))
    if check:
        _check("tdc_sytrd (device status)", sync_status(stream))
    return d[:n], e[:max(n - 1, 0)], tau[:max(n - 1, 0)], R


def ormtr(R: torch.Tensor, tau: torch.Tensor, X: torch.Tensor, opts: Opts | None = None, stream=None,
          check: bool = False) -> torch.Tensor:
    """X <- Q X in place for the Q of sytrd (R, tau as sytrd returned them); X a
    column-major n x ncols view (stride(0) == 1)."""
    n, ncols = X.shape
    if X.stride(0) != 1 and ncols > 1:
        raise ValueError("X must be column-major (a transposed view of row-major storage)")
    b = ctypes.c_size_t(0)
    _check("tdc_ormtr_workspace_size", lib().tdc_ormtr_workspace_size(n, ncols, ctypes.byref(b)))
    ws = workspace(b.value, X.device)
    ldx = X.stride(1) if ncols > 1 else max(n, 1)
    _check("tdc_ormtr", lib().tdc_ormtr(n, ncols, _ptr(R), max(R.stride(1), n, 1), _ptr(tau), _ptr(X), max(ldx, n, 1),
                                        _ptr(ws), ws.numel(), ctypes.byref(opts) if opts else None, _stream(stream)))
    if check:
        _check("tdc_ormtr (device status)", sync_status(stream))
    return X


def syevd_workspace_size(n: int, opts: Opts | None = None) -> int:
    b = ctypes.c_size_t(0)
    _check("tdc_syevd_workspace_size", lib().tdc_syevd_workspace_size(int(n), ctypes.byref(opts) if opts else None,
                                                                      ctypes.byref(b)))
    return b.value


def syevd(A: torch.Tensor, opts: Opts | None = None, ws: torch.Tensor | None = None, stream=None,
          check: bool = False, overwrite: bool = False):
    """A = Z diag(lam) Z^T for the dense symmetric A (device FP64, lower triangle read):
    reduction, the divide and conquer on T, back-transform.  Returns (lam, Z), Z a
    column-major view.  overwrite=True lets the call destroy a column-major A instead of
    copying it."""
    n = A.shape[0]
    R = A if (overwrite and (A.stride(0) == 1 or n <= 1)) else _colmajor_copy(A)
    lam = torch.empty(max(n, 1), dtype=torch.float64, device=A.device)
    Z = torch.empty(n, n, dtype=torch.float64, device=A.device).t()
    if ws is None:
        ws = workspace(syevd_workspace_size(n, opts), A.device)
    _check("tdc_syevd", lib().tdc_syevd(n, _ptr(R), max(R.stride(1) if n > 1 else n, n, 1), _ptr(lam), _ptr(Z),
                                        max(n, 1), _ptr(ws), ws.numel(), ctypes.byref(opts) if opts else None,
                                        _stream(stream)))
    if check:
        _check("tdc_syevd (device status)", sync_status(stream))
    return lam[:n], Z


TOEPLITZ, HANKEL, VANDERMONDE = 1, 2, 3


def structured_gemm(A: torch.Tensor, t: torch.Tensor, kind: int = TOEPLITZ, mode: int = MERGE_DENSE,
                    opts: Opts | None = None, stream=None, check: bool = False) -> torch.Tensor:
    """C = A * B with B the n x n Toeplitz (B_kj = t[k - j + n - 1]), Hankel (t[k + j]) or
    Vandermonde (t[k]^j) matrix of the generators t; A a column-major m x n view (device
    FP64); mode MERGE_DENSE (FP64) or MERGE_SPLIT (BF16 digit products on the tensor cores)."""
    m, n = A.shape
    lda = A.stride(1) if n > 1 else max(m, 1)
    C = torch.empty(n, m, dtype=torch.float64, device=A.device).t()
    b = ctypes.c_size_t(0)
    _check("tdc_structured_gemm_workspace_size",
           lib().tdc_structured_gemm_workspace_size(m, n, mode, ctypes.byref(opts) if opts else None,
                                                    ctypes.byref(b)))
    ws = workspace(b.value, A.device)
    _check("tdc_structured_gemm", lib().tdc_structured_gemm(m, n, _ptr(A), max(lda, m, 1), kind, _ptr(t), _ptr(C),
                                                            max(m, 1), mode, ctypes.byref(opts) if opts else None,
                                                            _ptr(ws), ws.numel(), _stream(stream)))
    if check:
        _check("tdc_structured_gemm (device status)", sync_status(stream))
    return C


def dft_gemm(A: torch.Tensor, mode: int = MERGE_DENSE, opts: Opts | None = None, stream=None, check: bool = False):
    """(Re, Im) of C = A F, F(k, j) = exp(-2 pi i k j / n), for a real column-major m x n A."""
    m, n = A.shape
    lda = A.stride(1) if n > 1 else max(m, 1)
    Cr = torch.empty(n, m, dtype=torch.float64, device=A.device).t()
    Ci = torch.empty(n, m, dtype=torch.float64, device=A.device).t()
    b = ctypes.c_size_t(0)
    _check("tdc_dft_gemm_workspace_size",
           lib().tdc_dft_gemm_workspace_size(m, n, mode, ctypes.byref(opts) if opts else None, ctypes.byref(b)))
    ws = workspace(b.value, A.device)
    _check("tdc_dft_gemm", lib().tdc_dft_gemm(m, n, _ptr(A), max(lda, m, 1), _ptr(Cr), _ptr(Ci), max(m, 1), mode,
                                              ctypes.byref(opts) if opts else None, _ptr(ws), ws.numel(),
                                              _stream(stream)))
    if check:
        _check("tdc_dft_gemm (device status)", sync_status(stream))
    return Cr, Ci


def sbevd(AB: torch.Tensor, opts: Opts | None = None, stream=None, check: bool = False):
    """A = Q diag(lam) Q^T for the symmetric band matrix in lower band storage AB
    ((b + 1) x n, AB[i - j, j] = A[i, j]; device FP64, any layout: copied column-major).
    Returns (lam, Q), Q a column-major n x n view."""
    b1, n = AB.shape
    b = b1 - 1
    ABc = _colmajor_copy(AB)
    lam = torch.empty(max(n, 1), dtype=torch.float64, device=AB.device)
    Q = torch.empty(n, n, dtype=torch.float64, device=AB.device).t()
    nb = ctypes.c_size_t(0)
    _check("tdc_sbevd_workspace_size", lib().tdc_sbevd_workspace_size(n, b, ctypes.byref(opts) if opts else None,
                                                                      ctypes.byref(nb)))
    ws = workspace(nb.value, AB.device)
    _check("tdc_sbevd", lib().tdc_sbevd(n, b, _ptr(ABc), max(b1, 1), _ptr(lam), _ptr(Q), max(n, 1), _ptr(ws),
                                        ws.numel(), ctypes.byref(opts) if opts else None, _stream(stream)))
    if check:
        _check("tdc_sbevd (device status)", sync_status(stream))
    return lam[:n], Q


def bdsdc(d: torch.Tensor, e: torch.Tensor, opts: Opts | None = None, stream=None, check: bool = False):
    """SVD B = U diag(sigma) VT of the upper bidiagonal B (diagonal d, superdiagonal e,
    device FP64) through the divide and conquer on the Golub-Kahan tridiagonal.  Returns
    (sigma, U, VT): sigma descending, U and VT column-major n x n views."""
    n = d.numel()
    dev = d.device
    sigma = torch.empty(max(n, 1), dtype=torch.float64, device=dev)
    U = torch.empty(n, n, dtype=torch.float64, device=dev).t()
    VT = torch.empty(n, n, dtype=torch.float64, device=dev).t()
    b = ctypes.c_size_t(0)
    _check("tdc_bdsdc_workspace_size", lib().tdc_bdsdc_workspace_size(n, ctypes.byref(opts) if opts else None,
                                                                      ctypes.byref(b)))
    ws = workspace(b.value, dev)
    _check("tdc_bdsdc", lib().tdc_bdsdc(n, _ptr(d), _ptr(e), _ptr(sigma), _ptr(U), max(n, 1), _ptr(VT), max(n, 1),
                                        _ptr(ws), ws.numel(), ctypes.byref(opts) if opts else None,
                                        _stream(stream)))
    if check:
        _check("tdc_bdsdc (device status)", sync_status(stream))
    return sigma[:n], U, VT


def eig_backward(lam: torch.Tensor, Q: torch.Tensor, lam_bar=None, Q_bar=None, stream=None):
    """Cotangents (d_bar, e_bar) of the tridiagonal entries (tdc_eig_backward).  Q is the
    column-major n x n eigenvector matrix; Q_bar any n x n tensor (copied column-major)."""
    n = lam.numel()
    dev = lam.device
    Qc = Q if (Q.stride(0) == 1 and Q.stride(1) >= max(n, 1)) else Q.t().contiguous().t()
    Qb = None if Q_bar is None else Q_bar.t().contiguous().t()
    if Qb is not None and Qb.stride(1) != Qc.stride(1):
        Qc = Q.t().contiguous().t()
    lb = None if lam_bar is None else lam_bar.contiguous().to(torch.float64)
    d_bar = torch.empty(n, dtype=torch.float64, device=dev)
    e_bar = torch.empty(max(n - 1, 0), dtype=torch.float64, device=dev)
    b = ctypes.c_size_t(0)
    _check("tdc_backward_workspace_size", lib().tdc_backward_workspace_size(n, ctypes.byref(b)))
    ws = workspace(b.value, dev)
    _check("tdc_eig_backward", lib().tdc_eig_backward(n, _ptr(lam), _ptr(Qc), max(Qc.stride(1), 1), _ptr(lb),
                                                      _ptr(Qb), _ptr(d_bar), _ptr(e_bar), _ptr(ws), ws.numel(),
                                                      _stream(stream)))
    return d_bar, e_bar


def eig_backward_batched(lam: torch.Tensor, Qs: torch.Tensor, lam_bar=None, Qs_bar=None, stream=None):
    """Batched adjoint: lam (B, n); Qs the (B, n, n) storage whose [b] is Q_b column-major
    (i.e. Q_b = Qs[b].t()); Qs_bar likewise."""
    B, n = lam.shape
    dev = lam.device
    d_bar = torch.empty(B, n, dtype=torch.float64, device=dev)
    e_bar = torch.empty(B, max(n - 1, 0), dtype=torch.float64, device=dev)
    b = ctypes.c_size_t(0)
    _check("tdc_backward_batched_workspace_size", lib().tdc_backward_batched_workspace_size(B, n, ctypes.byref(b)))
    ws = workspace(b.value, dev)
    lb = None if lam_bar is None else lam_bar.contiguous()
    qb = None if Qs_bar is None else Qs_bar.contiguous()
    _check("tdc_eig_backward_batched",
           lib().tdc_eig_backward_batched(B, n, _ptr(lam.contiguous()), _ptr(Qs.contiguous()), _ptr(lb), _ptr(qb),
                                          _ptr(d_bar), _ptr(e_bar), _ptr(ws), ws.numel(), _stream(stream)))
    return d_bar, e_bar


class _EighTridiagonal(torch.autograd.Function):
    """(lam, Q) = eig(T(d, e)) with the backward of tdc_eig_backward; d, e of shape
    (n,) / (n-1,) or batched (B, n) / (B, n-1)."""

    @staticmethod
    def forward(ctx, d, e, opts):
        if d.dim() == 1:
            lam, Q = eig(d.contiguous(), e.contiguous(), opts)
            ctx.save_for_backward(lam, Q)
            ctx.batched = False
            return lam, Q
        import numpy as np
        B, n = d.shape
        dev = d.device
        dd = d.contiguous().reshape(-1)
        ee = torch.zeros(B, n, dtype=torch.float64, device=dev)
        ee[:, : n - 1] = e
        lam = torch.empty(B, n, dtype=torch.float64, device=dev)
        Qs = torch.empty(B, n, n, dtype=torch.float64, device=dev)
        sizes = np.full(B, n, dtype=np.int64)
        eig_batched(sizes, dd, ee.reshape(-1), np.arange(B, dtype=np.int64) * n,
                    np.arange(B, dtype=np.int64) * n * n, lam.reshape(-1), Qs.reshape(-1), opts)
        ctx.save_for_backward(lam, Qs)
        ctx.batched = True
        return lam, Qs.transpose(1, 2)

    @staticmethod
    def backward(ctx, lam_bar, Q_bar):
        lam, Qx = ctx.saved_tensors
        if not ctx.batched:
            d_bar, e_bar = eig_backward(lam, Qx, lam_bar, Q_bar)
        else:
            qsb = None if Q_bar is None else Q_bar.transpose(1, 2).contiguous()
            d_bar, e_bar = eig_backward_batched(lam, Qx, lam_bar, qsb)
        return d_bar, e_bar, None


def eigh_tridiagonal(d: torch.Tensor, e: torch.Tensor, opts: Opts | None = None):
    """Differentiable eigen-decomposition of the symmetric tridiagonal (d, e)."""
    return _EighTridiagonal.apply(d, e, opts)


def sync_status(stream=None) -> int:
    return int(lib().tdc_sync_status(_stream(stream)))


def get_stats() -> dict:
    s = Stats()
    _check("tdc_get_stats", lib().tdc_get_stats(ctypes.byref(s)))
    return s.as_dict()


def strerror(status: int) -> str:
    return lib().tdc_strerror(int(status)).decode()
