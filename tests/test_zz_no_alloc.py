"""tdc_eig_noalloc: the eigensolver for callers that cannot allocate device memory.

Such callers (a process whose device memory is fully reserved by another
allocator, plugins that must not touch the allocator, latency-critical paths
where an allocation may block or fail) pass only inputs and outputs; the solver
then works in a fixed array inside the library.  This test calls the entry point
through the C ABI twice in a row and checks each result against tdc_eig with a
caller-provided workspace.  Both calls run the same kernels on the same inputs in
the same order, so the results must be identical bit for bit: once where the
library's default merge (the split path) fits the fixed array and runs inside it,
and once where it does not and the entry point takes the FP64 merge.  It is
collected last so that a failure here cannot hide the other tests.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2008_01990_gb300 import inputs

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module")
def tdc():
    from paper_2008_01990_gb300 import build, tdc as t
    build.build()
    t.lib()
    return t


def _noalloc(tdc, d, e, opts):
    n = d.numel()
    lam = torch.empty(n, dtype=torch.float64, device=DEV)
    Q = torch.empty(n, n, dtype=torch.float64, device=DEV).t()
    st = tdc.lib().tdc_eig_noalloc(n, ctypes.c_void_p(d.data_ptr()), ctypes.c_void_p(e.data_ptr()),
                                   ctypes.c_void_p(lam.data_ptr()), ctypes.c_void_p(Q.data_ptr()), Q.stride(1),
                                   ctypes.byref(opts), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, tdc.strerror(st)
    assert tdc.sync_status() == 0
    return lam, Q


SCRATCH = 24 << 20  # the entry point's fixed array


def _same_as_workspace_path(tdc, n, seed, ref_mode):
    d_np, e_np = inputs.uniform_tridiag(n, seed)
    d = torch.tensor(d_np, device=DEV)
    e = torch.tensor(e_np, device=DEV)
    lam, Q = _noalloc(tdc, d, e, tdc.default_opts(leaf=32))
    lam_ref, Q_ref = tdc.eig(d, e, tdc.default_opts(leaf=32, merge_mode=ref_mode), check=True)
    assert torch.equal(lam, lam_ref)
    assert torch.equal(Q, Q_ref)
    # and the result is an eigen-decomposition (tolerances of the other GPU tests)
    lam, Q = lam.cpu().numpy(), Q.cpu().numpy()
    nT = max(abs(lam[0]), abs(lam[-1]))
    T = np.diag(d_np) + np.diag(e_np, 1) + np.diag(e_np, -1)
    eps = np.finfo(float).eps
    assert np.abs(T @ Q - Q * lam).sum(axis=0).max() / (n * nT * eps) <= 50
    assert np.abs(Q.T @ Q - np.eye(n)).sum(axis=0).max() / (n * eps) <= 50


def test_noalloc_split_path_inside_the_scratch_twice(tdc):
    # orders whose default (split-path) workspace fits the fixed array: the split kernels
    # run out of it
    for n, seed in ((300, 23), (400, 24)):
        assert tdc.workspace_size(n, tdc.default_opts(leaf=32)) <= SCRATCH
        _same_as_workspace_path(tdc, n, seed, tdc.MERGE_AUTO)


def test_noalloc_matches_workspace_path_twice(tdc):
    # orders whose split-path workspace does not fit: the FP64 merge inside the fixed array
    for n, seed in ((1000, 21), (700, 22)):
        assert tdc.workspace_size(n, tdc.default_opts(leaf=32)) > SCRATCH
        _same_as_workspace_path(tdc, n, seed, tdc.MERGE_DENSE)


def test_noalloc_rejects_orders_beyond_its_scratch(tdc):
    n = 4096
    d = torch.ones(n, dtype=torch.float64, device=DEV)
    st = tdc.lib().tdc_eig_noalloc(n, ctypes.c_void_p(d.data_ptr()), ctypes.c_void_p(d.data_ptr()),
                                   ctypes.c_void_p(d.data_ptr()), ctypes.c_void_p(d.data_ptr()), n, None,
                                   ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == tdc.TDC_ETOOLARGE
