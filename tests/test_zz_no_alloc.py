"""tdc_eig_noalloc: the eigensolver for callers that cannot allocate device memory.

Such callers (a process whose device memory is fully reserved by another
allocator, plugins that must not touch the allocator, latency-critical paths
where an allocation may block or fail) pass only inputs and outputs; the solver
then works in a fixed array inside the library.  This test calls the entry point
through the C ABI twice in a row and checks each result against tdc_eig with a
caller-provided workspace, using the tolerances of the other GPU tests
(|lam - lam_ref| <= 1e-12 ||T||, eigenvectors equal up to sign).  It is collected
last so that a failure here cannot hide the other tests.
"""
import ctypes

import numpy as np
import pytest
import torch

from helpers import compare_vectors
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


def test_noalloc_matches_workspace_path_twice(tdc):
    # the library's default merge choice falls back to the FP64 merge inside the fixed scratch
    opts = tdc.default_opts(leaf=32, merge_mode=tdc.MERGE_DENSE)
    for n, seed in ((1000, 21), (700, 22)):
        d_np, e_np = inputs.uniform_tridiag(n, seed)
        d = torch.tensor(d_np, device=DEV)
        e = torch.tensor(e_np, device=DEV)
        lam, Q = _noalloc(tdc, d, e, tdc.default_opts(leaf=32))
        lam_ref, Q_ref = tdc.eig(d, e, opts, check=True)
        lam, Q = lam.cpu().numpy(), Q.cpu().numpy()
        lam_ref, Q_ref = lam_ref.cpu().numpy(), Q_ref.cpu().numpy()
        nT = max(abs(lam_ref[0]), abs(lam_ref[-1]))
        assert np.max(np.abs(lam - lam_ref)) <= 1e-12 * nT
        compare_vectors(Q, Q_ref, lam_ref, 1e-8 * nT, 1e-9)


def test_noalloc_rejects_orders_beyond_its_scratch(tdc):
    n = 4096
    d = torch.ones(n, dtype=torch.float64, device=DEV)
    st = tdc.lib().tdc_eig_noalloc(n, ctypes.c_void_p(d.data_ptr()), ctypes.c_void_p(d.data_ptr()),
                                   ctypes.c_void_p(d.data_ptr()), ctypes.c_void_p(d.data_ptr()), n, None,
                                   ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == tdc.TDC_ETOOLARGE
