"""The C-ABI library builds, loads without a GPU, exports every entry point that
include/tdc.h declares, and rejects invalid arguments on the host."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2008_01990_gb300 import build, tdc
    build.build()
    return tdc.lib()


def declared_functions():
    hdr = open(os.path.join(ROOT, "include", "tdc.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|void|const char\*)\s+(tdc_\w+)\s*\(", hdr, flags=re.M)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "tdc_eig" in names and "tdc_eig_batched" in names
    for nm in names:
        assert hasattr(lib, nm), nm


def test_default_opts_and_workspace(lib):
    from paper_2008_01990_gb300 import tdc
    o = tdc.default_opts()
    assert o.leaf == 16 and o.max_iter >= 1 and o.sign_normalise == 1
    assert o.split_chunk_k == 256 and ctypes.sizeof(o) == 64
    w1 = tdc.workspace_size(1024, o)
    w2 = tdc.workspace_size(2048, o)
    assert 2048 * 2048 * 8 < w2 and w1 < w2
    assert tdc.workspace_size(0, o) > 0
    # the structured merge on the split path needs its own scratch on top of the split path's
    w4 = tdc.workspace_size(16384, tdc.default_opts(leaf=64, merge_mode=tdc.MERGE_STRUCTURED_SPLIT))
    assert w4 > tdc.workspace_size(16384, tdc.default_opts(leaf=64, merge_mode=tdc.MERGE_SPLIT))
    assert w4 == tdc.workspace_size(16384, tdc.default_opts(leaf=64))  # the library's default merge
    assert tdc.cauchy_gemm_workspace_size(300, 1000, tdc.MERGE_STRUCTURED_SPLIT,
                                          tdc.default_opts(lr_tile=128)) > 300 * 1000 * 2
    # the chunk length of the split accumulators' drains changes no workspace
    assert tdc.workspace_size(2048, tdc.default_opts(split_chunk_k=512)) == w2
    assert tdc.workspace_size(2048, tdc.default_opts(split_chunk_k=0)) == w2


def test_host_argument_checks(lib):
    from paper_2008_01990_gb300 import tdc
    P = ctypes.c_void_p
    bogus = P(0x1000)
    assert lib.tdc_eig(-1, bogus, bogus, bogus, bogus, 1, bogus, 0, None, None) == -1
    assert lib.tdc_eig(0, None, None, None, None, 1, None, 0, None, None) == 0
    assert lib.tdc_eig(4, None, bogus, bogus, bogus, 4, bogus, 1 << 30, None, None) == -2
    assert lib.tdc_eig(4, bogus, None, bogus, bogus, 4, bogus, 1 << 30, None, None) == -3
    assert lib.tdc_eig(4, bogus, bogus, None, bogus, 4, bogus, 1 << 30, None, None) == -4
    assert lib.tdc_eig(4, bogus, bogus, bogus, None, 4, bogus, 1 << 30, None, None) == -5
    assert lib.tdc_eig(4, bogus, bogus, bogus, bogus, 3, bogus, 1 << 30, None, None) == -6
    o = tdc.default_opts(leaf=1)
    assert lib.tdc_eig(4, bogus, bogus, bogus, bogus, 4, bogus, 1 << 30, ctypes.byref(o), None) == -9
    o = tdc.default_opts()
    assert lib.tdc_eig(4, bogus, bogus, bogus, bogus, 4, bogus, 16, ctypes.byref(o), None) == tdc.TDC_ENOWS
    assert lib.tdc_eig(4, bogus, bogus, bogus, bogus, 4, None, 1 << 30, ctypes.byref(o), None) == tdc.TDC_ENOWS
    import numpy as np
    nh = np.array([5, -2, 7], dtype=np.int64)
    assert lib.tdc_eig_batched(3, nh.ctypes.data_as(P), nh.ctypes.data_as(P), nh.ctypes.data_as(P), bogus, bogus,
                               bogus, bogus, bogus, 1 << 30, None, None) == -1001
    assert lib.tdc_rank_one(4, bogus, bogus, -1.0, bogus, bogus, bogus, bogus, 8, bogus, 256, None) == -4
    # the rank-one workspace holds the FP32 copies of the poles (about 20 K bytes)
    b = ctypes.c_size_t(0)
    assert lib.tdc_rank_one_workspace_size(1000, ctypes.byref(b)) == 0 and b.value >= 20 * 1000
    assert lib.tdc_rank_one(1000, bogus, bogus, 1.0, bogus, bogus, bogus, bogus, 8, bogus, b.value - 1,
                            None) == tdc.TDC_ENOWS
    assert lib.tdc_rank_one(1000, bogus, bogus, 1.0, bogus, bogus, bogus, bogus, 8, None, b.value,
                            None) == tdc.TDC_ENOWS
    assert tdc.strerror(tdc.TDC_ENOWS).startswith("workspace")
    assert tdc.strerror(tdc.TDC_WPRECISION).startswith("warning")


@pytest.mark.parametrize("bad", [dict(leaf=1), dict(leaf=65), dict(merge_mode=5), dict(max_iter=0),
                                 dict(lr_tile=100), dict(split_slices=2), dict(split_slices=8),
                                 dict(split_min_K=0), dict(spin_budget=0), dict(lr_tol=0.0),
                                 dict(split_chunk_k=8), dict(split_chunk_k=-16)])
def test_invalid_options_rejected_on_host(lib, bad):
    """Every option outside its documented range is refused before anything is
    enqueued (the workspace query validates the same way)."""
    from paper_2008_01990_gb300 import tdc
    o = tdc.default_opts(**bad)
    P = ctypes.c_void_p
    bogus = P(0x1000)
    assert lib.tdc_eig(4, bogus, bogus, bogus, bogus, 4, bogus, 1 << 30, ctypes.byref(o), None) == -9
    nb = ctypes.c_size_t(0)
    assert lib.tdc_workspace_size(4, ctypes.byref(o), ctypes.byref(nb)) == -2


def test_dense_symmetric_entry_points_check_arguments_on_the_host(lib):
    from paper_2008_01990_gb300 import tdc
    bogus = ctypes.c_void_p(0x1000)
    big = 1 << 40
    assert lib.tdc_sytrd(-1, bogus, 1, bogus, bogus, bogus, bogus, big, None, None) == -1
    assert lib.tdc_sytrd(0, None, 1, None, None, None, None, 0, None, None) == 0
    assert lib.tdc_sytrd(4, None, 4, bogus, bogus, bogus, bogus, big, None, None) == -2
    assert lib.tdc_sytrd(4, bogus, 3, bogus, bogus, bogus, bogus, big, None, None) == -3
    assert lib.tdc_sytrd(4, bogus, 4, None, bogus, bogus, bogus, big, None, None) == -4
    assert lib.tdc_sytrd(4, bogus, 4, bogus, None, bogus, bogus, big, None, None) == -5
    assert lib.tdc_sytrd(4, bogus, 4, bogus, bogus, None, bogus, big, None, None) == -6
    assert lib.tdc_sytrd(4, bogus, 4, bogus, bogus, bogus, bogus, 16, None, None) == tdc.TDC_ENOWS
    assert lib.tdc_ormtr(-1, 1, bogus, 1, bogus, bogus, 1, bogus, big, None, None) == -1
    assert lib.tdc_ormtr(4, -1, bogus, 4, bogus, bogus, 4, bogus, big, None, None) == -2
    assert lib.tdc_ormtr(2, 5, None, 1, None, None, 1, None, 0, None, None) == 0  # no reflector
    assert lib.tdc_ormtr(6, 5, None, 6, bogus, bogus, 6, bogus, big, None, None) == -3
    assert lib.tdc_ormtr(6, 5, bogus, 5, bogus, bogus, 6, bogus, big, None, None) == -4
    assert lib.tdc_ormtr(6, 5, bogus, 6, None, bogus, 6, bogus, big, None, None) == -5
    assert lib.tdc_ormtr(6, 5, bogus, 6, bogus, None, 6, bogus, big, None, None) == -6
    assert lib.tdc_ormtr(6, 5, bogus, 6, bogus, bogus, 5, bogus, big, None, None) == -7
    assert lib.tdc_ormtr(6, 5, bogus, 6, bogus, bogus, 6, bogus, 16, None, None) == tdc.TDC_ENOWS
    assert lib.tdc_syevd(-1, bogus, 1, bogus, bogus, 1, bogus, big, None, None) == -1
    assert lib.tdc_syevd(5, None, 5, bogus, bogus, 5, bogus, big, None, None) == -2
    assert lib.tdc_syevd(5, bogus, 4, bogus, bogus, 5, bogus, big, None, None) == -3
    assert lib.tdc_syevd(5, bogus, 5, None, bogus, 5, bogus, big, None, None) == -4
    assert lib.tdc_syevd(5, bogus, 5, bogus, None, 5, bogus, big, None, None) == -5
    assert lib.tdc_syevd(5, bogus, 5, bogus, bogus, 4, bogus, big, None, None) == -6
    assert lib.tdc_syevd(5, bogus, 5, bogus, bogus, 5, bogus, 16, None, None) == tdc.TDC_ENOWS
    sz = [ctypes.c_size_t(0) for _ in range(3)]
    for i, n in enumerate((100, 1000, 4000)):
        assert lib.tdc_syevd_workspace_size(n, None, ctypes.byref(sz[i])) == 0
    assert sz[0].value < sz[1].value < sz[2].value
    w = ctypes.c_size_t(0)
    assert lib.tdc_workspace_size(4000, None, ctypes.byref(w)) == 0
    assert sz[2].value > w.value


def test_bdsdc_checks_arguments_on_the_host(lib):
    from paper_2008_01990_gb300 import tdc
    bogus = ctypes.c_void_p(0x1000)
    big = 1 << 40
    assert lib.tdc_bdsdc(-1, bogus, bogus, bogus, bogus, 1, bogus, 1, bogus, big, None, None) == -1
    assert lib.tdc_bdsdc(0, None, None, None, None, 1, None, 1, None, 0, None, None) == 0
    assert lib.tdc_bdsdc(4, None, bogus, bogus, bogus, 4, bogus, 4, bogus, big, None, None) == -2
    assert lib.tdc_bdsdc(4, bogus, None, bogus, bogus, 4, bogus, 4, bogus, big, None, None) == -3
    assert lib.tdc_bdsdc(4, bogus, bogus, None, bogus, 4, bogus, 4, bogus, big, None, None) == -4
    assert lib.tdc_bdsdc(4, bogus, bogus, bogus, None, 4, bogus, 4, bogus, big, None, None) == -5
    assert lib.tdc_bdsdc(4, bogus, bogus, bogus, bogus, 3, bogus, 4, bogus, big, None, None) == -6
    assert lib.tdc_bdsdc(4, bogus, bogus, bogus, bogus, 4, None, 4, bogus, big, None, None) == -7
    assert lib.tdc_bdsdc(4, bogus, bogus, bogus, bogus, 4, bogus, 3, bogus, big, None, None) == -8
    assert lib.tdc_bdsdc(4, bogus, bogus, bogus, bogus, 4, bogus, 4, bogus, 16, None, None) == tdc.TDC_ENOWS
    a, b = ctypes.c_size_t(0), ctypes.c_size_t(0)
    assert lib.tdc_bdsdc_workspace_size(1000, None, ctypes.byref(a)) == 0
    assert lib.tdc_workspace_size(2000, None, ctypes.byref(b)) == 0
    assert a.value > b.value + 8 * 2000 * 2000


def test_structured_gemm_checks_arguments_on_the_host(lib):
    from paper_2008_01990_gb300 import tdc
    bogus = ctypes.c_void_p(0x1000)
    big = 1 << 40
    f = lib.tdc_structured_gemm
    assert f(-1, 4, bogus, 1, 1, bogus, bogus, 1, 0, None, bogus, big, None) == -1
    assert f(4, -1, bogus, 4, 1, bogus, bogus, 4, 0, None, bogus, big, None) == -2
    assert f(0, 4, None, 1, 1, None, None, 1, 0, None, None, 0, None) == 0
    assert f(4, 4, None, 4, 1, bogus, bogus, 4, 0, None, bogus, big, None) == -3
    assert f(4, 4, bogus, 3, 1, bogus, bogus, 4, 0, None, bogus, big, None) == -4
    assert f(4, 4, bogus, 4, 5, bogus, bogus, 4, 0, None, bogus, big, None) == -5
    assert f(4, 4, bogus, 4, 1, None, bogus, 4, 0, None, bogus, big, None) == -6
    assert f(4, 4, bogus, 4, 1, bogus, None, 4, 0, None, bogus, big, None) == -7
    assert f(4, 4, bogus, 4, 1, bogus, bogus, 3, 0, None, bogus, big, None) == -8
    assert f(4, 4, bogus, 4, 1, bogus, bogus, 4, tdc.MERGE_STRUCTURED, None, bogus, big, None) == -9
    assert f(4, 4, bogus, 4, 1, bogus, bogus, 4, tdc.MERGE_DENSE, None, bogus, 8, None) == tdc.TDC_ENOWS

    g = lib.tdc_dft_gemm
    assert g(-1, 4, bogus, 1, bogus, bogus, 1, 1, None, bogus, big, None) == -1
    assert g(4, 4, None, 4, bogus, bogus, 4, 1, None, bogus, big, None) == -3
    assert g(4, 4, bogus, 4, None, bogus, 4, 1, None, bogus, big, None) == -5
    assert g(4, 4, bogus, 4, bogus, None, 4, 1, None, bogus, big, None) == -6
    assert g(4, 4, bogus, 4, bogus, bogus, 3, 1, None, bogus, big, None) == -7
    assert g(4, 4, bogus, 4, bogus, bogus, 4, 2, None, bogus, big, None) == -8
    assert g(4, 4, bogus, 4, bogus, bogus, 4, 1, None, bogus, 8, None) == tdc.TDC_ENOWS


def test_sbevd_checks_arguments_on_the_host(lib):
    from paper_2008_01990_gb300 import tdc
    bogus = ctypes.c_void_p(0x1000)
    big = 1 << 40
    f = lib.tdc_sbevd
    assert f(-1, 0, bogus, 1, bogus, bogus, 1, bogus, big, None, None) == -1
    assert f(0, 0, None, 1, None, None, 1, None, 0, None, None) == 0
    assert f(10, 10, bogus, 11, bogus, bogus, 10, bogus, big, None, None) == -2
    assert f(10, 65, bogus, 66, bogus, bogus, 10, bogus, big, None, None) == -2
    assert f(10, 2, None, 3, bogus, bogus, 10, bogus, big, None, None) == -3
    assert f(10, 2, bogus, 2, bogus, bogus, 10, bogus, big, None, None) == -4
    assert f(10, 2, bogus, 3, None, bogus, 10, bogus, big, None, None) == -5
    assert f(10, 2, bogus, 3, bogus, None, 10, bogus, big, None, None) == -6
    assert f(10, 2, bogus, 3, bogus, bogus, 9, bogus, big, None, None) == -7
    assert f(10, 2, bogus, 3, bogus, bogus, 10, bogus, 16, None, None) == tdc.TDC_ENOWS
    a = ctypes.c_size_t(0)
    assert lib.tdc_sbevd_workspace_size(1000, 8, None, ctypes.byref(a)) == 0 and a.value > 8 * 1000 * 1000
