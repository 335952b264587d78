"""The C ABI without a GPU: the library loads, exports every symbol
include/pylom.h declares, and host-side validation rejects bad calls with
the documented status codes before touching the device."""
import ctypes
import os
import re

import pytest

import paper_2405_15529_gb300 as pg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(pylom_\w+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2405_15529_gb300 import _build
    _build.build()
    return pg.load_library()


def test_exports_every_declared_symbol(lib):
    declared = _declared()
    assert len(declared) >= 12
    for name in declared:
        assert hasattr(lib, name), f"libpylom.so does not export {name}"
    assert set(pg.EXPORTS) <= set(declared)


def test_version_and_leaf_partition(lib):
    assert b"sm_103a" in lib.pylom_version()
    # P = max(1, floor(N / b)); every leaf has >= b rows
    assert pg.leaf_count(16384, 64, 1024) == 16
    assert pg.leaf_count(16384 + 1000, 64, 1024) == 16
    assert pg.leaf_count(100, 64, 1024) == 1
    assert pg.leaf_count(4194304, 256, 0) == 304
    assert pg.leaf_count(16384, 64, 0) == 16
    assert pg.leaf_count(10, 20, 0) == -1       # N < M
    assert pg.leaf_count(1000, 64, 32) == -1    # leaf height < M


def test_workspace_queries(lib):
    assert pg.pod_workspace_size(16384, 64, 1024, 64) > 16384 * 64 * 8
    assert pg.pod_workspace_size(16384, 64, 1024, 65) == 0      # r_max > M
    assert pg.pod_workspace_size(50, 64, 0, 10) == 0            # N < M
    assert lib.pylom_svd_small_workspace_size(64) > 0
    assert lib.pylom_svd_small_workspace_size(0) == 0
    assert lib.pylom_tsqr_workspace_size(1000, 10, 0, 1, pg.F64, pg.PREC_FP64) > 0
    assert lib.pylom_matmul_workspace_size(43, 256, 1 << 22) > 0


def _vp(x):
    return ctypes.c_void_p(x)


def test_host_validation_without_gpu(lib):
    fake = _vp(0x100000)  # never dereferenced: validation fails first
    st = lib.pylom_pod(None, 100, 10, 100, pg.F64, None, 1, 0.0, 10, 0, 0, fake, 100, fake, fake,
                       10, None, None, pg.PREC_FP64, fake, 1 << 30, None)
    assert st == pg.ERR_ARG
    st = lib.pylom_pod(fake, 5, 10, 5, pg.F64, None, 1, 0.0, 10, 0, 0, fake, 5, fake, fake, 10,
                       None, None, pg.PREC_FP64, fake, 1 << 30, None)
    assert st == pg.ERR_SHAPE
    st = lib.pylom_pod(fake, 100, 10, 50, pg.F64, None, 1, 0.0, 10, 0, 0, fake, 100, fake, fake,
                       10, None, None, pg.PREC_FP64, fake, 1 << 30, None)
    assert st == pg.ERR_ARG                      # ldx < N
    st = lib.pylom_pod(fake, 100, 10, 100, 7, None, 1, 0.0, 10, 0, 0, fake, 100, fake, fake, 10,
                       None, None, pg.PREC_FP64, fake, 1 << 30, None)
    assert st == pg.ERR_ARG                      # bad dtype
    st = lib.pylom_pod(fake, 100, 10, 100, pg.F64, None, 1, 0.0, 11, 0, 0, fake, 100, fake, fake,
                       10, None, None, pg.PREC_FP64, fake, 1 << 30, None)
    assert st == pg.ERR_SHAPE                    # r_max > M
    st = lib.pylom_pod(fake, 100, 10, 100, pg.F64, None, 1, 0.0, 10, 0, 0, fake, 100, fake, fake,
                       10, None, None, pg.PREC_FP64, fake, 64, None)
    assert st == pg.ERR_WORKSPACE
    st = lib.pylom_pod(fake, 100, 10, 100, pg.F64, None, 1, 0.0, 10, 0, 0, fake, 100, fake, fake,
                       10, None, None, pg.PREC_FP64, _vp(0x100008), 1 << 30, None)
    assert st == pg.ERR_WORKSPACE                # misaligned
    assert b"workspace" in lib.pylom_last_error()
    st = lib.pylom_svd_small(fake, 10, 10, fake, 10, fake, fake, 10, 0, fake, 1 << 20, None)
    assert st == pg.ERR_ARG                      # max_sweeps out of range
    st = lib.pylom_svd_small(fake, 10, 10, fake, 10, fake, fake, 10, 99, fake, 1 << 20, None)
    assert st == pg.ERR_ARG
    st = lib.pylom_tsqr(fake, 100, 10, 100, pg.F64, 5, fake, 10, None, 100, pg.PREC_FP64, fake,
                        1 << 30, None)
    assert st == pg.ERR_SHAPE                    # leaf height < M
    st = lib.pylom_matmul(0, fake, fake, fake, 10, 10, 10, 5, 10, 10, fake, 1 << 20, None)
    assert st == pg.ERR_ARG                      # lda < m


def test_no_cpu_fallback():
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    with pytest.raises(RuntimeError, match="no CUDA device"):
        pg.pod(torch.zeros(100, 10, dtype=torch.float64))


def test_streamed_dmd_spod_host_queries(lib):
    # streamed POD: the leaf height rule and the workspace query
    assert pg.pod_streamed_leaf_rows(1 << 22, 256, 0, 1 << 20) == max(256, 1024, (1 << 20) // 304)
    assert pg.pod_streamed_leaf_rows(1 << 22, 256, 2000, 1 << 20) == 2000
    assert pg.pod_streamed_leaf_rows(1 << 22, 256, 100, 1 << 20) == -1      # leaves shorter than M
    assert pg.pod_streamed_leaf_rows(1 << 22, 256, 0, 0) == -1               # no chunk
    small = lib.pylom_pod_streamed_workspace_size(1 << 22, 256, 0, 1 << 18, 256, pg.F64)
    large = lib.pylom_pod_streamed_workspace_size(1 << 22, 256, 0, 1 << 20, 256, pg.F64)
    assert 0 < small < large
    assert lib.pylom_pod_streamed_workspace_size(1 << 22, 256, 0, 1 << 20, 257, pg.F64) == 0
    # DMD: M >= 2, 1 <= r_max <= M - 1
    assert pg.dmd_workspace_size(10000, 64, 0, 63) > 10000 * 64 * 8
    assert pg.dmd_workspace_size(10000, 64, 0, 64) == 0
    assert pg.dmd_workspace_size(10000, 1, 0, 1) == 0
    # SPOD front end: block and frequency counts of Alg. 6, as the oracle states them
    from oracle import spod as osp
    for T, npwin, nolap in [(4128, 64, 32), (100, 60, 30), (64, 64, 0), (301, 15, 5)]:
        nb, nf = ctypes.c_int64(0), ctypes.c_int64(0)
        assert lib.pylom_spod_shape(T, npwin, nolap, ctypes.byref(nb), ctypes.byref(nf)) == pg.OK
        assert (nb.value, nf.value) == osp.spod_shape(T, npwin, nolap)
    nb, nf = ctypes.c_int64(0), ctypes.c_int64(0)
    assert lib.pylom_spod_shape(10, 32, 0, ctypes.byref(nb), ctypes.byref(nf)) == pg.ERR_SHAPE   # T < npwin


def test_dmd_and_streamed_host_validation(lib):
    fake = _vp(0x100000)  # never dereferenced: validation fails first
    i64 = ctypes.c_int64(0)
    st = lib.pylom_dmd(None, 1000, 20, 1000, pg.F64, 1, 0.0, 10, 0, fake, fake, fake, 1000, fake, None, fake,
                       fake, 1 << 30, None)
    assert st == pg.ERR_ARG
    st = lib.pylom_dmd(fake, 1000, 1, 1000, pg.F64, 1, 0.0, 1, 0, fake, fake, fake, 1000, fake, None, fake,
                       fake, 1 << 30, None)
    assert st == pg.ERR_SHAPE                     # one snapshot
    st = lib.pylom_dmd(fake, 1000, 20, 1000, pg.F64, 1, 0.0, 20, 0, fake, fake, fake, 1000, fake, None, fake,
                       fake, 1 << 30, None)
    assert st == pg.ERR_SHAPE                     # r_max > M - 1
    st = lib.pylom_pod_streamed(fake, 1000, 20, 1000, pg.F64, None, 1, 0.0, 20, 0, 0, 0, fake, fake, 1000,
                                fake, fake, 20, None, ctypes.byref(i64), fake, 1 << 30, None)
    assert st == pg.ERR_SHAPE                     # chunk_rows = 0
    st = lib.pylom_pod_streamed(fake, 1000, 20, 1000, pg.F64, None, 1, 0.0, 20, 0, 0, 1000, None, fake, 1000,
                                fake, fake, 20, None, ctypes.byref(i64), fake, 1 << 30, None)
    assert st == pg.ERR_ARG                       # no host scratch
