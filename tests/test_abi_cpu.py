"""The C ABI library builds, loads without a GPU, exports every function the
header declares, and rejects bad arguments on the host before touching CUDA."""
import ctypes as ct
import os
import re

import pytest

from tests.conftest import ROOT

HEADER = os.path.join(ROOT, "include", "sellcs.h")


def declared_functions():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"^SP_API\s+[\w\s\*]*?\b(sp_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def L():
    from paper_1507_08101_gb300 import build, sellcs
    build.build()
    return sellcs.lib()


def test_header_declares_api():
    names = declared_functions()
    for n in ("sp_mat_create_csr", "sp_spmv", "sp_dense_view", "sp_spmv_adjoint", "sp_mat_export_sell"):
        assert n in names
    assert len(names) >= 18


def test_every_declared_symbol_is_exported(L):
    from paper_1507_08101_gb300 import sellcs
    for n in declared_functions():
        assert hasattr(L, n), n
        assert n in sellcs.exported_symbols(), f"binding lacks {n}"


def test_binding_constants_match_header():
    """Every integer #define of the header that the binding mirrors has the same value there."""
    from paper_1507_08101_gb300 import sellcs
    defs = dict(re.findall(r"^#define\s+(SP_\w+)\s+(\d+)\s*(?:/\*.*)?$", open(HEADER).read(), flags=re.M))
    shared = [n for n in defs if hasattr(sellcs, n)]
    assert {"SP_DOT_RUN_F32", "SP_NOALLOC_MAX_W", "SP_MAX_VSHIFT"} <= set(shared)
    for n in shared:
        assert getattr(sellcs, n) == int(defs[n]), n


def test_error_strings(L):
    from paper_1507_08101_gb300 import sellcs
    assert sellcs.sp_error_string(0) == "ok"
    assert "malformed" in sellcs.sp_error_string(sellcs.SP_ERR_FORMAT)
    assert sellcs.sp_error_string(-99) == "unknown error"


def test_host_argument_checks(L):
    from paper_1507_08101_gb300 import sellcs as s
    h = ct.c_void_p()
    rp = (ct.c_int64 * 2)(0, 0)
    # null output handle / bad chunk height / bad sigma / bad dtype: rejected before any CUDA call
    assert L.sp_mat_create_csr(None, 1, 1, rp, None, None, 32, 1, 0, 0, None) == s.SP_ERR_ARG
    assert L.sp_mat_create_csr(ct.byref(h), 1, 1, rp, None, None, 0, 1, 0, 0, None) == s.SP_ERR_ARG
    assert L.sp_mat_create_csr(ct.byref(h), 1, 1, rp, None, None, 2048, 1, 0, 0, None) == s.SP_ERR_ARG
    assert L.sp_mat_create_csr(ct.byref(h), 1, 1, rp, None, None, 32, 0, 0, 0, None) == s.SP_ERR_ARG
    assert L.sp_mat_create_csr(ct.byref(h), 1, 1, rp, None, None, 32, 1, 7, 0, None) == s.SP_ERR_DTYPE
    assert L.sp_mat_create_csr(ct.byref(h), -1, 1, rp, None, None, 32, 1, 0, 0, None) == s.SP_ERR_DIM
    assert L.sp_mat_create_csr(ct.byref(h), 1, 1, rp, None, None, 32, 1, 0, 1 << 9, None) == s.SP_ERR_ARG
    assert L.sp_kpm_moments(None, None, 4, 1.0, 0.0, None, None) == s.SP_ERR_ARG
    assert L.sp_host_plan_create(None, None, 1, s.SP_F64) == s.SP_ERR_ARG
    assert L.sp_spmv_host(None, None, None, None, None, None, None, None) == s.SP_ERR_ARG
    assert L.sp_host_plan_sync(None) == s.SP_ERR_ARG
    assert L.sp_host_plan_destroy(None) == s.SP_ERR_ARG
    pt = s.SP_MAT_PERMUTED_SPACE | s.SP_MAT_WITH_TRANSPOSE  # the adjoint works in the user's order
    assert L.sp_mat_create_csr(ct.byref(h), 1, 1, rp, None, None, 32, 1, 0, pt, None) == s.SP_ERR_ARG
    assert L.sp_mat_create_csr(ct.byref(h), 1, 2, rp, None, None, 32, 1, 0, s.SP_MAT_PERMUTED_SPACE,
                               None) == s.SP_ERR_DIM  # square only
    assert L.sp_mat_permute(None, None, None, 1, None) == s.SP_ERR_ARG
    assert L.sp_tsmttsm(None, None, None, 1.0, 0.0, 0, None) == s.SP_ERR_ARG
    assert L.sp_tsmm(None, None, None, 1.0, 0.0, None) == s.SP_ERR_ARG
    both = s.SP_MAT_ORDER_FRONT | s.SP_MAT_ORDER_RANGES  # at most one work order
    assert L.sp_mat_create_csr(ct.byref(h), 1, 1, rp, None, None, 32, 1, 0, both, None) == s.SP_ERR_ARG
    # dense views: ld too small, bf16 vectors, null pointer
    buf = ct.c_void_p(0x1000)
    assert L.sp_dense_view(ct.byref(h), buf, 10, 4, 3, s.SP_F64, s.SP_ROW_MAJOR) == s.SP_ERR_DIM
    assert L.sp_dense_view(ct.byref(h), buf, 10, 4, 9, s.SP_F64, s.SP_COL_MAJOR) == s.SP_ERR_DIM
    assert L.sp_dense_view(ct.byref(h), buf, 10, 4, 4, s.SP_BF16, s.SP_ROW_MAJOR) == s.SP_ERR_DTYPE
    assert L.sp_dense_view(ct.byref(h), None, 10, 4, 4, s.SP_F64, s.SP_ROW_MAJOR) == s.SP_ERR_ARG
    # a valid view of a fake address never dereferences it
    assert L.sp_dense_view(ct.byref(h), buf, 10, 4, 4, s.SP_F64, s.SP_ROW_MAJOR) == 0
    v = ct.c_void_p()
    assert L.sp_dense_view_cols(ct.byref(v), h, 3, 2) == s.SP_ERR_DIM
    assert L.sp_dense_view_cols(ct.byref(v), h, 1, 2) == 0
    p = ct.c_void_p()
    ld = ct.c_int64()
    assert L.sp_dense_data(v, ct.byref(p), None, None, ct.byref(ld), None, None) == 0
    assert p.value == 0x1000 + 8 and ld.value == 4
    assert L.sp_dense_destroy(v, None) == 0
    assert L.sp_dense_destroy(h, None) == 0
    assert L.sp_spmv(None, None, None, None, None) == s.SP_ERR_ARG


def test_scattered_view_arguments_without_gpu(L):
    """Scattered views are host bookkeeping: their checks need no device."""
    import numpy as np
    from paper_1507_08101_gb300 import sellcs as s
    base = ct.c_void_p()
    assert L.sp_dense_view(ct.byref(base), ct.c_void_p(4096), 10, 6, 6, s.SP_F64, s.SP_ROW_MAJOR) == s.SP_OK
    v = ct.c_void_p()
    bad = np.array([1, 6], np.int32)
    assert L.sp_dense_view_scattered(ct.byref(v), base, 2, s._ptr(bad)) == s.SP_ERR_DIM
    rep = np.array([1, 1], np.int32)
    assert L.sp_dense_view_scattered(ct.byref(v), base, 2, s._ptr(rep)) == s.SP_ERR_ARG
    cols = np.array([5, 1, 3], np.int32)
    assert L.sp_dense_view_scattered(ct.byref(v), base, 3, s._ptr(cols)) == s.SP_OK
    got = np.empty(3, np.int32)
    assert L.sp_dense_columns(v, s._ptr(got)) == 1
    assert got.tolist() == [5, 1, 3]
    # a run of a scattered view, and a scattered view of a scattered view
    r = ct.c_void_p()
    assert L.sp_dense_view_cols(ct.byref(r), v, 1, 2) == s.SP_OK
    assert L.sp_dense_columns(r, s._ptr(got[:2])) == 1 and got[:2].tolist() == [1, 3]
    q = ct.c_void_p()
    sel = np.array([2, 0], np.int32)
    assert L.sp_dense_view_scattered(ct.byref(q), v, 2, s._ptr(sel)) == s.SP_OK
    assert L.sp_dense_columns(q, s._ptr(got[:2])) == 1 and got[:2].tolist() == [3, 5]
    assert L.sp_dense_columns(base, None) == 0
    for h in (q, r, v, base):
        L.sp_dense_destroy(h, None)
