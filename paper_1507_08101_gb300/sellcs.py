"""ctypes binding of the C ABI in ``include/sellcs.h``.

Argument marshalling only: every step of the product runs in the CUDA
library.  Functions carry the C names (``sp_mat_create_csr``, ``sp_spmv``,
...); :class:`SellMatrix` and :func:`spmv` wrap them for torch tensors, whose
device memory and current stream are passed through as raw pointers.  If the
library has not been built the import of this module still works, but the
first call raises -- there is no fallback.
"""
from __future__ import annotations

import ctypes as ct
import os

import numpy as np

from . import build as _build

# ------------------------------------------------------------------ constants (mirror of sellcs.h)
SP_OK = 0
SP_ERR_ARG, SP_ERR_DIM, SP_ERR_DTYPE, SP_ERR_CUDA, SP_ERR_OOM, SP_ERR_TIMEOUT, SP_ERR_FORMAT, \
    SP_ERR_UNSUPPORTED = -1, -2, -3, -4, -5, -6, -7, -8
SP_F64, SP_F32, SP_BF16 = 0, 1, 2
SP_ROW_MAJOR, SP_COL_MAJOR = 0, 1
SP_MAT_CSR_ON_DEVICE, SP_MAT_VAL_F32, SP_MAT_WITH_TRANSPOSE = 1, 2, 4
SP_MAT_ORDER_FRONT, SP_MAT_ORDER_RANGES = 8, 16
SP_MAT_PERMUTED_SPACE = 32
ORDERS = {"auto": 0, "front": SP_MAT_ORDER_FRONT, "ranges": SP_MAT_ORDER_RANGES}
SP_SPMV_SCALE = 1 << 0
SP_SPMV_SHIFT = 1 << 1
SP_SPMV_VSHIFT = 1 << 2
SP_SPMV_AXPBY = 1 << 3
SP_SPMV_DOT_YY = 1 << 4
SP_SPMV_DOT_XY = 1 << 5
SP_SPMV_DOT_XX = 1 << 6
SP_SPMV_CHAIN_AXPBY = 1 << 7
SP_SPMV_DOT_HOST = 1 << 8
SP_SPMV_DOT_ANY = SP_SPMV_DOT_YY | SP_SPMV_DOT_XY | SP_SPMV_DOT_XX

DTYPES = {"f64": SP_F64, "f32": SP_F32, "bf16": SP_BF16}


class sp_mat_info_t(ct.Structure):
    _fields_ = [("nrows", ct.c_int64), ("ncols", ct.c_int64), ("nnz", ct.c_int64), ("nchunks", ct.c_int64),
                ("nstored", ct.c_int64), ("C", ct.c_int32), ("maxrowlen", ct.c_int32), ("sigma", ct.c_int64),
                ("val_dtype", ct.c_int), ("has_transpose", ct.c_int32)]


class sp_spmv_opts(ct.Structure):
    _fields_ = [("flags", ct.c_uint32), ("alpha", ct.c_double), ("beta", ct.c_double), ("delta", ct.c_double),
                ("eta", ct.c_double), ("gamma", ct.POINTER(ct.c_double)), ("z", ct.c_void_p),
                ("dot", ct.c_void_p)]


class sp_cg_opts_t(ct.Structure):
    _fields_ = [("tol", ct.c_double), ("inner_tol", ct.c_double), ("max_outer", ct.c_int32),
                ("max_inner", ct.c_int32), ("graph_iters", ct.c_int32), ("inner_f64", ct.c_int32)]


class sp_cg_stats_t(ct.Structure):
    _fields_ = [("outer", ct.c_int32), ("inner", ct.c_int32), ("graph_launches", ct.c_int32),
                ("converged", ct.c_int32), ("max_rel_residual", ct.c_double)]


SP_BATCH_MAX_W = 8
SP_MAX_VSHIFT = 1024
SP_NOALLOC_MAX_W = 32
SP_DOT_RUN_F32 = 32  # float32-vector dots: longest float run of rows per lane


class SpError(RuntimeError):
    def __init__(self, code, what):
        self.code = code
        super().__init__(f"{what}: {sp_error_string(code)} ({code}) {sp_last_error_detail()}")


_lib = None
P = ct.c_void_p
PP = ct.POINTER(ct.c_void_p)
I = ct.c_int
I32 = ct.c_int32
I64 = ct.c_int64
U = ct.c_uint

_SIGS = {
    "sp_error_string": (ct.c_char_p, [I]),
    "sp_last_error_detail": (ct.c_char_p, []),
    "sp_device_sm_count": (I, [ct.POINTER(I)]),
    "sp_device_fp64_rate": (I, [ct.POINTER(ct.c_double), ct.POINTER(ct.c_double), P]),
    "sp_mat_create_csr": (I, [PP, I64, I64, P, P, P, I, I64, I, U, P]),
    "sp_mat_update_values": (I, [P, P, U, P]),
    "sp_mat_clone_values": (I, [PP, P, I, P]),
    "sp_mat_info": (I, [P, ct.POINTER(sp_mat_info_t)]),
    "sp_mat_export_sell": (I, [P, P, P, P, P, P, P, P]),
    "sp_mat_export_sell_transpose": (I, [P, P, P, P, P, P, P, P]),
    "sp_mat_to_csr": (I, [P, P, P, P, P]),
    "sp_mat_destroy": (I, [P, P]),
    "sp_dense_create": (I, [PP, I64, I32, I, I, P]),
    "sp_dense_view": (I, [PP, P, I64, I32, I64, I, I]),
    "sp_dense_view_cols": (I, [PP, P, I32, I32]),
    "sp_dense_data": (I, [P, PP, ct.POINTER(I64), ct.POINTER(I32), ct.POINTER(I64), ct.POINTER(I), ct.POINTER(I)]),
    "sp_dense_destroy": (I, [P, P]),
    "sp_dense_view_scattered": (I, [PP, P, I32, P]),
    "sp_dense_columns": (I, [P, P]),
    "sp_dense_clone": (I, [PP, P, I, P]),
    "sp_dense_copy": (I, [P, P, P]),
    "sp_spmv": (I, [P, P, P, ct.POINTER(sp_spmv_opts), P]),
    "sp_spmv_adjoint": (I, [P, P, P, P, P, P]),
    "sp_spmv_vty": (I, [P, P, P, ct.POINTER(sp_spmv_opts), P, P, I64, P]),
    "sp_batch_create": (I, [PP, I, P, P, P, I, P]),
    "sp_batch_bind": (I, [P, P, P, P, P]),
    "sp_batch_spmv": (I, [P, ct.c_uint32, ct.c_double, ct.c_double, P, P]),
    "sp_batch_info": (I, [P, P, P, P]),
    "sp_batch_destroy": (I, [P, P]),
    "sp_cg_create": (I, [PP, I, P, P, P, P, P]),
    "sp_cg_solve": (I, [P, P, P, ct.POINTER(sp_cg_opts_t), ct.POINTER(sp_cg_stats_t), P, P]),
    "sp_cg_destroy": (I, [P, P]),
    "sp_spmv_noalloc": (I, [P, I, P, P, P, P, I64, I64, I32, P, I64, P, I64, P, I64, I32, I, ct.c_uint32,
                            ct.c_double, ct.c_double, ct.POINTER(ct.c_double), ct.c_double, ct.c_double, P, P]),
    "sp_kpm_moments": (I, [P, P, I32, ct.c_double, ct.c_double, P, P]),
    "sp_mat_permute": (I, [P, P, P, I, P]),
    "sp_tsmttsm": (I, [P, P, P, ct.c_double, ct.c_double, I, P]),
    "sp_tsmm": (I, [P, P, P, ct.c_double, ct.c_double, P]),
    "sp_host_plan_create": (I, [PP, P, I32, I]),
    "sp_spmv_host": (I, [P, P, P, P, P, P, P, ct.POINTER(sp_spmv_opts)]),
    "sp_host_plan_sync": (I, [P]),
    "sp_host_plan_destroy": (I, [P]),
    "sp_dist_partition": (I, [I64, P, I, P, I, P]),
    "sp_dist_plan_create": (I, [PP, I64, I, P, I, P, P]),
    "sp_dist_plan_info": (I, [P, P, P, P, P, P]),
    "sp_dist_plan_halo": (I, [P, P, P]),
    "sp_dist_plan_columns": (I, [P, P]),
    "sp_dist_plan_split": (I, [P, P, P, P, P, P, P, P]),
    "sp_dist_plan_set_sends": (I, [P, P, P]),
    "sp_dist_plan_sends": (I, [P, P, P]),
    "sp_dist_plan_destroy": (I, [P]),
    "sp_dist_pack": (I, [P, P, P, P]),
    "sp_dist_split_opts": (I, [ct.POINTER(sp_spmv_opts), ct.POINTER(sp_spmv_opts), ct.POINTER(sp_spmv_opts)]),
    "sp_dist_spmv": (I, [P, P, P, P, ct.POINTER(sp_spmv_opts), P, P]),
}


def library_path() -> str:
    return _build.LIB


def lib():
    """The loaded CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library not built ({path}); run paper_1507_08101_gb300.build.build()")
        L = ct.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def exported_symbols():
    return list(_SIGS)


def device_fp64_rate(stream=None):
    """(TFLOP/s, ms) of the float64 fused multiply-add micro-benchmark."""
    t, ms = ct.c_double(), ct.c_double()
    check(lib().sp_device_fp64_rate(ct.byref(t), ct.byref(ms), _stream(stream)), "sp_device_fp64_rate")
    return t.value, ms.value


def sp_error_string(code: int) -> str:
    return lib().sp_error_string(code).decode()


def sp_last_error_detail() -> str:
    return lib().sp_last_error_detail().decode()


def check(rc: int, what: str):
    if rc != SP_OK:
        raise SpError(rc, what)


def _stream(stream):
    import torch
    if stream is None:
        return ct.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ct.c_void_p(stream)
    return ct.c_void_p(stream.cuda_stream)


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data_as(ct.c_void_p)
    return ct.c_void_p(a.data_ptr())


# ------------------------------------------------------------------ raw names


def sp_mat_create_csr(nrows, ncols, rowptr, col, val, C, sigma, val_dtype, flags, stream=None):
    h = ct.c_void_p()
    check(lib().sp_mat_create_csr(ct.byref(h), nrows, ncols, _ptr(rowptr), _ptr(col), _ptr(val), C, sigma,
                                  val_dtype, flags, _stream(stream)), "sp_mat_create_csr")
    return h


def sp_dense_view(t, layout=SP_ROW_MAJOR):
    """View of a 1-D or 2-D CUDA tensor (float64/float32), row-major by default.

    A column-major view of an (n, w) tensor expects its transposed strides
    (t.t() contiguous)."""
    import torch
    if t.dim() == 1:
        n, w, ld = t.shape[0], 1, 1
        if layout == SP_COL_MAJOR:
            ld = n
    elif layout == SP_ROW_MAJOR:
        n, w = t.shape
        assert t.stride(1) == 1, "row-major view needs unit column stride"
        ld = t.stride(0) if n > 1 else w
    else:
        n, w = t.shape
        assert t.stride(0) == 1, "column-major view needs unit row stride"
        ld = t.stride(1) if w > 1 else n
    dt = {torch.float64: SP_F64, torch.float32: SP_F32}[t.dtype]
    h = ct.c_void_p()
    check(lib().sp_dense_view(ct.byref(h), _ptr(t), n, w, max(ld, 1), dt, layout), "sp_dense_view")
    return h


def sp_dense_destroy(h, stream=None):
    check(lib().sp_dense_destroy(h, _stream(stream)), "sp_dense_destroy")


def sp_device_sm_count():
    n = ct.c_int()
    check(lib().sp_device_sm_count(ct.byref(n)), "sp_device_sm_count")
    return n.value


# ------------------------------------------------------------------ matrix wrapper


class SellMatrix:
    """Owning handle of a SELL-C-sigma matrix built from CSR arrays.

    ``csr`` is any object with nrows, ncols, rowptr, col, val (host numpy), or
    a tuple (nrows, ncols, rowptr, col, val) of CUDA tensors (then the CSR is
    read on the device)."""

    def __init__(self, csr, C=32, sigma=1, dtype="f64", with_transpose=False, stream=None, order="auto",
                 permuted=False):
        import torch
        self._lib = lib()
        flags = (SP_MAT_WITH_TRANSPOSE if with_transpose else 0) | ORDERS[order]
        if permuted:
            flags |= SP_MAT_PERMUTED_SPACE
        if isinstance(csr, tuple):
            nrows, ncols, rowptr, col, val = csr
            flags |= SP_MAT_CSR_ON_DEVICE
            if val.dtype == torch.float32:
                flags |= SP_MAT_VAL_F32
            keep = (rowptr, col, val)
        else:
            nrows, ncols = csr.nrows, csr.ncols
            rowptr = np.ascontiguousarray(csr.rowptr, np.int64)
            col = np.ascontiguousarray(csr.col, np.int32)
            val = np.ascontiguousarray(csr.val)
            if val.dtype == np.float32:
                flags |= SP_MAT_VAL_F32
            else:
                val = val.astype(np.float64, copy=False)
            keep = (rowptr, col, val)
        self.handle = sp_mat_create_csr(nrows, ncols, keep[0], keep[1], keep[2], C, sigma, DTYPES[dtype], flags,
                                        stream)
        self.dtype = dtype

    @classmethod
    def _from_handle(cls, h, dtype):
        obj = cls.__new__(cls)
        obj._lib = lib()
        obj.handle = h
        obj.dtype = dtype
        return obj

    def info(self) -> dict:
        inf = sp_mat_info_t()
        check(self._lib.sp_mat_info(self.handle, ct.byref(inf)), "sp_mat_info")
        return {f: getattr(inf, f) for f, _ in sp_mat_info_t._fields_}

    @property
    def shape(self):
        i = self.info()
        return i["nrows"], i["ncols"]

    def export_sell(self, transpose=False, stream=None) -> dict:
        i = self.info()
        if transpose:
            i = self.transpose_info()
        nch, C, nst = i["nchunks"], i["C"], i["nstored"]
        out = dict(chunkptr=np.empty(nch + 1, np.int64), chunklen=np.empty(nch, np.int32),
                   slotlen=np.empty(nch * C, np.int32), perm=np.empty(nch * C, np.int32),
                   col=np.empty(nst, np.int32), val=np.empty(nst, np.float64))
        fn = self._lib.sp_mat_export_sell_transpose if transpose else self._lib.sp_mat_export_sell
        check(fn(self.handle, *[_ptr(out[k]) for k in ("chunkptr", "chunklen", "slotlen", "perm", "col", "val")],
                 _stream(stream)), "sp_mat_export_sell")
        return out

    def transpose_info(self) -> dict:
        i = self.info()
        assert i["has_transpose"]
        e = dict(nrows=i["ncols"], ncols=i["nrows"], C=i["C"])
        # sizes of the transpose come from its own export; compute from a dry export of chunk counts
        nch = (e["nrows"] + e["C"] - 1) // e["C"]
        cp = np.empty(nch + 1, np.int64)
        check(self._lib.sp_mat_export_sell_transpose(self.handle, _ptr(cp), None, None, None, None, None,
                                                     _stream(None)), "sp_mat_export_sell_transpose")
        e.update(nchunks=nch, nstored=int(cp[-1]))
        return e

    def to_csr(self, stream=None):
        i = self.info()
        rp = np.empty(i["nrows"] + 1, np.int64)
        col = np.empty(i["nnz"], np.int32)
        val = np.empty(i["nnz"], np.float64)
        check(self._lib.sp_mat_to_csr(self.handle, _ptr(rp), _ptr(col), _ptr(val), _stream(stream)),
              "sp_mat_to_csr")
        return rp, col, val

    def update_values(self, val, stream=None):
        import torch
        flags = 0
        if isinstance(val, torch.Tensor):
            assert val.is_cuda and val.is_contiguous()
            flags |= SP_MAT_CSR_ON_DEVICE
            if val.dtype == torch.float32:
                flags |= SP_MAT_VAL_F32
            else:
                assert val.dtype == torch.float64
        else:
            val = np.ascontiguousarray(val)
            if val.dtype == np.float32:
                flags |= SP_MAT_VAL_F32
            else:
                val = val.astype(np.float64, copy=False)
        check(self._lib.sp_mat_update_values(self.handle, _ptr(val), flags, _stream(stream)),
              "sp_mat_update_values")

    def clone(self, dtype: str, stream=None) -> "SellMatrix":
        h = ct.c_void_p()
        check(self._lib.sp_mat_clone_values(ct.byref(h), self.handle, DTYPES[dtype], _stream(stream)),
              "sp_mat_clone_values")
        return SellMatrix._from_handle(h, dtype)

    def close(self):
        if getattr(self, "handle", None):
            self._lib.sp_mat_destroy(self.handle, _stream(None))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ product


def make_opts(w, *, alpha=None, gamma=None, beta=None, dot_yy=False, dot_xy=False, dot_xx=False, z_handle=None,
              delta=None, eta=None, dot_ptr=None, dot_host=False):
    o = sp_spmv_opts()
    f = 0
    o.alpha, o.beta, o.delta, o.eta = 1.0, 0.0, 0.0, 1.0
    keep = []
    if alpha is not None:
        f |= SP_SPMV_SCALE
        o.alpha = float(alpha)
    if gamma is not None:
        g = np.atleast_1d(np.asarray(gamma, np.float64))
        if g.size == 1 and w != 1:
            f |= SP_SPMV_SHIFT
        elif g.size == 1:
            f |= SP_SPMV_SHIFT
        else:
            assert g.size == w
            f |= SP_SPMV_VSHIFT
        g = np.ascontiguousarray(g)
        keep.append(g)
        o.gamma = g.ctypes.data_as(ct.POINTER(ct.c_double))
    if beta is not None:
        f |= SP_SPMV_AXPBY
        o.beta = float(beta)
    if dot_yy:
        f |= SP_SPMV_DOT_YY
    if dot_xy:
        f |= SP_SPMV_DOT_XY
    if dot_xx:
        f |= SP_SPMV_DOT_XX
    if z_handle is not None:
        f |= SP_SPMV_CHAIN_AXPBY
        o.z = z_handle
        o.delta = float(delta)
        o.eta = float(eta)
    if dot_host:
        f |= SP_SPMV_DOT_HOST
    o.flags = f
    o.dot = dot_ptr
    return o, keep


def spmv(A: SellMatrix, x, y, *, alpha=None, gamma=None, beta=None, dot_yy=False, dot_xy=False, dot_xx=False,
         z=None, delta=None, eta=None, dot=None, layout=SP_ROW_MAJOR, stream=None):
    """y = alpha (A - gamma I) x + beta y (+ dots into ``dot``, + z = delta z + eta y).

    x, y, z: CUDA tensors (n,) or (n, w); dot: CUDA float64 tensor of 3*w
    (written at [yy | xy | xx]).  Returns ``dot``."""
    L = lib()
    hx = sp_dense_view(x, layout)
    hy = sp_dense_view(y, layout)
    hz = sp_dense_view(z, layout) if z is not None else None
    w = 1 if x.dim() == 1 else x.shape[1]
    try:
        if (dot_yy or dot_xy or dot_xx) and dot is None:
            import torch
            dot = torch.full((3 * w,), float("nan"), dtype=torch.float64, device=x.device)
        o, keep = make_opts(w, alpha=alpha, gamma=gamma, beta=beta, dot_yy=dot_yy, dot_xy=dot_xy, dot_xx=dot_xx,
                            z_handle=hz, delta=delta, eta=eta, dot_ptr=_ptr(dot) if dot is not None else None)
        check(L.sp_spmv(hy, A.handle, hx, ct.byref(o), _stream(stream)), "sp_spmv")
    finally:
        L.sp_dense_destroy(hx, None)
        L.sp_dense_destroy(hy, None)
        if hz is not None:
            L.sp_dense_destroy(hz, None)
    return dot


def spmv_vty(A: SellMatrix, x, y, V, C, *, alpha=None, gamma=None, beta=None, z=None, delta=None, eta=None,
             stream=None):
    """y = alpha (A - gamma I) x + beta y (+ z = delta z + eta y) and C = V^T y
    in one pass (sp_spmv_vty); x, y, z: CUDA float64 (n,) or (n, w); V: (n, m);
    C: CUDA float64 (m, w) written.  Returns C."""
    L = lib()
    hx, hy, hv = sp_dense_view(x), sp_dense_view(y), sp_dense_view(V if V.dim() == 2 else V[:, None])
    hz = sp_dense_view(z) if z is not None else None
    w = 1 if x.dim() == 1 else x.shape[1]
    try:
        o, keep = make_opts(w, alpha=alpha, gamma=gamma, beta=beta, z_handle=hz, delta=delta, eta=eta)
        ldc = C.stride(0) if C.dim() == 2 else 1
        check(L.sp_spmv_vty(hy, A.handle, hx, ct.byref(o), hv, _ptr(C), int(max(ldc, w)), _stream(stream)),
              "sp_spmv_vty")
    finally:
        for h in (hx, hy, hv, hz):
            if h is not None:
                L.sp_dense_destroy(h, None)
    return C


def mat_permute(A: SellMatrix, out, inp, to_sell: bool, stream=None):
    """out = inp in A's SELL row order (to_sell) or back in the user's order
    (sp_mat_permute); CUDA tensors (n,) or (n, w), row-major."""
    L = lib()
    ho, hi = sp_dense_view(out), sp_dense_view(inp)
    try:
        check(L.sp_mat_permute(A.handle, ho, hi, 1 if to_sell else 0, _stream(stream)), "sp_mat_permute")
    finally:
        L.sp_dense_destroy(ho, None)
        L.sp_dense_destroy(hi, None)
    return out


def tsmttsm(X, V, W, alpha=1.0, beta=0.0, kahan=False, stream=None):
    """X <- alpha V^T W + beta X (sp_tsmttsm); CUDA tensors, row-major."""
    L = lib()
    hx, hv, hw = sp_dense_view(X), sp_dense_view(V), sp_dense_view(W)
    try:
        check(L.sp_tsmttsm(hx, hv, hw, float(alpha), float(beta), 1 if kahan else 0, _stream(stream)), "sp_tsmttsm")
    finally:
        for h in (hx, hv, hw):
            L.sp_dense_destroy(h, None)
    return X


def tsmm(W, V, X, alpha=1.0, beta=0.0, stream=None):
    """W <- alpha V X + beta W (sp_tsmm; W may be V); CUDA tensors, row-major."""
    L = lib()
    # separate views even when V is W: the library recognises the in-place
    # form by the shared storage and checks that the shapes agree
    hw, hv, hx = sp_dense_view(W), sp_dense_view(V), sp_dense_view(X)
    try:
        check(L.sp_tsmm(hw, hv, hx, float(alpha), float(beta), _stream(stream)), "sp_tsmm")
    finally:
        for h in (hw, hv, hx):
            L.sp_dense_destroy(h, None)
    return W


def kpm_moments(A: SellMatrix, x, nmom: int, a: float, b: float, stream=None) -> np.ndarray:
    """Chebyshev moments mu[k, c] = <x_c, T_k((A - b I) / a) x_c> (sp_kpm_moments);
    x: CUDA tensor (n,) or (n, w), row-major.  Returns an (nmom, w) array."""
    L = lib()
    w = 1 if x.dim() == 1 else x.shape[1]
    hx = sp_dense_view(x)
    mu = np.empty((int(nmom), w), np.float64)
    try:
        check(L.sp_kpm_moments(A.handle, hx, int(nmom), float(a), float(b), ct.c_void_p(mu.ctypes.data),
                               _stream(stream)), "sp_kpm_moments")
    finally:
        L.sp_dense_destroy(hx, None)
    return mu


def _host_ptr(a):
    """Address of a host (CPU) array: torch CPU tensor or numpy array, or None."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        assert not a.is_cuda, "host plan buffers live in host memory"
        return ct.c_void_p(a.data_ptr())
    return ct.c_void_p(a.ctypes.data)


class HostPlan:
    """Pipelined products over block vectors in host memory (sp_host_plan_*).

    ``spmv`` only enqueues (copy-in, product, copy-out on the plan's streams);
    the host buffers must stay untouched until ``sync``.  Page-locked buffers
    (torch ``pin_memory()``) let the copies of consecutive calls overlap."""

    def __init__(self, A: SellMatrix, w: int, vec_dtype: str = "f64"):
        self._lib = lib()
        self.A = A
        self.w = int(w)
        h = ct.c_void_p()
        check(self._lib.sp_host_plan_create(ct.byref(h), A.handle, self.w, DTYPES[vec_dtype]), "sp_host_plan_create")
        self.handle = h
        self._keep = []

    def spmv(self, x, y_out, *, y_in=None, alpha=None, gamma=None, beta=None, dot_yy=False, dot_xy=False,
             dot_xx=False, z_in=None, z_out=None, delta=None, eta=None, dot=None):
        o, keep = make_opts(self.w, alpha=alpha, gamma=gamma, beta=beta, dot_yy=dot_yy, dot_xy=dot_xy, dot_xx=dot_xx)
        if z_in is not None:
            o.flags |= SP_SPMV_CHAIN_AXPBY
            o.delta, o.eta = float(delta), float(eta)
        self._keep.append((x, y_in, y_out, z_in, z_out, dot))
        check(self._lib.sp_spmv_host(self.handle, _host_ptr(x), _host_ptr(y_in), _host_ptr(y_out), _host_ptr(z_in),
                                     _host_ptr(z_out), _host_ptr(dot), ct.byref(o)), "sp_spmv_host")

    def sync(self):
        check(self._lib.sp_host_plan_sync(self.handle), "sp_host_plan_sync")
        self._keep.clear()

    def close(self):
        if getattr(self, "handle", None):
            self._lib.sp_host_plan_destroy(self.handle)
            self.handle = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def spmv_adjoint(A: SellMatrix, g, x=None, dx=None, dvals=None, stream=None):
    """dx = A^T g (into ``dx``) and dvals[p] = sum_k g[row p] x[col p] (into ``dvals``)."""
    L = lib()
    hg = sp_dense_view(g)
    hx = sp_dense_view(x) if x is not None else None
    hdx = sp_dense_view(dx) if dx is not None else None
    try:
        check(L.sp_spmv_adjoint(hdx, _ptr(dvals) if dvals is not None else None, A.handle, hx, hg,
                                _stream(stream)), "sp_spmv_adjoint")
    finally:
        for h in (hg, hx, hdx):
            if h is not None:
                L.sp_dense_destroy(h, None)


# ------------------------------------------------------------------ batches


def _ptr_array(ptrs):
    arr = (ct.c_void_p * len(ptrs))()
    for i, p in enumerate(ptrs):
        arr[i] = p if isinstance(p, int) else (p.value if isinstance(p, ct.c_void_p) else p.data_ptr())
    return arr


class Batch:
    """Many SELL matrices multiplied in one persistent launch (sp_batch_*)."""

    def __init__(self, mats, widths, cols_per_lane=None, vec_dtype="f64", stream=None):
        self._lib = lib()
        self.mats = list(mats)  # keep alive
        self.count = len(self.mats)
        self.widths = np.ascontiguousarray(widths, np.int32)
        cpl = None if cols_per_lane is None else np.ascontiguousarray(cols_per_lane, np.int32)
        h = ct.c_void_p()
        check(self._lib.sp_batch_create(ct.byref(h), self.count, _ptr_array([m.handle.value for m in self.mats]),
                                        _ptr(self.widths), _ptr(cpl), DTYPES[vec_dtype], _stream(stream)),
              "sp_batch_create")
        self.handle = h

    def bind(self, xs, ys, y0s=None, stream=None):
        self._bound = (list(xs), list(ys), None if y0s is None else list(y0s))
        y0 = None if y0s is None else _ptr_array(y0s)
        check(self._lib.sp_batch_bind(self.handle, _ptr_array(xs), _ptr_array(ys), y0, _stream(stream)),
              "sp_batch_bind")

    def spmv(self, flags=0, alpha=1.0, beta=0.0, dots=None, stream=None):
        check(self._lib.sp_batch_spmv(self.handle, flags, alpha, beta, _ptr(dots), _stream(stream)),
              "sp_batch_spmv")

    def info(self):
        nu, gr = ct.c_int32(), ct.c_int32()
        cpl = np.zeros(self.count, np.int32)
        check(self._lib.sp_batch_info(self.handle, ct.byref(nu), ct.byref(gr), _ptr(cpl)), "sp_batch_info")
        return {"nunits": nu.value, "grid": gr.value, "cols_per_lane": cpl}

    def close(self):
        if getattr(self, "handle", None):
            self._lib.sp_batch_destroy(self.handle, _stream(None))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class CG:
    """Batched mixed-precision CG with iterative refinement (sp_cg_*)."""

    def __init__(self, mats, widths, cpl64=None, cpl32=None, stream=None):
        self._lib = lib()
        self.mats = list(mats)
        self.count = len(self.mats)
        self.widths = np.ascontiguousarray(widths, np.int32)
        c64 = None if cpl64 is None else np.ascontiguousarray(cpl64, np.int32)
        c32 = None if cpl32 is None else np.ascontiguousarray(cpl32, np.int32)
        h = ct.c_void_p()
        check(self._lib.sp_cg_create(ct.byref(h), self.count, _ptr_array([m.handle.value for m in self.mats]),
                                     _ptr(self.widths), _ptr(c64), _ptr(c32), _stream(stream)), "sp_cg_create")
        self.handle = h

    def solve(self, bs, xs, tol=1e-10, inner_tol=1e-4, max_outer=40, max_inner=20000, graph_iters=16,
              inner_f64=False, stream=None):
        o = sp_cg_opts_t(tol, inner_tol, max_outer, max_inner, graph_iters, int(inner_f64))
        st = sp_cg_stats_t()
        rel = np.zeros(int(self.widths.sum()))
        check(self._lib.sp_cg_solve(self.handle, _ptr_array(bs), _ptr_array(xs), ct.byref(o), ct.byref(st),
                                    _ptr(rel), _stream(stream)), "sp_cg_solve")
        return {f: getattr(st, f) for f, _ in sp_cg_stats_t._fields_}, rel

    def close(self):
        if getattr(self, "handle", None):
            self._lib.sp_cg_destroy(self.handle, _stream(None))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
