"""GB300 (sm_103a) wide/tall sparse SpMV and SpVTM (arXiv 1812.00904).

The functions below carry the names of the C ABI in ``include/spmv_gb300.h``
and only marshal arguments: tensors become device pointers, streams become
``cudaStream_t`` handles.  :class:`Plan` keeps the borrowed arrays alive for
the plan's lifetime; :class:`SparseMatVec` is the autograd form of y = A x
whose backward pass is the SpVTM kernel (dx) plus the dvalues kernel.
"""
from __future__ import annotations

import ctypes

from . import _lib
from ._lib import (SPMV_BF16, SPMV_CSC_WIDE, SPMV_CSR_TALL, SPMV_F16, SPMV_F32, SPMV_F64, SPMV_OP_AX, SPMV_OP_VTA,
                   SPMV_PLAN_BANK_ORDER, SPMV_PLAN_COO_UNSORTED, SPMV_PLAN_NO_VALIDATE, SPMV_PLAN_PROFILE,
                   SPMV_PLAN_ROW_BLOCKS, SPMV_PLAN_SHORT_IN_GLOBAL, SpmvError)

__all__ = [
    "spmv_plan", "spmv_plan_ex", "spmv_plan_coo", "spmv_plan_destroy", "spmv_plan_info", "spmv_plan_chunks", "spmv", "spvtm", "spmv_pair",
    "spmv_batch", "spmv_dvalues", "spmv_noalloc", "spmv_normal", "spmv_cgls", "spmv_check", "spmv_plan_export", "spmv_profile_read", "spmv_profile_reset", "spmv_profile_enable", "spmv_last_error",
    "spmv_version", "serve_create", "serve_register", "serve_register_host", "serve_submit", "serve_poll",
    "serve_wait", "serve_stats", "serve_destroy", "Plan", "SparseMatVec", "sparse_matvec", "SpmvError",
    "SPMV_CSC_WIDE", "SPMV_CSR_TALL", "SPMV_F64", "SPMV_F32", "SPMV_BF16", "SPMV_F16", "SPMV_OP_AX", "SPMV_OP_VTA",
    "SPMV_PLAN_NO_VALIDATE", "SPMV_PLAN_PROFILE", "SPMV_PLAN_SHORT_IN_GLOBAL", "SPMV_PLAN_BANK_ORDER",
    "SPMV_PLAN_COO_UNSORTED", "SPMV_PLAN_ROW_BLOCKS",
]


def _addr(a):
    """Address of a tensor / numpy array / int (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, int):
        return a
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    if hasattr(a, "ctypes"):
        return a.ctypes.data
    raise TypeError(f"cannot take the address of {type(a)}")


def _stream(s):
    if s is None:
        import torch

        return torch.cuda.current_stream().cuda_stream
    if isinstance(s, int):
        return s
    return s.cuda_stream


def dtype_code(dt) -> int:
    import torch

    table = {torch.float64: SPMV_F64, torch.float32: SPMV_F32, torch.bfloat16: SPMV_BF16, torch.float16: SPMV_F16}
    if dt not in table:
        raise TypeError(f"unsupported dtype {dt}")
    return table[dt]


# ---------------------------------------------------------------------------
# C ABI, same names


def spmv_plan(m, n, nnz, layout, ptr, idx, vals, val_dtype, vec_dtype, stream=None, flags=0):
    h = ctypes.c_void_p()
    _lib.call("spmv_plan", ctypes.byref(h), m, n, nnz, layout, _addr(ptr), _addr(idx), _addr(vals), val_dtype,
              vec_dtype, _stream(stream), flags)
    return h.value


def spmv_plan_ex(m, n, nnz, layout, ptr, idx, vals, val_dtype, vec_dtype, stream=None, flags=0, chunks=0,
                 warps_per_cta=0, tile_items=0, stages=0, chunk_tiles=0):
    h = ctypes.c_void_p()
    opts = _lib.spmv_plan_opts(chunks, warps_per_cta, tile_items, stages, chunk_tiles)
    _lib.call("spmv_plan_ex", ctypes.byref(h), m, n, nnz, layout, _addr(ptr), _addr(idx), _addr(vals), val_dtype,
              vec_dtype, _stream(stream), flags, ctypes.byref(opts))
    return h.value


def spmv_plan_coo(m, n, nnz, layout, rows, cols, vals, val_dtype, vec_dtype, stream=None, flags=0, chunks=0,
                  warps_per_cta=0, tile_items=0, stages=0, chunk_tiles=0):
    h = ctypes.c_void_p()
    opts = _lib.spmv_plan_opts(chunks, warps_per_cta, tile_items, stages, chunk_tiles)
    _lib.call("spmv_plan_coo", ctypes.byref(h), m, n, nnz, layout, _addr(rows), _addr(cols), _addr(vals), val_dtype,
              vec_dtype, _stream(stream), flags, ctypes.byref(opts))
    return h.value


def spmv_plan_destroy(plan):
    _lib.call("spmv_plan_destroy", plan)


def spmv_plan_info(plan) -> dict:
    info = _lib.spmv_plan_info_t()
    _lib.call("spmv_plan_info", plan, ctypes.byref(info))
    return info.as_dict()


def spmv_plan_chunks(plan, count: int):
    arr = (_lib.spmv_chunk_t * count)()
    _lib.call("spmv_plan_chunks", plan, arr, count)
    return [{k: getattr(c, k) for k, _ in _lib.spmv_chunk_t._fields_} for c in arr]


def spmv(plan, x, y, stream=None):
    _lib.call("spmv", plan, _addr(x), _addr(y), _stream(stream))


def spvtm(plan, v, u, stream=None):
    _lib.call("spvtm", plan, _addr(v), _addr(u), _stream(stream))


def spmv_pair(plan, x, y, v, u, stream=None):
    """y = A x and u = v^T A for independent x and v in one call (host vectors' copies overlap
    the other product's kernels)."""
    _lib.call("spmv_pair", plan, _addr(x), _addr(y), _addr(v), _addr(u), _stream(stream))


def spmv_batch(plan, op, k, inp, ld_in, out, ld_out, stream=None):
    _lib.call("spmv_batch", plan, op, k, _addr(inp), ld_in, _addr(out), ld_out, _stream(stream))


def spmv_dvalues(plan, r, x, g, stream=None):
    _lib.call("spmv_dvalues", plan, _addr(r), _addr(x), _addr(g), _stream(stream))


def spmv_check(plan, stream=None):
    _lib.call("spmv_check", plan, _stream(stream))


def spmv_plan_export(plan, idx_out, vals_out, stream=None):
    _lib.call("spmv_plan_export", plan, _addr(idx_out), _addr(vals_out), _stream(stream))


def spmv_profile_enable(plan, on):
    _lib.call("spmv_profile_enable", plan, 1 if on else 0)


def spmv_profile_read(plan, kernel: int):
    ms = ctypes.c_double()
    n = ctypes.c_int64()
    _lib.call("spmv_profile_read", plan, kernel, ctypes.byref(ms), ctypes.byref(n))
    return ms.value, n.value


def spmv_profile_reset(plan):
    _lib.call("spmv_profile_reset", plan)


def spmv_noalloc(m, n, nnz, ptr, idx, vals, x, y, stream=None):
    """y = A x (wide CSC, FP32) with no device allocation: scratch in the library's static device memory."""
    _lib.call("spmv_noalloc", m, n, nnz, _addr(ptr), _addr(idx), _addr(vals), _addr(x), _addr(y), _stream(stream))


def spmv_normal(plan, x, u, y=None, stream=None):
    """u = A^T (A x); y (optional) receives A x."""
    _lib.call("spmv_normal", plan, _addr(x), _addr(u), _addr(y), _stream(stream))


def spmv_cgls(plan, b, x, max_iters, tol, stream=None):
    """Least squares by CGLS on the device; x is updated in place.  Returns (iterations, ||A^T r|| / ||A^T r0||)."""
    it = ctypes.c_int32()
    rel = ctypes.c_double()
    _lib.call("spmv_cgls", plan, _addr(b), _addr(x), int(max_iters), float(tol), _stream(stream), ctypes.byref(it),
              ctypes.byref(rel))
    return it.value, rel.value


def spmv_last_error() -> str:
    return _lib.load().spmv_last_error().decode()


def spmv_version() -> str:
    return _lib.load().spmv_version().decode()


def serve_create(hbm_budget_bytes: int, k_max: int = 32, n_streams: int = 4):
    h = ctypes.c_void_p()
    _lib.call("serve_create", ctypes.byref(h), int(hbm_budget_bytes), k_max, n_streams)
    return h.value


def serve_register(srv, plan) -> int:
    mid = ctypes.c_int32()
    _lib.call("serve_register", srv, plan, ctypes.byref(mid))
    return mid.value


def serve_register_host(srv, m, n, nnz, layout, ptr, idx, vals, val_dtype, vec_dtype) -> int:
    mid = ctypes.c_int32()
    _lib.call("serve_register_host", srv, m, n, nnz, layout, _addr(ptr), _addr(idx), _addr(vals), val_dtype,
              vec_dtype, ctypes.byref(mid))
    return mid.value


def serve_submit(srv, mat_id, op, k, inp, out) -> int:
    rid = ctypes.c_uint64()
    _lib.call("serve_submit", srv, mat_id, op, k, _addr(inp), _addr(out), ctypes.byref(rid))
    return rid.value


def serve_poll(srv, req_id):
    done = ctypes.c_int32()
    lat = ctypes.c_double()
    _lib.call("serve_poll", srv, req_id, ctypes.byref(done), ctypes.byref(lat))
    return bool(done.value), lat.value


def serve_wait(srv, req_id, timeout_ms: int = 10000):
    _lib.call("serve_wait", srv, req_id, timeout_ms)


def serve_stats(srv) -> dict:
    st = _lib.serve_stats_t()
    _lib.call("serve_stats", srv, ctypes.byref(st))
    return st.as_dict()


def serve_destroy(srv):
    _lib.call("serve_destroy", srv)


# ---------------------------------------------------------------------------
# convenience: a plan that owns references to its borrowed device tensors


class Plan:
    """Plan over torch device tensors ``ptr``/``idx``/``vals`` (CSC for layout "csc", CSR for "csr")."""

    def __init__(self, m, n, ptr, idx, vals, layout="csc", vec_dtype=None, flags=0, chunks=0, warps_per_cta=0,
                 tile_items=0, stages=0, stream=None, chunk_tiles=0):
        import torch

        self.m, self.n = int(m), int(n)
        self.layout = SPMV_CSC_WIDE if layout in ("csc", SPMV_CSC_WIDE) else SPMV_CSR_TALL
        self.ptr, self.idx, self.vals = ptr, idx, vals
        self.val_dtype = vals.dtype
        if vec_dtype is None:
            vec_dtype = torch.float64 if vals.dtype == torch.float64 else torch.float32
        self.vec_dtype = vec_dtype
        self.nnz = int(idx.numel())
        self.handle = spmv_plan_ex(self.m, self.n, self.nnz, self.layout, ptr, idx, vals, dtype_code(vals.dtype),
                                   dtype_code(vec_dtype), stream, flags, chunks, warps_per_cta, tile_items, stages,
                                   chunk_tiles)

    @classmethod
    def from_matrix(cls, A, **kw):
        return cls(A.m, A.n, A.ptr, A.idx, A.vals, layout=A.layout, **kw)

    @classmethod
    def from_coo(cls, m, n, rows, cols, vals, layout="csc", vec_dtype=None, flags=0, stream=None, **opts):
        """Plan from device triples sorted by column ("csc") or by row ("csr"), or in any order with
        ``flags=SPMV_PLAN_COO_UNSORTED``; the plan builds the pointer array."""
        import torch

        self = cls.__new__(cls)
        self.m, self.n = int(m), int(n)
        self.layout = SPMV_CSC_WIDE if layout in ("csc", SPMV_CSC_WIDE) else SPMV_CSR_TALL
        self.rows, self.cols, self.vals = rows, cols, vals
        self.idx = rows if self.layout == SPMV_CSC_WIDE else cols
        self.ptr = None
        self.val_dtype = vals.dtype
        self.vec_dtype = vec_dtype or (torch.float64 if vals.dtype == torch.float64 else torch.float32)
        self.nnz = int(vals.numel())
        self.handle = spmv_plan_coo(self.m, self.n, self.nnz, self.layout, rows, cols, vals, dtype_code(vals.dtype),
                                    dtype_code(self.vec_dtype), stream, flags, opts.get("chunks", 0),
                                    opts.get("warps_per_cta", 0), opts.get("tile_items", 0), opts.get("stages", 0))
        return self

    def close(self):
        if getattr(self, "handle", None):
            spmv_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _empty(self, size):
        import torch

        return torch.empty(size, dtype=self.vec_dtype, device=self.vals.device)

    def spmv(self, x, out=None, stream=None):
        y = self._empty(self.m) if out is None else out
        spmv(self.handle, x, y, stream)
        return y

    def spvtm(self, v, out=None, stream=None):
        u = self._empty(self.n) if out is None else out
        spvtm(self.handle, v, u, stream)
        return u

    def batch(self, op, X, out=None, stream=None):
        """X: [k, len_in] contiguous; returns [k, len_out]."""
        import torch

        k = X.shape[0]
        len_out = self.m if op == SPMV_OP_AX else self.n
        Y = torch.empty((k, len_out), dtype=self.vec_dtype, device=X.device) if out is None else out
        spmv_batch(self.handle, op, k, X, X.stride(0), Y, Y.stride(0), stream)
        return Y

    def dvalues(self, r, x, out=None, stream=None):
        import torch

        g = torch.empty(self.nnz, dtype=self.val_dtype, device=self.vals.device) if out is None else out
        spmv_dvalues(self.handle, r, x, g, stream)
        return g

    def normal(self, x, out=None, stream=None):
        """A^T (A x)."""
        u = self._empty(self.n) if out is None else out
        spmv_normal(self.handle, x, u, None, stream)
        return u

    def cgls(self, b, x0=None, max_iters=100, tol=1e-6, stream=None):
        """Least squares min ||A x - b|| from x0 (zeros by default); returns (x, iterations, relative gradient)."""
        x = self._empty(self.n).zero_() if x0 is None else x0.clone()
        it, rel = spmv_cgls(self.handle, b, x, max_iters, tol, stream)
        return x, it, rel

    def info(self) -> dict:
        return spmv_plan_info(self.handle)

    def chunks(self):
        return spmv_plan_chunks(self.handle, self.info()["chunks"])

    def check(self, stream=None):
        spmv_check(self.handle, stream)

    def export(self, stream=None):
        """(idx, vals): device copies of the nonzeros in the plan's storage order."""
        import torch

        dev = self.vals.device
        idx = torch.empty(self.nnz, dtype=torch.int32, device=dev)
        vals = torch.empty(self.nnz, dtype=self.val_dtype, device=dev)
        spmv_plan_export(self.handle, idx, vals, stream)
        return idx, vals

    def profile(self, kernel: int):
        return spmv_profile_read(self.handle, kernel)


def _autograd():
    import torch

    class SparseMatVec(torch.autograd.Function):
        """y = A x with A's stored values as a differentiable input.

        forward:  y = A x (the chunked SpMV).
        backward: dx = A^T dy, i.e. u^T = dy^T A (the SpVTM kernel); dvalues[p] = dy_i x_j
        for the nonzero p = A_ij (the dvalues kernel).
        """

        @staticmethod
        def forward(ctx, vals, x, plan):
            if vals.data_ptr() != plan.vals.data_ptr():
                raise ValueError("the plan must be built over this values tensor")
            ctx.plan = plan
            ctx.save_for_backward(x)
            return plan.spmv(x)

        @staticmethod
        def backward(ctx, gy):
            (x,) = ctx.saved_tensors
            plan = ctx.plan
            gy = gy.contiguous()
            dvals = plan.dvalues(gy, x) if ctx.needs_input_grad[0] else None
            dx = plan.spvtm(gy) if ctx.needs_input_grad[1] else None
            return dvals, dx, None

    return SparseMatVec


class _LazyFn:
    _fn = None

    def __getattr__(self, name):
        if _LazyFn._fn is None:
            _LazyFn._fn = _autograd()
        return getattr(_LazyFn._fn, name)


SparseMatVec = _LazyFn()


def sparse_matvec(vals, x, plan):
    """Differentiable y = A(vals) x through the CUDA kernels."""
    return SparseMatVec.apply(vals, x, plan)
