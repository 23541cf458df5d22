"""FP64 CPU oracle for the wide/tall sparse products (arXiv 1812.00904).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by the package smoke check
and by the benchmark's CPU-baseline leg, never by the product library.  It
shares no code with the CUDA path; both receive their inputs from the seeded
generators in ``synth``.

* ``spmv`` / ``spvtm`` / ``dvalues`` call straight FP64 loops in ``oracle.c``
  (Sec. I problem statement, Sec. II storage orders); ``spmv_mt`` / ``spvtm_mt``
  run the same loops over balanced column (row) ranges on several host threads,
  for timing the CPU baseline on all cores.
* :mod:`oracle.plan` restates the nonzero partition of Sec. II and the
  overlap-zone set-up of Sec. IV-B step by step.

Every function here is pinned by ``tests/test_oracle.py`` against values the
paper prints (the worked example of Figs. 1-3 and Tables II-III), dense brute
force, closed forms and algebraic identities.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from types import SimpleNamespace

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-std=c99", "-fPIC", "-shared", "-pthread", "-ffp-contract=off", "-fno-fast-math"]


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``liboracle.so`` (plain gcc, no CUDA)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *CFLAGS, _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


def load_library(path: str = None):
    """Load (building first if needed) the oracle shared library."""
    global _lib
    with _lock:
        if path is not None:
            return _declare(ctypes.CDLL(path))
        if _lib is None:
            build()
            _lib = _declare(ctypes.CDLL(_LIB))
        return _lib


def _declare(lib):
    i64, p = ctypes.c_int64, ctypes.c_void_p
    for name in ("oracle_csc_matvec", "oracle_csc_vecmat", "oracle_csr_matvec", "oracle_csr_vecmat",
                 "oracle_csc_dvalues", "oracle_csr_dvalues"):
        f = getattr(lib, name)
        f.argtypes = [i64, i64, p, p, p, p, p]
        f.restype = None
    for name in ("oracle_csc_matvec_mt", "oracle_csc_vecmat_mt", "oracle_csr_matvec_mt", "oracle_csr_vecmat_mt"):
        f = getattr(lib, name, None)
        if f is not None:  # absent from mutant builds that predate them
            f.argtypes = [i64, i64, p, p, p, p, p, ctypes.c_int]
            f.restype = ctypes.c_int
    return lib


def _f64(a) -> np.ndarray:
    """Widen to a contiguous float64 host array (exact for f16/bf16/f32)."""
    if not isinstance(a, np.ndarray):
        import torch

        a = a.detach()
        if a.dtype in (torch.bfloat16, torch.float16):
            a = a.float()
        a = a.cpu().numpy()
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a) -> np.ndarray:
    if not isinstance(a, np.ndarray):
        a = a.detach().cpu().numpy()
    return np.ascontiguousarray(a, dtype=np.int32)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


class Oracle:
    """Bound oracle entry points (``lib`` may be a test-built variant)."""

    def __init__(self, lib=None):
        self.lib = lib if lib is not None else load_library()

    def _run(self, fname, A, vec_in, out_len):
        ptr, idx, val = _i32(A.ptr), _i32(A.idx), _f64(A.vals)
        vin = _f64(vec_in)
        out = np.empty(out_len, dtype=np.float64)
        getattr(self.lib, fname)(A.m, A.n, _ptr(ptr), _ptr(idx), _ptr(val), _ptr(vin), _ptr(out))
        return out

    def spmv(self, A, x) -> np.ndarray:
        """y = A x (Sec. I), FP64."""
        f = "oracle_csc_matvec" if A.layout == "csc" else "oracle_csr_matvec"
        assert len(x) == A.n
        return self._run(f, A, x, A.m)

    def spvtm(self, A, v) -> np.ndarray:
        """u = (v^T A)^T (Sec. I), FP64."""
        f = "oracle_csc_vecmat" if A.layout == "csc" else "oracle_csr_vecmat"
        assert len(v) == A.m
        return self._run(f, A, v, A.n)

    def _run_mt(self, fname, A, vec_in, out_len, threads):
        ptr, idx, val = _i32(A.ptr), _i32(A.idx), _f64(A.vals)
        vin = _f64(vec_in)
        out = np.empty(out_len, dtype=np.float64)
        rc = getattr(self.lib, fname)(A.m, A.n, _ptr(ptr), _ptr(idx), _ptr(val), _ptr(vin), _ptr(out), int(threads))
        if rc != 0:
            raise RuntimeError(f"{fname}: could not start {threads} threads")
        return out

    def spmv_mt(self, A, x, threads: int) -> np.ndarray:
        """y = A x on `threads` host threads (the serial loop over balanced column/row ranges)."""
        f = "oracle_csc_matvec_mt" if A.layout == "csc" else "oracle_csr_matvec_mt"
        assert len(x) == A.n
        return self._run_mt(f, A, x, A.m, threads)

    def spvtm_mt(self, A, v, threads: int) -> np.ndarray:
        """u = (v^T A)^T on `threads` host threads."""
        f = "oracle_csc_vecmat_mt" if A.layout == "csc" else "oracle_csr_vecmat_mt"
        assert len(v) == A.m
        return self._run_mt(f, A, v, A.n, threads)

    def dvalues(self, A, r, x) -> np.ndarray:
        """g[k] = r_i x_j for the stored nonzero k = A_ij (gradient of r^T A x)."""
        ptr, idx = _i32(A.ptr), _i32(A.idx)
        rr, xx = _f64(r), _f64(x)
        g = np.empty(idx.shape[0], dtype=np.float64)
        f = "oracle_csc_dvalues" if A.layout == "csc" else "oracle_csr_dvalues"
        getattr(self.lib, f)(A.m, A.n, _ptr(ptr), _ptr(idx), _ptr(rr), _ptr(xx), _ptr(g))
        return g

    def least_squares(self, A, x, b):
        """Loss 0.5||Ax - b||^2 and its gradients with respect to x and the values."""
        r = self.spmv(A, x) - _f64(b)
        loss = 0.5 * float(np.dot(r, r))
        return loss, self.spvtm(A, r), self.dvalues(A, r, x), r


    def cgls(self, A, b, x0, iters: int):
        """CGLS (conjugate gradients on the normal equations A^T A x = A^T b), FP64, from x0.

        Not part of the paper: the least-squares loop its SpMV-SpVTM pairs serve.  The
        standard recurrences: r = b - A x, s = A^T r, p = s, gamma = s.s; per iteration
        q = A p, alpha = gamma / q.q, x += alpha p, r -= alpha q, s = A^T r,
        gamma' = s.s, p = s + (gamma' / gamma) p.  Returns (x, ||s|| / ||s_0||).
        """
        x = _f64(x0).copy()
        r = _f64(b) - self.spmv(A, x)
        s = self.spvtm(A, r)
        p = s.copy()
        gamma0 = gamma = float(np.dot(s, s))
        for _ in range(iters):
            q = self.spmv(A, p)
            delta = float(np.dot(q, q))
            alpha = gamma / delta if delta > 0.0 else 0.0
            x += alpha * p
            r -= alpha * q
            s = self.spvtm(A, r)
            gamma_new = float(np.dot(s, s))
            beta = gamma_new / gamma if gamma > 0.0 else 0.0
            gamma = gamma_new
            p = s + beta * p
        return x, (np.sqrt(gamma / gamma0) if gamma0 > 0.0 else 0.0)


_default = None


def _get():
    global _default
    if _default is None:
        _default = Oracle()
    return _default


def spmv(A, x):
    return _get().spmv(A, x)


def spvtm(A, v):
    return _get().spvtm(A, v)


def dvalues(A, r, x):
    return _get().dvalues(A, r, x)


def spmv_mt(A, x, threads):
    return _get().spmv_mt(A, x, threads)


def spvtm_mt(A, v, threads):
    return _get().spvtm_mt(A, v, threads)


def least_squares(A, x, b):
    return _get().least_squares(A, x, b)


def cgls(A, b, x0, iters):
    return _get().cgls(A, b, x0, iters)


def abs_spmv(A, x):
    """|A| |x|: the per-element scale sum_j |A_ij x_j| used by the tolerances."""
    B = SimpleNamespace(layout=A.layout, m=A.m, n=A.n, ptr=A.ptr, idx=A.idx, vals=np.abs(_f64(A.vals)))
    return _get().spmv(B, np.abs(_f64(x)))


def abs_spvtm(A, v):
    """|v|^T |A|: the per-element scale sum_i |v_i A_ij|."""
    B = SimpleNamespace(layout=A.layout, m=A.m, n=A.n, ptr=A.ptr, idx=A.idx, vals=np.abs(_f64(A.vals)))
    return _get().spvtm(B, np.abs(_f64(v)))
