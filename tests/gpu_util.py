"""Helpers of the GPU parity tests: device copies of the seeded inputs and the tolerance checks.

Tolerances (per element, against the FP64 oracle run on the same stored values
and the same input vectors):
    |gpu_i - ref_i| <= tol * scale_i + tiny,   scale_i = sum_j |a_ij x_j|
with tol = 1e-12 for FP64 and 1e-5 for FP32 accumulation (BF16/FP16 values
accumulate in FP32); BF16/FP16 results are also held to 1e-2 normwise against
the oracle on the unrounded FP64 values.
"""
from __future__ import annotations

import numpy as np
import torch

import oracle
import synth
import paper_1812_00904_gb300 as pkg

DEV = torch.device("cuda:0")
TOL = {torch.float64: 1e-12, torch.float32: 1e-5, torch.bfloat16: 1e-5, torch.float16: 1e-5}


def vec_dtype_for(val_dtype):
    return torch.float64 if val_dtype == torch.float64 else torch.float32


def device_matrix(A: synth.SparseMatrix, val_dtype=torch.float32):
    """Copy a host matrix to the device with values rounded to val_dtype; returns (tensors, stored-values matrix)."""
    vals = torch.as_tensor(np.asarray(A.vals, dtype=np.float64)).to(val_dtype)
    t = dict(ptr=torch.from_numpy(np.ascontiguousarray(A.ptr, dtype=np.int32)).to(DEV),
             idx=torch.from_numpy(np.ascontiguousarray(A.idx, dtype=np.int32)).to(DEV),
             vals=vals.to(DEV))
    stored = synth.SparseMatrix(A.layout, A.m, A.n, A.ptr, A.idx, vals.double().numpy())
    return t, stored


def make_plan(A, val_dtype=torch.float32, **kw):
    t, stored = device_matrix(A, val_dtype)
    plan = pkg.Plan(A.m, A.n, t["ptr"], t["idx"], t["vals"], layout=A.layout, vec_dtype=vec_dtype_for(val_dtype), **kw)
    return plan, stored


def dev_vec(x: np.ndarray, dtype):
    return torch.from_numpy(np.asarray(x, dtype=np.float64)).to(dtype).to(DEV)


def host_of(t) -> np.ndarray:
    return t.detach().double().cpu().numpy()


def assert_close(got, ref, scale, tol, what=""):
    got = np.asarray(got, dtype=np.float64)
    err = np.abs(got - ref)
    bound = tol * scale + 1e-300
    bad = np.nonzero(err > bound)[0]
    if bad.size:
        i = bad[0]
        raise AssertionError(f"{what}: {bad.size} of {got.size} elements outside tolerance {tol}; first at {i}: "
                             f"got {got[i]!r} ref {ref[i]!r} scale {scale[i]!r} (max ratio "
                             f"{np.max(err / np.maximum(scale, 1e-300)):.3e})")


def check_products(plan, stored, x, v, tol, what=""):
    """SpMV and SpVTM of the plan against the oracle on the stored values and the rounded vectors."""
    xd, vd = dev_vec(x, plan.vec_dtype), dev_vec(v, plan.vec_dtype)
    y = host_of(plan.spmv(xd))
    u = host_of(plan.spvtm(vd))
    plan.check()
    xs, vs = host_of(xd), host_of(vd)
    assert_close(y, oracle.spmv(stored, xs), oracle.abs_spmv(stored, xs), tol, f"spmv {what}")
    assert_close(u, oracle.spvtm(stored, vs), oracle.abs_spvtm(stored, vs), tol, f"spvtm {what}")
    return y, u
