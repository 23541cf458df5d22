"""Seeded synthetic inputs for the wide-CSC / tall-CSR sparse products.

This module is shared by the CUDA path's tests and benchmark and by the FP64
oracle's tests.  It holds none of the products' arithmetic: it only draws
random sparsity structure, values and dense vectors, and assembles them into
compressed-sparse arrays.

Matrices are described by :class:`SparseMatrix`:

* ``layout == "csc"`` (wide, m << n): ``ptr`` has n+1 entries, column j holds
  the nonzeros ``ptr[j]:ptr[j+1]`` with row ids in ``idx`` (Sec. II: a wide
  matrix stored in column-major order).
* ``layout == "csr"`` (tall, m >> n): ``ptr`` has m+1 entries, row i holds
  ``ptr[i]:ptr[i+1]`` with column ids in ``idx`` (Sec. II: the same method with
  the roles of rows and columns reversed).

All index arrays are int32 and 0-based.  Within each compressed segment the
indices are distinct and sorted ascending.

Workload recipes (document-term-like, standing in for the paper's News20
matrix, Sec. VI):

* ``wide_fp64_small`` -- m=1,000, n=100,000, FP64.  Column degrees Zipf(2)
  clipped to [1, 1000]; 5 fully dense columns at seeded random positions;
  rows uniform without replacement; values U(0,1); x, v ~ U(-1,1).
* ``wide_fp32_large`` -- m=20,000, n=5,000,000, FP32 values.  Column degree a
  discrete bounded power law with density exponent 2 (tail P(D>=d) =
  (d_min/d)^1), capped at m, with d_min chosen so that the expected total is
  about 200M nonzeros; 50 dense columns at 50% density; values lognormal(0,1).
* ``tall_fp32_large`` -- m=10,000,000, n=2,000, CSR, FP32.  Row degree power
  law with density exponent 2.2 capped at n, expected total about 150M; 20
  dense rows at 60% density; values lognormal(0,1).
* ``serving_specs`` -- 64 matrices with m, n and Z log-uniform in the serving
  ranges, wide or tall with equal odds.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

__all__ = [
    "SparseMatrix",
    "power_law_dmin",
    "power_law_degrees",
    "zipf_degrees",
    "random_matrix",
    "wide_fp64_small",
    "wide_fp32_large",
    "tall_fp32_large",
    "serving_specs",
    "uniform_vector",
]


@dataclasses.dataclass
class SparseMatrix:
    """Compressed sparse matrix (arrays are numpy or torch, host or device)."""

    layout: str  # "csc" (wide) or "csr" (tall)
    m: int
    n: int
    ptr: object  # int32 [major + 1]
    idx: object  # int32 [nnz]
    vals: object  # [nnz] float64 / float32 / bfloat16 / float16
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.idx.shape[0])

    @property
    def n_major(self) -> int:
        return self.n if self.layout == "csc" else self.m

    @property
    def n_minor(self) -> int:
        return self.m if self.layout == "csc" else self.n

    def to_numpy(self) -> "SparseMatrix":
        def cv(a):
            if isinstance(a, np.ndarray):
                return a
            import torch

            a = a.detach()
            if a.dtype in (torch.bfloat16,):
                return a.float().cpu().numpy()
            return a.cpu().numpy()

        return SparseMatrix(self.layout, self.m, self.n, cv(self.ptr), cv(self.idx), cv(self.vals), self.name)


# ----------------------------------------------------------------------------
# degree laws


def power_law_expected(d_min: float, alpha: float, cap: int) -> float:
    """E[min(cap, floor(d_min * U**(-1/alpha)))] for U ~ U(0,1], d_min >= 1."""
    k = np.arange(1, cap + 1, dtype=np.float64)
    return float(np.minimum(1.0, (d_min / k) ** alpha).sum())


def power_law_dmin(mean: float, exponent: float, cap: int) -> float:
    """d_min of the bounded discrete power law whose expectation is ``mean``.

    ``exponent`` is the density exponent gamma (P(D=d) ~ d^-gamma), so the
    tail exponent is alpha = gamma - 1.
    """
    alpha = exponent - 1.0
    lo, hi = 1.0, float(cap)
    if power_law_expected(lo, alpha, cap) >= mean:
        return lo
    for _ in range(100):
        mid = 0.5 * (lo + hi)
        if power_law_expected(mid, alpha, cap) < mean:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def power_law_degrees(count: int, exponent: float, cap: int, mean: float, rng: np.random.Generator) -> np.ndarray:
    d_min = power_law_dmin(mean, exponent, cap)
    alpha = exponent - 1.0
    u = 1.0 - rng.random(count)  # (0, 1]
    d = np.floor(d_min * u ** (-1.0 / alpha))
    return np.minimum(d, cap).astype(np.int64)


def zipf_degrees(count: int, a: float, lo: int, hi: int, rng: np.random.Generator) -> np.ndarray:
    d = rng.zipf(a, count)
    return np.clip(d, lo, hi).astype(np.int64)


# ----------------------------------------------------------------------------
# distinct sorted indices per segment (numpy, host)


def _distinct_rows_numpy(deg: np.ndarray, m: int, rng: np.random.Generator) -> np.ndarray:
    """For each segment s draw deg[s] distinct ids in [0, m), uniformly.

    Returns the int64 keys ``s * m + id`` sorted ascending (so segment-major
    with sorted ids).  Segments with deg > m/2 draw a random-key permutation;
    the others draw with replacement and redraw the shortfall until every
    segment holds deg[s] distinct ids.
    """
    deg = deg.astype(np.int64)
    nseg = deg.shape[0]
    heavy = np.nonzero(deg > m // 2)[0]
    light_deg = deg.copy()
    light_deg[heavy] = 0
    keys = np.empty(0, dtype=np.int64)
    need = light_deg.copy()
    while need.sum() > 0:
        seg = np.repeat(np.arange(nseg, dtype=np.int64), need)
        ids = rng.integers(0, m, size=seg.shape[0], dtype=np.int64)
        keys = np.unique(np.concatenate([keys, seg * m + ids]))
        have = np.bincount(keys // m, minlength=nseg)
        need = light_deg - have
        if (need < 0).any():  # cannot happen: unique keys per segment <= drawn
            raise AssertionError("overfull segment")
    parts = [keys]
    for s in heavy:
        ids = np.argsort(rng.random(m))[: deg[s]]
        parts.append(np.int64(s) * m + np.sort(ids).astype(np.int64))
    keys = np.sort(np.concatenate(parts))
    return keys


def _assemble_numpy(deg: np.ndarray, keys: np.ndarray, m_minor: int):
    nseg = deg.shape[0]
    ptr = np.zeros(nseg + 1, dtype=np.int64)
    np.cumsum(deg, out=ptr[1:])
    idx = (keys % m_minor).astype(np.int32)
    return ptr.astype(np.int32), idx


# ----------------------------------------------------------------------------
# distinct sorted indices per segment (torch, any device)


def _distinct_rows_torch(deg, m: int, gen, device):
    import torch

    deg = deg.to(torch.int64)
    nseg = deg.shape[0]
    heavy_mask = deg > (m // 2)
    light = torch.where(heavy_mask, torch.zeros_like(deg), deg)
    keys = torch.empty(0, dtype=torch.int64, device=device)
    need = light.clone()
    segs = torch.arange(nseg, dtype=torch.int64, device=device)
    while int(need.sum()) > 0:
        seg = torch.repeat_interleave(segs, need)
        ids = torch.randint(0, m, (seg.shape[0],), generator=gen, device=device, dtype=torch.int64)
        keys = torch.unique(torch.cat([keys, seg * m + ids]))  # sorted
        have = torch.bincount(keys // m, minlength=nseg)
        need = light - have
    parts = [keys]
    heavy = torch.nonzero(heavy_mask).flatten()
    # heavy segments: random-key permutation, in batches bounded in memory
    hb = max(1, (1 << 26) // max(m, 1))
    for b in range(0, heavy.shape[0], hb):
        hs = heavy[b : b + hb]
        r = torch.rand((hs.shape[0], m), generator=gen, device=device)
        order = torch.argsort(r, dim=1)
        take = torch.arange(m, device=device).unsqueeze(0) < deg[hs].unsqueeze(1)
        ids = order[take]
        seg = torch.repeat_interleave(hs, deg[hs])
        parts.append(seg * m + ids)
        del r, order, take
    keys = torch.sort(torch.cat(parts)).values
    return keys


def _assemble_torch(deg, keys, m_minor: int):
    import torch

    nseg = deg.shape[0]
    ptr = torch.zeros(nseg + 1, dtype=torch.int64, device=deg.device)
    ptr[1:] = torch.cumsum(deg.to(torch.int64), 0)
    idx = (keys % m_minor).to(torch.int32)
    return ptr.to(torch.int32), idx


# ----------------------------------------------------------------------------
# small random matrices for tests


def random_matrix(
    m: int,
    n: int,
    layout: str = "csc",
    density: float = 0.1,
    dtype=np.float64,
    seed: int = 0,
    int_values: Optional[int] = None,
    degrees: Optional[np.ndarray] = None,
    duplicates: bool = False,
) -> SparseMatrix:
    """Small random sparse matrix on the host (numpy arrays).

    ``int_values=K`` draws integer values in [-K, K] (so products and sums are
    exact in FP32/FP64 as long as they stay below 2^24 / 2^53).  ``degrees``
    overrides the per-segment nonzero counts.  ``duplicates=True`` allows
    repeated indices inside a segment (the products then add up).
    """
    rng = np.random.default_rng(seed)
    n_major, n_minor = (n, m) if layout == "csc" else (m, n)
    if degrees is None:
        deg = rng.binomial(n_minor, density, size=n_major).astype(np.int64) if n_minor > 0 else np.zeros(n_major, np.int64)
    else:
        deg = np.asarray(degrees, dtype=np.int64)
        assert deg.shape[0] == n_major
    if duplicates:
        ptr = np.zeros(n_major + 1, dtype=np.int64)
        np.cumsum(deg, out=ptr[1:])
        idx = rng.integers(0, max(n_minor, 1), size=int(ptr[-1])).astype(np.int32)
        ptr = ptr.astype(np.int32)
    else:
        assert (deg <= n_minor).all()
        keys = _distinct_rows_numpy(deg, n_minor, rng) if deg.sum() > 0 else np.empty(0, np.int64)
        ptr, idx = _assemble_numpy(deg, keys, max(n_minor, 1))
    z = idx.shape[0]
    if int_values is not None:
        vals = rng.integers(-int_values, int_values + 1, size=z).astype(np.float64)
    else:
        vals = rng.uniform(-1.0, 1.0, size=z)
    vals = _cast_np(vals, dtype)
    return SparseMatrix(layout, m, n, ptr, idx, vals, name=f"random_{layout}_{m}x{n}")


def _cast_np(vals: np.ndarray, dtype):
    if dtype in ("bf16", "bfloat16"):
        import torch

        return torch.from_numpy(np.asarray(vals, dtype=np.float32)).to(torch.bfloat16)
    return np.asarray(vals).astype(dtype)


def uniform_vector(size: int, seed: int, dtype=np.float64, lo: float = -1.0, hi: float = 1.0, int_values: Optional[int] = None):
    rng = np.random.default_rng(seed)
    if int_values is not None:
        return rng.integers(-int_values, int_values + 1, size=size).astype(dtype)
    return rng.uniform(lo, hi, size=size).astype(dtype)


# ----------------------------------------------------------------------------
# the paper-shaped workloads


def wide_fp64_small(seed: int = 0) -> SparseMatrix:
    """m=1,000 x n=100,000 wide CSC, FP64 values (about 0.5M nonzeros).

    Column degrees Zipf(2.0) clipped to [1, 1000]; 5 columns at seeded random
    positions are made fully dense (1,000 nonzeros each); row ids uniform
    without replacement, sorted; values U(0, 1).
    """
    m, n = 1000, 100_000
    rng = np.random.default_rng(seed)
    deg = zipf_degrees(n, 2.0, 1, m, rng)
    dense = rng.choice(n, size=5, replace=False)
    deg[dense] = m
    keys = _distinct_rows_numpy(deg, m, rng)
    ptr, idx = _assemble_numpy(deg, keys, m)
    vals = rng.uniform(0.0, 1.0, size=idx.shape[0])
    return SparseMatrix("csc", m, n, ptr, idx, vals, name="wide_csc_m1000_n100000_fp64")


def _large_torch(layout: str, n_major: int, n_minor: int, exponent: float, target_nnz: float,
                 n_dense: int, dense_frac: float, seed: int, device, value_dtype, name: str,
                 scale: float = 1.0) -> SparseMatrix:
    import torch

    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    rng = np.random.default_rng(seed)
    n_major_s = max(1, int(round(n_major * scale)))
    dense_deg = int(round(dense_frac * n_minor))
    mean = (target_nnz * scale - n_dense * dense_deg) / max(1, n_major_s - n_dense)
    d_min = power_law_dmin(mean, exponent, n_minor)
    alpha = exponent - 1.0
    u = 1.0 - torch.rand(n_major_s, generator=gen, device=device, dtype=torch.float64)
    deg = torch.clamp(torch.floor(d_min * u ** (-1.0 / alpha)), max=n_minor).to(torch.int64)
    dense = torch.from_numpy(rng.choice(n_major_s, size=min(n_dense, n_major_s), replace=False)).to(device)
    deg[dense] = dense_deg
    keys = _distinct_rows_torch(deg, n_minor, gen, device)
    ptr, idx = _assemble_torch(deg, keys, n_minor)
    del keys
    vals = torch.empty(idx.shape[0], dtype=torch.float32, device=device)
    vals.log_normal_(0.0, 1.0, generator=gen)
    vals = vals.to(value_dtype)
    if layout == "csc":
        m, n = n_minor, n_major_s
    else:
        m, n = n_major_s, n_minor
    return SparseMatrix(layout, m, n, ptr, idx, vals, name=name)


def wide_fp32_large(seed: int = 1, device="cuda", scale: float = 1.0, value_dtype=None) -> SparseMatrix:
    """m=20,000 x n=5,000,000 wide CSC, FP32 values, about 200M nonzeros.

    ``scale`` < 1 keeps the column count (and expected nonzeros) in that
    proportion, for bounded samples of the same workload.
    """
    import torch

    return _large_torch("csc", 5_000_000, 20_000, 2.0, 200e6, 50, 0.5, seed, device,
                        value_dtype or torch.float32, "wide_csc_m20000_n5000000_fp32", scale)


def wide_fp32_short(m: int = 2000, seed: int = 5, device="cuda", scale: float = 0.25) -> SparseMatrix:
    """The recipe of wide_fp32_large with a short dimension of m rows (2,000 by default), so that
    8 short vectors (m x 8 x 4 B) fit in one SM's shared memory; ``scale`` of the 5M columns
    (a quarter by default: about 50M nonzeros)."""
    import torch

    return _large_torch("csc", 5_000_000, m, 2.0, 200e6, 50, 0.5, seed, device, torch.float32,
                        f"wide_csc_m{m}_n5000000_fp32", scale)


def tall_fp32_large(seed: int = 2, device="cuda", scale: float = 1.0, value_dtype=None) -> SparseMatrix:
    """m=10,000,000 x n=2,000 tall CSR, FP32 values, about 150M nonzeros."""
    import torch

    return _large_torch("csr", 10_000_000, 2_000, 2.2, 150e6, 20, 0.6, seed, device,
                        value_dtype or torch.float32, "tall_csr_m10000000_n2000_fp32", scale)


def serving_specs(seed: int = 4, count: int = 64, budget_bytes: float = 120e9):
    """Shapes of the resident serving matrices: list of dicts.

    m in [1k, 50k], n in [100k, 5M] (multiples of 4), Z in [1M, 100M] (each log-uniform), Z
    capped at m*n/4; wide CSC or tall CSR with equal odds (a tall matrix
    swaps the roles: its long dimension is the row count).  The total stored
    bytes (8 per nonzero plus the pointer array) stay under ``budget_bytes``.
    """
    rng = np.random.default_rng(seed)
    specs = []
    total = 0.0
    for i in range(count):
        # dimensions rounded to multiples of 4, so that the vectors of a k-vector request
        # packed back to back each start on a 16-byte boundary
        short = 4 * int(round(math.exp(rng.uniform(math.log(1e3), math.log(5e4))) / 4))
        long_ = 4 * int(round(math.exp(rng.uniform(math.log(1e5), math.log(5e6))) / 4))
        z = int(round(math.exp(rng.uniform(math.log(1e6), math.log(1e8)))))
        z = min(z, short * long_ // 4)
        layout = "csc" if rng.random() < 0.5 else "csr"
        m, n = (short, long_) if layout == "csc" else (long_, short)
        b = 8.0 * z + 4.0 * (long_ + 1)
        if total + b > budget_bytes:
            z = max(1_000_000, int((budget_bytes - total - 4.0 * (long_ + 1)) / 8.0))
            b = 8.0 * z + 4.0 * (long_ + 1)
        total += b
        specs.append(dict(id=i, layout=layout, m=m, n=n, nnz=z, seed=seed * 1000 + i))
    return specs


def serving_matrix(spec: dict, device="cuda", exponent: float = 2.0) -> SparseMatrix:
    """One serving matrix of the given spec (power-law degrees, FP32 values)."""
    import torch

    layout = spec["layout"]
    short = spec["m"] if layout == "csc" else spec["n"]
    long_ = spec["n"] if layout == "csc" else spec["m"]
    return _large_torch(layout, long_, short, exponent, float(spec["nnz"]), 0, 0.0, spec["seed"], device,
                        torch.float32, f"serve_{spec['id']}_{layout}_{spec['m']}x{spec['n']}")
