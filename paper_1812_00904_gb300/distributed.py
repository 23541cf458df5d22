"""Nonzero-partitioned products over several ranks (one process per GPU): the paper's
distributed method, with torch.distributed for the two exchange steps.

Sec. II: rank r of R holds the r-th of R contiguous groups of the nonzeros in storage order
(column-major for a wide CSC matrix, row-major for a tall CSR one; the first Z mod R groups
one nonzero larger), whatever the column boundaries, and the entries of the long vector
its columns need: its window, long-vector entries first .. last.

Products that accumulate into the short vector (Sec. III: y = A x of a wide matrix; by
role reversal u^T = v^T A of a tall one): every rank multiplies its group with its window
into a full-length short vector, and an all-reduce in FP64 adds them (step 2).

Products that dot the long dimension with the short vector (Sec. IV-A: u^T = v^T A of a
wide matrix; y = A x of a tall one): every rank dots its group's columns with the short
vector.  A column split between ranks (an overlap zone) is completed from the ranks'
partial sums: one all-gather brings every rank's partial sums of its first and last
column to all ranks, the zones come from the Sec. IV-B set-up run over the ranks' first
and last columns, and every rank of a zone adds the zone's partials in rank order in
FP64 (the first rank's last-column partial, the whole-window partials of the ranks
inside the zone, the last rank's first-column partial) and keeps the sum, so every copy
of a shared entry holds the same value.

The local products run in the CUDA library (a plan over the rank's group); the
``local`` argument replaces them, for tests on CPU ranks.
"""
from __future__ import annotations

import dataclasses
from typing import Callable, List, Optional, Tuple

import numpy as np


def group_range(nnz: int, world: int, rank: int) -> Tuple[int, int]:
    """Sec. II: the nonzeros [a, b) of group `rank` of `world` (the first nnz mod world one larger)."""
    q, r = divmod(nnz, world)
    a = rank * q + min(rank, r)
    return a, a + q + (1 if rank < r else 0)


def owner_of(ptr: np.ndarray, k: int) -> int:
    """Major index (column of a wide matrix) whose segment holds storage position k."""
    return int(np.searchsorted(ptr, k, side="right")) - 1


@dataclasses.dataclass
class ZoneSetup:
    """Sec. IV-B over the ranks: flags, group numbers and extents, and the zones (first rank,
    last rank, long-vector index) in zone order."""
    needLeft: List[int]
    needRight: List[int]
    leftGroupEnd: List[int]
    rightGroup: List[int]
    leftGroup: List[int]
    procsOnLeft: List[int]
    procsOnRight: List[int]
    zones: List[Tuple[int, int, int]]


def zone_setup(first: List[int], last: List[int], nonempty: List[bool]) -> ZoneSetup:
    """The overlap-zone set-up of Sec. IV-B from every rank's first and last column.

    needLeft_r: rank r's first column is rank r-1's last; needRight_r: its last column is
    rank r+1's first (empty ranks have neither).  leftGroupEnd_r marks the rank that closes
    a zone on the right (needLeft and, unless the rank holds a single column, not needRight);
    rightGroup is the inclusive running count of those and leftGroup = rightGroup -
    leftGroupEnd.  procsOnLeft (procsOnRight) counts the ranks further left (right) in the
    same zone: the segmented running sum (s, k) o (t, l) = (s + t, l) if k == l, else (t, l),
    of (needLeft, leftGroup) forward and of (needRight, rightGroup) backward.
    """
    R = len(first)
    nl = [1 if (r > 0 and nonempty[r] and nonempty[r - 1] and first[r] == last[r - 1]) else 0 for r in range(R)]
    nr = [1 if (r < R - 1 and nonempty[r] and nonempty[r + 1] and last[r] == first[r + 1]) else 0 for r in range(R)]
    lge = [1 if (nl[r] and (not nr[r] or first[r] != last[r])) else 0 for r in range(R)]
    rg, lg, run = [], [], 0
    for r in range(R):
        run += lge[r]
        rg.append(run)
        lg.append(run - lge[r])

    def seg_scan(vals, keys, order):
        out = [0] * R
        acc = None
        for r in order:
            cur = (vals[r], keys[r])
            acc = cur if acc is None else ((acc[0] + cur[0], cur[1]) if acc[1] == cur[1] else cur)
            out[r] = acc[0]
        return out

    pol = seg_scan(nl, lg, range(R))
    por = seg_scan(nr, rg, range(R - 1, -1, -1))
    zones = [(r - pol[r], r, first[r]) for r in range(R) if lge[r]]
    return ZoneSetup(nl, nr, lge, rg, lg, pol, por, zones)


class _DeviceLocal:
    """The rank's group as a plan of the CUDA library."""

    def __init__(self, layout, m, n, ptr, idx, vals, device, flags, vec_dtype):
        import torch

        from . import Plan

        self.m, self.n = m, n
        self.ptr = torch.from_numpy(np.ascontiguousarray(ptr, dtype=np.int32)).to(device)
        self.idx = torch.from_numpy(np.ascontiguousarray(idx, dtype=np.int32)).to(device)
        self.vals = torch.as_tensor(vals).to(device)
        self.plan = Plan(m, n, self.ptr, self.idx, self.vals, layout=layout, flags=flags, vec_dtype=vec_dtype)

    def spmv(self, x):
        return self.plan.spmv(x)

    def spvtm(self, v):
        return self.plan.spvtm(v)


class DistributedMatrix:
    """The rank's share of a wide (CSC) or tall (CSR) matrix and the two distributed products.

    ptr is the global pointer array (host, every rank reads it to find its group); idx and
    vals are the global index and value arrays, of which only the rank's group is read.

    Wide CSC:  spmv(x_window) -> y (all m entries, the same on every rank);
               spvtm(v) -> u_window (entries first .. last of u, zones completed).
    Tall CSR:  spmv(x) -> y_window (rows first .. last of y, zones completed);
               spvtm(v_window) -> u (all n entries, the same on every rank).
    """

    def __init__(self, layout: str, m: int, n: int, ptr, idx, vals, group=None, device=None, flags: int = 0,
                 local: Optional[Callable] = None, vec_dtype=None):
        import torch
        import torch.distributed as dist

        self.layout, self.m, self.n = layout, int(m), int(n)
        self.group = group
        self.world = dist.get_world_size(group)
        self.rank = dist.get_rank(group)
        ptr = np.asarray(ptr, dtype=np.int64)
        nnz = int(ptr[-1])
        self.a, self.b = group_range(nnz, self.world, self.rank)
        self.nonempty = self.b > self.a
        if self.nonempty:
            self.first, self.last = owner_of(ptr, self.a), owner_of(ptr, self.b - 1)
        else:
            self.first, self.last = 0, -1
        n_local = self.last - self.first + 1
        lptr = np.clip(ptr[self.first:self.last + 2], self.a, self.b) - self.a if self.nonempty else np.zeros(1)
        lidx = np.asarray(idx[self.a:self.b])
        lvals = vals[self.a:self.b]
        self.short = self.m if layout == "csc" else self.n
        self.n_local = max(n_local, 0)
        self.device = device if device is not None else torch.device("cpu")
        lm, ln = (self.short, self.n_local) if layout == "csc" else (self.n_local, self.short)
        if not self.nonempty:
            self.local = None
        elif local is not None:
            self.local = local(layout, lm, ln, lptr, lidx, lvals)
        else:
            self.local = _DeviceLocal(layout, lm, ln, lptr, lidx, lvals, self.device, flags, vec_dtype)
        # Sec. IV-B over the ranks: every rank's first and last column, by one all-gather
        mine = torch.tensor([self.first, self.last, 1 if self.nonempty else 0], dtype=torch.int64,
                            device=self._comm_device())
        allv = [torch.empty_like(mine) for _ in range(self.world)]
        dist.all_gather(allv, mine, group=group)
        rows = [t.cpu().tolist() for t in allv]
        self.setup = zone_setup([r[0] for r in rows], [r[1] for r in rows], [bool(r[2]) for r in rows])

    def _comm_device(self):
        import torch.distributed as dist

        return self.device if dist.get_backend(self.group) == "nccl" else "cpu"

    @property
    def window(self) -> Tuple[int, int]:
        """Long-vector entries first .. last held by this rank (first > last when the group is empty)."""
        return self.first, self.last

    # ---- Sec. III: per-rank short vectors, added by an FP64 all-reduce
    def _accumulate(self, w):
        import torch
        import torch.distributed as dist

        if self.local is None:
            part = torch.zeros(self.short, dtype=torch.float64, device=self._comm_device())
        else:
            res = self.local.spmv(w) if self.layout == "csc" else self.local.spvtm(w)
            part = torch.as_tensor(res).to(self._comm_device()).double()
        dist.all_reduce(part, op=dist.ReduceOp.SUM, group=self.group)
        return part

    # ---- Sec. IV-A: per-rank dot products, split columns completed across the zone
    def _dot(self, w):
        import torch
        import torch.distributed as dist

        if self.local is None:
            out = torch.zeros(0, dtype=torch.float64)
        else:
            res = self.local.spvtm(w) if self.layout == "csc" else self.local.spmv(w)
            out = torch.as_tensor(res).detach().to("cpu").double().clone()
        mine = torch.zeros(2, dtype=torch.float64)
        if self.nonempty and self.n_local > 0:
            mine[0] = out[0]   # partial sum of the first column
            mine[1] = out[-1]  # of the last (the same entry when the rank holds one column)
        allp = [torch.empty(2, dtype=torch.float64, device=self._comm_device()) for _ in range(self.world)]
        dist.all_gather(allp, mine.to(self._comm_device()), group=self.group)
        parts = [t.cpu() for t in allp]
        for first, last, col in self.setup.zones:
            if not (first <= self.rank <= last):
                continue
            s = float(parts[first][1])
            for q in range(first + 1, last):
                s += float(parts[q][1])
            s += float(parts[last][0])
            if self.first == col:
                out[0] = s
            if self.last == col:
                out[-1] = s
        return out

    def spmv(self, x):
        """Wide CSC: x_window (entries first .. last of x) -> y (m entries, all-reduced).
        Tall CSR: x (n entries) -> y_window (rows first .. last, zones completed)."""
        return self._accumulate(x) if self.layout == "csc" else self._dot(x)

    def spvtm(self, v):
        """Wide CSC: v (m entries) -> u_window (entries first .. last, zones completed).
        Tall CSR: v_window (rows first .. last of v) -> u (n entries, all-reduced)."""
        return self._dot(v) if self.layout == "csc" else self._accumulate(v)
