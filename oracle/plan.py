"""Oracle of the nonzero partition (Sec. II) and the overlap-zone set-up (Sec. IV-B).

TEST INFRASTRUCTURE ONLY (see the package docstring).  Plain Python over
numpy arrays; P is at most a few thousand, so loops are fine.

Everything follows the paper's steps in its order, 0-based:

1. Sec. II: split the Z nonzeros, in storage order, into P contiguous groups;
   the first Z mod P groups hold ceil(Z/P) nonzeros and the others floor(Z/P).
2. Sec. II: J_i is the set of columns (rows for a tall CSR matrix) holding a
   nonzero of group i; Sec. IV-B: j^f_i and j^l_i are its first and last.
3. Sec. IV-B "Determine overlap zones": needLeft_i = [j^f_i = j^l_{i-1}]
   (i >= 1), needRight_i = [j^l_i = j^f_{i+1}] (i <= P-2), zero at the ends.
4. "Determine ranks of overlap groups": leftGroupEnd = needLeft and
   (not needRight or j^f != j^l); rightGroup = inclusive additive forward
   scan of leftGroupEnd; leftGroup = rightGroup - leftGroupEnd.
5. "Determine group extents": procsOnLeft is the first component of the
   inclusive forward scan of (needLeft, leftGroup) under the segmented
   operator o; procsOnRight the same for a backward scan of
   (needRight, rightGroup).

Readings where the paper is silent: a group may be empty when Z < P (with the
Sec. II rule those are the trailing groups); an empty group has no columns and
all its flags are zero, and its neighbours compare unequal with it.
"""
from __future__ import annotations

import dataclasses
from typing import List, Tuple

import numpy as np


def seg_op(a: Tuple[int, int], b: Tuple[int, int]) -> Tuple[int, int]:
    """The segmented addition o of Sec. IV-B: (s,k) o (t,l) = (s+t, l) if k == l else (t, l)."""
    s, k = a
    t, l = b
    return (s + t, l) if k == l else (t, l)


def group_bounds(Z: int, P: int) -> Tuple[np.ndarray, np.ndarray]:
    """Sec. II: [begin, end) of each of the P nonzero groups."""
    q, r = divmod(Z, P)
    sizes = [q + 1 if i < r else q for i in range(P)]
    begin = np.zeros(P, dtype=np.int64)
    end = np.zeros(P, dtype=np.int64)
    pos = 0
    for i in range(P):
        begin[i] = pos
        pos += sizes[i]
        end[i] = pos
    assert pos == Z
    return begin, end


def column_of(ptr: np.ndarray, k: int) -> int:
    """Column (major index) holding storage position k: ptr[j] <= k < ptr[j+1]."""
    # ptr is non-decreasing; the last j with ptr[j] <= k is the (non-empty) owner.
    return int(np.searchsorted(ptr, k, side="right")) - 1


@dataclasses.dataclass
class PlanOracle:
    P: int
    Z: int
    begin: np.ndarray
    end: np.ndarray
    nonempty: np.ndarray
    jf: np.ndarray
    jl: np.ndarray
    needLeft: np.ndarray
    needRight: np.ndarray
    leftGroupEnd: np.ndarray
    rightGroup: np.ndarray
    leftGroup: np.ndarray
    procsOnLeft: np.ndarray
    procsOnRight: np.ndarray
    zones: List[Tuple[int, int, List[int]]]  # (rank k, column j_k, processors S_k)

    @property
    def z(self) -> int:
        return len(self.zones)


def plan(ptr, P: int) -> PlanOracle:
    """Run steps 1-5 above on the pointer array of a CSC (or CSR) matrix."""
    ptr = np.asarray(ptr, dtype=np.int64)
    Z = int(ptr[-1])
    begin, end = group_bounds(Z, P)
    nonempty = end > begin
    # step 2: first and last column of each group
    jf = np.full(P, -1, dtype=np.int64)
    jl = np.full(P, -1, dtype=np.int64)
    for i in range(P):
        if nonempty[i]:
            jf[i] = column_of(ptr, begin[i])
            jl[i] = column_of(ptr, end[i] - 1)
    # step 3
    needLeft = np.zeros(P, dtype=np.int64)
    needRight = np.zeros(P, dtype=np.int64)
    for i in range(1, P):
        if nonempty[i] and nonempty[i - 1] and jf[i] == jl[i - 1]:
            needLeft[i] = 1
    for i in range(P - 1):
        if nonempty[i] and nonempty[i + 1] and jl[i] == jf[i + 1]:
            needRight[i] = 1
    # step 4
    leftGroupEnd = np.zeros(P, dtype=np.int64)
    for i in range(P):
        leftGroupEnd[i] = int(needLeft[i] == 1 and (needRight[i] == 0 or jf[i] != jl[i]))
    rightGroup = np.zeros(P, dtype=np.int64)
    acc = 0
    for i in range(P):
        acc += int(leftGroupEnd[i])
        rightGroup[i] = acc
    leftGroup = rightGroup - leftGroupEnd
    # step 5: forward o-scan of (needLeft, leftGroup), backward o-scan of (needRight, rightGroup)
    procsOnLeft = np.zeros(P, dtype=np.int64)
    run = None
    for i in range(P):
        pair = (int(needLeft[i]), int(leftGroup[i]))
        run = pair if run is None else seg_op(run, pair)
        procsOnLeft[i] = run[0]
    procsOnRight = np.zeros(P, dtype=np.int64)
    run = None
    for i in range(P - 1, -1, -1):
        pair = (int(needRight[i]), int(rightGroup[i]))
        run = pair if run is None else seg_op(run, pair)
        procsOnRight[i] = run[0]
    # zones: the processor that closes a left group names its rank, column and extent
    zones = []
    for i in range(P):
        if leftGroupEnd[i]:
            k = int(leftGroup[i])
            first = i - int(procsOnLeft[i])
            zones.append((k, int(jf[i]), list(range(first, i + 1))))
    zones.sort()
    return PlanOracle(P, Z, begin, end, nonempty, jf, jl, needLeft, needRight, leftGroupEnd, rightGroup,
                      leftGroup, procsOnLeft, procsOnRight, zones)


def brute_force_zones(ptr, P: int):
    """Walk every nonzero, note which groups touch each column, and list the
    columns touched by two or more groups (the overlap zones of Sec. II) with
    their processor sets, left to right.  Independent of steps 3-5."""
    ptr = np.asarray(ptr, dtype=np.int64)
    Z = int(ptr[-1])
    begin, end = group_bounds(Z, P)
    owner = np.empty(Z, dtype=np.int64)
    for i in range(P):
        owner[begin[i]:end[i]] = i
    zones = []
    for j in range(len(ptr) - 1):
        holders = sorted(set(owner[ptr[j]:ptr[j + 1]].tolist()))
        if len(holders) >= 2:
            zones.append((len(zones), j, holders))
    return zones
