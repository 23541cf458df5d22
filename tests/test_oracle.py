"""The FP64 oracle against what the paper and the mathematics fix (CPU only)."""
import itertools
import json
import os
import zlib

import numpy as np
import pytest

import oracle
import pins
import synth
from oracle import plan as plan_oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "worked_example.json")


@pytest.mark.parametrize("pin", pins.ALL_PINS, ids=lambda f: f.__name__)
def test_oracle_pin(pin, oracle_impl):
    pin(oracle_impl)


# ---------------------------------------------------------------------------
# Sec. II partition and Sec. IV-B set-up: the worked example (Figs. 1-3, Tables II-III)


@pytest.fixture(scope="module")
def golden():
    with open(GOLDEN) as f:
        return json.load(f)


def _example_ptr(golden):
    counts = golden["column_counts"]["value"]
    return np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)


def test_example_partition(golden):
    ptr = _example_ptr(golden)
    po = plan_oracle.plan(ptr, golden["P"])
    assert po.Z == golden["Z"]
    assert (po.end - po.begin).tolist() == golden["nonzeros_per_processor"]["value"]
    # J_i: every column holding a nonzero of group i (1-based as printed)
    cols = []
    for i in range(po.P):
        owners = [plan_oracle.column_of(ptr, k) + 1 for k in range(po.begin[i], po.end[i])]
        cols.append(sorted(set(owners)))
    assert cols == golden["processor_columns_1based"]["value"]
    assert cols[:2] == golden["J0_J1_1based"]["value"]
    # the first/last columns of step 2 bound J_i
    assert [[c[0], c[-1]] for c in cols] == [[a + 1, b + 1] for a, b in zip(po.jf, po.jl)]
    # Fig. 3: number of copies of each x coefficient
    copies = {str(j): sum(j in c for c in cols) for j in range(1, 9)}
    for j, cnt in golden["x_replication_1based"]["value"].items():
        assert copies[j] == cnt
    assert all(copies[str(j)] == 1 for j in (1, 3, 5, 7, 8))


def test_example_zones_table2(golden):
    ptr = _example_ptr(golden)
    po = plan_oracle.plan(ptr, golden["P"])
    got = [[k, j + 1, S] for (k, j, S) in po.zones]
    assert got == golden["zones"]["value"]
    assert plan_oracle.brute_force_zones(ptr, golden["P"]) == po.zones


def test_example_variables_table3(golden):
    ptr = _example_ptr(golden)
    po = plan_oracle.plan(ptr, golden["P"])
    t3 = golden["table3"]
    for name in ("needLeft", "needRight", "leftGroupEnd", "rightGroup", "leftGroup", "procsOnLeft", "procsOnRight"):
        assert getattr(po, name).tolist() == t3[name], name


def test_group_sizes_rule():
    """Sec. II: the first Z mod P groups hold ceil(Z/P) nonzeros, the rest floor(Z/P)."""
    for Z, P, want in [(10, 4, [3, 3, 2, 2]), (21, 7, [3] * 7), (2, 5, [1, 1, 0, 0, 0]), (0, 3, [0, 0, 0])]:
        b, e = plan_oracle.group_bounds(Z, P)
        assert (e - b).tolist() == want
        assert b[0] == 0 and e[-1] == Z and (b[1:] == e[:-1]).all()


def test_seg_op_associative():
    """Sec. IV-B calls o associative.  That holds on sequences whose equal keys are
    contiguous (the scanned group ranks are non-decreasing); with a key that
    returns after a different one it does not, e.g. (1,0),(0,1),(0,0)."""
    vals = [(s, k) for s in range(3) for k in range(3)]
    op = plan_oracle.seg_op
    for a, b, c in itertools.product(vals, repeat=3):
        if a[1] <= b[1] <= c[1]:
            assert op(op(a, b), c) == op(a, op(b, c))
    assert op(op((1, 0), (0, 1)), (0, 0)) != op((1, 0), op((0, 1), (0, 0)))
    assert op((1, 0), (2, 1)) != op((2, 1), (1, 0))  # not commutative


def _random_ptr(rng, n, kind):
    if kind == "powerlaw":
        deg = np.minimum(rng.zipf(1.8, n), 500)
    elif kind == "empties":
        deg = rng.integers(0, 3, n) * rng.integers(0, 2, n)
    elif kind == "one_column":
        deg = np.zeros(n, np.int64)
        deg[rng.integers(0, n)] = rng.integers(1, 400)
    elif kind == "singletons":
        deg = np.ones(n, np.int64)
    else:
        deg = rng.integers(0, 20, n)
    return np.concatenate([[0], np.cumsum(deg)]).astype(np.int64)


@pytest.mark.parametrize("kind", ["powerlaw", "empties", "one_column", "singletons", "uniform"])
def test_plan_rules_match_brute_force(kind):
    rng = np.random.default_rng(zlib.crc32(kind.encode()))
    for trial in range(25):
        n = int(rng.integers(1, 300))
        ptr = _random_ptr(rng, n, kind)
        Z = int(ptr[-1])
        for P in sorted({1, 2, 3, int(rng.integers(1, 64)), int(rng.integers(1, 700))}):
            po = plan_oracle.plan(ptr, P)
            # Sec. II: sizes differ by at most one, larger groups first
            sizes = po.end - po.begin
            assert sizes.max() - sizes.min() <= 1
            assert (np.diff(sizes) <= 0).all()
            assert sizes.sum() == Z
            # the rule-based zones of Sec. IV-B equal a direct walk of the nonzeros
            bf = plan_oracle.brute_force_zones(ptr, P)
            assert po.zones == bf
            # Sec. IV-A: z <= P-1; consecutive S_k meet in at most one processor; others are disjoint
            assert po.z <= max(P - 1, 0)
            for a in range(po.z):
                for b in range(a + 1, po.z):
                    inter = set(po.zones[a][2]) & set(po.zones[b][2])
                    assert len(inter) <= (1 if b == a + 1 else 0)
            # procsOnRight of each zone's first processor is |S_k| - 1
            for k, j, S in po.zones:
                assert po.needRight[S[0]] == 1 and po.rightGroup[S[0]] == k
                assert po.procsOnRight[S[0]] == len(S) - 1
                assert all(po.jf[p] == j or po.jl[p] == j for p in S)


def test_oracle_cgls_reaches_the_least_squares_solution():
    """CGLS from zero converges to the least-squares solution of a tall full-rank problem and to
    the minimum-norm solution of a wide one (both given by numpy's lstsq); one step is the
    steepest-descent step."""
    pins.pin_cgls_least_squares(oracle.Oracle())
