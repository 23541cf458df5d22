"""Plant plausible mistakes in copies of the oracle (on the CPU) and check that the pins catch each.

The real oracle sources are never modified: each mutant is a text substitution
in a temporary copy of ``oracle.c`` (compiled with the same flags) or a
monkeypatched step of ``oracle.plan``.
"""
import json
import os
import subprocess

import numpy as np
import pytest

import oracle
import pins
from oracle import plan as plan_oracle

SRC = os.path.join(os.path.dirname(oracle.__file__), "oracle.c")

C_MUTANTS = {
    # dropped last term of every column (CSC matvec)
    "csc_matvec_drop_last": ("for (int64_t k = ptr[j]; k < ptr[j + 1]; ++k) {\n            y[idx[k]]",
                             "for (int64_t k = ptr[j]; k < ptr[j + 1] - 1; ++k) {\n            y[idx[k]]"),
    # wrong sign of the column dot product (CSC vecmat)
    "csc_vecmat_sign": ("s += v[idx[k]] * val[k];", "s -= v[idx[k]] * val[k];"),
    # transposed operand: indexes v by the column instead of the row
    "csc_vecmat_transposed": ("s += v[idx[k]] * val[k];", "s += v[j % m] * val[k];"),
    # wrong index into x (CSR matvec)
    "csr_matvec_index": ("s += val[k] * x[idx[k]];", "s += val[k] * x[k % n];"),
    # accumulates into the wrong output position (CSR vecmat)
    "csr_vecmat_target": ("u[idx[k]] += v[i] * val[k];", "u[i % n] += v[i] * val[k];"),
    # missing initialisation of y (CSC matvec) -> stale values
    "csc_matvec_no_zero": ("for (int64_t i = 0; i < m; ++i) y[i] = 0.0;", "for (int64_t i = 0; i < m; ++i) y[i] = 1.0;"),
    # gradient with x of the row index instead of the column
    "csc_dvalues_index": ("g[k] = r[idx[k]] * x[j];", "g[k] = r[idx[k]] * x[idx[k] % n];"),
    "csr_dvalues_index": ("g[k] = r[i] * x[idx[k]];", "g[k] = r[idx[k] % m] * x[idx[k]];"),
    # all-core loops: the last thread's private copy left out of the final sum
    "mt_sum_drops_thread": ("for (int t = 0; t < threads; ++t) s += priv", "for (int t = 0; t + 1 < threads; ++t) s += priv"),
    # all-core loops: neighbouring ranges skip the column (row) between them
    "mt_range_gap": ("if (t > 0) J->lo = jobs[t - 1].hi;", "if (t > 0) J->lo = jobs[t - 1].hi + (jobs[t - 1].hi < n_major);"),
}


def _build_mutant(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not unique"
    path = tmp_path / f"{name}.c"
    path.write_text(src.replace(old, new))
    so = tmp_path / f"lib{name}.so"
    subprocess.check_call(["gcc", *oracle.CFLAGS, str(path), "-o", str(so)])
    return oracle.Oracle(oracle.load_library(str(so)))


@pytest.mark.parametrize("name", sorted(C_MUTANTS))
def test_c_mutant_is_caught(tmp_path, name):
    old, new = C_MUTANTS[name]
    orc = _build_mutant(tmp_path, name, old, new)
    caught = []
    for pin in pins.ALL_PINS:
        try:
            pin(orc)
        except AssertionError:
            caught.append(pin.__name__)
    assert caught, f"no pin caught mutant {name}"


GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "worked_example.json")


def _golden_check():
    g = json.load(open(GOLDEN))
    ptr = np.concatenate([[0], np.cumsum(g["column_counts"]["value"])]).astype(np.int64)
    po = plan_oracle.plan(ptr, g["P"])
    ok = (po.end - po.begin).tolist() == g["nonzeros_per_processor"]["value"]
    ok &= [[k, j + 1, S] for (k, j, S) in po.zones] == g["zones"]["value"]
    for name in ("needLeft", "needRight", "leftGroupEnd", "rightGroup", "leftGroup", "procsOnLeft", "procsOnRight"):
        ok &= getattr(po, name).tolist() == g["table3"][name]
    # Sec. II stated rule with Z mod P != 0: 10 nonzeros over 4 groups -> 3, 3, 2, 2
    b, e = plan_oracle.group_bounds(10, 4)
    ok &= (np.asarray(e) - np.asarray(b)).tolist() == [3, 3, 2, 2]
    return ok


def _uneven_bounds(Z, P):
    # mistake: the extra nonzeros go to the last groups instead of the first
    q, r = divmod(Z, P)
    sizes = [q + 1 if i >= P - r else q for i in range(P)]
    end = np.cumsum(sizes)
    return end - np.array(sizes), end


def _non_segmented(a, b):
    # mistake: plain addition that ignores the keys
    return (a[0] + b[0], b[1])


def _swapped_keys(a, b):
    # mistake: keeps the left key
    s, k = a
    t, l = b
    return (s + t, k) if k == l else (t, k)


@pytest.mark.parametrize("mutant", ["uneven_bounds", "non_segmented", "swapped_keys"])
def test_plan_mutant_is_caught(monkeypatch, mutant):
    assert _golden_check()
    if mutant == "uneven_bounds":
        monkeypatch.setattr(plan_oracle, "group_bounds", _uneven_bounds)
    elif mutant == "non_segmented":
        monkeypatch.setattr(plan_oracle, "seg_op", _non_segmented)
    else:
        monkeypatch.setattr(plan_oracle, "seg_op", _swapped_keys)
    caught = not _golden_check()
    if not caught:  # the brute-force walk is the second line of defence
        rng = np.random.default_rng(3)
        for _ in range(20):
            deg = np.minimum(rng.zipf(1.8, 100), 300)
            ptr = np.concatenate([[0], np.cumsum(deg)])
            P = int(rng.integers(2, 60))
            if plan_oracle.plan(ptr, P).zones != plan_oracle.brute_force_zones(ptr, P):
                caught = True
                break
    assert caught


def _cgls_mutant(kind):
    """CGLS recurrences with one plausible mistake, on the real products."""

    def cgls(self, A, b, x0, iters):
        x = np.array(x0, dtype=np.float64)
        r = np.asarray(b, dtype=np.float64) - self.spmv(A, x)
        s = self.spvtm(A, r)
        p = s.copy()
        gamma0 = gamma = float(s @ s)
        for _ in range(iters):
            q = self.spmv(A, p)
            delta = float((p @ p) if kind == "alpha_denominator" else (q @ q))
            alpha = gamma / delta if delta > 0 else 0.0
            x += alpha * p
            r = r + alpha * q if kind == "residual_sign" else r - alpha * q
            s = self.spvtm(A, q if kind == "gradient_of_q" else r)
            gamma_new = float(s @ s)
            beta = (gamma / gamma_new if gamma_new > 0 else 0.0) if kind == "beta_inverted" else \
                (gamma_new / gamma if gamma > 0 else 0.0)
            gamma = gamma_new
            p = s if kind == "no_momentum" else s + beta * p
        return x, (np.sqrt(gamma / gamma0) if gamma0 > 0 else 0.0)

    return cgls


@pytest.mark.parametrize("kind", ["alpha_denominator", "residual_sign", "gradient_of_q", "beta_inverted",
                                  "no_momentum"])
def test_cgls_mutant_is_caught(monkeypatch, kind):
    orc = oracle.Oracle()
    pins.pin_cgls_least_squares(orc)  # the real recurrences pass
    monkeypatch.setattr(oracle.Oracle, "cgls", _cgls_mutant(kind))
    with pytest.raises(AssertionError), np.errstate(all="ignore"):  # some mutants diverge
        pins.pin_cgls_least_squares(oracle.Oracle())
