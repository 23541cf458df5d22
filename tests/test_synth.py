"""The seeded synthetic workloads follow their stated recipes (CPU only).

Shapes, dense columns (rows), degree laws, index structure and value distributions of
the generators in synth/, checked on the generated arrays; the generators hold no
arithmetic of the method, so these checks are about the inputs only.
"""
import math

import numpy as np
import pytest

import synth


def _np(a):
    return a.cpu().numpy() if hasattr(a, "cpu") else np.asarray(a)


def _check_structure(A):
    ptr, idx = _np(A.ptr).astype(np.int64), _np(A.idx).astype(np.int64)
    assert ptr[0] == 0 and ptr[-1] == A.nnz and np.all(np.diff(ptr) >= 0)
    assert idx.min() >= 0 and idx.max() < A.n_minor
    # indices distinct and ascending inside every segment
    starts = np.zeros(A.nnz, dtype=bool)
    starts[ptr[:-1][np.diff(ptr) > 0]] = True
    d = np.diff(idx)
    assert np.all((d > 0) | starts[1:])
    return np.diff(ptr)


def test_wide_fp64_small_recipe():
    """m = 1,000, n = 100,000; Zipf(2) degrees clipped to [1, 1000]; 5 fully dense columns;
    values U(0, 1); seeded."""
    A = synth.wide_fp64_small(0)
    assert (A.m, A.n, A.layout) == (1000, 100_000, "csc")
    deg = _check_structure(A)
    assert deg.min() >= 1 and deg.max() <= 1000
    assert np.sum(deg == 1000) >= 5
    zeta2 = math.pi ** 2 / 6
    assert abs(np.mean(deg == 1) - 1 / zeta2) < 0.01  # P(D = 1) of Zipf(2)
    assert abs(np.mean(deg == 2) - 0.25 / zeta2) < 0.01
    assert 480_000 < A.nnz < 540_000
    vals = _np(A.vals)
    assert vals.min() >= 0 and vals.max() < 1 and abs(vals.mean() - 0.5) < 0.005
    B = synth.wide_fp64_small(0)
    assert np.array_equal(_np(A.ptr), _np(B.ptr)) and np.array_equal(_np(A.idx), _np(B.idx))


def _tail_check(deg, d_min, alpha):
    for mult in (4, 16):
        d = math.ceil(mult * d_min)
        want = (d_min / d) ** alpha
        got = np.mean(deg >= d)
        assert abs(got - want) < 0.1 * want, (d, got, want)


def test_wide_fp32_large_recipe_on_a_scaled_sample():
    """m = 20,000 rows; 50 columns at 50% density; the other columns a bounded power law with
    density exponent 2 (tail P(D >= d) = d_min / d); lognormal(0, 1) values."""
    scale = 0.05
    A = synth.wide_fp32_large(1, device="cpu", scale=scale)
    assert (A.m, A.n, A.layout) == (20_000, 250_000, "csc")
    deg = _check_structure(A)
    dense = deg == 10_000
    assert dense.sum() >= 50
    rest = deg[~dense]
    mean = (200e6 * scale - 50 * 10_000) / (A.n - 50)
    d_min = synth.power_law_dmin(mean, 2.0, 20_000)
    _tail_check(rest, d_min, 1.0)
    assert abs(A.nnz - 200e6 * scale) < 0.06 * 200e6 * scale
    lv = np.log(_np(A.vals).astype(np.float64))
    assert abs(lv.mean()) < 0.01 and abs(lv.std() - 1) < 0.01


def test_tall_fp32_large_recipe_on_a_scaled_sample():
    """n = 2,000 columns; 20 rows at 60% density; the other rows a bounded power law with density
    exponent 2.2."""
    scale = 0.01
    A = synth.tall_fp32_large(2, device="cpu", scale=scale)
    assert (A.m, A.n, A.layout) == (100_000, 2_000, "csr")
    deg = _check_structure(A)
    dense = deg == 1200
    assert dense.sum() >= 20
    rest = deg[~dense]
    mean = (150e6 * scale - 20 * 1200) / (A.m - 20)
    d_min = synth.power_law_dmin(mean, 2.2, 2_000)
    _tail_check(rest, d_min, 1.2)
    assert abs(A.nnz - 150e6 * scale) < 0.05 * 150e6 * scale


def test_serving_specs_recipe():
    """64 matrices, m in [1k, 50k], n in [100k, 5M] (the long side of a tall matrix), Z in [1M, 100M],
    at most a quarter dense, dimensions multiples of 4, total stored bytes within 120 GB."""
    specs = synth.serving_specs()
    assert len(specs) == 64
    assert {s["layout"] for s in specs} == {"csc", "csr"}
    total = 0.0
    for s in specs:
        short, long_ = (s["m"], s["n"]) if s["layout"] == "csc" else (s["n"], s["m"])
        assert 1_000 <= short <= 50_000 and 100_000 <= long_ <= 5_000_000
        assert short % 4 == 0 and long_ % 4 == 0
        assert 1_000_000 <= s["nnz"] <= 100_000_000 and s["nnz"] <= short * long_ / 4
        total += 8.0 * s["nnz"] + 4.0 * (long_ + 1)
    assert total <= 120e9
    assert synth.serving_specs() == specs


@pytest.mark.parametrize("seed", [0, 1])
def test_uniform_vectors_are_seeded(seed):
    a, b = synth.uniform_vector(1000, seed), synth.uniform_vector(1000, seed)
    assert np.array_equal(a, b) and a.min() >= -1 and a.max() <= 1
    assert not np.array_equal(a, synth.uniform_vector(1000, seed + 7))
