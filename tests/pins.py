"""Pins of the FP64 oracle: checks against things the oracle does not compute itself.

Each ``pin_*`` function takes an oracle object (``oracle.Oracle`` or a variant
built from a deliberately broken copy of its source) and raises
``AssertionError`` on a mismatch.  ``tests/test_oracle.py`` runs them on the
real oracle; ``tests/test_oracle_mutants.py`` checks that every planted
mistake trips at least one of them.
"""
from __future__ import annotations

import numpy as np

from synth import SparseMatrix, random_matrix, uniform_vector


def dense_of(A: SparseMatrix) -> np.ndarray:
    """Dense m x n matrix assembled by direct placement (duplicates add)."""
    D = np.zeros((A.m, A.n), dtype=np.float64)
    ptr = np.asarray(A.ptr, dtype=np.int64)
    vals = np.asarray(A.vals, dtype=np.float64)
    for s in range(len(ptr) - 1):
        for k in range(ptr[s], ptr[s + 1]):
            if A.layout == "csc":
                D[A.idx[k], s] += vals[k]
            else:
                D[s, A.idx[k]] += vals[k]
    return D


def dense_dvalues(A: SparseMatrix, r, x) -> np.ndarray:
    """Gradient of r^T A x w.r.t. each stored value: the outer product r x^T read at its position."""
    G = np.outer(np.asarray(r, np.float64), np.asarray(x, np.float64))
    ptr = np.asarray(A.ptr, dtype=np.int64)
    g = np.empty(A.nnz, dtype=np.float64)
    for s in range(len(ptr) - 1):
        for k in range(ptr[s], ptr[s + 1]):
            g[k] = G[A.idx[k], s] if A.layout == "csc" else G[s, A.idx[k]]
    return g


def _int_cases():
    """Small integer-valued matrices (all sums exact in FP64) covering the edge cases."""
    cases = []
    seed = 100
    for layout in ("csc", "csr"):
        for (m, n, dens) in [(7, 13, 0.3), (13, 7, 0.3), (1, 9, 0.6), (9, 1, 0.6), (5, 8, 0.5), (16, 40, 0.05), (40, 16, 0.05)]:
            cases.append(random_matrix(m, n, layout, density=dens, seed=seed, int_values=9))
            seed += 1
        # duplicates inside a segment
        cases.append(random_matrix(6, 11, layout, density=0.4, seed=seed, int_values=5, duplicates=True))
        seed += 1
        # empty segments everywhere but two
        n_major = 12
        deg = np.zeros(n_major, dtype=np.int64)
        deg[3] = 4
        deg[9] = 2
        m, n = (5, n_major) if layout == "csc" else (n_major, 5)
        cases.append(random_matrix(m, n, layout, degrees=deg, seed=seed, int_values=7))
        seed += 1
        # no nonzeros at all
        cases.append(random_matrix(4, 6, layout, degrees=np.zeros(6 if layout == "csc" else 4, np.int64), seed=seed))
        seed += 1
    return cases


def pin_dense_bruteforce(orc) -> None:
    """y = A x and u = v^T A equal the dense products exactly on integer data."""
    for A in _int_cases():
        D = dense_of(A)
        x = uniform_vector(A.n, 7, int_values=6)
        v = uniform_vector(A.m, 8, int_values=6)
        y = orc.spmv(A, x)
        u = orc.spvtm(A, v)
        assert np.array_equal(y, D @ x), f"spmv != dense ({A.name})"
        assert np.array_equal(u, v @ D), f"spvtm != dense ({A.name})"


def pin_dvalues_bruteforce(orc) -> None:
    """g[k] = r_i x_j read from the dense outer product, exactly."""
    for A in _int_cases():
        r = uniform_vector(A.m, 9, int_values=5)
        x = uniform_vector(A.n, 10, int_values=5)
        g = orc.dvalues(A, r, x)
        assert np.array_equal(g, dense_dvalues(A, r, x)), f"dvalues != outer product ({A.name})"


def pin_adjoint_linearity(orc) -> None:
    """v^T (A x) = (v^T A) x, and both products are linear in their vector and in the values."""
    for layout in ("csc", "csr"):
        for seed, (m, n) in enumerate([(50, 400), (400, 50), (33, 33)]):
            A = random_matrix(m, n, layout, density=0.05, seed=200 + seed)
            x = uniform_vector(n, 300 + seed)
            x2 = uniform_vector(n, 301 + seed)
            v = uniform_vector(m, 400 + seed)
            v2 = uniform_vector(m, 401 + seed)
            y = orc.spmv(A, x)
            u = orc.spvtm(A, v)
            lhs, rhs = float(v @ y), float(u @ x)
            scale = float(np.abs(v) @ dense_of(SparseMatrix(A.layout, m, n, A.ptr, A.idx, np.abs(A.vals))) @ np.abs(x))
            assert abs(lhs - rhs) <= 1e-12 * scale + 1e-300, "adjoint identity"
            a, b = 0.75, -2.5
            assert np.allclose(orc.spmv(A, a * x + b * x2), a * y + b * orc.spmv(A, x2), rtol=1e-12, atol=1e-12)
            assert np.allclose(orc.spvtm(A, a * v + b * v2), a * u + b * orc.spvtm(A, v2), rtol=1e-12, atol=1e-12)
            B = SparseMatrix(A.layout, m, n, A.ptr, A.idx, 3.0 * np.asarray(A.vals))
            assert np.allclose(orc.spmv(B, x), 3.0 * y, rtol=1e-13, atol=1e-13)
            assert np.allclose(orc.spvtm(B, v), 3.0 * u, rtol=1e-13, atol=1e-13)


def pin_closed_forms(orc) -> None:
    """Identity matrix, a single dense column/row, and the all-ones matrix."""
    for layout in ("csc", "csr"):
        N = 17
        I = SparseMatrix(layout, N, N, np.arange(N + 1, dtype=np.int32), np.arange(N, dtype=np.int32), np.ones(N))
        x = uniform_vector(N, 1)
        assert np.array_equal(orc.spmv(I, x), x) and np.array_equal(orc.spvtm(I, x), x), "identity"
        # all-ones m x n: y_i = sum(x), u_j = sum(v)
        m, n = 6, 9
        n_major, n_minor = (n, m) if layout == "csc" else (m, n)
        ptr = (np.arange(n_major + 1) * n_minor).astype(np.int32)
        idx = np.tile(np.arange(n_minor, dtype=np.int32), n_major)
        J = SparseMatrix(layout, m, n, ptr, idx, np.ones(m * n))
        xi = uniform_vector(n, 2, int_values=9)
        vi = uniform_vector(m, 3, int_values=9)
        assert np.array_equal(orc.spmv(J, xi), np.full(m, xi.sum())), "ones spmv"
        assert np.array_equal(orc.spvtm(J, vi), np.full(n, vi.sum())), "ones spvtm"
    # one dense column j0 in a wide CSC matrix: u_j0 = v . a, y = a x_j0
    m, n, j0 = 8, 5, 3
    a = np.arange(1, m + 1, dtype=np.float64)
    ptr = np.array([0, 0, 0, 0, m, m], dtype=np.int32)
    A = SparseMatrix("csc", m, n, ptr, np.arange(m, dtype=np.int32), a)
    x = np.array([1.0, 2.0, 3.0, -4.0, 5.0])
    v = np.arange(m, dtype=np.float64) - 3.0
    assert np.array_equal(orc.spmv(A, x), a * x[j0]), "dense column spmv"
    u = orc.spvtm(A, v)
    assert u[j0] == float(v @ a) and np.count_nonzero(u) == 1, "dense column spvtm"


def pin_gradients_fd(orc) -> None:
    """Central finite differences of 0.5||Ax-b||^2 match the oracle gradients."""
    for layout in ("csc", "csr"):
        A = random_matrix(12, 30, layout, density=0.2, seed=77)
        x = uniform_vector(30, 78)
        b = uniform_vector(12, 79)
        loss, gx, gv, _ = orc.least_squares(A, x, b)
        h = 1e-6
        rng = np.random.default_rng(5)
        for j in rng.choice(30, 6, replace=False):
            e = np.zeros(30)
            e[j] = h
            fd = (orc.least_squares(A, x + e, b)[0] - orc.least_squares(A, x - e, b)[0]) / (2 * h)
            assert abs(fd - gx[j]) <= 1e-7 * max(1.0, abs(gx[j])), "d/dx"
        for k in rng.choice(A.nnz, 6, replace=False):
            vp = np.array(A.vals, dtype=np.float64)
            vm = vp.copy()
            vp[k] += h
            vm[k] -= h
            Ap = SparseMatrix(A.layout, A.m, A.n, A.ptr, A.idx, vp)
            Am = SparseMatrix(A.layout, A.m, A.n, A.ptr, A.idx, vm)
            fd = (orc.least_squares(Ap, x, b)[0] - orc.least_squares(Am, x, b)[0]) / (2 * h)
            assert abs(fd - gv[k]) <= 1e-7 * max(1.0, abs(gv[k])), "d/dvalues"


def pin_cgls_least_squares(orc) -> None:
    """CGLS from zero reaches numpy's least-squares solution (tall full rank) and the minimum-norm
    solution (wide); its first step is the steepest-descent step on the normal equations, and its
    k-th iterate the least-squares solution over the k-dimensional Krylov space."""
    for m, n in ((60, 12), (12, 60)):
        layout = "csr" if m > n else "csc"
        A = random_matrix(m, n, layout, density=0.5, seed=31)
        b = uniform_vector(m, 32)
        D = dense_of(A)
        x_ref = np.linalg.lstsq(D, b, rcond=None)[0]
        x, rel = orc.cgls(A, b, np.zeros(n), iters=4 * min(m, n))
        assert rel < 1e-8, "gradient norm"
        assert np.allclose(x, x_ref, rtol=1e-7, atol=1e-9 * np.abs(x_ref).max()), "least-squares solution"
        g = D.T @ b
        alpha = g @ g / np.sum((D @ g) ** 2)
        x1, _ = orc.cgls(A, b, np.zeros(n), iters=1)
        assert np.allclose(x1, alpha * g, rtol=1e-12, atol=1e-15), "first step"
        # the k-th iterate minimises ||b - A x|| over the Krylov space span{g, M g, ..., M^(k-1) g},
        # M = A^T A (the defining property of CG on the normal equations)
        M = D.T @ D
        K = [g]
        for k in (2, 3):
            K.append(M @ K[-1])
            B = np.stack(K, axis=1)
            c = np.linalg.lstsq(D @ B, b, rcond=None)[0]
            xk, _ = orc.cgls(A, b, np.zeros(n), iters=k)
            assert np.allclose(xk, B @ c, rtol=1e-8, atol=1e-10 * np.abs(B @ c).max()), f"iterate {k}"


def pin_threaded_loops(orc) -> None:
    """The all-core loops equal the dense products exactly on integer data, for thread counts
    below, at and above the number of columns (rows); the dot-product directions equal the
    serial loop bit for bit on random data too (one thread computes each entry)."""
    for A in _int_cases():
        D = dense_of(A)
        x = uniform_vector(A.n, 17, int_values=6)
        v = uniform_vector(A.m, 18, int_values=6)
        for t in (1, 2, 3, 7, 16):
            assert np.array_equal(orc.spmv_mt(A, x, t), D @ x), f"spmv_mt({t}) != dense ({A.name})"
            assert np.array_equal(orc.spvtm_mt(A, v, t), v @ D), f"spvtm_mt({t}) != dense ({A.name})"
    for layout in ("csc", "csr"):
        A = random_matrix(120, 900, layout, density=0.03, seed=31)
        x, v = uniform_vector(A.n, 32), uniform_vector(A.m, 33)
        dot_mt, dot = (orc.spvtm_mt(A, v, 5), orc.spvtm(A, v)) if layout == "csc" else (orc.spmv_mt(A, x, 5), orc.spmv(A, x))
        assert np.array_equal(dot_mt, dot), f"dot-product direction differs from the serial loop ({layout})"


ALL_PINS = [pin_dense_bruteforce, pin_dvalues_bruteforce, pin_adjoint_linearity, pin_closed_forms, pin_gradients_fd,
            pin_cgls_least_squares, pin_threaded_loops]
