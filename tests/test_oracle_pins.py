"""The CPU oracle against facts the paper and the mathematics fix (no GPU)."""

import os

import numpy as np
import pytest

import oracle
from paper_2308_08417_gb300 import workloads as W
from tests import pins

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.mark.parametrize("check", pins.ALL_CHECKS, ids=lambda c: c.__name__)
def test_pin(check):
    fails = check()
    assert not fails, "\n".join(fails)


def test_format_equivalence_bitwise():
    """Sec. 3.1: the three formats store the same entries; SpMV and every solver
    agree bit for bit when entries are summed in column order."""
    wl = W.plain_at_scale(32, grid=6)
    rng = np.random.default_rng(1)
    xin = rng.uniform(-1, 1, (32, wl.pattern.n))
    ys = []
    for fmt in ("csr", "ell", "dense"):
        A = wl.matrix(fmt)
        ys.append(oracle.spmv(fmt, A.n, A.nnz, A.ell_k, A.row_ptrs, A.col_idxs, A.values, xin))
    assert np.array_equal(ys[0], ys[1]) and np.array_equal(ys[0], ys[2])
    dense = W.to_dense(wl.pattern, wl.csr_values).reshape(32, wl.pattern.n, wl.pattern.n)
    assert np.allclose(ys[0], np.einsum("bij,bj->bi", dense, xin), rtol=1e-14, atol=1e-15)
    for solver in ("bicgstab", "cg", "gmres"):
        outs = [oracle.solve_batch(wl.matrix(f), wl.b, solver=solver) for f in ("csr", "ell", "dense")]
        for o in outs[1:]:
            assert np.array_equal(o[0], outs[0][0]) and np.array_equal(o[1], outs[0][1])


def _golden_rows():
    rows = []
    with open(os.path.join(HERE, "golden", "storage_formulas.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            name, B, n, nnz = line.split()
            rows.append((name, int(B), int(n), int(nnz)))
    return rows


def test_storage_counts_match_section_3_1():
    rows = _golden_rows()
    assert len(rows) == 6
    for name, B, n, nnz in rows:
        assert W.storage_entries("csr", B, n, nnz) == B * nnz + (n + 1) + nnz
        assert W.storage_entries("dense", B, n, nnz) == B * n * n
    # the 3-point stencil row: the pattern builder gives 3n-2 entries
    name, B, n, nnz = rows[-1]
    pat = W.stencil_pattern("1d3", n)
    assert pat.nnz == nnz == 3 * n - 2
    # entry counts of the arrays the builders actually produce
    wl = W.plain_at_scale(8)
    for fmt in ("csr", "ell", "dense"):
        A = wl.matrix(fmt)
        stored = A.values.size + (A.col_idxs.size if fmt != "dense" else 0)
        stored += A.row_ptrs.size if fmt == "csr" else 0
        assert stored == W.storage_entries(fmt, 8, A.n, A.nnz, A.ell_k)


def test_stencil_pattern_counts():
    assert W.stencil_pattern("2d5", 12, 12).nnz == 5 * 144 - 4 * 12 == 672
    assert W.stencil_pattern("2d9", 32, 32).nnz == (3 * 32 - 2) ** 2 == 8836
    assert W.stencil_pattern("2d9", 32, 32).max_row == 9
    assert W.stencil_pattern("1d3", 32).nnz == 94


def test_generated_values_recipe():
    wl = W.plain_at_scale(256)
    pat = wl.pattern
    rows = np.repeat(np.arange(pat.n), np.diff(pat.row_ptrs))
    off = rows != pat.col_idxs
    v = wl.csr_values
    assert (v[:, off] <= 0).all() and (v[:, off] >= -1.1).all()
    diag = v[:, ~off]
    offsum = np.add.reduceat(np.abs(np.where(off, v, 0.0)), pat.row_ptrs[:-1], axis=1)
    ratio = diag / offsum
    assert ratio.min() >= 1.05 - 1e-12 and ratio.max() <= 1.5 + 1e-12
    sym = W.plain_at_scale(16, symmetric=True)
    D = W.to_dense(sym.pattern, sym.csr_values).reshape(16, 144, 144)
    assert np.array_equal(D, np.transpose(D, (0, 2, 1)))
    assert (np.linalg.eigvalsh(D) > 0).all()


# ----------------------------------------------------------------- edges

def test_zero_rhs_gives_zero_solution():
    wl = W.tiny_tridiagonal(8)
    b = wl.b.copy()
    b[3] = 0.0
    x0 = np.ones_like(b)
    for solver in ("bicgstab", "cg", "gmres"):
        x, it, rel, st = oracle.solve_batch(wl.matrix(), b, x0, solver=solver)
        assert it[3] == 0 and st[3] == 0 and rel[3] == 0.0 and (x[3] == 0).all()


def test_nan_is_isolated_per_system():
    wl = W.tiny_tridiagonal(16)
    A = wl.matrix()
    clean = oracle.solve_batch(A, wl.b)
    A2 = A.subset(np.arange(16))
    A2.values = A.values.copy()
    A2.values[5, 7] = np.nan
    b2 = wl.b.copy()
    b2[9, 0] = np.inf
    for solver in ("bicgstab", "cg", "gmres"):
        ref = oracle.solve_batch(A, wl.b, solver=solver)
        x, it, rel, st = oracle.solve_batch(A2, b2, solver=solver)
        assert st[5] == 3 and st[9] == 3
        keep = np.setdiff1d(np.arange(16), [5, 9])
        assert np.array_equal(x[keep], ref[0][keep]) and np.array_equal(it[keep], ref[1][keep])
    assert clean[3].max() == 0


def test_zero_diagonal_falls_back_to_one():
    """Jacobi with a zero diagonal entry uses 1 for that row, i.e. behaves as no
    preconditioner on a matrix whose diagonal is all zero."""
    P = np.array([[0.0, 2.0, 0.0], [1.0, 0.0, 1.0], [0.0, 3.0, 0.0]])
    P[2, 2] = 0.0
    A = [np.array([[0.0, 2.0, 1.0], [1.0, 0.0, 1.0], [1.0, 3.0, 0.0]])]
    b = np.array([[1.0, 2.0, 3.0]])
    for solver in ("bicgstab", "gmres"):
        a = pins.solve_dense(A, b, solver=solver, precond="jacobi", tol=1e-12)
        c = pins.solve_dense(A, b, solver=solver, precond="none", tol=1e-12)
        assert np.array_equal(a[0], c[0]) and np.array_equal(a[1], c[1])
        assert a[3][0] == 0
        assert np.allclose(A[0] @ a[0][0], b[0], atol=1e-10)


def test_max_iters_zero_and_singular():
    wl = W.tiny_tridiagonal(4)
    x0 = np.full_like(wl.b, 0.25)
    for solver in ("bicgstab", "cg", "gmres"):
        x, it, rel, st = oracle.solve_batch(wl.matrix(), wl.b, x0, solver=solver, max_iters=0)
        assert (it == 0).all() and (st == 1).all() and np.array_equal(x, x0)
    Z = [np.zeros((4, 4))]
    b = np.array([[1.0, -1.0, 0.5, 2.0]])
    for solver in ("bicgstab", "cg", "gmres"):
        x, it, rel, st = pins.solve_dense(Z, b, solver=solver, max_iters=50)
        assert st[0] == 2 and it[0] == 1 and np.array_equal(x[0], np.zeros(4))


def test_absolute_tolerance():
    wl = W.plain_at_scale(32)
    D = W.to_dense(wl.pattern, wl.csr_values).reshape(32, 144, 144)
    x, it, rel, st = oracle.solve_batch(wl.matrix(), wl.b, tol_type="absolute", tol=1e-9)
    r = wl.b - np.einsum("bij,bj->bi", D, x)
    assert (st == 0).all() and (np.linalg.norm(r, axis=1) <= 1e-9).all()


def test_refinement_reaches_fp64_tolerance():
    wl = W.mixed_precision(16, grid=12)
    A = wl.matrix("ell")
    D = W.to_dense(wl.pattern, wl.csr_values).reshape(16, wl.pattern.n, wl.pattern.n)
    xs = np.linalg.solve(D, wl.b[..., None])[..., 0]
    x, it, rel, st, inner = oracle.refine(A, wl.b, tol=1e-10, inner_tol=1e-4)
    tr = pins._true_rel(D, x, wl.b)
    assert (st == 0).all() and (tr <= 1e-10).all()
    assert pins.relerr(x, xs).max() <= 1e-8
    assert (it >= 2).all() and (inner >= it).all()
    # the FP32 inner alone cannot reach 1e-10: one outer step is not enough
    x1, it1, rel1, st1, _ = oracle.refine(A, wl.b, tol=1e-10, inner_tol=1e-12, max_outer=1)
    assert (st1 == 1).all() and (rel1 > 1e-10).all()


def test_varsize_matches_shared_pattern_solves():
    vb = W.uneven(60, n_min=16, n_max=80)
    x, it, rel, st = oracle.solve_varsize(vb)
    assert (st == 0).all()
    for i in range(0, 60, 7):
        p, vals, b, x0 = vb.system(i)
        xi, iti, reli, sti = oracle.solve("csr", p.n, p.nnz, 0, p.row_ptrs, p.col_idxs,
                                          vals[None], b[None])
        o = int(vb.vec_off[i])
        assert np.array_equal(xi[0], x[o:o + p.n]) and iti[0] == it[i]
