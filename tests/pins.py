"""Checks that tie the CPU oracle to facts outside itself.

Each check returns a list of failure strings (empty = pass) so that the same
checks serve the pin tests and the mutation tests, which plant a mistake in a
copy of the oracle and expect at least one check to fail.

Independent facts used:
  * dense LU with partial pivoting (numpy.linalg.solve) on tiny systems;
  * closed forms: diagonal A under Jacobi is solved in one iteration,
    A = I gives x = b exactly;
  * finite termination in exact arithmetic: CG on an SPD system within n
    steps, BiCGSTAB within n steps absent breakdown, GMRES with restart >= n
    within n steps;
  * optimality: after k steps GMRES attains the least-squares minimum of
    ||b - A x|| over x0 + M K_k(AM, r0); preconditioned CG attains the A-norm
    Galerkin solution over x0 + K_k(MA, M r0) (both computed with numpy);
  * the stopping invariant ||b - A x|| / ||b|| <= tol, recomputed in long double;
  * exact invariances: power-of-two scaling and batch order.
"""

from __future__ import annotations

import numpy as np

import oracle
from paper_2308_08417_gb300 import workloads as W


def dense_system_batch(mats):
    B, n = len(mats), mats[0].shape[0]
    vals = np.stack([np.asarray(m, dtype=np.float64).ravel() for m in mats])
    return dict(fmt="dense", n=n, nnz=n * n, ell_k=0, row_ptrs=None, col_idxs=None, values=vals,
                num_batch=B)


def solve_dense(mats, b, x0=None, **kw):
    d = dense_system_batch(mats)
    return oracle.solve("dense", d["n"], d["nnz"], 0, None, None, d["values"], b, x0, **kw)


def random_dd(rng, n, factor=1.3, count=40):
    out = []
    for _ in range(count):
        M = rng.uniform(-1, 1, (n, n))
        M += np.diag(np.abs(M).sum(1) * factor)
        out.append(M)
    return out


def relerr(x, y):
    return np.linalg.norm(x - y, axis=-1) / np.linalg.norm(y, axis=-1)


# ---------------------------------------------------------------- checks

def check_lu(solvers=("bicgstab", "cg", "gmres"), fmts=("csr", "ell", "dense")):
    fails = []
    wl = W.tiny_tridiagonal()
    D = W.to_dense(wl.pattern, wl.csr_values).reshape(-1, wl.pattern.n, wl.pattern.n)
    xs = np.linalg.solve(D, wl.b[..., None])[..., 0]
    sym = W.plain_at_scale(16, grid=4, symmetric=True)
    Ds = W.to_dense(sym.pattern, sym.csr_values).reshape(-1, 16, 16)
    xss = np.linalg.solve(Ds, sym.b[..., None])[..., 0]
    for solver in solvers:
        for fmt in fmts:
            A = wl.matrix(fmt)
            x, it, rel, st = oracle.solve_batch(A, wl.b, solver=solver, tol=1e-12, max_iters=400)
            e = relerr(x, xs).max()
            if not (st == 0).all() or not e <= 1e-9:
                fails.append(f"LU {solver}/{fmt}: err {e:.2e} status {np.unique(st)}")
            x, it, rel, st = oracle.solve_batch(sym.matrix(fmt), sym.b, solver=solver, tol=1e-12)
            e = relerr(x, xss).max()
            if not (st == 0).all() or not e <= 1e-9:
                fails.append(f"LU sym {solver}/{fmt}: err {e:.2e}")
    return fails


def check_diagonal():
    fails = []
    rng = np.random.default_rng(11)
    n = 20
    mats = [np.diag(rng.uniform(0.5, 4.0, n)) for _ in range(8)]
    b = rng.uniform(-1, 1, (8, n))
    exact = np.stack([b[i] / np.diag(m) for i, m in enumerate(mats)])
    for solver in ("bicgstab", "cg", "gmres"):
        x, it, rel, st = solve_dense(mats, b, solver=solver, tol=1e-12)
        if not (it == 1).all() or not (st == 0).all():
            fails.append(f"diagonal {solver}: iters {np.unique(it)} status {np.unique(st)}")
        e = relerr(x, exact).max()
        if not e <= 4e-16:
            fails.append(f"diagonal {solver}: err {e:.2e}")
    return fails


def check_identity():
    fails = []
    rng = np.random.default_rng(12)
    n = 16
    mats = [np.eye(n) for _ in range(4)]
    b = rng.uniform(-1, 1, (4, n))
    for solver in ("bicgstab", "cg", "gmres"):
        for precond in ("jacobi", "none"):
            x, it, rel, st = solve_dense(mats, b, solver=solver, precond=precond, tol=1e-14)
            # BiCGSTAB and CG reproduce b exactly (alpha = 1 exactly); GMRES
            # scales by 1/||r|| and back, which costs a rounding or two.
            same = (np.array_equal(x, b) if solver != "gmres"
                    else np.abs(x - b).max() <= 4 * np.finfo(float).eps * np.abs(b).max())
            if not (it == 1).all() or not same:
                fails.append(f"identity {solver}/{precond}: iters {np.unique(it)} "
                             f"maxdiff {np.abs(x - b).max():.2e}")
            x, it, rel, st = solve_dense(mats, b, b, solver=solver, precond=precond)
            if not (it == 0).all() or not np.array_equal(x, b):
                fails.append(f"identity x0=b {solver}/{precond}: iters {np.unique(it)}")
    return fails


def check_finite_termination():
    fails = []
    rng = np.random.default_rng(13)
    # SPD tridiagonal under CG (unpreconditioned and Jacobi): n steps in exact
    # arithmetic; one extra allowed for the rounding of the last step
    n = 24
    mats = []
    for _ in range(16):
        off = -rng.uniform(0.2, 1.0, n - 1)
        d = np.zeros(n)
        d[:-1] += -off
        d[1:] += -off
        M = np.diag(d * rng.uniform(1.05, 1.5, n)) + np.diag(off, 1) + np.diag(off, -1)
        mats.append(M)
    b = rng.uniform(-1, 1, (16, n))
    for precond in ("none", "jacobi"):
        x, it, rel, st = solve_dense(mats, b, solver="cg", precond=precond, tol=1e-11)
        if not (st == 0).all() or it.max() > n + 1 or it.mean() > n + 0.5:
            fails.append(f"CG finite termination ({precond}): iters {np.bincount(it)}")
    # BiCGSTAB on tiny nonsymmetric systems: n steps (one extra allowed for rounding)
    for n in (3, 5, 8):
        mats = random_dd(rng, n)
        b = rng.uniform(-1, 1, (len(mats), n))
        x, it, rel, st = solve_dense(mats, b, solver="bicgstab", tol=1e-12, max_iters=60)
        if not (st == 0).all() or it.max() > n + 1 or it.mean() > n + 0.2:
            fails.append(f"BiCGSTAB finite termination n={n}: iters {np.bincount(it)}")
    # GMRES with restart >= n: at most n Arnoldi steps
    for n in (4, 9):
        mats = random_dd(rng, n, factor=0.6)
        b = rng.uniform(-1, 1, (len(mats), n))
        x, it, rel, st = solve_dense(mats, b, solver="gmres", restart=n, tol=1e-12, max_iters=60)
        if not (st == 0).all() or it.max() > n:
            fails.append(f"GMRES finite termination n={n}: iters {np.bincount(it)}")
    return fails


def _krylov(Op, v, k):
    cols = [v]
    for _ in range(k - 1):
        cols.append(Op @ cols[-1])
    Q, _ = np.linalg.qr(np.stack(cols, axis=1))
    return Q


def check_gmres_optimal():
    fails = []
    rng = np.random.default_rng(14)
    n = 12
    mats = random_dd(rng, n, factor=0.4, count=12)
    b = rng.uniform(-1, 1, (12, n))
    x0 = rng.uniform(-1, 1, (12, n)) * 0.1
    for k in (1, 2, 4, 7):
        x, it, rel, st = solve_dense(mats, b, x0, solver="gmres", restart=10, tol=1e-300,
                                     max_iters=k)
        for i, A in enumerate(mats):
            Minv = np.diag(1.0 / np.diag(A))
            r0 = b[i] - A @ x0[i]
            Q = _krylov(A @ Minv, r0, k)
            y, *_ = np.linalg.lstsq(A @ Minv @ Q, r0, rcond=None)
            best = np.linalg.norm(r0 - A @ Minv @ Q @ y)
            got = np.linalg.norm(b[i] - A @ x[i])
            if abs(got - best) > 1e-9 * np.linalg.norm(r0):
                fails.append(f"GMRES k={k} sys {i}: residual {got:.6e} vs least squares {best:.6e}")
                break
    return fails


def check_cg_optimal():
    fails = []
    rng = np.random.default_rng(15)
    n = 14
    mats = []
    for _ in range(10):
        G = rng.uniform(-1, 1, (n, n))
        S = 0.5 * (G + G.T)
        S += np.diag(np.abs(S).sum(1) * rng.uniform(1.05, 2.0, n))
        mats.append(S)
    b = rng.uniform(-1, 1, (10, n))
    for k in (1, 2, 3, 5):
        x, it, rel, st = solve_dense(mats, b, solver="cg", tol=1e-300, max_iters=k)
        for i, A in enumerate(mats):
            Minv = np.diag(1.0 / np.diag(A))
            Z = _krylov(Minv @ A, Minv @ b[i], k)
            y = np.linalg.solve(Z.T @ A @ Z, Z.T @ b[i])
            xg = Z @ y
            e = np.linalg.norm(x[i] - xg) / np.linalg.norm(xg)
            if e > 1e-9:
                fails.append(f"CG k={k} sys {i}: Galerkin mismatch {e:.2e}")
                break
    return fails


def _true_rel(A_dense, x, b):
    Al = A_dense.astype(np.longdouble)
    r = b.astype(np.longdouble) - np.einsum("bij,bj->bi", Al, x.astype(np.longdouble))
    return np.sqrt((r * r).sum(1)) / np.sqrt((b.astype(np.longdouble) ** 2).sum(1))


def check_stopping_invariant():
    fails = []
    wl = W.plain_at_scale(128)
    D = W.to_dense(wl.pattern, wl.csr_values).reshape(-1, wl.pattern.n, wl.pattern.n)
    for solver in ("bicgstab", "gmres"):
        x, it, rel, st = oracle.solve_batch(wl.matrix("csr"), wl.b, solver=solver, tol=1e-10)
        tr = _true_rel(D, x, wl.b)
        conv = st == 0
        if not conv.all() or (tr[conv] > 1e-10).any():
            fails.append(f"stopping invariant {solver}: max {float(tr.max()):.3e}")
        if np.abs(rel - tr.astype(np.float64)).max() > 1e-12:
            fails.append(f"logged rel_res {solver} differs from the true residual")
    sym = W.plain_at_scale(128, symmetric=True)
    Ds = W.to_dense(sym.pattern, sym.csr_values).reshape(-1, sym.pattern.n, sym.pattern.n)
    x, it, rel, st = oracle.solve_batch(sym.matrix("csr"), sym.b, solver="cg", tol=1e-10)
    tr = _true_rel(Ds, x, sym.b)
    if not (st == 0).all() or (tr > 1e-10).any():
        fails.append("stopping invariant cg")
    return fails


def check_scaling_and_order():
    fails = []
    wl = W.plain_at_scale(64)
    A = wl.matrix("csr")
    for solver in ("bicgstab", "gmres"):
        x, it, rel, st = oracle.solve_batch(A, wl.b, solver=solver)
        for k in (-3, 5):
            As = A.subset(np.arange(64))
            As.values = A.values * 2.0 ** k
            xs, its, rels, sts = oracle.solve_batch(As, wl.b * 2.0 ** k, solver=solver)
            if not (np.array_equal(x, xs) and np.array_equal(it, its)):
                fails.append(f"power-of-two scaling {solver} k={k}")
        perm = np.random.default_rng(3).permutation(64)
        xp, itp, relp, stp = oracle.solve_batch(A.subset(perm), wl.b[perm], solver=solver)
        if not (np.array_equal(xp, x[perm]) and np.array_equal(itp, it[perm])):
            fails.append(f"batch order {solver}")
    return fails


ALL_CHECKS = [check_lu, check_diagonal, check_identity, check_finite_termination,
              check_gmres_optimal, check_cg_optimal, check_stopping_invariant,
              check_scaling_and_order]


def check_refine():
    """Mixed mode against dense LU: FP64 refinement around an FP32 inner solve
    must still reach the FP64 tolerance and the LU solution."""
    fails = []
    wl = W.mixed_precision(12, grid=10)
    D = W.to_dense(wl.pattern, wl.csr_values).reshape(12, wl.pattern.n, wl.pattern.n)
    xs = np.linalg.solve(D, wl.b[..., None])[..., 0]
    x, it, rel, st, inner = oracle.refine(wl.matrix("ell"), wl.b, tol=1e-10, inner_tol=1e-4)
    e = relerr(x, xs).max()
    tr = _true_rel(D, x, wl.b)
    if not (st == 0).all() or e > 1e-8 or (tr > 1e-10).any() or it.max() > 6:
        fails.append(f"refinement: status {np.unique(st)} err {e:.2e} outer {it.max()}")
    return fails


ALL_CHECKS.append(check_refine)


def _dense_lu_of(row_ptrs, col_idxs, lu_vals, n):
    L = np.eye(n)
    U = np.zeros((n, n))
    for i in range(n):
        for e in range(row_ptrs[i], row_ptrs[i + 1]):
            j = col_idxs[e]
            if j < i:
                L[i, j] = lu_vals[e]
            else:
                U[i, j] = lu_vals[e]
    return L, U


def check_ilu():
    """ILU(0): exact on a tridiagonal matrix (no fill-in exists), so the
    preconditioned solvers finish in one iteration with the LU solution; on a
    general pattern L U reproduces A on the pattern; solutions match LU."""
    fails = []
    wl = W.tiny_tridiagonal(16)
    A = wl.matrix("csr")
    D = W.to_dense(wl.pattern, wl.csr_values).reshape(-1, 32, 32)
    xs = np.linalg.solve(D, wl.b[..., None])[..., 0]
    for solver in ("bicgstab", "gmres"):
        x, it, rel, st = oracle.solve_batch(A, wl.b, solver=solver, precond="ilu0", tol=1e-12)
        if not (it == 1).all() or relerr(x, xs).max() > 1e-12 or not (st == 0).all():
            fails.append(f"ILU tridiagonal {solver}: iters {np.unique(it)} err {relerr(x, xs).max():.2e}")
    for wl in (W.plain_at_scale(8, grid=6), W.pele_like("drm19", 8)):
        p = wl.pattern
        lu = oracle.ilu0(p.row_ptrs, p.col_idxs, wl.csr_values)
        Dn = W.to_dense(p, wl.csr_values).reshape(-1, p.n, p.n)
        rows = np.repeat(np.arange(p.n), np.diff(p.row_ptrs))
        for k in range(len(lu)):
            L, U = _dense_lu_of(p.row_ptrs, p.col_idxs, lu[k], p.n)
            with np.errstate(all="ignore"):  # a broken factorisation may overflow
                prod = L @ U
            e = np.abs(prod[rows, p.col_idxs] - Dn[k][rows, p.col_idxs]).max() / np.abs(Dn[k]).max()
            if e > 1e-13:
                fails.append(f"ILU pattern identity on {wl.name}: {e:.2e}")
                break
        xs = np.linalg.solve(Dn, wl.b[..., None])[..., 0]
        for solver in ("bicgstab", "gmres"):
            x, it, rel, st = oracle.solve_batch(wl.matrix("csr"), wl.b, solver=solver, precond="ilu0",
                                                tol=1e-12)
            if not (st == 0).all() or relerr(x, xs).max() > 1e-9:
                fails.append(f"ILU {solver} on {wl.name}: err {relerr(x, xs).max():.2e}")
    return fails


ALL_CHECKS.append(check_ilu)
