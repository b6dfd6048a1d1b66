"""CPU oracle of the batched Krylov solvers (plain FP64 C, see bbs_oracle.c).

TEST INFRASTRUCTURE: only tests/, the smoke check and the benchmark's
CPU-baseline leg import this package. It shares no code with the CUDA library.

Parity unpinned (no value outside the oracle fixes them): exact iteration
counts on the random workloads, and the inner tolerance of the mixed mode.
"""

from __future__ import annotations

import contextlib
import ctypes as C

import numpy as np

from . import build as _build

SOLVERS = {"bicgstab": 0, "cg": 1, "gmres": 2}
PRECONDS = {"none": 0, "jacobi": 1, "ilu0": 2}
TOL_TYPES = {"absolute": 0, "relative": 1}
FORMATS = {"csr": 0, "ell": 1, "dense": 2}
STATUS = {0: "converged", 1: "max_iter", 2: "breakdown", 3: "nan"}

_lib = None


def _configure(L):
    p_i32 = np.ctypeslib.ndpointer(np.int32, flags="C")
    p_i64 = np.ctypeslib.ndpointer(np.int64, flags="C")
    p_f64 = np.ctypeslib.ndpointer(np.float64, flags="C")
    p_f32 = np.ctypeslib.ndpointer(np.float32, flags="C")
    ci, cd = C.c_int, C.c_double
    L.om_num_threads.restype = ci
    L.om_spmv_batch.argtypes = [ci, ci, ci, ci, p_i32, p_i32, p_f64, ci, p_f64, p_f64]
    L.om_spmv_batch.restype = None
    L.om_solve_batch.argtypes = [ci, ci, ci, ci, ci, ci, p_i32, p_i32, p_f64, ci, p_f64,
                                 p_f64, ci, cd, ci, ci, p_i32, p_f64, p_i32, ci]
    L.om_solve_batch.restype = None
    L.om_refine_batch.argtypes = [ci, ci, ci, ci, ci, p_i32, p_i32, p_f64, p_f32, ci, p_f64,
                                  p_f64, ci, cd, ci, cd, ci, p_i32, p_f64, p_i32, p_i32, ci]
    L.om_refine_batch.restype = None
    L.om_solve_varsize.argtypes = [ci, ci, ci, p_i32, p_i64, p_i64, p_i32, p_i32, p_i32,
                                   p_i64, p_i64, p_f64, p_f64, p_f64, ci, cd, ci, ci, p_i32,
                                   p_f64, p_i32, ci]
    L.om_solve_varsize.restype = None
    L.om_ilu0_batch.argtypes = [ci, p_i32, p_i32, p_f64, ci, p_f64]
    L.om_ilu0_batch.restype = None
    return L


def lib():
    global _lib
    if _lib is None:
        _lib = _configure(C.CDLL(_build.build()))
    return _lib


@contextlib.contextmanager
def using(path: str):
    """Run the oracle API on another build of the oracle (mutation tests)."""
    global _lib
    saved = _lib
    _lib = _configure(C.CDLL(path))
    try:
        yield
    finally:
        _lib = saved


def num_threads() -> int:
    return int(lib().om_num_threads())


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _pattern_arrays(fmt, row_ptrs, col_idxs, n):
    rp = _i32(row_ptrs if row_ptrs is not None else np.zeros(n + 1))
    ci = _i32(col_idxs if col_idxs is not None else np.zeros(1))
    return rp, ci


def spmv(fmt: str, n: int, nnz: int, ell_k: int, row_ptrs, col_idxs, values, x):
    """y_i = A_i x_i for every system of a batch (values [B, per-system])."""
    values = _f64(values)
    B = values.shape[0]
    x = _f64(x).reshape(B, n)
    y = np.empty((B, n), dtype=np.float64)
    rp, ci = _pattern_arrays(fmt, row_ptrs, col_idxs, n)
    lib().om_spmv_batch(FORMATS[fmt], n, nnz, ell_k, rp, ci, values, B, x, y)
    return y


def solve(fmt: str, n: int, nnz: int, ell_k: int, row_ptrs, col_idxs, values, b, x0=None, *,
          solver="bicgstab", precond="jacobi", tol_type="relative", tol=1e-10,
          max_iters=500, restart=10, threads=0):
    """Solve every system; returns (x [B,n], iters, rel_res, status)."""
    if precond == "ilu0" and (fmt != "csr" or solver == "cg"):
        raise ValueError("ILU(0) preconditions BiCGSTAB and GMRES on BatchCsr")
    values = _f64(values)
    B = values.shape[0]
    b = _f64(b).reshape(B, n)
    x = np.zeros((B, n)) if x0 is None else np.array(x0, dtype=np.float64).reshape(B, n)
    x = np.ascontiguousarray(x)
    iters = np.zeros(B, np.int32)
    rel = np.zeros(B, np.float64)
    status = np.zeros(B, np.int32)
    rp, ci = _pattern_arrays(fmt, row_ptrs, col_idxs, n)
    nt = threads if threads > 0 else num_threads()
    lib().om_solve_batch(SOLVERS[solver], PRECONDS[precond], FORMATS[fmt], n, nnz, ell_k, rp, ci,
                         values, B, b, x, TOL_TYPES[tol_type], float(tol), int(max_iters),
                         int(restart), iters, rel, status, nt)
    return x, iters, rel, status


def solve_batch(A, b, x0=None, **kw):
    """Same as solve() for a workloads.BatchMatrix-like object A."""
    return solve(A.fmt, A.n, A.nnz, A.ell_k, A.row_ptrs, A.col_idxs, A.values, b, x0, **kw)


def refine(A, b, x0=None, *, values32=None, precond="jacobi", tol_type="relative", tol=1e-10,
           max_inner=100, inner_tol=1e-4, max_outer=30, threads=0):
    """Mixed mode: FP32 inner BiCGSTAB in FP64 refinement.

    Returns (x, outer_iters, rel_res, status, inner_iters).
    """
    values = _f64(A.values)
    v32 = np.ascontiguousarray(values.astype(np.float32) if values32 is None else values32,
                               dtype=np.float32)
    B, n = values.shape[0], A.n
    b = _f64(b).reshape(B, n)
    x = np.zeros((B, n)) if x0 is None else np.array(x0, dtype=np.float64).reshape(B, n)
    x = np.ascontiguousarray(x)
    iters = np.zeros(B, np.int32)
    rel = np.zeros(B, np.float64)
    status = np.zeros(B, np.int32)
    inner = np.zeros(B, np.int32)
    rp, ci = _pattern_arrays(A.fmt, A.row_ptrs, A.col_idxs, n)
    nt = threads if threads > 0 else num_threads()
    lib().om_refine_batch(PRECONDS[precond], FORMATS[A.fmt], n, A.nnz, A.ell_k, rp, ci, values,
                          v32, B, b, x, TOL_TYPES[tol_type], float(tol), int(max_inner),
                          float(inner_tol), int(max_outer), iters, rel, status, inner, nt)
    return x, iters, rel, status, inner


def solve_varsize(vb, *, solver="bicgstab", precond="jacobi", tol_type="relative", tol=1e-10,
                  max_iters=500, restart=10, systems=None, threads=0):
    """Solve an uneven batch (workloads.VarBatch); `systems` picks a subset.

    Returns (x_flat, iters, rel_res, status) for the chosen systems, with
    x_flat laid out like vb.b restricted to those systems (same offsets).
    """
    pat_n, pat_nnz, rp_off, ci_off, rps, cis = vb.pools()
    sel = np.arange(vb.num_batch) if systems is None else np.asarray(systems)
    sp = _i32(vb.sys_pattern[sel])
    voff = np.ascontiguousarray(vb.val_off[sel], dtype=np.int64)
    xoff = np.ascontiguousarray(vb.vec_off[sel], dtype=np.int64)
    x = np.array(vb.x0, dtype=np.float64)
    B = len(sel)
    iters = np.zeros(B, np.int32)
    rel = np.zeros(B, np.float64)
    status = np.zeros(B, np.int32)
    nt = threads if threads > 0 else num_threads()
    lib().om_solve_varsize(SOLVERS[solver], PRECONDS[precond], B, pat_n, rp_off, ci_off, rps, cis,
                           sp, voff, xoff, _f64(vb.values), _f64(vb.b), x, TOL_TYPES[tol_type],
                           float(tol), int(max_iters), int(restart), iters, rel, status, nt)
    return x, iters, rel, status


def ilu0(row_ptrs, col_idxs, values):
    """ILU(0) factors (unit L below the diagonal, U on and above) of every
    system of a BatchCsr batch, in the pattern's layout."""
    values = _f64(values)
    B = values.shape[0]
    rp, ci = _i32(row_ptrs), _i32(col_idxs)
    lu = np.empty_like(values)
    lib().om_ilu0_batch(len(rp) - 1, rp, ci, values, B, lu)
    return lu
