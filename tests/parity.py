"""Comparison of a GPU solve with the CPU oracle on the same seeded inputs.

Bar (stated per system):
  * status codes equal exactly;
  * iteration counts within +-2 (tree vs serial reductions change rounding),
    or, where a test says so, within +-2 plus the oracle's own spread when
    the values are perturbed at rounding level (iteration_spread);
  * relative solution error <= 1e-8 for converged systems at tol 1e-10;
  * the logged relative residual of every converged system is <= tol and
    matches the residual of the returned x recomputed on the host in long
    double to 1e-3 relative (the residual of a converged x is itself a
    cancellation result with a few significant digits).
"""

from __future__ import annotations

import numpy as np

SOL_TOL = 1e-8
ITER_TOL = 2


def host_rel_residual(dense, x, b):
    """||b - A x|| / ||b|| per system in long double; dense is [B, n, n]."""
    xl = x.astype(np.longdouble)
    r = b.astype(np.longdouble) - np.einsum("bij,bj->bi", dense.astype(np.longdouble), xl)
    return (np.sqrt((r * r).sum(1)) / np.sqrt((b.astype(np.longdouble) ** 2).sum(1))).astype(np.float64)


def compare(x_gpu, it_gpu, rel_gpu, st_gpu, x_ref, it_ref, st_ref, *, tol=1e-10, rel_host=None,
            iter_tol=ITER_TOL, sol_tol=SOL_TOL, label=""):
    fails = []
    if not np.array_equal(st_gpu, st_ref):
        bad = np.nonzero(st_gpu != st_ref)[0][:8]
        fails.append(f"{label} status differs at {bad}: gpu {st_gpu[bad]} oracle {st_ref[bad]}")
    d = np.abs(it_gpu.astype(np.int64) - it_ref.astype(np.int64))
    over = d - np.broadcast_to(np.asarray(iter_tol, dtype=np.int64), d.shape)
    if over.max(initial=0) > 0:
        i = int(np.argmax(over))
        fails.append(f"{label} iterations differ by {d[i]} (system {i}: gpu {it_gpu[i]} oracle {it_ref[i]}, "
                     f"allowed {np.broadcast_to(iter_tol, d.shape)[i]})")
    conv = (st_ref == 0) & (st_gpu == 0)
    if conv.any():
        e = np.linalg.norm(x_gpu[conv] - x_ref[conv], axis=1) / np.maximum(
            np.linalg.norm(x_ref[conv], axis=1), 1e-300)
        if e.max() > sol_tol:
            fails.append(f"{label} relative solution error {e.max():.3e} > {sol_tol}")
        if (rel_gpu[conv] > tol).any():
            fails.append(f"{label} logged rel_res above tol: {rel_gpu[conv].max():.3e}")
        if rel_host is not None:
            rh = rel_host[conv]
            dev = np.abs(rel_gpu[conv] - rh) / np.maximum(rh, 1e-300)
            if (dev > 1e-3).any() and (np.abs(rel_gpu[conv] - rh) > 1e-15).any():
                fails.append(f"{label} logged rel_res differs from the host recomputation by {dev.max():.2e}")
            if (rh > tol * (1 + 1e-6)).any():
                fails.append(f"{label} host-recomputed residual above tol: {rh.max():.3e}")
    return fails


def iteration_spread(solve, A, b, *args, seeds=range(1, 9), rel=1e-15, **kw):
    """Per system, the range of the oracle's own iteration counts when the
    matrix values are perturbed by `rel` relative (eight seeds): how far
    rounding alone moves that system's count."""
    its = []
    for s in seeds:
        rng = np.random.default_rng(s)
        Ap = A.subset(np.arange(A.num_batch))
        Ap.values = A.values * (1.0 + rel * rng.uniform(-1.0, 1.0, A.values.shape))
        its.append(np.asarray(solve(Ap, b, *args, **kw)[1], dtype=np.int64))
    its = np.array(its)
    return its.max(axis=0) - its.min(axis=0)
