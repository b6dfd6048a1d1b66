"""How much of a time step's change of solution the learned guess's inputs can
predict, measured on the time-stepped workload itself (CPU, dense LU).

The learned initial guess sees diag(A(t)), b(t) and x(t-1). The change
x(t) - x(t-1) = A(t)^-1 (b(t) - A(t) x(t-1)) depends on the off-diagonals of
A(t) and on the drift of b, which those inputs do not show. This test fits,
at each step separately (an upper bound on what a network trained on other
steps can do), the best linear predictor of the change from local features
of the inputs (a row's own and its stencil neighbours' values, and their
products with diag(A(t))'s mean, which encodes t), and checks that it
removes only a small part of the residual of x0 = x(t-1). The numbers behind
the learned guess's measured result: it can only match x(t-1) in iterations,
so its cost decides the comparison.
"""

import numpy as np

from paper_2308_08417_gb300 import workloads as W


def _solutions(ts, steps):
    pat, n = ts.pattern, ts.pattern.n
    rows = np.repeat(np.arange(n), np.diff(pat.row_ptrs))

    def dense(vals):
        M = np.zeros((vals.shape[0], n, n))
        M[:, rows, pat.col_idxs] = vals
        return M

    xs = [np.linalg.solve(dense(ts.values_at(t)), ts.rhs_at(t)[..., None])[..., 0] for t in range(steps)]
    return np.array(xs), dense, rows


def test_inputs_predict_little_of_the_change():
    B, steps = 48, 97
    ts = W.time_stepped(num_batch=B, steps=steps)
    xs, dense, rows = _solutions(ts, steps)
    pat, n = ts.pattern, ts.pattern.n
    diagpos = np.nonzero(rows == pat.col_idxs)[0]
    off = rows != pat.col_idxs
    adj = np.zeros((n, n))
    adj[rows[off], pat.col_idxs[off]] = 1.0

    def feats(t):
        d = ts.values_at(t)[:, diagpos]
        b = ts.rhs_at(t)
        x = xs[t - 1]
        s = d.mean(axis=1, keepdims=True)
        base = [x, b, b / d, x * d, x @ adj.T, b @ adj.T, (b / d) @ adj.T]
        return np.stack(base + [f * s for f in base], axis=-1)

    def rel_residual(t, x0):
        r = ts.rhs_at(t) - np.einsum("bij,bj->bi", dense(ts.values_at(t)), x0)
        return float(np.mean(np.linalg.norm(r, axis=1) / np.linalg.norm(ts.rhs_at(t), axis=1)))

    for t in (64, 80, 96):
        F = feats(t)
        dx = xs[t] - xs[t - 1]
        coef, *_ = np.linalg.lstsq(F.reshape(-1, F.shape[-1]), dx.reshape(-1), rcond=None)
        pred = F @ coef
        # least squares on the change: never a larger solution error than x(t-1)
        assert np.linalg.norm(dx - pred) <= np.linalg.norm(dx) * (1 + 1e-12)
        persist = rel_residual(t, xs[t - 1])
        best = rel_residual(t, xs[t - 1] + pred)
        # yet the best per-step linear fit removes under a fifth of the residual
        assert best > 0.8 * persist, (t, persist, best)
