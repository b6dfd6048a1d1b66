"""Parity at the benchmark workloads' full sizes, in the launch configurations
the bench times, on sampled systems that the oracle solves one by one."""

import numpy as np
import pytest
import torch

import oracle
from paper_2308_08417_gb300 import workloads as W
from tests.parity import compare
from tests.test_gpu_varsize import check_against_oracle, run_plan

pytestmark = pytest.mark.gpu

# the bench's mixed-refinement options (inner tolerance from its sweep)
MIXED = dict(precision="mixed", inner_tol=3e-3, max_iters=200, max_outer=30)


@pytest.fixture(scope="module")
def bbs():
    from paper_2308_08417_gb300 import _build, bbs as mod

    _build.build()
    return mod


@pytest.fixture(scope="module")
def handle(bbs):
    return bbs.Handle(0)


def solve(bbs, handle, A, b, **opts):
    dA = bbs.DeviceBatch.from_batch(A, "cuda")
    x, log = bbs.solve(dA, torch.as_tensor(b, device="cuda"), handle=handle, **opts)
    torch.cuda.synchronize()
    inner = None if log.inner_iters is None else log.inner_iters.cpu().numpy()
    return (x.cpu().numpy(), log.iters.cpu().numpy(), log.rel_res.cpu().numpy(),
            log.status.cpu().numpy(), inner)


def sample(num_batch, k, seed):
    return np.sort(np.random.default_rng(seed).choice(num_batch, k, replace=False))


def csr_rel_residual(pattern, values, x, b):
    """||b - A x|| / ||b|| per system in long double, A from the CSR pattern."""
    rows = np.repeat(np.arange(pattern.n), np.diff(pattern.row_ptrs))
    xl, bl = x.astype(np.longdouble), b.astype(np.longdouble)
    out = np.empty(len(x))
    for i in range(len(x)):
        ax = np.zeros(pattern.n, dtype=np.longdouble)
        np.add.at(ax, rows, values[i].astype(np.longdouble) * xl[i][pattern.col_idxs])
        r = bl[i] - ax
        out[i] = float(np.sqrt((r * r).sum()) / np.sqrt((bl[i] * bl[i]).sum()))
    return out


@pytest.mark.parametrize("solver,precond", [("cg", "jacobi"), ("gmres", "jacobi"), ("bicgstab", "ilu0")])
def test_headline_batch_other_solvers_sampled(bbs, handle, solver, precond):
    """65,536 systems of n = 144 (packed, 2 per warp): CG on the symmetrised
    copy, GMRES(10) and BiCGSTAB + ILU(0), 512 systems checked."""
    wl = W.plain_at_scale(symmetric=(solver == "cg"))
    A = wl.matrix("csr")
    g = solve(bbs, handle, A, wl.b, solver=solver, precond=precond)
    idx = sample(wl.num_batch, 512, 5)
    r = oracle.solve_batch(A.subset(idx), wl.b[idx], solver=solver, precond=precond)
    assert (g[3] == 0).all()
    rh = csr_rel_residual(wl.pattern, wl.csr_values[idx], g[0][idx], wl.b[idx])
    fails = compare(g[0][idx], g[1][idx], g[2][idx], g[3][idx], r[0], r[1], r[3], rel_host=rh,
                    label=f"{solver}+{precond} full size")
    assert not fails, "\n".join(fails)


def test_mixed_batch_full_size_sampled(bbs, handle):
    """16,384 systems of n = 1,024 (9-point, ELL) through FP32-inner / FP64-outer
    refinement: every system reaches the FP64 tolerance, and 32 sampled
    systems match the FP64 oracle's solution within 1e-8 and the oracle's
    refinement in outer steps within 1."""
    wl = W.mixed_precision()
    A = wl.matrix("ell")
    g = solve(bbs, handle, A, wl.b, **MIXED)
    assert (g[3] == 0).all() and (g[2] <= 1e-10).all()
    idx = sample(wl.num_batch, 32, 3)
    x64 = oracle.solve_batch(A.subset(idx), wl.b[idx], max_iters=2000)[0]
    xr, itr, relr, str_, inr = oracle.refine(A.subset(idx), wl.b[idx], inner_tol=MIXED["inner_tol"],
                                             max_inner=MIXED["max_iters"], max_outer=MIXED["max_outer"])
    e = np.linalg.norm(g[0][idx] - x64, axis=1) / np.linalg.norm(x64, axis=1)
    assert e.max() <= 1e-8
    assert (str_ == 0).all() and np.abs(g[1][idx].astype(int) - itr).max() <= 1
    rh = csr_rel_residual(wl.pattern, wl.csr_values[idx], g[0][idx], wl.b[idx])
    assert (rh <= 1e-10 * (1 + 1e-6)).all()


def test_uneven_batch_full_size_tuned_sampled(bbs, handle):
    """100,000 systems of n in [16, 1024] through the tuned, graph-captured
    persistent launch (the bench's configuration), 300 systems checked."""
    vb = W.uneven(100000)
    vbd = bbs.VarDeviceBatch.from_varbatch(vb)
    b = torch.as_tensor(vb.b, device="cuda")
    x0 = torch.as_tensor(vb.x0, device="cuda")
    opts = bbs.bbs_default_options()
    tuning = bbs.bbs_var_tune(handle, vbd, b, x0, opts, sample=512)
    plan = bbs.VarPlan(handle, vbd, opts, tuning)
    got = run_plan(bbs, plan, vb)
    assert (got[3] == 0).all()
    fails = check_against_oracle(vb, got, sample=300)
    assert not fails, "\n".join(fails[:10])
