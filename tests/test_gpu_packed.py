"""Packed BiCGSTAB, CG and GMRES (several systems per warp in lockstep) against the CPU oracle.

Each aligned group of L = 4, 8 or 16 lanes owns one system. The tests cover:
every lane width; rows per lane from 1 to the maximum of 10, ragged in n;
batches that leave part of the last warp empty; all three formats; Jacobi
and no preconditioner; and warps whose systems stop at different iterations
and for different reasons (per-system predication).
"""

import numpy as np
import pytest
import torch

import oracle
from paper_2308_08417_gb300 import workloads as W
from tests.parity import compare, host_rel_residual, iteration_spread
from tests.test_gpu_parity import dense_of, gpu_solve

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bbs():
    from paper_2308_08417_gb300 import _build, bbs as mod

    _build.build()
    return mod


@pytest.fixture(scope="module")
def handle(bbs):
    return bbs.Handle(0)


def stencil_batch(n, B, seed, kind="1d3"):
    if kind == "1d3":
        pat = W.stencil_pattern("1d3", n)
    else:
        g = int(round(n ** 0.5))
        pat = W.stencil_pattern(kind, g, g)
    rng = np.random.default_rng(seed)
    vals = W.stencil_values(pat, B, rng, 0.05, 0.5)
    b = rng.uniform(-1, 1, (B, pat.n))
    return pat, vals, b


@pytest.mark.parametrize("L", [4, 8, 16])
@pytest.mark.parametrize("R", [1, 2, 3, 5, 7, 9, 10])
def test_lane_widths_and_rows(bbs, handle, L, R):
    """n = L*R - (L // 2 if R > 1) is ragged in the last row group; 37 systems
    leave the last warp partly empty."""
    n = L * R - (L // 2 if R > 1 else 0)
    pat, vals, b = stencil_batch(n, 37, 100 * L + R)
    A = W.make_batch(pat, vals, "csr")
    g = gpu_solve(bbs, handle, A, b, threads_per_system=L, max_iters=1000)
    r = oracle.solve_batch(A, b, max_iters=1000)
    D = W.to_dense(pat, vals).reshape(-1, n, n)
    fails = compare(*g[:4], r[0], r[1], r[3], rel_host=host_rel_residual(D, g[0], b),
                    label=f"L={L} R={R} n={n}")
    assert not fails, "\n".join(fails)


@pytest.mark.parametrize("fmt", ["csr", "ell", "dense"])
@pytest.mark.parametrize("precond", ["jacobi", "none"])
def test_formats_and_preconditioners(bbs, handle, fmt, precond):
    wl = W.plain_at_scale(203, grid=8)  # n = 64: L = 8 by default (R = 8)
    A = wl.matrix(fmt)
    for L in (0, 16):
        g = gpu_solve(bbs, handle, A, wl.b, threads_per_system=L, precond=precond, max_iters=2000)
        r = oracle.solve_batch(A, wl.b, precond=precond, max_iters=2000)
        # Without preconditioning some iteration counts of this batch are
        # sensitive to rounding (the oracle itself moves by up to 4 iterations
        # on one system when the values are perturbed by 1e-15 relative): each
        # system gets +-2 plus its own spread. Solutions and residuals keep
        # the full bar.
        spread = iteration_spread(oracle.solve_batch, A, wl.b, precond=precond, max_iters=2000)
        fails = compare(*g[:4], r[0], r[1], r[3], rel_host=host_rel_residual(dense_of(wl), g[0], wl.b),
                        iter_tol=2 + spread, label=f"{fmt}/{precond}/L={L}")
        assert not fails, "\n".join(fails)


def test_pele_shaped(bbs, handle):
    """Random structurally symmetric patterns (dense-ish rows of uneven length)."""
    for mech in ("drm19", "gri12"):
        wl = W.pele_like(mech, 300)
        A = wl.matrix("csr")
        for L in (4, 8):
            g = gpu_solve(bbs, handle, A, wl.b, threads_per_system=L)
            r = oracle.solve_batch(A, wl.b)
            fails = compare(*g[:4], r[0], r[1], r[3], rel_host=host_rel_residual(dense_of(wl), g[0], wl.b),
                            label=f"{mech}/L={L}")
            assert not fails, "\n".join(fails)


def test_mixed_outcomes_in_one_warp(bbs, handle):
    """Eight systems in one warp (L = 4) that stop at different iterations and
    for different reasons; each must match the oracle on its own."""
    n = 24
    pat, vals, b = stencil_batch(n, 8, 7)
    is_diag = pat.col_idxs == np.repeat(np.arange(n), np.diff(pat.row_ptrs))
    vals = vals.copy()
    off = np.abs(np.where(is_diag, 0.0, vals[6]))
    row_off = np.add.reduceat(off, pat.row_ptrs[:-1])
    vals[6, is_diag] = 1.01 * row_off                # barely dominant: many iterations
    b = b.copy()
    D = W.to_dense(pat, vals).reshape(-1, n, n)
    x0 = np.zeros_like(b)
    x0[4] = np.linalg.solve(D[4], b[4])              # starts converged
    x0[7] = np.linalg.solve(D[7], b[7]) * (1 + 1e-7)  # a few iterations
    b[1] = 0.0                                       # b = 0: x = 0, 0 iterations
    b[3, 2] = np.inf                                 # Inf in the right-hand side
    A = W.make_batch(pat, vals, "csr")
    A.values[2, 5] = np.nan                          # NaN in the matrix
    A.values[5] = 0.0                                # zero matrix: breakdown
    g = gpu_solve(bbs, handle, A, b, x0, threads_per_system=4, max_iters=300)
    r = oracle.solve_batch(A, b, x0, max_iters=300)
    assert list(g[3]) == list(r[3]), (g[3], r[3])
    assert g[3][1] == 0 and g[1][1] == 0 and (g[0][1] == 0).all()
    assert g[3][2] == 3 and g[3][3] == 3 and g[3][5] == 2
    assert g[1][4] == 0 and np.array_equal(g[0][4], x0[4])
    assert r[1][7] < r[1][0] < r[1][6]
    keep = np.array([0, 4, 6, 7])
    fails = compare(g[0][keep], g[1][keep], g[2][keep], g[3][keep], r[0][keep], r[1][keep], r[3][keep],
                    label="mixed outcomes")
    assert not fails, "\n".join(fails)
    # an iteration cap between the easy and the hard systems stops the hard
    # ones with MAX_ITER while the easy one converges
    cap = int(r[1][7]) + 3
    if r[1][0] > cap + 3:
        g = gpu_solve(bbs, handle, A, b, x0, threads_per_system=4, max_iters=cap)
        assert g[3][7] == 0 and g[3][0] == 1 and g[3][6] == 1 and g[1][0] == cap
    # max_iters = 0 moves nothing
    g = gpu_solve(bbs, handle, A, b, x0 + 0.5, threads_per_system=4, max_iters=0)
    ok = np.array([0, 4, 6, 7])
    assert (g[1] == 0).all() and (g[3][ok] == 1).all() and np.array_equal(g[0][ok], (x0 + 0.5)[ok])


@pytest.mark.parametrize("L", [4, 8, 16])
@pytest.mark.parametrize("R", [1, 3, 6, 10])
def test_cg_lane_widths_and_rows(bbs, handle, L, R):
    """Packed CG on symmetric positive definite batches (1D and 2D stencils)."""
    n = L * R - (L // 2 if R > 1 else 0)
    pat = W.stencil_pattern("1d3", n)
    rng = np.random.default_rng(500 + 10 * L + R)
    vals = W.stencil_values(pat, 37, rng, 0.05, 0.5, symmetric=True)
    b = rng.uniform(-1, 1, (37, n))
    for fmt in ("csr", "ell"):
        A = W.make_batch(pat, vals, fmt)
        g = gpu_solve(bbs, handle, A, b, solver="cg", threads_per_system=L, max_iters=1000)
        r = oracle.solve_batch(A, b, solver="cg", max_iters=1000)
        D = W.to_dense(pat, vals).reshape(-1, n, n)
        fails = compare(*g[:4], r[0], r[1], r[3], rel_host=host_rel_residual(D, g[0], b),
                        label=f"cg {fmt} L={L} R={R} n={n}")
        assert not fails, "\n".join(fails)


def test_cg_default_and_edges(bbs, handle):
    sym = W.plain_at_scale(301, symmetric=True)
    A = sym.matrix("csr")
    dA = bbs.DeviceBatch.from_batch(A, "cuda")
    assert handle.describe(dA, bbs.bbs_default_options(solver="cg"))["kernel"] == "cg_packed_kernel"
    vals = A.values.copy()
    b = sym.b.copy()
    b[3] = 0.0
    vals[5, 7] = np.nan
    b[9, 0] = np.inf
    A2 = A.subset(np.arange(301))
    A2.values = vals
    x0 = np.full_like(b, 0.1)
    for precond in ("jacobi", "none"):
        g = gpu_solve(bbs, handle, A2, b, x0, solver="cg", precond=precond)
        r = oracle.solve_batch(A2, b, x0, solver="cg", precond=precond)
        assert g[3][5] == 3 and g[3][9] == 3 and g[3][3] == 0 and g[1][3] == 0 and (g[0][3] == 0).all()
        keep = np.setdiff1d(np.arange(301), [5, 9])
        fails = compare(g[0][keep], g[1][keep], g[2][keep], g[3][keep], r[0][keep], r[1][keep], r[3][keep],
                        label=f"cg edges {precond}")
        assert not fails, "\n".join(fails)
    g0 = gpu_solve(bbs, handle, A, sym.b, x0, solver="cg", max_iters=0)
    assert (g0[1] == 0).all() and (g0[3] == 1).all() and np.array_equal(g0[0], x0)


@pytest.mark.parametrize("L", [4, 8, 16])
@pytest.mark.parametrize("R,restart", [(1, 10), (3, 3), (6, 10), (9, 1), (10, 32)])
def test_gmres_lane_widths_rows_and_restarts(bbs, handle, L, R, restart):
    """Packed GMRES(m) on nonsymmetric batches: every lane width, rows per lane
    up to 10, restart lengths from 1 to 32, a partly empty last warp."""
    n = L * R - (L // 2 if R > 1 else 0)
    pat, vals, b = stencil_batch(n, 37, 900 + 10 * L + R)
    for fmt in ("csr", "ell"):
        A = W.make_batch(pat, vals, fmt)
        g = gpu_solve(bbs, handle, A, b, solver="gmres", gmres_restart=restart, threads_per_system=L,
                      max_iters=2000)
        r = oracle.solve_batch(A, b, solver="gmres", restart=restart, max_iters=2000)
        D = W.to_dense(pat, vals).reshape(-1, n, n)
        fails = compare(*g[:4], r[0], r[1], r[3], rel_host=host_rel_residual(D, g[0], b),
                        label=f"gmres({restart}) {fmt} L={L} R={R} n={n}")
        assert not fails, "\n".join(fails)


def test_gmres_default_and_edges(bbs, handle):
    wl = W.plain_at_scale(301)
    A = wl.matrix("csr")
    dA = bbs.DeviceBatch.from_batch(A, "cuda")
    info = handle.describe(dA, bbs.bbs_default_options(solver="gmres"))
    assert info["kernel"] == "gmres_packed_kernel" and info["threads_per_system"] == 16
    vals = A.values.copy()
    b = wl.b.copy()
    b[3] = 0.0
    vals[5, 7] = np.nan
    b[9, 0] = np.inf
    A2 = A.subset(np.arange(301))
    A2.values = vals
    x0 = np.full_like(b, 0.1)
    for precond in ("jacobi", "none"):
        g = gpu_solve(bbs, handle, A2, b, x0, solver="gmres", precond=precond)
        r = oracle.solve_batch(A2, b, x0, solver="gmres", precond=precond)
        assert g[3][5] == 3 and g[3][9] == 3 and g[3][3] == 0 and g[1][3] == 0 and (g[0][3] == 0).all()
        keep = np.setdiff1d(np.arange(301), [5, 9])
        spread = iteration_spread(oracle.solve_batch, A2.subset(keep), b[keep], x0[keep], solver="gmres",
                                  precond=precond)
        fails = compare(g[0][keep], g[1][keep], g[2][keep], g[3][keep], r[0][keep], r[1][keep], r[3][keep],
                        iter_tol=2 + spread, label=f"gmres edges {precond}")
        assert not fails, "\n".join(fails)
    g0 = gpu_solve(bbs, handle, A, wl.b, x0, solver="gmres", max_iters=0)
    assert (g0[1] == 0).all() and (g0[3] == 1).all() and np.array_equal(g0[0], x0)
    # a cap in the middle of a cycle stops every system with MAX_ITER after exactly 7 steps
    g7 = gpu_solve(bbs, handle, A, wl.b, solver="gmres", max_iters=7)
    assert (g7[3] == 1).all() and (g7[1] == 7).all()


def test_results_do_not_depend_on_warp_partners(bbs, handle):
    """A system's bits do not depend on which systems share its warp."""
    wl = W.plain_at_scale(512)
    A = wl.matrix("csr")
    base = gpu_solve(bbs, handle, A, wl.b, threads_per_system=16)
    perm = np.random.default_rng(3).permutation(512)
    pr = gpu_solve(bbs, handle, A.subset(perm), wl.b[perm], threads_per_system=16)
    assert np.array_equal(pr[0], base[0][perm]) and np.array_equal(pr[1], base[1][perm])
    one = gpu_solve(bbs, handle, A.subset(np.array([77])), wl.b[77:78], threads_per_system=16)
    assert np.array_equal(one[0][0], base[0][77])


def test_default_plan_is_packed_for_small_systems(bbs, handle):
    wl = W.plain_at_scale(64)
    A = bbs.DeviceBatch.from_batch(wl.matrix("csr"), "cuda")
    info = handle.describe(A, bbs.bbs_default_options())
    assert info["kernel"] == "bicgstab_packed_kernel" and info["threads_per_system"] == 16
    assert info["rows"] == 9 and info["launches"] == 2  # the CSR column table, then the solver
    assert info["block"] == 32 and info["grid"] == 32
    # without the row-length bound a CSR batch runs one system per warp
    nohint = bbs.DeviceBatch("csr", A.n, A.nnz, 0, A.row_ptrs, A.col_idxs, A.values)
    info = handle.describe(nohint, bbs.bbs_default_options())
    assert info["kernel"] == "bicgstab_folded_kernel" and info["launches"] == 1
    big = W.mixed_precision(4)
    info = handle.describe(bbs.DeviceBatch.from_batch(big.matrix("ell"), "cuda"), bbs.bbs_default_options())
    assert info["kernel"] == "bicgstab_folded_kernel" and info["threads_per_system"] == 128


def test_packed_argument_errors(bbs, handle):
    wl = W.tiny_tridiagonal(4)
    dA = bbs.DeviceBatch.from_batch(wl.matrix("csr"), "cuda")
    b = torch.as_tensor(wl.b, device="cuda")
    x = torch.zeros_like(b)
    log = bbs.Log.empty(4)
    bad = [dict(threads_per_system=8, solver="gmres", precond="ilu0"), dict(threads_per_system=16, solver="gmres", precision="mixed"),
           dict(threads_per_system=4, precision="mixed"), dict(threads_per_system=16, values_in_smem=-1),
           dict(threads_per_system=2), dict(threads_per_system=4, precond="ilu0")]
    for kw in bad:
        with pytest.raises(bbs.BBSError):
            handle.solve(dA, b, x, bbs.bbs_default_options(**kw), log)
    # packed CSR needs the row-length bound
    nohint = bbs.DeviceBatch("csr", dA.n, dA.nnz, 0, dA.row_ptrs, dA.col_idxs, dA.values)
    with pytest.raises(bbs.BBSError):
        handle.solve(nohint, b, x, bbs.bbs_default_options(threads_per_system=8), log)
    # n = 41 on 4 lanes would need 11 rows per lane
    pat, vals, bb = stencil_batch(41, 4, 1)
    dB = bbs.DeviceBatch.from_batch(W.make_batch(pat, vals, "csr"), "cuda")
    with pytest.raises(bbs.BBSError):
        handle.solve(dB, torch.as_tensor(bb, device="cuda"), torch.zeros(4, 41, dtype=torch.float64, device="cuda"),
                     bbs.bbs_default_options(threads_per_system=4), log)


def test_csr_row_longer_than_bound_is_an_argument_error(bbs, handle):
    """A CSR bound (ell_k) below the longest row: bbs_solve and bbs_solve_host
    return BBS_ERR_INVALID_ARG before any launch and x is left alone; the right
    bound solves the batch."""
    wl = W.tiny_tridiagonal(40)
    A = wl.matrix("csr")
    good = bbs.DeviceBatch.from_batch(A, "cuda")
    assert good.ell_k == 3
    bad = bbs.DeviceBatch("csr", good.n, good.nnz, 2, good.row_ptrs, good.col_idxs, good.values)
    b = torch.as_tensor(wl.b, device="cuda")
    x0 = torch.full_like(b, 0.25)
    for tps in (4, 8):
        x = x0.clone()
        log = bbs.Log.empty(40)
        o = bbs.bbs_default_options(threads_per_system=tps)
        for _ in range(2):  # the second call answers from the handle's record
            with pytest.raises(bbs.BBSError) as err:
                handle.solve(bad, b, x, o, log, handle.workspace(bad, o))
            assert err.value.status == 1
        torch.cuda.synchronize()
        assert torch.equal(x, x0)
        g = gpu_solve(bbs, handle, A, wl.b, threads_per_system=tps)
        assert (g[3] == 0).all()
    hbad = bbs.DeviceBatch("csr", good.n, good.nnz, 2, good.row_ptrs.cpu(), good.col_idxs.cpu(),
                           good.values.cpu())
    hx = x0.cpu()
    with pytest.raises(bbs.BBSError) as err:
        handle.solve_host(hbad, b.cpu(), hx, bbs.bbs_default_options(threads_per_system=4),
                          bbs.Log.empty(40, device="cpu"))
    assert err.value.status == 1 and torch.equal(hx, x0.cpu())


def test_csr_pattern_rewritten_in_place_reports_nan(bbs, handle):
    """The device-side guard behind the handle's record: a pattern checked once
    and then rewritten in place (same address, n, nnz and bound) with a row
    longer than the bound makes every system report NAN, x untouched."""
    wl = W.tiny_tridiagonal(40)
    A = wl.matrix("csr")
    dA = bbs.DeviceBatch.from_batch(A, "cuda")
    b = torch.as_tensor(wl.b, device="cuda")
    o = bbs.bbs_default_options(threads_per_system=8)
    x = torch.zeros_like(b)
    log = bbs.Log.empty(40)
    handle.solve(dA, b, x, o, log, handle.workspace(dA, o))  # the pattern is checked and remembered
    torch.cuda.synchronize()
    assert (log.status.cpu().numpy() == 0).all()
    # same n = 32 and nnz = 94: row 0 holds columns 0..3, row 1 only its diagonal
    n = A.n
    rows = [[0, 1, 2, 3], [1]] + [[i - 1, i, i + 1] for i in range(2, n - 1)] + [[n - 2, n - 1]]
    rp = np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int32)
    assert rp[-1] == A.nnz
    dA.row_ptrs.copy_(torch.as_tensor(rp))
    dA.col_idxs.copy_(torch.as_tensor(np.concatenate(rows).astype(np.int32)))
    x0 = torch.full_like(b, 0.25)
    x = x0.clone()
    handle.solve(dA, b, x, o, log, handle.workspace(dA, o))
    torch.cuda.synchronize()
    assert (log.status.cpu().numpy() == 3).all() and (log.iters.cpu().numpy() == 0).all()
    assert torch.equal(x, x0)


def test_host_buffer_chunks_match_the_device_solve(bbs, handle):
    """bbs_solve_host splits a batch of more than 128 MB of input into chunks
    on two streams (here 20,001 systems, 154 MB, ragged last chunk); every
    system's bits equal those of one device-buffer solve."""
    wl = W.plain_at_scale(20001)
    A = wl.matrix("csr")
    dev = gpu_solve(bbs, handle, A, wl.b)
    hA = bbs.DeviceBatch.from_batch(A, "cpu", pin=True)
    hb = torch.as_tensor(wl.b).pin_memory()
    hx = torch.zeros_like(hb).pin_memory()
    log = bbs.Log.empty(20001, device="cpu", pin=True)
    handle.solve_host(hA, hb, hx, bbs.bbs_default_options(), log)
    assert np.array_equal(hx.numpy(), dev[0])
    assert np.array_equal(log.iters.numpy(), dev[1]) and np.array_equal(log.status.numpy(), dev[3])
    assert np.array_equal(log.rel_res.numpy(), dev[2])


@pytest.mark.parametrize("exp", [300, -300])
def test_extreme_scales_take_the_plain_divisions(bbs, handle, exp):
    """b scaled by 2^exp: every iterate scales exactly, but (t, t) rho (t, s)
    overflows or underflows, so omega and the next beta fall back to plain
    divisions. The packed BiCGSTAB and CG and the one-system-per-warp
    BiCGSTAB still meet the oracle bar on the scaled batch and take the
    iterations of the unscaled one (within the bar)."""
    scale = 2.0 ** exp
    for solver, symmetric in (("bicgstab", False), ("cg", True)):
        wl = W.plain_at_scale(97, symmetric=symmetric)
        A = wl.matrix("csr")
        b = wl.b * scale
        r = oracle.solve_batch(A, b, solver=solver)
        r1 = oracle.solve_batch(A, wl.b, solver=solver)
        assert np.array_equal(r[1], r1[1])  # the oracle's iterates scale exactly
        for tps in (0, 32):
            g = gpu_solve(bbs, handle, A, b, solver=solver, threads_per_system=tps)
            fails = compare(*g[:4], r[0], r[1], r[3], rel_host=host_rel_residual(dense_of(wl), g[0], b),
                            label=f"{solver} tps={tps} 2^{exp}")
            assert not fails, "\n".join(fails)
            g1 = gpu_solve(bbs, handle, A, wl.b, solver=solver, threads_per_system=tps)
            assert np.abs(g[1].astype(int) - g1[1].astype(int)).max() <= 2
