"""GPU solves through the C ABI against the CPU oracle (same seeded inputs)."""

import numpy as np
import pytest
import torch

import oracle
from paper_2308_08417_gb300 import workloads as W
from tests.parity import compare, host_rel_residual

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bbs():
    from paper_2308_08417_gb300 import _build, bbs as mod

    _build.build()
    return mod


@pytest.fixture(scope="module")
def handle(bbs):
    return bbs.Handle(0)


def gpu_solve(bbs, handle, A, b, x0=None, *, values_f32=False, **opts):
    dA = bbs.DeviceBatch.from_batch(A, "cuda", values_f32=values_f32)
    bt = torch.as_tensor(np.ascontiguousarray(b), device="cuda")
    x0t = None if x0 is None else torch.as_tensor(np.ascontiguousarray(x0), device="cuda")
    x, log = bbs.solve(dA, bt, x0t, handle=handle, **opts)
    torch.cuda.synchronize()
    inner = None if log.inner_iters is None else log.inner_iters.cpu().numpy()
    return (x.cpu().numpy(), log.iters.cpu().numpy(), log.rel_res.cpu().numpy(),
            log.status.cpu().numpy(), inner)


def dense_of(wl):
    n = wl.pattern.n
    return W.to_dense(wl.pattern, wl.csr_values).reshape(-1, n, n)


# ------------------------------------------------------------ tiny batch

@pytest.mark.parametrize("fmt", ["csr", "ell", "dense"])
@pytest.mark.parametrize("solver", ["bicgstab", "cg", "gmres"])
def test_tiny_tridiagonal(bbs, handle, solver, fmt):
    wl = W.tiny_tridiagonal()
    A = wl.matrix(fmt)
    g = gpu_solve(bbs, handle, A, wl.b, solver=solver, max_iters=200)
    r = oracle.solve_batch(A, wl.b, solver=solver, max_iters=200)
    fails = compare(*g[:4], r[0], r[1], r[3], rel_host=host_rel_residual(dense_of(wl), g[0], wl.b),
                    label=f"{solver}/{fmt}")
    assert not fails, "\n".join(fails)


@pytest.mark.parametrize("threads", [32, 64, 96, 128, 256, 512, 1024])
def test_launch_shapes_agree(bbs, handle, threads):
    """Every rows-per-thread instantiation (R = ceil(n/threads)) meets the bar,
    including ragged tails (n not a multiple of the block)."""
    wl = W.plain_at_scale(96, grid=13)  # n = 169
    A = wl.matrix("csr")
    R = -(-169 // threads)
    if threads > (1024 if R <= 1 else 512 if R <= 4 else 256) or R > 8:
        pytest.skip("shape outside the register tiers")
    g = gpu_solve(bbs, handle, A, wl.b, threads_per_system=threads)
    r = oracle.solve_batch(A, wl.b)
    fails = compare(*g[:4], r[0], r[1], r[3], label=f"threads={threads}")
    assert not fails, "\n".join(fails)


@pytest.mark.parametrize("n", [1, 2, 7, 31, 33, 100, 257, 1000, 2048])
def test_ragged_sizes(bbs, handle, n):
    wl = W.plain_at_scale(8, grid=1) if n == 1 else None
    pat = W.stencil_pattern("1d3", n)
    rng = np.random.default_rng(n)
    vals = W.stencil_values(pat, 8, rng, 0.05, 0.5) if n > 1 else rng.uniform(1, 2, (8, 1))
    b = rng.uniform(-1, 1, (8, n))
    A = W.make_batch(pat, vals, "csr")
    for solver in ("bicgstab", "gmres"):
        g = gpu_solve(bbs, handle, A, b, solver=solver, max_iters=2000)
        r = oracle.solve_batch(A, b, solver=solver, max_iters=2000)
        fails = compare(*g[:4], r[0], r[1], r[3], label=f"n={n} {solver}")
        assert not fails, "\n".join(fails)
    del wl


# ------------------------------------------------- full-size scale batch

@pytest.fixture(scope="module")
def scale():
    return W.plain_at_scale()


@pytest.mark.parametrize("fmt", ["csr", "ell"])
def test_scale_bicgstab_sampled(bbs, handle, scale, fmt):
    """65,536 systems, n = 144, the benchmark's launch configuration; the oracle
    solves a sample of 1,024 systems one by one."""
    A = scale.matrix(fmt)
    g = gpu_solve(bbs, handle, A, scale.b, max_iters=500)
    idx = np.random.default_rng(7).choice(scale.num_batch, 1024, replace=False)
    idx.sort()
    r = oracle.solve_batch(A.subset(idx), scale.b[idx], max_iters=500)
    assert (g[3] == 0).all()
    D = W.to_dense(scale.pattern, scale.csr_values[idx]).reshape(-1, 144, 144)
    fails = compare(g[0][idx], g[1][idx], g[2][idx], g[3][idx], r[0], r[1], r[3],
                    rel_host=host_rel_residual(D, g[0][idx], scale.b[idx]), label=f"scale/{fmt}")
    assert not fails, "\n".join(fails)


def test_scale_gmres_and_cg_sampled(bbs, handle):
    wl = W.plain_at_scale(8192)
    A = wl.matrix("csr")
    g = gpu_solve(bbs, handle, A, wl.b, solver="gmres", gmres_restart=10)
    idx = np.arange(0, 8192, 16)
    r = oracle.solve_batch(A.subset(idx), wl.b[idx], solver="gmres", restart=10)
    fails = compare(g[0][idx], g[1][idx], g[2][idx], g[3][idx], r[0], r[1], r[3], label="gmres")
    sym = W.plain_at_scale(8192, symmetric=True)
    As = sym.matrix("ell")
    g = gpu_solve(bbs, handle, As, sym.b, solver="cg")
    r = oracle.solve_batch(As.subset(idx), sym.b[idx], solver="cg")
    fails += compare(g[0][idx], g[1][idx], g[2][idx], g[3][idx], r[0], r[1], r[3], label="cg")
    assert not fails, "\n".join(fails)


# ---------------------------------------------------------- mixed mode

@pytest.mark.parametrize("given_f32", [False, True])
def test_mixed_refinement(bbs, handle, given_f32):
    """FP32 inner BiCGSTAB inside FP64 refinement: reaches the FP64 tolerance;
    its solution is within 1e-8 of the FP64 oracle's."""
    wl = W.mixed_precision(256)
    A = wl.matrix("ell")
    g = gpu_solve(bbs, handle, A, wl.b, values_f32=given_f32, precision="mixed", inner_tol=1e-4,
                  max_iters=200, max_outer=30)
    x64, it64, rel64, st64 = oracle.solve_batch(A, wl.b, max_iters=2000)
    xr, itr, relr, str_, inr = oracle.refine(A, wl.b, inner_tol=1e-4, max_inner=200)
    assert (g[3] == 0).all() and (str_ == 0).all()
    e64 = np.linalg.norm(g[0] - x64, axis=1) / np.linalg.norm(x64, axis=1)
    er = np.linalg.norm(g[0] - xr, axis=1) / np.linalg.norm(xr, axis=1)
    assert e64.max() <= 1e-8 and er.max() <= 1e-8
    assert (g[2] <= 1e-10).all()
    rh = host_rel_residual(dense_of(wl), g[0], wl.b)
    assert (rh <= 1e-10 * (1 + 1e-6)).all()
    assert np.abs(g[1].astype(int) - itr).max() <= 1
    assert (g[4] >= g[1]).all()


@pytest.mark.parametrize("fmt", ["ell", "csr"])
def test_mixed_fp32_rounding_paths_agree(bbs, handle, fmt):
    """The three ways the FP32 values reach the inner solve give the same
    bits: the caller's copy (rounded to nearest on the host), rounding while
    staging into shared memory (no copy, no workspace, one launch), and the
    library's conversion into the workspace (values not staged)."""
    wl = W.mixed_precision(96, grid=16)
    A = wl.matrix(fmt)
    kw = dict(precision="mixed", inner_tol=3e-3, max_iters=200, max_outer=30)
    given = gpu_solve(bbs, handle, A, wl.b, values_f32=True, **kw)
    fused = gpu_solve(bbs, handle, A, wl.b, **kw)
    unstaged = gpu_solve(bbs, handle, A, wl.b, values_in_smem=-1, **kw)
    for other in (fused, unstaged):
        for a, b in zip(given, other):
            assert np.array_equal(a, b)
    assert (given[3] == 0).all()
    dA = bbs.DeviceBatch.from_batch(A, "cuda")
    info = handle.describe(dA, bbs.bbs_default_options(**kw))
    assert info["kernel"] == "refine_kernel" and info["staged"] and info["launches"] == 1
    assert handle.workspace_size(dA, bbs.bbs_default_options(**kw)) == 0


# ---------------------------------------------------------- edge cases

def test_edge_cases(bbs, handle):
    wl = W.tiny_tridiagonal(16)
    A = wl.matrix("csr")
    vals = A.values.copy()
    b = wl.b.copy()
    b[3] = 0.0                      # b = 0 -> x = 0, 0 iterations
    vals[5, 7] = np.nan             # NaN in one system's matrix
    b[9, 0] = np.inf                # Inf in one system's rhs
    A2 = A.subset(np.arange(16))
    A2.values = vals
    x0 = np.full_like(b, 0.1)
    for solver in ("bicgstab", "cg", "gmres"):
        g = gpu_solve(bbs, handle, A2, b, x0, solver=solver)
        r = oracle.solve_batch(A2, b, x0, solver=solver)
        assert g[3][5] == 3 and g[3][9] == 3 and g[3][3] == 0
        assert g[1][3] == 0 and (g[0][3] == 0).all() and g[2][3] == 0.0
        keep = np.setdiff1d(np.arange(16), [5, 9])
        fails = compare(g[0][keep], g[1][keep], g[2][keep], g[3][keep], r[0][keep], r[1][keep],
                        r[3][keep], label=f"edges/{solver}")
        assert not fails, "\n".join(fails)
        # max_iters = 0: nothing moves
        g0 = gpu_solve(bbs, handle, A, wl.b, x0, solver=solver, max_iters=0)
        assert (g0[1] == 0).all() and (g0[3] == 1).all() and np.array_equal(g0[0], x0)


def test_singular_and_zero_diagonal(bbs, handle):
    n = 4
    Z = W.BatchMatrix("dense", n, n * n, 0, None, None, np.zeros((2, n * n)))
    b = np.array([[1.0, -1.0, 0.5, 2.0]] * 2)
    for solver in ("bicgstab", "cg", "gmres"):
        g = gpu_solve(bbs, handle, Z, b, solver=solver, max_iters=50)
        assert (g[3] == 2).all() and (g[1] == 1).all() and (g[0] == 0).all()
    M = np.array([[0.0, 2.0, 1.0], [1.0, 0.0, 1.0], [1.0, 3.0, 0.0]])
    Ad = W.BatchMatrix("dense", 3, 9, 0, None, None, np.stack([M.ravel()] * 3))
    b = np.array([[1.0, 2.0, 3.0]] * 3)
    for solver in ("bicgstab", "gmres"):
        g = gpu_solve(bbs, handle, Ad, b, solver=solver, tol=1e-12)
        r = oracle.solve_batch(Ad, b, solver=solver, tol=1e-12)
        assert (g[3] == r[3]).all() and np.allclose(g[0], r[0], rtol=1e-9, atol=1e-12)


def test_absolute_tolerance(bbs, handle):
    wl = W.plain_at_scale(64)
    A = wl.matrix("csr")
    g = gpu_solve(bbs, handle, A, wl.b, tol_type="absolute", tol=1e-9)
    r = oracle.solve_batch(A, wl.b, tol_type="absolute", tol=1e-9)
    fails = compare(*g[:4], r[0], r[1], r[3], tol=1e9, label="absolute")
    assert not fails, "\n".join(fails)
    res = np.linalg.norm(wl.b - np.einsum("bij,bj->bi", dense_of(wl), g[0]), axis=1)
    assert (res <= 1e-9 * (1 + 1e-6)).all()


# ------------------------------------------------------- exact invariants

def test_staging_chunking_order_and_host_path_bitwise(bbs, handle):
    """Staged or streamed values, one call or chunked calls (the collective-free
    multi-GPU split), batch order, host-buffer path: per-system results are bit
    for bit the same (each system is computed by one block with a fixed
    reduction order)."""
    wl = W.plain_at_scale(1024)
    A = wl.matrix("csr")
    base = gpu_solve(bbs, handle, A, wl.b, values_in_smem=-1)
    st = gpu_solve(bbs, handle, A, wl.b, values_in_smem=1)
    # staged values run BiCGSTAB with Jacobi folded into the matrix: the same
    # method up to rounding, so the parity bar applies rather than bit equality
    fails = compare(*st[:4], base[0], base[1], base[3], label="staged vs streamed")
    assert not fails, "\n".join(fails)
    base = st
    parts = [gpu_solve(bbs, handle, A.subset(np.arange(c, c + 256)), wl.b[c:c + 256], values_in_smem=1)
             for c in range(0, 1024, 256)]
    assert np.array_equal(np.concatenate([p[0] for p in parts]), base[0])
    perm = np.random.default_rng(5).permutation(1024)
    pr = gpu_solve(bbs, handle, A.subset(perm), wl.b[perm], values_in_smem=1)
    assert np.array_equal(pr[0], base[0][perm]) and np.array_equal(pr[1], base[1][perm])
    again = gpu_solve(bbs, handle, A, wl.b, values_in_smem=1)
    assert np.array_equal(again[0], base[0])
    # host-buffer entry point
    hA = bbs.DeviceBatch.from_batch(A, "cpu", pin=True)
    hb = torch.as_tensor(wl.b).pin_memory()
    hx = torch.zeros_like(hb).pin_memory()
    log = bbs.Log.empty(1024, device="cpu", pin=True)
    o = bbs.bbs_default_options()
    handle.solve_host(hA, hb, hx, o, log)
    dflt = gpu_solve(bbs, handle, A, wl.b)
    assert np.array_equal(hx.numpy(), dflt[0]) and np.array_equal(log.iters.numpy(), dflt[1])


def test_argument_errors(bbs, handle):
    wl = W.tiny_tridiagonal(4)
    dA = bbs.DeviceBatch.from_batch(wl.matrix("csr"), "cuda")
    b = torch.as_tensor(wl.b, device="cuda")
    x = torch.zeros_like(b)
    log = bbs.Log.empty(4)
    bad = [dict(tol=0.0), dict(max_iters=-1), dict(solver=7), dict(threads_per_system=48),
           dict(threads_per_system=1024 + 32), dict(gmres_restart=0, solver="gmres"),
           dict(precision="mixed", solver="cg"), dict(values_in_smem=2)]
    for kw in bad:
        with pytest.raises(bbs.BBSError):
            handle.solve(dA, b, x, bbs.bbs_default_options(**kw), log)
    big = bbs.DeviceBatch("csr", 4096, 4096, 0, dA.row_ptrs, dA.col_idxs, dA.values)
    with pytest.raises(bbs.BBSError):
        handle.solve(big, b, x, bbs.bbs_default_options(), log)
    empty = bbs.DeviceBatch("csr", 32, 94, 0, dA.row_ptrs, dA.col_idxs, dA.values[:0])
    handle.solve(empty, b[:0], x[:0], bbs.bbs_default_options(), log)  # no launch, OK
