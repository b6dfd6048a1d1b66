"""bbs_solve_noalloc against bbs_solve, through the C ABI, on the GPU.

bbs_solve_noalloc is for callers that cannot allocate device memory: a host
whose device memory another allocator already holds (a framework's caching
pool, a server's arena), or a loop that must not wait on cudaMalloc/cudaFree.
It takes its scratch from a static array inside the library instead of a
caller workspace, and solves a batch whose scratch is larger than that array
in consecutive chunks. Its results must be bit for bit those of bbs_solve
with a workspace, on two calls in a row (the second reuses the array with the
first call's contents in it), and a call must leave the device's free memory
unchanged. This file is collected last on purpose.
"""

import numpy as np
import pytest
import torch

from paper_2308_08417_gb300 import workloads as W

pytestmark = pytest.mark.gpu

SCRATCH = 64 << 20  # the library's static scratch


@pytest.fixture(scope="module")
def bbs():
    from paper_2308_08417_gb300 import _build, bbs as mod

    _build.build()
    return mod


def _outputs(bbs, dA, b, opts):
    x = torch.zeros_like(b)
    log = bbs.Log.empty(dA.num_batch, device=b.device, inner=(opts.precision == 1))
    return x, log


def _host(x, log):
    return (x.cpu().numpy(), log.iters.cpu().numpy(), log.status.cpu().numpy(), log.rel_res.cpu().numpy())


def _check_noalloc(bbs, dA, b, opts, expect_ws):
    handle = bbs.Handle(0)
    ws_bytes = handle.workspace_size(dA, opts)
    # the case must need more scratch than the array holds, so the chunked path runs
    assert ws_bytes == expect_ws and ws_bytes > SCRATCH
    x, log = _outputs(bbs, dA, b, opts)
    handle.solve(dA, b, x, opts, log, handle.workspace(dA, opts))
    torch.cuda.synchronize()
    ref = _host(x, log)
    outs = [_outputs(bbs, dA, b, opts) for _ in range(2)]
    free = []
    for xo, lo in outs:  # two calls in a row, outputs allocated beforehand
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
        handle.solve_noalloc(dA, b, xo, opts, lo)
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
    # the first call may load the library's scratch module; the second allocates nothing
    assert free[2] == free[3]
    for xo, lo in outs:
        got = _host(xo, lo)
        for g, r in zip(got, ref):
            assert np.array_equal(g, r)
    assert (ref[2] == 0).all() and (ref[3] <= 1e-10).all()


def test_noalloc_mixed_fp32_copy_in_scratch(bbs):
    """Mixed precision with unstaged values: the FP32 copy of 2,200 systems
    (81 MB) goes through the 64 MiB scratch in two chunks."""
    B = 2200
    wl = W.mixed_precision(B)
    dA = bbs.DeviceBatch.from_batch(wl.matrix("ell"), "cuda")
    b = torch.as_tensor(wl.b, device="cuda")
    opts = bbs.bbs_default_options(precision="mixed", inner_tol=1e-4, max_iters=200, max_outer=30,
                                   values_in_smem=-1)
    vps = dA.ell_k * dA.n
    _check_noalloc(bbs, dA, b, opts, expect_ws=(vps * 4 * B + 255) // 256 * 256)


def test_noalloc_gmres_basis_in_scratch(bbs):
    """GMRES(20) at n = 2048: the Krylov basis (344 KB per system) does not fit
    in shared memory; 200 systems (69 MB) go through the scratch in two chunks."""
    B, n, m = 200, 2048, 20
    pat = W.stencil_pattern("1d3", n)
    rng = np.random.default_rng(3)
    vals = W.stencil_values(pat, B, rng, 0.05, 0.5)
    b_np = rng.uniform(-1, 1, (B, n))
    dA = bbs.DeviceBatch.from_batch(W.make_batch(pat, vals, "csr"), "cuda")
    b = torch.as_tensor(b_np, device="cuda")
    opts = bbs.bbs_default_options(solver="gmres", gmres_restart=m, max_iters=3000)
    _check_noalloc(bbs, dA, b, opts, expect_ws=(m + 1) * n * 8 * B)
