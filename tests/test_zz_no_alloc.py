"""bbs_solve_noalloc against bbs_solve, through the C ABI, on the GPU.

bbs_solve_noalloc serves callers that cannot allocate device memory (stream
capture, allocator-free loops, hosts with their own memory pools): it takes
its scratch from a static array inside the library instead of a workspace.
Its results must be those of bbs_solve with a caller workspace. Two calls in
a row are checked, so a second call that reuses the shared array (holding the
first call's contents) is covered. This file is collected last on purpose.
"""

import numpy as np
import pytest
import torch

from paper_2308_08417_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bbs():
    from paper_2308_08417_gb300 import _build, bbs as mod

    _build.build()
    return mod


def _run(bbs, handle, dA, b, opts, noalloc):
    x = torch.zeros_like(b)
    log = bbs.Log.empty(dA.num_batch, device=b.device, inner=(opts.precision == 1))
    if noalloc:
        handle.solve_noalloc(dA, b, x, opts, log)
    else:
        handle.solve(dA, b, x, opts, log, handle.workspace(dA, opts))
    torch.cuda.synchronize()
    return x.cpu().numpy(), log.iters.cpu().numpy(), log.status.cpu().numpy(), log.rel_res.cpu().numpy()


@pytest.mark.parametrize("num_batch", [300, 2200])  # 2200 systems need two chunks of 64 MiB
def test_noalloc_matches_workspace_solve(bbs, num_batch):
    wl = W.mixed_precision(num_batch)
    dA = bbs.DeviceBatch.from_batch(wl.matrix("ell"), "cuda")
    b = torch.as_tensor(wl.b, device="cuda")
    opts = bbs.bbs_default_options(precision="mixed", inner_tol=1e-4, max_iters=200, max_outer=30)
    handle = bbs.Handle(0)
    ref = _run(bbs, handle, dA, b, opts, noalloc=False)
    for _ in range(2):
        got = _run(bbs, handle, dA, b, opts, noalloc=True)
        err = np.linalg.norm(got[0] - ref[0], axis=1) / np.linalg.norm(ref[0], axis=1)
        assert err.max() <= 1e-8
        assert np.abs(got[1].astype(int) - ref[1]).max() <= 2
        assert np.array_equal(got[2], ref[2]) and (got[2] == 0).all()
        assert (got[3] <= 1e-10).all()


def test_noalloc_gmres_basis_in_scratch(bbs):
    """GMRES with a basis too large for shared memory keeps it in the scratch."""
    pat = W.stencil_pattern("1d3", 2048)
    rng = np.random.default_rng(3)
    vals = W.stencil_values(pat, 64, rng, 0.05, 0.5)
    b_np = rng.uniform(-1, 1, (64, 2048))
    dA = bbs.DeviceBatch.from_batch(W.make_batch(pat, vals, "csr"), "cuda")
    b = torch.as_tensor(b_np, device="cuda")
    opts = bbs.bbs_default_options(solver="gmres", gmres_restart=20, max_iters=3000)
    handle = bbs.Handle(0)
    assert handle.workspace_size(dA, opts) > 0
    ref = _run(bbs, handle, dA, b, opts, noalloc=False)
    for _ in range(2):
        got = _run(bbs, handle, dA, b, opts, noalloc=True)
        err = np.linalg.norm(got[0] - ref[0], axis=1) / np.linalg.norm(ref[0], axis=1)
        assert err.max() <= 1e-8 and np.array_equal(got[2], ref[2])
