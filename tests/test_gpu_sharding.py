"""The collective-free multi-GPU split on one GPU: the slices a sharded run
gives its ranks (sharding.shard_range for uniform batches, cost_shard_range
for uneven ones), solved one after another through libbbs.so, reassemble bit
for bit into the result of one call over the whole batch. The ranks of a
real run solve the same slices on their own GPUs with no exchange."""

import numpy as np
import pytest
import torch

from paper_2308_08417_gb300 import workloads as W
from paper_2308_08417_gb300.sharding import cost_shard_range, shard_range

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bbs():
    from paper_2308_08417_gb300 import _build, bbs as mod

    _build.build()
    return mod


def _uniform(bbs, h, wl, fmt, opts, span):
    b0, b1 = span
    A = wl.matrix(fmt).subset(np.arange(b0, b1))
    dA = bbs.DeviceBatch.from_batch(A, "cuda")
    b = torch.as_tensor(wl.b[b0:b1], device="cuda")
    x = torch.zeros_like(b)
    log = bbs.Log.empty(b1 - b0, inner=(opts.precision == 1))
    h.solve(dA, b, x, opts, log, h.workspace(dA, opts))
    torch.cuda.synchronize()
    return x.cpu().numpy(), log.iters.cpu().numpy(), log.status.cpu().numpy(), log.rel_res.cpu().numpy()


@pytest.mark.parametrize("case", ["plain_csr", "mixed_ell"])
@pytest.mark.parametrize("world", [2, 3])
def test_uniform_shards_reassemble_bitwise(bbs, case, world):
    h = bbs.Handle(0)
    if case == "plain_csr":
        wl, fmt, opts = W.plain_at_scale(6001), "csr", bbs.bbs_default_options()
    else:
        wl, fmt = W.mixed_precision(601), "ell"
        opts = bbs.bbs_default_options(precision="mixed", inner_tol=3e-3, max_iters=200, max_outer=30)
    whole = _uniform(bbs, h, wl, fmt, opts, (0, wl.num_batch))
    parts = [_uniform(bbs, h, wl, fmt, opts, shard_range(wl.num_batch, r, world)) for r in range(world)]
    for k in range(4):
        assert np.array_equal(np.concatenate([p[k] for p in parts]), whole[k])
    assert (whole[2] == 0).all()


def test_uneven_cost_shards_reassemble_bitwise(bbs):
    h = bbs.Handle(0)
    vb = W.uneven(4000)
    n = vb.sys_n().astype(np.float64)
    cost = (2 * vb.sys_nnz() + 14 * n) * np.sqrt(n)
    opts = bbs.bbs_default_options()
    tuning = bbs.bbs_var_default_tuning(int(vb.sys_n().max()))

    def solve(v):
        vbd = bbs.VarDeviceBatch.from_varbatch(v)
        plan = bbs.VarPlan(h, vbd, opts, tuning)
        b = torch.as_tensor(v.b, device="cuda")
        x = torch.as_tensor(v.x0, device="cuda").clone()
        log = bbs.Log.empty(v.num_batch)
        plan.solve(b, x, log)
        torch.cuda.synchronize()
        return x.cpu().numpy(), log.iters.cpu().numpy(), log.status.cpu().numpy(), log.rel_res.cpu().numpy()

    whole = solve(vb)
    parts = [solve(vb.slice(*cost_shard_range(cost, r, 3))) for r in range(3)]
    for k in range(4):
        assert np.array_equal(np.concatenate([p[k] for p in parts]), whole[k])
    assert (whole[2] == 0).all()
