"""PeleLM-shaped batches (random patterns with the n and nonzeros of the
paper's mechanisms; denser rows than the stencils) against the oracle."""

import numpy as np
import pytest
import torch

import oracle
from paper_2308_08417_gb300 import workloads as W
from tests.parity import compare

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bbs():
    from paper_2308_08417_gb300 import _build, bbs as mod

    _build.build()
    return mod


@pytest.mark.parametrize("mech", list(W.MECHANISMS))
@pytest.mark.parametrize("fmt", ["csr", "ell", "dense"])
def test_pele_like_batches(bbs, mech, fmt):
    wl = W.pele_like(mech, 2048)
    A = wl.matrix(fmt)
    dA = bbs.DeviceBatch.from_batch(A, "cuda")
    b = torch.as_tensor(wl.b, device="cuda")
    h = bbs.Handle(0)
    x, log = bbs.solve(dA, b, handle=h)
    torch.cuda.synchronize()
    idx = np.arange(0, 2048, 7)
    r = oracle.solve_batch(A.subset(idx), wl.b[idx])
    g = (x.cpu().numpy()[idx], log.iters.cpu().numpy()[idx], log.rel_res.cpu().numpy()[idx],
         log.status.cpu().numpy()[idx])
    fails = compare(*g, r[0], r[1], r[3], label=f"{mech}/{fmt}")
    assert not fails, "\n".join(fails)
