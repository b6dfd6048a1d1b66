"""BiCGSTAB with the batched ILU(0) preconditioner against the CPU oracle."""

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


def run(bbs, A, b, hint=True, **kw):
    dA = bbs.DeviceBatch.from_batch(A, "cuda")
    if not hint:  # no CSR row-length bound: one system per warp
        dA = bbs.DeviceBatch(dA.fmt, dA.n, dA.nnz, 0, dA.row_ptrs, dA.col_idxs, dA.values)
    bt = torch.as_tensor(b, device="cuda")
    x, log = bbs.solve(dA, bt, handle=bbs.Handle(0), precond="ilu0", **kw)
    torch.cuda.synchronize()
    return x.cpu().numpy(), log.iters.cpu().numpy(), log.rel_res.cpu().numpy(), log.status.cpu().numpy()


@pytest.mark.parametrize("tps", [0, 4, 8, 16, 32])
def test_ilu_exact_on_tridiagonal(bbs, tps):
    """No fill-in exists for a tridiagonal pattern: ILU(0) is the exact LU and
    BiCGSTAB finishes in one iteration with the solution (packed or not)."""
    wl = W.tiny_tridiagonal(64)
    x, it, rel, st = run(bbs, wl.matrix("csr"), wl.b, tol=1e-12, threads_per_system=tps)
    D = W.to_dense(wl.pattern, wl.csr_values).reshape(-1, 32, 32)
    xs = np.linalg.solve(D, wl.b[..., None])[..., 0]
    assert (it == 1).all() and (st == 0).all()
    assert (np.linalg.norm(x - xs, axis=1) / np.linalg.norm(xs, axis=1)).max() < 1e-12


@pytest.mark.parametrize("hint,tps", [(True, 0), (True, 8), (True, 16), (False, 0)])
def test_ilu_packed_and_unpacked_match_oracle(bbs, hint, tps):
    """65 systems (the last warp partly empty) of the 12x12 stencil: packed
    2 or 4 systems per warp, and one system per warp without the CSR bound."""
    wl = W.plain_at_scale(65)
    A = wl.matrix("csr")
    if tps == 8:  # 144 rows would need 18 rows per lane on 8 lanes: use an 8x8 grid
        wl = W.plain_at_scale(65, grid=8)
        A = wl.matrix("csr")
    g = run(bbs, A, wl.b, hint=hint, threads_per_system=tps)
    r = oracle.solve_batch(A, wl.b, precond="ilu0")
    fails = compare(*g, r[0], r[1], r[3], label=f"ilu hint={hint} tps={tps}")
    assert not fails, "\n".join(fails)
    if hint and tps == 0:
        h = bbs.Handle(0)
        info = h.describe(bbs.DeviceBatch.from_batch(A, "cuda"), bbs.bbs_default_options(precond="ilu0"))
        assert info["kernel"] == "bicgstab_ilu_packed_kernel" and info["launches"] == 3


@pytest.mark.parametrize("name", ["stencil", "stencil9", "drm19", "gri12", "gri30", "dodecane_lu",
                                  "isooctane"])
def test_ilu_matches_oracle(bbs, name):
    if name == "stencil":
        wl = W.plain_at_scale(4096)
    elif name == "stencil9":
        wl = W.mixed_precision(256, grid=16)
    else:
        wl = W.pele_like(name, 1024)
    A = wl.matrix("csr")
    g = run(bbs, A, wl.b)
    idx = np.arange(0, wl.num_batch, 5)
    r = oracle.solve_batch(A.subset(idx), wl.b[idx], precond="ilu0")
    fails = compare(g[0][idx], g[1][idx], g[2][idx], g[3][idx], r[0], r[1], r[3], label=f"ilu/{name}")
    assert not fails, "\n".join(fails)


def test_ilu_rejects_unsupported_combinations(bbs):
    wl = W.tiny_tridiagonal(4)
    b = torch.as_tensor(wl.b, device="cuda")
    h = bbs.Handle(0)
    for fmt, kw in (("ell", {}), ("csr", dict(solver="cg")), ("csr", dict(solver="gmres")),
                    ("csr", dict(precision="mixed"))):
        dA = bbs.DeviceBatch.from_batch(wl.matrix(fmt), "cuda")
        with pytest.raises(bbs.BBSError):
            bbs.solve(dA, b, handle=h, precond="ilu0", **kw)
