"""bbs_check_pattern: the device check of a shared pattern. Only the checker
runs on the broken patterns below; no solver ever sees them."""

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


def csr_batch(bbs, rp, ci, n, nnz, k=0):
    vals = torch.ones(2, max(nnz, 1), dtype=torch.float64, device="cuda")
    return bbs.DeviceBatch("csr", n, nnz, k, torch.as_tensor(rp, dtype=torch.int32, device="cuda"),
                           torch.as_tensor(ci, dtype=torch.int32, device="cuda"), vals)


def test_valid_patterns_pass(bbs):
    h = bbs.Handle(0)
    for wl in (W.plain_at_scale(4), W.mixed_precision(2, grid=8), W.pele_like("gri12", 4)):
        for fmt in ("csr", "ell", "dense"):
            dA = bbs.DeviceBatch.from_batch(wl.matrix(fmt), "cuda")
            assert h.check_pattern(dA) == 0, (wl.name, fmt)


def test_broken_csr_patterns_are_counted(bbs):
    h = bbs.Handle(0)
    pat = W.stencil_pattern("1d3", 8)  # rows 0 and 7 have 2 entries, the others 3
    rp, ci, nnz = pat.row_ptrs.copy(), pat.col_idxs.copy(), pat.nnz
    assert h.check_pattern(csr_batch(bbs, rp, ci, 8, nnz, k=3)) == 0
    bad = ci.copy()
    bad[4] = 8                                  # column out of range (row 1)
    assert h.check_pattern(csr_batch(bbs, rp, bad, 8, nnz)) == 1
    bad = ci.copy()
    bad[[3, 4]] = bad[[4, 3]]                   # unsorted row 1
    assert h.check_pattern(csr_batch(bbs, rp, bad, 8, nnz)) == 1
    bad = ci.copy()
    bad[2] = -3                                 # negative column (row 1)
    assert h.check_pattern(csr_batch(bbs, rp, bad, 8, nnz)) == 1
    brp = rp.copy()
    brp[3] = brp[2] - 1                         # decreasing row pointers: rows 2 and 3
    assert h.check_pattern(csr_batch(bbs, brp, ci, 8, nnz)) == 2
    brp = rp.copy()
    brp[8] = nnz + 5                            # past the end of col_idxs (row 7)
    assert h.check_pattern(csr_batch(bbs, brp, ci, 8, nnz)) >= 1
    assert h.check_pattern(csr_batch(bbs, rp, ci, 8, nnz, k=2)) == 6  # 6 rows longer than 2


def test_broken_ell_patterns_are_counted(bbs):
    h = bbs.Handle(0)
    A = W.plain_at_scale(2, grid=4).matrix("ell")  # 16 rows, k = 5
    good = bbs.DeviceBatch.from_batch(A, "cuda")
    assert h.check_pattern(good) == 0
    ci = A.col_idxs.copy().reshape(5, 16)
    row0 = ci[:, 0].copy()                      # corner row: 3 entries then 2 pads
    assert (row0[3:] == -1).all()
    ci[:, 0] = [row0[0], -1, row0[1], row0[2], -1]   # a pad before stored entries
    ci[:, 5] = ci[::-1, 5]                      # unsorted interior row
    ci[2, 9] = 16                               # column out of range
    bad = bbs.DeviceBatch("ell", 16, A.nnz, 5, None, torch.as_tensor(ci.ravel(), device="cuda"), good.values)
    assert h.check_pattern(bad) == 3
