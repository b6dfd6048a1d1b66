"""The C-ABI library loads and exports every symbol include/bbs.h declares;
host-only logic (no GPU compute) behaves as specified."""

import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2308_08417_gb300 import _build, bbs

    _build.build()
    return bbs.lib()


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "bbs.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(bbs_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(L):
    names = declared_symbols()
    assert "bbs_solve" in names and "bbs_create" in names
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, f"not exported: {missing}"


def test_paper_block_size_rule():
    """Sec. 3.6: at least n, a multiple of the sub-group (warp) size, at most the
    device maximum; rows divisible by 32 use n itself."""
    from paper_2308_08417_gb300 import bbs

    for n in range(1, 3000):
        w = bbs.bbs_paper_block_size(n, 1024)
        assert w % 32 == 0 and w <= 1024
        if n <= 1024:
            assert w >= n and w - n < 32
        else:
            assert w == 1024
        if n % 32 == 0 and n <= 1024:
            assert w == n
    assert bbs.bbs_paper_block_size(0, 1024) == 0
    assert bbs.bbs_paper_block_size(100, 16) == 0


def test_default_block_size_respects_register_tiers():
    from paper_2308_08417_gb300 import bbs

    for n in range(1, 2049):
        t = bbs.bbs_default_block_size(n, 5)
        assert t % 32 == 0 and 32 <= t <= 1024
        R = -(-n // t)
        assert R <= 8
        assert t <= (1024 if R <= 1 else 512 if R <= 4 else 256)
    assert bbs.bbs_default_block_size(144, 5) == 32
    assert bbs.bbs_default_block_size(2049, 5) == 0


def test_default_options_and_version(L):
    from paper_2308_08417_gb300 import bbs

    o = bbs.bbs_default_options()
    assert (o.solver, o.precond, o.tol_type, o.max_iters, o.gmres_restart) == (0, 1, 1, 500, 10)
    assert o.tol == 1e-10 and o.inner_tol == 1e-4 and o.max_outer == 30
    assert "sm_103a" in bbs.bbs_version()


def test_struct_layouts_match_header():
    import ctypes as C

    from paper_2308_08417_gb300 import bbs

    assert C.sizeof(bbs.bbs_options) == 56
    assert bbs.bbs_options.tol.offset == 16 and bbs.bbs_options.inner_tol.offset == 32
    assert C.sizeof(bbs.bbs_batch_matrix) == 24 + 4 * 8
    assert C.sizeof(bbs.bbs_log) == 32
    assert C.sizeof(bbs.bbs_launch_info) == 40 and bbs.bbs_launch_info.smem_bytes.offset == 24
