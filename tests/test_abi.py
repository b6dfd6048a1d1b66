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


def test_struct_layouts_match_the_c_compiler(tmp_path):
    """Every struct the binding mirrors has the size and field offsets that a
    C compiler gives the header's declaration."""
    import ctypes as C
    import shutil
    import subprocess

    from paper_2308_08417_gb300 import bbs

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = [bbs.bbs_options, bbs.bbs_batch_matrix, bbs.bbs_log, bbs.bbs_launch_info, bbs.bbs_var_batch,
               bbs.bbs_var_host_info, bbs.bbs_var_tuning, bbs.bbs_var_plan_desc]
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "bbs.h"', "int main(void) {"]
    for st in structs:
        lines.append(f'    printf("{st.__name__} size %zu\\n", sizeof({st.__name__}));')
        for f, _ in st._fields_:
            lines.append(f'    printf("{st.__name__} {f} %zu\\n", offsetof({st.__name__}, {f}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l}
    for st in structs:
        assert got[(st.__name__, "size")] == C.sizeof(st), st.__name__
        for f, _ in st._fields_:
            assert got[(st.__name__, f)] == getattr(st, f).offset, f"{st.__name__}.{f}"


def test_host_chunk_plan():
    """bbs_solve_host's chunks: in order, the batch covered once, at least
    2,048 systems each but the last, led by a quarter and a half chunk, about
    128 MB of input per full chunk and never more than 8 of them."""
    from paper_2308_08417_gb300 import bbs

    for B in (1, 7, 2047, 2048, 4096, 20001, 65536, 100001, 1 << 20):
        for per in (0, 8, 8848, 90112, 1 << 20):
            plan = bbs.bbs_host_chunk_plan(B, per)
            assert plan and plan[0][0] == 0
            assert all(a + n == b for (a, n), (b, _) in zip(plan, plan[1:]))
            assert plan[-1][0] + plan[-1][1] == B
            assert all(n >= min(2048, B) for _, n in plan[:-1]) and plan[-1][1] >= 1
            full = max(n for _, n in plan)
            assert sum(1 for _, n in plan if n == full) <= 8 and len(plan) <= 10
            if len(plan) >= 4:  # plan[2] is a full chunk: the ramp leads it
                c = plan[2][1]
                assert plan[0][1] == max(2048, c // 4) and plan[1][1] == max(2048, c // 2)
    # the headline batch: 65,536 systems of 672 values, b and x0 (7,680 bytes,
    # 503 MB) in chunks of 4,096, 8,192, then 16,384 systems
    assert [n for _, n in bbs.bbs_host_chunk_plan(65536, 672 * 8 + 2 * 144 * 8)] == [4096, 8192, 16384, 16384,
                                                                                     16384, 4096]
    assert bbs.bbs_host_chunk_plan(0, 100) == []
    assert bbs.bbs_host_chunk_plan(-1, 100) is None
    assert bbs.bbs_host_chunk_plan(65536, 8848, max_chunks=3) is None
