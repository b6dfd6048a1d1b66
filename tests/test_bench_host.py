"""Host-side logic of bench.py (no GPU): the traffic table is looked up by
kernel and workload shape, and never scaled onto another workload."""

import importlib.util
import os

import pytest

from paper_2308_08417_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_workload_shape_drops_only_the_batch_size(bench):
    assert bench.workload_shape("stencil2d5_12x12_B65536") == "stencil2d5_12x12"
    assert bench.workload_shape("sym_stencil2d5_12x12_B16384_cg+jacobi") == "sym_stencil2d5_12x12_cg+jacobi"
    assert bench.workload_shape("uneven_n16-1024_B100000") == "uneven_n16-1024"
    assert bench.workload_shape("stencil2d5_12x12_B65536[:16384]") == "stencil2d5_12x12"


def test_traffic_scales_by_systems_within_a_shape(bench):
    captured, systems = bench.TRAFFIC[("bicgstab_packed_kernel", "stencil2d5_12x12")]
    assert systems == 16384 and 120e6 < captured < 150e6  # about the compulsory 145 MB
    b16 = bench.traffic_bytes("bicgstab_packed_kernel", "stencil2d5_12x12_B16384", 16384)
    b64 = bench.traffic_bytes("bicgstab_packed_kernel", "stencil2d5_12x12_B65536", 65536)
    assert b16 == pytest.approx(captured) and b64 == pytest.approx(4 * b16)


def test_no_traffic_from_another_workload(bench):
    # the folded kernel was captured on the 12x12 5-point batch only: its run
    # on the 32x32 9-point batch (the mixed batch's FP64 baseline) has none
    assert bench.traffic_bytes("bicgstab_folded_kernel", "stencil2d9_32x32_B16384", 16384) is None
    assert bench.traffic_bytes("bicgstab_packed_kernel", "stencil2d9_32x32_B16384", 16384) is None


def test_every_table_entry_names_a_workload_the_bench_runs(bench):
    shapes = {
        bench.workload_shape(W.plain_at_scale(64).name),
        bench.workload_shape(W.plain_at_scale(64, symmetric=True).name + "_cg+jacobi"),
        bench.workload_shape(W.plain_at_scale(64).name + "_bicgstab+ilu0"),
        bench.workload_shape(W.plain_at_scale(64).name + "_gmres+jacobi"),
        bench.workload_shape(W.mixed_precision(8, grid=32).name),
        bench.workload_shape(W.uneven(64).name),
    }
    for kernel, shape in bench.TRAFFIC:
        assert shape in shapes, (kernel, shape)
