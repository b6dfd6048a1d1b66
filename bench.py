"""Benchmark: systems solved per second to relative residual 1e-10.

Default workload: 65,536 nonsymmetric 5-point-stencil systems on a 12x12 grid
(n = 144, nnz = 672), BatchCsr FP64, BiCGSTAB + scalar Jacobi, relative
tolerance 1e-10, max 500 iterations, x0 = 0. One step = one bbs_solve over
the whole batch (one kernel launch). Inputs (352 MB of values) exceed L2
(129 MB), so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload scale|mixed]

--impl reference times the CPU oracle (plain C, OpenMP) on a bounded sample
of the same workload, on the host cores.
Multi-GPU: one process per GPU (torchrun), each solving its own full batch
(weak scaling, no data-path collective); rank 0 prints the line.
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2308_08417_gb300 import workloads as W  # noqa: E402

METRIC = "systems solved/s to rel. residual 1e-10"

# FP64 throughput of one GB300 SM per clock (FLOP/clk/SM, FMA = 2), from the
# nominal 1.25 TFLOP/s at 2,070 MHz over 152 SMs: 1.25e12 / (152 * 2.07e9) = 3.97.
FP64_FLOP_PER_CLK_SM = 4.0
NUM_SMS = 152

# dram bytes (read + write) per launch of the dominant kernel from an ncu
# capture of this kernel (profiles/bicgstab_kernel_stencil2d5_n144.md: 280.0 MB
# for 32,768 systems, scaled by 2 to the 65,536-system launch); an entry is
# removed when its kernel changes.
TRAFFIC_BYTES = {"bicgstab_kernel": 560.0e6}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=30)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="scale", choices=["scale", "mixed"])
    p.add_argument("--systems", type=int, default=0,
                   help="solve only the first N systems of the workload (profiling runs)")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    return p.parse_args()


def workload(name):
    if name == "mixed":
        wl = W.mixed_precision()
        return wl, "ell", dict(precision="mixed", inner_tol=1e-4, max_iters=200, max_outer=30)
    wl = W.plain_at_scale()
    return wl, "csr", dict()


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        rows = [r.split(",") for r in self.out.strip().splitlines() if r.count(",") >= 8]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def cpu_oracle_run(A, b, threads, opts, budget_s=10.0):
    """Oracle on whole-batch passes until ~budget_s of CPU time; systems/s."""
    import oracle

    kw = dict(max_iters=opts.get("max_iters", 500))
    t0 = time.perf_counter()
    done = 0
    while True:
        if opts.get("precision") == "mixed":
            oracle.refine(A, b, inner_tol=opts["inner_tol"], max_inner=opts["max_iters"],
                          max_outer=opts["max_outer"], threads=threads)
        else:
            oracle.solve_batch(A, b, threads=threads, **kw)
        done += A.num_batch
        if time.perf_counter() - t0 >= budget_s:
            break
    return done / (time.perf_counter() - t0), done


def reference_arm(args, rank):
    """The CPU oracle as the reference arm (rank 0 only)."""
    if rank != 0:
        return
    import oracle

    wl, fmt, opts = workload(args.workload)
    A = wl.matrix(fmt)
    sample = 8192 if args.workload == "scale" else 512
    As, bs = A.subset(np.arange(sample)), wl.b[:sample]
    threads = oracle.num_threads()
    for _ in range(args.warmup):
        cpu_oracle_run(As, bs, threads, opts, budget_s=0.0)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        cpu_oracle_run(As, bs, threads, opts, budget_s=0.0)
    dt = time.perf_counter() - t0
    value = sample * args.steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "systems/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl.name, "sample_systems": sample},
            "cpu_baseline": {"value": value, "unit": "systems/s", "cores": threads, "kind": "oracle",
                             "sample": f"first {sample} systems of {wl.name}, one pass per step"},
            "e2e": {"value": value, "unit": "systems/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        reference_arm(args, rank)
        return

    import torch

    from paper_2308_08417_gb300 import _build, bbs

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    _build.build()

    wl, fmt, extra = workload(args.workload)
    if args.systems:
        wl = W.Workload(f"{wl.name}[:{args.systems}]", wl.pattern, wl.csr_values[:args.systems],
                        wl.b[:args.systems], wl.x0[:args.systems])
    A = wl.matrix(fmt)
    dev = torch.device("cuda", local)
    dA = bbs.DeviceBatch.from_batch(A, dev)
    b = torch.as_tensor(wl.b, device=dev)
    x0 = torch.as_tensor(wl.x0, device=dev)
    x = x0.clone()
    h = bbs.Handle(local)
    opts = bbs.bbs_default_options(**extra)
    mixed = opts.precision == 1
    log = bbs.Log.empty(wl.num_batch, device=dev, inner=mixed)
    ws = h.workspace(dA, opts)
    stream = torch.cuda.current_stream(dev)

    def step():
        x.copy_(x0)
        h.solve(dA, b, x, opts, log, ws, stream)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t_start.record(stream)
        for k in range(args.steps):
            x.copy_(x0)
            ev[k][0].record(stream)
            h.solve(dA, b, x, opts, log, ws, stream)
            ev[k][1].record(stream)
        t_end.record(stream)
        torch.cuda.synchronize()
    total_ms = t_start.elapsed_time(t_end)
    solve_ms = [a.elapsed_time(z) for a, z in ev]
    if dist is not None:
        t = torch.tensor([total_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    clocks = clk.summary()

    iters = log.iters.cpu().numpy().astype(np.int64)
    status = log.status.cpu().numpy()
    B = wl.num_batch
    value = B * world * args.steps / (total_ms / 1e3)
    avg_solve_s = statistics.mean(solve_ms) / 1e3
    if mixed:
        inner = log.inner_iters.cpu().numpy().astype(np.int64)
        flops = float(inner.sum()) * (4 * A.nnz + 26 * A.n)
        bound, unit = "alu", "TFLOP/s"
    else:
        flops = float(iters.sum()) * (4 * A.nnz + 26 * A.n)
        bound, unit = "alu", "TFLOP/s"
    mhz = clocks.get("sm_mhz") or 2070.0
    peak = FP64_FLOP_PER_CLK_SM * NUM_SMS * mhz * 1e6 / 1e12
    achieved = flops / avg_solve_s / 1e12
    kname = "refine_kernel" if mixed else "bicgstab_kernel"
    roofline = {"bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
                "frac": achieved / peak, "traffic": TRAFFIC_BYTES.get(kname),
                "kernel": kname, "peak_source": f"FP64 {FP64_FLOP_PER_CLK_SM} FLOP/clk/SM x {NUM_SMS} SMs x median SM clock {mhz:.0f} MHz"}
    hbm_bytes = 8 * (B * A.values.shape[1] + 3 * B * A.n) + 16 * B
    hbm_gbs = hbm_bytes / avg_solve_s / 1e9

    line = {"metric": METRIC, "value": value, "unit": "systems/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64+f32" if mixed else "f64", "data": "synthetic",
            "config": {"workload": wl.name, "format": fmt, "solver": "bicgstab+jacobi",
                       "num_batch_per_gpu": B, "n": A.n, "nnz": A.nnz, "tol": 1e-10,
                       "l2": "inputs larger than L2 (no flush)"},
            "gpu_launches": args.steps * (1 + (1 if ws is not None and mixed else 0)),
            "clocks": clocks, "roofline": roofline,
            "iterations": {"mean": float(iters.mean()), "max": int(iters.max()),
                           "converged": int((status == 0).sum())},
            "compulsory_hbm": {"bytes": hbm_bytes, "GB/s": hbm_gbs,
                               "frac_of_hbm": hbm_gbs / 6789.0}}

    if rank == 0 and not args.no_e2e:
        hA = bbs.DeviceBatch.from_batch(A, "cpu", pin=True)
        hb = torch.as_tensor(wl.b).pin_memory()
        hx0 = torch.as_tensor(wl.x0).pin_memory()
        hx = hx0.clone().pin_memory()
        hlog = bbs.Log.empty(B, device="cpu", pin=True, inner=mixed)
        h.solve_host(hA, hb, hx, opts, hlog)
        reps = max(2, min(args.steps, 5))
        t0 = time.perf_counter()
        for _ in range(reps):
            hx.copy_(hx0)
            h.solve_host(hA, hb, hx, opts, hlog)
        e2e_s = (time.perf_counter() - t0) / reps
        h2d = (hA.values.numel() * 8 + (hA.row_ptrs.numel() * 4 if hA.row_ptrs is not None else 0)
               + (hA.col_idxs.numel() * 4 if hA.col_idxs is not None else 0) + 2 * hb.numel() * 8)
        d2h = hx.numel() * 8 + B * (4 + 8 + 4 + (4 if mixed else 0))
        line["e2e"] = {"value": B / e2e_s, "unit": "systems/s", "h2d_bytes_per_step": h2d,
                       "d2h_bytes_per_step": d2h}
    if rank == 0 and world == 1 and not args.no_cpu:
        import oracle

        threads = oracle.num_threads()
        sample = 8192 if args.workload == "scale" else 256
        As, bs = A.subset(np.arange(sample)), wl.b[:sample]
        v, done = cpu_oracle_run(As, bs, threads, extra, budget_s=10.0)
        line["cpu_baseline"] = {"value": v, "unit": "systems/s", "cores": threads, "kind": "oracle",
                                "sample": f"first {sample} systems of {wl.name}, repeated to "
                                          f"{done} solves (~10 s)"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
