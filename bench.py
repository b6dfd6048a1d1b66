"""Benchmark: systems solved per second to relative residual 1e-10.

Headline workload (default, --workload scale): 65,536 nonsymmetric
5-point-stencil systems on a 12x12 grid (n = 144, nnz = 672), BatchCsr FP64,
BiCGSTAB + scalar Jacobi, relative tolerance 1e-10, max 500 iterations,
x0 = 0. One step = one bbs_solve over the whole batch (one kernel launch).
Its inputs (352 MB of values) exceed L2 (129 MB), so no flush is needed.

Other workloads (--workload): mixed (16,384 9-point systems, n = 1024, ELL;
FP32-inner / FP64-outer refinement against plain FP64 BiCGSTAB) and uneven
(100,000 systems, n log-uniform in [16, 1024], one persistent graph launch
with autotuned team sizes). The default line carries short measurements of
these under "extras".

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload scale|mixed|uneven|learned|pele|sweep|peaks|mlp_predict]
                  [--systems N] [--shard] [--no-extras]

--impl reference times the CPU oracle (plain C, OpenMP) on a bounded sample
of the same workload, on the host cores.
Multi-GPU: one process per GPU (torchrun), each solving its own full batch
(weak scaling, no data-path collective); rank 0 prints the line. With
--shard the ranks split one batch instead (strong scaling): rank r solves a
contiguous range of systems (balanced by estimated cost for the uneven
batch), and rank 0 gathers the iteration counts and statuses on the host.

The default line ends with "speedups": the mixed-precision and learned-guess
forms against plain FP64 on the same GPU (the metric's second half).
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
from paper_2308_08417_gb300.sharding import max_over_ranks  # noqa: E402

METRIC = "systems solved/s to rel. residual 1e-10"

# FP64 throughput of one GB300 SM per clock (FLOP/clk/SM, FMA = 2), from the
# nominal 1.25 TFLOP/s at 2,070 MHz over 152 SMs: 1.25e12 / (152 * 2.07e9) = 3.97.
FP64_FLOP_PER_CLK_SM = 4.0
# FP32 (non-tensor) FMA lanes: 128 per SM per clock = 256 FLOP/clk/SM.
FP32_FLOP_PER_CLK_SM = 256.0
NUM_SMS = 152
HBM_GBS = 6789.0  # measured copy bandwidth of the GB300s

# dram bytes (read + write) of one launch of a kernel from an ncu capture of
# it, with the number of systems that launch solved, keyed by kernel and
# workload shape (the workload label without its batch size); the bench
# scales them to its own launch of the same shape by systems (traffic is the
# compulsory bytes, which grow in proportion). A kernel run on a workload
# without a capture reports null, and an entry is removed when its kernel
# changes. The uneven batch's entries are captures of its first 20,000
# systems (the persistent launch alone, and the graph of persistent, packed
# and wide launches: the sum over its launches); per-system bytes vary with n,
# so their scaling is approximate.
TRAFFIC = {("bicgstab_packed_kernel", "stencil2d5_12x12"): (135.11e6, 16384),
           ("bicgstab_folded_kernel", "stencil2d5_12x12"): (280.72e6, 32768),
           ("cg_packed_kernel", "sym_stencil2d5_12x12_cg+jacobi"): (133.00e6, 16384),
           ("gmres_packed_kernel", "stencil2d5_12x12_gmres+jacobi"): (147.83e6, 16384),
           ("bicgstab_ilu_packed_kernel", "stencil2d5_12x12_bicgstab+ilu0"): (134.60e6, 16384),
           ("refine_kernel", "stencil2d9_32x32"): (396.44e6, 4096),
           ("varsize_kernel", "uneven_n16-1024"): (333.05e6, 20000),
           ("varsize_kernel+varpacked_kernel", "uneven_n16-1024"): (336.46e6, 20000),
           ("varsize_kernel+varpacked_kernel+varwide_kernel", "uneven_n16-1024"): (332.21e6, 20000)}


# mixed refinement of the 32x32 9-point batch: the inner FP32 tolerance from a
# sweep on GB300 (3e-2: 1.13 M systems/s, 1e-2: 1.29 M, 5e-3: 1.18 M,
# 3e-3: 1.33 M, 1e-3: 1.17 M, 1e-4: 1.17 M); both arms use it
MIXED_OPTS = dict(precision="mixed", inner_tol=3e-3, max_iters=200, max_outer=30)


def workload_shape(label):
    """A workload label without its batch size (`_B<count>`, and the `[:k]` of
    a --systems subset)."""
    import re

    return re.sub(r"_B[0-9]+|\[:[0-9]+\]", "", label)


def traffic_bytes(kernel, label, systems):
    key = (kernel, workload_shape(label))
    if key not in TRAFFIC:
        return None
    b, s = TRAFFIC[key]
    return b / s * systems


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=30)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="scale",
                   choices=["scale", "mixed", "uneven", "learned", "pele", "sweep", "peaks", "mlp_predict"])
    p.add_argument("--format", default="csr", choices=["csr", "ell", "dense"],
                   help="batch format of the scale workload")
    p.add_argument("--solver", default="bicgstab", choices=["bicgstab", "cg", "gmres"],
                   help="solver of the scale workload (cg runs on its symmetrised copy)")
    p.add_argument("--precond", default="jacobi", choices=["jacobi", "none", "ilu0"],
                   help="preconditioner of the scale workload")
    p.add_argument("--threads-per-system", type=int, default=0,
                   help="launch shape of the scale and mixed workloads (0: the library's choice)")
    p.add_argument("--systems", type=int, default=0,
                   help="solve only the first N systems of the workload (profiling runs)")
    p.add_argument("--inner-tol", type=float, default=0.0,
                   help="mixed workload: inner FP32 tolerance (0: the tuned default)")
    p.add_argument("--shard", action="store_true",
                   help="ranks split one batch (strong scaling) instead of each solving a full batch")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-extras", action="store_true")
    p.add_argument("--no-tune", action="store_true", help="uneven workload: default launch choices")
    p.add_argument("--tuning", default="", help="uneven workload: launch choices as JSON (an earlier line's "
                   "iterations.tuning), instead of tuning")
    return p.parse_args()


# --------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.out = ""

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


# ------------------------------------------------------------ workloads

def subset_workload(wl, k):
    if not k:
        return wl
    return W.Workload(f"{wl.name}[:{k}]", wl.pattern, wl.csr_values[:k], wl.b[:k], wl.x0[:k])


def span_workload(wl, span):
    """Systems [begin, end) of a workload, under the whole workload's name (a
    rank's share of a sharded batch)."""
    if span is None:
        return wl
    b0, b1 = span
    return W.Workload(wl.name, wl.pattern, wl.csr_values[b0:b1], wl.b[b0:b1], wl.x0[b0:b1])


def uneven_cost(vb):
    """Per-system cost estimate of an uneven batch, (2 nnz + 14 n) sqrt(n):
    the work of one iteration times an iteration count growing like sqrt(n)."""
    n = vb.sys_n().astype(np.float64)
    return (2 * vb.sys_nnz() + 14 * n) * np.sqrt(n)


def shard_span(workload, systems, rank, world):
    """This rank's [begin, end) of the batch the workload names."""
    from paper_2308_08417_gb300.sharding import cost_shard_range, shard_range

    if workload == "uneven":
        return cost_shard_range(uneven_cost(W.uneven(systems or 100000)), rank, world)
    total = {"mixed": 16384, "scale": 65536}[workload]
    return shard_range(min(systems, total) if systems else total, rank, world)


class Uniform:
    """bbs_solve over a shared-pattern batch (one launch per step)."""

    def __init__(self, bbs, torch, dev, wl, fmt, opts_kw, label, values_f32=False):
        self.bbs, self.torch, self.dev = bbs, torch, dev
        self.wl, self.fmt, self.label = wl, fmt, label
        self.A = wl.matrix(fmt)
        self.dA = bbs.DeviceBatch.from_batch(self.A, dev, values_f32=values_f32)
        self.b = torch.as_tensor(wl.b, device=dev)
        self.x0 = torch.as_tensor(wl.x0, device=dev)
        self.x = self.x0.clone()
        self.h = bbs.Handle(dev.index or 0)
        self.opts = bbs.bbs_default_options(**opts_kw)
        self.mixed = self.opts.precision == 1
        self.log = bbs.Log.empty(wl.num_batch, device=dev, inner=self.mixed)
        self.ws = self.h.workspace(self.dA, self.opts)
        self.num_batch = wl.num_batch
        # the library's own account of the launch (kernel, shape, launches per solve)
        self.launch = self.h.describe(self.dA, self.opts)
        self.kernel = self.launch["kernel"]
        self.launches_per_step = self.launch["launches"]

    def reset(self):
        self.x.copy_(self.x0)

    def step(self, stream):
        self.h.solve(self.dA, self.b, self.x, self.opts, self.log, self.ws, stream)

    def work(self):
        """(algorithmic FLOPs of the last solve, arithmetic) per launch. Per
        iteration: BiCGSTAB 4 nnz + 26 n; with ILU(0) two triangular solves
        more, 2 (2 (nnz - n) + n); CG 2 nnz + 10 n; GMRES(m) per Arnoldi step j
        2 nnz + (4 j + 7) n, taken at the cycle's mean j = (m - 1) / 2."""
        A, o = self.A, self.opts
        nnz = A.nnz if A.fmt == "csr" else int(np.count_nonzero(A.values[0]))
        if o.solver == 1:
            per_it = 2 * nnz + 10 * A.n
        elif o.solver == 2:
            per_it = 2 * nnz + (4 * (o.gmres_restart - 1) / 2 + 7) * A.n
        else:
            per_it = 4 * nnz + 26 * A.n
            if o.precond == 2:
                per_it += 2 * (2 * (nnz - A.n) + A.n)
        if self.mixed:
            inner = self.log.inner_iters.cpu().numpy().astype(np.int64)
            return float(inner.sum()) * per_it, "fp32"
        it = self.log.iters.cpu().numpy().astype(np.int64)
        return float(it.sum()) * per_it, "fp64"

    def compulsory_bytes(self):
        B, A = self.num_batch, self.A
        return 8 * (B * A.values.shape[1] + 3 * B * A.n) + 16 * B

    def streamed_bytes(self):
        """The matrix values re-read by every SpMV (two per iteration, plus the
        initial and confirming residuals) as if nothing stayed on chip, plus
        the compulsory vector bytes: the HBM traffic of an unstaged design."""
        it = self.log.iters.cpu().numpy().astype(np.int64)
        spmvs = 2 * it.sum() + 2 * self.num_batch
        return 8 * self.A.values.shape[1] * int(spmvs) + 8 * 3 * self.num_batch * self.A.n + 16 * self.num_batch

    def summary(self):
        it = self.log.iters.cpu().numpy()
        st = self.log.status.cpu().numpy()
        out = {"mean": float(it.mean()), "max": int(it.max()), "converged": int((st == 0).sum())}
        if self.mixed:
            out["inner_mean"] = float(self.log.inner_iters.cpu().numpy().mean())
        return out

    def e2e(self, reps):
        bbs, torch = self.bbs, self.torch
        with host_memory_near(torch, self.dev) as near:
            hA = bbs.DeviceBatch.from_batch(self.A, "cpu", pin=True)
            hb = torch.as_tensor(self.wl.b).pin_memory()
            hx0 = torch.as_tensor(self.wl.x0)
            # x is in/out: every call gets its own pinned copy of x0, made
            # before the timed region (restoring one buffer on the host would
            # time a host memcpy of the whole x that is not part of the call)
            hxs = [hx0.clone().pin_memory() for _ in range(reps + 1)]
            hlog = bbs.Log.empty(self.num_batch, device="cpu", pin=True, inner=self.mixed)
        hx = hxs[0]
        self.h.solve_host(hA, hb, hxs[reps], self.opts, hlog)
        per = []
        for i in range(reps):  # each call returns once its results are back on the host
            t0 = time.perf_counter()
            self.h.solve_host(hA, hb, hxs[i], self.opts, hlog)
            per.append(time.perf_counter() - t0)
        h2d = (hA.values.numel() * 8 + (hA.row_ptrs.numel() * 4 if hA.row_ptrs is not None else 0)
               + (hA.col_idxs.numel() * 4 if hA.col_idxs is not None else 0) + 2 * hb.numel() * 8)
        d2h = hx.numel() * 8 + self.num_batch * (4 + 8 + 4 + (4 if self.mixed else 0))
        # the median call: a call now and then runs much slower on a shared host
        # (host copies, not the device), which the mean would carry
        return {"value": self.num_batch / statistics.median(per), "unit": "systems/s",
                "mean_value": self.num_batch * reps / sum(per), "per_call_ms": [round(1e3 * t, 3) for t in per],
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "path": "bbs_solve_host (host buffers)",
                "host_numa_node": near.node}

    def cpu(self, threads, budget_s):
        import oracle

        k = min(8192 if not self.mixed else 256, self.num_batch)
        As, bs = self.A.subset(np.arange(k)), self.wl.b[:k]
        t0 = time.perf_counter()
        done = 0
        while True:
            if self.mixed:
                oracle.refine(As, bs, inner_tol=self.opts.inner_tol, max_inner=self.opts.max_iters,
                              max_outer=self.opts.max_outer, threads=threads)
            else:
                oracle.solve_batch(As, bs, max_iters=self.opts.max_iters, threads=threads)
            done += As.num_batch
            if time.perf_counter() - t0 >= budget_s:
                break
        return (done / (time.perf_counter() - t0),
                f"first {As.num_batch} systems of {self.wl.name}, repeated to {done} solves")


class Uneven:
    """One graph launch of the persistent uneven-batch plan per step."""

    def __init__(self, bbs, torch, dev, vb, tune=True, tuning=None):
        self.bbs, self.torch, self.dev, self.vb = bbs, torch, dev, vb
        self.label = vb.name
        self.vbd = bbs.VarDeviceBatch.from_varbatch(vb, dev)
        self.b = torch.as_tensor(vb.b, device=dev)
        self.x0 = torch.as_tensor(vb.x0, device=dev)
        self.x = self.x0.clone()
        self.h = bbs.Handle(dev.index or 0)
        self.opts = bbs.bbs_default_options()
        t0 = time.perf_counter()
        if tuning is not None:  # a pinned tuning (the dict of an earlier run's line)
            self.tuning = bbs.bbs_var_tuning.from_dict(tuning)
        else:
            self.tuning = (bbs.bbs_var_tune(self.h, self.vbd, self.b, self.x0, self.opts, sample=512)
                           if tune else None)
        self.tune_s = time.perf_counter() - t0
        self.plan = bbs.VarPlan(self.h, self.vbd, self.opts, self.tuning)
        self.desc = self.plan.describe()
        self.log = bbs.Log.empty(vb.num_batch, device=dev)
        self.num_batch = vb.num_batch
        # one graph: the persistent team launch (with its counter reset), one
        # launch per packed class of small systems and per wide-team class
        d = self.desc
        persistent = 1 if d["persistent_grid"] else 0
        self.kernel = "+".join(k for k, c in (("varsize_kernel", persistent), ("varpacked_kernel", d["packed_launches"]),
                                              ("varwide_kernel", d["wide_launches"])) if c)
        self.launches_per_step = persistent + d["packed_launches"] + d["wide_launches"]
        self.mixed = False

    def reset(self):
        self.x.copy_(self.x0)

    def step(self, stream):
        self.plan.solve(self.b, self.x, self.log, stream)

    def work(self):
        it = self.log.iters.cpu().numpy().astype(np.int64)
        per_it = 4 * self.vb.sys_nnz().astype(np.int64) + 26 * self.vb.sys_n().astype(np.int64)
        return float((it * per_it).sum()), "fp64"

    def compulsory_bytes(self):
        return 8 * (self.vb.values.size + 3 * self.vb.b.size) + 16 * self.num_batch

    def summary(self):
        it = self.log.iters.cpu().numpy()
        st = self.log.status.cpu().numpy()
        return {"mean": float(it.mean()), "max": int(it.max()), "converged": int((st == 0).sum()),
                "tuning": self.tuning.as_dict() if self.tuning is not None else "default",
                "tune_s": self.tune_s, "plan": self.desc}

    def e2e(self, reps):
        torch = self.torch
        hb = torch.as_tensor(self.vb.b).pin_memory()
        hv = torch.as_tensor(self.vb.values).pin_memory()
        hx0 = torch.as_tensor(self.vb.x0).pin_memory()
        hx = hx0.clone().pin_memory()
        hit = torch.empty(self.num_batch, dtype=torch.int32).pin_memory()
        vals = self.vbd.tensors["values"]
        stream = torch.cuda.current_stream(self.dev)
        t0 = time.perf_counter()
        for _ in range(reps):
            vals.copy_(hv, non_blocking=True)
            self.b.copy_(hb, non_blocking=True)
            self.x.copy_(hx0, non_blocking=True)
            self.plan.solve(self.b, self.x, self.log, stream)
            hx.copy_(self.x, non_blocking=True)
            hit.copy_(self.log.iters, non_blocking=True)
            torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / reps
        return {"value": self.num_batch / dt, "unit": "systems/s",
                "h2d_bytes_per_step": hv.numel() * 8 + 2 * hb.numel() * 8,
                "d2h_bytes_per_step": hx.numel() * 8 + self.num_batch * 4,
                "path": "host copies + bbs_var_solve (graph launch)"}

    def cpu(self, threads, budget_s):
        import oracle

        sel = np.arange(0, self.num_batch, 10)
        t0 = time.perf_counter()
        done = 0
        while True:
            oracle.solve_varsize(self.vb, systems=sel, threads=threads)
            done += len(sel)
            if time.perf_counter() - t0 >= budget_s:
                break
        return (done / (time.perf_counter() - t0),
                f"every 10th system of {self.vb.name}, repeated to {done} solves")


def make_runner(name, bbs, torch, dev, systems=0, tune=True, fmt="csr", tps=0, solver="bicgstab",
                precond="jacobi", span=None, inner_tol=0.0, tuning=None):
    if name == "mixed":
        wl = span_workload(subset_workload(W.mixed_precision(), systems), span)
        kw = dict(MIXED_OPTS)
        if inner_tol:
            kw["inner_tol"] = inner_tol
        if tps:
            kw["threads_per_system"] = tps
        return Uniform(bbs, torch, dev, wl, "ell", kw, wl.name)
    if name == "mixed_fp64":
        wl = subset_workload(W.mixed_precision(), systems)
        return Uniform(bbs, torch, dev, wl, "ell", dict(max_iters=2000), wl.name)
    if name == "uneven":
        vb = W.uneven(systems or 100000)
        if span is not None:
            vb = vb.slice(*span)
            vb.name = vb.name.split("[")[0]
        return Uneven(bbs, torch, dev, vb, tune=tune, tuning=tuning)
    wl = span_workload(subset_workload(W.plain_at_scale(symmetric=(solver == "cg")), systems), span)
    opts = {"threads_per_system": tps} if tps else {}
    opts.update(solver=solver, precond=precond)
    label = wl.name if fmt == "csr" else f"{wl.name}_{fmt}"
    if (solver, precond) != ("bicgstab", "jacobi"):
        label = f"{label}_{solver}+{precond}"
    return Uniform(bbs, torch, dev, wl, fmt, opts, label)


def gpu_numa_cpus(torch, dev):
    """(NUMA node, its CPUs) of the GPU's host memory, from sysfs; (None,
    None) when the machine does not say."""
    try:
        p = torch.cuda.get_device_properties(dev)
        bdf = f"{p.pci_domain_id:04x}:{p.pci_bus_id:02x}:{p.pci_device_id:02x}.0"
        with open(f"/sys/bus/pci/devices/{bdf}/numa_node") as f:
            node = int(f.read())
        if node < 0:
            return None, None
        cpus = set()
        with open(f"/sys/devices/system/node/node{node}/cpulist") as f:
            for part in f.read().strip().split(","):
                a, _, b = part.partition("-")
                cpus.update(range(int(a), int(b or a) + 1))
        return node, (cpus & os.sched_getaffinity(0)) or None
    except (OSError, ValueError, AttributeError, RuntimeError):
        return None, None


class host_memory_near:
    """Run the block on the CPUs of the GPU's NUMA node (when known), so that
    pinned buffers made there are first touched in memory next to the GPU."""

    def __init__(self, torch, dev):
        self.node, self.cpus = gpu_numa_cpus(torch, dev)

    def __enter__(self):
        self.saved = os.sched_getaffinity(0)
        if self.cpus:
            os.sched_setaffinity(0, self.cpus)
        return self

    def __exit__(self, *exc):
        os.sched_setaffinity(0, self.saved)
        return False


def timed_solve(bbs, torch, h, dA, b, opts, reps=3):
    """Best-of-reps CUDA-event time (ms) of one bbs_solve from x0 = 0, and the log."""
    x = torch.zeros_like(b)
    log = bbs.Log.empty(dA.num_batch, device=b.device)
    ws = h.workspace(dA, opts)
    h.solve(dA, b, x, opts, log, ws)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    best = float("inf")
    for _ in range(reps):
        x.zero_()
        e0.record()
        h.solve(dA, b, x, opts, log, ws)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    st = log.status.cpu().numpy()
    return best, float(log.iters.double().mean()), int((st == 0).sum())


def pele_runs(bbs, torch, dev, num_batch=131072):
    """The five PeleLM-shaped batches (BatchCsr, BiCGSTAB + scalar Jacobi, the
    paper's Sec. 5.2 setup), each unique matrix repeated on the device."""
    h = bbs.Handle(dev.index or 0)
    out = {}
    for mech, (U, n, nnz) in W.MECHANISMS.items():
        wl = W.pele_like(mech, U)  # the unique matrices
        uniq = torch.as_tensor(wl.csr_values, device=dev)
        idx = torch.arange(num_batch, device=dev) % U
        vals = uniq[idx].contiguous()
        g = np.random.Generator(np.random.PCG64(W.SEED_BASE + 11))
        b = torch.as_tensor(g.uniform(-1, 1, (num_batch, n)), device=dev)
        res = {}
        for fmt in ("csr", "dense"):
            if fmt == "csr":
                kmax = int(np.diff(wl.pattern.row_ptrs).max())  # the CSR row-length bound
                dA = bbs.DeviceBatch("csr", n, nnz, kmax, torch.as_tensor(wl.pattern.row_ptrs, device=dev),
                                     torch.as_tensor(wl.pattern.col_idxs, device=dev), vals)
            else:
                dense = torch.zeros(num_batch, n * n, dtype=torch.float64, device=dev)
                rows = np.repeat(np.arange(n), np.diff(wl.pattern.row_ptrs))
                pos = torch.as_tensor(rows * n + wl.pattern.col_idxs, device=dev)
                dense[:, pos] = vals
                dA = bbs.DeviceBatch("dense", n, nnz, 0, None, None, dense)
            opts = bbs.bbs_default_options()
            ms, it, conv = timed_solve(bbs, torch, h, dA, b, opts)
            per_it = 4 * (nnz if fmt == "csr" else n * n) + 26 * n
            res[fmt] = {"ms": ms, "systems_per_s": num_batch / (ms / 1e3), "iters_mean": it,
                        "converged": conv, "launch": h.describe(dA, opts),
                        "fp64_tflops": num_batch * it * (4 * nnz + 26 * n) / (ms / 1e3) / 1e12,
                        "executed_tflops": num_batch * it * per_it / (ms / 1e3) / 1e12}
            del dA
        out[mech] = {"n": n, "nnz": nnz, "unique": U, "num_batch": num_batch, **res}
        del vals, uniq
        torch.cuda.empty_cache()
    return out


def sweep_runs(bbs, torch, dev):
    """Scaling study of Sec. 5.1 on the 3-point SPD batch: matrix size at 2^17
    systems and batch count at n = 64, for CG and BiCGSTAB (+ Jacobi)."""
    h = bbs.Handle(dev.index or 0)
    out = {"size": [], "batch": []}
    for n in (16, 32, 64, 128, 256, 512, 1024):
        wl = W.spd_tridiagonal(131072, n)
        dA = bbs.DeviceBatch.from_batch(wl.matrix("csr"), dev)
        b = torch.as_tensor(wl.b, device=dev)
        for solver in ("cg", "bicgstab"):
            ms, it, conv = timed_solve(bbs, torch, h, dA, b, bbs.bbs_default_options(solver=solver))
            out["size"].append({"n": n, "solver": solver, "ms": ms, "iters_mean": it, "converged": conv,
                                "systems_per_s": 131072 / (ms / 1e3)})
        del dA, b, wl
    wl = W.spd_tridiagonal(131072, 64)
    for lb in range(13, 18):
        B = 2 ** lb
        A = wl.matrix("csr").subset(np.arange(B))
        dA = bbs.DeviceBatch.from_batch(A, dev)
        b = torch.as_tensor(wl.b[:B], device=dev)
        for solver in ("cg", "bicgstab"):
            ms, it, conv = timed_solve(bbs, torch, h, dA, b, bbs.bbs_default_options(solver=solver))
            out["batch"].append({"num_batch": B, "solver": solver, "ms": ms, "iters_mean": it,
                                 "converged": conv, "systems_per_s": B / (ms / 1e3)})
    return out


def learned_run(bbs, torch, dev, eval_steps=192, num_batch=16384):
    """Time-stepped batch: train on steps 0..63, then per step time (MLP
    prediction + solve) against (solve from x(t-1))."""
    from paper_2308_08417_gb300.learned import TimeStepped

    ts = W.time_stepped(num_batch=num_batch, steps=64 + eval_steps)
    run = TimeStepped(ts, device=str(dev), hidden=256, seed=0)
    rep = run.run(train_steps=64, eval_steps=eval_steps, epochs=6, batch=4096)
    s = rep.summary()
    s["workload"] = f"timestepped_stencil2d5_12x12_B{num_batch}_T{64 + eval_steps}"
    return s


def mlp_predict_run(bbs, torch, dev, stream, args, num_batch=16384, n=144, hidden=256):
    """bbs_mlp_predict alone: the learned guess's network over one step of the
    time-stepped batch (a network of the bench's shape, its initial weights;
    the work does not depend on their values)."""
    ts = W.time_stepped(num_batch=num_batch, steps=3)
    A = bbs.DeviceBatch.from_batch(W.make_batch(ts.pattern, ts.values_at(2), "csr"), dev)
    b = torch.as_tensor(ts.rhs_at(2), device=dev)
    xp = torch.as_tensor(np.random.default_rng(1).uniform(-1, 1, (num_batch, n)), device=dev)
    net = bbs.MLP(bbs.Handle(dev.index or 0), n, hidden=hidden, seed=1, max_batch=num_batch)
    x0 = torch.empty_like(xp)
    for _ in range(max(args.warmup, 3)):
        net.predict(A, b, xp, x0)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    torch.cuda.nvtx.range_push("bbs.timed")
    with ClockSampler(dev.index or 0) as clk:
        for e0, e1 in ev:
            e0.record(stream)
            net.predict(A, b, xp, x0)
            e1.record(stream)
        torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    net.check()
    ms = [a.elapsed_time(z) for a, z in ev]
    flop = 2.0 * num_batch * (3 * n * hidden + 2 * hidden * hidden + hidden * n)
    achieved = flop / (statistics.mean(ms) / 1e3) / 1e12
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peak, src = float(json.load(f)["bf16_tflops"]), "MEASURED_PEAKS.json bf16_tflops (burst)"
    except (OSError, KeyError, ValueError):
        peak, src = 1900.0, "profiling recipe fallback (1.9 PFLOP/s bf16 burst)"
    return {"metric": "bbs_mlp_predict time per step", "value": statistics.mean(ms), "unit": "ms",
            "higher_is_better": False, "steps": args.steps, "warmup": args.warmup, "dtype": "bf16+f32",
            "data": "synthetic", "config": {"workload": f"timestepped_stencil2d5_12x12_B{num_batch}_predict",
                                            "network": f"{3 * n}-{hidden}-{hidden}-{hidden}-{n}"},
            "gpu_launches": args.steps, "clocks": clk.summary(),
            "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": None, "kernel": "mlp_infer_kernel",
                         "peak_source": src, "flop_per_launch": flop}}


def time_steps(r, torch, stream, steps, warmup, dist=None, sample_clocks=False, dev_index=0):
    for _ in range(max(warmup, 3)):
        r.reset()
        r.step(stream)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(dev_index) if sample_clocks else None
    if clk:
        clk.__enter__()
    nvtx = torch.cuda.nvtx
    nvtx.range_push("bbs.timed")  # NVTX ranges for timeline tools
    t0.record(stream)
    for k in range(steps):
        nvtx.range_push("bbs.step")
        r.reset()
        ev[k][0].record(stream)
        r.step(stream)
        ev[k][1].record(stream)
        nvtx.range_pop()
    t1.record(stream)
    torch.cuda.synchronize()
    nvtx.range_pop()
    if dist is not None:
        dist.barrier()
    if clk:
        clk.__exit__()
    total_ms = t0.elapsed_time(t1)
    solve_ms = [a.elapsed_time(z) for a, z in ev]
    return total_ms, solve_ms, (clk.summary() if clk else None)


def measured_peaks(bbs, h):
    """FP64 and FP32 FMA rates of this GPU in TFLOP/s (bbs_fma_rate: 8 FMA
    chains per thread, 8 blocks of 256 threads per SM, CUDA events)."""
    try:
        return {"fp64": bbs.bbs_fma_rate(h, "fp64") / 1e12, "fp32": bbs.bbs_fma_rate(h, "fp32") / 1e12,
                "source": "bbs_fma_rate in this run (8 independent FMA chains per thread, "
                          "8 x 256 threads per SM, one ~20 ms launch timed with CUDA events)"}
    except Exception as e:  # report, do not hide
        return {"error": repr(e)}


def roofline(r, solve_ms, mhz, peaks=None):
    flops, arith = r.work()
    avg_s = statistics.mean(solve_ms) / 1e3
    per_clk = FP64_FLOP_PER_CLK_SM if arith == "fp64" else FP32_FLOP_PER_CLK_SM
    peak = per_clk * NUM_SMS * mhz * 1e6 / 1e12
    achieved = flops / avg_s / 1e12
    out = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
           "frac": achieved / peak, "traffic": traffic_bytes(r.kernel, r.label, r.num_batch), "kernel": r.kernel,
           "arith": arith,
           "peak_source": f"nominal: {arith.upper()} {per_clk:g} FLOP/clk/SM x {NUM_SMS} SMs x median SM clock "
                          f"{mhz:.0f} MHz"}
    if peaks and arith in peaks:
        out["measured_peak"] = peaks[arith]
        out["frac_measured_peak"] = achieved / peaks[arith]
        out["measured_peak_source"] = peaks["source"]
    return out


def extras(bbs, torch, dev, stream, mhz, peaks=None):
    """Short measurements of the other forms on the same GPU."""
    out = {}
    try:
        f64 = make_runner("mixed_fp64", bbs, torch, dev)
        tot64, ms64, _ = time_steps(f64, torch, stream, 3, 1)
        mix = make_runner("mixed", bbs, torch, dev)
        tot, ms, _ = time_steps(mix, torch, stream, 5, 2)
        v64 = f64.num_batch * 3 / (tot64 / 1e3)
        vm = mix.num_batch * 5 / (tot / 1e3)
        x64 = f64.x.cpu().numpy()
        xm = mix.x.cpu().numpy()
        err = float((np.linalg.norm(xm - x64, axis=1) / np.linalg.norm(x64, axis=1)).max())
        out["mixed"] = {"workload": mix.label, "value": vm, "fp64_value": v64, "unit": "systems/s",
                        "speedup_vs_fp64": vm / v64, "max_rel_diff_vs_fp64": err,
                        "iterations": mix.summary(), "fp64_iterations": f64.summary(),
                        "roofline": roofline(mix, ms, mhz, peaks), "fp64_roofline": roofline(f64, ms64, mhz, peaks)}
        del f64, mix
        torch.cuda.empty_cache()
        # the same solve with the caller's FP32 copy of the values: the
        # difference is the cost of rounding the values while staging them
        wl = W.mixed_precision()
        given = Uniform(bbs, torch, dev, wl, "ell",
                        dict(MIXED_OPTS), wl.name,
                        values_f32=True)
        totg, _, _ = time_steps(given, torch, stream, 5, 2)
        vg = given.num_batch * 5 / (totg / 1e3)
        out["mixed"]["value_with_f32_copy_given"] = vg
        out["mixed"]["rounding_ms_per_step"] = (tot - totg) / 5
        del given
    except Exception as e:  # report, do not hide
        out["mixed"] = {"error": repr(e)}
    try:  # the same headline batch with one system per warp (no packing)
        wl = W.plain_at_scale()
        ow = Uniform(bbs, torch, dev, wl, "csr", dict(threads_per_system=32), wl.name)
        tot, ms, _ = time_steps(ow, torch, stream, 5, 2)
        out["one_system_per_warp"] = {"workload": ow.wl.name, "value": ow.num_batch * 5 / (tot / 1e3),
                                      "unit": "systems/s", "launch": ow.launch, "iterations": ow.summary(),
                                      "roofline": roofline(ow, ms, mhz, peaks)}
        del ow
    except Exception as e:
        out["one_system_per_warp"] = {"error": repr(e)}
    for solver in ("cg", "gmres"):  # the other Krylov solvers on the headline shape
        try:
            wl = W.plain_at_scale(symmetric=(solver == "cg"))
            kr = Uniform(bbs, torch, dev, wl, "csr", dict(solver=solver), f"{wl.name}_{solver}+jacobi")
            tot, ms, _ = time_steps(kr, torch, stream, 5, 2)
            out[solver] = {"workload": kr.label, "value": kr.num_batch * 5 / (tot / 1e3), "unit": "systems/s",
                           "launch": kr.launch, "iterations": kr.summary(), "roofline": roofline(kr, ms, mhz, peaks)}
            del kr
        except Exception as e:
            out[solver] = {"error": repr(e)}
    try:  # the same headline batch with the batched ILU(0) preconditioner
        wl = W.plain_at_scale()
        il = Uniform(bbs, torch, dev, wl, "csr", dict(precond="ilu0"), f"{wl.name}_bicgstab+ilu0")
        tot, ms, _ = time_steps(il, torch, stream, 5, 2)
        out["ilu0"] = {"workload": il.label, "value": il.num_batch * 5 / (tot / 1e3),
                       "unit": "systems/s", "iterations": il.summary(), "launch": il.launch,
                       "roofline": roofline(il, ms, mhz, peaks),
                       "note": "BiCGSTAB + ILU(0) (level-scheduled factorisation and triangular solves)"}
        del il
    except Exception as e:
        out["ilu0"] = {"error": repr(e)}
    try:
        out["learned"] = learned_run(bbs, torch, dev, eval_steps=192)
    except Exception as e:
        out["learned"] = {"error": repr(e)}
    try:
        un = make_runner("uneven", bbs, torch, dev)
        tot, ms, _ = time_steps(un, torch, stream, 5, 2)
        out["uneven"] = {"workload": un.label, "value": un.num_batch * 5 / (tot / 1e3),
                         "unit": "systems/s", "iterations": un.summary(),
                         "roofline": roofline(un, ms, mhz, peaks),
                         "launches_per_step": f"1 graph ({un.launches_per_step} kernels)"}
        del un
    except Exception as e:
        out["uneven"] = {"error": repr(e)}
    return out


# ---------------------------------------------------------- reference arm

def reference_arm(args, rank):
    """The CPU oracle as the reference arm (rank 0 only)."""
    if rank != 0:
        return
    import oracle

    threads = oracle.num_threads()
    if args.workload == "uneven":
        vb = W.uneven(args.systems or 100000)
        sel = np.arange(0, vb.num_batch, 10)
        run = lambda: oracle.solve_varsize(vb, systems=sel, threads=threads)  # noqa: E731
        sample, name = len(sel), vb.name
    else:
        if args.workload == "mixed":
            wl, fmt, k = W.mixed_precision(), "ell", 512
        else:
            wl, fmt, k = W.plain_at_scale(), "csr", 8192
        A = wl.matrix(fmt)
        As, bs = A.subset(np.arange(k)), wl.b[:k]
        if args.workload == "mixed":
            run = lambda: oracle.refine(As, bs, inner_tol=MIXED_OPTS["inner_tol"],  # noqa: E731
                                        max_inner=MIXED_OPTS["max_iters"], max_outer=MIXED_OPTS["max_outer"],
                                        threads=threads)
        else:
            run = lambda: oracle.solve_batch(As, bs, threads=threads)  # noqa: E731
        sample, name = k, wl.name
    for _ in range(args.warmup):
        run()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        run()
    dt = time.perf_counter() - t0
    value = sample * args.steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "systems/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": name, "sample_systems": sample},
            "cpu_baseline": {"value": value, "unit": "systems/s", "cores": threads, "kind": "oracle",
                             "sample": f"{sample} systems of {name}, one pass per step"},
            "e2e": {"value": value, "unit": "systems/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ main

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
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)

    if args.workload == "peaks":
        h = bbs.Handle(local)
        with ClockSampler(local) as clk:
            pk = measured_peaks(bbs, h)
        if rank == 0:
            print(json.dumps({"workload": "peaks", "unit": "TFLOP/s", **pk, "clocks": clk.summary(),
                              "nominal_fp64": FP64_FLOP_PER_CLK_SM * NUM_SMS * 2.07e9 / 1e12,
                              "nominal_fp32": FP32_FLOP_PER_CLK_SM * NUM_SMS * 2.07e9 / 1e12}), flush=True)
        return
    if args.workload == "mlp_predict":
        line = mlp_predict_run(bbs, torch, dev, stream, args)
        if rank == 0:
            print(json.dumps(line), flush=True)
        return
    if args.workload in ("pele", "sweep"):
        res = pele_runs(bbs, torch, dev) if args.workload == "pele" else sweep_runs(bbs, torch, dev)
        if rank == 0:
            print(json.dumps({"metric": METRIC, "workload": args.workload, "unit": "systems/s",
                              "n_gpus": world, "dtype": "f64", "data": "synthetic", "results": res}),
                  flush=True)
        return
    if args.workload == "learned":
        s = learned_run(bbs, torch, dev, eval_steps=192, num_batch=args.systems or 16384)
        line = {"metric": METRIC, "value": s["systems_per_s_learned"], "unit": "systems/s",
                "n_gpus": world, "steps": s["eval_steps"], "warmup": 64,
                "ms_per_step": 1e3 * s["num_batch"] / s["systems_per_s_learned"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64+bf16",
                "data": "synthetic", "config": {"workload": s["workload"], "train_steps": 64},
                "gpu_launches": None, "learned": s}
        if rank == 0:
            print(json.dumps(line), flush=True)
        return
    span = shard_span(args.workload, args.systems, rank, world) if args.shard else None
    r = make_runner(args.workload, bbs, torch, dev, args.systems, tune=not args.no_tune, fmt=args.format,
                    tps=args.threads_per_system, solver=args.solver, precond=args.precond, span=span,
                    inner_tol=args.inner_tol, tuning=json.loads(args.tuning) if args.tuning else None)
    total_ms, solve_ms, clocks = time_steps(r, torch, stream, args.steps, args.warmup, dist,
                                            sample_clocks=True, dev_index=local)
    total_ms = max_over_ranks(total_ms, dist, dev)  # the job's time is its slowest rank's
    mhz = clocks.get("sm_mhz") or 2070.0
    if args.shard:  # one batch split over the ranks
        job_systems = int(r.num_batch)
        if dist is not None:
            t = torch.tensor([job_systems], dtype=torch.int64, device=dev)
            dist.all_reduce(t)
            job_systems = int(t.item())
    else:  # every rank solves its own full batch
        job_systems = r.num_batch * world
    value = job_systems * args.steps / (total_ms / 1e3)
    avg_solve_s = statistics.mean(solve_ms) / 1e3
    hbm_bytes = r.compulsory_bytes()
    line = {"metric": METRIC, "value": value, "unit": "systems/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "strong" if args.shard else "weak", "vs_baseline": None,
            "dtype": "f64+f32" if r.mixed else "f64", "data": "synthetic",
            "config": {"workload": r.label, "num_batch_per_gpu": r.num_batch, "tol": 1e-10,
                       "solver": f"{args.solver}+{args.precond}" if args.workload == "scale" else "bicgstab+jacobi",
                       "l2": "inputs larger than L2 (no flush)"},
            "gpu_launches": args.steps * r.launches_per_step,
            "launch": getattr(r, "launch", None),
            "clocks": clocks, "roofline": None,
            "iterations": r.summary(),
            "compulsory_hbm": {"bytes": hbm_bytes, "GB/s": hbm_bytes / avg_solve_s / 1e9,
                               "frac_of_hbm": hbm_bytes / avg_solve_s / 1e9 / HBM_GBS}}
    if args.shard:
        line["config"]["shard"] = {"span": list(span), "job_systems": job_systems,
                                   "split": "cost-balanced contiguous ranges" if args.workload == "uneven"
                                   else "contiguous ranges"}
        line["gathered"] = gather_logs(r, torch, dist, dev)
    if hasattr(r, "streamed_bytes"):
        sb = r.streamed_bytes()
        line["streamed_matrix_hbm"] = {"bytes": sb, "GB/s": sb / avg_solve_s / 1e9,
                                       "frac_of_hbm": sb / avg_solve_s / 1e9 / HBM_GBS,
                                       "note": "values re-read by every SpMV, as an unstaged design would"}
    if rank == 0 and not args.no_e2e and not args.shard:
        line["e2e"] = r.e2e(max(3, min(args.steps, 7)))
    if rank == 0 and world == 1 and not args.no_cpu:
        import oracle

        threads = oracle.num_threads()
        v, sample = r.cpu(threads, 10.0)
        v1, sample1 = r.cpu(1, 3.0)
        line["cpu_baseline"] = {"value": v, "unit": "systems/s", "cores": threads, "kind": "oracle",
                                "sample": sample + " (~10 s)",
                                "one_thread": {"value": v1, "sample": sample1 + " (~3 s)"}}
    # the FMA-rate probe runs after the host-buffer timing: its seconds of
    # full-occupancy FMA chains would otherwise change the clocks that timing sees
    peaks = measured_peaks(bbs, r.h)
    line["roofline"] = roofline(r, solve_ms, mhz, peaks)
    if rank == 0 and world == 1 and args.workload == "scale" and not args.no_extras and not args.systems:
        del r
        torch.cuda.empty_cache()
        ex = extras(bbs, torch, dev, stream, mhz, peaks)
        line["extras"] = ex
        line["speedups"] = speedups(ex, value)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def gather_logs(r, torch, dist, dev):
    """Host-side collection of a sharded run's per-system outcome (after the
    timed region): every rank's iteration counts and statuses, concatenated in
    rank order on rank 0."""
    its = r.log.iters.cpu().numpy()
    st = r.log.status.cpu().numpy()
    parts = [(its, st)]
    if dist is not None:
        parts = [None] * dist.get_world_size()
        dist.all_gather_object(parts, (its, st))
    it = np.concatenate([p[0] for p in parts])
    sa = np.concatenate([p[1] for p in parts])
    return {"systems": int(it.size), "converged": int((sa == 0).sum()), "iters_mean": float(it.mean()),
            "collective": "host-side gather of the logs after the timed region"}


def speedups(ex, plain_value):
    """The metric's second half, compact: each form against plain FP64 BiCGSTAB
    on the same GPU (ratios of systems/s at rel. residual 1e-10)."""
    out = {"plain_fp64_systems_per_s": round(plain_value)}
    m = ex.get("mixed", {})
    if "speedup_vs_fp64" in m:
        out["mixed_vs_fp64"] = round(m["speedup_vs_fp64"], 3)
        out["mixed"] = {"systems_per_s": round(m["value"]), "fp64_systems_per_s": round(m["fp64_value"]),
                        "workload": m["workload"], "max_rel_diff_vs_fp64": m["max_rel_diff_vs_fp64"]}
    lr = ex.get("learned", {})
    if "speedup" in lr:
        out["learned_vs_prev_x"] = round(lr["speedup"], 3)
        out["learned_vs_zero"] = round(lr["speedup_vs_zero_guess"], 3)
        out["learned"] = {"workload": lr["workload"], "eval_steps": lr["eval_steps"],
                          "iters": [round(lr["iters_learned"], 2), round(lr["iters_base"], 2),
                                    round(lr["iters_zero_guess"], 2)],
                          "iters_order": "learned, x(t-1), zero"}
    return out


if __name__ == "__main__":
    main()
