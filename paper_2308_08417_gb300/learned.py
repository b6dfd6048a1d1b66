"""Time-stepped batches with a learned initial guess (orchestration only).

A_i(t) = A_i + 0.01 t B_i and b_i(t) = b_i + 0.01 t c_i (workloads.TimeSeries)
are solved step after step; each step's solve starts from an initial guess.
The baseline guess is the previous solution x(t-1). The learned guess is
x(t-1) plus gamma times the change an MLP predicts from (diag A(t), b(t),
x(t-1)); the network is trained on the changes the solver produced in the
first steps, and the gate gamma in [0, 1] is the least-squares scale of its
prediction on the last training steps, which the network does not train on.

Every step of the method runs in libbbs.so: the solves (bbs_solve), the
input statistics (bbs_mlp_observe / bbs_mlp_finalize_stats), the training
samples (bbs_mlp_make_samples), the forward/backward passes and Adam
(bbs_mlp_train_step), the gate (bbs_mlp_gate_observe / bbs_mlp_gate_finalize)
and the prediction (bbs_mlp_predict). This module only builds each step's
inputs (an elementwise A + 0.01 t B on the device), sequences the calls and
tallies the report.
"""

from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import bbs as B
from . import workloads as W


@dataclass
class StepRecord:
    t: int
    iters_base: float
    iters_learned: float
    ms_base: float
    ms_learned: float
    res0_base: float = 0.0
    res0_learned: float = 0.0
    converged: int = 0
    iters_zero: float = 0.0
    ms_zero: float = 0.0
    ms_predict: float = 0.0


@dataclass
class LearnedReport:
    train_steps: int
    eval_steps: int
    num_batch: int
    train_s: float
    collect_s: float
    losses: list = field(default_factory=list)
    records: list = field(default_factory=list)
    gate: float = 1.0
    gate_steps: int = 0
    gate_err_learned: float = 0.0
    gate_err_base: float = 0.0

    def summary(self) -> dict:
        r = self.records
        base_ms = sum(x.ms_base for x in r)
        learn_ms = sum(x.ms_learned for x in r)
        n = self.num_batch * len(r)
        return {
            "eval_steps": len(r), "num_batch": self.num_batch,
            "iters_base": float(np.mean([x.iters_base for x in r])),
            "iters_learned": float(np.mean([x.iters_learned for x in r])),
            "systems_per_s_base": n / (base_ms / 1e3),
            "systems_per_s_learned": n / (learn_ms / 1e3),
            "speedup": base_ms / learn_ms,
            "iters_zero_guess": float(np.mean([x.iters_zero for x in r])),
            "systems_per_s_zero_guess": n / (sum(x.ms_zero for x in r) / 1e3),
            "speedup_vs_zero_guess": sum(x.ms_zero for x in r) / learn_ms,
            "init_residual_base": float(np.mean([x.res0_base for x in r])),
            "init_residual_learned": float(np.mean([x.res0_learned for x in r])),
            "train_s": self.train_s, "collect_s": self.collect_s,
            "final_loss": self.losses[-1] if self.losses else None,
            "first_loss": self.losses[0] if self.losses else None,
            "predict_ms_per_step": float(np.mean([x.ms_predict for x in r])),
            "solve_ms_per_step_base": base_ms / len(r),
            "gate": self.gate, "gate_steps": self.gate_steps,
            "gate_steps_error_ratio": (self.gate_err_learned / self.gate_err_base
                                       if self.gate_err_base > 0 else None),
        }


class TimeStepped:
    def __init__(self, ts: W.TimeSeries, device="cuda", hidden=256, seed=0, max_batch=None):
        self.ts = ts
        self.dev = torch.device(device)
        self.h = B.Handle(self.dev.index or 0)
        pat = ts.pattern
        self.n, self.nnz = pat.n, pat.nnz
        self.rp = torch.as_tensor(pat.row_ptrs, dtype=torch.int32, device=self.dev)
        self.ci = torch.as_tensor(pat.col_idxs, dtype=torch.int32, device=self.dev)
        self.A0 = torch.as_tensor(ts.A, device=self.dev)
        self.Bn = torch.as_tensor(ts.Bn, device=self.dev)
        self.b0 = torch.as_tensor(ts.b, device=self.dev)
        self.c = torch.as_tensor(ts.c, device=self.dev)
        self.vals = torch.empty_like(self.A0)
        self.rhs = torch.empty_like(self.b0)
        self.opts = B.bbs_default_options()
        self.log = B.Log.empty(ts.num_batch, device=self.dev)
        # rows the network handles per launch: the whole batch by default, so a
        # prediction is one pass of four GEMMs over every system
        if max_batch is None:
            max_batch = max(4096, (ts.num_batch + 63) // 64 * 64)
        self.mlp = B.MLP(self.h, self.n, hidden=hidden, seed=seed, max_batch=max_batch)
        self.max_batch = max_batch

    # inputs of step t (input construction, not the method)
    def set_step(self, t: int):
        torch.add(self.A0, self.Bn, alpha=0.01 * t, out=self.vals)
        torch.add(self.b0, self.c, alpha=0.01 * t, out=self.rhs)

    def matrix(self):
        return B.DeviceBatch("csr", self.n, self.nnz, 0, self.rp, self.ci, self.vals)

    def solve(self, x):
        self.h.solve(self.matrix(), self.rhs, x, self.opts, self.log)

    def init_residual(self, x):
        """Mean relative residual of a guess, through a zero-iteration solve."""
        o = B.bbs_default_options(max_iters=0)
        y = x.clone()
        lg = B.Log.empty(self.ts.num_batch, device=self.dev)
        self.h.solve(self.matrix(), self.rhs, y, o, lg)
        return float(lg.rel_res.mean())

    def run(self, train_steps=64, eval_steps=16, epochs=6, lr=1e-3, batch=4096, progress=None,
            gate_steps=8) -> LearnedReport:
        """Solve steps 0..train_steps-1 from x(t-1); train the network on the
        changes of steps 1..train_steps-gate_steps-1; fit the gate on the last
        gate_steps training steps (held out from the network's training); then
        time eval_steps steps of (prediction + solve) against a solve from
        x(t-1) and one from x0 = 0."""
        Bsz, n = self.ts.num_batch, self.n
        fit_end = train_steps - gate_steps  # samples of steps 1..fit_end-1
        # 1. solve the training steps from the previous solution; keep x(t)
        t0 = time.perf_counter()
        xs = [torch.zeros(Bsz, n, dtype=torch.float64, device=self.dev)]  # x(-1) = 0
        for t in range(train_steps):
            self.set_step(t)
            x = xs[-1].clone()
            self.solve(x)
            xs.append(x)
        torch.cuda.synchronize()
        collect_s = time.perf_counter() - t0
        # 2. statistics and samples from steps 1..train_steps-1 (x(t-1) from the solver)
        t1 = time.perf_counter()
        for t in range(1, fit_end):
            self.set_step(t)
            self.mlp.observe(self.matrix(), self.rhs, xs[t], xs[t + 1])
        self.mlp.finalize_stats()
        S = (fit_end - 1) * Bsz
        feats = torch.empty(S, self.mlp.in_pad, dtype=torch.bfloat16, device=self.dev)
        targets = torch.empty(S, n, dtype=torch.float32, device=self.dev)
        for k, t in enumerate(range(1, fit_end)):
            self.set_step(t)
            self.mlp.make_samples(self.matrix(), self.rhs, xs[t], xs[t + 1],
                                  feats[k * Bsz:(k + 1) * Bsz], targets[k * Bsz:(k + 1) * Bsz])
        # 3. Adam over shuffled minibatches
        gen = torch.Generator(device=self.dev)
        gen.manual_seed(1234)
        losses = []
        mb = min(batch, self.max_batch)
        steps_per_epoch = S // mb
        loss = torch.zeros(1, dtype=torch.float32, device=self.dev)
        for ep in range(epochs):
            perm = torch.randperm(S, device=self.dev, generator=gen).to(torch.int32)
            acc = torch.zeros(1, dtype=torch.float64, device=self.dev)
            lr_ep = lr if ep < epochs - 2 else lr * 0.3
            for s in range(steps_per_epoch):
                rows = perm[s * mb:(s + 1) * mb]
                self.mlp.train_step(feats, targets, rows, lr_ep, loss)
                acc += loss.double()
            losses.append(float(acc) / steps_per_epoch)
            if progress:
                progress(f"epoch {ep}: loss {losses[-1]:.4f}")
        torch.cuda.synchronize()
        train_s = time.perf_counter() - t1
        del feats, targets
        rep = LearnedReport(train_steps, eval_steps, Bsz, train_s, collect_s, losses)
        # 4. the gate, fitted on the held-out training steps; the squared
        # error of the gated guess there against that of x(t-1)
        if gate_steps > 0:
            for t in range(fit_end, train_steps):
                self.set_step(t)
                self.mlp.gate_observe(self.matrix(), self.rhs, xs[t], xs[t + 1])
            self.mlp.gate_finalize()
            rep.gate, rep.gate_steps = self.mlp.gate(), gate_steps
            for t in range(fit_end, train_steps):
                self.set_step(t)
                x0 = self.mlp.predict(self.matrix(), self.rhs, xs[t])
                rep.gate_err_learned += float(((xs[t + 1] - x0) ** 2).sum())
                rep.gate_err_base += float(((xs[t + 1] - xs[t]) ** 2).sum())
        # 5. evaluation steps: same x(t-1) for every guess
        x_prev = xs[-1]
        del xs
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for t in range(train_steps, train_steps + eval_steps):
            self.set_step(t)
            xb = x_prev.clone()
            r0b = self.init_residual(xb)
            torch.cuda.synchronize()
            e0.record()
            self.solve(xb)
            e1.record()
            torch.cuda.synchronize()
            ms_b = e0.elapsed_time(e1)
            it_b = float(self.log.iters.double().mean())
            xl = torch.empty_like(x_prev)
            e0.record()
            self.mlp.predict(self.matrix(), self.rhs, x_prev, xl)
            e1.record()
            torch.cuda.synchronize()
            ms_p = e0.elapsed_time(e1)
            r0l = self.init_residual(xl)
            e0.record()
            self.solve(xl)
            e1.record()
            torch.cuda.synchronize()
            ms_l = e0.elapsed_time(e1) + ms_p
            it_l = float(self.log.iters.double().mean())
            conv = int((self.log.status == 0).sum())
            xz = torch.zeros_like(x_prev)
            e0.record()
            self.solve(xz)
            e1.record()
            torch.cuda.synchronize()
            ms_z = e0.elapsed_time(e1)
            it_z = float(self.log.iters.double().mean())
            rep.records.append(StepRecord(t, it_b, it_l, ms_b, ms_l, r0b, r0l, conv, it_z, ms_z, ms_p))
            x_prev = xl
        return rep
