"""ctypes binding of libbbs.so (include/bbs.h), argument marshalling only.

Every step of a solve runs in the CUDA library; this module only turns torch
tensors into the pointers and structs the C ABI takes. If the library has not
been built, loading raises: there is no fallback of any kind.
"""

from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np
import torch

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libbbs.so")

BBS_OK = 0
FMT = {"csr": 0, "ell": 1, "dense": 2}
SOLVER = {"bicgstab": 0, "cg": 1, "gmres": 2}
PRECOND = {"none": 0, "jacobi": 1, "ilu0": 2}
TOL = {"absolute": 0, "relative": 1}
PRECISION = {"fp64": 0, "mixed": 1}
SYS_STATUS = {0: "converged", 1: "max_iter", 2: "breakdown", 3: "nan"}
GEMM = {"mma": 0, "tcgen05": 1}


class bbs_batch_matrix(C.Structure):
    _fields_ = [("fmt", C.c_int32), ("num_batch", C.c_int32), ("n", C.c_int32),
                ("nnz", C.c_int32), ("ell_k", C.c_int32), ("row_ptrs", C.c_void_p),
                ("col_idxs", C.c_void_p), ("values", C.c_void_p), ("values_f32", C.c_void_p)]


class bbs_options(C.Structure):
    _fields_ = [("solver", C.c_int32), ("precond", C.c_int32), ("tol_type", C.c_int32),
                ("max_iters", C.c_int32), ("tol", C.c_double), ("gmres_restart", C.c_int32),
                ("precision", C.c_int32), ("inner_tol", C.c_double), ("max_outer", C.c_int32),
                ("threads_per_system", C.c_int32), ("values_in_smem", C.c_int32),
                ("reserved", C.c_int32)]


class bbs_log(C.Structure):
    _fields_ = [("iters", C.c_void_p), ("rel_res", C.c_void_p), ("status", C.c_void_p),
                ("inner_iters", C.c_void_p)]


class bbs_launch_info(C.Structure):
    _fields_ = [("kernel", C.c_char_p), ("grid", C.c_int32), ("block", C.c_int32),
                ("threads_per_system", C.c_int32), ("rows_per_thread", C.c_int32),
                ("smem_bytes", C.c_int64), ("values_staged", C.c_int32), ("launches", C.c_int32)]


class bbs_var_batch(C.Structure):
    _fields_ = [("num_batch", C.c_int32), ("num_patterns", C.c_int32), ("pat_n", C.c_void_p),
                ("pat_nnz", C.c_void_p), ("pat_rp_off", C.c_void_p), ("pat_ci_off", C.c_void_p),
                ("row_ptrs", C.c_void_p), ("col_idxs", C.c_void_p), ("sys_pattern", C.c_void_p),
                ("val_off", C.c_void_p), ("vec_off", C.c_void_p), ("values", C.c_void_p)]


class bbs_var_host_info(C.Structure):
    _fields_ = [("pat_n", C.c_void_p), ("pat_nnz", C.c_void_p), ("sys_pattern", C.c_void_p)]


class bbs_var_plan_desc(C.Structure):
    _fields_ = [("team_systems", C.c_int32), ("packed_systems", C.c_int32),
                ("packed_launches", C.c_int32), ("persistent_grid", C.c_int32),
                ("wide_systems", C.c_int32), ("wide_launches", C.c_int32)]


class bbs_var_tuning(C.Structure):
    _fields_ = [("num_buckets", C.c_int32), ("bucket_max_n", C.c_int32 * 8),
                ("team_warps", C.c_int32 * 8), ("stage_values", C.c_int32 * 8),
                ("pack", C.c_int32 * 8), ("wide", C.c_int32 * 8), ("block_warps", C.c_int32),
                ("reserved", C.c_int32)]

    def as_dict(self) -> dict:
        k = self.num_buckets
        return {"bucket_max_n": list(self.bucket_max_n[:k]), "team_warps": list(self.team_warps[:k]),
                "stage_values": list(self.stage_values[:k]), "pack": list(self.pack[:k]),
                "wide": list(self.wide[:k]),
                "block_warps": self.block_warps}

    @classmethod
    def from_dict(cls, d: dict) -> "bbs_var_tuning":
        t = cls()
        k = len(d["bucket_max_n"])
        t.num_buckets = k
        for i in range(k):
            t.bucket_max_n[i] = d["bucket_max_n"][i]
            t.team_warps[i] = d["team_warps"][i]
            t.stage_values[i] = d["stage_values"][i]
            t.pack[i] = d.get("pack", [1] * k)[i]
            t.wide[i] = d.get("wide", [1] * k)[i]
        t.block_warps = d["block_warps"]
        return t


_lib = None


def lib():
    """The loaded libbbs.so; raises if it was not built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                               "(python -c 'import __graft_entry__ as g; g.build()')")
        L = C.CDLL(LIB_PATH)
        P = C.POINTER
        L.bbs_default_options.argtypes = [P(bbs_options)]
        L.bbs_create.argtypes = [P(C.c_void_p), C.c_int]
        L.bbs_destroy.argtypes = [C.c_void_p]
        L.bbs_workspace_size.argtypes = [C.c_void_p, P(bbs_batch_matrix), P(bbs_options),
                                         P(C.c_size_t)]
        L.bbs_describe.argtypes = [C.c_void_p, P(bbs_batch_matrix), P(bbs_options), P(bbs_launch_info)]
        L.bbs_check_pattern.argtypes = [C.c_void_p, P(bbs_batch_matrix), P(C.c_int32)]
        L.bbs_solve.argtypes = [C.c_void_p, P(bbs_batch_matrix), C.c_void_p, C.c_void_p,
                                P(bbs_options), P(bbs_log), C.c_void_p, C.c_size_t, C.c_void_p]
        L.bbs_solve_host.argtypes = [C.c_void_p, P(bbs_batch_matrix), C.c_void_p, C.c_void_p,
                                     P(bbs_options), P(bbs_log)]
        L.bbs_solve_noalloc.argtypes = [C.c_void_p, P(bbs_batch_matrix), C.c_void_p, C.c_void_p,
                                        P(bbs_options), P(bbs_log), C.c_void_p]
        L.bbs_var_default_tuning.argtypes = [C.c_int32, P(bbs_var_tuning)]
        L.bbs_var_plan_create.argtypes = [C.c_void_p, P(bbs_var_batch), P(bbs_var_host_info),
                                          P(bbs_options), P(bbs_var_tuning), P(C.c_void_p)]
        L.bbs_var_solve.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, P(bbs_log), C.c_void_p]
        L.bbs_var_plan_destroy.argtypes = [C.c_void_p]
        L.bbs_var_plan_describe.argtypes = [C.c_void_p, P(bbs_var_plan_desc)]
        L.bbs_var_tune.argtypes = [C.c_void_p, P(bbs_var_batch), P(bbs_var_host_info), C.c_void_p,
                                   C.c_void_p, P(bbs_options), C.c_int32, P(bbs_var_tuning)]
        vp, i32, st = C.c_void_p, C.c_int32, C.c_void_p
        L.bbs_mlp_create.argtypes = [vp, i32, i32, C.c_uint64, i32, P(C.c_void_p)]
        L.bbs_mlp_destroy.argtypes = [vp]
        L.bbs_mlp_param_count.argtypes = [vp, P(C.c_int64)]
        L.bbs_mlp_get_params.argtypes = [vp, vp, st]
        L.bbs_mlp_set_params.argtypes = [vp, vp, st]
        L.bbs_mlp_get_grads.argtypes = [vp, vp, st]
        L.bbs_mlp_observe.argtypes = [vp, P(bbs_batch_matrix), vp, vp, vp, st]
        L.bbs_mlp_finalize_stats.argtypes = [vp, st]
        L.bbs_mlp_make_samples.argtypes = [vp, P(bbs_batch_matrix), vp, vp, vp, vp, vp, st]
        L.bbs_mlp_gradients.argtypes = [vp, vp, vp, vp, i32, vp, st]
        L.bbs_mlp_train_step.argtypes = [vp, vp, vp, vp, i32, C.c_float, vp, st]
        L.bbs_mlp_forward.argtypes = [vp, vp, i32, vp, st]
        L.bbs_mlp_predict.argtypes = [vp, P(bbs_batch_matrix), vp, vp, vp, st]
        L.bbs_mlp_gate_observe.argtypes = [vp, P(bbs_batch_matrix), vp, vp, vp, st]
        L.bbs_mlp_gate_finalize.argtypes = [vp, st]
        L.bbs_mlp_get_gate.argtypes = [vp, P(C.c_double)]
        L.bbs_mlp_set_gemm.argtypes = [vp, i32]
        L.bbs_mlp_check.argtypes = [vp]
        L.bbs_gemm_bf16.argtypes = [vp, i32, vp, i32, vp, i32, i32, i32, i32, vp, i32]
        L.bbs_paper_block_size.argtypes = [C.c_int32, C.c_int32]
        L.bbs_paper_block_size.restype = C.c_int32
        L.bbs_default_block_size.argtypes = [C.c_int32, C.c_int32]
        L.bbs_default_block_size.restype = C.c_int32
        L.bbs_host_chunk_plan.argtypes = [C.c_int64, C.c_int64, C.c_void_p, C.c_void_p, C.c_int32]
        L.bbs_fma_rate.argtypes = [C.c_void_p, C.c_int32, P(C.c_double)]
        L.bbs_host_chunk_plan.restype = C.c_int32
        L.bbs_last_error.restype = C.c_char_p
        L.bbs_version.restype = C.c_char_p
        for name in ("bbs_default_options", "bbs_create", "bbs_destroy", "bbs_workspace_size", "bbs_describe", "bbs_check_pattern",
                     "bbs_solve", "bbs_solve_host", "bbs_solve_noalloc", "bbs_var_default_tuning",
                     "bbs_var_plan_create", "bbs_var_solve", "bbs_var_plan_destroy", "bbs_var_tune",
                     "bbs_var_plan_describe",
                     "bbs_mlp_create", "bbs_mlp_destroy", "bbs_mlp_param_count", "bbs_mlp_get_params",
                     "bbs_mlp_set_params", "bbs_mlp_get_grads", "bbs_mlp_observe",
                     "bbs_mlp_finalize_stats", "bbs_mlp_make_samples", "bbs_mlp_gradients",
                     "bbs_mlp_train_step", "bbs_mlp_forward", "bbs_mlp_predict", "bbs_mlp_set_gemm",
                     "bbs_mlp_check", "bbs_gemm_bf16", "bbs_fma_rate", "bbs_mlp_gate_observe",
                     "bbs_mlp_gate_finalize", "bbs_mlp_get_gate"):
            getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


class BBSError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = lib().bbs_last_error().decode()
        super().__init__(f"{where} failed with status {status}: {msg}")
        self.status = status


def _check(status: int, where: str):
    if status != BBS_OK:
        raise BBSError(status, where)


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def bbs_default_options(**overrides) -> bbs_options:
    o = bbs_options()
    _check(lib().bbs_default_options(C.byref(o)), "bbs_default_options")
    for k, v in overrides.items():
        if k == "solver":
            v = SOLVER[v] if isinstance(v, str) else v
        elif k == "precond":
            v = PRECOND[v] if isinstance(v, str) else v
        elif k == "tol_type":
            v = TOL[v] if isinstance(v, str) else v
        elif k == "precision":
            v = PRECISION[v] if isinstance(v, str) else v
        setattr(o, k, v)
    return o


def bbs_paper_block_size(n: int, max_threads: int = 1024) -> int:
    return int(lib().bbs_paper_block_size(n, max_threads))


def bbs_default_block_size(n: int, rows_per_thread: int = 5) -> int:
    return int(lib().bbs_default_block_size(n, rows_per_thread))


def bbs_host_chunk_plan(num_batch: int, input_bytes_per_system: int, max_chunks: int = 16):
    """bbs_host_chunk_plan: the (first, count) chunks bbs_solve_host cuts a
    batch into, or None when it returns -1."""
    first = (C.c_int64 * max(max_chunks, 1))()
    count = (C.c_int64 * max(max_chunks, 1))()
    n = int(lib().bbs_host_chunk_plan(num_batch, input_bytes_per_system, first, count, max_chunks))
    return None if n < 0 else [(int(first[i]), int(count[i])) for i in range(n)]


def bbs_fma_rate(handle: "Handle", precision: str = "fp64") -> float:
    """bbs_fma_rate: measured FMA throughput of the handle's device in FLOP/s
    (precision "fp64" or "fp32")."""
    out = C.c_double()
    _check(lib().bbs_fma_rate(handle._h, {"fp64": 0, "fp32": 1}[precision], C.byref(out)), "bbs_fma_rate")
    return float(out.value)


def bbs_version() -> str:
    return lib().bbs_version().decode()


@dataclass
class DeviceBatch:
    """Tensors of one batch matrix (Sec. 3.1 layouts), on one device or on the host."""

    fmt: str
    n: int
    nnz: int
    ell_k: int
    row_ptrs: torch.Tensor | None
    col_idxs: torch.Tensor | None
    values: torch.Tensor
    values_f32: torch.Tensor | None = None

    @property
    def num_batch(self) -> int:
        return int(self.values.shape[0])

    @classmethod
    def from_batch(cls, A, device="cuda", values_f32: bool = False, pin: bool = False):
        """From a workloads.BatchMatrix (numpy) to tensors on `device`."""
        def t(a, dtype):
            if a is None:
                return None
            x = torch.as_tensor(a).to(dtype)
            if device == "cpu":
                return x.pin_memory() if pin else x.contiguous()
            return x.to(device)
        vals = t(A.values, torch.float64)
        rp = t(A.row_ptrs, torch.int32) if A.fmt == "csr" else None
        ci = t(A.col_idxs, torch.int32) if A.fmt in ("csr", "ell") else None
        v32 = vals.to(torch.float32) if values_f32 else None
        # CSR: pass the largest row length, which lets small systems run packed
        k = int(np.diff(A.row_ptrs).max()) if A.fmt == "csr" and A.n > 0 else A.ell_k
        return cls(A.fmt, A.n, A.nnz, k, rp, ci, vals, v32)

    def struct(self) -> bbs_batch_matrix:
        return bbs_batch_matrix(FMT[self.fmt], self.num_batch, self.n, self.nnz, self.ell_k,
                                _ptr(self.row_ptrs), _ptr(self.col_idxs), _ptr(self.values),
                                _ptr(self.values_f32))


@dataclass
class Log:
    iters: torch.Tensor
    rel_res: torch.Tensor
    status: torch.Tensor
    inner_iters: torch.Tensor | None = None

    @classmethod
    def empty(cls, num_batch: int, device="cuda", inner: bool = False, pin: bool = False):
        kw = dict(device=device)
        mk = (lambda *a, **k: torch.empty(*a, **k).pin_memory()) if pin else torch.empty
        return cls(mk(num_batch, dtype=torch.int32, **kw), mk(num_batch, dtype=torch.float64, **kw),
                   mk(num_batch, dtype=torch.int32, **kw),
                   mk(num_batch, dtype=torch.int32, **kw) if inner else None)

    def struct(self) -> bbs_log:
        return bbs_log(_ptr(self.iters), _ptr(self.rel_res), _ptr(self.status), _ptr(self.inner_iters))


class Handle:
    """Owns a bbs_handle for one device."""

    def __init__(self, device: int = 0):
        h = C.c_void_p()
        _check(lib().bbs_create(C.byref(h), int(device)), "bbs_create")
        self._h = h
        self.device = int(device)

    def close(self):
        if self._h:
            lib().bbs_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def workspace_size(self, A: DeviceBatch, opts: bbs_options) -> int:
        out = C.c_size_t()
        s = A.struct()
        _check(lib().bbs_workspace_size(self._h, C.byref(s), C.byref(opts), C.byref(out)),
               "bbs_workspace_size")
        return int(out.value)

    def describe(self, A: DeviceBatch, opts: bbs_options) -> dict:
        """bbs_describe: the launch a solve of A with opts makes."""
        info = bbs_launch_info()
        s = A.struct()
        _check(lib().bbs_describe(self._h, C.byref(s), C.byref(opts), C.byref(info)), "bbs_describe")
        return {"kernel": info.kernel.decode(), "grid": info.grid, "block": info.block,
                "threads_per_system": info.threads_per_system, "rows": info.rows_per_thread,
                "smem": info.smem_bytes, "staged": bool(info.values_staged), "launches": info.launches}

    def check_pattern(self, A: DeviceBatch) -> int:
        """bbs_check_pattern: the number of rows of A's shared pattern that break its format's rules."""
        bad = C.c_int32()
        s = A.struct()
        _check(lib().bbs_check_pattern(self._h, C.byref(s), C.byref(bad)), "bbs_check_pattern")
        return int(bad.value)

    def workspace(self, A: DeviceBatch, opts: bbs_options) -> torch.Tensor | None:
        nb = self.workspace_size(A, opts)
        if nb == 0:
            return None
        return torch.empty(nb, dtype=torch.uint8, device=A.values.device)

    def solve(self, A: DeviceBatch, b: torch.Tensor, x: torch.Tensor, opts: bbs_options,
              log: Log, workspace: torch.Tensor | None = None, stream=None):
        """bbs_solve: x (in: x0, out: solution) and log are written asynchronously."""
        s = A.struct()
        lg = log.struct()
        ws_bytes = 0 if workspace is None else workspace.numel() * workspace.element_size()
        st = stream if stream is not None else torch.cuda.current_stream(A.values.device)
        _check(lib().bbs_solve(self._h, C.byref(s), _ptr(b), _ptr(x), C.byref(opts), C.byref(lg),
                               _ptr(workspace), ws_bytes, C.c_void_p(st.cuda_stream)), "bbs_solve")

    def solve_noalloc(self, A: DeviceBatch, b: torch.Tensor, x: torch.Tensor, opts: bbs_options,
                      log: Log, stream=None):
        """bbs_solve_noalloc: like solve() with the library's static scratch
        instead of a workspace (for callers that cannot allocate)."""
        s = A.struct()
        lg = log.struct()
        st = stream if stream is not None else torch.cuda.current_stream(A.values.device)
        _check(lib().bbs_solve_noalloc(self._h, C.byref(s), _ptr(b), _ptr(x), C.byref(opts),
                                       C.byref(lg), C.c_void_p(st.cuda_stream)), "bbs_solve_noalloc")

    def solve_host(self, A: DeviceBatch, b: torch.Tensor, x: torch.Tensor, opts: bbs_options,
                   log: Log):
        """bbs_solve_host: every tensor in host memory; returns when results are back."""
        s = A.struct()
        lg = log.struct()
        _check(lib().bbs_solve_host(self._h, C.byref(s), _ptr(b), _ptr(x), C.byref(opts),
                                    C.byref(lg)), "bbs_solve_host")


def solve(A: DeviceBatch, b: torch.Tensor, x0: torch.Tensor | None = None, handle: Handle | None = None,
          **opts):
    """Convenience: allocate x, log and workspace, solve on the current stream.

    Returns (x, Log). opts are bbs_options fields (strings allowed for enums).
    """
    dev = A.values.device
    h = handle or Handle(dev.index or 0)
    o = bbs_default_options(**opts)
    x = (torch.zeros_like(b) if x0 is None else x0.clone()).contiguous()
    log = Log.empty(A.num_batch, device=dev, inner=(o.precision == 1))
    ws = h.workspace(A, o)
    h.solve(A, b.contiguous(), x, o, log, ws)
    return x, log


# ------------------------------------------------------------ uneven batches

@dataclass
class VarDeviceBatch:
    """An uneven batch (workloads.VarBatch) on the device, plus the host metadata
    the planner reads."""

    tensors: dict
    host: dict
    num_batch: int
    num_patterns: int
    vec_len: int

    @classmethod
    def from_varbatch(cls, vb, device="cuda"):
        import numpy as np

        pat_n, pat_nnz, rp_off, ci_off, rps, cis = vb.pools()
        t = {
            "pat_n": torch.as_tensor(pat_n, dtype=torch.int32, device=device),
            "pat_nnz": torch.as_tensor(pat_nnz, dtype=torch.int32, device=device),
            "pat_rp_off": torch.as_tensor(rp_off, dtype=torch.int64, device=device),
            "pat_ci_off": torch.as_tensor(ci_off, dtype=torch.int64, device=device),
            "row_ptrs": torch.as_tensor(rps, dtype=torch.int32, device=device),
            "col_idxs": torch.as_tensor(cis, dtype=torch.int32, device=device),
            "sys_pattern": torch.as_tensor(vb.sys_pattern, dtype=torch.int32, device=device),
            "val_off": torch.as_tensor(vb.val_off, dtype=torch.int64, device=device),
            "vec_off": torch.as_tensor(vb.vec_off, dtype=torch.int64, device=device),
            "values": torch.as_tensor(vb.values, dtype=torch.float64, device=device),
        }
        host = {"pat_n": np.ascontiguousarray(pat_n, dtype=np.int32),
                "pat_nnz": np.ascontiguousarray(pat_nnz, dtype=np.int32),
                "sys_pattern": np.ascontiguousarray(vb.sys_pattern, dtype=np.int32)}
        return cls(t, host, vb.num_batch, len(vb.patterns), int(vb.b.shape[0]))

    def struct(self) -> bbs_var_batch:
        t = self.tensors
        return bbs_var_batch(self.num_batch, self.num_patterns, *[_ptr(t[k]) for k in (
            "pat_n", "pat_nnz", "pat_rp_off", "pat_ci_off", "row_ptrs", "col_idxs", "sys_pattern",
            "val_off", "vec_off", "values")])

    def host_struct(self) -> bbs_var_host_info:
        h = self.host
        return bbs_var_host_info(*[C.c_void_p(h[k].ctypes.data) for k in ("pat_n", "pat_nnz", "sys_pattern")])


def bbs_var_default_tuning(max_n: int) -> bbs_var_tuning:
    t = bbs_var_tuning()
    _check(lib().bbs_var_default_tuning(int(max_n), C.byref(t)), "bbs_var_default_tuning")
    return t


def bbs_var_tune(handle: Handle, vbd: VarDeviceBatch, b: torch.Tensor, x0: torch.Tensor,
                 opts: bbs_options, sample: int = 512) -> bbs_var_tuning:
    t = bbs_var_tuning()
    s, hs = vbd.struct(), vbd.host_struct()
    _check(lib().bbs_var_tune(handle._h, C.byref(s), C.byref(hs), _ptr(b), _ptr(x0), C.byref(opts),
                              int(sample), C.byref(t)), "bbs_var_tune")
    return t


class VarPlan:
    """bbs_var_plan: a planned, graph-captured persistent solve of an uneven batch."""

    def __init__(self, handle: Handle, vbd: VarDeviceBatch, opts: bbs_options,
                 tuning: bbs_var_tuning | None = None):
        p = C.c_void_p()
        s, hs = vbd.struct(), vbd.host_struct()
        _check(lib().bbs_var_plan_create(handle._h, C.byref(s), C.byref(hs), C.byref(opts),
                                         None if tuning is None else C.byref(tuning), C.byref(p)),
               "bbs_var_plan_create")
        self._p = p
        self._keep = (handle, vbd)

    def solve(self, b: torch.Tensor, x: torch.Tensor, log: Log, stream=None):
        lg = log.struct()
        st = stream if stream is not None else torch.cuda.current_stream(b.device)
        _check(lib().bbs_var_solve(self._p, _ptr(b), _ptr(x), C.byref(lg), C.c_void_p(st.cuda_stream)),
               "bbs_var_solve")

    def describe(self) -> dict:
        d = bbs_var_plan_desc()
        _check(lib().bbs_var_plan_describe(self._p, C.byref(d)), "bbs_var_plan_describe")
        return {f: getattr(d, f) for f, _ in d._fields_}

    def close(self):
        if self._p:
            lib().bbs_var_plan_destroy(self._p)
            self._p = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------- learned guess

def _stream(t):
    return C.c_void_p(torch.cuda.current_stream(t.device).cuda_stream)


class MLP:
    """bbs_mlp: the initial-guess network (weights, statistics, activations on
    the device; every step runs in the library's kernels)."""

    def __init__(self, handle: Handle, n: int, hidden: int = 256, seed: int = 0, max_batch: int = 4096):
        p = C.c_void_p()
        _check(lib().bbs_mlp_create(handle._h, int(n), int(hidden), int(seed), int(max_batch), C.byref(p)),
               "bbs_mlp_create")
        self._p = p
        self._handle = handle
        self.n, self.hidden, self.max_batch = int(n), int(hidden), int(max_batch)
        self.in_pad = (3 * self.n + 63) // 64 * 64
        cnt = C.c_int64()
        _check(lib().bbs_mlp_param_count(p, C.byref(cnt)), "bbs_mlp_param_count")
        self.param_count = int(cnt.value)
        self.device = torch.device("cuda", handle.device)

    def close(self):
        if self._p:
            lib().bbs_mlp_destroy(self._p)
            self._p = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_gemm(self, kind: str):
        _check(lib().bbs_mlp_set_gemm(self._p, GEMM[kind]), "bbs_mlp_set_gemm")

    def check(self):
        _check(lib().bbs_mlp_check(self._p), "bbs_mlp_check")

    def get_params(self) -> torch.Tensor:
        out = torch.empty(self.param_count, dtype=torch.float32, device=self.device)
        _check(lib().bbs_mlp_get_params(self._p, _ptr(out), _stream(out)), "bbs_mlp_get_params")
        return out

    def set_params(self, params: torch.Tensor):
        params = params.to(self.device, torch.float32).contiguous()
        _check(lib().bbs_mlp_set_params(self._p, _ptr(params), _stream(params)), "bbs_mlp_set_params")

    def get_grads(self) -> torch.Tensor:
        out = torch.empty(self.param_count, dtype=torch.float32, device=self.device)
        _check(lib().bbs_mlp_get_grads(self._p, _ptr(out), _stream(out)), "bbs_mlp_get_grads")
        return out

    def observe(self, A: DeviceBatch, b, x_prev, x_next):
        s = A.struct()
        _check(lib().bbs_mlp_observe(self._p, C.byref(s), _ptr(b), _ptr(x_prev), _ptr(x_next), _stream(b)),
               "bbs_mlp_observe")

    def finalize_stats(self):
        _check(lib().bbs_mlp_finalize_stats(self._p, C.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)),
               "bbs_mlp_finalize_stats")

    def make_samples(self, A: DeviceBatch, b, x_prev, x_next=None, feats=None, targets=None):
        B = A.num_batch
        if feats is None:
            feats = torch.empty(B, self.in_pad, dtype=torch.bfloat16, device=self.device)
        if x_next is not None and targets is None:
            targets = torch.empty(B, self.n, dtype=torch.float32, device=self.device)
        s = A.struct()
        _check(lib().bbs_mlp_make_samples(self._p, C.byref(s), _ptr(b), _ptr(x_prev), _ptr(x_next),
                                          _ptr(feats), _ptr(targets), _stream(b)), "bbs_mlp_make_samples")
        return feats, targets

    def gradients(self, feats, targets, rows, loss=None):
        loss = torch.zeros(1, dtype=torch.float32, device=self.device) if loss is None else loss
        _check(lib().bbs_mlp_gradients(self._p, _ptr(feats), _ptr(targets), _ptr(rows), int(rows.numel()),
                                       _ptr(loss), _stream(feats)), "bbs_mlp_gradients")
        return loss

    def train_step(self, feats, targets, rows, lr, loss=None):
        loss = torch.zeros(1, dtype=torch.float32, device=self.device) if loss is None else loss
        _check(lib().bbs_mlp_train_step(self._p, _ptr(feats), _ptr(targets), _ptr(rows), int(rows.numel()),
                                        float(lr), _ptr(loss), _stream(feats)), "bbs_mlp_train_step")
        return loss

    def forward(self, feats) -> torch.Tensor:
        M = int(feats.shape[0])
        out = torch.empty(M, self.n, dtype=torch.float32, device=self.device)
        _check(lib().bbs_mlp_forward(self._p, _ptr(feats), M, _ptr(out), _stream(feats)), "bbs_mlp_forward")
        return out

    def gate_observe(self, A: DeviceBatch, b, x_prev, x_next):
        s = A.struct()
        _check(lib().bbs_mlp_gate_observe(self._p, C.byref(s), _ptr(b), _ptr(x_prev), _ptr(x_next), _stream(b)),
               "bbs_mlp_gate_observe")

    def gate_finalize(self):
        _check(lib().bbs_mlp_gate_finalize(self._p, C.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)),
               "bbs_mlp_gate_finalize")

    def gate(self) -> float:
        g = C.c_double()
        _check(lib().bbs_mlp_get_gate(self._p, C.byref(g)), "bbs_mlp_get_gate")
        return float(g.value)

    def predict(self, A: DeviceBatch, b, x_prev, x0=None):
        x0 = torch.empty_like(x_prev) if x0 is None else x0
        s = A.struct()
        _check(lib().bbs_mlp_predict(self._p, C.byref(s), _ptr(b), _ptr(x_prev), _ptr(x0), _stream(b)),
               "bbs_mlp_predict")
        return x0


def bbs_gemm_bf16(handle: Handle, kind: str, A: torch.Tensor, B: torch.Tensor) -> torch.Tensor:
    """C = A B^T (A [M, K], B [N, K] bfloat16 on the device) through a tensor-core path."""
    M, K = A.shape
    N = B.shape[0]
    C_ = torch.empty(M, N, dtype=torch.float32, device=A.device)
    _check(lib().bbs_gemm_bf16(handle._h, GEMM[kind], _ptr(A), A.stride(0), _ptr(B), B.stride(0), M, N, K,
                               _ptr(C_), N), "bbs_gemm_bf16")
    return C_

