"""Seeded synthetic batches shaped like the paper's workloads.

This module only builds inputs: stencil sparsity patterns (one pattern shared
by every system of a batch, Sec. 3.1), random matrix values with the stated
distributions, right-hand sides and initial guesses, and re-layouts of the
same entries into the three batch formats (BatchCsr, BatchEll column-major,
BatchDense row-major; Sec. 3.1). No step of a Krylov solve happens here. Both
the CUDA library and the CPU oracle consume what it returns, so this is the one
module the two sides share.

Value recipe (the paper's 3-point stencil SPD study, Sec. 5.1, and the PeleLM
inputs, Table "Reference for data inputs", are stood in for by these):
  * for every undirected stencil edge {i, j}: s ~ U[-1, 0], then
    a_ij = s * (1 + U[-0.1, 0.1]) and a_ji = s * (1 + U[-0.1, 0.1]), drawn
    independently, so the matrix is nonsymmetric;
  * a_ii = (sum_{j != i} |a_ij|) * (1 + U[lo, hi]) (strict diagonal dominance);
  * b ~ U[-1, 1], x0 = 0.
All draws use NumPy's PCG64 seeded with SEED_BASE + workload index.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 230808417

FMT_CSR, FMT_ELL, FMT_DENSE = 0, 1, 2
FMT_NAMES = {"csr": FMT_CSR, "ell": FMT_ELL, "dense": FMT_DENSE}

_CHUNK = 4096  # systems drawn per RNG call; part of the recipe's draw order


@dataclass
class Pattern:
    """One shared CSR sparsity pattern (0-based, columns sorted per row)."""

    n: int
    row_ptrs: np.ndarray  # int32 [n+1]
    col_idxs: np.ndarray  # int32 [nnz]
    kind: str = ""
    kx: int = 0
    ky: int = 0

    @property
    def nnz(self) -> int:
        return int(self.row_ptrs[-1])

    @property
    def max_row(self) -> int:
        return int(np.max(np.diff(self.row_ptrs))) if self.n else 0


@dataclass
class BatchMatrix:
    """A batch of matrices with one shared pattern, in one storage format.

    Layout is row-of-systems: system i's values are contiguous.
      csr:   row_ptrs [n+1], col_idxs [nnz],   values [B, nnz]
      ell:   col_idxs [k*n] column-major (slot j of row r at j*n + r, pad -1),
             values [B, k*n] in the same order (pad 0)
      dense: values [B, n*n] row-major
    """

    fmt: str
    n: int
    nnz: int
    ell_k: int
    row_ptrs: np.ndarray
    col_idxs: np.ndarray
    values: np.ndarray
    pattern: Pattern = field(repr=False, default=None)

    @property
    def num_batch(self) -> int:
        return int(self.values.shape[0])

    @property
    def fmt_code(self) -> int:
        return FMT_NAMES[self.fmt]

    def subset(self, idx) -> "BatchMatrix":
        idx = np.asarray(idx)
        return BatchMatrix(self.fmt, self.n, self.nnz, self.ell_k, self.row_ptrs,
                           self.col_idxs, np.ascontiguousarray(self.values[idx]),
                           self.pattern)


# --------------------------------------------------------------------------
# patterns
# --------------------------------------------------------------------------

def stencil_pattern(kind: str, kx: int, ky: int = 1) -> Pattern:
    """Sparsity pattern of a 1D 3-point, 2D 5-point or 2D 9-point stencil.

    Grid node (ix, iy) is row iy*kx + ix. Columns are sorted ascending.
    """
    if kind == "1d3":
        offsets = [(-1, 0), (0, 0), (1, 0)]
        ky = 1
    elif kind == "2d5":
        offsets = [(0, -1), (-1, 0), (0, 0), (1, 0), (0, 1)]
    elif kind == "2d9":
        offsets = [(dx, dy) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
    else:
        raise ValueError(f"unknown stencil {kind!r}")
    n = kx * ky
    rows = []
    for iy in range(ky):
        for ix in range(kx):
            cols = []
            for dx, dy in offsets:
                jx, jy = ix + dx, iy + dy
                if 0 <= jx < kx and 0 <= jy < ky:
                    cols.append(jy * kx + jx)
            rows.append(sorted(cols))
    row_ptrs = np.zeros(n + 1, dtype=np.int32)
    row_ptrs[1:] = np.cumsum([len(r) for r in rows])
    col_idxs = np.array([c for r in rows for c in r], dtype=np.int32)
    return Pattern(n, row_ptrs, col_idxs, kind, kx, ky)


def _entry_tables(pat: Pattern):
    """Positions of diagonal entries and of both halves of each edge."""
    rows = np.repeat(np.arange(pat.n), np.diff(pat.row_ptrs))
    cols = pat.col_idxs.astype(np.int64)
    pos = {(int(r), int(c)): e for e, (r, c) in enumerate(zip(rows, cols))}
    diag = np.array([pos[(i, i)] for i in range(pat.n)], dtype=np.int64)
    upper = [(r, c) for (r, c) in pos if r < c]
    upper.sort()
    pos_ij = np.array([pos[(r, c)] for r, c in upper], dtype=np.int64)
    pos_ji = np.array([pos[(c, r)] for r, c in upper], dtype=np.int64)
    return rows, diag, pos_ij, pos_ji


def stencil_values(pat: Pattern, num_batch: int, rng: np.random.Generator,
                   diag_lo: float, diag_hi: float, symmetric: bool = False) -> np.ndarray:
    """Values [B, nnz] of a strictly diagonally dominant batch on `pat`.

    With symmetric=True the same draws are used, the off-diagonal pair is
    replaced by its mean (a_ij + a_ji)/2 and every diagonal is recomputed from
    the symmetric off-diagonals with the same dominance draw, which gives a
    symmetric, strictly diagonally dominant matrix with a positive diagonal
    (SPD by Gershgorin).
    """
    rows, diag, pos_ij, pos_ji = _entry_tables(pat)
    nnz, n, E = pat.nnz, pat.n, len(pos_ij)
    out = np.empty((num_batch, nnz), dtype=np.float64)
    starts = pat.row_ptrs[:-1].astype(np.int64)
    for c0 in range(0, num_batch, _CHUNK):
        bc = min(_CHUNK, num_batch - c0)
        s = rng.uniform(-1.0, 0.0, (bc, E))
        f1 = rng.uniform(-0.1, 0.1, (bc, E))
        f2 = rng.uniform(-0.1, 0.1, (bc, E))
        u = rng.uniform(diag_lo, diag_hi, (bc, n))
        v = np.zeros((bc, nnz), dtype=np.float64)
        a_ij = s * (1.0 + f1)
        a_ji = s * (1.0 + f2)
        if symmetric:
            m = 0.5 * (a_ij + a_ji)
            a_ij, a_ji = m, m
        v[:, pos_ij] = a_ij
        v[:, pos_ji] = a_ji
        offsum = np.add.reduceat(np.abs(v), starts, axis=1)
        v[:, diag] = offsum * (1.0 + u)
        out[c0:c0 + bc] = v
    return out


# --------------------------------------------------------------------------
# format re-layouts (pure data movement of the same entries)
# --------------------------------------------------------------------------

def to_ell(pat: Pattern, csr_values: np.ndarray):
    """Column-major ELL layout of a CSR batch: (k, col_idxs[k*n], values[B, k*n])."""
    n, k = pat.n, pat.max_row
    lens = np.diff(pat.row_ptrs)
    rows = np.repeat(np.arange(n), lens)
    slot_in_row = np.arange(pat.nnz) - np.repeat(pat.row_ptrs[:-1], lens)
    dest = slot_in_row.astype(np.int64) * n + rows
    cols = np.full(k * n, -1, dtype=np.int32)
    cols[dest] = pat.col_idxs
    vals = np.zeros((csr_values.shape[0], k * n), dtype=csr_values.dtype)
    vals[:, dest] = csr_values
    return k, cols, vals


def to_dense(pat: Pattern, csr_values: np.ndarray) -> np.ndarray:
    """Row-major dense layout [B, n*n] of a CSR batch."""
    n = pat.n
    lens = np.diff(pat.row_ptrs)
    rows = np.repeat(np.arange(n), lens)
    dest = rows.astype(np.int64) * n + pat.col_idxs
    vals = np.zeros((csr_values.shape[0], n * n), dtype=csr_values.dtype)
    vals[:, dest] = csr_values
    return vals


def make_batch(pat: Pattern, csr_values: np.ndarray, fmt: str) -> BatchMatrix:
    if fmt == "csr":
        return BatchMatrix("csr", pat.n, pat.nnz, 0, pat.row_ptrs, pat.col_idxs,
                           np.ascontiguousarray(csr_values), pat)
    if fmt == "ell":
        k, cols, vals = to_ell(pat, csr_values)
        return BatchMatrix("ell", pat.n, pat.nnz, k, pat.row_ptrs, cols, vals, pat)
    if fmt == "dense":
        return BatchMatrix("dense", pat.n, pat.nnz, 0, pat.row_ptrs, pat.col_idxs,
                           to_dense(pat, csr_values), pat)
    raise ValueError(fmt)


def storage_entries(fmt: str, num_batch: int, n: int, nnz: int, ell_k: int = 0) -> int:
    """Number of stored array entries of a batch (values + shared index arrays).

    Sec. 3.1 lists the storage of the three formats; dense counts n*n values
    per system and ELL counts its padded k*n value slots per system.
    """
    if fmt == "dense":
        return num_batch * n * n
    if fmt == "csr":
        return num_batch * nnz + (n + 1) + nnz
    if fmt == "ell":
        return num_batch * ell_k * n + ell_k * n
    raise ValueError(fmt)


# --------------------------------------------------------------------------
# the named workloads
# --------------------------------------------------------------------------

@dataclass
class Workload:
    name: str
    pattern: Pattern
    csr_values: np.ndarray
    b: np.ndarray
    x0: np.ndarray
    meta: dict = field(default_factory=dict)

    @property
    def num_batch(self) -> int:
        return int(self.b.shape[0])

    def matrix(self, fmt: str = "csr") -> BatchMatrix:
        return make_batch(self.pattern, self.csr_values, fmt)


def _rng(index: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(SEED_BASE + index))


def tiny_tridiagonal(num_batch: int = 64, n: int = 32) -> Workload:
    """64 nonsymmetric tridiagonal systems, n=32, dominance factor 1+U[0.05,0.5]."""
    rng = _rng(0)
    pat = stencil_pattern("1d3", n)
    vals = stencil_values(pat, num_batch, rng, 0.05, 0.5)
    b = rng.uniform(-1.0, 1.0, (num_batch, n))
    return Workload(f"tridiag_n{n}_B{num_batch}", pat, vals, b, np.zeros_like(b))


def plain_at_scale(num_batch: int = 65536, grid: int = 12, symmetric: bool = False) -> Workload:
    """5-point stencil on a grid x grid mesh (n=144 at 12x12), factor 1+U[0.05,0.5].

    symmetric=True gives the symmetrised copy used for CG (same draws).
    """
    rng = _rng(1)
    pat = stencil_pattern("2d5", grid, grid)
    vals = stencil_values(pat, num_batch, rng, 0.05, 0.5, symmetric=symmetric)
    b = rng.uniform(-1.0, 1.0, (num_batch, pat.n))
    tag = "sym_" if symmetric else ""
    return Workload(f"{tag}stencil2d5_{grid}x{grid}_B{num_batch}", pat, vals, b, np.zeros_like(b))


def mixed_precision(num_batch: int = 16384, grid: int = 32) -> Workload:
    """9-point stencil on a grid x grid mesh (n=1024 at 32x32), factor 1+U[0.01,0.1]."""
    rng = _rng(2)
    pat = stencil_pattern("2d9", grid, grid)
    vals = stencil_values(pat, num_batch, rng, 0.01, 0.1)
    b = rng.uniform(-1.0, 1.0, (num_batch, pat.n))
    return Workload(f"stencil2d9_{grid}x{grid}_B{num_batch}", pat, vals, b, np.zeros_like(b))


# --------------------------------------------------------------------------
# uneven batch: many patterns, log-uniform sizes
# --------------------------------------------------------------------------

@dataclass
class VarBatch:
    """Systems of uneven size: a pool of CSR patterns plus per-system records.

    sys_pattern[i] names system i's pattern; its values start at
    values[val_off[i]] (nnz of its pattern) and its vectors at b[vec_off[i]]
    (n of its pattern).
    """

    patterns: list
    sys_pattern: np.ndarray  # int32 [B]
    val_off: np.ndarray      # int64 [B]
    vec_off: np.ndarray      # int64 [B]
    values: np.ndarray       # float64 [sum nnz]
    b: np.ndarray            # float64 [sum n]
    x0: np.ndarray           # float64 [sum n]
    name: str = ""

    @property
    def num_batch(self) -> int:
        return int(self.sys_pattern.shape[0])

    def sys_n(self) -> np.ndarray:
        ns = np.array([p.n for p in self.patterns], dtype=np.int32)
        return ns[self.sys_pattern]

    def sys_nnz(self) -> np.ndarray:
        nz = np.array([p.nnz for p in self.patterns], dtype=np.int32)
        return nz[self.sys_pattern]

    def pools(self):
        """Concatenated pattern arrays: (pat_n, pat_nnz, rp_off, ci_off, row_ptrs, col_idxs)."""
        pat_n = np.array([p.n for p in self.patterns], dtype=np.int32)
        pat_nnz = np.array([p.nnz for p in self.patterns], dtype=np.int32)
        rp_off = np.zeros(len(self.patterns), dtype=np.int64)
        ci_off = np.zeros(len(self.patterns), dtype=np.int64)
        rps, cis = [], []
        a = c = 0
        for i, p in enumerate(self.patterns):
            rp_off[i], ci_off[i] = a, c
            rps.append(p.row_ptrs)
            cis.append(p.col_idxs)
            a += p.n + 1
            c += p.nnz
        return (pat_n, pat_nnz, rp_off, ci_off,
                np.concatenate(rps).astype(np.int32), np.concatenate(cis).astype(np.int32))

    def slice(self, begin: int, end: int) -> "VarBatch":
        """Systems [begin, end) as a batch of their own (views of the values
        and vectors, offsets re-based; the pattern pool is kept whole)."""
        if not 0 <= begin <= end <= self.num_batch:
            raise ValueError("need 0 <= begin <= end <= num_batch")
        nnz, nn = self.sys_nnz().astype(np.int64), self.sys_n().astype(np.int64)
        v0 = int(self.val_off[begin]) if begin < self.num_batch else self.values.size
        x0 = int(self.vec_off[begin]) if begin < self.num_batch else self.b.size
        v1 = v0 + int(nnz[begin:end].sum())
        x1 = x0 + int(nn[begin:end].sum())
        return VarBatch(self.patterns, self.sys_pattern[begin:end], self.val_off[begin:end] - v0,
                        self.vec_off[begin:end] - x0, self.values[v0:v1], self.b[x0:x1], self.x0[x0:x1],
                        f"{self.name}[{begin}:{end}]")

    def system(self, i: int):
        """(pattern, values[nnz], b[n], x0[n]) of system i (views)."""
        p = self.patterns[int(self.sys_pattern[i])]
        vo, xo = int(self.val_off[i]), int(self.vec_off[i])
        return p, self.values[vo:vo + p.nnz], self.b[xo:xo + p.n], self.x0[xo:xo + p.n]


def uneven(num_batch: int = 100000, n_min: int = 16, n_max: int = 1024) -> VarBatch:
    """n log-uniform in [n_min, n_max] over 1D 3-pt, 2D 5-pt and 2D 9-pt stencils.

    1D uses n as drawn; 2D uses kx = round(sqrt(n)), ky = max(1, round(n/kx)),
    clipped so kx*ky stays within [n_min, n_max]. One pattern per distinct
    (stencil, kx, ky). Value recipe of the tiny tridiagonal batch.
    """
    rng = _rng(3)
    n_draw = np.rint(np.exp(rng.uniform(math.log(n_min), math.log(n_max), num_batch))).astype(np.int64)
    kinds = np.array(["1d3", "2d5", "2d9"])
    kind_draw = rng.integers(0, 3, num_batch)
    keys = []
    for n, kd in zip(n_draw, kind_draw):
        kind = kinds[kd]
        if kind == "1d3":
            keys.append((kind, int(n), 1))
            continue
        kx = int(round(math.sqrt(n)))
        ky = max(1, int(round(n / kx)))
        while kx * ky > n_max:
            ky -= 1
        while kx * ky < n_min:
            ky += 1
        keys.append((kind, kx, ky))
    uniq = sorted(set(keys))
    index = {k: i for i, k in enumerate(uniq)}
    patterns = [stencil_pattern(k, kx, ky) for (k, kx, ky) in uniq]
    sys_pattern = np.array([index[k] for k in keys], dtype=np.int32)
    nnz = np.array([p.nnz for p in patterns], dtype=np.int64)[sys_pattern]
    nn = np.array([p.n for p in patterns], dtype=np.int64)[sys_pattern]
    val_off = np.zeros(num_batch, dtype=np.int64)
    vec_off = np.zeros(num_batch, dtype=np.int64)
    val_off[1:] = np.cumsum(nnz)[:-1]
    vec_off[1:] = np.cumsum(nn)[:-1]
    values = np.empty(int(nnz.sum()), dtype=np.float64)
    b = np.empty(int(nn.sum()), dtype=np.float64)
    for pi, p in enumerate(patterns):
        members = np.nonzero(sys_pattern == pi)[0]
        sub = np.random.Generator(np.random.PCG64(SEED_BASE + 3 + 1000 * (pi + 1)))
        v = stencil_values(p, len(members), sub, 0.05, 0.5)
        bb = sub.uniform(-1.0, 1.0, (len(members), p.n))
        vidx = val_off[members][:, None] + np.arange(p.nnz)[None, :]
        bidx = vec_off[members][:, None] + np.arange(p.n)[None, :]
        values[vidx] = v
        b[bidx] = bb
    return VarBatch(patterns, sys_pattern, val_off, vec_off, values, b, np.zeros_like(b),
                    name=f"uneven_n{n_min}-{n_max}_B{num_batch}")


# --------------------------------------------------------------------------
# time-stepped batch for the learned initial guess
# --------------------------------------------------------------------------

@dataclass
class TimeSeries:
    """A_i(t) = A_i + 0.01 t B_i, b_i(t) = b_i + 0.01 t c_i on one shared pattern."""

    pattern: Pattern
    A: np.ndarray   # [B, nnz]
    Bn: np.ndarray  # [B, nnz] diagonally dominant noise, same pattern
    b: np.ndarray   # [B, n]
    c: np.ndarray   # [B, n]
    steps: int

    @property
    def num_batch(self) -> int:
        return int(self.b.shape[0])

    def values_at(self, t: int) -> np.ndarray:
        return self.A + (0.01 * t) * self.Bn

    def rhs_at(self, t: int) -> np.ndarray:
        return self.b + (0.01 * t) * self.c


def time_stepped(num_batch: int = 16384, steps: int = 256, grid: int = 12) -> TimeSeries:
    rng = _rng(4)
    pat = stencil_pattern("2d5", grid, grid)
    A = stencil_values(pat, num_batch, rng, 0.05, 0.5)
    b = rng.uniform(-1.0, 1.0, (num_batch, pat.n))
    c = rng.uniform(-1.0, 1.0, (num_batch, pat.n))
    noise = np.random.Generator(np.random.PCG64(SEED_BASE + 4 + 7919))
    Bn = stencil_values(pat, num_batch, noise, 0.05, 0.5)
    return TimeSeries(pat, A, Bn, b, c, steps)


# --------------------------------------------------------------------------
# PeleLM-shaped batches (Table "Reference for data inputs": n, nonzeros per
# matrix, number of unique matrices; the matrices themselves are not
# available, so random patterns of the same size and density stand in)
# --------------------------------------------------------------------------

MECHANISMS = {
    # name: (unique matrices, n, nnz per matrix)
    "drm19": (67, 22, 438),
    "gri12": (73, 33, 978),
    "gri30": (90, 54, 2560),
    "dodecane_lu": (78, 54, 2332),
    "isooctane": (72, 144, 6135),
}


def random_pattern(n: int, nnz: int, rng: np.random.Generator) -> Pattern:
    """Full diagonal plus nnz - n off-diagonal entries at random positions,
    placed in mirrored pairs (structurally symmetric, as reaction Jacobians of
    a species set nearly are) with one unpaired entry when the count is odd."""
    off = nnz - n
    if off < 0 or off > n * (n - 1):
        raise ValueError("nnz out of range")
    pairs = [(i, j) for i in range(n) for j in range(i + 1, n)]
    chosen = rng.choice(len(pairs), off // 2, replace=False)
    entries = {(i, i) for i in range(n)}
    for c in chosen:
        i, j = pairs[c]
        entries.add((i, j))
        entries.add((j, i))
    if off % 2:
        free = [(j, i) for (i, j) in pairs if (j, i) not in entries]
        entries.add(free[rng.integers(len(free))])
    rows = [sorted(c for (r, c) in entries if r == i) for i in range(n)]
    row_ptrs = np.zeros(n + 1, dtype=np.int32)
    row_ptrs[1:] = np.cumsum([len(r) for r in rows])
    col_idxs = np.array([c for r in rows for c in r], dtype=np.int32)
    return Pattern(n, row_ptrs, col_idxs, "random")


def general_values(pat: Pattern, count: int, rng: np.random.Generator, diag_lo: float,
                   diag_hi: float) -> np.ndarray:
    """Values [count, nnz]: every off-diagonal entry U[-1, 0] * (1 + U[-0.1, 0.1]),
    diagonal = sum |off-diagonal| * (1 + U[lo, hi])."""
    rows = np.repeat(np.arange(pat.n), np.diff(pat.row_ptrs))
    diag = rows == pat.col_idxs
    v = rng.uniform(-1.0, 0.0, (count, pat.nnz)) * (1.0 + rng.uniform(-0.1, 0.1, (count, pat.nnz)))
    v[:, diag] = 0.0
    offsum = np.add.reduceat(np.abs(v), pat.row_ptrs[:-1].astype(np.int64), axis=1)
    v[:, diag] = offsum * (1.0 + rng.uniform(diag_lo, diag_hi, (count, pat.n)))
    return v


def pele_like(mechanism: str, num_batch: int = 131072) -> Workload:
    """A batch of num_batch systems made of the mechanism's unique matrices
    repeated in turn (system i uses matrix i mod U, as the paper replicates a
    few cells' matrices to emulate a larger mesh); b ~ U[-1, 1] per system."""
    U, n, nnz = MECHANISMS[mechanism]
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + 5 + list(MECHANISMS).index(mechanism)))
    pat = random_pattern(n, nnz, rng)
    uniq = general_values(pat, U, rng, 0.05, 0.5)
    vals = uniq[np.arange(num_batch) % U]
    b = rng.uniform(-1.0, 1.0, (num_batch, n))
    return Workload(f"{mechanism}_n{n}_nnz{nnz}_B{num_batch}", pat, vals, b, np.zeros_like(b),
                    meta={"unique": U})


def spd_tridiagonal(num_batch: int, n: int) -> Workload:
    """The 3-point-stencil SPD batch of the scaling study (Sec. 5.1): symmetric
    tridiagonal, strictly diagonally dominant, positive diagonal."""
    rng = _rng(6)
    pat = stencil_pattern("1d3", n)
    vals = stencil_values(pat, num_batch, rng, 0.05, 0.5, symmetric=True)
    b = rng.uniform(-1.0, 1.0, (num_batch, n))
    return Workload(f"spd3pt_n{n}_B{num_batch}", pat, vals, b, np.zeros_like(b))
