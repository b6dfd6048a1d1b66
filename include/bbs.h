/*
 * bbs.h - batched sparse iterative solvers for GB300 (sm_103a), C ABI.
 *
 * Solves many small independent systems A_i x_i = b_i, i = 0..B-1, that share
 * one sparsity pattern (Sec. 3.1), one CUDA thread block per system (Sec.
 * 3.2), all systems in one kernel launch (Sec. 3.4). Each system is monitored
 * and stops on its own residual test (Sec. 2.1); a per-system log records
 * iterations, final residual and status.
 *
 * Conventions for every call:
 *   - Pointers named in a struct or argument as DEVICE point to device memory
 *     owned by the caller; the library never frees them. HOST pointers point
 *     to host memory (pinned memory gives full copy bandwidth).
 *   - Argument errors are reported before any launch with a bbs_status and a
 *     message from bbs_last_error(); nothing is written then.
 *   - Numerical trouble in one system is not an API error: it is recorded in
 *     that system's log status (bbs_sys_status) and no other system is
 *     affected.
 *   - Calls taking a stream are asynchronous on it; the *_host calls return
 *     after the results are back in host memory.
 *   - Indices are 0-based int32; columns are sorted ascending within a row.
 *   - Every device loop is bounded by the iteration caps given in
 *     bbs_options, so no kernel can run forever.
 */
#ifndef BBS_H
#define BBS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    BBS_OK = 0,
    BBS_ERR_INVALID_ARG = 1, /* a size, pointer, enum or option is out of range */
    BBS_ERR_UNSUPPORTED = 2, /* valid but not provided (e.g. n too large)       */
    BBS_ERR_CUDA = 3,        /* a CUDA runtime call failed (message has detail) */
    BBS_ERR_NO_MEMORY = 4    /* workspace too small or a library buffer failed  */
} bbs_status;

/* Batch matrix formats, Sec. 3.1 and Table "Batched feature support". */
typedef enum { BBS_FMT_CSR = 0, BBS_FMT_ELL = 1, BBS_FMT_DENSE = 2 } bbs_format;
/* Solvers, Table "Batched feature support": BatchBicgstab, BatchCg (Alg. 1),
 * BatchGmres (restarted). */
typedef enum { BBS_SOLVER_BICGSTAB = 0, BBS_SOLVER_CG = 1, BBS_SOLVER_GMRES = 2 } bbs_solver;
/* Preconditioners (Table "Batched feature support"): none; scalar
 * BatchJacobi M = D^-1 (1 for a zero or missing diagonal entry); BatchIlu
 * read as ILU(0): A ~ L U with unit lower L and upper U on A's pattern (zero
 * fill-in, a zero pivot replaced by 1), applied by forward and backward
 * triangular solves (BatchTrsv). ILU(0) preconditions FP64 BiCGSTAB on
 * BatchCsr; the factors of a system must fit in shared memory (about 27,000
 * nonzeros). */
typedef enum { BBS_PREC_NONE = 0, BBS_PREC_JACOBI = 1, BBS_PREC_ILU0 = 2 } bbs_precond;
/* Stopping criteria, Table "Batched feature support": stop when
 * ||b - A x||_2 <= tol (absolute) or <= tol * ||b||_2 (relative). */
typedef enum { BBS_TOL_ABSOLUTE = 0, BBS_TOL_RELATIVE = 1 } bbs_tol_type;
/* FP64 throughout, or FP32 inner BiCGSTAB inside FP64 iterative refinement
 * (residual, update and exit test in FP64). */
typedef enum { BBS_PRECISION_FP64 = 0, BBS_PRECISION_MIXED_IR = 1 } bbs_precision;
/* Per-system outcome written to bbs_log.status. */
typedef enum {
    BBS_SYS_CONVERGED = 0, /* true residual passed the test                      */
    BBS_SYS_MAX_ITER = 1,  /* iteration cap reached (or confirmation restarts ran out) */
    BBS_SYS_BREAKDOWN = 2, /* an exact-zero denominator stopped the method       */
    BBS_SYS_NAN = 3        /* a non-finite scalar appeared                       */
} bbs_sys_status;

/* A batch of matrices sharing one pattern (Sec. 3.1). All pointers DEVICE.
 *   CSR:   row_ptrs [n+1], col_idxs [nnz], values [num_batch * nnz]
 *   ELL:   col_idxs [ell_k * n] column-major (slot j of row r at j*n + r,
 *          padding column -1), values [num_batch * ell_k * n] same order,
 *          padding value 0; row_ptrs unused (may be NULL)
 *   DENSE: values [num_batch * n * n] row-major; row_ptrs/col_idxs unused
 * System i's values start at values + i * (nnz | ell_k*n | n*n).
 * values_f32: optional FP32 copy in the same layout, used by the mixed mode.
 * With NULL, each block rounds its system's FP64 values to FP32 (to nearest)
 * as it stages them into shared memory; values too large to stage are
 * converted into the workspace inside the call instead. Either way the
 * results equal those with a copy rounded to nearest. */
typedef struct {
    int32_t fmt; /* bbs_format */
    int32_t num_batch;
    int32_t n;
    int32_t nnz;   /* CSR: pattern nonzeros; ELL/DENSE: informational */
    int32_t ell_k; /* ELL: width (max nonzeros per row). CSR: 0, or the
                      largest number of nonzeros in any row; with it, small
                      systems can run packed several to a warp (their values
                      staged in ELL order). A packed CSR solve whose pattern
                      has a row longer than ell_k returns
                      BBS_ERR_INVALID_ARG before any launch. The first such
                      solve with a given row_ptrs address (and n, nnz,
                      ell_k) reads the row pointers back on its stream and
                      waits for them; the handle remembers the answer for
                      the next 16 patterns. A pattern rewritten in place
                      under a remembered address is caught on the device
                      instead: every system of the call reports
                      BBS_SYS_NAN. DENSE: ignored. */
    const int32_t *row_ptrs;
    const int32_t *col_idxs;
    const double *values;
    const float *values_f32;
} bbs_batch_matrix;

typedef struct {
    int32_t solver;   /* bbs_solver */
    int32_t precond;  /* bbs_precond */
    int32_t tol_type; /* bbs_tol_type */
    int32_t max_iters;     /* FP64: iteration cap per system (>= 0);
                              mixed: cap of each inner FP32 solve (>= 1) */
    double tol;            /* > 0 */
    int32_t gmres_restart; /* GMRES restart length m, 1..32 */
    int32_t precision;     /* bbs_precision; mixed requires BiCGSTAB */
    double inner_tol;      /* mixed: relative tolerance of each inner solve, (0,1) */
    int32_t max_outer;     /* mixed: cap on refinement steps (>= 0) */
    int32_t threads_per_system; /* 0: library choice; 4, 8 or 16: packed
                                   systems, 32 / threads of them per warp in
                                   lockstep (FP64 BiCGSTAB with Jacobi, none
                                   or ILU(0), CG or GMRES with Jacobi or none;
                                   staged values; CSR needs ell_k;
                                   ceil(n / threads) <= 10); else a multiple
                                   of 32 in [32, 1024] with
                                   ceil(n / threads) <= 8. The library choice
                                   packs systems of n <= 160 rows when enough
                                   of them fit in an SM's shared memory. */
    int32_t values_in_smem;     /* 0: library choice, 1: stage each system's
                                   values in shared memory, -1: read them from
                                   global memory in every SpMV */
    int32_t reserved;
} bbs_options;

/* Per-system log, DEVICE arrays of length num_batch (HOST for *_host calls).
 *   iters:       iterations taken (FP64 and varsize: Krylov iterations; a
 *                half-step exit of BiCGSTAB counts as one; GMRES counts
 *                Arnoldi steps; mixed: refinement steps)
 *   rel_res:     ||b - A x||_2 / ||b||_2 of the returned x (0 when b = 0)
 *   status:      bbs_sys_status
 *   inner_iters: mixed only, total inner FP32 iterations (may be NULL)   */
typedef struct {
    int32_t *iters;
    double *rel_res;
    int32_t *status;
    int32_t *inner_iters;
} bbs_log;

typedef struct bbs_handle bbs_handle;

/* Fill *opts with the defaults: BiCGSTAB, Jacobi, relative tol 1e-10,
 * max_iters 500, GMRES restart 10, FP64, inner_tol 1e-4, max_outer 30,
 * library-chosen launch shape. Host only; cannot fail for non-NULL opts. */
bbs_status bbs_default_options(bbs_options *opts);

/* Create a handle bound to CUDA device `device` (queries its SM count and
 * shared-memory limit). The handle owns only the buffers of the *_host calls. */
bbs_status bbs_create(bbs_handle **handle, int device);
/* Release the handle and the buffers it owns. NULL is accepted. */
bbs_status bbs_destroy(bbs_handle *handle);

/* Bytes of DEVICE workspace bbs_solve needs for this problem (0 is possible).
 * Workspace use: the FP32 copy of the values in mixed mode when values_f32
 * is NULL and the values are not staged in shared memory, the GMRES Krylov
 * basis ((restart + 1) * n_pad doubles per system; always for packed
 * systems, else when it does not fit in shared memory), the
 * ILU(0) level schedule of the shared pattern, and for packed systems on CSR
 * the pattern as an ELL column table (2 * ell_k * n int32 + 256 bytes). */
bbs_status bbs_workspace_size(const bbs_handle *handle, const bbs_batch_matrix *A,
                              const bbs_options *opts, size_t *bytes);

/* The launch bbs_solve makes for (A, opts) on this handle's device (the
 * multi-level dispatch of Sec. 3.3 made visible). Host-only: no GPU work,
 * A's arrays are not read. `kernel` points at a static string naming the
 * solver kernel: "bicgstab_packed_kernel", "cg_packed_kernel", "gmres_packed_kernel",
 * "bicgstab_ilu_packed_kernel", "bicgstab_folded_kernel",
 * "bicgstab_kernel", "bicgstab_ilu_kernel", "cg_kernel", "gmres_kernel" or
 * "refine_kernel". threads_per_system is the lanes of one system (4, 8 or
 * 16 when systems are packed 32 / lanes to a warp). launches counts every
 * kernel of one bbs_solve (an FP32 conversion, an ILU(0) analysis or the
 * CSR column table of packed systems runs before the solver kernel). Errors
 * as bbs_solve's argument checks. */
typedef struct bbs_launch_info {
    const char *kernel;
    int32_t grid;               /* blocks of the solver kernel */
    int32_t block;              /* threads per block */
    int32_t threads_per_system;
    int32_t rows_per_thread;    /* R: rows each thread owns */
    int64_t smem_bytes;         /* dynamic shared memory per block */
    int32_t values_staged;      /* 1: the values are staged in shared memory */
    int32_t launches;
} bbs_launch_info;

bbs_status bbs_describe(const bbs_handle *handle, const bbs_batch_matrix *A, const bbs_options *opts,
                        bbs_launch_info *info);

/* Check the shared pattern of A on the device, which the solvers trust:
 *   CSR:   row_ptrs[0] = 0, row_ptrs non-decreasing, row_ptrs[n] = nnz;
 *          columns in [0, n) and strictly increasing within each row; with
 *          ell_k > 0, no row longer than ell_k;
 *   ELL:   columns in [-1, n), strictly increasing within each row, and
 *          padding (-1) only after the last stored entry of the row;
 *   DENSE: nothing to check.
 * *bad_rows receives the number of rows that break a rule (0: the pattern
 * is valid). Reads only row_ptrs[0..n] and col_idxs[0..nnz) (CSR) or
 * col_idxs[0..ell_k*n) (ELL), whatever they hold. Synchronous. Values are
 * not inspected: non-finite values are reported per system (BBS_SYS_NAN). */
bbs_status bbs_check_pattern(bbs_handle *handle, const bbs_batch_matrix *A, int32_t *bad_rows);

/* Solve every system of the batch (Sec. 3.2-3.4: one thread block per system,
 * one launch for the batch; Sec. 2.1: x holds the initial guess on entry and
 * the solution on return). b, x: DEVICE [num_batch * n], system i at i*n.
 * log: DEVICE arrays (see bbs_log). workspace: DEVICE, >= bbs_workspace_size
 * bytes, 256-byte aligned, may be NULL when that size is 0. stream: a
 * cudaStream_t (NULL = legacy default stream). Asynchronous. */
bbs_status bbs_solve(bbs_handle *handle, const bbs_batch_matrix *A, const double *b, double *x,
                     const bbs_options *opts, const bbs_log *log, void *workspace,
                     size_t workspace_bytes, void *stream);

/* Same as bbs_solve with every array in HOST memory: A's pointers, b, x (in:
 * x0, out: x) and log are HOST pointers. The library copies the inputs to
 * device buffers owned by the handle, solves, copies x and the log back and
 * waits for completion. The batch goes in chunks of about 128 MB of input
 * (at least 2,048 systems each), led by a quarter and a half chunk. The
 * inputs are copied in on a stream of their own, chunk after chunk; each
 * chunk's solve waits for its copy only, and the solves and the copies out
 * alternate between two more streams, so copies overlap solves and
 * consecutive solves overlap each other (with page-locked host memory);
 * results are the same as one bbs_solve of the whole batch. */
bbs_status bbs_solve_host(bbs_handle *handle, const bbs_batch_matrix *A_host,
                          const double *b_host, double *x_host, const bbs_options *opts,
                          const bbs_log *log_host);

/* The chunks bbs_solve_host cuts a batch into (host only, no GPU): for
 * num_batch systems of input_bytes_per_system bytes of input each (values,
 * b and x0), writes chunk c as systems [first[c], first[c] + count[c]) for
 * up to max_chunks chunks, in order and covering the batch once, and
 * returns the number of chunks: 0 for an empty batch, -1 when an argument
 * is negative or NULL or more than max_chunks chunks would be needed (16
 * always suffice). */
int32_t bbs_host_chunk_plan(int64_t num_batch, int64_t input_bytes_per_system, int64_t *first,
                            int64_t *count, int32_t max_chunks);

/* bbs_solve without any caller workspace and without allocating, for callers
 * that cannot call cudaMalloc: hosts whose device memory is already reserved
 * by another allocator (a framework's caching pool, a server's arena, a fixed
 * budget), and loops that must not wait on the allocator (cudaFree
 * synchronises the device). The paper has no counterpart: it is an interface
 * addition of this library.
 * Arguments and results are those of bbs_solve (all DEVICE pointers, x in/out,
 * asynchronous on `stream`); the results are bit for bit those of bbs_solve
 * with a workspace. The scratch bbs_solve would take from the workspace (the
 * FP32 copy of the values in mixed mode when they are not staged, the GMRES
 * basis when it does not fit in shared memory) comes instead from one static
 * 64 MiB device array inside the library, which every GPU that loads the
 * library keeps until the process exits. A batch whose scratch exceeds 64 MiB
 * is solved in consecutive chunks of systems on `stream`; a single system
 * needing more than 64 MiB is rejected with BBS_ERR_UNSUPPORTED. The first
 * call on a device looks up the array's device address, so make that call
 * before any stream capture. Every call shares the one array, which keeps the
 * last call's contents: calls that overlap on the GPU (other streams, other
 * host threads) race on it and must be serialised by the caller. Calls no
 * cudaMalloc, cudaFree or allocating library routine. */
bbs_status bbs_solve_noalloc(bbs_handle *handle, const bbs_batch_matrix *A, const double *b,
                             double *x, const bbs_options *opts, const bbs_log *log,
                             void *stream);

/* ------------------------------------------------------------------------
 * Uneven batches: systems of different sizes and patterns in one persistent,
 * graph-captured launch. The paper's batch shares one pattern (Sec. 3.1) and
 * tunes launch thresholds per device experimentally (Sec. 3.6); this
 * extension keeps one thread team per system but lets the team size follow
 * the system size, chosen per size bucket by a measured autotuner.
 * ------------------------------------------------------------------------ */

/* Systems of uneven size in BatchCsr: a pool of patterns and one record per
 * system. All pointers DEVICE. System i uses pattern sys_pattern[i]: its
 * row_ptrs start at row_ptrs + pat_rp_off[p] (n+1 entries, values relative to
 * the pattern's first entry), its col_idxs at col_idxs + pat_ci_off[p]; its
 * values start at values + val_off[i] (pat_nnz[p] entries) and its vectors
 * at b + vec_off[i], x + vec_off[i] (pat_n[p] entries). */
typedef struct {
    int32_t num_batch;
    int32_t num_patterns;
    const int32_t *pat_n;
    const int32_t *pat_nnz;
    const int64_t *pat_rp_off;
    const int64_t *pat_ci_off;
    const int32_t *row_ptrs;
    const int32_t *col_idxs;
    const int32_t *sys_pattern;
    const int64_t *val_off;
    const int64_t *vec_off;
    const double *values;
} bbs_var_batch;

/* HOST copies of the metadata the planner reads: pat_n and pat_nnz
 * [num_patterns], sys_pattern [num_batch]. */
typedef struct {
    const int32_t *pat_n;
    const int32_t *pat_nnz;
    const int32_t *sys_pattern;
} bbs_var_host_info;

/* Launch choices for an uneven batch. Systems fall in size buckets
 * (bucket b holds n <= bucket_max_n[b], ascending); each bucket has the number
 * of warps that solve one of its systems (1, 2, 4, 8 or 16; at most
 * block_warps), whether its systems' values are staged in shared memory, and
 * whether its small systems are packed (pack[b] = 1: a system of at most 160
 * rows whose group fits shared memory is solved by 4, 8 or 16 lanes, with
 * 8, 4 or 2 systems per warp in lockstep, as bbs_solve packs uniform batches;
 * 0: one team per system), and which of its large systems run as wide teams
 * (wide[b], BiCGSTAB with Jacobi only, a bit set: 1 = systems whose rows hold
 * at most 4 stored values on average, 2 = the others, 3 = both, 0 = none. Such
 * a system, if it needs more than 8 rows per thread on the fewest warps that
 * hold it in at most 16 rows per thread (1, 2 or 4 warps), is solved by that
 * many warps, one block per system, values staged, in a launch of its own,
 * where such blocks still leave an SM 8 warps; the others run in the
 * persistent launch). block_warps is 8 (up to 8 rows per thread) or 16 (up to 4 rows per
 * thread). The planner lowers a bucket's warps to those of the next larger
 * bucket if they exceed them and raises them to the minimum its rows need. */
typedef struct {
    int32_t num_buckets; /* 1..8 */
    int32_t bucket_max_n[8];
    int32_t team_warps[8];
    int32_t stage_values[8];
    int32_t pack[8];
    int32_t wide[8];
    int32_t block_warps;
    int32_t reserved;
} bbs_var_tuning;

typedef struct bbs_var_plan bbs_var_plan;

/* Default tuning: power-of-two buckets up to max_n, one warp per 5 rows per
 * thread (as bbs_default_block_size), values streamed, small systems packed,
 * wide teams for the sparse rows (wide = 1) of the buckets above 512 rows,
 * 8-warp blocks. Host only. */
bbs_status bbs_var_default_tuning(int32_t max_n, bbs_var_tuning *tuning);

/* Plan the persistent solve of `batch` (FP64, BiCGSTAB or CG, Jacobi or
 * none). The systems that run packed (see bbs_var_tuning.pack) are grouped by
 * (lanes per system, rows per lane), one launch per group, and so are the
 * wide teams (bbs_var_tuning.wide) by (warps, rows per thread); the planner reads
 * their patterns' row pointers (rejecting, with BBS_ERR_INVALID_ARG, row
 * pointers that do not ascend within [0, nnz]) and builds an ELL column table
 * of each such pattern on the device. The other systems are ordered longest
 * first and grouped in segments of equal team size for one persistent launch
 * whose grid fills every SM. The CUDA graph holds "reset the work counters ->
 * the persistent launch" and, beside it, the packed and wide launches. Allocates the
 * plan's own device buffers (system order, counters, tables). The patterns
 * must not change while the plan lives (values, b and x may). tuning NULL =
 * default tuning. */
bbs_status bbs_var_plan_create(bbs_handle *handle, const bbs_var_batch *batch,
                               const bbs_var_host_info *host, const bbs_options *opts,
                               const bbs_var_tuning *tuning, bbs_var_plan **plan);

/* Run a plan: one graph launch on `stream`. b, x (in: x0, out: solution) are
 * DEVICE arrays laid out by vec_off; log is DEVICE (inner_iters unused).
 * Asynchronous. Plans of the same handle must not run concurrently. */
bbs_status bbs_var_solve(bbs_var_plan *plan, const double *b, double *x, const bbs_log *log,
                         void *stream);

/* What a plan runs: systems solved by teams in the persistent launch, systems
 * solved packed and the number of packed launches, the persistent grid (0 when
 * every system runs packed or wide), and systems solved by wide teams and the
 * number of wide launches. Host only. */
typedef struct {
    int32_t team_systems;
    int32_t packed_systems;
    int32_t packed_launches;
    int32_t persistent_grid;
    int32_t wide_systems;
    int32_t wide_launches;
} bbs_var_plan_desc;

bbs_status bbs_var_plan_describe(const bbs_var_plan *plan, bbs_var_plan_desc *desc);

/* Release a plan (waits for its graph to finish). NULL is accepted. */
bbs_status bbs_var_plan_destroy(bbs_var_plan *plan);

/* Autotuner: for every size bucket that holds systems, time the persistent
 * kernel on a sample of the bucket's systems (at least `sample`, and at least
 * four times the systems the GPU holds at once, so that each trial measures
 * throughput; all of them when the bucket is smaller) for each team
 * size and staging choice (and both block shapes), then packing and wide
 * teams where the bucket has such systems, and write the fastest choices to
 * *tuning (packing and wide teams keep the default tuning's choice unless the
 * other one times at least 3 % faster; then the sample of the whole batch
 * decides whether to pack the small systems that buckets timed alone left
 * unpacked, and whether to keep the wide teams, each by a 1 % margin). b and x0 are DEVICE arrays of the batch; x0 is not
 * modified (trials run on a private copy). Synchronous; allocates and frees
 * its own scratch. */
bbs_status bbs_var_tune(bbs_handle *handle, const bbs_var_batch *batch,
                        const bbs_var_host_info *host, const double *b, const double *x0,
                        const bbs_options *opts, int32_t sample, bbs_var_tuning *tuning);

/* ------------------------------------------------------------------------
 * Learned initial guess for time-stepped batches (an extension: the paper
 * motivates it with the solver's use of an initial guess, Sec. 2.1). A small
 * MLP predicts each system's change of solution from its diagonal, its
 * right-hand side and its previous solution: 3n standardised inputs ->
 * hidden -> hidden -> hidden -> n, GELU (tanh form) after each hidden layer,
 * BF16 tensor-core GEMMs with FP32 accumulation, FP32 master weights, Adam
 * (beta 0.9 / 0.999, eps 1e-8), mean-squared-error loss on the standardised
 * change. The solver itself is unchanged: it still iterates to its tolerance
 * from whatever guess it is given.
 * Parameter layout (FP32, flat): W1 b1 W2 b2 W3 b3 W4 b4, W_l row-major
 * [out, in] (y = x W^T + b); W1 is [hidden, 3n], W4 is [n, hidden].
 * Feature rows (BF16, stored as uint16_t) have ceil(3n/64)*64 columns:
 * standardised diag(A) (n), b (n), x_prev (n), then zeros.
 * ------------------------------------------------------------------------ */
typedef struct bbs_mlp bbs_mlp;

/* Tensor-core paths of the network's GEMMs: tcgen05 MMAs with the FP32
 * accumulator in tensor memory (K-tiles of 64), or warp-level mma.sync. */
typedef enum { BBS_GEMM_MMA_SYNC = 0, BBS_GEMM_TCGEN05 = 1 } bbs_gemm_kind;

/* Create a network for systems of n rows (1..2048) with `hidden` units (a
 * multiple of 64, 64..4096) and minibatches of up to max_batch rows (a
 * multiple of 64). Weights are drawn from U(-1/sqrt(in), 1/sqrt(in)) by a
 * counter-based hash of `seed` (output layer scaled by 0.1), biases zero.
 * Allocates all its device buffers here. */
bbs_status bbs_mlp_create(bbs_handle *handle, int32_t n, int32_t hidden, uint64_t seed,
                          int32_t max_batch, bbs_mlp **mlp);
bbs_status bbs_mlp_destroy(bbs_mlp *mlp);
/* Number of FP32 parameters (length of the flat layout). */
bbs_status bbs_mlp_param_count(const bbs_mlp *mlp, int64_t *count);
/* Copy the FP32 master parameters to / from a DEVICE array (set also
 * refreshes the BF16 copies). Asynchronous on stream. */
bbs_status bbs_mlp_get_params(bbs_mlp *mlp, float *params, void *stream);
bbs_status bbs_mlp_set_params(bbs_mlp *mlp, const float *params, void *stream);
/* Accumulate the input and target moments of one time step: A (DEVICE
 * BatchCsr with this network's n), b, x_prev, x_next (DEVICE, num_batch*n). */
bbs_status bbs_mlp_observe(bbs_mlp *mlp, const bbs_batch_matrix *A, const double *b,
                           const double *x_prev, const double *x_next, void *stream);
/* Turn the accumulated moments into the standardisation (mean, std). */
bbs_status bbs_mlp_finalize_stats(bbs_mlp *mlp, void *stream);
/* Standardised feature rows [num_batch, ceil(3n/64)*64] (BF16) and, when
 * x_next is given, standardised targets [num_batch, n] (FP32), DEVICE. */
bbs_status bbs_mlp_make_samples(bbs_mlp *mlp, const bbs_batch_matrix *A, const double *b,
                                const double *x_prev, const double *x_next, uint16_t *feats,
                                float *targets, void *stream);
/* Loss and parameter gradients of the minibatch made of rows `rows` (DEVICE
 * int32 [M]) of the sample store (feats, targets); M a multiple of 64 up to
 * max_batch. *loss (DEVICE) receives the mean squared error; the gradients
 * stay in the network (flat layout, see bbs_mlp_get_grads). */
bbs_status bbs_mlp_gradients(bbs_mlp *mlp, const uint16_t *feats, const float *targets,
                             const int32_t *rows, int32_t M, float *loss, void *stream);
/* bbs_mlp_gradients followed by one Adam step with learning rate lr. */
bbs_status bbs_mlp_train_step(bbs_mlp *mlp, const uint16_t *feats, const float *targets,
                              const int32_t *rows, int32_t M, float lr, float *loss, void *stream);
/* Choose the tensor-core path of the network's GEMMs (default tcgen05). */
bbs_status bbs_mlp_set_gemm(bbs_mlp *mlp, int32_t kind);
/* Wait for the network's work and report whether a tcgen05 GEMM gave up on
 * a bounded wait (BBS_ERR_CUDA) since creation. */
bbs_status bbs_mlp_check(bbs_mlp *mlp);
/* C[m][n] = sum_k A[m*lda + k] B[n*ldb + k] for BF16 A [M, K] and B [N, K]
 * (both K-contiguous, DEVICE), FP32 C [M, ldc] (DEVICE), through the chosen
 * tensor-core path; K a multiple of 64 (tcgen05) or 32 (mma.sync), lda and
 * ldb multiples of 8. Synchronous; the building block of the network. */
bbs_status bbs_gemm_bf16(bbs_handle *handle, int32_t kind, const uint16_t *A, int32_t lda,
                         const uint16_t *B, int32_t ldb, int32_t M, int32_t N, int32_t K, float *C,
                         int32_t ldc);
/* Copy the gradients (flat layout) of the last bbs_mlp_gradients /
 * bbs_mlp_train_step to a DEVICE array. Asynchronous on stream. */
bbs_status bbs_mlp_get_grads(bbs_mlp *mlp, float *grads, void *stream);
/* Network output (standardised change) for M feature rows: out [M, n] FP32. */
bbs_status bbs_mlp_forward(bbs_mlp *mlp, const uint16_t *feats, int32_t M, float *out, void *stream);
/* Initial guesses for a whole batch: x0 = x_prev + gamma * predicted change
 * (DEVICE FP64 [num_batch * n]); gamma is 1 until a gate is fitted. */
bbs_status bbs_mlp_predict(bbs_mlp *mlp, const bbs_batch_matrix *A, const double *b,
                           const double *x_prev, double *x0, void *stream);
/* The gate on the predicted change c, fitted on steps held out from training.
 * An initial guess is there to speed the solve up (Sec. 2.1); with the gate
 * the guess falls back to x_prev where the network carries no signal.
 * gate_observe runs the network on one step (A, b, x_prev as for predict)
 * and accumulates sum c.d and sum c.c over the batch in FP64, d = x_next -
 * x_prev the true change (DEVICE, num_batch*n). gate_finalize sets gamma =
 * sum c.d / sum c.c limited to [0, 1] (0 if sum c.c = 0), the least-squares
 * scale: on the observed steps, sum ||d - gamma c||^2 <= sum ||d||^2, the
 * error of x0 = x_prev; it clears the sums. Asynchronous on stream.
 * get_gate copies gamma to the host (synchronous). */
bbs_status bbs_mlp_gate_observe(bbs_mlp *mlp, const bbs_batch_matrix *A, const double *b,
                                const double *x_prev, const double *x_next, void *stream);
bbs_status bbs_mlp_gate_finalize(bbs_mlp *mlp, void *stream);
bbs_status bbs_mlp_get_gate(bbs_mlp *mlp, double *gamma);

/* Threads per system by the rule of Sec. 3.6: at least n, a multiple of the
 * warp size 32, at most `max_threads` (the device maximum, 1024 on GB300).
 * Returns 0 for n <= 0 or max_threads < 32. Host only. */
int32_t bbs_paper_block_size(int32_t n, int32_t max_threads);

/* Threads per system for an n-row system at up to `rows_per_thread` rows per
 * thread: the fewest warps that keep at most that many rows per thread (which
 * keeps the working vectors in registers). The library uses 8 for the FP64
 * solvers (fewest FP64 instructions per system) and 4 for the mixed mode.
 * Host only. */
int32_t bbs_default_block_size(int32_t n, int32_t rows_per_thread);

/* Measured arithmetic peak of the handle's device, the denominator of the
 * FP64 solvers' roofline (the paper compares each GPU's FP64 peak, Table "GPUs
 * specifications", and places its solver on a roofline, Sec. "Roofline
 * analysis"). precision 0 measures FP64 FMAs, 1 FP32 FMAs: 8 blocks of 256
 * threads per SM, 8 independent FMA chains per thread, timed with CUDA events
 * over one launch of about 20 ms on a stream of its own. *flop_per_s receives
 * the rate (an FMA counts 2 FLOP). Synchronous; allocates no device memory.
 * BBS_ERR_INVALID_ARG for a NULL argument or another precision. */
bbs_status bbs_fma_rate(bbs_handle *handle, int32_t precision, double *flop_per_s);

/* Message of the last failed call on this host thread ("" if none). */
const char *bbs_last_error(void);

/* Library version string. */
const char *bbs_version(void);

#ifdef __cplusplus
}
#endif
#endif /* BBS_H */
