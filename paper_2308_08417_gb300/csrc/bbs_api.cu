// Host side of the C ABI declared in include/bbs.h: argument checks, the
// launch-shape choice, the kernel dispatch over (solver, format, precision,
// rows per thread) (Sec. 3.3's multi-level dispatch) and the host-buffer path.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/bbs.h"
#include "bbs_ilu.cuh"
#include "bbs_internal.h"
#include "bbs_kernels.h"
#include "bbs_params.h"

struct bbs_handle {
    int device = 0;
    int sms = 0;
    int max_smem_optin = 0;
    int max_threads = 1024;
    // bbs_solve_host: the inputs go in on `copy_in`, chunk after chunk, each
    // chunk signalling `chunk_in[c]`; the solves and the copies out alternate
    // between `stream` and `stream2`, so consecutive solves overlap
    cudaStream_t stream = nullptr;
    cudaStream_t stream2 = nullptr;
    cudaStream_t copy_in = nullptr;
    cudaEvent_t chunk_in[16] = {nullptr};
    // device buffers owned for bbs_solve_host (grow only)
    void* buf[12] = {nullptr};
    size_t cap[12] = {0};
    // CSR patterns whose row-length bound (ell_k) has been checked against
    // their row pointers, most recent first (see csr_bound_ok)
    struct CheckedPattern {
        const int32_t* row_ptrs;
        int32_t n, nnz, ell_k, longest;
    };
    static constexpr int kChecked = 16;
    CheckedPattern checked[kChecked] = {};
    int num_checked = 0;
    std::mutex checked_mutex;
};

namespace {

thread_local std::string g_last_error;

bbs_status fail(bbs_status s, const char* fmt, ...) {
    char msg[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(msg, sizeof msg, fmt, ap);
    va_end(ap);
    g_last_error = msg;
    return s;
}

bbs_status cuda_fail(cudaError_t e, const char* what) {
    return fail(BBS_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

size_t vals_per_system(const bbs_batch_matrix* A) {
    switch (A->fmt) {
        case BBS_FMT_CSR: return (size_t)A->nnz;
        case BBS_FMT_ELL: return (size_t)A->ell_k * (size_t)A->n;
        default: return (size_t)A->n * (size_t)A->n;
    }
}

// Default rows per thread: FP64 arithmetic is the scarce resource, so the FP64
// solvers use the fewest warps per system (up to 8 rows per thread); the mixed
// mode's FP32 inner loop is latency-bound and prefers 4 rows per thread.
constexpr int kDefaultRowsPerThread = 8;
constexpr int kMixedRowsPerThread = 4;
// Values are staged in shared memory by default when a block's shared memory
// stays within this size (two blocks per SM).
constexpr size_t kAutoStageBytes = 116 * 1024;

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Launch plan for one solve.
struct Plan {
    int threads = 0, R = 0, n_pad = 0;
    size_t smem = 0;        // dynamic shared memory bytes
    size_t stage_off = 0;
    bool stage = false;
    bool gmres_ws = false;  // GMRES basis in the workspace
    bool ilu = false;       // ILU(0): level schedule in the workspace, factors in shared memory
    int lanes = 32;         // < 32: packed kernel, 32 / lanes systems per one-warp block
    size_t slice = 0;       // packed: shared-memory bytes per system
    size_t ws_gmres = 0, ws_f32 = 0, ws_ilu = 0;
    size_t ws_tables = 0;   // packed CSR: ELL column table, value map and flag
};

bbs_status validate(const bbs_batch_matrix* A, const bbs_options* o) {
    if (A == nullptr || o == nullptr) return fail(BBS_ERR_INVALID_ARG, "null matrix or options");
    if (A->fmt < 0 || A->fmt > 2) return fail(BBS_ERR_INVALID_ARG, "unknown format %d", A->fmt);
    if (A->num_batch < 0) return fail(BBS_ERR_INVALID_ARG, "num_batch < 0");
    if (A->n <= 0) return fail(BBS_ERR_INVALID_ARG, "n must be positive (got %d)", A->n);
    if (A->fmt == BBS_FMT_CSR && (A->nnz < 0 || A->row_ptrs == nullptr || A->col_idxs == nullptr))
        return fail(BBS_ERR_INVALID_ARG, "CSR needs nnz >= 0, row_ptrs and col_idxs");
    if (A->fmt == BBS_FMT_ELL) {
        if (A->ell_k <= 0 || A->col_idxs == nullptr)
            return fail(BBS_ERR_INVALID_ARG, "ELL needs ell_k > 0 and col_idxs");
        if ((long long)A->ell_k * A->n > 0x7fffffffLL)
            return fail(BBS_ERR_INVALID_ARG, "ELL ell_k*n overflows int32");
    }
    if (A->fmt == BBS_FMT_CSR && A->ell_k < 0)
        return fail(BBS_ERR_INVALID_ARG, "CSR ell_k must be 0 (unknown) or the largest row length");
    if (A->fmt == BBS_FMT_DENSE && (long long)A->n * A->n > 0x7fffffffLL)
        return fail(BBS_ERR_INVALID_ARG, "dense n*n overflows int32");
    if (A->num_batch > 0 && A->values == nullptr) return fail(BBS_ERR_INVALID_ARG, "values is NULL");
    if (o->solver < 0 || o->solver > 2) return fail(BBS_ERR_INVALID_ARG, "unknown solver %d", o->solver);
    if (o->precond < 0 || o->precond > 2) return fail(BBS_ERR_INVALID_ARG, "unknown preconditioner %d", o->precond);
    if (o->precond == BBS_PREC_ILU0 &&
        (A->fmt != BBS_FMT_CSR || o->solver != BBS_SOLVER_BICGSTAB || o->precision != BBS_PRECISION_FP64))
        return fail(BBS_ERR_UNSUPPORTED, "ILU(0) preconditions FP64 BiCGSTAB on BatchCsr");
    if (o->tol_type < 0 || o->tol_type > 1) return fail(BBS_ERR_INVALID_ARG, "unknown tolerance type %d", o->tol_type);
    if (!(o->tol > 0.0)) return fail(BBS_ERR_INVALID_ARG, "tol must be > 0");
    if (o->max_iters < 0) return fail(BBS_ERR_INVALID_ARG, "max_iters must be >= 0");
    if (o->precision < 0 || o->precision > 1) return fail(BBS_ERR_INVALID_ARG, "unknown precision %d", o->precision);
    if (o->solver == BBS_SOLVER_GMRES && (o->gmres_restart < 1 || o->gmres_restart > 32))
        return fail(BBS_ERR_INVALID_ARG, "gmres_restart must be in [1, 32]");
    if (o->precision == BBS_PRECISION_MIXED_IR) {
        if (o->solver != BBS_SOLVER_BICGSTAB)
            return fail(BBS_ERR_UNSUPPORTED, "mixed precision is provided for BiCGSTAB only");
        if (!(o->inner_tol > 0.0 && o->inner_tol < 1.0))
            return fail(BBS_ERR_INVALID_ARG, "inner_tol must be in (0, 1)");
        if (o->max_outer < 0 || o->max_iters < 1)
            return fail(BBS_ERR_INVALID_ARG, "mixed mode needs max_outer >= 0 and max_iters >= 1");
    }
    const int t = o->threads_per_system;
    if (t == 4 || t == 8 || t == 16) {
        if (o->precision != BBS_PRECISION_FP64 || o->values_in_smem == -1 ||
            (o->solver == BBS_SOLVER_GMRES && o->precond == BBS_PREC_ILU0))
            return fail(BBS_ERR_UNSUPPORTED,
                        "threads_per_system %d (packed systems) is provided for FP64 solvers with staged "
                        "values", t);
    } else if (t != 0 && (t < 32 || t > 1024 || (t % 32) != 0)) {
        return fail(BBS_ERR_INVALID_ARG,
                    "threads_per_system must be 0, 4, 8, 16 or a multiple of 32 in [32, 1024]");
    }
    if (o->values_in_smem < -1 || o->values_in_smem > 1)
        return fail(BBS_ERR_INVALID_ARG, "values_in_smem must be -1, 0 or 1");
    return BBS_OK;
}

int max_row_len(const bbs_batch_matrix* A) { return A->fmt == BBS_FMT_ELL ? A->ell_k : 0; }

// Shared memory of a packed system: xa [n_pad] | xb [n_pad] | values. The
// slice is padded to 8 L bytes past a multiple of 128, so the groups that
// share a half-warp's shared-memory wavefront start on different banks.
size_t packed_slice(int n_pad, size_t vps, int L, size_t* stage_off, size_t extra = 0) {
    *stage_off = align_up(2 * (size_t)n_pad * 8, 16);
    const size_t raw = *stage_off + align_up(vps * 8, 16) + extra;
    const size_t shift = (size_t)(8 * L) % 128;
    return align_up(raw + 128 - shift, 128) - 128 + shift;
}

// Warps an SM keeps resident for a packed launch: one-warp blocks, limited by
// the register cap of the kernel's launch bounds and by shared memory.
int packed_warps_per_sm(size_t smem, int R) {
    const size_t sm_bytes = 228 * 1024;  // per SM, with 1 KB reserved per block
    const int by_smem = smem + 1024 > sm_bytes ? 0 : (int)(sm_bytes / (smem + 1024));
    const int by_regs = R <= 5 ? 16 : 12;  // packed_min_blocks
    return by_smem < by_regs ? by_smem : by_regs;
}

// The library's packing: the narrowest group of 4, 8 or 16 lanes that covers
// n in at most kMaxPackedR rows per lane and still leaves kPackedMinWarps
// warps resident per SM (narrower groups put more systems on each FP64
// instruction; fewer warps leave the FP64 pipe idle). Measured on GB300
// (BiCGSTAB + Jacobi, 32,768 systems): 22 rows, 438 values: 8 lanes (14
// warps) 31.0 M systems/s, 4 lanes (7 warps) 28.5 M, one per warp 16.9 M;
// 33 rows, 978 values (CSR): 16 lanes (13 warps) 13.4 M, 8 lanes (6 warps)
// 12.7 M, one per warp 9.4 M; 54 rows, 2,560 values: 16 lanes (5 warps)
// 5.1 M, one per warp 6.5 M.
constexpr int kPackedMinWarps = 8;

bbs_status make_plan(const bbs_handle* h, const bbs_batch_matrix* A, const bbs_options* o, Plan* p) {
    const int n = A->n;
    const int tps = o->threads_per_system;
    // ILU(0) packs too (BiCGSTAB on CSR; validate() rejects the rest): its
    // factors are staged in the values' place and 1/u_ii after them
    const bool ilu = o->precond == BBS_PREC_ILU0;
    const bool gmres = o->solver == BBS_SOLVER_GMRES;
    // (the packed ILU(0) kernel keeps CSR indices in 16 bits)
    const bool packable = o->precision == BBS_PRECISION_FP64 && o->values_in_smem != -1 && !(gmres && ilu) &&
                          !(ilu && A->nnz >= 32768);
    // CSR packs through an ELL table of width ell_k (the caller's bound on
    // the row length); the library packs it only while the padding stays
    // small, and needs the bound in any case.
    const bool csr = A->fmt == BBS_FMT_CSR;
    const bool csr_ok = !csr || (A->ell_k > 0 && (size_t)A->ell_k * (size_t)n <= (size_t)A->nnz * 3 / 2);
    if (packable && tps != 0 && csr && A->ell_k <= 0)
        return fail(BBS_ERR_INVALID_ARG,
                    "packed systems on CSR need ell_k = the largest number of nonzeros in a row");
    if (packable && (tps == 4 || tps == 8 || tps == 16 || (tps == 0 && csr_ok))) {
        const int n_pad = (n + 1) & ~1;
        const size_t vps = csr ? (size_t)A->ell_k * (size_t)n : vals_per_system(A);
        for (int L = tps ? tps : 4; L <= (tps ? tps : 16); L *= 2) {
            const int R = (n + L - 1) / L;
            size_t off = 0;
            // after the values: the GMRES Hessenberg, rotations, right-hand side,
            // solution and control words
            const size_t mr = (size_t)o->gmres_restart;
            const size_t extra = gmres ? (mr * (mr + 3) / 2 + 2 * mr + (mr + 1) + mr + 2) * 8 : 0;
            const size_t slice = packed_slice(n_pad, vps, L, &off, extra);
            // ILU(0) blocks also hold one copy of the pattern for their groups
            const size_t smem = slice * (size_t)(32 / L) + (ilu ? bbs::ilu_pattern_smem(n, A->ell_k) : 0);
            if (tps != 0) {
                if (R > bbs::kMaxPackedR)
                    return fail(BBS_ERR_INVALID_ARG, "threads_per_system %d leaves %d rows per lane (max %d)",
                                tps, R, bbs::kMaxPackedR);
                if (smem > (size_t)h->max_smem_optin)
                    return fail(BBS_ERR_UNSUPPORTED, "packed block needs %zu bytes of shared memory (max %d)",
                                smem, h->max_smem_optin);
            } else if (R > bbs::kMaxPackedR || smem > (size_t)h->max_smem_optin ||
                       packed_warps_per_sm(smem, R) < kPackedMinWarps) {
                continue;
            }
            p->lanes = L;
            p->R = R;
            p->threads = 32;
            p->n_pad = n_pad;
            p->stage = true;
            p->stage_off = off;
            p->slice = slice;
            p->smem = smem;
            if (csr) p->ws_tables = align_up(2 * vps * 4, 256) + 256;
            if (ilu) {
                p->ilu = true;
                p->ws_ilu = align_up(bbs::ilu_workspace_bytes(n), 256);
            }
            if (gmres) {  // the Krylov basis in the workspace, (m + 1) x n_pad per system
                p->gmres_ws = true;
                p->ws_gmres = (mr + 1) * (size_t)n_pad * 8 * (size_t)A->num_batch;
            }
            return BBS_OK;
        }
    }
    const int rpt = o->precision == BBS_PRECISION_MIXED_IR ? kMixedRowsPerThread : kDefaultRowsPerThread;
    p->threads = tps ? tps : bbs_default_block_size(n, rpt);
    if (p->threads <= 0)
        return fail(BBS_ERR_UNSUPPORTED, "n = %d exceeds the largest supported system (%d rows)", n,
                    bbs::kMaxRows);
    p->R = (n + p->threads - 1) / p->threads;
    if (p->R > bbs::kMaxR || p->threads > bbs::max_threads_for(p->R))
        return fail(BBS_ERR_INVALID_ARG,
                    "threads_per_system %d leaves %d rows per thread; R = 1 allows 1024 threads, "
                    "R <= 4 512, R <= 8 256", p->threads, p->R);
    p->n_pad = (n + 1) & ~1;
    const bool mixed = o->precision == BBS_PRECISION_MIXED_IR;
    const size_t vps = vals_per_system(A);
    size_t base;
    if (mixed) {  // FP32 SpMV inputs keep a zero after their last entry
        base = 256 * 8 + (size_t)p->n_pad * 8 + 256 * 4 + 2 * ((size_t)p->n_pad + 2) * 4;
    } else {
        base = 256 * 8 + 2 * (size_t)p->n_pad * 8;
        if (o->solver == BBS_SOLVER_GMRES) {
            const size_t m = (size_t)o->gmres_restart;
            base += ((m + 1) * m + 2 * m + (m + 1) + m + 2) * 8;
            const size_t vbytes = (m + 1) * (size_t)p->n_pad * 8;
            if (base + vbytes <= (size_t)h->max_smem_optin) {
                base += vbytes;
            } else {
                p->gmres_ws = true;
                p->ws_gmres = vbytes * (size_t)A->num_batch;
            }
        }
    }
    base = align_up(base, 16);
    if (o->precond == BBS_PREC_ILU0) {  // factors (nnz) and inverse U diagonal (n_pad) in shared memory
        p->ilu = true;
        p->stage = true;
        p->stage_off = base;
        p->smem = base + align_up(vps * 8, 16) + (size_t)p->n_pad * 8;
        if (p->smem > (size_t)h->max_smem_optin)
            return fail(BBS_ERR_UNSUPPORTED, "ILU(0) factors need %zu bytes of shared memory (max %d)", p->smem,
                        h->max_smem_optin);
        p->ws_ilu = align_up(bbs::ilu_workspace_bytes(n), 256);
        return BBS_OK;
    }
    // mixed mode on ELL stages an FP32 value and a 16-bit column for every row
    // slot of the block, R * ell_k * threads of each (the refinement kernel's
    // PairOp32); otherwise the values in their own layout
    const size_t stage_bytes = (mixed && A->fmt == BBS_FMT_ELL)
                                   ? align_up((size_t)p->R * (size_t)A->ell_k * (size_t)p->threads * 6, 16)
                                   : align_up(vps * (mixed ? 4 : 8), 16);
    const size_t limit = (size_t)h->max_smem_optin;
    bool stage = false;
    if (o->values_in_smem == 1)
        stage = base + stage_bytes <= limit;
    else if (o->values_in_smem == 0)
        stage = base + stage_bytes <= kAutoStageBytes;
    if (base > limit) return fail(BBS_ERR_UNSUPPORTED, "shared memory need %zu exceeds %zu", base, limit);
    p->stage = stage;
    p->stage_off = base;
    p->smem = base + (stage ? stage_bytes : 0);
    // without the caller's FP32 copy, staged values are rounded as the kernel
    // stages them; only unstaged values need a converted copy in the workspace
    if (mixed && A->values_f32 == nullptr && !stage) p->ws_f32 = align_up(vps * 4 * (size_t)A->num_batch, 256);
    return BBS_OK;
}

size_t workspace_bytes(const Plan& p) {
    return align_up(p.ws_gmres, 256) + p.ws_f32 + p.ws_ilu + p.ws_tables;
}

// BiCGSTAB with staged values and Jacobi runs the Jacobi-folded kernel; the
// mixed mode on ELL with staged values takes an instance for its ELL width
// when there is one and the block has at most 256 threads (those instances
// are compiled for three resident blocks).
const void* pick_kernel(const bbs_options* o, int fmt, int R, bool staged, int ell_k, int threads) {
    if (o->precision == BBS_PRECISION_MIXED_IR) {
        const void* fn = (fmt == BBS_FMT_ELL && staged && threads <= 256) ? bbs::refine_ell_fn(R, ell_k) : nullptr;
        return fn != nullptr ? fn : bbs::refine_fn(fmt, R);
    }
    switch (o->solver) {
        case BBS_SOLVER_CG: return bbs::cg_fn(fmt, R);
        case BBS_SOLVER_GMRES: return bbs::gmres_fn(fmt, R);
        default:
            return (staged && o->precond == BBS_PREC_JACOBI) ? bbs::bicgstab_folded_fn(fmt, R)
                                                             : bbs::bicgstab_fn(fmt, R);
    }
}

std::mutex g_attr_mutex;

cudaError_t allow_smem(const void* fn, size_t smem) {
    if (smem <= 48 * 1024) return cudaSuccess;
    std::lock_guard<std::mutex> lock(g_attr_mutex);
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

// Packed CSR solves stage each system's values through an ELL table of
// width ell_k, so a row longer than ell_k is an argument error. The row
// pointers are device data: the first solve with a pattern (keyed by its
// row_ptrs address, n, nnz and ell_k) copies them back on the solve's stream
// and waits for them, and the handle remembers the result, so later solves
// with the same pattern launch without waiting. (A pattern rewritten in place
// behind a remembered key is still caught on the device, where every system
// then reports BBS_SYS_NAN.)
void remember_pattern(bbs_handle* h, const bbs_batch_matrix* A, int32_t longest) {
    std::lock_guard<std::mutex> lock(h->checked_mutex);
    int keep = h->num_checked < bbs_handle::kChecked ? h->num_checked : bbs_handle::kChecked - 1;
    for (int i = 0; i < h->num_checked; ++i) {
        const auto& c = h->checked[i];
        if (c.row_ptrs == A->row_ptrs && c.n == A->n && c.nnz == A->nnz && c.ell_k == A->ell_k) {
            keep = i;
            break;
        }
    }
    for (int i = keep; i > 0; --i) h->checked[i] = h->checked[i - 1];
    h->checked[0] = {A->row_ptrs, A->n, A->nnz, A->ell_k, longest};
    if (keep == h->num_checked) ++h->num_checked;
}

bbs_status csr_bound_ok(bbs_handle* h, const bbs_batch_matrix* A, cudaStream_t st) {
    int32_t longest = -1;
    {
        std::lock_guard<std::mutex> lock(h->checked_mutex);
        for (int i = 0; i < h->num_checked; ++i) {
            const auto& c = h->checked[i];
            if (c.row_ptrs == A->row_ptrs && c.n == A->n && c.nnz == A->nnz && c.ell_k == A->ell_k) {
                longest = c.longest;
                break;
            }
        }
    }
    if (longest < 0) {
        std::vector<int32_t> rp((size_t)A->n + 1);
        cudaError_t e = cudaMemcpyAsync(rp.data(), A->row_ptrs, rp.size() * sizeof(int32_t),
                                        cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "reading the CSR row pointers back");
        longest = 0;
        for (int32_t i = 0; i < A->n; ++i) longest = std::max(longest, rp[(size_t)i + 1] - rp[i]);
        remember_pattern(h, A, longest);
    }
    if (longest > A->ell_k)
        return fail(BBS_ERR_INVALID_ARG, "a CSR row has %d nonzeros, more than ell_k = %d", longest, A->ell_k);
    return BBS_OK;
}

}  // namespace

namespace bbs {
bbs_status record_error(bbs_status s, const char* msg) { return fail(s, "%s", msg); }
int handle_device(const bbs_handle* h) { return h->device; }
}  // namespace bbs

extern "C" {

bbs_status bbs_default_options(bbs_options* o) {
    if (o == nullptr) return fail(BBS_ERR_INVALID_ARG, "null options");
    std::memset(o, 0, sizeof *o);
    o->solver = BBS_SOLVER_BICGSTAB;
    o->precond = BBS_PREC_JACOBI;
    o->tol_type = BBS_TOL_RELATIVE;
    o->tol = 1e-10;
    o->max_iters = 500;
    o->gmres_restart = 10;
    o->precision = BBS_PRECISION_FP64;
    o->inner_tol = 1e-4;
    o->max_outer = 30;
    return BBS_OK;
}

int32_t bbs_paper_block_size(int32_t n, int32_t max_threads) {
    if (n <= 0 || max_threads < 32) return 0;
    const int32_t cap = max_threads / 32 * 32;
    const int32_t up = (n + 31) / 32 * 32;
    return up < cap ? up : cap;
}

int32_t bbs_default_block_size(int32_t n, int32_t rows_per_thread) {
    if (n <= 0 || rows_per_thread <= 0 || n > bbs::kMaxRows) return 0;
    const int32_t rpt = rows_per_thread < bbs::kMaxR ? rows_per_thread : bbs::kMaxR;
    for (int32_t r = rpt; r >= 1; --r) {  // fewest warps at <= r rows per thread
        const int32_t threads = (n + 32 * r - 1) / (32 * r) * 32;
        if (threads > 1024) continue;
        const int32_t R = (n + threads - 1) / threads;
        if (threads <= bbs::max_threads_for(R)) return threads;
    }
    return 0;
}

const char* bbs_last_error(void) { return g_last_error.c_str(); }

const char* bbs_version(void) { return "bbs 0.1 sm_103a"; }

bbs_status bbs_create(bbs_handle** handle, int device) {
    if (handle == nullptr) return fail(BBS_ERR_INVALID_ARG, "null handle pointer");
    *handle = nullptr;
    int count = 0;
    cudaError_t e = cudaGetDeviceCount(&count);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
    if (device < 0 || device >= count) return fail(BBS_ERR_INVALID_ARG, "device %d out of range", device);
    bbs_handle* h = new bbs_handle();
    h->device = device;
    if ((e = cudaSetDevice(device)) != cudaSuccess) { delete h; return cuda_fail(e, "cudaSetDevice"); }
    cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, device);
    cudaDeviceGetAttribute(&h->max_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    cudaDeviceGetAttribute(&h->max_threads, cudaDevAttrMaxThreadsPerBlock, device);
    if ((e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking)) == cudaSuccess &&
        (e = cudaStreamCreateWithFlags(&h->stream2, cudaStreamNonBlocking)) == cudaSuccess)
        e = cudaStreamCreateWithFlags(&h->copy_in, cudaStreamNonBlocking);
    for (cudaEvent_t& ev : h->chunk_in)
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        bbs_destroy(h);
        return cuda_fail(e, "stream or event creation");
    }
    *handle = h;
    return BBS_OK;
}

bbs_status bbs_destroy(bbs_handle* h) {
    if (h == nullptr) return BBS_OK;
    cudaSetDevice(h->device);
    for (int i = 0; i < 12; ++i)
        if (h->buf[i]) cudaFree(h->buf[i]);
    if (h->stream) cudaStreamDestroy(h->stream);
    if (h->stream2) cudaStreamDestroy(h->stream2);
    if (h->copy_in) cudaStreamDestroy(h->copy_in);
    for (cudaEvent_t ev : h->chunk_in)
        if (ev) cudaEventDestroy(ev);
    delete h;
    return BBS_OK;
}

bbs_status bbs_workspace_size(const bbs_handle* h, const bbs_batch_matrix* A, const bbs_options* o,
                              size_t* bytes) {
    if (h == nullptr || bytes == nullptr) return fail(BBS_ERR_INVALID_ARG, "null handle or output");
    bbs_status s = validate(A, o);
    if (s != BBS_OK) return s;
    Plan p;
    if ((s = make_plan(h, A, o, &p)) != BBS_OK) return s;
    *bytes = workspace_bytes(p);
    return BBS_OK;
}

bbs_status bbs_describe(const bbs_handle* h, const bbs_batch_matrix* A, const bbs_options* o,
                        bbs_launch_info* info) {
    if (h == nullptr || info == nullptr) return fail(BBS_ERR_INVALID_ARG, "null handle or output");
    bbs_status s = validate(A, o);
    if (s != BBS_OK) return s;
    Plan p;
    if ((s = make_plan(h, A, o, &p)) != BBS_OK) return s;
    std::memset(info, 0, sizeof *info);
    const bool mixed = o->precision == BBS_PRECISION_MIXED_IR;
    if (p.lanes < 32) {
        info->kernel = p.ilu ? "bicgstab_ilu_packed_kernel"
                       : o->solver == BBS_SOLVER_CG ? "cg_packed_kernel"
                       : o->solver == BBS_SOLVER_GMRES ? "gmres_packed_kernel" : "bicgstab_packed_kernel";
        info->grid = (A->num_batch + 32 / p.lanes - 1) / (32 / p.lanes);
        info->threads_per_system = p.lanes;
    } else {
        info->kernel = p.ilu ? "bicgstab_ilu_kernel"
                       : mixed ? "refine_kernel"
                       : o->solver == BBS_SOLVER_CG ? "cg_kernel"
                       : o->solver == BBS_SOLVER_GMRES ? "gmres_kernel"
                       : (p.stage && o->precond == BBS_PREC_JACOBI) ? "bicgstab_folded_kernel"
                                                                     : "bicgstab_kernel";
        info->grid = A->num_batch;
        info->threads_per_system = p.threads;
    }
    info->block = p.threads;
    info->rows_per_thread = p.R;
    info->smem_bytes = (int64_t)p.smem;
    info->values_staged = p.stage ? 1 : 0;
    info->launches = A->num_batch == 0 ? 0 : 1 + ((p.ws_f32 > 0 || p.ilu) ? 1 : 0) + (p.ws_tables > 0 ? 1 : 0);
    return BBS_OK;
}

bbs_status bbs_check_pattern(bbs_handle* h, const bbs_batch_matrix* A, int32_t* bad_rows) {
    if (h == nullptr || A == nullptr || bad_rows == nullptr) return fail(BBS_ERR_INVALID_ARG, "null argument");
    if (A->fmt < 0 || A->fmt > 2) return fail(BBS_ERR_INVALID_ARG, "unknown format %d", A->fmt);
    if (A->n <= 0) return fail(BBS_ERR_INVALID_ARG, "n must be positive (got %d)", A->n);
    *bad_rows = 0;
    if (A->fmt == BBS_FMT_DENSE) return BBS_OK;
    if (A->fmt == BBS_FMT_CSR && (A->nnz < 0 || A->row_ptrs == nullptr || A->col_idxs == nullptr || A->ell_k < 0))
        return fail(BBS_ERR_INVALID_ARG, "CSR needs nnz >= 0, ell_k >= 0, row_ptrs and col_idxs");
    if (A->fmt == BBS_FMT_ELL && (A->ell_k <= 0 || A->col_idxs == nullptr))
        return fail(BBS_ERR_INVALID_ARG, "ELL needs ell_k > 0 and col_idxs");
    cudaSetDevice(h->device);
    int* d_bad = nullptr;
    cudaError_t e = cudaMalloc(&d_bad, sizeof(int));
    if (e != cudaSuccess) return fail(BBS_ERR_NO_MEMORY, "check buffer: %s", cudaGetErrorString(e));
    int bad = 0;
    if ((e = cudaMemsetAsync(d_bad, 0, sizeof(int), h->stream)) == cudaSuccess &&
        (e = bbs::launch_check_pattern(A->fmt, A->n, A->nnz, A->ell_k, A->row_ptrs, A->col_idxs, d_bad, h->stream)) ==
            cudaSuccess &&
        (e = cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, h->stream)) == cudaSuccess)
        e = cudaStreamSynchronize(h->stream);
    cudaFree(d_bad);
    if (e != cudaSuccess) return cuda_fail(e, "pattern check");
    *bad_rows = bad;
    return BBS_OK;
}

bbs_status bbs_solve(bbs_handle* h, const bbs_batch_matrix* A, const double* b, double* x,
                     const bbs_options* o, const bbs_log* log, void* workspace,
                     size_t ws_bytes, void* stream) {
    if (h == nullptr) return fail(BBS_ERR_INVALID_ARG, "null handle");
    bbs_status s = validate(A, o);
    if (s != BBS_OK) return s;
    if (log == nullptr || log->iters == nullptr || log->rel_res == nullptr || log->status == nullptr)
        return fail(BBS_ERR_INVALID_ARG, "log arrays iters, rel_res and status are required");
    if (A->num_batch > 0 && (b == nullptr || x == nullptr))
        return fail(BBS_ERR_INVALID_ARG, "b and x are required");
    Plan p;
    if ((s = make_plan(h, A, o, &p)) != BBS_OK) return s;
    const size_t need = workspace_bytes(p);
    if (ws_bytes < need || (need > 0 && workspace == nullptr))
        return fail(BBS_ERR_NO_MEMORY, "workspace of %zu bytes needed, %zu given", need, ws_bytes);
    if (need > 0 && (reinterpret_cast<uintptr_t>(workspace) & 255) != 0)
        return fail(BBS_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
    if (A->num_batch == 0) return BBS_OK;
    cudaSetDevice(h->device);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (p.ws_tables > 0 && (s = csr_bound_ok(h, A, st)) != BBS_OK) return s;

    bbs::SolveParams P{};
    P.n = A->n;
    P.n_pad = p.n_pad;
    P.k = max_row_len(A);
    P.num_batch = A->num_batch;
    P.vps = vals_per_system(A);
    P.row_ptrs = A->row_ptrs;
    P.cols = A->col_idxs;
    P.values = A->values;
    P.values32 = A->values_f32;
    P.b = b;
    P.x = x;
    P.iters = log->iters;
    P.rel_res = log->rel_res;
    P.status = log->status;
    P.inner_iters = log->inner_iters;
    P.precond = o->precond;
    P.tol_type = o->tol_type;
    P.tol = o->tol;
    P.max_iters = o->max_iters;
    P.restart = o->gmres_restart;
    P.inner_tol = o->inner_tol;
    P.max_outer = o->max_outer;
    P.stage = p.stage ? 1 : 0;
    P.stage_off = p.stage_off;
    unsigned char* ws = static_cast<unsigned char*>(workspace);
    P.ws = p.gmres_ws ? reinterpret_cast<double*>(ws) : nullptr;
    cudaError_t e;
    if (p.ws_f32 > 0) {
        float* f32 = reinterpret_cast<float*>(ws + align_up(p.ws_gmres, 256));
        if ((e = bbs::launch_convert_f32(A->values, f32, P.vps * (size_t)A->num_batch, st)) != cudaSuccess)
            return cuda_fail(e, "FP32 conversion launch");
        P.values32 = f32;
    }
    const int* csched = nullptr;
    if (p.ilu) {
        int* sched = reinterpret_cast<int*>(ws);
        if ((e = bbs::launch_ilu_analysis(A->n, A->row_ptrs, A->col_idxs, sched, st)) != cudaSuccess)
            return cuda_fail(e, "ILU(0) analysis launch");
        csched = sched;
    }
    if (p.ilu && p.lanes == 32) {
        const void* fn = bbs::bicgstab_ilu_fn(p.R);
        if ((e = allow_smem(fn, p.smem)) != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
        void* args[] = {&P, &csched};
        e = cudaLaunchKernel(fn, dim3((unsigned)A->num_batch), dim3((unsigned)p.threads), args, p.smem, st);
        return e == cudaSuccess ? BBS_OK : cuda_fail(e, "ILU(0) solver launch");
    }
    if (p.lanes < 32) {
        const int per_block = 32 / p.lanes;
        P.slice = p.slice;
        if (p.ws_tables > 0) {  // after the other workspace parts, 256-byte aligned
            unsigned char* t = ws + (need - p.ws_tables);
            const size_t cells = (size_t)A->ell_k * (size_t)A->n;
            int32_t* xcols = reinterpret_cast<int32_t*>(t);
            int32_t* xsrc = xcols + cells;
            int32_t* flag = reinterpret_cast<int32_t*>(t + align_up(2 * cells * 4, 256));
            if ((e = bbs::launch_csr_ell_tables(A->n, A->ell_k, A->row_ptrs, A->col_idxs, xcols, xsrc, flag, st)) !=
                cudaSuccess)
                return cuda_fail(e, "CSR table launch");
            P.xcols = xcols;
            P.xsrc = xsrc;
            P.xflag = flag;
            P.xk = A->ell_k;
        }
        const void* fn = p.ilu ? bbs::bicgstab_ilu_packed_fn(p.lanes, p.R)
                         : o->solver == BBS_SOLVER_CG ? bbs::cg_packed_fn(A->fmt, p.lanes, p.R)
                         : o->solver == BBS_SOLVER_GMRES ? bbs::gmres_packed_fn(A->fmt, p.lanes, p.R)
                                                         : bbs::bicgstab_packed_fn(A->fmt, p.lanes, p.R);
        if ((e = allow_smem(fn, p.smem)) != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
        void* args[] = {&P, &csched};  // the ILU(0) kernels take the schedule as a second argument
        const unsigned blocks = (unsigned)((A->num_batch + per_block - 1) / per_block);
        e = cudaLaunchKernel(fn, dim3(blocks), dim3(32), args, p.smem, st);
        return e == cudaSuccess ? BBS_OK : cuda_fail(e, "packed solver launch");
    }
    const void* fn = pick_kernel(o, A->fmt, p.R, p.stage, A->ell_k, p.threads);
    if ((e = allow_smem(fn, p.smem)) != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
    void* args[] = {&P};
    e = cudaLaunchKernel(fn, dim3((unsigned)A->num_batch), dim3((unsigned)p.threads), args, p.smem, st);
    if (e != cudaSuccess) return cuda_fail(e, "solver launch");
    return BBS_OK;
}

static bbs_status ensure(bbs_handle* h, int slot, size_t bytes, void** out) {
    if (bytes == 0) {
        *out = nullptr;
        return BBS_OK;
    }
    if (h->cap[slot] < bytes) {
        if (h->buf[slot]) cudaFree(h->buf[slot]);
        h->buf[slot] = nullptr;
        h->cap[slot] = 0;
        cudaError_t e = cudaMalloc(&h->buf[slot], bytes);
        if (e != cudaSuccess) return fail(BBS_ERR_NO_MEMORY, "device buffer of %zu bytes: %s", bytes, cudaGetErrorString(e));
        h->cap[slot] = bytes;
    }
    *out = h->buf[slot];
    return BBS_OK;
}

// bbs_solve_host cuts a batch into chunks of about kHostChunkBytes of input
// (at most kHostChunks of that size, at least kHostMinChunk systems each),
// led by a ramp of a quarter and a half chunk so that the first solve starts
// after a short copy. The inputs stream in on their own stream, chunk after
// chunk, never waiting for a solve; each solve waits only for its chunk and
// alternates with the next between two streams, so their partial last waves
// overlap. Per-system results do not depend on the chunking.
constexpr size_t kHostChunkBytes = 128u << 20;
constexpr size_t kHostMinChunk = 2048;
constexpr size_t kHostChunks = 8;

int32_t bbs_host_chunk_plan(int64_t num_batch, int64_t input_bytes_per_system, int64_t* first, int64_t* count,
                            int32_t max_chunks) {
    if (num_batch < 0 || input_bytes_per_system < 0 || first == nullptr || count == nullptr || max_chunks < 0)
        return -1;
    const size_t B = (size_t)num_batch;
    if (B == 0) return 0;
    const size_t in_bytes = B * (size_t)input_bytes_per_system;
    const size_t want = std::min(kHostChunks, std::max<size_t>(1, (in_bytes + kHostChunkBytes - 1) / kHostChunkBytes));
    const size_t chunk = std::min(B, std::max(kHostMinChunk, (B + want - 1) / want));
    // at most 2 + kHostChunks chunks: the ramp, then chunks of `chunk`
    int32_t nc = 0;
    for (size_t c0 = 0; c0 < B; c0 += (size_t)count[nc++]) {
        if (nc == max_chunks) return -1;
        const size_t ramp = nc == 0 ? chunk / 4 : nc == 1 ? chunk / 2 : chunk;
        first[nc] = (int64_t)c0;
        count[nc] = (int64_t)std::min(B - c0, std::max(kHostMinChunk, ramp));
    }
    return nc;
}

bbs_status bbs_solve_host(bbs_handle* h, const bbs_batch_matrix* Ah, const double* b_host,
                          double* x_host, const bbs_options* o, const bbs_log* log_host) {
    if (h == nullptr) return fail(BBS_ERR_INVALID_ARG, "null handle");
    bbs_status s = validate(Ah, o);
    if (s != BBS_OK) return s;
    if (log_host == nullptr || log_host->iters == nullptr || log_host->rel_res == nullptr ||
        log_host->status == nullptr)
        return fail(BBS_ERR_INVALID_ARG, "log arrays iters, rel_res and status are required");
    const size_t B = (size_t)Ah->num_batch, n = (size_t)Ah->n;
    if (B == 0) return BBS_OK;
    if (b_host == nullptr || x_host == nullptr) return fail(BBS_ERR_INVALID_ARG, "b and x are required");
    cudaSetDevice(h->device);
    const size_t vps = vals_per_system(Ah);
    const size_t rp_bytes = Ah->fmt == BBS_FMT_CSR ? (n + 1) * 4 : 0;
    const size_t ci_bytes = Ah->fmt == BBS_FMT_CSR ? (size_t)Ah->nnz * 4
                            : Ah->fmt == BBS_FMT_ELL ? (size_t)Ah->ell_k * n * 4 : 0;
    void *d_rp, *d_ci, *d_v, *d_v32, *d_b, *d_x, *d_it, *d_rr, *d_st, *d_in, *d_ws0, *d_ws1;
    if ((s = ensure(h, 0, rp_bytes, &d_rp)) || (s = ensure(h, 1, ci_bytes, &d_ci)) ||
        (s = ensure(h, 2, B * vps * 8, &d_v)) ||
        (s = ensure(h, 3, Ah->values_f32 ? B * vps * 4 : 0, &d_v32)) ||
        (s = ensure(h, 4, B * n * 8, &d_b)) || (s = ensure(h, 5, B * n * 8, &d_x)) ||
        (s = ensure(h, 6, B * 4, &d_it)) || (s = ensure(h, 7, B * 8, &d_rr)) ||
        (s = ensure(h, 8, B * 4, &d_st)) ||
        (s = ensure(h, 9, log_host->inner_iters ? B * 4 : 0, &d_in)))
        return s;
    int64_t first[16], count[16];
    const int32_t planned = bbs_host_chunk_plan((int64_t)B, (int64_t)(vps * (Ah->values_f32 ? 12 : 8) + 2 * n * 8),
                                                first, count, 16);
    if (planned < 1) return fail(BBS_ERR_UNSUPPORTED, "host batch cut into too many chunks");
    const size_t nchunks = (size_t)planned;
    size_t chunk = 0;  // the largest chunk sizes the workspaces
    for (size_t c = 0; c < nchunks; ++c) chunk = std::max(chunk, (size_t)count[c]);
    bbs_batch_matrix Ad = *Ah;
    Ad.row_ptrs = static_cast<const int32_t*>(d_rp);
    Ad.col_idxs = static_cast<const int32_t*>(d_ci);
    Ad.values = static_cast<const double*>(d_v);
    Ad.values_f32 = static_cast<const float*>(d_v32);
    Ad.num_batch = (int32_t)chunk;
    if (Ah->fmt == BBS_FMT_CSR && Ah->ell_k > 0) {
        // the row pointers are on the host here: check the row-length bound
        // directly, and record the result for the device copy that bbs_solve
        // will see (the handle's buffer may have held another pattern before)
        int32_t longest = 0;
        for (int32_t i = 0; i < Ah->n; ++i) longest = std::max(longest, Ah->row_ptrs[i + 1] - Ah->row_ptrs[i]);
        if (longest > Ah->ell_k)
            return fail(BBS_ERR_INVALID_ARG, "a CSR row has %d nonzeros, more than ell_k = %d", longest, Ah->ell_k);
        remember_pattern(h, &Ad, longest);
    }
    size_t ws_bytes = 0;  // the largest chunk's workspace; one per stream
    if ((s = bbs_workspace_size(h, &Ad, o, &ws_bytes)) != BBS_OK) return s;
    if ((s = ensure(h, 10, ws_bytes, &d_ws0)) != BBS_OK ||
        (s = ensure(h, 11, nchunks > 1 ? ws_bytes : 0, &d_ws1)) != BBS_OK)
        return s;
    cudaStream_t streams[2] = {h->stream, h->stream2};
    cudaError_t e = cudaSuccess;
    // an error after the first copy waits for the work already queued, so
    // that no copy still reads or writes the caller's buffers on return
    const auto drain = [h]() {
        for (cudaStream_t st : {h->copy_in, h->stream, h->stream2}) cudaStreamSynchronize(st);
    };
#define BBS_CP(dst, src, bytes, kind, st)                                          \
    if ((bytes) > 0 && e == cudaSuccess) e = cudaMemcpyAsync(dst, src, bytes, kind, st)
    BBS_CP(d_rp, Ah->row_ptrs, rp_bytes, cudaMemcpyHostToDevice, h->copy_in);
    BBS_CP(d_ci, Ah->col_idxs, ci_bytes, cudaMemcpyHostToDevice, h->copy_in);
    if (e != cudaSuccess) {
        drain();
        return cuda_fail(e, "pattern copy");
    }
    for (size_t c = 0; c < nchunks; ++c) {
        cudaStream_t st = streams[c & 1];
        const size_t c0 = (size_t)first[c], cb = (size_t)count[c];
        char* v = static_cast<char*>(d_v) + c0 * vps * 8;
        char* v32 = Ah->values_f32 ? static_cast<char*>(d_v32) + c0 * vps * 4 : nullptr;
        double* bd = static_cast<double*>(d_b) + c0 * n;
        double* xd = static_cast<double*>(d_x) + c0 * n;
        BBS_CP(v, reinterpret_cast<const char*>(Ah->values) + c0 * vps * 8, cb * vps * 8, cudaMemcpyHostToDevice,
               h->copy_in);
        if (Ah->values_f32)
            BBS_CP(v32, reinterpret_cast<const char*>(Ah->values_f32) + c0 * vps * 4, cb * vps * 4,
                   cudaMemcpyHostToDevice, h->copy_in);
        BBS_CP(bd, b_host + c0 * n, cb * n * 8, cudaMemcpyHostToDevice, h->copy_in);
        BBS_CP(xd, x_host + c0 * n, cb * n * 8, cudaMemcpyHostToDevice, h->copy_in);
        if (e == cudaSuccess) e = cudaEventRecord(h->chunk_in[c], h->copy_in);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, h->chunk_in[c], 0);
        if (e != cudaSuccess) {
            drain();
            return cuda_fail(e, "host-to-device copy");
        }
        bbs_batch_matrix Ac = Ad;
        Ac.num_batch = (int32_t)cb;
        Ac.values = reinterpret_cast<const double*>(v);
        Ac.values_f32 = reinterpret_cast<const float*>(v32);
        bbs_log dlog{static_cast<int32_t*>(d_it) + c0, static_cast<double*>(d_rr) + c0,
                     static_cast<int32_t*>(d_st) + c0, d_in ? static_cast<int32_t*>(d_in) + c0 : nullptr};
        if ((s = bbs_solve(h, &Ac, bd, xd, o, &dlog, (c & 1) ? d_ws1 : d_ws0, ws_bytes, st)) != BBS_OK) {
            drain();
            return s;
        }
        BBS_CP(x_host + c0 * n, xd, cb * n * 8, cudaMemcpyDeviceToHost, st);
        BBS_CP(log_host->iters + c0, dlog.iters, cb * 4, cudaMemcpyDeviceToHost, st);
        BBS_CP(log_host->rel_res + c0, dlog.rel_res, cb * 8, cudaMemcpyDeviceToHost, st);
        BBS_CP(log_host->status + c0, dlog.status, cb * 4, cudaMemcpyDeviceToHost, st);
        if (log_host->inner_iters) BBS_CP(log_host->inner_iters + c0, dlog.inner_iters, cb * 4, cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) {
            drain();
            return cuda_fail(e, "device-to-host copy");
        }
    }
#undef BBS_CP
    for (cudaStream_t st : {h->copy_in, h->stream, h->stream2})
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "solve");
    return BBS_OK;
}

}  // extern "C"
