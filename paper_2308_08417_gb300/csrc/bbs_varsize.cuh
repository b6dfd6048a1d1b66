// Device side of the uneven-batch solver (parameters, team loop, kernel
// template). The host planner, tuner and graph capture live in
// bbs_varsize.cu; each kernel instantiation has a translation unit of its own.
//
// Uneven batches: one persistent, graph-captured launch over systems of
// different sizes and patterns, with the team size per size bucket chosen by
// a measured autotuner (the per-device experimental thresholds of Sec. 3.6).
//
// Scheduling. The planner orders the systems by team size (largest first)
// and, within a team size, by estimated cost (longest first), and cuts the
// order into segments of equal (team size, staging). Every block of the
// persistent grid starts as one team per `seg_warps[0]` warps; a team pulls
// system indices from its segment's atomic counter until the segment is
// exhausted, then moves to the next segment. Team sizes never grow along the
// order, so a team only ever splits (8 warps -> two teams of 4 -> ...), and a
// split needs no synchronisation with the rest of the block. A team of w warps
// starting at warp w0 synchronises on named barrier 1 + w0 (unique among the
// teams alive at any time), a full-block team on barrier 0, a single warp on
// __syncwarp. Each team solves its system with the same device functions as
// the one-block-per-system kernels.
#pragma once

#include <cstdint>

#include "bbs_solvers.cuh"

namespace bbs {

constexpr int kMaxSeg = 16;

struct VarParams {
    const int32_t* pat_n;
    const int32_t* pat_nnz;
    const int64_t* rp_off;
    const int64_t* ci_off;
    const int32_t* row_ptrs;
    const int32_t* col_idxs;
    const int32_t* sys_pattern;
    const int64_t* val_off;
    const int64_t* vec_off;
    const double* values;
    const double* b;
    double* x;
    int32_t* iters;
    double* rel_res;
    int32_t* status;
    const int32_t* order;
    int32_t* counters;
    int num_segments;
    int seg_begin[kMaxSeg];
    int seg_count[kMaxSeg];
    int seg_warps[kMaxSeg];
    int seg_stage[kMaxSeg];
    int slice_bytes;
    int solver;
    SolveCfg cfg;
};

// Not inlined: each rows-per-thread variant is compiled as a function of its
// own (one call per system), which keeps the persistent kernel's compile time
// linear in the number of variants. Everything is passed by value, so that
// the solver loops keep it in registers (a reference would leave it in the
// caller's local memory).
template <int R>
__device__ __noinline__ void var_run(int solver, const SolveCfg cfg, const Mat<double> A, int nnz,
                                     const SysIO io, const TeamSmem sm, double* stage, const Team tm) {
    const auto op = make_op<FMT_CSR, R>(A, (size_t)nnz, stage, tm);
    if (solver == 1)
        cg_system<FMT_CSR, R>(op, io, cfg, sm, tm);
    else
        bicgstab_any<FMT_CSR, R>(op, io, cfg, sm, tm);
}

template <int R, int RMAX>
__device__ __forceinline__ void var_dispatch(int rows, const VarParams& P, const Mat<double>& A,
                                             int nnz, const SysIO& io, const TeamSmem& sm,
                                             double* stage, const Team& tm) {
    if constexpr (R == RMAX) {
        var_run<R>(P.solver, P.cfg, A, nnz, io, sm, stage, tm);
    } else {
        if (rows <= R)
            var_run<R>(P.solver, P.cfg, A, nnz, io, sm, stage, tm);
        else
            var_dispatch<R + 1, RMAX>(rows, P, A, nnz, io, sm, stage, tm);
    }
}

// Team area: red [256 doubles] | xa [n_pad] | xb [n_pad] | staged values
template <int RMAX>
__device__ __forceinline__ void var_solve_one(const VarParams& P, int sys, const Team& tm,
                                              unsigned char* area, bool stage_values_flag) {
    const int pat = P.sys_pattern[sys];
    const int n = P.pat_n[pat];
    const int nnz = P.pat_nnz[pat];
    const Mat<double> A{P.values + P.val_off[sys], P.row_ptrs + P.rp_off[pat],
                        P.col_idxs + P.ci_off[pat], n, 0};
    SysIO io;
    io.b = P.b + P.vec_off[sys];
    io.x = P.x + P.vec_off[sys];
    io.iters = P.iters + sys;
    io.rel_res = P.rel_res + sys;
    io.status = P.status + sys;
    io.inner = nullptr;
    io.n = n;
    const TeamSmem sm = team_smem(area, (n + 1) & ~1);
    double* stage = stage_values_flag ? sm.extra : nullptr;
    const int rows = (n + tm.nt - 1) / tm.nt;
    var_dispatch<1, RMAX>(rows, P, A, nnz, io, sm, stage, tm);
}

template <int RMAX>
__global__ void __launch_bounds__(RMAX <= 4 ? 512 : 256, 1) varsize_kernel(const __grid_constant__ VarParams P) {
    extern __shared__ __align__(16) unsigned char raw[];
    const int warp = threadIdx.x >> 5;
    for (int seg = 0; seg < P.num_segments; ++seg) {
        const int W = P.seg_warps[seg];
        const int w0 = warp - warp % W;
        const Team tm = Team::group(w0, W);
        unsigned char* base = raw + (size_t)w0 * P.slice_bytes;
        int* cell = reinterpret_cast<int*>(base);
        const int count = P.seg_count[seg];
        for (;;) {
            int item;
            if (W == 1) {
                int v = 0;
                if (tm.lane == 0) v = atomicAdd(P.counters + seg, 1);
                item = __shfl_sync(kFull, v, 0);
            } else {
                if (tm.tid == 0) *cell = atomicAdd(P.counters + seg, 1);
                tm.sync();
                item = *cell;
                tm.sync();  // the cell is rewritten by the next grab
            }
            if (item >= count) break;
            var_solve_one<RMAX>(P, P.order[P.seg_begin[seg] + item], tm, base + 16,
                                P.seg_stage[seg] != 0);
        }
    }
}

}  // namespace bbs


namespace bbs {
const void* varsize_kernel4_fn();
const void* varsize_kernel8_fn();
}  // namespace bbs
