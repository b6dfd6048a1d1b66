// Uneven batches, small systems: several systems of different patterns
// packed to a warp (the packing of bbs_packed.cuh, with each group of L lanes
// reading its own system's pattern).
//
// The planner (bbs_varsize.cu) puts every system of up to L * kMaxPackedR
// rows whose group fits the shared-memory rule into a class (L, R): the
// narrowest L of 4, 8, 16 that covers its n in R <= kMaxPackedR rows per lane.
// Each class is one launch of varpacked_kernel<SOLVER, L, R> over the class's
// systems (one warp per block, 32 / L systems per warp, in lockstep), and the
// plan's CUDA graph holds these launches beside the persistent team kernel.
// Each pattern of a packed system has an ELL column table built once when
// the plan is made; the values are gathered through it into shared memory in
// ELL order at the start of every solve, as in the uniform packed kernels.
// The solver device functions are those of the uniform packed kernels: every
// quantity they use per system (n, the pattern, the staged values, the
// vectors) is held per lane, so groups of different sizes and patterns share
// a warp; rows past a group's n stay inert.
#pragma once

#include <cstdint>

#include "bbs_kernels.h"
#include "bbs_packed.cuh"

namespace bbs {

struct VarPackedParams {
    const int32_t* pat_n;
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
    // ELL tables of the packed patterns: slot j of row r of pattern p is
    // entry tab_off[p] + j n_p + r of xcols (its column, -1 for padding) and
    // of xsrc (the CSR index of its value, -1 for padding); tab_k[p] = width
    const int64_t* tab_off;
    const int32_t* tab_k;
    const int32_t* xcols;
    const int32_t* xsrc;
    const int32_t* order;  // the class's systems
    int count;
    int slice;  // shared-memory bytes per group: xa [n_pad] | xb [n_pad] | staged values
    SolveCfg cfg;
};

// SOLVER: 0 = BiCGSTAB, 1 = CG (the uneven path's two solvers).
template <int SOLVER, int L, int R>
__global__ void __launch_bounds__(32, packed_min_blocks(R)) varpacked_kernel(const __grid_constant__ VarPackedParams P) {
    extern __shared__ __align__(16) unsigned char raw[];
    constexpr int G = 32 / L;
    const int lane = threadIdx.x & 31, g = lane / L;
    const int item = blockIdx.x * G + g;
    // groups past the end of the class solve its last system and never write
    const bool valid = item < P.count;
    const int sys = ldg(P.order + (valid ? item : P.count - 1));
    const int pat = ldg(P.sys_pattern + sys);
    const int n = ldg(P.pat_n + pat);
    const int k = ldg(P.tab_k + pat);
    const int64_t toff = ldg(P.tab_off + pat);
    Team tm;
    tm.tid = lane & (L - 1);
    tm.nt = L;
    tm.lane = lane;
    tm.warp = 0;
    tm.nwarps = 1;
    tm.bar = 0;
    const int n_pad = (n + 1) & ~1;
    unsigned char* slice = raw + (size_t)g * P.slice;
    TeamSmem sm;
    sm.red = nullptr;
    sm.xa = reinterpret_cast<double*>(slice);
    sm.xb = sm.xa + n_pad;
    sm.extra = nullptr;
    double* as = reinterpret_cast<double*>(slice + (((size_t)2 * n_pad * 8 + 15) & ~(size_t)15));
    const double* vals = P.values + ldg(P.val_off + sys);
    const int32_t* xsrc = P.xsrc + toff;
    const int count = k * n;
#pragma unroll 4
    for (int i = tm.tid; i < count; i += L) {
        const int src = ldg(xsrc + i);
        if (src >= 0)
            cp_async8(as + i, vals + src);
        else
            as[i] = 0.0;
    }
    cp_async_wait_all();
    PackedOp<FMT_CSR, R> op;
    op.A = Mat<double>{vals, P.row_ptrs + ldg(P.rp_off + pat), P.col_idxs + ldg(P.ci_off + pat), n, 0};
    op.S = Mat<double>{as, nullptr, P.xcols + toff, n, k};
    __syncwarp();
    const int64_t vo = ldg(P.vec_off + sys);
    SysIO io;
    io.b = P.b + vo;
    io.x = P.x + vo;
    io.iters = P.iters + sys;
    io.rel_res = P.rel_res + sys;
    io.status = P.status + sys;
    io.inner = nullptr;
    io.n = n;
    if constexpr (SOLVER == 1)
        cg_packed_system<FMT_CSR, L, R>(op, io, valid, P.cfg, sm, tm);
    else
        bicgstab_packed_system<FMT_CSR, L, R>(op, io, valid, P.cfg, sm, tm);
}

// Kernel of class (L, R) for the solver (0 BiCGSTAB, 1 CG); one table per L.
const void* varpacked_fn(int solver, int L, int R);
const void* varpacked_fn_l4(int solver, int R);
const void* varpacked_fn_l8(int solver, int R);
const void* varpacked_fn_l16(int solver, int R);

}  // namespace bbs
