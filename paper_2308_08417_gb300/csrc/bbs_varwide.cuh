// Uneven batches, wide teams: systems solved one per block with 9 to 16 rows
// per thread, each a launch of its own beside the persistent team launch.
//
// On GB300 the FP64 pipe bounds these solvers, and a team with fewer warps
// spends less of each iteration in block barriers: for a batch of n = 784
// systems, 2 warps at 13 rows per thread ran 19 % faster than 4 warps at 7 (the
// same register budget per SM). The persistent kernel holds every team size
// and rows-per-thread variant in one kernel, which limits it to 8 rows per
// thread (each further variant roughly doubles its compile time). Systems of
// a bucket marked wide (bbs_var_tuning.wide) that need more than 8 rows per
// thread on their fewest warps run here instead: the planner groups them by
// (warps, rows per thread), and each group is one launch of
// varwide_kernel<R> with one block of 32, 64 or 128 threads per system, in the
// plan's CUDA graph beside the other launches. The solver is the Jacobi-folded
// BiCGSTAB of the team kernels (values staged in shared memory).
#pragma once

#include <cstdint>

#include "bbs_solvers.cuh"

namespace bbs {

constexpr int kVarWideMinR = 9;
constexpr int kVarWideMaxR = 16;

struct VarWideParams {
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
    const int32_t* order;  // the group's systems, one per block
    int count;
    SolveCfg cfg;
};

// Block area: red [256 doubles] | xa [n_pad] | xb [n_pad] | staged values.
template <int R>
__global__ void __launch_bounds__(128, 1) varwide_kernel(const __grid_constant__ VarWideParams P) {
    extern __shared__ __align__(16) unsigned char raw[];
    const Team tm = Team::block();
    const int sys = ldg(P.order + blockIdx.x);
    const int pat = ldg(P.sys_pattern + sys);
    const int n = ldg(P.pat_n + pat);
    const int nnz = ldg(P.pat_nnz + pat);
    const Mat<double> A{P.values + ldg(P.val_off + sys), P.row_ptrs + ldg(P.rp_off + pat),
                        P.col_idxs + ldg(P.ci_off + pat), n, 0};
    const int64_t vo = ldg(P.vec_off + sys);
    SysIO io;
    io.b = P.b + vo;
    io.x = P.x + vo;
    io.iters = P.iters + sys;
    io.rel_res = P.rel_res + sys;
    io.status = P.status + sys;
    io.inner = nullptr;
    io.n = n;
    const TeamSmem sm = team_smem(raw, (n + 1) & ~1);
    const auto op = make_op<FMT_CSR, R>(A, (size_t)nnz, sm.extra, tm);
    bicgstab_scaled_system<FMT_CSR, R>(op, io, P.cfg, sm, tm);
}

// Shared-memory bytes of a wide block for a system of n rows and nnz values.
__host__ __device__ constexpr size_t varwide_smem(int n, int nnz) {
    return (256 + 2 * (size_t)((n + 1) & ~1)) * 8 + (((size_t)nnz * 8 + 15) & ~(size_t)15);
}

// Kernel of R rows per thread (kVarWideMinR..kVarWideMaxR).
const void* varwide_fn(int R);
const void* varwide_fn_lo(int R);
const void* varwide_fn_hi(int R);

}  // namespace bbs
