// The level schedule of ILU(0) on a shared CSR pattern, as the analysis
// kernel (bbs_ilu.cu) leaves it in the workspace.
#pragma once

#include <cstddef>

namespace bbs {

// Workspace layout (int32): nlevL, nlevU, levL_ptr[n+1], rowsL[n],
// levU_ptr[n+1], rowsU[n], diag_pos[n], level scratch[n].
struct IluSchedule {
    const int* levL_ptr;
    const int* rowsL;
    const int* levU_ptr;
    const int* rowsU;
    const int* diag_pos;  // CSR index of a_ii, -1 when the pattern has none
    int nlevL, nlevU;
};

__host__ __device__ inline size_t ilu_schedule_ints(int n) { return 2 + 2 * ((size_t)n + 1) + 4 * (size_t)n; }

// Shared-memory bytes of a packed ILU(0) block's copy of the pattern (n <=
// 160, nnz < 2^15): 16-bit CSR row starts [n], then 8-bit column table [k n]
// (255 past the row end), row lengths [n], diagonal slots [n], lower level
// pointers [n + 1] and rows [n], upper level pointers [n + 1] and rows [n].
__host__ __device__ inline size_t ilu_pattern_smem(int n, int k) {
    return (2 * (size_t)n + (size_t)k * n + 6 * (size_t)n + 2 + 15) & ~(size_t)15;
}

__device__ __forceinline__ IluSchedule ilu_schedule(const int* sched, int n) {
    IluSchedule S;
    S.nlevL = sched[0];
    S.nlevU = sched[1];
    S.levL_ptr = sched + 2;
    S.rowsL = S.levL_ptr + n + 1;
    S.levU_ptr = S.rowsL + n;
    S.rowsU = S.levU_ptr + n + 1;
    S.diag_pos = S.rowsU + n;
    return S;
}

}  // namespace bbs
