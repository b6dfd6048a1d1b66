// Kernel tables: one instantiation per (format, rows per thread R = 1..kMaxR).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace bbs {

constexpr int kMaxR = 8;

// Largest block a kernel with R rows per thread is compiled for. The bound
// sets the register budget (65536 / threads, with one block per SM assumed):
// 64 registers hold one row of every working vector, 128 hold R <= 4, 255
// hold R <= 8. The largest system is therefore 2048 rows (the paper targets
// 10 to 2,000 rows, Sec. 2.1).
__host__ __device__ constexpr int max_threads_for(int R) { return R <= 1 ? 1024 : R <= 4 ? 512 : 256; }
constexpr int kMaxRows = 2048;

#define BBS_DECL(S)                  \
    const void* S##_fn(int fmt, int R);  \
    const void* S##_fn_csr(int R);       \
    const void* S##_fn_ell(int R);       \
    const void* S##_fn_dense(int R);
BBS_DECL(bicgstab)
BBS_DECL(bicgstab_folded)
BBS_DECL(cg)
BBS_DECL(gmres)
BBS_DECL(refine)
#undef BBS_DECL
// Mixed-mode refinement on ELL with staged values, ELL width K in {3, 5, 7, 9}
// fixed at compile time, R = 1..4; nullptr for other (R, K).
const void* refine_ell_fn(int R, int K);

// Packed BiCGSTAB, CG and GMRES (32 / L systems per warp): L = 4, 8 or 16
// lanes per system, R = 1..kMaxPackedR rows per lane.
constexpr int kMaxPackedR = 10;
#define BBS_DECL_PACKED(S)                       \
    const void* S##_packed_fn(int fmt, int L, int R); \
    const void* S##_packed_fn_csr_l4(int R);          \
    const void* S##_packed_fn_csr_l8(int R);          \
    const void* S##_packed_fn_csr_l16(int R);         \
    const void* S##_packed_fn_ell_l4(int R);          \
    const void* S##_packed_fn_ell_l8(int R);          \
    const void* S##_packed_fn_ell_l16(int R);         \
    const void* S##_packed_fn_dense_l4(int R);        \
    const void* S##_packed_fn_dense_l8(int R);        \
    const void* S##_packed_fn_dense_l16(int R);
BBS_DECL_PACKED(bicgstab)
BBS_DECL_PACKED(cg)
BBS_DECL_PACKED(gmres)
#undef BBS_DECL_PACKED

cudaError_t launch_check_pattern(int fmt, int n, int nnz, int k, const int32_t* rp, const int32_t* cols,
                                 int* bad, cudaStream_t stream);
cudaError_t launch_csr_ell_tables(int n, int k, const int32_t* row_ptrs, const int32_t* cols, int32_t* xcols,
                                  int32_t* xsrc, int32_t* flag, cudaStream_t stream);

const void* bicgstab_ilu_fn(int R);
// Packed BiCGSTAB + ILU(0) on CSR (L = 4, 8, 16 lanes per system).
const void* bicgstab_ilu_packed_fn(int L, int R);
const void* bicgstab_ilu_packed_fn_l4(int R);
const void* bicgstab_ilu_packed_fn_l8(int R);
const void* bicgstab_ilu_packed_fn_l16(int R);
size_t ilu_workspace_bytes(int n);
cudaError_t launch_ilu_analysis(int n, const int32_t* row_ptrs, const int32_t* col_idxs, int* ws,
                                cudaStream_t stream);
cudaError_t launch_convert_f32(const double* src, float* dst, size_t count, cudaStream_t stream);

}  // namespace bbs
