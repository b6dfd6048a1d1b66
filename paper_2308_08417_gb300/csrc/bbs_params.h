// Kernel parameter block shared by the host dispatcher and the kernels.
#pragma once

#include <cstddef>
#include <cstdint>

namespace bbs {

struct SolveParams {
    int n, n_pad, k;          // rows, rows rounded up to 2, ELL width / CSR max row
    int num_batch;
    size_t vps;               // values per system
    const int32_t* row_ptrs;  // CSR
    const int32_t* cols;      // CSR nnz / ELL k*n
    const double* values;
    const float* values32;    // mixed mode FP32 copy
    const double* b;
    double* x;
    int32_t* iters;
    double* rel_res;
    int32_t* status;
    int32_t* inner_iters;
    int precond;   // 0 none, 1 Jacobi
    int tol_type;  // 0 absolute, 1 relative
    double tol;
    int max_iters;
    int restart;
    double inner_tol;
    int max_outer;
    int stage;          // stage the system's values in shared memory
    size_t stage_off;   // byte offset of the staged values in dynamic shared memory
    double* ws;         // workspace (GMRES basis when it does not fit in shared memory)
    size_t slice;       // packed kernels: shared-memory bytes per system
    // packed kernels on CSR: the pattern as an ELL column table [xk * n]
    // (column-major, -1 padding), the CSR index of each slot's value (-1
    // padding), and a flag set when a row is longer than xk
    const int32_t* xcols;
    const int32_t* xsrc;
    const int32_t* xflag;
    int xk;
};

}  // namespace bbs
