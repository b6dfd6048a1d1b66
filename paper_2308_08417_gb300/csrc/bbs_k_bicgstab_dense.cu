// bicgstab kernels (plain and Jacobi-folded) instantiated for the DENSE format, R = 1..kMaxR rows per thread.
#include "bbs_kernels.h"
#include "bbs_solvers.cuh"

namespace bbs {
const void* bicgstab_fn_dense(int R) {
    static const void* const kTable[kMaxR] = {
        (const void*)bicgstab_kernel<FMT_DENSE, 1>, (const void*)bicgstab_kernel<FMT_DENSE, 2>,
        (const void*)bicgstab_kernel<FMT_DENSE, 3>, (const void*)bicgstab_kernel<FMT_DENSE, 4>,
        (const void*)bicgstab_kernel<FMT_DENSE, 5>, (const void*)bicgstab_kernel<FMT_DENSE, 6>,
        (const void*)bicgstab_kernel<FMT_DENSE, 7>, (const void*)bicgstab_kernel<FMT_DENSE, 8>};
    return kTable[R - 1];
}
const void* bicgstab_folded_fn_dense(int R) {
    static const void* const kTable[kMaxR] = {
        (const void*)bicgstab_folded_kernel<FMT_DENSE, 1>, (const void*)bicgstab_folded_kernel<FMT_DENSE, 2>,
        (const void*)bicgstab_folded_kernel<FMT_DENSE, 3>, (const void*)bicgstab_folded_kernel<FMT_DENSE, 4>,
        (const void*)bicgstab_folded_kernel<FMT_DENSE, 5>, (const void*)bicgstab_folded_kernel<FMT_DENSE, 6>,
        (const void*)bicgstab_folded_kernel<FMT_DENSE, 7>, (const void*)bicgstab_folded_kernel<FMT_DENSE, 8>};
    return kTable[R - 1];
}
}  // namespace bbs
