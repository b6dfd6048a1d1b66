// bicgstab kernels (plain and Jacobi-folded) instantiated for the ELL format, R = 1..kMaxR rows per thread.
#include "bbs_kernels.h"
#include "bbs_solvers.cuh"

namespace bbs {
const void* bicgstab_fn_ell(int R) {
    static const void* const kTable[kMaxR] = {
        (const void*)bicgstab_kernel<FMT_ELL, 1>, (const void*)bicgstab_kernel<FMT_ELL, 2>,
        (const void*)bicgstab_kernel<FMT_ELL, 3>, (const void*)bicgstab_kernel<FMT_ELL, 4>,
        (const void*)bicgstab_kernel<FMT_ELL, 5>, (const void*)bicgstab_kernel<FMT_ELL, 6>,
        (const void*)bicgstab_kernel<FMT_ELL, 7>, (const void*)bicgstab_kernel<FMT_ELL, 8>};
    return kTable[R - 1];
}
const void* bicgstab_folded_fn_ell(int R) {
    static const void* const kTable[kMaxR] = {
        (const void*)bicgstab_folded_kernel<FMT_ELL, 1>, (const void*)bicgstab_folded_kernel<FMT_ELL, 2>,
        (const void*)bicgstab_folded_kernel<FMT_ELL, 3>, (const void*)bicgstab_folded_kernel<FMT_ELL, 4>,
        (const void*)bicgstab_folded_kernel<FMT_ELL, 5>, (const void*)bicgstab_folded_kernel<FMT_ELL, 6>,
        (const void*)bicgstab_folded_kernel<FMT_ELL, 7>, (const void*)bicgstab_folded_kernel<FMT_ELL, 8>};
    return kTable[R - 1];
}
}  // namespace bbs
