// bicgstab kernels (plain and Jacobi-folded) instantiated for the CSR format, R = 1..kMaxR rows per thread.
#include "bbs_kernels.h"
#include "bbs_solvers.cuh"

namespace bbs {
const void* bicgstab_fn_csr(int R) {
    static const void* const kTable[kMaxR] = {
        (const void*)bicgstab_kernel<FMT_CSR, 1>, (const void*)bicgstab_kernel<FMT_CSR, 2>,
        (const void*)bicgstab_kernel<FMT_CSR, 3>, (const void*)bicgstab_kernel<FMT_CSR, 4>,
        (const void*)bicgstab_kernel<FMT_CSR, 5>, (const void*)bicgstab_kernel<FMT_CSR, 6>,
        (const void*)bicgstab_kernel<FMT_CSR, 7>, (const void*)bicgstab_kernel<FMT_CSR, 8>};
    return kTable[R - 1];
}
const void* bicgstab_folded_fn_csr(int R) {
    static const void* const kTable[kMaxR] = {
        (const void*)bicgstab_folded_kernel<FMT_CSR, 1>, (const void*)bicgstab_folded_kernel<FMT_CSR, 2>,
        (const void*)bicgstab_folded_kernel<FMT_CSR, 3>, (const void*)bicgstab_folded_kernel<FMT_CSR, 4>,
        (const void*)bicgstab_folded_kernel<FMT_CSR, 5>, (const void*)bicgstab_folded_kernel<FMT_CSR, 6>,
        (const void*)bicgstab_folded_kernel<FMT_CSR, 7>, (const void*)bicgstab_folded_kernel<FMT_CSR, 8>};
    return kTable[R - 1];
}
}  // namespace bbs
