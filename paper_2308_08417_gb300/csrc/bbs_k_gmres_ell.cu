// gmres kernel instantiated for the ELL format, R = 1..kMaxR rows per thread.
#include "bbs_kernels.h"
#include "bbs_solvers.cuh"

namespace bbs {
const void* gmres_fn_ell(int R) {
    static const void* const kTable[kMaxR] = {
        (const void*)gmres_kernel<FMT_ELL, 1>, (const void*)gmres_kernel<FMT_ELL, 2>,
        (const void*)gmres_kernel<FMT_ELL, 3>, (const void*)gmres_kernel<FMT_ELL, 4>,
        (const void*)gmres_kernel<FMT_ELL, 5>, (const void*)gmres_kernel<FMT_ELL, 6>,
        (const void*)gmres_kernel<FMT_ELL, 7>, (const void*)gmres_kernel<FMT_ELL, 8>};
    return kTable[R - 1];
}
}  // namespace bbs
