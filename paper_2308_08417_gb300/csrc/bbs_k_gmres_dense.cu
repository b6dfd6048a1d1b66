// gmres kernel instantiated for the DENSE format, R = 1..kMaxR rows per thread.
#include "bbs_kernels.h"
#include "bbs_solvers.cuh"

namespace bbs {
const void* gmres_fn_dense(int R) {
    static const void* const kTable[kMaxR] = {
        (const void*)gmres_kernel<FMT_DENSE, 1>, (const void*)gmres_kernel<FMT_DENSE, 2>,
        (const void*)gmres_kernel<FMT_DENSE, 3>, (const void*)gmres_kernel<FMT_DENSE, 4>,
        (const void*)gmres_kernel<FMT_DENSE, 5>, (const void*)gmres_kernel<FMT_DENSE, 6>,
        (const void*)gmres_kernel<FMT_DENSE, 7>, (const void*)gmres_kernel<FMT_DENSE, 8>};
    return kTable[R - 1];
}
}  // namespace bbs
