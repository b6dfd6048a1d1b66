// Uneven batches: wide-team kernels with 9..12 rows per thread.
#include "bbs_varwide.cuh"

namespace bbs {
const void* varwide_fn_lo(int R) {
    static const void* const kTable[4] = {(const void*)varwide_kernel<9>, (const void*)varwide_kernel<10>,
                                          (const void*)varwide_kernel<11>, (const void*)varwide_kernel<12>};
    return kTable[R - 9];
}
}  // namespace bbs
