// Uneven batches: wide-team kernels with 13..16 rows per thread.
#include "bbs_varwide.cuh"

namespace bbs {
const void* varwide_fn_hi(int R) {
    static const void* const kTable[4] = {(const void*)varwide_kernel<13>, (const void*)varwide_kernel<14>,
                                          (const void*)varwide_kernel<15>, (const void*)varwide_kernel<16>};
    return kTable[R - 13];
}
}  // namespace bbs
