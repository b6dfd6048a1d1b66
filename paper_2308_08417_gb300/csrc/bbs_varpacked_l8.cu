// Uneven batches: packed small-system kernels with L = 8 lanes per system,
// R = 1..kMaxPackedR rows per lane, for BiCGSTAB and CG.
#include "bbs_varpacked.cuh"

namespace bbs {
#define BBS_ROW(S)                                                                                    \
    {(const void*)varpacked_kernel<S, 8, 1>, (const void*)varpacked_kernel<S, 8, 2>,                  \
     (const void*)varpacked_kernel<S, 8, 3>, (const void*)varpacked_kernel<S, 8, 4>,                  \
     (const void*)varpacked_kernel<S, 8, 5>, (const void*)varpacked_kernel<S, 8, 6>,                  \
     (const void*)varpacked_kernel<S, 8, 7>, (const void*)varpacked_kernel<S, 8, 8>,                  \
     (const void*)varpacked_kernel<S, 8, 9>, (const void*)varpacked_kernel<S, 8, 10>}
static_assert(kMaxPackedR == 10, "tables cover R = 1..10");
const void* varpacked_fn_l8(int solver, int R) {
    static const void* const kTable[2][kMaxPackedR] = {BBS_ROW(0), BBS_ROW(1)};
    return kTable[solver == 1 ? 1 : 0][R - 1];
}
#undef BBS_ROW
}  // namespace bbs
