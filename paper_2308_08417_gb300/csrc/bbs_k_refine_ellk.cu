// refine kernel for ELL batches with staged values and an ELL width fixed at
// compile time: K = 3, 5, 7, 9 (1D 3-point, 2D 5-point, 3D 7-point and 2D
// 9-point stencils) at R = 1..4 rows per thread, the mixed mode's default
// launch shapes.
#include "bbs_kernels.h"
#include "bbs_refine.cuh"

namespace bbs {
const void* refine_ell_fn(int R, int K) {
#define BBS_ROW(K_) {(const void*)refine_kernel<FMT_ELL, 1, K_>, (const void*)refine_kernel<FMT_ELL, 2, K_>, \
                     (const void*)refine_kernel<FMT_ELL, 3, K_>, (const void*)refine_kernel<FMT_ELL, 4, K_>}
    static const void* const kTable[4][4] = {BBS_ROW(3), BBS_ROW(5), BBS_ROW(7), BBS_ROW(9)};
#undef BBS_ROW
    if (R < 1 || R > 4 || K < 3 || K > 9 || (K & 1) == 0) return nullptr;
    return kTable[(K - 3) / 2][R - 1];
}
}  // namespace bbs
