// Packed BiCGSTAB + ILU(0) kernels (32 / L systems per warp), CSR, L = 4
// lanes per system, R = 1..kMaxPackedR rows per lane.
#include "bbs_ilu_packed.cuh"
#include "bbs_kernels.h"

namespace bbs {
#define BBS_P(R) (const void*)bicgstab_ilu_packed_kernel<4, R>
const void* bicgstab_ilu_packed_fn_l4(int R) {
    static_assert(kMaxPackedR == 10, "table covers R = 1..10");
    static const void* const kTable[kMaxPackedR] = {BBS_P(1), BBS_P(2), BBS_P(3), BBS_P(4), BBS_P(5),
                                                    BBS_P(6), BBS_P(7), BBS_P(8), BBS_P(9), BBS_P(10)};
    return kTable[R - 1];
}
#undef BBS_P
}  // namespace bbs
