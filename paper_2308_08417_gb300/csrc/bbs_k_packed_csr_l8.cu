// Packed BiCGSTAB, CG and GMRES kernels (32 / L systems per warp), CSR format,
// L = 8 lanes per system, R = 1..kMaxPackedR rows per lane.
#include "bbs_kernels.h"
#include "bbs_packed.cuh"

namespace bbs {
#define BBS_TABLE(K)                                                                          \
    static const void* const kTable[kMaxPackedR] = {                                         \
        (const void*)K<FMT_CSR, 8, 1>, (const void*)K<FMT_CSR, 8, 2>, (const void*)K<FMT_CSR, 8, 3>,   \
        (const void*)K<FMT_CSR, 8, 4>, (const void*)K<FMT_CSR, 8, 5>, (const void*)K<FMT_CSR, 8, 6>,   \
        (const void*)K<FMT_CSR, 8, 7>, (const void*)K<FMT_CSR, 8, 8>, (const void*)K<FMT_CSR, 8, 9>,   \
        (const void*)K<FMT_CSR, 8, 10>};                                                   \
    return kTable[R - 1];
static_assert(kMaxPackedR == 10, "tables cover R = 1..10");
const void* bicgstab_packed_fn_csr_l8(int R) { BBS_TABLE(bicgstab_packed_kernel) }
const void* gmres_packed_fn_csr_l8(int R) { BBS_TABLE(gmres_packed_kernel) }
const void* cg_packed_fn_csr_l8(int R) { BBS_TABLE(cg_packed_kernel) }
#undef BBS_TABLE
}  // namespace bbs
