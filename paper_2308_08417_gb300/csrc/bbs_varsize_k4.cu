// Uneven-batch persistent kernel, up to 4 rows per thread.
#include "bbs_varsize.cuh"

namespace bbs {
const void* varsize_kernel4_fn() { return (const void*)varsize_kernel<4>; }
}  // namespace bbs
