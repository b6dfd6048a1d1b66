// Uneven-batch persistent kernel, up to 8 rows per thread.
#include "bbs_varsize.cuh"

namespace bbs {
const void* varsize_kernel8_fn() { return (const void*)varsize_kernel<8>; }
}  // namespace bbs
