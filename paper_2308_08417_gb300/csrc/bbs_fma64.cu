// Elementwise fma64_int over device arrays: the check that the integer-pipe
// FP64 FMA equals the hardware fma bit for bit.
#include <cstdint>

#include <cuda_runtime.h>

#include "../../include/bbs.h"
#include "bbs_fma64.cuh"
#include "bbs_internal.h"

namespace bbs {
__global__ void fma64_int_kernel(const double* __restrict__ a, const double* __restrict__ b,
                                 const double* __restrict__ c, double* __restrict__ out, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = fma64_int(a[i], b[i], c[i]);
}
}  // namespace bbs

extern "C" bbs_status bbs_fma64_int(const double* a, const double* b, const double* c, double* out, int64_t n,
                                    void* stream) {
    if (n < 0 || (n > 0 && (!a || !b || !c || !out)))
        return bbs::record_error(BBS_ERR_INVALID_ARG, "null array or negative length");
    if (n == 0) return BBS_OK;
    const int64_t blocks = (n + 255) / 256 < 65536 ? (n + 255) / 256 : 65536;
    bbs::fma64_int_kernel<<<(unsigned)blocks, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(a, b, c, out, n);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? BBS_OK : bbs::record_error(BBS_ERR_CUDA, cudaGetErrorString(e));
}
