// FP32 conversion of the values for the mixed mode when the caller supplies
// no FP32 copy, and the per-format kernel-table front ends.
#include "bbs_kernels.h"
#include "bbs_refine.cuh"

namespace bbs {

// Grid-stride conversion, two values per thread per step (16-byte loads).
__global__ void convert_f32_kernel(const double* __restrict__ src, float* __restrict__ dst,
                                   size_t count) {
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    const size_t pairs = count / 2;
    const double2* s2 = reinterpret_cast<const double2*>(src);
    float2* d2 = reinterpret_cast<float2*>(dst);
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < pairs; i += stride) {
        const double2 v = __ldg(s2 + i);
        d2[i] = make_float2((float)v.x, (float)v.y);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && (count & 1)) dst[count - 1] = (float)src[count - 1];
}

cudaError_t launch_convert_f32(const double* src, float* dst, size_t count, cudaStream_t stream) {
    if (count == 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t pairs = (count + 1) / 2;
    size_t blocks = (pairs + 255) / 256;
    const size_t cap = (size_t)(sms > 0 ? sms : 152) * 8;
    if (blocks > cap) blocks = cap;
    convert_f32_kernel<<<(unsigned)blocks, 256, 0, stream>>>(src, dst, count);
    return cudaGetLastError();
}

#define BBS_FRONT(S)                                   \
    const void* S##_fn(int fmt, int R) {               \
        if (fmt == FMT_CSR) return S##_fn_csr(R);      \
        if (fmt == FMT_ELL) return S##_fn_ell(R);      \
        return S##_fn_dense(R);                        \
    }
BBS_FRONT(bicgstab)
BBS_FRONT(bicgstab_folded)
BBS_FRONT(cg)
BBS_FRONT(gmres)
BBS_FRONT(refine)

}  // namespace bbs
