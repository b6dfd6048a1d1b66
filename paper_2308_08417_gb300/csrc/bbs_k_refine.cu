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

// The CSR pattern as an ELL column table for the packed kernels: one thread
// per row writes slot j of row r at j n + r (column, and the CSR index of the
// value; -1 past the row's end). A row longer than k sets *flag and keeps
// its first k entries.
__global__ void csr_ell_tables_kernel(int n, int k, const int32_t* __restrict__ row_ptrs,
                                      const int32_t* __restrict__ cols, int32_t* __restrict__ xcols,
                                      int32_t* __restrict__ xsrc, int32_t* __restrict__ flag) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int e0 = row_ptrs[r];
    int len = row_ptrs[r + 1] - e0;
    if (len > k) {
        atomicOr(flag, 1);
        len = k;
    }
    for (int j = 0; j < k; ++j) {
        const size_t i = (size_t)j * n + r;
        xcols[i] = j < len ? cols[e0 + j] : -1;
        xsrc[i] = j < len ? e0 + j : -1;
    }
}

cudaError_t launch_csr_ell_tables(int n, int k, const int32_t* row_ptrs, const int32_t* cols, int32_t* xcols,
                                  int32_t* xsrc, int32_t* flag, cudaStream_t stream) {
    cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(int32_t), stream);
    if (e != cudaSuccess) return e;
    csr_ell_tables_kernel<<<(n + 127) / 128, 128, 0, stream>>>(n, k, row_ptrs, cols, xcols, xsrc, flag);
    return cudaGetLastError();
}

// One thread per row: counts the rows of a shared pattern that break the
// format's rules (see bbs_check_pattern). Every read stays inside the arrays
// whatever they hold.
__global__ void check_pattern_kernel(int fmt, int n, int nnz, int k, const int32_t* __restrict__ rp,
                                     const int32_t* __restrict__ cols, int* __restrict__ bad) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    bool ok = true;
    if (fmt == FMT_CSR) {
        const int e0 = rp[i], e1 = rp[i + 1];
        if (i == 0 && e0 != 0) ok = false;
        if (i == n - 1 && e1 != nnz) ok = false;
        if (e0 < 0 || e1 < e0 || e1 > nnz) {
            ok = false;
        } else {
            if (k > 0 && e1 - e0 > k) ok = false;
            int prev = -1;
            for (int e = e0; e < e1; ++e) {
                const int c = cols[e];
                if (c < 0 || c >= n || c <= prev) ok = false;
                prev = c;
            }
        }
    } else if (fmt == FMT_ELL) {
        int prev = -1;
        bool padded = false;
        for (int j = 0; j < k; ++j) {
            const int c = cols[(size_t)j * n + i];
            if (c == -1) {
                padded = true;
                continue;
            }
            if (padded || c < 0 || c >= n || c <= prev) ok = false;
            prev = c;
        }
    }
    if (!ok) atomicAdd(bad, 1);
}

cudaError_t launch_check_pattern(int fmt, int n, int nnz, int k, const int32_t* rp, const int32_t* cols,
                                 int* bad, cudaStream_t stream) {
    check_pattern_kernel<<<(n + 127) / 128, 128, 0, stream>>>(fmt, n, nnz, k, rp, cols, bad);
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

#define BBS_PACKED_FRONT(S)                                                                  \
    const void* S##_packed_fn(int fmt, int L, int R) {                                       \
        if (fmt == FMT_CSR)                                                                  \
            return L == 4 ? S##_packed_fn_csr_l4(R) : L == 8 ? S##_packed_fn_csr_l8(R)       \
                                                             : S##_packed_fn_csr_l16(R);     \
        if (fmt == FMT_ELL)                                                                  \
            return L == 4 ? S##_packed_fn_ell_l4(R) : L == 8 ? S##_packed_fn_ell_l8(R)       \
                                                             : S##_packed_fn_ell_l16(R);     \
        return L == 4 ? S##_packed_fn_dense_l4(R) : L == 8 ? S##_packed_fn_dense_l8(R)       \
                                                           : S##_packed_fn_dense_l16(R);     \
    }
BBS_PACKED_FRONT(bicgstab)
BBS_PACKED_FRONT(cg)
BBS_PACKED_FRONT(gmres)
#undef BBS_PACKED_FRONT

}  // namespace bbs
