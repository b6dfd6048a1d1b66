// bbs_fma_rate: the measured FP64 or FP32 FMA throughput of the device.
//
// The paper judges its solvers against each GPU's FP64 peak (Table "GPUs
// specifications") and places them on a roofline (Sec. "Roofline analysis").
// On GB300 the FP64 pipe, not HBM, is the roof of the FP64 solvers, and a
// datasheet figure is only nominal, so the library measures the rate it
// reports fractions against: every SM runs 8 blocks of 256 threads, each
// thread 8 independent FMA chains a <- a * m + c (m just below 1, so the
// values settle near c / (1 - m) and stay normal), timed with CUDA events.
#include <cstdio>

#include <cuda_runtime.h>

#include "../../include/bbs.h"
#include "bbs_internal.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 8;

__device__ double g_sink64;
__device__ float g_sink32;

template <typename T>
__global__ void __launch_bounds__(kThreads) fma_chain_kernel(int iters, T m, T c) {
    T a[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) a[j] = T(threadIdx.x + j) * T(1e-3);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < kChains; ++j) a[j] = fma(a[j], m, c);
    }
    T s = T(0);
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += a[j];
    if (s == T(-1)) {  // never true: keeps the chains from being removed
        if constexpr (sizeof(T) == 8)
            g_sink64 = s;
        else
            g_sink32 = s;
    }
}

template <typename T>
cudaError_t timed(int sms, int iters, cudaStream_t st, float* ms) {
    const dim3 grid((unsigned)(sms * kBlocksPerSm));
    const T m = T(0.999999), c = T(1e-6);
    fma_chain_kernel<T><<<grid, kThreads, 0, st>>>(iters / 8 + 1, m, c);  // warm-up
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if ((e = cudaEventCreate(&e0)) != cudaSuccess) return e;
    if ((e = cudaEventCreate(&e1)) != cudaSuccess) {
        cudaEventDestroy(e0);
        return e;
    }
    cudaEventRecord(e0, st);
    fma_chain_kernel<T><<<grid, kThreads, 0, st>>>(iters, m, c);
    e = cudaGetLastError();
    cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return e;
}

}  // namespace

extern "C" bbs_status bbs_fma_rate(bbs_handle* handle, int32_t precision, double* flop_per_s) {
    if (handle == nullptr || flop_per_s == nullptr)
        return bbs::record_error(BBS_ERR_INVALID_ARG, "null handle or output");
    if (precision != 0 && precision != 1)
        return bbs::record_error(BBS_ERR_INVALID_ARG, "precision must be 0 (FP64) or 1 (FP32)");
    const int device = bbs::handle_device(handle);
    cudaError_t e = cudaSetDevice(device);
    int sms = 0;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    cudaStream_t st = nullptr;
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    // about 30 ms per timed launch at GB300's rates (FP64 ~0.5 T FMA/s, FP32 ~40 T)
    const int iters = precision == 0 ? 4096 : 262144;
    float ms = 0.0f;
    if (e == cudaSuccess) e = precision == 0 ? timed<double>(sms, iters, st, &ms) : timed<float>(sms, iters, st, &ms);
    if (st != nullptr) cudaStreamDestroy(st);
    if (e != cudaSuccess) {
        char msg[256];
        snprintf(msg, sizeof msg, "FMA rate probe: %s", cudaGetErrorString(e));
        return bbs::record_error(BBS_ERR_CUDA, msg);
    }
    const double fmas = (double)sms * kBlocksPerSm * kThreads * kChains * (double)iters;
    *flop_per_s = 2.0 * fmas / (ms * 1e-3);
    return BBS_OK;
}
