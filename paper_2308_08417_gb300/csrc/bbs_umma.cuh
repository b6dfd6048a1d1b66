// BF16 GEMM on the 5th-generation tensor cores (tcgen05) with the FP32
// accumulator in tensor memory:
//   C[m][n] = sum_k A[m*lda + k] * B[n*ldb + k]     (both operands K-major)
// K must be a multiple of 64 and the row strides multiples of 8 elements.
//
// One block of 4 warps computes a 128 x BN tile (BN a multiple of 16, <= 256):
//   * all threads stage 128x64 A and BNx64 B k-tiles into shared memory with
//     cp.async, two stages, in the no-swizzle K-major "core matrix" layout
//     (8 rows x 16 bytes per 128-byte core matrix; core matrices adjacent in
//     K are 128 bytes apart, 8-row groups 1024 bytes apart);
//   * thread 0 issues four tcgen05.mma (M=128, N=BN, K=16 each) per k-tile
//     and commits them to the stage's mbarrier, which frees the stage;
//   * after the last commit every warp reads its 32 accumulator lanes (rows)
//     with tcgen05.ld and runs the epilogue functor epi(m, n, value).
// Every mbarrier wait is bounded; a wait that runs out sets *err, skips the
// remaining work and still releases the tensor memory.
#pragma once

#include <cstdint>

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "bbs_mlp_gemm.cuh"

namespace bbs {
namespace umma {

constexpr int kBM = 128, kBK = 64;

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor (tcgen05): start address, leading-dimension
// byte offset (K direction), stride-dimension byte offset (M/N direction),
// descriptor version 1, base offset 0, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Byte offset of 16-byte chunk `kc` (8 elements along K) of row `r` in a
// tile stored as 8-row groups of core matrices, 8 chunks per row (K = 64).
__device__ __forceinline__ uint32_t core_off(int r, int kc) {
    return (uint32_t)((((r >> 3) * 8 + kc) << 7) + ((r & 7) << 4));
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    for (int i = 0; i < (1 << 22); ++i) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void umma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
        "%12, %13, %14, %15}, [%16];\n"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
          "=r"(v[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
}

// Dynamic shared memory the kernel needs for a BN-wide tile.
__host__ __device__ constexpr size_t smem_bytes(int BN) {
    return 2 * ((size_t)kBM * kBK * 2 + (size_t)BN * kBK * 2) + 64;
}

template <class Epi>
__device__ __forceinline__ void gemm_tn_umma(const __nv_bfloat16* __restrict__ A, int lda,
                                             const __nv_bfloat16* __restrict__ B, int ldb, int M, int N,
                                             int K, int BN, const Epi& epi, int* err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * BN;
    const uint32_t a_bytes = kBM * kBK * 2, b_bytes = (uint32_t)BN * kBK * 2;
    const uint32_t stage_bytes = a_bytes + b_bytes;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + 2 * stage_bytes);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mbar + 2);
    const uint32_t tmem_cols = BN <= 32 ? 32u : BN <= 64 ? 64u : BN <= 128 ? 128u : 256u;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(saddr(tmem_slot)),
                     "r"(tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(saddr(&mbar[0])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(saddr(&mbar[1])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    const uint32_t idesc = idesc_bf16(kBM, BN);

    auto load = [&](int s, int kt) {
        unsigned char* a = smem + s * stage_bytes;
        unsigned char* b = a + a_bytes;
        const int k0 = kt * kBK;
        for (int c = tid; c < kBM * 8; c += 128) {
            const int r = c >> 3, kc = c & 7, gm = m0 + r;
            mlp::cp_async16(a + core_off(r, kc), A + (size_t)(gm < M ? gm : 0) * lda + k0 + kc * 8, gm < M ? 16 : 0);
        }
        for (int c = tid; c < BN * 8; c += 128) {
            const int r = c >> 3, kc = c & 7, gn = n0 + r;
            mlp::cp_async16(b + core_off(r, kc), B + (size_t)(gn < N ? gn : 0) * ldb + k0 + kc * 8, gn < N ? 16 : 0);
        }
        mlp::cp_async_commit();
    };

    const int nk = K / kBK;
    uint32_t phase[2] = {0u, 0u};
    bool ok = true;
    load(0, 0);
    for (int kt = 0; kt < nk; ++kt) {
        const int s = kt & 1;
        if (kt + 1 < nk) {
            if (kt >= 1) {  // the other stage is free once the MMAs of k-tile kt-1 completed
                ok = ok && mbar_wait(saddr(&mbar[s ^ 1]), phase[s ^ 1]);
                phase[s ^ 1] ^= 1u;
            }
            load(s ^ 1, kt + 1);
            mlp::cp_async_wait<1>();
        } else {
            mlp::cp_async_wait<0>();
        }
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        __syncthreads();
        if (tid == 0 && ok) {
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            const uint32_t a_addr = saddr(smem + s * stage_bytes), b_addr = a_addr + a_bytes;
#pragma unroll
            for (int ks = 0; ks < kBK / 16; ++ks)
                umma_bf16(tmem, smem_desc(a_addr + ks * 256, 128, 1024), smem_desc(b_addr + ks * 256, 128, 1024),
                          idesc, (kt > 0 || ks > 0) ? 1u : 0u);
            umma_commit(saddr(&mbar[s]));
        }
    }
    {
        const int s = (nk - 1) & 1;  // completion of the last commit covers all earlier MMAs
        ok = ok && mbar_wait(saddr(&mbar[s]), phase[s]);
    }
    ok = __syncthreads_and(ok ? 1 : 0) != 0;  // the tensor-memory loads below are warp-collective
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (ok) {
        const int m = m0 + warp * 32 + lane;
        for (int c0 = 0; c0 < BN; c0 += 16) {
            uint32_t v[16];
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
            if (m < M) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int n = n0 + c0 + j;
                    if (n < N && c0 + j < BN) epi(m, n, __uint_as_float(v[j]));
                }
            }
        }
    } else if (tid == 0) {
        atomicExch(err, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(tmem_cols)
                     : "memory");
}

}  // namespace umma
}  // namespace bbs
