// BF16 GEMM on the 5th-generation tensor cores (tcgen05) with the FP32
// accumulator in tensor memory and TMA-fed shared-memory stages:
//   C[m][n] = sum_k A[m*lda + k] * B[n*ldb + k]     (both operands K-major)
// K must be a multiple of 64 and the row strides multiples of 8 elements.
//
// One block of 4 warps computes a 128 x BN tile (BN a multiple of 16, <= 256)
// over the k-tiles [kt0, kt1) of its split (blockIdx.z):
//   * thread 0 of warp 0 is the producer: for each 64-wide k-tile it issues
//     TMA copies (cp.async.bulk.tensor.2d) of eight 16-byte-wide column boxes
//     of A (128 rows) and of B (BN rows) into one of kStages stages, laid out
//     as the no-swizzle K-major "core matrix" canonical form (8 rows x 16
//     bytes per 128-byte core matrix; 8-row groups 128 bytes apart, 16-byte
//     K chunks 16 * rows bytes apart), and arms the stage's "full" mbarrier
//     with the byte count;
//   * thread 0 of warp 1 issues four tcgen05.mma (M = 128, N = BN, K = 16)
//     per k-tile once the stage is full, and tcgen05.commit frees the stage
//     through its "empty" mbarrier; a last commit signals "done";
//   * then every warp reads its 32 accumulator lanes (rows) with tcgen05.ld
//     and runs the epilogue functor epi(m, n, value).
// Rows past M and N are zero-filled by TMA. Every mbarrier wait is bounded;
// a wait that runs out sets *err, the block stops issuing, waits (bounded)
// for the copies and MMAs it already issued, and still frees its tensor
// memory.
#pragma once

#include <cstdint>

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace bbs {
namespace umma {

constexpr int kBM = 128, kBK = 64, kStages = 4;
constexpr int kWaitIters = 1 << 22;

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

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    for (int i = 0; i < kWaitIters; ++i) {
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

// 2D tiled TMA load of box (x = K element offset, y = row) into shared memory,
// completing on mbarrier `bar` (byte count armed by mbar_expect_tx).
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::"r"(
            dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
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

// Dynamic shared memory of a BN-wide tile: kStages stages of A and B, then
// the barriers (full[kStages], empty[kStages], done) and the TMEM slot.
__host__ __device__ constexpr size_t stage_bytes(int BN) { return (size_t)kBM * kBK * 2 + (size_t)BN * kBK * 2; }
__host__ __device__ constexpr size_t smem_bytes(int BN) { return kStages * stage_bytes(BN) + 128 + 1024; }

template <class Epi>
__device__ __forceinline__ void gemm_tn_tma(const CUtensorMap* ta, const CUtensorMap* tb, int M, int N, int K,
                                            int BN, int ktiles_per_split, const Epi& epi, int* err) {
    extern __shared__ unsigned char smem_raw[];
    // TMA destinations and MMA operands: 1024-byte aligned base
    unsigned char* smem = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * BN;
    const int nk = K / kBK;
    const int kt0 = blockIdx.z * ktiles_per_split;
    const int kt1 = min(nk, kt0 + ktiles_per_split);
    const uint32_t a_bytes = kBM * kBK * 2, b_bytes = (uint32_t)BN * kBK * 2;
    const uint32_t sbytes = a_bytes + b_bytes;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kStages * sbytes);
    uint64_t* full = bars;
    uint64_t* empty = bars + kStages;
    uint64_t* done = bars + 2 * kStages;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
    const uint32_t tmem_cols = BN <= 32 ? 32u : BN <= 64 ? 64u : BN <= 128 ? 128u : 256u;
    // K-major no-swizzle layout written by the column boxes
    const uint32_t lbo_a = kBM * 16, lbo_b = (uint32_t)BN * 16, sbo = 128;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(saddr(tmem_slot)),
                     "r"(tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (tid == 32) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(saddr(&full[s]), 1);
            mbar_init(saddr(&empty[s]), 1);
        }
        mbar_init(saddr(done), 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    const uint32_t idesc = idesc_bf16(kBM, BN);
    const uint32_t base = saddr(smem);
    bool ok = true;

    if (tid == 0) {  // producer
        int issued = 0;
        for (int kt = kt0; kt < kt1; ++kt, ++issued) {
            const int s = issued % kStages;
            if (issued >= kStages && !mbar_wait(saddr(&empty[s]), ((issued / kStages) - 1) & 1)) {
                ok = false;
                break;
            }
            const uint32_t a = base + s * sbytes, b = a + a_bytes, fb = saddr(&full[s]);
            mbar_expect_tx(fb, sbytes);
            const int k0 = kt * kBK;
#pragma unroll
            for (int kc = 0; kc < kBK / 8; ++kc) {
                tma_load_2d(a + kc * lbo_a, ta, k0 + 8 * kc, m0, fb);
                tma_load_2d(b + kc * lbo_b, tb, k0 + 8 * kc, n0, fb);
            }
        }
        // the copies of the last (up to kStages) stages land before the block
        // ends, whether or not the MMA side consumed them
        for (int j = issued > kStages ? issued - kStages : 0; j < issued; ++j)
            if (!mbar_wait(saddr(&full[j % kStages]), (j / kStages) & 1)) ok = false;
    } else if (tid == 32) {  // MMA issuer
        int i = 0;
        for (int kt = kt0; kt < kt1; ++kt, ++i) {
            const int s = i % kStages;
            if (!mbar_wait(saddr(&full[s]), (i / kStages) & 1)) {
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            const uint32_t a = base + s * sbytes, b = a + a_bytes;
#pragma unroll
            for (int ks = 0; ks < kBK / 16; ++ks)
                umma_bf16(tmem, smem_desc(a + ks * 2 * lbo_a, lbo_a, sbo), smem_desc(b + ks * 2 * lbo_b, lbo_b, sbo),
                          idesc, (i > 0 || ks > 0) ? 1u : 0u);
            umma_commit(saddr(&empty[s]));
        }
        umma_commit(saddr(done));  // arrives once every MMA issued above has completed
    }
    ok = ok && mbar_wait(saddr(done), 0);
    ok = __syncthreads_and(ok ? 1 : 0) != 0;  // the tensor-memory loads below are warp-collective
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (ok && kt1 > kt0) {
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
    } else if (!ok && tid == 0) {
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
