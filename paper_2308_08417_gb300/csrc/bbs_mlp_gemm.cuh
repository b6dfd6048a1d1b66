// BF16 GEMM with FP32 accumulation for the MLP:
//   C[m][n] = sum_k A[m*lda + k] * B[n*ldb + k]
// Both operands are K-contiguous ("TN"); K must be a multiple of 32 and the
// row strides multiples of 8 elements (16-byte rows for cp.async). Rows of A
// beyond M and of B beyond N are zero-filled. Each result goes through the
// epilogue functor epi(m, n, value) (bias, activation, transposed stores).
//
// Tiles: 128 x 64 x 32 per block of 8 warps (4 x 2), each warp a 32 x 32
// sub-tile of mma.sync m16n8k16 (BF16 in, FP32 accumulate); two shared-memory
// stages filled with cp.async.
#pragma once

#include <cstdint>

#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace bbs {
namespace mlp {

constexpr int kBM = 128, kBN = 64, kBK = 32, kSkew = 8;

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, int src_bytes) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(src_bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

__device__ __forceinline__ void ldmatrix_x4(uint32_t (&r)[4], const void* p) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(s));
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, "
        "{%8, %9}, {%0, %1, %2, %3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

template <class Epi>
__device__ __forceinline__ void gemm_tn_mma(const __nv_bfloat16* __restrict__ A, int lda,
                                            const __nv_bfloat16* __restrict__ B, int ldb, int M, int N,
                                            int K, const Epi& epi) {
    __shared__ __align__(16) __nv_bfloat16 As[2][kBM][kBK + kSkew];
    __shared__ __align__(16) __nv_bfloat16 Bs[2][kBN][kBK + kSkew];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int wm = warp >> 1, wn = warp & 1;
    const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * kBN;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.0f;

    auto load = [&](int stage, int k0) {
#pragma unroll
        for (int c = tid; c < kBM * 4; c += 256) {
            const int r = c >> 2, cc = (c & 3) * 8;
            const int gm = m0 + r;
            const __nv_bfloat16* src = A + (size_t)(gm < M ? gm : 0) * lda + k0 + cc;
            cp_async16(&As[stage][r][cc], src, gm < M ? 16 : 0);
        }
        {
            const int r = tid >> 2, cc = (tid & 3) * 8;
            const int gn = n0 + r;
            const __nv_bfloat16* src = B + (size_t)(gn < N ? gn : 0) * ldb + k0 + cc;
            cp_async16(&Bs[stage][r][cc], src, gn < N ? 16 : 0);
        }
        cp_async_commit();
    };

    const int nk = K / kBK;
    load(0, 0);
    for (int kt = 0; kt < nk; ++kt) {
        if (kt + 1 < nk) {
            load((kt + 1) & 1, (kt + 1) * kBK);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        const int st = kt & 1;
#pragma unroll
        for (int kk = 0; kk < kBK; kk += 16) {
            uint32_t a[2][4], b[4][2];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int row = wm * 32 + i * 16 + (lane & 15);
                const int col = kk + (lane >> 4) * 8;
                ldmatrix_x4(a[i], &As[st][row][col]);
            }
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int row = wn * 32 + j * 16 + (lane & 7) + ((lane >> 4) << 3);
                const int col = kk + ((lane >> 3) & 1) * 8;
                uint32_t r4[4];
                ldmatrix_x4(r4, &Bs[st][row][col]);
                b[2 * j][0] = r4[0];
                b[2 * j][1] = r4[1];
                b[2 * j + 1][0] = r4[2];
                b[2 * j + 1][1] = r4[3];
            }
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], a[i], b[j][0], b[j][1]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int m = m0 + wm * 32 + i * 16 + (lane >> 2) + h * 8;
                const int n = n0 + wn * 32 + j * 8 + (lane & 3) * 2;
                if (m < M) {
                    if (n < N) epi(m, n, acc[i][j][2 * h]);
                    if (n + 1 < N) epi(m, n + 1, acc[i][j][2 * h + 1]);
                }
            }
}

}  // namespace mlp
}  // namespace bbs
