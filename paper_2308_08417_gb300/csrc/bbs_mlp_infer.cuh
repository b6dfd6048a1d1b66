// Fused inference of the initial-guess network: one kernel runs all four
// layers for a tile of 128 systems, with the activations in shared memory and
// the accumulator in tensor memory between the layers.
//
// Per block (10 warps):
//   * warps 0-7 (256 threads) assemble the tile's standardised BF16 features
//     [diag(A), b, x_prev] with coalesced loads straight into the K-major
//     no-swizzle core-matrix layout the MMAs read (8 rows x 16 bytes per core
//     matrix, 16-byte K chunks 128 * 16 bytes apart), then run every
//     epilogue: thread (warp w,
//     lane l) owns TMEM lane / tile row 32 (w % 4) + l and every other
//     16-column chunk (w / 4 picks which). Hidden layers: bias + GELU, BF16,
//     written back over the layer's own input (its MMAs have completed).
//     Output layer: bias, staged as FP32 in shared memory, then a coalesced
//     pass writes x0 = x_prev + gamma (out * sigma + mu), or accumulates the
//     gate statistics sum c.d and sum c.c (c = out * sigma + mu, d = x_next -
//     x_prev) into acc.
//   * warp 8, one lane: streams every layer's weights through a ring of
//     kInferStages stages, each a 64-wide K tile of W_l [N_l, K_l] copied by
//     TMA (eight 16-byte-wide column boxes) with an mbarrier armed by bytes.
//   * warp 9 allocates the tensor memory; one lane issues the MMAs: per K
//     tile four tcgen05.mma kind::f16 (M = 128, N = N_l, K = 16) into the
//     FP32 accumulator, a commit that frees the stage, and after each layer a
//     commit to "accumulator ready".
// Handshakes: act_ready (256 arrivals: the layer's BF16 input is in shared
// memory, fenced to the async proxy) and acc_ready (one commit per layer).
// Every wait is bounded; a wait that runs out sets *err, the role stops, and
// the block still waits (bounded) for its copies and MMAs before it frees the
// tensor memory.
#pragma once

#include <cstdint>

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "bbs_umma.cuh"

namespace bbs {
namespace mlp {

constexpr int kInferRows = 128;
constexpr int kInferStages = 3;
constexpr int kInferEpiWarps = 8;
constexpr int kInferThreads = (kInferEpiWarps + 2) * 32;

struct InferParams {
    int num_batch, n, nnz, in_pad, hidden, n_mma;
    const int32_t* row_ptrs;
    const int32_t* cols;
    const double* values;
    const double* b;
    const double* xp;
    const double* xn;  // gate mode: x_next
    double* x0;        // predict mode: output
    double* acc;       // gate mode: [sum c.d, sum c.c]
    const float* bias[4];
    const float* mean;
    const float* inv_std;
    const float* stdv;
    const double* gamma;
    int* err;
};

// Shared-memory layout of the fused kernel, from a 1024-byte aligned base.
struct InferSmem {
    size_t act, stage, stage_bytes, bars, dpos, bias, total;
};

__host__ __device__ inline InferSmem infer_smem(int n, int in_pad, int hidden, int n_mma) {
    InferSmem s;
    const int act_k = in_pad > hidden ? in_pad : hidden;
    size_t act_bytes = (size_t)kInferRows * act_k * 2;
    const size_t out_bytes = (size_t)kInferRows * (n + 1) * 4;  // the output layer's FP32 staging
    if (out_bytes > act_bytes) act_bytes = out_bytes;
    const int wrows = hidden > n_mma ? hidden : n_mma;
    s.act = 0;
    s.stage = (act_bytes + 1023) / 1024 * 1024;
    s.stage_bytes = (size_t)wrows * 64 * 2;
    s.bars = s.stage + kInferStages * s.stage_bytes;
    s.dpos = s.bars + 128;
    s.bias = (s.dpos + (size_t)n * 4 + 15) / 16 * 16;  // the four layers' biases, FP32
    s.total = s.bias + (size_t)(3 * hidden + n_mma) * 4 + 1024;  // + alignment slack of the base
    return s;
}

// GELU (tanh form) on the MUFU tanh: its 2^-10.7 relative error is below the
// BF16 rounding the hidden activations get anyway.
__device__ __forceinline__ float gelu_fast(float z) {
    const float u = kSqrt2OverPi * fmaf(kGeluC * z * z, z, z);
    float t;
    asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(u));
    return 0.5f * z * (1.0f + t);
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(bar) : "memory");
}

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&h);
}

template <bool GATE>
__global__ void __launch_bounds__(kInferThreads, 1)
    mlp_infer_kernel(const __grid_constant__ CUtensorMap w0, const __grid_constant__ CUtensorMap w1,
                     const __grid_constant__ CUtensorMap w2, const __grid_constant__ CUtensorMap w3,
                     const InferParams p) {
    using namespace umma;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    const InferSmem L = infer_smem(p.n, p.in_pad, p.hidden, p.n_mma);
    unsigned char* act = smem + L.act;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L.bars);
    uint64_t* full = bars;
    uint64_t* empty = bars + kInferStages;
    uint64_t* act_ready = bars + 2 * kInferStages;
    uint64_t* acc_ready = act_ready + 1;
    uint64_t* done = acc_ready + 1;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
    int* dpos = reinterpret_cast<int*>(smem + L.dpos);
    float* sbias = reinterpret_cast<float*>(smem + L.bias);  // [3 hidden + n_mma]

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int n = p.n;
    const int row0 = blockIdx.x * kInferRows;
    const int wrows = p.hidden > p.n_mma ? p.hidden : p.n_mma;
    const uint32_t tmem_cols = wrows <= 32 ? 32u : wrows <= 64 ? 64u : wrows <= 128 ? 128u : 256u;
    const CUtensorMap* maps[4] = {&w0, &w1, &w2, &w3};
    constexpr uint32_t kLboA = kInferRows * 16;  // 16-byte K chunks of the activation tile

    if (warp == kInferEpiWarps + 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(saddr(tmem_slot)),
                     "r"(tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (tid == kInferEpiWarps * 32) {
        for (int s = 0; s < kInferStages; ++s) {
            mbar_init(saddr(&full[s]), 1);
            mbar_init(saddr(&empty[s]), 1);
        }
        mbar_init(saddr(act_ready), kInferEpiWarps * 32);
        mbar_init(saddr(acc_ready), 1);
        mbar_init(saddr(done), 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (tid < kInferEpiWarps * 32) {  // CSR position of each row's diagonal (-1: none), the biases
        for (int j = tid; j < n; j += kInferEpiWarps * 32) {
            int d = -1;
            for (int e = p.row_ptrs[j]; e < p.row_ptrs[j + 1]; ++e)
                if (p.cols[e] == j) d = e;
            dpos[j] = d;
        }
        for (int j = tid; j < 3 * p.hidden + p.n_mma; j += kInferEpiWarps * 32) {
            const int l = j < 3 * p.hidden ? j / p.hidden : 3;
            const int c = j - l * p.hidden;
            sbias[j] = (l < 3 || c < n) ? p.bias[l][c] : 0.0f;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    const uint32_t act_base = saddr(act);
    const uint32_t stage_base = saddr(smem + L.stage);
    bool ok = true;

    if (warp == kInferEpiWarps) {
        if (lane == 0) {  // TMA producer of the weight tiles
            int i = 0;
            for (int l = 0; l < 4 && ok; ++l) {
                const int N = l < 3 ? p.hidden : p.n_mma;
                const int K = l == 0 ? p.in_pad : p.hidden;
                for (int kt = 0; kt < K / 64; ++kt, ++i) {
                    const int s = i % kInferStages;
                    if (i >= kInferStages &&
                        !mbar_wait(saddr(&empty[s]), ((i / kInferStages) - 1) & 1)) {
                        ok = false;
                        break;
                    }
                    const uint32_t dst = stage_base + (uint32_t)(s * L.stage_bytes), fb = saddr(&full[s]);
                    mbar_expect_tx(fb, (uint32_t)N * 64 * 2);
#pragma unroll
                    for (int kc = 0; kc < 8; ++kc)
                        tma_load_2d(dst + (uint32_t)(kc * N * 16), maps[l], kt * 64 + 8 * kc, 0, fb);
                }
            }
            // the last copies land before the block ends
            for (int j = i > kInferStages ? i - kInferStages : 0; j < i; ++j)
                if (!mbar_wait(saddr(&full[j % kInferStages]), (j / kInferStages) & 1)) ok = false;
        }
    } else if (warp == kInferEpiWarps + 1) {
        if (lane == 0) {  // MMA issuer
            int i = 0;
            for (int l = 0; l < 4 && ok; ++l) {
                const int N = l < 3 ? p.hidden : p.n_mma;
                const int K = l == 0 ? p.in_pad : p.hidden;
                const uint32_t idesc = idesc_bf16(kInferRows, N);
                const uint32_t lbo_b = (uint32_t)N * 16;
                if (!mbar_wait(saddr(act_ready), l & 1)) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                for (int kt = 0; kt < K / 64; ++kt, ++i) {
                    const int s = i % kInferStages;
                    if (!mbar_wait(saddr(&full[s]), (i / kInferStages) & 1)) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                    const uint32_t b = stage_base + (uint32_t)(s * L.stage_bytes);
#pragma unroll
                    for (int ks = 0; ks < 4; ++ks)
                        umma_bf16(tmem, smem_desc(act_base + (uint32_t)(kt * 8 + ks * 2) * kLboA, kLboA, 128),
                                  smem_desc(b + (uint32_t)ks * 2 * lbo_b, lbo_b, 128), idesc,
                                  (kt > 0 || ks > 0) ? 1u : 0u);
                    umma_commit(saddr(&empty[s]));
                }
                if (ok) umma_commit(saddr(acc_ready));
            }
            umma_commit(saddr(done));  // arrives once every MMA issued above has completed
        }
    } else {  // epilogue warps
        const int q = warp & 3, half = warp >> 2;
        const int r = q * 32 + lane;
        const uint32_t lane_addr = tmem + ((uint32_t)(q * 32) << 16);
        // the tile's features: the 256 threads walk the tile's rows of b and
        // x_prev (contiguous across the tile's systems) and its diagonal
        // entries with coalesced loads, and scatter the standardised BF16
        // values into the core-matrix layout; padding columns get zeros
        {
            const int rows = min(kInferRows, p.num_batch - row0);
            const int et = tid;  // 0..255
            unsigned char* actb = act;
            const auto put = [&](int rr, int f, float v) {
                *reinterpret_cast<__nv_bfloat16*>(actb + (size_t)(f >> 3) * kLboA + (size_t)rr * 16 + (f & 7) * 2) =
                    __float2bfloat16_rn(v);
            };
#pragma unroll 4
            for (int idx = et; idx < kInferRows * n; idx += kInferEpiWarps * 32) {
                const int rr = idx / n, f = idx - rr * n;
                float vd = 0.0f, vb = 0.0f, vx = 0.0f;
                if (rr < rows) {  // standardised in FP32 (the FP64 pipe is scarce; BF16 follows)
                    const size_t sysr = (size_t)(row0 + rr);
                    const int d = dpos[f];
                    const float dg = d >= 0 ? (float)p.values[sysr * p.nnz + d] : 0.0f;
                    vd = (dg - p.mean[f]) * p.inv_std[f];
                    vb = ((float)p.b[sysr * n + f] - p.mean[n + f]) * p.inv_std[n + f];
                    vx = ((float)p.xp[sysr * n + f] - p.mean[2 * n + f]) * p.inv_std[2 * n + f];
                }
                put(rr, f, vd);
                put(rr, n + f, vb);
                put(rr, 2 * n + f, vx);
            }
            const int padw = p.in_pad - 3 * n;
            for (int idx = et; idx < kInferRows * padw; idx += kInferEpiWarps * 32)
                put(idx / padw, 3 * n + idx % padw, 0.0f);
        }
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        mbar_arrive(saddr(act_ready));
        for (int l = 0; l < 3 && ok; ++l) {  // hidden layers: bias + GELU, BF16, in place
            if (!mbar_wait(saddr(acc_ready), l & 1)) {
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            const float* bias = sbias + l * p.hidden;
            for (int c0 = half * 16; c0 < p.hidden; c0 += 32) {
                uint32_t v[16];
                tmem_ld16(lane_addr + (uint32_t)c0, v);
                uint32_t w[8];
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    w[j] = pack_bf16x2(gelu_fast(__uint_as_float(v[2 * j]) + bias[c0 + 2 * j]),
                                       gelu_fast(__uint_as_float(v[2 * j + 1]) + bias[c0 + 2 * j + 1]));
                unsigned char* dst = act + (size_t)(c0 / 8) * kLboA + (size_t)r * 16;
                *reinterpret_cast<uint4*>(dst) = make_uint4(w[0], w[1], w[2], w[3]);
                *reinterpret_cast<uint4*>(dst + kLboA) = make_uint4(w[4], w[5], w[6], w[7]);
            }
            asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            mbar_arrive(saddr(act_ready));
        }
        // output layer: bias, FP32 staging [128][n + 1] over the activations
        float* out = reinterpret_cast<float*>(act);
        if (ok && !mbar_wait(saddr(acc_ready), 1)) ok = false;
        if (ok) {
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            const float* bias = sbias + 3 * p.hidden;
            for (int c0 = half * 16; c0 < p.n_mma; c0 += 32) {
                uint32_t v[16];
                tmem_ld16(lane_addr + (uint32_t)c0, v);
#pragma unroll
                for (int j = 0; j < 16; ++j)
                    if (c0 + j < n) out[(size_t)r * (n + 1) + c0 + j] = __uint_as_float(v[j]) + bias[c0 + j];
            }
        }
        asm volatile("bar.sync 1, %0;" ::"r"(kInferEpiWarps * 32) : "memory");
        // every epilogue thread agrees on whether the output is there
        ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
        const int rows = min(kInferRows, p.num_batch - row0);
        if (ok) {
            const double g = GATE ? 0.0 : *p.gamma;
            double cd = 0.0, cc = 0.0;
#pragma unroll 4
            for (int idx = tid; idx < rows * n; idx += kInferEpiWarps * 32) {
                const int rr = idx / n, j = idx - rr * n;
                const size_t gi = (size_t)(row0 + rr) * n + j;
                // the de-standardised change in FP32, added to x_prev in FP64
                const float c = fmaf(out[(size_t)rr * (n + 1) + j], p.stdv[3 * n + j], p.mean[3 * n + j]);
                if constexpr (GATE) {
                    cd = fma((double)c, p.xn[gi] - p.xp[gi], cd);
                    cc = fma((double)c, (double)c, cc);
                } else {
                    p.x0[gi] = fma(g, (double)c, p.xp[gi]);
                }
            }
            if constexpr (GATE) {
                for (int m = 16; m; m >>= 1) {
                    cd += __shfl_xor_sync(0xffffffffu, cd, m);
                    cc += __shfl_xor_sync(0xffffffffu, cc, m);
                }
                if (lane == 0) {
                    atomicAdd(p.acc, cd);
                    atomicAdd(p.acc + 1, cc);
                }
            }
        }
    }
    // every MMA has completed (or the waits ran out) before the tensor memory is freed
    ok = ok && mbar_wait(saddr(done), 0);
    ok = __syncthreads_and(ok ? 1 : 0) != 0;
    if (!ok && tid == 0) atomicExch(p.err, 1);
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == kInferEpiWarps + 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(tmem_cols)
                     : "memory");
}

}  // namespace mlp
}  // namespace bbs
