// Learned initial guess for time-stepped batches: a small MLP that predicts
// each system's change of solution from its diagonal, right-hand side and
// previous solution, trained and run on the GPU by this file's kernels
// (BF16 tensor-core GEMMs with FP32 accumulation -- tcgen05 MMAs with the
// accumulator in tensor memory by default, mma.sync as the alternative --
// FP32 master weights, Adam).
// The paper has no such network; it motivates it: the solver accepts an
// initial guess (Sec. 2.1), and a better guess means fewer iterations.
//
// Network: 3n inputs (standardised diag(A), b, x_prev) -> H -> H -> H -> n,
// GELU (tanh form) after each hidden layer; output = standardised dx; the
// predicted initial guess is x_prev + dx * sigma + mu. Loss: mean squared
// error over the outputs. Weights W_l are [out, in] (y = x W^T + b).
//
// Storage (all owned by the bbs_mlp object):
//   master FP32 parameters, flat: W1 b1 W2 b2 W3 b3 W4 b4 (W row-major)
//   BF16 copies W_l [out, in_pad] (K-major, forward) and W_l^T [in, out_pad]
//   (K-major for the input-gradient GEMM), zero-padded to multiples of 32
//   activations of a minibatch: row-major and transposed BF16 copies (the
//   transposed ones feed the weight-gradient GEMMs, which reduce over rows)
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include "../../include/bbs.h"
#include "bbs_internal.h"
#include "bbs_mlp_gemm.cuh"
#include "bbs_umma.cuh"

namespace bbs {
namespace mlp {

constexpr int kLayers = 4;
constexpr float kGeluC = 0.044715f;
constexpr float kSqrt2OverPi = 0.7978845608028654f;

__device__ __forceinline__ float gelu(float z) {
    return 0.5f * z * (1.0f + tanhf(kSqrt2OverPi * (z + kGeluC * z * z * z)));
}
__device__ __forceinline__ float gelu_grad(float z) {
    const float t = tanhf(kSqrt2OverPi * (z + kGeluC * z * z * z));
    const float du = kSqrt2OverPi * (1.0f + 3.0f * kGeluC * z * z);
    return 0.5f * (1.0f + t) + 0.5f * z * (1.0f - t * t) * du;
}

// ---------------------------------------------------------- epilogues

enum EpiMode { EPI_F32 = 0, EPI_BIAS_GELU = 1, EPI_BIAS = 2, EPI_GELU_BWD = 3 };

struct Epi {
    int mode;
    float* c;                 // EPI_F32 / EPI_BIAS: output; EPI_BIAS_GELU: pre-activation store
    int ldc;
    size_t zstride;           // EPI_F32: split-K part blockIdx.z goes to c + blockIdx.z * zstride
    const float* bias;        // EPI_BIAS_GELU / EPI_BIAS
    __nv_bfloat16* y;         // BF16 row-major output (EPI_BIAS_GELU, EPI_GELU_BWD)
    int ldy;
    __nv_bfloat16* yt;        // BF16 transposed output, may be null
    int ldyt;
    const float* z;           // EPI_GELU_BWD: pre-activation of the layer below
    int ldz;

    __device__ __forceinline__ void operator()(int m, int n, float v) const {
        switch (mode) {
            case EPI_F32:
                c[(size_t)blockIdx.z * zstride + (size_t)m * ldc + n] = v;
                break;
            case EPI_BIAS:
                c[(size_t)m * ldc + n] = v + bias[n];
                break;
            case EPI_BIAS_GELU: {
                const float zz = v + bias[n];
                c[(size_t)m * ldc + n] = zz;
                const __nv_bfloat16 h = __float2bfloat16_rn(gelu(zz));
                y[(size_t)m * ldy + n] = h;
                if (yt) yt[(size_t)n * ldyt + m] = h;
                break;
            }
            default: {  // EPI_GELU_BWD
                const __nv_bfloat16 g = __float2bfloat16_rn(v * gelu_grad(z[(size_t)m * ldz + n]));
                y[(size_t)m * ldy + n] = g;
                if (yt) yt[(size_t)n * ldyt + m] = g;
                break;
            }
        }
    }
};

__global__ void __launch_bounds__(256) gemm_kernel(const __nv_bfloat16* __restrict__ A, int lda,
                                                   const __nv_bfloat16* __restrict__ B, int ldb, int M,
                                                   int N, int K, Epi epi) {
    gemm_tn_mma<Epi>(A, lda, B, ldb, M, N, K, epi);
}

__global__ void __launch_bounds__(128, 1) gemm_umma_kernel(const __grid_constant__ CUtensorMap ta,
                                                           const __grid_constant__ CUtensorMap tb, int M, int N,
                                                           int K, int BN, int ktiles_per_split, Epi epi,
                                                           int* err) {
    umma::gemm_tn_tma<Epi>(&ta, &tb, M, N, K, BN, ktiles_per_split, epi, err);
}

// c[m][n] = sum over the splits of part[z][m][n] (split-K, fixed order).
__global__ void splitk_reduce_kernel(int M, int N, int splits, const float* __restrict__ part, float* __restrict__ c,
                                     int ldc) {
    const size_t total = (size_t)M * N;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        float s = 0.0f;
        for (int z = 0; z < splits; ++z) s += part[(size_t)z * total + i];
        c[(i / N) * ldc + i % N] = s;
    }
}

// ---------------------------------------------------- small kernels

// Per-feature (3n inputs) and per-output (n) first and second moments of one
// time step's samples, accumulated in FP64: inputs diag(A), b, x_prev;
// outputs x_next - x_prev.
__global__ void observe_kernel(int num_batch, int n, const int32_t* __restrict__ row_ptrs,
                               const int32_t* __restrict__ cols, const double* __restrict__ values,
                               int nnz, const double* __restrict__ b, const double* __restrict__ xp,
                               const double* __restrict__ xn, double* __restrict__ sums,
                               double* __restrict__ sumsq) {
    const int F = 4 * n;
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= F) return;
    double s = 0.0, s2 = 0.0;
    for (int i = blockIdx.y; i < num_batch; i += gridDim.y) {
        double v;
        if (f < n) {
            v = 0.0;
            for (int e = row_ptrs[f]; e < row_ptrs[f + 1]; ++e)
                if (cols[e] == f) v = values[(size_t)i * nnz + e];
        } else if (f < 2 * n) {
            v = b[(size_t)i * n + f - n];
        } else if (f < 3 * n) {
            v = xp[(size_t)i * n + f - 2 * n];
        } else {
            v = xn[(size_t)i * n + f - 3 * n] - xp[(size_t)i * n + f - 3 * n];
        }
        s += v;
        s2 += v * v;
    }
    atomicAdd(sums + f, s);
    atomicAdd(sumsq + f, s2);
}

__global__ void finalize_stats_kernel(int F, double count, const double* sums, const double* sumsq,
                                      float* mean, float* inv_std, float* stdv) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= F) return;
    const double mu = sums[f] / count;
    const double var = fmax(sumsq[f] / count - mu * mu, 0.0);
    // a (numerically) constant quantity is centred but not scaled
    const double sd = var > 1e-12 * (mu * mu) + 1e-300 ? sqrt(var) : 1.0;
    mean[f] = (float)mu;
    stdv[f] = (float)sd;
    inv_std[f] = (float)(1.0 / sd);
}

// Standardised BF16 features [M, in_pad] (columns >= 3n zero) and, when xn is
// given, standardised FP32 targets [M, n].
__global__ void samples_kernel(int num_batch, int n, int in_pad, const int32_t* __restrict__ row_ptrs,
                               const int32_t* __restrict__ cols, const double* __restrict__ values, int nnz,
                               const double* __restrict__ b, const double* __restrict__ xp,
                               const double* __restrict__ xn, const float* __restrict__ mean,
                               const float* __restrict__ inv_std, __nv_bfloat16* __restrict__ feats,
                               float* __restrict__ targets) {
    const int i = blockIdx.x;
    for (int f = threadIdx.x; f < in_pad; f += blockDim.x) {
        float out = 0.0f;
        if (f < 3 * n) {
            double v;
            if (f < n) {
                v = 0.0;
                for (int e = row_ptrs[f]; e < row_ptrs[f + 1]; ++e)
                    if (cols[e] == f) v = values[(size_t)i * nnz + e];
            } else if (f < 2 * n) {
                v = b[(size_t)i * n + f - n];
            } else {
                v = xp[(size_t)i * n + f - 2 * n];
            }
            out = (float)((v - (double)mean[f]) * (double)inv_std[f]);
        }
        feats[(size_t)i * in_pad + f] = __float2bfloat16_rn(out);
    }
    if (xn != nullptr)
        for (int k = threadIdx.x; k < n; k += blockDim.x) {
            const int f = 3 * n + k;
            const double d = xn[(size_t)i * n + k] - xp[(size_t)i * n + k];
            targets[(size_t)i * n + k] = (float)((d - (double)mean[f]) * (double)inv_std[f]);
        }
}

// Minibatch gather: rows idx[r] of the sample store into X [M, in_pad] and
// X^T [in_pad, M], targets into T [M, n].
__global__ void gather_kernel(int M, int in_pad, int n, const int32_t* __restrict__ idx,
                              const __nv_bfloat16* __restrict__ feats, const float* __restrict__ targets,
                              __nv_bfloat16* __restrict__ X, __nv_bfloat16* __restrict__ XT,
                              float* __restrict__ T) {
    const int r = blockIdx.x;
    const size_t src = (size_t)idx[r];
    for (int f = threadIdx.x; f < in_pad; f += blockDim.x) {
        const __nv_bfloat16 v = feats[src * in_pad + f];
        X[(size_t)r * in_pad + f] = v;
        XT[(size_t)f * M + r] = v;
    }
    for (int k = threadIdx.x; k < n; k += blockDim.x) T[(size_t)r * n + k] = targets[src * n + k];
}

// dOut = 2 (out - t) / (M n) as BF16 [M, n_pad] and [n_pad, M]; loss sum.
__global__ void loss_kernel(int M, int n, int n_pad, const float* __restrict__ out,
                            const float* __restrict__ t, __nv_bfloat16* __restrict__ d,
                            __nv_bfloat16* __restrict__ dT, float* __restrict__ loss) {
    const int r = blockIdx.x;
    const float scale = 2.0f / ((float)M * (float)n);
    float acc = 0.0f;
    for (int k = threadIdx.x; k < n_pad; k += blockDim.x) {
        float g = 0.0f;
        if (k < n) {
            const float diff = out[(size_t)r * n + k] - t[(size_t)r * n + k];
            acc += diff * diff;
            g = diff * scale;
        }
        const __nv_bfloat16 gb = __float2bfloat16_rn(g);
        d[(size_t)r * n_pad + k] = gb;
        dT[(size_t)k * M + r] = gb;
    }
    for (int m = 16; m; m >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, m);
    __shared__ float part[32];
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.0f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += part[w];
        atomicAdd(loss, s / ((float)M * (float)n));
    }
}

// db[j] = sum over the row j of dT [N, M] (BF16), one warp per row.
__global__ void bias_grad_kernel(int N, int M, const __nv_bfloat16* __restrict__ dT, float* __restrict__ db) {
    const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (j >= N) return;
    float s = 0.0f;
    for (int m = threadIdx.x & 31; m < M; m += 32) s += __bfloat162float(dT[(size_t)j * M + m]);
    for (int k = 16; k; k >>= 1) s += __shfl_xor_sync(0xffffffffu, s, k);
    if ((threadIdx.x & 31) == 0) db[j] = s;
}

__global__ void adam_kernel(size_t count, float* __restrict__ p, const float* __restrict__ g,
                            float* __restrict__ m, float* __restrict__ v, float lr, float b1, float b2,
                            float eps, float c1, float c2) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (size_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// BF16 copies of one layer: W [out, in_pad] and W^T [in, out_pad], zero pads.
__global__ void pack_kernel(int out, int in, int in_pad, int out_pad, const float* __restrict__ W,
                            __nv_bfloat16* __restrict__ Wb, __nv_bfloat16* __restrict__ WTb) {
    const int total = out_pad * in_pad;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const int r = i / in_pad, k = i % in_pad;  // r over out_pad, k over in_pad
        const float w = (r < out && k < in) ? W[(size_t)r * in + k] : 0.0f;
        const __nv_bfloat16 h = __float2bfloat16_rn(w);
        if (r < out) Wb[(size_t)r * in_pad + k] = h;
        if (k < in) WTb[(size_t)k * out_pad + r] = h;
    }
}

// Deterministic initialisation from a counter-based hash (splitmix64):
// uniform in [-bound, bound].
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
    x += 0x9e3779b97f4a7c15ULL;
    x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ULL;
    x = (x ^ (x >> 27)) * 0x94d049bb133111ebULL;
    return x ^ (x >> 31);
}

__global__ void init_kernel(size_t count, float* __restrict__ p, uint64_t seed, size_t offset, float bound) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (size_t)gridDim.x * blockDim.x) {
        const uint64_t r = splitmix64(seed ^ splitmix64(offset + i));
        const double u = (double)(r >> 11) * (1.0 / 9007199254740992.0);  // [0, 1)
        p[i] = (float)((2.0 * u - 1.0) * bound);
    }
}

// x0 = x_prev + gamma * (predicted change), the change de-standardised.
__global__ void predict_epilogue_kernel(int num_batch, int n, const float* __restrict__ out,
                                        const double* __restrict__ xp, const float* __restrict__ mean,
                                        const float* __restrict__ stdv, const double* __restrict__ gamma,
                                        double* __restrict__ x0) {
    const size_t total = (size_t)num_batch * n;
    const double g = *gamma;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (size_t)gridDim.x * blockDim.x) {
        const int k = (int)(i % n);
        x0[i] = xp[i] + g * ((double)out[i] * (double)stdv[3 * n + k] + (double)mean[3 * n + k]);
    }
}

// Gate statistics of one time step: sums over the batch of c.d and c.c, with
// c the predicted change (de-standardised network output) and d the true
// change x_next - x_prev, accumulated in FP64 (acc[0], acc[1]).
__global__ void gate_observe_kernel(int num_batch, int n, const float* __restrict__ out,
                                    const double* __restrict__ xp, const double* __restrict__ xn,
                                    const float* __restrict__ mean, const float* __restrict__ stdv,
                                    double* __restrict__ acc) {
    const size_t total = (size_t)num_batch * n;
    double cd = 0.0, cc = 0.0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (size_t)gridDim.x * blockDim.x) {
        const int k = (int)(i % n);
        const double c = (double)out[i] * (double)stdv[3 * n + k] + (double)mean[3 * n + k];
        cd += c * (xn[i] - xp[i]);
        cc += c * c;
    }
    for (int m = 16; m; m >>= 1) {
        cd += __shfl_xor_sync(0xffffffffu, cd, m);
        cc += __shfl_xor_sync(0xffffffffu, cc, m);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(acc, cd);
        atomicAdd(acc + 1, cc);
    }
}

// gamma = acc[0] / acc[1], the least-squares scale of the predicted change,
// limited to [0, 1]; 0 when no change was predicted. Clears the sums.
__global__ void gate_finalize_kernel(double* __restrict__ acc, double* __restrict__ gamma) {
    const double num = acc[0], den = acc[1];
    double g = den > 0.0 ? num / den : 0.0;
    g = isfinite(g) ? fmin(fmax(g, 0.0), 1.0) : 0.0;
    *gamma = g;
    acc[0] = 0.0;
    acc[1] = 0.0;
}

}  // namespace mlp
}  // namespace bbs

#include "bbs_mlp_infer.cuh"

// ------------------------------------------------------------------ host

using bbs::mlp::Epi;

struct bbs_mlp {
    int device = 0;
    int n = 0, hidden = 0, in = 0, in_pad = 0, n_pad = 0, max_batch = 0;
    int dims_in[4], dims_out[4], pad_in[4], pad_out[4];
    size_t off_W[4], off_b[4], count = 0;
    float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
    __nv_bfloat16* Wb[4] = {};
    __nv_bfloat16* WTb[4] = {};
    int adam_t = 0;
    // statistics
    double *sums = nullptr, *sumsq = nullptr;
    double observed = 0.0;
    float *mean = nullptr, *inv_std = nullptr, *stdv = nullptr;
    // minibatch activations (max_batch rows)
    __nv_bfloat16 *X = nullptr, *XT = nullptr;
    float* T = nullptr;
    float* Z[3] = {};
    __nv_bfloat16* Y[3] = {};
    __nv_bfloat16* YT[3] = {};
    float* out = nullptr;
    __nv_bfloat16 *D = nullptr, *DT = nullptr;
    __nv_bfloat16* DZ[3] = {};
    __nv_bfloat16* DZT[3] = {};
    int32_t* idx = nullptr;
    int* err = nullptr;     // set by a tensor-core GEMM whose waits ran out
    double* gate = nullptr;  // [gamma, sum c.d, sum c.c] (see bbs_mlp_gate_observe)
    float* part = nullptr;  // split-K partial sums of the weight-gradient GEMMs
    size_t part_cap = 0;    // floats
    int sms = 0;
    int gemm_kind = BBS_GEMM_TCGEN05;  // or BBS_GEMM_MMA_SYNC
    // fused inference (bbs_mlp_infer.cuh): TMA maps of the BF16 weights, the
    // padded output width and the kernel's shared memory; fused = usable
    CUtensorMap infer_maps[4];
    int n_mma = 0;
    size_t infer_smem = 0;
    bool fused = false;
    std::vector<void*> allocs;
};

namespace {

bbs_status errf(bbs_status s, const char* fmt, ...) {
    char msg[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(msg, sizeof msg, fmt, ap);
    va_end(ap);
    return bbs::record_error(s, msg);
}

int round_up(int v, int a) { return (v + a - 1) / a * a; }

template <typename T>
bool dev_alloc(bbs_mlp* m, T** ptr, size_t count) {
    void* p = nullptr;
    if (cudaMalloc(&p, std::max<size_t>(count, 1) * sizeof(T)) != cudaSuccess) return false;
    cudaMemset(p, 0, std::max<size_t>(count, 1) * sizeof(T));
    m->allocs.push_back(p);
    *ptr = static_cast<T*>(p);
    return true;
}

// cuTensorMapEncodeTiled from the driver, through the runtime (no -lcuda).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// TMA map of a K-major BF16 operand [rows, K] (row stride ld elements) read
// in boxes of 8 K-elements (16 bytes) by box_rows rows; rows past the end
// read as zeros.
bool make_operand_map(CUtensorMap* map, const __nv_bfloat16* ptr, int rows, int K, int ld, int box_rows) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (enc == nullptr) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    const cuuint32_t box[2] = {8, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16*>(ptr), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// C = A B^T through the chosen tensor-core path (kind 1: tcgen05 with the
// accumulator in tensor memory, K a multiple of 64; kind 0: mma.sync).
// tcgen05 tiles: 128 rows x BN columns, BN <= 64 so that the layer GEMMs
// over thousands of samples launch hundreds of blocks. An FP32-output GEMM
// with few tiles and a long K (the weight gradients, K = samples) is split
// over K when `part` has room: each split writes its partial tile, and
// splitk_reduce_kernel adds them in a fixed order.
cudaError_t gemm_any(int kind, const __nv_bfloat16* A, int lda, const __nv_bfloat16* B, int ldb, int M, int N,
                     int K, const Epi& e, int* err, cudaStream_t st, float* part = nullptr, size_t part_cap = 0,
                     int sms = 152) {
    if (kind == BBS_GEMM_TCGEN05) {
        const int ntile = (N + 63) / 64;
        const int BN = std::max(16, round_up((N + ntile - 1) / ntile, 16));
        const int mt = (M + bbs::umma::kBM - 1) / bbs::umma::kBM, nt = (N + BN - 1) / BN;
        const int nk = K / bbs::umma::kBK;
        int splits = 1, kps = nk;
        const int want = 2 * sms;  // two blocks per SM fit (96 KB of stages each)
        if (e.mode == bbs::mlp::EPI_F32 && part != nullptr && mt * nt < want && nk >= 8) {
            splits = std::min((want + mt * nt - 1) / (mt * nt), nk / 4);
            while (splits > 1 && (size_t)splits * M * N > part_cap) --splits;
            if (splits > 1) {
                kps = (nk + splits - 1) / splits;
                splits = (nk + kps - 1) / kps;  // every split has k-tiles
            }
        }
        CUtensorMap ta, tb;
        if (!make_operand_map(&ta, A, M, K, lda, bbs::umma::kBM) || !make_operand_map(&tb, B, N, K, ldb, BN))
            return cudaErrorInvalidValue;
        const size_t smem = bbs::umma::smem_bytes(BN);
        static bool attr_set = false;
        if (!attr_set) {
            cudaError_t a = cudaFuncSetAttribute(bbs::mlp::gemm_umma_kernel,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)bbs::umma::smem_bytes(64));
            if (a != cudaSuccess) return a;
            attr_set = true;
        }
        dim3 grid(nt, mt, splits);
        if (splits == 1) {
            bbs::mlp::gemm_umma_kernel<<<grid, 128, smem, st>>>(ta, tb, M, N, K, BN, kps, e, err);
            return cudaGetLastError();
        }
        Epi pe = e;
        pe.c = part;
        pe.ldc = N;
        pe.zstride = (size_t)M * N;
        bbs::mlp::gemm_umma_kernel<<<grid, 128, smem, st>>>(ta, tb, M, N, K, BN, kps, pe, err);
        const size_t total = (size_t)M * N;
        const int blocks = (int)std::min<size_t>((total + 255) / 256, (size_t)sms * 8);
        bbs::mlp::splitk_reduce_kernel<<<blocks, 256, 0, st>>>(M, N, splits, part, e.c, e.ldc);
        return cudaGetLastError();
    }
    dim3 grid((N + bbs::mlp::kBN - 1) / bbs::mlp::kBN, (M + bbs::mlp::kBM - 1) / bbs::mlp::kBM);
    bbs::mlp::gemm_kernel<<<grid, 256, 0, st>>>(A, lda, B, ldb, M, N, K, e);
    return cudaGetLastError();
}

cudaError_t gemm(bbs_mlp* m, const __nv_bfloat16* A, int lda, const __nv_bfloat16* B, int ldb, int M, int N,
                 int K, const Epi& e, cudaStream_t st) {
    return gemm_any(m->gemm_kind, A, lda, B, ldb, M, N, K, e, m->err, st, m->part, m->part_cap, m->sms);
}

Epi epi_f32(float* c, int ldc) {
    Epi e{};
    e.mode = bbs::mlp::EPI_F32;
    e.c = c;
    e.ldc = ldc;
    return e;
}

void pack_all(bbs_mlp* m, cudaStream_t st) {
    for (int l = 0; l < bbs::mlp::kLayers; ++l) {
        const int total = m->pad_out[l] * m->pad_in[l];
        bbs::mlp::pack_kernel<<<(total + 255) / 256, 256, 0, st>>>(m->dims_out[l], m->dims_in[l], m->pad_in[l],
                                                                   m->pad_out[l], m->p + m->off_W[l], m->Wb[l],
                                                                   m->WTb[l]);
    }
}

// Forward pass of M rows of X [M, in_pad]; activations kept for backward.
cudaError_t forward(bbs_mlp* m, const __nv_bfloat16* X, int M, bool keep_transposed, cudaStream_t st) {
    const __nv_bfloat16* h = X;
    int ldh = m->in_pad;
    cudaError_t e = cudaSuccess;
    for (int l = 0; l < 3 && e == cudaSuccess; ++l) {
        Epi ep{};
        ep.mode = bbs::mlp::EPI_BIAS_GELU;
        ep.c = m->Z[l];
        ep.ldc = m->hidden;
        ep.bias = m->p + m->off_b[l];
        ep.y = m->Y[l];
        ep.ldy = m->hidden;
        ep.yt = keep_transposed ? m->YT[l] : nullptr;
        ep.ldyt = M;
        e = gemm(m, h, ldh, m->Wb[l], m->pad_in[l], M, m->hidden, m->pad_in[l], ep, st);
        h = m->Y[l];
        ldh = m->hidden;
    }
    if (e != cudaSuccess) return e;
    Epi ep{};
    ep.mode = bbs::mlp::EPI_BIAS;
    ep.c = m->out;
    ep.ldc = m->n;
    ep.bias = m->p + m->off_b[3];
    return gemm(m, h, ldh, m->Wb[3], m->pad_in[3], M, m->n, m->pad_in[3], ep, st);
}

// Loss and gradients of the minibatch in X/XT/T (M rows) into m->g.
cudaError_t backward(bbs_mlp* m, int M, float* loss, cudaStream_t st) {
    using namespace bbs::mlp;
    cudaError_t e = forward(m, m->X, M, true, st);
    if (e != cudaSuccess) return e;
    loss_kernel<<<M, 160, 0, st>>>(M, m->n, m->n_pad, m->out, m->T, m->D, m->DT, loss);
    // layer 4
    const __nv_bfloat16* dT = m->DT;  // [out_pad, M]
    const __nv_bfloat16* d = m->D;    // [M, out_pad]
    int ld_d = m->n_pad;
    for (int l = 3; l >= 0; --l) {
        const int out = m->dims_out[l], in = m->dims_in[l];
        // dW_l = d^T [out, M] . h_{l-1}^T [in, M]^T  -> [out, in]
        const __nv_bfloat16* hT = (l == 0) ? m->XT : m->YT[l - 1];
        if ((e = gemm(m, dT, M, hT, M, out, in, M, epi_f32(m->g + m->off_W[l], in), st)) != cudaSuccess) return e;
        bias_grad_kernel<<<(out + 7) / 8, 256, 0, st>>>(out, M, dT, m->g + m->off_b[l]);
        if (l == 0) break;
        // d_{l-1} = (d . W_l) * gelu'(z_{l-1}):  [M, in] = d [M, out_pad] . W_l^T [in, out_pad]^T
        Epi ep{};
        ep.mode = EPI_GELU_BWD;
        ep.z = m->Z[l - 1];
        ep.ldz = m->hidden;
        ep.y = m->DZ[l - 1];
        ep.ldy = m->hidden;
        ep.yt = m->DZT[l - 1];
        ep.ldyt = M;
        if ((e = gemm(m, d, ld_d, m->WTb[l], m->pad_out[l], M, in, m->pad_out[l], ep, st)) != cudaSuccess) return e;
        d = m->DZ[l - 1];
        dT = m->DZT[l - 1];
        ld_d = m->hidden;
    }
    return cudaGetLastError();
}

}  // namespace

extern "C" {

bbs_status bbs_mlp_create(bbs_handle* h, int32_t n, int32_t hidden, uint64_t seed, int32_t max_batch,
                          bbs_mlp** out) {
    if (h == nullptr || out == nullptr) return errf(BBS_ERR_INVALID_ARG, "null handle or output");
    *out = nullptr;
    if (n < 1 || n > 2048 || hidden < 64 || hidden % 64 != 0 || hidden > 4096)
        return errf(BBS_ERR_INVALID_ARG, "need 1 <= n <= 2048 and hidden a multiple of 64 in [64, 4096]");
    if (max_batch < 64 || max_batch % 64 != 0)
        return errf(BBS_ERR_INVALID_ARG, "max_batch must be a positive multiple of 64");
    cudaSetDevice(bbs::handle_device(h));
    bbs_mlp* m = new bbs_mlp();
    m->device = bbs::handle_device(h);
    m->n = n;
    m->hidden = hidden;
    m->in = 3 * n;
    m->in_pad = round_up(3 * n, 64);
    m->n_pad = round_up(n, 64);
    m->max_batch = max_batch;
    const int ins[4] = {3 * n, hidden, hidden, hidden}, outs[4] = {hidden, hidden, hidden, n};
    size_t o = 0;
    for (int l = 0; l < 4; ++l) {
        m->dims_in[l] = ins[l];
        m->dims_out[l] = outs[l];
        m->pad_in[l] = round_up(ins[l], 64);
        m->pad_out[l] = round_up(outs[l], 64);
        m->off_W[l] = o;
        o += (size_t)ins[l] * outs[l];
        m->off_b[l] = o;
        o += outs[l];
    }
    m->count = o;
    bool ok = dev_alloc(m, &m->p, o) && dev_alloc(m, &m->g, o) && dev_alloc(m, &m->m, o) &&
              dev_alloc(m, &m->v, o);
    for (int l = 0; l < 4 && ok; ++l)
        ok = dev_alloc(m, &m->Wb[l], (size_t)outs[l] * m->pad_in[l]) &&
             dev_alloc(m, &m->WTb[l], (size_t)ins[l] * m->pad_out[l]);
    const int F = 4 * n;
    ok = ok && dev_alloc(m, &m->sums, F) && dev_alloc(m, &m->sumsq, F) && dev_alloc(m, &m->mean, F) &&
         dev_alloc(m, &m->inv_std, F) && dev_alloc(m, &m->stdv, F);
    const size_t MB = (size_t)max_batch;
    ok = ok && dev_alloc(m, &m->X, MB * m->in_pad) && dev_alloc(m, &m->XT, MB * m->in_pad) &&
         dev_alloc(m, &m->T, MB * n) && dev_alloc(m, &m->out, MB * n) &&
         dev_alloc(m, &m->D, MB * m->n_pad) && dev_alloc(m, &m->DT, MB * m->n_pad) &&
         dev_alloc(m, &m->idx, MB) && dev_alloc(m, &m->err, 1) && dev_alloc(m, &m->gate, 3);
    for (int l = 0; l < 3 && ok; ++l)
        ok = dev_alloc(m, &m->Z[l], MB * hidden) && dev_alloc(m, &m->Y[l], MB * hidden) &&
             dev_alloc(m, &m->YT[l], MB * hidden) && dev_alloc(m, &m->DZ[l], MB * hidden) &&
             dev_alloc(m, &m->DZT[l], MB * hidden);
    // split-K partials of the weight gradients: up to 32 splits of the largest [out, in]
    size_t wmax = 0;
    for (int l = 0; l < 4; ++l) wmax = std::max(wmax, (size_t)outs[l] * ins[l]);
    m->part_cap = 32 * wmax;
    ok = ok && dev_alloc(m, &m->part, m->part_cap);
    cudaDeviceGetAttribute(&m->sms, cudaDevAttrMultiProcessorCount, m->device);
    if (m->sms <= 0) m->sms = 152;
    if (!ok) {
        bbs_mlp_destroy(m);
        return errf(BBS_ERR_NO_MEMORY, "MLP buffers");
    }
    // init: weights U(-1/sqrt(in), 1/sqrt(in)), the output layer scaled by 0.1 so
    // the first predictions stay near the mean change; biases zero
    for (int l = 0; l < 4; ++l) {
        const float bound = (float)(1.0 / std::sqrt((double)ins[l])) * (l == 3 ? 0.1f : 1.0f);
        const size_t cnt = (size_t)ins[l] * outs[l];
        bbs::mlp::init_kernel<<<(unsigned)std::min<size_t>((cnt + 255) / 256, 4096), 256>>>(
            cnt, m->p + m->off_W[l], seed, m->off_W[l], bound);
    }
    // standardisation defaults to identity until statistics are finalised
    std::vector<float> ones(F, 1.0f);
    cudaMemcpy(m->inv_std, ones.data(), F * sizeof(float), cudaMemcpyHostToDevice);
    cudaMemcpy(m->stdv, ones.data(), F * sizeof(float), cudaMemcpyHostToDevice);
    const double gamma_one = 1.0;  // ungated until bbs_mlp_gate_finalize
    cudaMemcpy(m->gate, &gamma_one, sizeof(double), cudaMemcpyHostToDevice);
    pack_all(m, nullptr);
    // fused inference (one kernel for the whole network) when its tiles fit:
    // hidden and the 16-padded output width up to 256 (one MMA's N and the
    // tensor-memory columns), the activation tile and weight ring in shared
    // memory
    m->n_mma = round_up(n, 16);
    const bbs::mlp::InferSmem L = bbs::mlp::infer_smem(n, m->in_pad, hidden, m->n_mma);
    m->infer_smem = L.total;
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, m->device);
    m->fused = hidden <= 256 && m->n_mma <= 256 && L.total <= (size_t)optin;
    for (int l = 0; l < 4 && m->fused; ++l)
        m->fused = make_operand_map(&m->infer_maps[l], m->Wb[l], outs[l], m->pad_in[l], m->pad_in[l],
                                    l < 3 ? hidden : m->n_mma);
    if (m->fused)
        m->fused = cudaFuncSetAttribute(bbs::mlp::mlp_infer_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)L.total) == cudaSuccess &&
                   cudaFuncSetAttribute(bbs::mlp::mlp_infer_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)L.total) == cudaSuccess;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        bbs_mlp_destroy(m);
        return errf(BBS_ERR_CUDA, "MLP init: %s", cudaGetErrorString(e));
    }
    *out = m;
    return BBS_OK;
}

bbs_status bbs_mlp_destroy(bbs_mlp* m) {
    if (m == nullptr) return BBS_OK;
    cudaSetDevice(m->device);
    for (void* p : m->allocs) cudaFree(p);
    delete m;
    return BBS_OK;
}

bbs_status bbs_mlp_param_count(const bbs_mlp* m, int64_t* count) {
    if (m == nullptr || count == nullptr) return errf(BBS_ERR_INVALID_ARG, "null argument");
    *count = (int64_t)m->count;
    return BBS_OK;
}

bbs_status bbs_mlp_get_params(bbs_mlp* m, float* params, void* stream) {
    if (m == nullptr || params == nullptr) return errf(BBS_ERR_INVALID_ARG, "null argument");
    cudaError_t e = cudaMemcpyAsync(params, m->p, m->count * sizeof(float), cudaMemcpyDeviceToDevice,
                                    reinterpret_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? BBS_OK : errf(BBS_ERR_CUDA, "%s", cudaGetErrorString(e));
}

bbs_status bbs_mlp_set_params(bbs_mlp* m, const float* params, void* stream) {
    if (m == nullptr || params == nullptr) return errf(BBS_ERR_INVALID_ARG, "null argument");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemcpyAsync(m->p, params, m->count * sizeof(float), cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return errf(BBS_ERR_CUDA, "%s", cudaGetErrorString(e));
    pack_all(m, st);
    e = cudaGetLastError();
    return e == cudaSuccess ? BBS_OK : errf(BBS_ERR_CUDA, "%s", cudaGetErrorString(e));
}

static bbs_status check_csr_batch(const bbs_mlp* m, const bbs_batch_matrix* A) {
    if (A == nullptr || A->fmt != BBS_FMT_CSR || A->n != m->n || !A->row_ptrs || !A->col_idxs || !A->values)
        return errf(BBS_ERR_INVALID_ARG, "the MLP reads a BatchCsr matrix with n = %d", m->n);
    return BBS_OK;
}

bbs_status bbs_mlp_observe(bbs_mlp* m, const bbs_batch_matrix* A, const double* b, const double* x_prev,
                           const double* x_next, void* stream) {
    if (m == nullptr || !b || !x_prev || !x_next) return errf(BBS_ERR_INVALID_ARG, "null argument");
    bbs_status s = check_csr_batch(m, A);
    if (s != BBS_OK) return s;
    if (A->num_batch == 0) return BBS_OK;
    const int F = 4 * m->n;
    dim3 grid((F + 127) / 128, std::min(A->num_batch, 256));
    bbs::mlp::observe_kernel<<<grid, 128, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        A->num_batch, m->n, A->row_ptrs, A->col_idxs, A->values, A->nnz, b, x_prev, x_next, m->sums, m->sumsq);
    m->observed += A->num_batch;
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? BBS_OK : errf(BBS_ERR_CUDA, "%s", cudaGetErrorString(e));
}

bbs_status bbs_mlp_finalize_stats(bbs_mlp* m, void* stream) {
    if (m == nullptr || m->observed <= 0) return errf(BBS_ERR_INVALID_ARG, "no samples observed");
    const int F = 4 * m->n;
    bbs::mlp::finalize_stats_kernel<<<(F + 127) / 128, 128, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        F, m->observed, m->sums, m->sumsq, m->mean, m->inv_std, m->stdv);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? BBS_OK : errf(BBS_ERR_CUDA, "%s", cudaGetErrorString(e));
}

bbs_status bbs_mlp_make_samples(bbs_mlp* m, const bbs_batch_matrix* A, const double* b, const double* x_prev,
                                const double* x_next, uint16_t* feats, float* targets, void* stream) {
    if (m == nullptr || !b || !x_prev || !feats || (x_next && !targets))
        return errf(BBS_ERR_INVALID_ARG, "null argument");
    bbs_status s = check_csr_batch(m, A);
    if (s != BBS_OK) return s;
    if (A->num_batch == 0) return BBS_OK;
    bbs::mlp::samples_kernel<<<A->num_batch, 128, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        A->num_batch, m->n, m->in_pad, A->row_ptrs, A->col_idxs, A->values, A->nnz, b, x_prev, x_next, m->mean,
        m->inv_std, reinterpret_cast<__nv_bfloat16*>(feats), targets);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? BBS_OK : errf(BBS_ERR_CUDA, "%s", cudaGetErrorString(e));
}

bbs_status bbs_mlp_gradients(bbs_mlp* m, const uint16_t* feats, const float* targets, const int32_t* rows,
                             int32_t M, float* loss, void* stream) {
    if (m == nullptr || !feats || !targets || !rows || !loss) return errf(BBS_ERR_INVALID_ARG, "null argument");
    if (M < 64 || M > m->max_batch || M % 64 != 0)
        return errf(BBS_ERR_INVALID_ARG, "minibatch must be a multiple of 64 up to %d", m->max_batch);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaMemcpyAsync(m->idx, rows, sizeof(int32_t) * M, cudaMemcpyDeviceToDevice, st);
    bbs::mlp::gather_kernel<<<M, 128, 0, st>>>(M, m->in_pad, m->n, m->idx,
                                               reinterpret_cast<const __nv_bfloat16*>(feats), targets, m->X,
                                               m->XT, m->T);
    cudaMemsetAsync(loss, 0, sizeof(float), st);
    cudaError_t e = backward(m, M, loss, st);
    return e == cudaSuccess ? BBS_OK : errf(BBS_ERR_CUDA, "%s", cudaGetErrorString(e));
}

bbs_status bbs_mlp_train_step(bbs_mlp* m, const uint16_t* feats, const float* targets, const int32_t* rows,
                              int32_t M, float lr, float* loss, void* stream) {
    bbs_status s = bbs_mlp_gradients(m, feats, targets, rows, M, loss, stream);
    if (s != BBS_OK) return s;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    m->adam_t += 1;
    const float c1 = 1.0f - powf(0.9f, (float)m->adam_t), c2 = 1.0f - powf(0.999f, (float)m->adam_t);
    bbs::mlp::adam_kernel<<<(unsigned)std::min<size_t>((m->count + 255) / 256, 2048), 256, 0, st>>>(
        m->count, m->p, m->g, m->m, m->v, lr, 0.9f, 0.999f, 1e-8f, c1, c2);
    pack_all(m, st);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? BBS_OK : errf(BBS_ERR_CUDA, "%s", cudaGetErrorString(e));
}

bbs_status bbs_mlp_set_gemm(bbs_mlp* m, int32_t kind) {
    if (m == nullptr || (kind != BBS_GEMM_MMA_SYNC && kind != BBS_GEMM_TCGEN05))
        return errf(BBS_ERR_INVALID_ARG, "unknown GEMM kind");
    m->gemm_kind = kind;
    return BBS_OK;
}

bbs_status bbs_mlp_check(bbs_mlp* m) {
    if (m == nullptr) return errf(BBS_ERR_INVALID_ARG, "null network");
    int flag = 0;
    cudaError_t e = cudaMemcpy(&flag, m->err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return errf(BBS_ERR_CUDA, "%s", cudaGetErrorString(e));
    return flag ? errf(BBS_ERR_CUDA, "a tensor-core GEMM gave up waiting for its MMAs") : BBS_OK;
}

bbs_status bbs_gemm_bf16(bbs_handle* h, int32_t kind, const uint16_t* A, int32_t lda, const uint16_t* B,
                         int32_t ldb, int32_t M, int32_t N, int32_t K, float* C, int32_t ldc) {
    if (h == nullptr || !A || !B || !C || M < 0 || N < 0 || K < 0)
        return errf(BBS_ERR_INVALID_ARG, "null pointer or negative size");
    if (kind != BBS_GEMM_MMA_SYNC && kind != BBS_GEMM_TCGEN05) return errf(BBS_ERR_INVALID_ARG, "unknown GEMM kind");
    const int kmul = kind == BBS_GEMM_TCGEN05 ? 64 : 32;
    if (K % kmul != 0 || lda % 8 != 0 || ldb % 8 != 0 || lda < K || ldb < K || ldc < N)
        return errf(BBS_ERR_INVALID_ARG, "K must be a multiple of %d, lda/ldb multiples of 8 and >= K", kmul);
    if (M == 0 || N == 0) return BBS_OK;
    cudaSetDevice(bbs::handle_device(h));
    int* err = nullptr;
    cudaError_t e = cudaMalloc(&err, sizeof(int));
    if (e != cudaSuccess) return errf(BBS_ERR_NO_MEMORY, "%s", cudaGetErrorString(e));
    cudaMemset(err, 0, sizeof(int));
    Epi ep = epi_f32(C, ldc);
    if (K == 0) {
        cudaFree(err);
        return errf(BBS_ERR_INVALID_ARG, "K must be positive");
    }
    float* part = nullptr;
    const size_t part_cap = (size_t)32 * M * N;
    if (kind == BBS_GEMM_TCGEN05 && cudaMalloc(&part, part_cap * sizeof(float)) != cudaSuccess) part = nullptr;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, bbs::handle_device(h));
    e = gemm_any(kind, reinterpret_cast<const __nv_bfloat16*>(A), lda, reinterpret_cast<const __nv_bfloat16*>(B),
                 ldb, M, N, K, ep, err, nullptr, part, part ? part_cap : 0, sms > 0 ? sms : 152);
    int flag = 0;
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(&flag, err, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(err);
    if (part) cudaFree(part);
    if (e != cudaSuccess) return errf(BBS_ERR_CUDA, "%s", cudaGetErrorString(e));
    return flag ? errf(BBS_ERR_CUDA, "the tensor-core GEMM gave up waiting for its MMAs") : BBS_OK;
}

bbs_status bbs_mlp_get_grads(bbs_mlp* m, float* grads, void* stream) {
    if (m == nullptr || grads == nullptr) return errf(BBS_ERR_INVALID_ARG, "null argument");
    cudaError_t e = cudaMemcpyAsync(grads, m->g, m->count * sizeof(float), cudaMemcpyDeviceToDevice,
                                    reinterpret_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? BBS_OK : errf(BBS_ERR_CUDA, "%s", cudaGetErrorString(e));
}

bbs_status bbs_mlp_forward(bbs_mlp* m, const uint16_t* feats, int32_t M, float* out, void* stream) {
    if (m == nullptr || !feats || !out) return errf(BBS_ERR_INVALID_ARG, "null argument");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    for (int r0 = 0; r0 < M; r0 += m->max_batch) {
        const int rows = std::min(m->max_batch, M - r0);
        cudaError_t e = forward(m, reinterpret_cast<const __nv_bfloat16*>(feats) + (size_t)r0 * m->in_pad, rows,
                                false, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(out + (size_t)r0 * m->n, m->out, sizeof(float) * rows * m->n,
                                cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return errf(BBS_ERR_CUDA, "%s", cudaGetErrorString(e));
    }
    return BBS_OK;
}

}  // extern "C"

// The tcgen05 path runs predictions and gate statistics through the fused
// kernel when the network's tiles fit it.
static bool uses_fused(const bbs_mlp* m) { return m->fused && m->gemm_kind == BBS_GEMM_TCGEN05; }

// One launch of the fused network over the batch (128 systems per block):
// x0 = x_prev + gamma * change (x_next == nullptr), or the gate statistics of
// the change against x_next - x_prev.
static bbs_status infer_fused(bbs_mlp* m, const bbs_batch_matrix* A, const double* b, const double* x_prev,
                              const double* x_next, double* x0, cudaStream_t st) {
    if (A->num_batch == 0) return BBS_OK;
    bbs::mlp::InferParams p{};
    p.num_batch = A->num_batch;
    p.n = m->n;
    p.nnz = A->nnz;
    p.in_pad = m->in_pad;
    p.hidden = m->hidden;
    p.n_mma = m->n_mma;
    p.row_ptrs = A->row_ptrs;
    p.cols = A->col_idxs;
    p.values = A->values;
    p.b = b;
    p.xp = x_prev;
    p.xn = x_next;
    p.x0 = x0;
    p.acc = m->gate + 1;
    for (int l = 0; l < 4; ++l) p.bias[l] = m->p + m->off_b[l];
    p.mean = m->mean;
    p.inv_std = m->inv_std;
    p.stdv = m->stdv;
    p.gamma = m->gate;
    p.err = m->err;
    const unsigned grid = (unsigned)((A->num_batch + bbs::mlp::kInferRows - 1) / bbs::mlp::kInferRows);
    const auto& w = m->infer_maps;
    if (x_next != nullptr)
        bbs::mlp::mlp_infer_kernel<true><<<grid, bbs::mlp::kInferThreads, m->infer_smem, st>>>(w[0], w[1], w[2], w[3], p);
    else
        bbs::mlp::mlp_infer_kernel<false><<<grid, bbs::mlp::kInferThreads, m->infer_smem, st>>>(w[0], w[1], w[2], w[3],
                                                                                              p);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? BBS_OK : errf(BBS_ERR_CUDA, "%s", cudaGetErrorString(e));
}

// The network over a batch, max_batch rows at a time; `tail(r0, rows)`
// consumes each piece's output in m->out.
template <class Tail>
static bbs_status run_batch(bbs_mlp* m, const bbs_batch_matrix* A, const double* b, const double* x_prev,
                            cudaStream_t st, Tail tail) {
    const int n = m->n;
    for (int r0 = 0; r0 < A->num_batch; r0 += m->max_batch) {
        const int rows = std::min(m->max_batch, A->num_batch - r0);
        bbs::mlp::samples_kernel<<<rows, 128, 0, st>>>(
            rows, n, m->in_pad, A->row_ptrs, A->col_idxs, A->values + (size_t)r0 * A->nnz, A->nnz,
            b + (size_t)r0 * n, x_prev + (size_t)r0 * n, nullptr, m->mean, m->inv_std, m->X, nullptr);
        cudaError_t e = forward(m, m->X, rows, false, st);
        if (e != cudaSuccess) return errf(BBS_ERR_CUDA, "%s", cudaGetErrorString(e));
        tail(r0, rows);
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? BBS_OK : errf(BBS_ERR_CUDA, "%s", cudaGetErrorString(e));
}

extern "C" {

bbs_status bbs_mlp_predict(bbs_mlp* m, const bbs_batch_matrix* A, const double* b, const double* x_prev,
                           double* x0, void* stream) {
    if (m == nullptr || !b || !x_prev || !x0) return errf(BBS_ERR_INVALID_ARG, "null argument");
    bbs_status s = check_csr_batch(m, A);
    if (s != BBS_OK) return s;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (uses_fused(m)) return infer_fused(m, A, b, x_prev, nullptr, x0, st);
    const int n = m->n;
    return run_batch(m, A, b, x_prev, st, [&](int r0, int rows) {
        bbs::mlp::predict_epilogue_kernel<<<std::min((rows * n + 255) / 256, 4096), 256, 0, st>>>(
            rows, n, m->out, x_prev + (size_t)r0 * n, m->mean, m->stdv, m->gate, x0 + (size_t)r0 * n);
    });
}

bbs_status bbs_mlp_gate_observe(bbs_mlp* m, const bbs_batch_matrix* A, const double* b, const double* x_prev,
                                const double* x_next, void* stream) {
    if (m == nullptr || !b || !x_prev || !x_next) return errf(BBS_ERR_INVALID_ARG, "null argument");
    bbs_status s = check_csr_batch(m, A);
    if (s != BBS_OK) return s;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (uses_fused(m)) return infer_fused(m, A, b, x_prev, x_next, nullptr, st);
    const int n = m->n;
    return run_batch(m, A, b, x_prev, st, [&](int r0, int rows) {
        bbs::mlp::gate_observe_kernel<<<std::min((rows * n + 255) / 256, 1024), 256, 0, st>>>(
            rows, n, m->out, x_prev + (size_t)r0 * n, x_next + (size_t)r0 * n, m->mean, m->stdv, m->gate + 1);
    });
}

bbs_status bbs_mlp_gate_finalize(bbs_mlp* m, void* stream) {
    if (m == nullptr) return errf(BBS_ERR_INVALID_ARG, "null argument");
    bbs::mlp::gate_finalize_kernel<<<1, 1, 0, reinterpret_cast<cudaStream_t>(stream)>>>(m->gate + 1, m->gate);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? BBS_OK : errf(BBS_ERR_CUDA, "%s", cudaGetErrorString(e));
}

bbs_status bbs_mlp_get_gate(bbs_mlp* m, double* gamma) {
    if (m == nullptr || gamma == nullptr) return errf(BBS_ERR_INVALID_ARG, "null argument");
    cudaError_t e = cudaMemcpy(gamma, m->gate, sizeof(double), cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? BBS_OK : errf(BBS_ERR_CUDA, "%s", cudaGetErrorString(e));
}

}  // extern "C"
