// Device building blocks of the fused batched solvers (Sec. 3.2): SpMV per
// batch format, block-wide dot products and norms, Jacobi setup.
//
// Thread mapping. One thread block owns one system. Thread `tid` of a block
// of `nt` threads owns rows tid, tid + nt, ..., tid + (R-1)*nt (R is a
// compile-time bound, ceil(n / nt) <= R). Every vector the method updates
// element-wise (r, r^, p, v, x, dinv ...) lives in the owner's registers;
// only the SpMV input vectors, which every thread reads at arbitrary columns,
// go through shared memory. This is the GB300 counterpart of the paper's
// "vectors in SLM by priority" (Sec. 3.5): registers are the faster and
// larger store here, so the priority list collapses to "SpMV inputs in shared
// memory, everything else in registers".
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "bbs_kernels.h"

namespace bbs {

enum Fmt { FMT_CSR = 0, FMT_ELL = 1, FMT_DENSE = 2 };
enum SysStatus { ST_CONVERGED = 0, ST_MAX_ITER = 1, ST_BREAKDOWN = 2, ST_NAN = 3 };
constexpr int kMaxRestarts = 3;  // confirmation restarts before MAX_ITER
constexpr unsigned kFull = 0xffffffffu;

// One system's matrix. vals points at this system's first value.
template <typename V>
struct Mat {
    const V* __restrict__ vals;
    const int32_t* __restrict__ row_ptrs;  // CSR
    const int32_t* __restrict__ cols;      // CSR: nnz, ELL: k*n column-major
    int n;
    int k;  // ELL width
};

// A team of whole warps that solves one system: the whole block (bar == 0,
// synchronised with __syncthreads), a single warp (__syncwarp), or a group of
// warps inside a persistent block (named barrier `bar`, 1..15).
struct Team {
    int tid, nt, lane, warp, nwarps, bar;
    __device__ __forceinline__ static Team block() {
        Team t;
        t.tid = threadIdx.x;
        t.nt = blockDim.x;
        t.lane = threadIdx.x & 31;
        t.warp = threadIdx.x >> 5;
        t.nwarps = blockDim.x >> 5;
        t.bar = 0;
        return t;
    }
    // Warps [first_warp, first_warp + nwarps) of the block.
    __device__ __forceinline__ static Team group(int first_warp, int nwarps) {
        Team t;
        t.tid = threadIdx.x - first_warp * 32;
        t.nt = nwarps * 32;
        t.lane = threadIdx.x & 31;
        t.warp = (threadIdx.x >> 5) - first_warp;
        t.nwarps = nwarps;
        t.bar = (nwarps * 32 == (int)blockDim.x) ? 0 : 1 + first_warp;
        return t;
    }
    __device__ __forceinline__ int row(int q) const { return tid + q * nt; }
    __device__ __forceinline__ void sync() const {
        if (nwarps == 1)
            __syncwarp();
        else if (bar == 0)
            __syncthreads();
        else
            asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(nt) : "memory");
    }
};

template <typename V>
__device__ __forceinline__ V ldg(const V* p) { return __ldg(p); }

template <typename T>
__device__ __forceinline__ bool finite(T v) { return isfinite(v); }

// FP64 tests done on the integer pipe (the FP64 pipe is the scarce resource
// of the FP64 solvers): finiteness, exact zero, and a <= b for a, b >= +0
// (the bit patterns of non-negative doubles order like the values).
__device__ __forceinline__ bool finite64(double v) {
    return (__double_as_longlong(v) & 0x7ff0000000000000LL) != 0x7ff0000000000000LL;
}
__device__ __forceinline__ bool zero64(double v) { return (__double_as_longlong(v) << 1) == 0; }
// Neither zero, subnormal, infinite nor NaN (its exponent field is neither 0 nor all ones).
__device__ __forceinline__ bool normal64(double v) {
    const long long e = __double_as_longlong(v) & 0x7ff0000000000000LL;
    return e != 0 && e != 0x7ff0000000000000LL;
}
__device__ __forceinline__ bool le_nonneg64(double a, double b) {
    return __double_as_longlong(a) <= __double_as_longlong(b);
}

// a_ii of row `row` (0 when the pattern stores none).
template <int FMT, typename V>
__device__ __forceinline__ V diag_entry(const Mat<V>& A, int row) {
    if constexpr (FMT == FMT_CSR) {
        const int e0 = ldg(A.row_ptrs + row), e1 = ldg(A.row_ptrs + row + 1);
        for (int e = e0; e < e1; ++e)
            if (ldg(A.cols + e) == row) return ldg(A.vals + e);
        return V(0);
    } else if constexpr (FMT == FMT_ELL) {
        for (int j = 0; j < A.k; ++j)
            if (ldg(A.cols + (size_t)j * A.n + row) == row) return ldg(A.vals + (size_t)j * A.n + row);
        return V(0);
    } else {
        return ldg(A.vals + (size_t)row * A.n + row);
    }
}

// Scalar Jacobi (Table "Batched feature support": BatchJacobi): 1/a_ii, with
// 1 for a zero or missing diagonal; without preconditioning all ones. Rows
// beyond n get 0 so that they stay inert in every update and dot product.
template <int FMT, int R, typename T, typename V>
__device__ __forceinline__ void jacobi_setup(const Mat<V>& A, bool jacobi, T (&dinv)[R],
                                             const Team& tm) {
#pragma unroll
    for (int q = 0; q < R; ++q) {
        const int row = tm.row(q);
        T d = T(0);
        if (row < A.n) {
            const T a = jacobi ? T(diag_entry<FMT>(A, row)) : T(0);
            d = (a != T(0)) ? T(1) / a : T(1);
        }
        dinv[q] = d;
    }
}

// y = A x for the caller's rows; x is a shared-memory vector of length n.
// Entries are accumulated in stored (ascending column) order with FMA. The
// CSR loop runs the warp's longest row with a predicate, so the warp never
// diverges on row lengths.
template <int FMT, int R, typename T, typename V>
__device__ __forceinline__ void spmv(const Mat<V>& A, const T* __restrict__ xs, T (&y)[R],
                                     const Team& tm) {
#pragma unroll
    for (int q = 0; q < R; ++q) {
        const int row = tm.row(q);
        T sum = T(0);
        if constexpr (FMT == FMT_CSR) {
            const bool ok = row < A.n;
            const int e0 = ok ? ldg(A.row_ptrs + row) : 0;
            const int len = ok ? ldg(A.row_ptrs + row + 1) - e0 : 0;
            const int longest = __reduce_max_sync(kFull, len);
            for (int j = 0; j < longest; ++j)
                if (j < len) sum = fma(T(ldg(A.vals + e0 + j)), xs[ldg(A.cols + e0 + j)], sum);
        } else if (row < A.n) {
            if constexpr (FMT == FMT_ELL) {
                // the value load does not wait for the column test (every
                // slot of the k*n table exists), so the slots' loads overlap
                const int32_t* c = A.cols + row;
                const V* a = A.vals + row;
#pragma unroll 3
                for (int j = 0; j < A.k; ++j) {
                    const int col = ldg(c + (size_t)j * A.n);
                    const V av = ldg(a + (size_t)j * A.n);
                    const T prod = col >= 0 ? fma(T(av), xs[col], sum) : sum;
                    sum = prod;
                }
            } else {
                const V* a = A.vals + (size_t)row * A.n;
                for (int j = 0; j < A.n; ++j) sum = fma(T(ldg(a + j)), xs[j], sum);
            }
        }
        y[q] = sum;
    }
}

// Same SpMV with the system's values staged in shared memory (as, laid out
// exactly like the global values of the system).
template <int FMT, int R, typename T, typename V>
__device__ __forceinline__ void spmv_staged(const Mat<V>& A, const V* __restrict__ as,
                                            const T* __restrict__ xs, T (&y)[R], const Team& tm) {
#pragma unroll
    for (int q = 0; q < R; ++q) {
        const int row = tm.row(q);
        T sum = T(0);
        if constexpr (FMT == FMT_CSR) {
            const bool ok = row < A.n;
            const int e0 = ok ? ldg(A.row_ptrs + row) : 0;
            const int len = ok ? ldg(A.row_ptrs + row + 1) - e0 : 0;
            const int longest = __reduce_max_sync(kFull, len);
            for (int j = 0; j < longest; ++j)
                if (j < len) sum = fma(T(as[e0 + j]), xs[ldg(A.cols + e0 + j)], sum);
        } else if (row < A.n) {
            if constexpr (FMT == FMT_ELL) {
                if constexpr (sizeof(T) == 8) {  // FP64: unrolled slots overlap their loads
#pragma unroll 3
                    for (int j = 0; j < A.k; ++j) {
                        const int col = ldg(A.cols + (size_t)j * A.n + row);
                        if (col >= 0) sum = fma(T(as[(size_t)j * A.n + row]), xs[col], sum);
                    }
                } else {
                    for (int j = 0; j < A.k; ++j) {
                        const int col = ldg(A.cols + (size_t)j * A.n + row);
                        if (col >= 0) sum = fma(T(as[(size_t)j * A.n + row]), xs[col], sum);
                    }
                }
            } else {
                const V* a = as + (size_t)row * A.n;
                for (int j = 0; j < A.n; ++j) sum = fma(T(a[j]), xs[j], sum);
            }
        }
        y[q] = sum;
    }
}

// Asynchronous global -> shared copies (cp.async): the data never pass
// through registers, so a thread's whole share of a staging loop is in
// flight at once instead of one load latency per element. The copies land
// after cp_async_wait_all() in the issuing thread and are visible to the
// others after the team's next barrier. 16-byte copies bypass L1 (the
// values are read once); 8-byte copies (gathers) go through it.
__device__ __forceinline__ void cp_async16(void* s, const void* g) {
    const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(s));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async8(void* s, const void* g) {
    const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(s));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Copy `count` values from global to shared memory with the whole team:
// 16-byte asynchronous copies when the source is 16-byte aligned (the
// destination always is), the ragged tail by plain loads. The caller
// synchronises the team afterwards.
template <typename V>
__device__ __forceinline__ void stage_values(const V* __restrict__ g, V* __restrict__ s,
                                             size_t count, const Team& tm) {
    constexpr int kVec = 16 / sizeof(V);
    const bool aligned = ((reinterpret_cast<uintptr_t>(g) & 15) == 0);
    size_t i = 0;
    if (aligned) {
        const size_t nv = count / kVec;
        const uint4* gv = reinterpret_cast<const uint4*>(g);
        uint4* sv = reinterpret_cast<uint4*>(s);
        for (size_t j = tm.tid; j < nv; j += tm.nt) cp_async16(sv + j, gv + j);
        i = nv * kVec;
    }
    for (size_t j = i + tm.tid; j < count; j += tm.nt) s[j] = ldg(g + j);
    cp_async_wait_all();
}

// ------------------------------------------------------------ reductions
//
// Block-wide sums of NV values at once, returned to every thread with
// identical bits. Within a warp the NV values are reduced "transposed": the
// first butterfly levels exchange half of the values instead of all, so NV
// sums cost about NV-1+5 additions instead of 5*NV (FP64 additions are the
// scarce resource on GB300). IEEE addition is commutative, so butterfly
// partners always hold identical sums. Across warps, lane partials go through
// shared memory (two alternating buffers, so one barrier per reduction).

template <typename T>
__device__ __forceinline__ T shfl_xor(T v, int m) { return __shfl_xor_sync(kFull, v, m); }
template <typename T>
__device__ __forceinline__ T shfl(T v, int src) { return __shfl_sync(kFull, v, src); }

// Sums of NV values over each aligned group of L lanes (L a power of two,
// 4..32), returned to every lane of the group with identical bits. All 32
// lanes of the warp must take part (every group runs the same instructions).
template <int L, typename T, int NV>
__device__ __forceinline__ void group_sum(T (&v)[NV], int lane) {
    static_assert(NV >= 1 && NV <= 4, "group_sum handles 1..4 values");
    static_assert(L >= 4 && L <= 32 && (L & (L - 1)) == 0, "L is a power of two in [4, 32]");
    const int base = lane & ~(L - 1);
    if constexpr (NV == 1) {
        T a = v[0];
#pragma unroll
        for (int m = L / 2; m; m >>= 1) a += shfl_xor(a, m);
        v[0] = a;
    } else if constexpr (NV == 2) {
        const bool hi = lane & (L / 2);
        T keep = hi ? v[1] : v[0];
        const T send = hi ? v[0] : v[1];
        keep += shfl_xor(send, L / 2);
#pragma unroll
        for (int m = L / 4; m; m >>= 1) keep += shfl_xor(keep, m);
        v[0] = shfl(keep, base);
        v[1] = shfl(keep, base + L / 2);
    } else {
        const T w3 = (NV == 4) ? v[NV - 1] : T(0);
        const bool b4 = lane & (L / 2);
        T k0 = b4 ? v[2] : v[0];
        T k1 = b4 ? w3 : v[1];
        const T s0 = b4 ? v[0] : v[2];
        const T s1 = b4 ? v[1] : w3;
        k0 += shfl_xor(s0, L / 2);
        k1 += shfl_xor(s1, L / 2);
        const bool b3 = lane & (L / 4);
        T keep = b3 ? k1 : k0;
        const T send = b3 ? k0 : k1;
        keep += shfl_xor(send, L / 4);
#pragma unroll
        for (int m = L / 8; m; m >>= 1) keep += shfl_xor(keep, m);
        v[0] = shfl(keep, base);
        v[1] = shfl(keep, base + L / 4);
        v[2] = shfl(keep, base + L / 2);
        if constexpr (NV == 4) v[3] = shfl(keep, base + 3 * L / 4);
    }
}

template <typename T, int NV>
__device__ __forceinline__ void warp_sum(T (&v)[NV], int lane) {
    group_sum<32, T, NV>(v, lane);
}

// red: shared scratch of 2 * 32 * 4 elements; parity alternates per call.
template <typename T, int NV>
__device__ __forceinline__ void block_sum(T (&v)[NV], T* red, int& parity, const Team& tm) {
    warp_sum<T, NV>(v, tm.lane);
    if (tm.nwarps == 1) return;
    T* buf = red + parity * 128;
    parity ^= 1;
    if constexpr (sizeof(T) == 4) {
        if (tm.nwarps <= 32) {  // FP32: one 16-byte slot per warp, read back as 16-byte broadcasts
            float4* b4 = reinterpret_cast<float4*>(buf);
            if (tm.lane == 0)
                b4[tm.warp] = make_float4(v[0], NV > 1 ? v[NV > 1 ? 1 : 0] : 0.0f, NV > 2 ? v[NV > 2 ? 2 : 0] : 0.0f,
                                          NV > 3 ? v[NV > 3 ? 3 : 0] : 0.0f);
            tm.sync();
            float4 s = b4[0];
            for (int w = 1; w < tm.nwarps; ++w) {
                const float4 t = b4[w];
                s.x += t.x;
                s.y += t.y;
                s.z += t.z;
                s.w += t.w;
            }
            v[0] = s.x;
            if constexpr (NV > 1) v[1] = s.y;
            if constexpr (NV > 2) v[2] = s.z;
            if constexpr (NV > 3) v[3] = s.w;
            return;
        }
    }
    if (tm.lane == 0) {
#pragma unroll
        for (int j = 0; j < NV; ++j) buf[tm.warp * 4 + j] = v[j];
    }
    tm.sync();
    // serial sums over the warps' partials: FP64 up to 4 warps (FP64 adds are
    // scarce), FP32 up to 8 (a short dependent chain beats a second shuffle
    // tree there)
    if (tm.nwarps <= (sizeof(T) == 4 ? 8 : 4)) {
#pragma unroll
        for (int j = 0; j < NV; ++j) {
            T s = buf[j];
            for (int w = 1; w < tm.nwarps; ++w) s += buf[w * 4 + j];
            v[j] = s;
        }
    } else {
#pragma unroll
        for (int j = 0; j < NV; ++j) v[j] = (tm.lane < tm.nwarps) ? buf[tm.lane * 4 + j] : T(0);
        warp_sum<T, NV>(v, tm.lane);
    }
}

// FP32 block sums of 5..8 values, identical bits on every thread. Blocks of
// up to 16 warps use one barrier (two 16-byte slots per warp in the same
// 128-float buffer); larger blocks reduce the first four values and the rest
// in two rounds.
template <int NV>
__device__ __forceinline__ void block_sum_wide(float (&v)[NV], float* red, int& parity, const Team& tm) {
    static_assert(NV > 4 && NV <= 8, "block_sum_wide handles 5..8 values");
    float a[4] = {v[0], v[1], v[2], v[3]};
    float c[NV - 4];
#pragma unroll
    for (int j = 0; j < NV - 4; ++j) c[j] = v[4 + j];
    if (tm.nwarps > 16) {
        block_sum(a, red, parity, tm);
        block_sum(c, red, parity, tm);
    } else {
        warp_sum<float, 4>(a, tm.lane);
        warp_sum<float, NV - 4>(c, tm.lane);
        if (tm.nwarps > 1) {
            float4* b4 = reinterpret_cast<float4*>(red + parity * 128);
            parity ^= 1;
            if (tm.lane == 0) {
                float e[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
                for (int j = 0; j < NV - 4; ++j) e[j] = c[j];
                b4[2 * tm.warp] = make_float4(a[0], a[1], a[2], a[3]);
                b4[2 * tm.warp + 1] = make_float4(e[0], e[1], e[2], e[3]);
            }
            tm.sync();
            float4 s = b4[0], u = b4[1];
            for (int w = 1; w < tm.nwarps; ++w) {
                const float4 p = b4[2 * w], q = b4[2 * w + 1];
                s.x += p.x;
                s.y += p.y;
                s.z += p.z;
                s.w += p.w;
                u.x += q.x;
                u.y += q.y;
                u.z += q.z;
                u.w += q.w;
            }
            a[0] = s.x;
            a[1] = s.y;
            a[2] = s.z;
            a[3] = s.w;
            const float uu[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
            for (int j = 0; j < NV - 4; ++j) c[j] = uu[j];
        }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) v[j] = a[j];
#pragma unroll
    for (int j = 0; j < NV - 4; ++j) v[4 + j] = c[j];
}

// Partial dot products over the caller's rows (rows beyond n hold zeros).
template <int R, typename T>
__device__ __forceinline__ T pdot(const T (&a)[R], const T (&b)[R]) {
    T s = T(0);
#pragma unroll
    for (int q = 0; q < R; ++q) s = fma(a[q], b[q], s);
    return s;
}

// Write the caller's rows of a register vector to a shared vector.
template <int R, typename T, typename U>
__device__ __forceinline__ void put(U* __restrict__ s, const T (&a)[R], const Team& tm, int n) {
#pragma unroll
    for (int q = 0; q < R; ++q) {
        const int row = tm.row(q);
        if (row < n) s[row] = U(a[q]);
    }
}

}  // namespace bbs
