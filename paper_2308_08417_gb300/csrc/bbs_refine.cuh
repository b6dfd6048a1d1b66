// Mixed-precision iterative refinement, fused in one kernel per batch.
//
// The paper makes the arithmetic precision a dispatch parameter of the
// solver kernel (Sec. 3.3-3.4) and notes that iteration counts depend on the
// precision used (Sec. 2.1). Here the outer loop keeps the residual
// r = b - A x, its norm, the exit test and the update x += ||r|| d in FP64,
// and the correction d solves A32 d = r/||r|| by BiCGSTAB + Jacobi entirely
// in FP32 (values, vectors, reductions), to a relative inner tolerance.
#pragma once

#include "bbs_solvers.cuh"

namespace bbs {

// FP32 BiCGSTAB from d = 0 on A32 d = w; stops when the recursive residual
// passes inner_tol*||w||, on a breakdown or non-finite scalar, or after
// max_inner iterations. Returns the iteration at which it stopped. Two block
// reductions per iteration instead of three: the norm of the new residual
// and the next rho come from the dot products of s and t (the inner solve
// only needs to shrink the residual; the FP64 outer loop judges the result).
template <int R, class Op32>
__device__ __forceinline__ int inner_bicgstab32(const Op32& op,
                                                const float (&dinv)[R], const float (&w)[R],
                                                float (&d)[R], float inner_tol, int max_inner,
                                                float* xa, float* xb, float* red, int& parity,
                                                const Team& tm, int n) {
    float r[R], rh[R], p[R], v[R], t[R];
#pragma unroll
    for (int q = 0; q < R; ++q) {
        d[q] = 0.0f;
        r[q] = w[q];
        rh[q] = w[q];
        p[q] = 0.0f;
        v[q] = 0.0f;
    }
    float s0[1] = {pdot(w, w)};
    block_sum(s0, red, parity, tm);
    const float tau2 = inner_tol * inner_tol * s0[0];
    float rho = s0[0], rho_old = 1.0f, alpha = 1.0f, omega = 1.0f;
    for (int it = 1; it <= max_inner; ++it) {
        if (!finite(rho) || rho == 0.0f) return it;
        const float beta = (rho * alpha) / (rho_old * omega);
#pragma unroll
        for (int q = 0; q < R; ++q) p[q] = fmaf(beta, fmaf(-omega, v[q], p[q]), r[q]);
        {
            float ph[R];
#pragma unroll
            for (int q = 0; q < R; ++q) ph[q] = dinv[q] * p[q];
            put(xa, ph, tm, n);
        }
        tm.sync();
        op.apply(xa, v, tm);
        float s1[1] = {pdot(rh, v)};
        block_sum(s1, red, parity, tm);
        const float sigma = s1[0];
        if (!finite(sigma) || sigma == 0.0f) return it;
        alpha = rho / sigma;
#pragma unroll
        for (int q = 0; q < R; ++q) r[q] = fmaf(-alpha, v[q], r[q]);
        {
            float sh[R];
#pragma unroll
            for (int q = 0; q < R; ++q) sh[q] = dinv[q] * r[q];
            put(xb, sh, tm, n);
        }
        tm.sync();
        op.apply(xb, t, tm);
        // One reduction closes the step. With r = s - omega t (s held in r):
        // (r, r) = (s, s) - omega (2 (t, s) - omega (t, t)) and
        // (rh, r) = (rh, s) - omega (rh, t), exact in exact arithmetic.
        float s3[5] = {pdot(r, r), pdot(t, t), pdot(t, r), pdot(rh, r), pdot(rh, t)};
        block_sum_wide(s3, red, parity, tm);
        if (s3[0] <= tau2) {
#pragma unroll
            for (int q = 0; q < R; ++q) {
                const int row = tm.row(q);
                if (row < n) d[q] = fmaf(alpha, xa[row], d[q]);
            }
            return it;
        }
        omega = (s3[1] == 0.0f) ? 0.0f : s3[2] / s3[1];
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const int row = tm.row(q);
            if (row < n) d[q] = fmaf(omega, xb[row], fmaf(alpha, xa[row], d[q]));
            r[q] = fmaf(-omega, t[q], r[q]);
        }
        const float rr = fmaf(-omega, fmaf(-omega, s3[1], 2.0f * s3[2]), s3[0]);
        if (!finite(rr) || rr <= tau2 || omega == 0.0f) return it;
        rho_old = rho;
        rho = fmaf(-omega, s3[4], s3[3]);
    }
    return max_inner;
}

// Copy `count` FP64 values to shared memory rounded to FP32 (to nearest, as
// convert_f32_kernel rounds), with 16-byte loads when the source allows.
__device__ __forceinline__ void stage_values_rounded(const double* __restrict__ g, float* __restrict__ s,
                                                     size_t count, const Team& tm) {
    size_t i = 0;
    if ((reinterpret_cast<uintptr_t>(g) & 15) == 0) {
        const size_t nv = count / 2;
        const double2* gv = reinterpret_cast<const double2*>(g);
        float2* sv = reinterpret_cast<float2*>(s);
        for (size_t j = tm.tid; j < nv; j += tm.nt) {
            const double2 v = __ldg(gv + j);
            sv[j] = make_float2((float)v.x, (float)v.y);
        }
        i = nv * 2;
    }
    for (size_t j = i + tm.tid; j < count; j += tm.nt) s[j] = (float)ldg(g + j);
}

// Staged FP32 ELL values in each thread's own order: slot j of row t + q nt
// is entry (q k + j) nt + t of an FP32 value array and of a 16-bit column
// array after it (6 bytes a slot, so that three 256-thread blocks of the
// n = 1,024 batch fit in an SM's shared memory), and consecutive threads read
// consecutive entries. Padding slots and rows past n carry value 0 and column
// n, a zero kept after the end of every FP32 SpMV input vector, so the SpMV
// has no branch. The values are the FP32 copy's, or the FP64 values rounded
// to nearest as they are staged.
//
// With the width compiled in (K > 0, always odd: 3-, 5-, 7- and 9-point
// rows), the first K - 1 slots of each of a thread's rows are stored in
// groups side by side: quads of slots 4i..4i + 3 (one 16-byte load brings
// their values, one 8-byte load their columns), then a pair when K - 1 is not
// a multiple of 4 (8- and 4-byte loads), then the row's last slot alone.
// Same bytes, fewer shared-memory loads in the SpMV (for K = 9: 15 per row
// instead of 27), and the same order of accumulation.
template <int K>
struct SlotGroups {
    static_assert(K % 2 == 1, "the grouped layout is for odd ELL widths");
    static constexpr int NQ = (K - 1) / 4;        // quads per row
    static constexpr int NP = ((K - 1) % 4) / 2;  // pairs per row (0 or 1)
};

template <int R, int K>
__device__ __forceinline__ int paired_slot(int q, int j, int nt, int tid) {
    constexpr int NQ = SlotGroups<K>::NQ, NP = SlotGroups<K>::NP;
    if (j < 4 * NQ) return ((q * NQ + (j >> 2)) * nt + tid) * 4 + (j & 3);
    if (j < 4 * NQ + 2 * NP) return 4 * R * NQ * nt + (q * nt + tid) * 2 + ((j - 4 * NQ) & 1);
    return (4 * NQ + 2 * NP) * R * nt + q * nt + tid;
}

template <int R, int K = 0>
__device__ __forceinline__ void stage_pairs_ell(const double* __restrict__ g64, const float* __restrict__ g32,
                                                const int32_t* __restrict__ cols, float* __restrict__ vals,
                                                int n, int k, const Team& tm) {
    uint16_t* cl = reinterpret_cast<uint16_t*>(vals + (size_t)R * k * tm.nt);
#pragma unroll
    for (int q = 0; q < R; ++q) {
        const int row = tm.row(q);
        for (int j = 0; j < k; ++j) {
            float v = 0.0f;
            int c = n;
            if (row < n) {
                const size_t i = (size_t)j * n + row;
                const int cc = ldg(cols + i);
                if (cc >= 0) {
                    c = cc;
                    v = g32 != nullptr ? ldg(g32 + i) : (float)ldg(g64 + i);
                }
            }
            size_t o;
            if constexpr (K > 0)
                o = (size_t)paired_slot<R, K>(q, j, tm.nt, tm.tid);
            else
                o = (size_t)(q * k + j) * tm.nt + tm.tid;
            vals[o] = v;
            cl[o] = (uint16_t)c;
        }
    }
}

// y = A x over the staged values and columns (slots in ascending column
// order, FMA). K > 0 fixes the ELL width at compile time (the multi-level
// dispatch of Sec. 3.3 applied to the stencil width): the slot loop then
// unrolls fully, every entry sits at a constant multiple of the thread
// stride, and the R rows' FMA chains interleave. K = 0 takes the width k at
// run time.
template <int R, int K = 0>
struct PairOp32 {
    const float* __restrict__ vals;
    int k;
    __device__ __forceinline__ void apply(const float* __restrict__ xs, float (&y)[R], const Team& tm) const {
        const int kk = K > 0 ? K : k;
        const uint16_t* cl = reinterpret_cast<const uint16_t*>(vals + (size_t)R * kk * tm.nt);
        const int nt = tm.nt;
        if constexpr (K > 0) {  // the grouped layout of stage_pairs_ell
            constexpr int NQ = SlotGroups<K>::NQ, NP = SlotGroups<K>::NP;
            const float4* v4 = reinterpret_cast<const float4*>(vals);
            const uint2* c4 = reinterpret_cast<const uint2*>(cl);
            const float2* v2 = reinterpret_cast<const float2*>(vals + 4 * R * NQ * nt);
            const uint32_t* c2 = reinterpret_cast<const uint32_t*>(cl + 4 * R * NQ * nt);
            const float* v1 = vals + (4 * NQ + 2 * NP) * R * nt;
            const uint16_t* c1 = cl + (4 * NQ + 2 * NP) * R * nt;
            float sum[R];
#pragma unroll
            for (int q = 0; q < R; ++q) sum[q] = 0.0f;
#pragma unroll
            for (int g = 0; g < NQ; ++g) {
#pragma unroll
                for (int q = 0; q < R; ++q) {
                    const int o = (q * NQ + g) * nt + tm.tid;
                    const float4 a = v4[o];
                    const uint2 cc = c4[o];
                    sum[q] = fmaf(a.x, xs[cc.x & 0xffffu], sum[q]);
                    sum[q] = fmaf(a.y, xs[cc.x >> 16], sum[q]);
                    sum[q] = fmaf(a.z, xs[cc.y & 0xffffu], sum[q]);
                    sum[q] = fmaf(a.w, xs[cc.y >> 16], sum[q]);
                }
            }
            if constexpr (NP > 0) {
#pragma unroll
                for (int q = 0; q < R; ++q) {
                    const int o = q * nt + tm.tid;
                    const float2 a = v2[o];
                    const uint32_t cc = c2[o];
                    sum[q] = fmaf(a.x, xs[cc & 0xffffu], sum[q]);
                    sum[q] = fmaf(a.y, xs[cc >> 16], sum[q]);
                }
            }
#pragma unroll
            for (int q = 0; q < R; ++q) {
                const int o = q * nt + tm.tid;
                y[q] = fmaf(v1[o], xs[c1[o]], sum[q]);
            }
        } else {
#pragma unroll
            for (int q = 0; q < R; ++q) {
                float sum = 0.0f;
                for (int j = 0; j < kk; ++j) {
                    const int o = (q * kk + j) * nt + tm.tid;
                    sum = fmaf(vals[o], xs[cl[o]], sum);
                }
                y[q] = sum;
            }
        }
    }
};

// The refinement loop of one system: r = b - A x in FP64, exit test, FP32
// inner solve for the correction direction d, x += ||r|| d in FP64.
template <int FMT, int R, class Op32>
__device__ __forceinline__ void refine_system(const SolveParams& P, const SysIO& io,
                                              const Op<FMT, R, double, double>& op64, const Op32& op32,
                                              const float (&dinv)[R], double* red64, double* xd, float* red32,
                                              float* xa, float* xb, const Team& tm) {
    const int n = P.n;
    int par64 = 0, par32 = 0;
    // Neither b nor x is held in registers through the inner solves (which
    // need every register): b is re-read from memory for each residual, and
    // x lives in xd, the shared FP64 vector the residual's SpMV reads (each
    // thread updates its own rows).
    double r[R];
    float w[R], d[R];
    double bb = 0.0;
#pragma unroll
    for (int q = 0; q < R; ++q) {
        const int row = tm.row(q);
        if (row < n) {
            const double bq = io.b[row];
            xd[row] = io.x[row];
            bb = fma(bq, bq, bb);
        }
    }
    double s0[1] = {bb};
    block_sum(s0, red64, par64, tm);
    const double nb2 = s0[0];
    if (!finite(nb2) || nb2 == 0.0) {  // x stays x0, or x = 0
        double x[R];
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const int row = tm.row(q);
            x[q] = (nb2 == 0.0 || row >= n) ? 0.0 : xd[row];
        }
        if (nb2 == 0.0)
            write_result(io, x, ST_CONVERGED, 0, 0.0, 0, tm);
        else
            write_result(io, x, ST_NAN, 0, quiet_nan(), 0, tm);
        return;
    }
    const double tau2 = (P.tol_type == 1) ? P.tol * P.tol * nb2 : P.tol * P.tol;
    int status = -1, k = 0, inner_total = 0;
    double rr = 0.0;
    for (k = 0;; ++k) {
        {  // r = b - A x in FP64
            tm.sync();
            double ax[R];
            op64.apply(xd, ax, tm);
#pragma unroll
            for (int q = 0; q < R; ++q) {
                const int row = tm.row(q);
                r[q] = (row < n ? io.b[row] : 0.0) - ax[q];
            }
            double s1[1] = {pdot(r, r)};
            block_sum(s1, red64, par64, tm);
            rr = s1[0];
        }
        if (!finite(rr)) { status = ST_NAN; break; }
        if (rr <= tau2) { status = ST_CONVERGED; break; }
        if (k >= P.max_outer) { status = ST_MAX_ITER; break; }
        const double rn = sqrt(rr);
        const double rinv = 1.0 / rn;
#pragma unroll
        for (int q = 0; q < R; ++q) w[q] = (float)(r[q] * rinv);
        inner_total += inner_bicgstab32<R>(op32, dinv, w, d, (float)P.inner_tol, P.max_iters, xa, xb, red32,
                                           par32, tm, n);
        tm.sync();  // every thread is done reading xd (the inner solve has no FP64 reads of it)
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const int row = tm.row(q);
            if (row < n) xd[row] = fma(rn, (double)d[q], xd[row]);
        }
    }
    double x[R];
#pragma unroll
    for (int q = 0; q < R; ++q) {
        const int row = tm.row(q);
        x[q] = row < n ? xd[row] : 0.0;
    }
    write_result(io, x, status, k, sqrt(rr / nb2), inner_total, tm);
}

// Shared memory: red64[256] | xd[n_pad] (FP64) | red32[256] | xa[n_pad + 2] |
// xb[n_pad + 2] (FP32; entry n stays 0) | staged FP32 values (optional; on
// ELL values and 16-bit columns, 6 bytes a slot). K > 0 (ELL with staged
// values, at most 256 threads): the SpMV for an ELL width of exactly K, and
// three resident blocks per SM (80 registers), which hide more of the inner
// iteration's reduction and barrier latency than two.
template <int FMT, int R, int K = 0>
__global__ void __launch_bounds__(K > 0 ? 256 : max_threads_for(R), K > 0 ? 3 : 1)
    refine_kernel(const SolveParams P) {
    extern __shared__ __align__(16) unsigned char raw[];
    const Team tm = Team::block();
    const int sys = blockIdx.x;
    const int n = P.n;
    const SysIO io = sys_io(P, sys);
    double* red64 = reinterpret_cast<double*>(raw);
    double* xd = red64 + 256;
    float* red32 = reinterpret_cast<float*>(xd + P.n_pad);
    float* xa = red32 + 256;
    float* xb = xa + P.n_pad + 2;

    const Mat<double> A64{P.values + (size_t)sys * P.vps, P.row_ptrs, P.cols, n, P.k};
    const Op<FMT, R, double, double> op64{A64, nullptr};
    // Without an FP32 copy (values32 == nullptr, only when the values are
    // staged) the block rounds the FP64 values to FP32 as it stages them.
    const bool copy32 = P.values32 != nullptr;
    const Mat<float> A32{copy32 ? P.values32 + (size_t)sys * P.vps : nullptr, P.row_ptrs, P.cols, n, P.k};
    float dinv[R];
    if (copy32)
        jacobi_setup<FMT, R>(A32, P.precond == 1, dinv, tm);
    else  // 1 / a_ii in FP32 of the FP32-rounded diagonal, as from a copy
        jacobi_setup<FMT, R>(A64, P.precond == 1, dinv, tm);
    if (tm.tid == 0) {
        xa[n] = 0.0f;
        xb[n] = 0.0f;
    }
    if constexpr (FMT == FMT_ELL) {
        if (P.stage) {
            float* vals = reinterpret_cast<float*>(raw + P.stage_off);
            stage_pairs_ell<R, K>(A64.vals, A32.vals, P.cols, vals, n, P.k, tm);
            tm.sync();
            const PairOp32<R, K> op32{vals, P.k};
            refine_system<FMT, R>(P, io, op64, op32, dinv, red64, xd, red32, xa, xb, tm);
            return;
        }
    }
    const float* as = nullptr;
    if (P.stage) {
        float* s = reinterpret_cast<float*>(raw + P.stage_off);
        if (copy32)
            stage_values(A32.vals, s, P.vps, tm);
        else
            stage_values_rounded(A64.vals, s, P.vps, tm);
        as = s;
    }
    tm.sync();
    const Op<FMT, R, float, float> op32{A32, as};
    refine_system<FMT, R>(P, io, op64, op32, dinv, red64, xd, red32, xa, xb, tm);
}

// FP32 copy of the values for the mixed mode (when the caller gives none).
__global__ void convert_f32_kernel(const double* __restrict__ src, float* __restrict__ dst,
                                   size_t count);

}  // namespace bbs
