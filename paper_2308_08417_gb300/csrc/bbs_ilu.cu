// BiCGSTAB with a batched ILU(0) preconditioner on BatchCsr (Table "Batched
// feature support": BatchIlu, applied through BatchTrsv-style triangular
// solves), one block per system.
//
// ILU(0) keeps the sparsity pattern: A ~ L U with L unit lower and U upper on
// the pattern of A, computed row by row (for each k < i stored in row i:
// a_ik /= u_kk, then a_ij -= a_ik u_kj for every j > k stored in rows i and
// k). Row i needs the finished rows k < i of its lower part, so rows are
// processed by level: level(i) = 1 + max level(k) over those k. The pattern is
// shared by the batch, so one analysis kernel computes the level schedule
// once per solve into the workspace; every block then factors its system in
// shared memory level by level, and applies M^-1 = U^-1 L^-1 by a forward and
// a backward level-scheduled triangular solve in place in the SpMV input
// buffer. The SpMV itself keeps reading the original values.
#include <cstdint>

#include <cuda_runtime.h>

#include "bbs_ilu.cuh"
#include "bbs_kernels.h"
#include "bbs_solvers.cuh"

namespace bbs {


// Serial analysis of the shared pattern by one thread (n <= 2048).
__global__ void ilu_analysis_kernel(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                    int* __restrict__ ws) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    int* levL_ptr = ws + 2;
    int* rowsL = levL_ptr + n + 1;
    int* levU_ptr = rowsL + n;
    int* rowsU = levU_ptr + n + 1;
    int* diag_pos = rowsU + n;
    int* lev = diag_pos + n;
    for (int pass = 0; pass < 2; ++pass) {
        int* ptr = pass == 0 ? levL_ptr : levU_ptr;
        int* rows = pass == 0 ? rowsL : rowsU;
        int nlev = 0;
        for (int t = 0; t < n; ++t) {
            const int i = pass == 0 ? t : n - 1 - t;
            int L = 0;
            for (int e = rp[i]; e < rp[i + 1]; ++e) {
                const int k = ci[e];
                if ((pass == 0 && k < i) || (pass == 1 && k > i)) L = max(L, lev[k] + 1);
            }
            lev[i] = L;
            nlev = max(nlev, L + 1);
        }
        for (int l = 0; l <= nlev; ++l) ptr[l] = 0;
        for (int i = 0; i < n; ++i) ++ptr[lev[i] + 1];
        for (int l = 0; l < nlev; ++l) ptr[l + 1] += ptr[l];
        for (int t = 0; t < n; ++t) {  // stable placement, ascending (lower) / descending (upper) rows
            const int i = pass == 0 ? t : n - 1 - t;
            rows[ptr[lev[i]]++] = i;
        }
        for (int l = nlev; l > 0; --l) ptr[l] = ptr[l - 1];
        ptr[0] = 0;
        ws[pass] = nlev;
    }
    for (int i = 0; i < n; ++i) {
        int d = -1;
        for (int e = rp[i]; e < rp[i + 1]; ++e)
            if (ci[e] == i) d = e;
        diag_pos[i] = d;
    }
}

// In-place factorisation of the staged values `lu` (level by level).
__device__ __forceinline__ void ilu_factor(const Mat<double>& A, double* lu, double* udinv,
                                           const IluSchedule& S, const Team& tm) {
    for (int l = 1; l < S.nlevL; ++l) {  // level-0 rows have no lower part
        for (int t = S.levL_ptr[l] + tm.tid; t < S.levL_ptr[l + 1]; t += tm.nt) {
            const int i = S.rowsL[t];
            const int e0 = ldg(A.row_ptrs + i), e1 = ldg(A.row_ptrs + i + 1);
            for (int e = e0; e < e1; ++e) {
                const int k = ldg(A.cols + e);
                if (k >= i) break;
                const int dk = S.diag_pos[k];
                double piv = dk >= 0 ? lu[dk] : 0.0;
                if (piv == 0.0) piv = 1.0;
                const double lik = lu[e] / piv;
                lu[e] = lik;
                // a_ij -= l_ik u_kj for j > k present in both rows (merge of sorted rows)
                int f = ldg(A.row_ptrs + k);
                const int f1 = ldg(A.row_ptrs + k + 1);
                for (int g = e + 1; g < e1; ++g) {
                    const int j = ldg(A.cols + g);
                    while (f < f1 && ldg(A.cols + f) < j) ++f;
                    if (f < f1 && ldg(A.cols + f) == j) lu[g] = fma(-lik, lu[f], lu[g]);
                }
            }
        }
        tm.sync();
    }
    for (int i = tm.tid; i < A.n; i += tm.nt) {
        const int d = S.diag_pos[i];
        const double u = d >= 0 ? lu[d] : 0.0;
        udinv[i] = (u != 0.0) ? 1.0 / u : 1.0;
    }
    tm.sync();
}

// z = U^-1 L^-1 v in place in the shared vector `buf`.
__device__ __forceinline__ void ilu_apply(const Mat<double>& A, const double* lu, const double* udinv,
                                          double* buf, const IluSchedule& S, const Team& tm) {
    for (int l = 1; l < S.nlevL; ++l) {
        for (int t = S.levL_ptr[l] + tm.tid; t < S.levL_ptr[l + 1]; t += tm.nt) {
            const int i = S.rowsL[t];
            double sum = buf[i];
            const int e1 = ldg(A.row_ptrs + i + 1);
            for (int e = ldg(A.row_ptrs + i); e < e1; ++e) {
                const int k = ldg(A.cols + e);
                if (k >= i) break;
                sum = fma(-lu[e], buf[k], sum);
            }
            buf[i] = sum;
        }
        tm.sync();
    }
    for (int l = 0; l < S.nlevU; ++l) {
        for (int t = S.levU_ptr[l] + tm.tid; t < S.levU_ptr[l + 1]; t += tm.nt) {
            const int i = S.rowsU[t];
            double sum = buf[i];
            const int e0 = ldg(A.row_ptrs + i);
            for (int e = ldg(A.row_ptrs + i + 1) - 1; e >= e0; --e) {
                const int j = ldg(A.cols + e);
                if (j <= i) break;
                sum = fma(-lu[e], buf[j], sum);
            }
            buf[i] = sum * udinv[i];
        }
        tm.sync();
    }
}

// Right-preconditioned BiCGSTAB, M = (L U)^-1 from ILU(0); same exit,
// confirmation, breakdown and logging rules as the Jacobi solvers.
// Shared memory: red [256] | xa [n_pad] | xb [n_pad] | lu [nnz, 16-aligned] | udinv [n_pad]
template <int R>
__global__ void __launch_bounds__(max_threads_for(R), 1) bicgstab_ilu_kernel(const SolveParams P, const int* sched) {
    extern __shared__ __align__(16) unsigned char raw[];
    const Team tm = Team::block();
    const int sys = blockIdx.x;
    const int n = P.n;
    const TeamSmem sm = team_smem(raw, P.n_pad);
    double* lu = reinterpret_cast<double*>(raw + P.stage_off);
    double* udinv = lu + ((P.vps + 1) & ~(size_t)1);
    const Mat<double> A{P.values + (size_t)sys * P.vps, P.row_ptrs, P.cols, n, 0};
    const Op<FMT_CSR, R, double, double> op{A, nullptr};
    const IluSchedule S = ilu_schedule(sched, n);
    stage_values(A.vals, lu, P.vps, tm);
    tm.sync();
    ilu_factor(A, lu, udinv, S, tm);

    const SysIO io = sys_io(P, sys);
    int parity = 0;
    double b[R], x[R], r[R], rh[R], p[R], v[R], t[R];
    load_system<R>(io, b, x, tm);
    double rr = true_residual(op, b, x, r, sm.xa, sm.red, parity, tm, n);
    double s0[1] = {pdot(b, b)};
    block_sum(s0, sm.red, parity, tm);
    const double nb2 = s0[0];
    if (!finite64(nb2)) {
        write_result(io, x, ST_NAN, 0, quiet_nan(), 0, tm);
        return;
    }
    if (zero64(nb2)) {
#pragma unroll
        for (int q = 0; q < R; ++q) x[q] = 0.0;
        write_result(io, x, ST_CONVERGED, 0, 0.0, 0, tm);
        return;
    }
    const double tau2 = (P.tol_type == 1) ? P.tol * P.tol * nb2 : P.tol * P.tol;
    int status = -1, iters = 0;
    double res2 = rr;
    bool have_res = true;
    if (!finite64(rr)) {
        status = ST_NAN;
    } else if (le_nonneg64(rr, tau2)) {
        status = ST_CONVERGED;
    } else {
        double rho = rr, rho_old = 1.0, alpha = 1.0, omega = 1.0;
        int restarts = 0;
#pragma unroll
        for (int q = 0; q < R; ++q) {
            rh[q] = r[q];
            p[q] = 0.0;
            v[q] = 0.0;
        }
        have_res = false;
        for (int it = 1; it <= P.max_iters; ++it) {
            iters = it;
            if (!finite64(rho)) { status = ST_NAN; break; }
            if (zero64(rho)) { status = ST_BREAKDOWN; break; }
            const double beta = (rho * alpha) / (rho_old * omega);
#pragma unroll
            for (int q = 0; q < R; ++q) p[q] = fma(beta, fma(-omega, v[q], p[q]), r[q]);
            put(sm.xa, p, tm, n);
            tm.sync();
            ilu_apply(A, lu, udinv, sm.xa, S, tm);  // xa = p^
            op.apply(sm.xa, v, tm);
            double s1[1] = {pdot(rh, v)};
            block_sum(s1, sm.red, parity, tm);
            const double sigma = s1[0];
            if (!finite64(sigma)) { status = ST_NAN; break; }
            if (zero64(sigma)) { status = ST_BREAKDOWN; break; }
            alpha = rho / sigma;
#pragma unroll
            for (int q = 0; q < R; ++q) r[q] = fma(-alpha, v[q], r[q]);  // r holds s
            put(sm.xb, r, tm, n);
            tm.sync();
            ilu_apply(A, lu, udinv, sm.xb, S, tm);  // xb = s^
            op.apply(sm.xb, t, tm);
            double s3[3] = {pdot(r, r), pdot(t, t), pdot(t, r)};
            block_sum(s3, sm.red, parity, tm);
            const double ss = s3[0], tt = s3[1], ts = s3[2];
            if (!finite64(ss)) { status = ST_NAN; break; }
            bool candidate;
            double rho_next = 0.0;
            if (le_nonneg64(ss, tau2)) {
#pragma unroll
                for (int q = 0; q < R; ++q) {
                    const int row = tm.row(q);
                    if (row < n) x[q] = fma(alpha, sm.xa[row], x[q]);
                }
                candidate = true;
            } else {
                if (!finite64(tt) || !finite64(ts)) { status = ST_NAN; break; }
                omega = zero64(tt) ? 0.0 : ts / tt;
#pragma unroll
                for (int q = 0; q < R; ++q) {
                    const int row = tm.row(q);
                    if (row < n) x[q] = fma(omega, sm.xb[row], fma(alpha, sm.xa[row], x[q]));
                    r[q] = fma(-omega, t[q], r[q]);
                }
                double s2[2] = {pdot(r, r), pdot(rh, r)};
                block_sum(s2, sm.red, parity, tm);
                rr = s2[0];
                rho_next = s2[1];
                if (!finite64(rr)) { status = ST_NAN; break; }
                candidate = le_nonneg64(rr, tau2);
            }
            if (candidate) {
                res2 = true_residual(op, b, x, r, sm.xa, sm.red, parity, tm, n);
                have_res = true;
                if (!finite64(res2)) { status = ST_NAN; break; }
                if (le_nonneg64(res2, tau2)) { status = ST_CONVERGED; break; }
                if (++restarts > kMaxRestarts) { status = ST_MAX_ITER; break; }
                have_res = false;
#pragma unroll
                for (int q = 0; q < R; ++q) {
                    rh[q] = r[q];
                    p[q] = 0.0;
                    v[q] = 0.0;
                }
                rho = res2;
                rho_old = alpha = omega = 1.0;
                continue;
            }
            if (zero64(omega)) { status = ST_BREAKDOWN; break; }
            rho_old = rho;
            rho = rho_next;
        }
        if (status < 0) status = ST_MAX_ITER;
    }
    if (!have_res) res2 = true_residual(op, b, x, r, sm.xa, sm.red, parity, tm, n);
    write_result(io, x, status, iters, sqrt(res2 / nb2), 0, tm);
}

const void* bicgstab_ilu_fn(int R) {
    static const void* const kTable[kMaxR] = {
        (const void*)bicgstab_ilu_kernel<1>, (const void*)bicgstab_ilu_kernel<2>,
        (const void*)bicgstab_ilu_kernel<3>, (const void*)bicgstab_ilu_kernel<4>,
        (const void*)bicgstab_ilu_kernel<5>, (const void*)bicgstab_ilu_kernel<6>,
        (const void*)bicgstab_ilu_kernel<7>, (const void*)bicgstab_ilu_kernel<8>};
    return kTable[R - 1];
}

const void* bicgstab_ilu_packed_fn(int L, int R) {
    return L == 4 ? bicgstab_ilu_packed_fn_l4(R) : L == 8 ? bicgstab_ilu_packed_fn_l8(R)
                                                        : bicgstab_ilu_packed_fn_l16(R);
}

size_t ilu_workspace_bytes(int n) { return ilu_schedule_ints(n) * sizeof(int); }

cudaError_t launch_ilu_analysis(int n, const int32_t* rp, const int32_t* ci, int* ws, cudaStream_t st) {
    ilu_analysis_kernel<<<1, 32, 0, st>>>(n, rp, ci, ws);
    return cudaGetLastError();
}

}  // namespace bbs
