// Fused batched Krylov kernels: one thread block per system, one launch per
// batch (Sec. 3.2, 3.4). Each kernel is instantiated per (format, rows per
// thread R) and chosen on the host (the multi-level dispatch of Sec. 3.3).
//
// Common rules (identical in every solver):
//   * stop when ||r||_2 <= tau, tau = tol*||b||_2 (relative) or tol
//     (absolute); compared as ||r||^2 <= tau^2;
//   * a passing recursive residual is confirmed with the true residual
//     b - A x; a failed confirmation restarts the method from the true
//     residual, at most kMaxRestarts times, then the system stops with
//     MAX_ITER;
//   * b = 0 gives x = 0 after 0 iterations;
//   * exact-zero denominators stop the system with BREAKDOWN, a non-finite
//     scalar with NAN;
//   * the log holds ||b - A x|| / ||b|| of the returned x.
#pragma once

#include "bbs_device.cuh"
#include "bbs_params.h"

namespace bbs {

template <int FMT, int R, typename T, typename V>
struct Op {
    Mat<V> A;
    const V* as;  // staged values (shared memory) or nullptr
    __device__ __forceinline__ void apply(const T* xs, T (&y)[R], const Team& tm) const {
        if (as != nullptr)
            spmv_staged<FMT, R>(A, as, xs, y, tm);
        else
            spmv<FMT, R>(A, xs, y, tm);
    }
};

// Shared memory of one team: red [256] | xa [n_pad] | xb [n_pad] | extra
struct TeamSmem {
    double* red;
    double* xa;
    double* xb;
    double* extra;
};

__device__ __forceinline__ TeamSmem team_smem(unsigned char* raw, int n_pad) {
    TeamSmem s;
    s.red = reinterpret_cast<double*>(raw);
    s.xa = s.red + 256;
    s.xb = s.xa + n_pad;
    s.extra = s.xb + n_pad;
    return s;
}

// One system's vectors and log entries.
struct SysIO {
    const double* b;
    double* x;
    int32_t* iters;
    double* rel_res;
    int32_t* status;
    int32_t* inner;  // may be null
    int n;
};

struct SolveCfg {
    int precond, tol_type, max_iters, restart, max_outer;
    double tol, inner_tol;
    double* ws;  // this system's workspace slice (GMRES basis) or null
};

__device__ __forceinline__ SysIO sys_io(const SolveParams& P, int sys) {
    SysIO io;
    io.b = P.b + (size_t)sys * P.n;
    io.x = P.x + (size_t)sys * P.n;
    io.iters = P.iters + sys;
    io.rel_res = P.rel_res + sys;
    io.status = P.status + sys;
    io.inner = P.inner_iters != nullptr ? P.inner_iters + sys : nullptr;
    io.n = P.n;
    return io;
}

__device__ __forceinline__ SolveCfg solve_cfg(const SolveParams& P, int sys) {
    SolveCfg c;
    c.precond = P.precond;
    c.tol_type = P.tol_type;
    c.max_iters = P.max_iters;
    c.restart = P.restart;
    c.max_outer = P.max_outer;
    c.tol = P.tol;
    c.inner_tol = P.inner_tol;
    c.ws = P.ws != nullptr ? P.ws + (size_t)sys * (P.restart + 1) * P.n_pad : nullptr;
    return c;
}

// Residual r = b - A x (x staged through xs) and ||r||^2.
template <int FMT, int R, typename V>
__device__ __forceinline__ double true_residual(const Op<FMT, R, double, V>& op,
                                                const double (&b)[R], const double (&x)[R],
                                                double (&r)[R], double* xs, double* red,
                                                int& parity, const Team& tm, int n) {
    put(xs, x, tm, n);
    tm.sync();
    double ax[R];
    op.apply(xs, ax, tm);
#pragma unroll
    for (int q = 0; q < R; ++q) r[q] = b[q] - ax[q];
    double s[1] = {pdot(r, r)};
    block_sum(s, red, parity, tm);
    return s[0];
}

template <int R>
__device__ __forceinline__ void write_result(const SysIO& io, const double (&x)[R], int status,
                                             int iters, double rel, int inner, const Team& tm) {
#pragma unroll
    for (int q = 0; q < R; ++q) {
        const int row = tm.row(q);
        if (row < io.n) io.x[row] = x[q];
    }
    if (tm.tid == 0) {
        *io.iters = iters;
        *io.rel_res = rel;
        *io.status = status;
        if (io.inner != nullptr) *io.inner = inner;
    }
}

template <int R>
__device__ __forceinline__ void load_system(const SysIO& io, double (&b)[R], double (&x)[R],
                                            const Team& tm) {
#pragma unroll
    for (int q = 0; q < R; ++q) {
        const int row = tm.row(q);
        b[q] = (row < io.n) ? io.b[row] : 0.0;
        x[q] = (row < io.n) ? io.x[row] : 0.0;
    }
}

// The default quiet NaN (sign 0, exponent all ones, top fraction bit set).
__device__ __forceinline__ double quiet_nan() { return __longlong_as_double(0x7ff8000000000000LL); }

// The system's values, staged in shared memory at `stage` when non-null.
template <int FMT, int R>
__device__ __forceinline__ Op<FMT, R, double, double> make_op(const Mat<double>& A, size_t vps,
                                                              double* stage, const Team& tm) {
    if (stage != nullptr) {
        stage_values(A.vals, stage, vps, tm);
        tm.sync();
    }
    return Op<FMT, R, double, double>{A, stage};
}

template <int FMT, int R>
__device__ __forceinline__ Op<FMT, R, double, double> make_op(const SolveParams& P, int sys,
                                                              unsigned char* raw, const Team& tm) {
    const Mat<double> A{P.values + (size_t)sys * P.vps, P.row_ptrs, P.cols, P.n, P.k};
    double* stage = P.stage ? reinterpret_cast<double*>(raw + P.stage_off) : nullptr;
    return make_op<FMT, R>(A, P.vps, stage, tm);
}

// ------------------------------------------------------------- BiCGSTAB

// omega = ts / tt and alpha / (rho omega) = alpha tt / (rho ts), the factor
// of the next beta = (rho' alpha) / (rho omega), from one division (one
// reciprocal of tt rho ts); where that product or a quotient leaves the
// normal range (systems scaled far from 1), plain divisions in the original
// form. omega = 0 for tt = 0.
__device__ __forceinline__ void omega_and_cfac(double tt, double ts, double rho, double alpha, double& omega,
                                               double& cfac) {
    const double den = tt * rho * ts;
    const double inv = 1.0 / den;
    const double qs = ts * inv, qt = tt * inv;  // 1 / (tt rho), 1 / (rho ts)
    omega = qs * (rho * ts);
    cfac = qt * (alpha * tt);
    if (!(normal64(den) && normal64(qs) && normal64(qt) && finite64(omega) && finite64(cfac))) {
        omega = zero64(tt) ? 0.0 : ts / tt;
        cfac = alpha / (rho * omega);
    }
}

// Right-preconditioned BiCGSTAB (van der Vorst), M = D^-1, per system:
//   rho = r^.r ; beta = (rho alpha)/(rho_old omega) ; p = r + beta (p - omega v)
//   p^ = M p ; v = A p^ ; alpha = rho / r^.v ; s = r - alpha v
//   s^ = M s ; t = A s^ ; omega = t.s / t.t ; x += alpha p^ + omega s^
//   r = s - omega t
// The three reductions per iteration are (r^.v), (s.s, t.t, t.s) and
// (r.r, r^.r); t is computed before the half-step test on ||s|| so that the
// s-test shares a reduction with omega (the t of an exiting iteration is
// simply unused).
template <int FMT, int R>
__device__ __forceinline__ void bicgstab_system(const Op<FMT, R, double, double>& op, const SysIO& io,
                                          const SolveCfg& C, const TeamSmem& sm, const Team& tm) {
    const int n = io.n;
    int parity = 0;
    double b[R], x[R], r[R], rh[R], p[R], v[R], dinv[R], t[R];
    load_system<R>(io, b, x, tm);
    jacobi_setup<FMT, R>(op.A, C.precond == 1, dinv, tm);

    put(sm.xa, x, tm, n);
    tm.sync();
    op.apply(sm.xa, t, tm);
#pragma unroll
    for (int q = 0; q < R; ++q) r[q] = b[q] - t[q];
    double s0[2] = {pdot(b, b), pdot(r, r)};
    block_sum(s0, sm.red, parity, tm);
    const double nb2 = s0[0];
    double rr = s0[1];

    int status = -1, iters = 0;
    double res2 = rr;  // squared true residual of x (valid when have_res)
    bool have_res = true;
    if (!finite(nb2)) {
        write_result(io, x, ST_NAN, 0, quiet_nan(), 0, tm);
        return;
    }
    if (nb2 == 0.0) {
#pragma unroll
        for (int q = 0; q < R; ++q) x[q] = 0.0;
        write_result(io, x, ST_CONVERGED, 0, 0.0, 0, tm);
        return;
    }
    const double tau2 = (C.tol_type == 1) ? C.tol * C.tol * nb2 : C.tol * C.tol;
    if (!finite(rr)) {
        status = ST_NAN;
    } else if (rr <= tau2) {
        status = ST_CONVERGED;
    } else {
        double rho = rr;  // r^ = r, so r^.r = ||r||^2
        double alpha = 1.0, omega = 1.0, cfac = 1.0;  // cfac: as in bicgstab_scaled_system
        int restarts = 0;
#pragma unroll
        for (int q = 0; q < R; ++q) {
            rh[q] = r[q];
            p[q] = 0.0;
            v[q] = 0.0;
        }
        have_res = false;
        for (int it = 1; it <= C.max_iters; ++it) {
            iters = it;
            if (!finite(rho)) { status = ST_NAN; break; }
            if (rho == 0.0) { status = ST_BREAKDOWN; break; }
            const double beta = rho * cfac;
#pragma unroll
            for (int q = 0; q < R; ++q) p[q] = fma(beta, fma(-omega, v[q], p[q]), r[q]);
            {
                double ph[R];
#pragma unroll
                for (int q = 0; q < R; ++q) ph[q] = dinv[q] * p[q];
                put(sm.xa, ph, tm, n);
            }
            tm.sync();
            op.apply(sm.xa, v, tm);
            double s1[1] = {pdot(rh, v)};
            block_sum(s1, sm.red, parity, tm);
            const double sigma = s1[0];
            if (!finite(sigma)) { status = ST_NAN; break; }
            if (sigma == 0.0) { status = ST_BREAKDOWN; break; }
            alpha = rho / sigma;
#pragma unroll
            for (int q = 0; q < R; ++q) r[q] = fma(-alpha, v[q], r[q]);  // r now holds s
            {
                double sh[R];
#pragma unroll
                for (int q = 0; q < R; ++q) sh[q] = dinv[q] * r[q];
                put(sm.xb, sh, tm, n);
            }
            tm.sync();
            op.apply(sm.xb, t, tm);
            double s3[3] = {pdot(r, r), pdot(t, t), pdot(t, r)};
            block_sum(s3, sm.red, parity, tm);
            const double ss = s3[0], tt = s3[1], ts = s3[2];
            if (!finite(ss)) { status = ST_NAN; break; }
            bool candidate;
            double rho_next = 0.0;
            if (ss <= tau2) {  // half-step exit: x += alpha p^
#pragma unroll
                for (int q = 0; q < R; ++q) {
                    const int row = tm.row(q);
                    if (row < n) x[q] = fma(alpha, sm.xa[row], x[q]);
                }
                candidate = true;
            } else {
                if (!finite(tt) || !finite(ts)) { status = ST_NAN; break; }
                omega_and_cfac(tt, ts, rho, alpha, omega, cfac);
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
                if (!finite(rr)) { status = ST_NAN; break; }
                candidate = (rr <= tau2);
            }
            if (candidate) {
                res2 = true_residual(op, b, x, r, sm.xa, sm.red, parity, tm, n);
                have_res = true;
                if (!finite(res2)) { status = ST_NAN; break; }
                if (res2 <= tau2) { status = ST_CONVERGED; break; }
                if (++restarts > kMaxRestarts) { status = ST_MAX_ITER; break; }
                have_res = false;
#pragma unroll
                for (int q = 0; q < R; ++q) {
                    rh[q] = r[q];
                    p[q] = 0.0;
                    v[q] = 0.0;
                }
                rho = res2;
                alpha = omega = cfac = 1.0;
                continue;
            }
            if (omega == 0.0) { status = ST_BREAKDOWN; break; }
            rho = rho_next;
        }
        if (status < 0) status = ST_MAX_ITER;
    }
    if (!have_res) res2 = true_residual(op, b, x, r, sm.xa, sm.red, parity, tm, n);
    write_result(io, x, status, iters, sqrt(res2 / nb2), 0, tm);
}

// Scale the staged values in place by the Jacobi inverse diagonal of their
// column, As = A D^-1 (each thread rescales the entries of its own rows; dinv
// is shared through `tmp` for the column lookups).
template <int FMT, int R>
__device__ __forceinline__ void scale_columns(const Mat<double>& A, double* as, const double (&dinv)[R],
                                              double* tmp, const Team& tm) {
    put(tmp, dinv, tm, A.n);
    tm.sync();
#pragma unroll
    for (int q = 0; q < R; ++q) {
        const int row = tm.row(q);
        if (row >= A.n) continue;
        if constexpr (FMT == FMT_CSR) {
            const int e1 = ldg(A.row_ptrs + row + 1);
            for (int e = ldg(A.row_ptrs + row); e < e1; ++e) as[e] *= tmp[ldg(A.cols + e)];
        } else if constexpr (FMT == FMT_ELL) {
            for (int j = 0; j < A.k; ++j) {
                const int col = ldg(A.cols + (size_t)j * A.n + row);
                if (col >= 0) as[(size_t)j * A.n + row] *= tmp[col];
            }
        } else {
            for (int j = 0; j < A.n; ++j) as[(size_t)row * A.n + j] *= tmp[j];
        }
    }
    tm.sync();
}

// BiCGSTAB with the Jacobi preconditioner folded into the staged matrix:
// with As = A D^-1 and x~ = D x, right-preconditioned BiCGSTAB on A x = b is
// plain BiCGSTAB on As x~ = b (p^ = D^-1 p and s^ = D^-1 s never need forming;
// x~ += alpha p + omega s). Same iterates as bicgstab_system up to rounding,
// two FP64 multiplies per row and iteration fewer. Scalar tests run on the
// integer pipe. Only the six vectors the iteration updates stay in registers
// (b, x0 and the diagonal are re-read from memory when needed), which keeps
// the register count, and so the number of resident systems, up. x = D^-1 x~
// on exit; a system that takes no iteration returns its x0 untouched.
template <int FMT, int R>
__device__ __forceinline__ double residual_from_global(const Op<FMT, R, double, double>& op,
                                                       const double* __restrict__ bg,
                                                       const double (&x)[R], double (&r)[R],
                                                       double* xs, double* red, int& parity,
                                                       const Team& tm, int n) {
    put(xs, x, tm, n);
    tm.sync();
    double ax[R];
    op.apply(xs, ax, tm);
#pragma unroll
    for (int q = 0; q < R; ++q) {
        const int row = tm.row(q);
        r[q] = (row < n ? bg[row] : 0.0) - ax[q];
    }
    double s[1] = {pdot(r, r)};
    block_sum(s, red, parity, tm);
    return s[0];
}

template <int FMT, int R>
__device__ __forceinline__ void bicgstab_scaled_system(const Op<FMT, R, double, double>& op,
                                                       const SysIO& io, const SolveCfg& C,
                                                       const TeamSmem& sm, const Team& tm) {
    const int n = io.n;
    int parity = 0;
    // p lives in shared memory only (xa, the SpMV input it is copied to
    // anyway), which leaves five register vectors
    double xs[R], r[R], rh[R], v[R], t[R];
    {
        double dinv[R];
        jacobi_setup<FMT, R>(op.A, true, dinv, tm);
        scale_columns<FMT, R>(op.A, const_cast<double*>(op.as), dinv, sm.xb, tm);
    }
#pragma unroll
    for (int q = 0; q < R; ++q) {  // x~ = D x0 (1 for a zero diagonal)
        const int row = tm.row(q);
        const double d = row < n ? diag_entry<FMT>(op.A, row) : 0.0;
        const double x0 = row < n ? io.x[row] : 0.0;
        xs[q] = (d != 0.0) ? d * x0 : x0;
    }
    double nb2;
    {
        double bb = 0.0;
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const int row = tm.row(q);
            const double bq = row < n ? io.b[row] : 0.0;
            bb = fma(bq, bq, bb);
        }
        double s0[1] = {bb};
        block_sum(s0, sm.red, parity, tm);
        nb2 = s0[0];
    }
    if (!finite64(nb2)) {  // x stays x0
        if (tm.tid == 0) {
            *io.iters = 0;
            *io.rel_res = quiet_nan();
            *io.status = ST_NAN;
        }
        return;
    }
    if (zero64(nb2)) {
#pragma unroll
        for (int q = 0; q < R; ++q) xs[q] = 0.0;
        write_result(io, xs, ST_CONVERGED, 0, 0.0, 0, tm);
        return;
    }
    double rr = residual_from_global(op, io.b, xs, r, sm.xa, sm.red, parity, tm, n);
    int status = -1, iters = 0;
    double res2 = rr;
    bool have_res = true;
    const double tau2 = (C.tol_type == 1) ? C.tol * C.tol * nb2 : C.tol * C.tol;
    if (!finite64(rr)) {
        status = ST_NAN;
    } else if (le_nonneg64(rr, tau2)) {
        status = ST_CONVERGED;
    } else {
        // beta = (rho alpha) / (rho_old omega): cfac holds alpha / (rho omega)
        // of the previous step, found with omega from one division
        double rho = rr, alpha = 1.0, omega = 1.0, cfac = 1.0;
        int restarts = 0;
        tm.sync();  // every thread is done reading xa (the residual's SpMV input)
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const int row = tm.row(q);
            rh[q] = r[q];
            v[q] = 0.0;
            if (row < n) sm.xa[row] = 0.0;  // p = 0
        }
        have_res = false;
        for (int it = 1; it <= C.max_iters; ++it) {
            iters = it;
            if (!finite64(rho)) { status = ST_NAN; break; }
            if (zero64(rho)) { status = ST_BREAKDOWN; break; }
            const double beta = rho * cfac;
#pragma unroll
            for (int q = 0; q < R; ++q) {
                const int row = tm.row(q);
                if (row < n) sm.xa[row] = fma(beta, fma(-omega, v[q], sm.xa[row]), r[q]);
            }
            tm.sync();
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
                    xs[q] = fma(alpha, row < n ? sm.xa[row] : 0.0, xs[q]);
                }
                candidate = true;
            } else {
                if (!finite64(tt) || !finite64(ts)) { status = ST_NAN; break; }
                omega_and_cfac(tt, ts, rho, alpha, omega, cfac);
#pragma unroll
                for (int q = 0; q < R; ++q) {
                    const int row = tm.row(q);
                    xs[q] = fma(omega, r[q], fma(alpha, row < n ? sm.xa[row] : 0.0, xs[q]));
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
                res2 = residual_from_global(op, io.b, xs, r, sm.xa, sm.red, parity, tm, n);
                have_res = true;
                if (!finite64(res2)) { status = ST_NAN; break; }
                if (le_nonneg64(res2, tau2)) { status = ST_CONVERGED; break; }
                if (++restarts > kMaxRestarts) { status = ST_MAX_ITER; break; }
                have_res = false;
                tm.sync();  // every thread is done reading xa (the residual's SpMV input)
#pragma unroll
                for (int q = 0; q < R; ++q) {
                    const int row = tm.row(q);
                    rh[q] = r[q];
                    v[q] = 0.0;
                    if (row < n) sm.xa[row] = 0.0;  // p = 0
                }
                rho = res2;
                alpha = omega = cfac = 1.0;
                continue;
            }
            if (zero64(omega)) { status = ST_BREAKDOWN; break; }
            rho = rho_next;
        }
        if (status < 0) status = ST_MAX_ITER;
    }
    if (!have_res) res2 = residual_from_global(op, io.b, xs, r, sm.xa, sm.red, parity, tm, n);
    if (iters > 0) {  // x = D^-1 x~ (1 for a zero diagonal)
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const int row = tm.row(q);
            if (row >= n) continue;
            const double d = diag_entry<FMT>(op.A, row);
            io.x[row] = (d != 0.0) ? xs[q] / d : xs[q];
        }
    }
    if (tm.tid == 0) {
        *io.iters = iters;
        *io.rel_res = sqrt(res2 / nb2);
        *io.status = status;
        if (io.inner != nullptr) *io.inner = 0;
    }
}

// BiCGSTAB entry: the folded form when the values are staged and Jacobi is on.
template <int FMT, int R>
__device__ __forceinline__ void bicgstab_any(const Op<FMT, R, double, double>& op, const SysIO& io,
                                             const SolveCfg& C, const TeamSmem& sm, const Team& tm) {
    if (op.as != nullptr && C.precond == 1)
        bicgstab_scaled_system<FMT, R>(op, io, C, sm, tm);
    else
        bicgstab_system<FMT, R>(op, io, C, sm, tm);
}

// ------------------------------------------------------------------- CG

// Alg. 1 (BatchCg) with the exit test on ||r||: t = A p ; alpha = rho/(p.t) ;
// x += alpha p ; r -= alpha t ; z = M r ; rho^ = r.z ; p = z + (rho^/rho) p.
// Two reductions per iteration: (p.t) and (r.r, r.z).
template <int FMT, int R>
__device__ __forceinline__ void cg_system(const Op<FMT, R, double, double>& op, const SysIO& io,
                                          const SolveCfg& C, const TeamSmem& sm, const Team& tm) {
    const int n = io.n;
    int parity = 0;
    double b[R], x[R], r[R], z[R], p[R], t[R], dinv[R];
    load_system<R>(io, b, x, tm);
    jacobi_setup<FMT, R>(op.A, C.precond == 1, dinv, tm);

    put(sm.xa, x, tm, n);
    tm.sync();
    op.apply(sm.xa, t, tm);
#pragma unroll
    for (int q = 0; q < R; ++q) {
        r[q] = b[q] - t[q];
        z[q] = dinv[q] * r[q];
    }
    double s0[3] = {pdot(b, b), pdot(r, r), pdot(r, z)};
    block_sum(s0, sm.red, parity, tm);
    const double nb2 = s0[0];
    double rr = s0[1], rho = s0[2];

    int status = -1, iters = 0;
    double res2 = rr;
    bool have_res = true;
    if (!finite(nb2)) {
        write_result(io, x, ST_NAN, 0, quiet_nan(), 0, tm);
        return;
    }
    if (nb2 == 0.0) {
#pragma unroll
        for (int q = 0; q < R; ++q) x[q] = 0.0;
        write_result(io, x, ST_CONVERGED, 0, 0.0, 0, tm);
        return;
    }
    const double tau2 = (C.tol_type == 1) ? C.tol * C.tol * nb2 : C.tol * C.tol;
    if (!finite(rr)) {
        status = ST_NAN;
    } else if (rr <= tau2) {
        status = ST_CONVERGED;
    } else {
        have_res = false;
        int restarts = 0;
#pragma unroll
        for (int q = 0; q < R; ++q) p[q] = z[q];
        for (int it = 1; it <= C.max_iters; ++it) {
            iters = it;
            if (!finite(rho)) { status = ST_NAN; break; }
            if (rho == 0.0) { status = ST_BREAKDOWN; break; }
            put(sm.xa, p, tm, n);
            tm.sync();
            op.apply(sm.xa, t, tm);
            double s1[1] = {pdot(p, t)};
            block_sum(s1, sm.red, parity, tm);
            const double pt = s1[0];
            if (!finite(pt)) { status = ST_NAN; break; }
            if (pt == 0.0) { status = ST_BREAKDOWN; break; }
            const double alpha = rho / pt;
#pragma unroll
            for (int q = 0; q < R; ++q) {
                x[q] = fma(alpha, p[q], x[q]);
                r[q] = fma(-alpha, t[q], r[q]);
                z[q] = dinv[q] * r[q];
            }
            double s2[2] = {pdot(r, r), pdot(r, z)};
            block_sum(s2, sm.red, parity, tm);
            rr = s2[0];
            const double rho_hat = s2[1];
            if (!finite(rr)) { status = ST_NAN; break; }
            if (rr <= tau2) {
                put(sm.xa, x, tm, n);
                tm.sync();
                op.apply(sm.xa, t, tm);
#pragma unroll
                for (int q = 0; q < R; ++q) {
                    r[q] = b[q] - t[q];
                    z[q] = dinv[q] * r[q];
                }
                double s3[2] = {pdot(r, r), pdot(r, z)};
                block_sum(s3, sm.red, parity, tm);
                res2 = s3[0];
                have_res = true;
                if (!finite(res2)) { status = ST_NAN; break; }
                if (res2 <= tau2) { status = ST_CONVERGED; break; }
                if (++restarts > kMaxRestarts) { status = ST_MAX_ITER; break; }
                have_res = false;
#pragma unroll
                for (int q = 0; q < R; ++q) p[q] = z[q];
                rho = s3[1];
                continue;
            }
            const double ratio = rho_hat / rho;
#pragma unroll
            for (int q = 0; q < R; ++q) p[q] = fma(ratio, p[q], z[q]);
            rho = rho_hat;
        }
        if (status < 0) status = ST_MAX_ITER;
    }
    if (!have_res) res2 = true_residual(op, b, x, r, sm.xa, sm.red, parity, tm, n);
    write_result(io, x, status, iters, sqrt(res2 / nb2), 0, tm);
}

// ---------------------------------------------------------------- GMRES

// Restarted GMRES(m), right-preconditioned: Arnoldi with modified
// Gram-Schmidt (one reduction per basis vector), Givens rotations applied by
// thread 0 to the Hessenberg column in shared memory, residual estimate
// |g_{j+1}|; each Arnoldi step is one iteration. The basis V (m+1 vectors)
// lives in shared memory or, when it does not fit, in the workspace; each
// thread only touches its own rows of it.
template <int FMT, int R>
__device__ __forceinline__ void gmres_system(const Op<FMT, R, double, double>& op, const SysIO& io,
                                          const SolveCfg& C, const TeamSmem& sm, const Team& tm) {
    const int n = io.n;
    const int m = C.restart;
    int parity = 0;
    // extra: H[(m+1)*m] | cs[m] | sn[m] | g[m+1] | y[m] | ctl[4] | V (if in smem)
    double* H = sm.extra;
    double* cs = H + (m + 1) * m;
    double* sn = cs + m;
    double* g = sn + m;
    double* y = g + m + 1;
    int* ctl = reinterpret_cast<int*>(y + m);
    double* V = (C.ws != nullptr) ? C.ws : y + m + 2;
    const size_t vstride = (size_t)((n + 1) & ~1);

    double b[R], x[R], r[R], w[R], dinv[R];
    load_system<R>(io, b, x, tm);
    jacobi_setup<FMT, R>(op.A, C.precond == 1, dinv, tm);
    put(sm.xa, x, tm, n);
    tm.sync();
    op.apply(sm.xa, w, tm);
#pragma unroll
    for (int q = 0; q < R; ++q) r[q] = b[q] - w[q];
    double s0[2] = {pdot(b, b), pdot(r, r)};
    block_sum(s0, sm.red, parity, tm);
    const double nb2 = s0[0];
    double beta2 = s0[1];
    if (!finite(nb2)) {
        write_result(io, x, ST_NAN, 0, quiet_nan(), 0, tm);
        return;
    }
    if (nb2 == 0.0) {
#pragma unroll
        for (int q = 0; q < R; ++q) x[q] = 0.0;
        write_result(io, x, ST_CONVERGED, 0, 0.0, 0, tm);
        return;
    }
    const double tau2 = (C.tol_type == 1) ? C.tol * C.tol * nb2 : C.tol * C.tol;
    const double tau = sqrt(tau2);
    int status = -1, it = 0, restarts = 0;
    if (!finite(beta2))
        status = ST_NAN;
    else if (beta2 <= tau2)
        status = ST_CONVERGED;
    while (status < 0) {
        if (it >= C.max_iters) { status = ST_MAX_ITER; break; }
        const double beta = sqrt(beta2);
        const double binv = 1.0 / beta;
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const int row = tm.row(q);
            if (row < n) V[row] = r[q] * binv;
        }
        if (tm.tid == 0) {
            for (int i = 0; i <= m; ++i) g[i] = 0.0;
            g[0] = beta;
        }
        int k = 0, singular = 0, estimate_ok = 0;
        for (int j = 0; j < m; ++j) {
            ++it;
            const double* vj = V + (size_t)j * vstride;
            {
                double u[R];
#pragma unroll
                for (int q = 0; q < R; ++q) {
                    const int row = tm.row(q);
                    u[q] = (row < n) ? dinv[q] * vj[row] : 0.0;
                }
                put(sm.xa, u, tm, n);
            }
            tm.sync();
            op.apply(sm.xa, w, tm);
            bool bad = false;
            for (int i = 0; i <= j; ++i) {  // modified Gram-Schmidt
                const double* vi = V + (size_t)i * vstride;
                double vr[R];
#pragma unroll
                for (int q = 0; q < R; ++q) {
                    const int row = tm.row(q);
                    vr[q] = (row < n) ? vi[row] : 0.0;
                }
                double h[1] = {pdot(w, vr)};
                block_sum(h, sm.red, parity, tm);
                bad |= !finite(h[0]);
#pragma unroll
                for (int q = 0; q < R; ++q) w[q] = fma(-h[0], vr[q], w[q]);
                if (tm.tid == 0) H[i * m + j] = h[0];
            }
            double hw[1] = {pdot(w, w)};
            block_sum(hw, sm.red, parity, tm);
            const double hn = sqrt(hw[0]);
            bad |= !finite(hn);
            if (bad) { status = ST_NAN; break; }
            if (tm.tid == 0) {
                H[(j + 1) * m + j] = hn;
                for (int i = 0; i < j; ++i) {
                    const double a = H[i * m + j], c = H[(i + 1) * m + j];
                    H[i * m + j] = cs[i] * a + sn[i] * c;
                    H[(i + 1) * m + j] = -sn[i] * a + cs[i] * c;
                }
                const double a = H[j * m + j];
                const double denom = sqrt(a * a + hn * hn);
                int c0 = 0, c1 = 0, c2 = 0;
                if (denom == 0.0) {
                    c0 = j;
                    c1 = 1;
                } else {
                    cs[j] = a / denom;
                    sn[j] = hn / denom;
                    H[j * m + j] = denom;
                    H[(j + 1) * m + j] = 0.0;
                    g[j + 1] = -sn[j] * g[j];
                    g[j] = cs[j] * g[j];
                    c0 = j + 1;
                    c2 = (hn == 0.0 || fabs(g[j + 1]) <= tau) ? 1 : 0;
                }
                ctl[0] = c0;
                ctl[1] = c1;
                ctl[2] = c2;
            }
            tm.sync();
            k = ctl[0];
            singular = ctl[1];
            estimate_ok = ctl[2];
            tm.sync();  // ctl is rewritten by thread 0 in the next step
            if (singular || estimate_ok || it >= C.max_iters) break;
            const double hinv = 1.0 / hn;
            double* vn = V + (size_t)(j + 1) * vstride;
#pragma unroll
            for (int q = 0; q < R; ++q) {
                const int row = tm.row(q);
                if (row < n) vn[row] = w[q] * hinv;
            }
        }
        if (status >= 0) break;
        // y = H(0:k,0:k)^-1 g(0:k) ; x += M (V y)
        if (tm.tid == 0) {
            for (int i = k - 1; i >= 0; --i) {
                double sum = g[i];
                for (int l = i + 1; l < k; ++l) sum -= H[i * m + l] * y[l];
                y[i] = sum / H[i * m + i];
            }
        }
        tm.sync();
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const int row = tm.row(q);
            if (row < n) {
                double sum = 0.0;
                for (int i = 0; i < k; ++i) sum = fma(y[i], V[(size_t)i * vstride + row], sum);
                x[q] = fma(dinv[q], sum, x[q]);
            }
        }
        beta2 = true_residual(op, b, x, r, sm.xa, sm.red, parity, tm, n);
        if (!finite(beta2)) { status = ST_NAN; break; }
        if (beta2 <= tau2) { status = ST_CONVERGED; break; }
        if (singular) { status = ST_BREAKDOWN; break; }
        if (it >= C.max_iters) { status = ST_MAX_ITER; break; }
        if (estimate_ok && ++restarts > kMaxRestarts) { status = ST_MAX_ITER; break; }
    }
    double res2 = beta2;
    if (status == ST_NAN) res2 = true_residual(op, b, x, r, sm.xa, sm.red, parity, tm, n);
    if (C.ws != nullptr) {  // a basis in the workspace is dead scratch now: drop its
                            // whole 128-byte lines from L2 without a write-back
        tm.sync();
        const uintptr_t first = (reinterpret_cast<uintptr_t>(V) + 127) & ~static_cast<uintptr_t>(127);
        const uintptr_t end =
            (reinterpret_cast<uintptr_t>(V) + (size_t)(m + 1) * vstride * 8) & ~static_cast<uintptr_t>(127);
        for (uintptr_t a = first + (uintptr_t)tm.tid * 128; a < end; a += (uintptr_t)tm.nt * 128)
            asm volatile("discard.global.L2 [%0], 128;" ::"l"(a) : "memory");
    }
    write_result(io, x, status, it, sqrt(res2 / nb2), 0, tm);
}

// ----------------------------------------------------- one block per system

#define BBS_UNIFORM_KERNEL(NAME, SYSTEM)                                                       \
    template <int FMT, int R>                                                                  \
    __global__ void __launch_bounds__(max_threads_for(R), 1) NAME(const SolveParams P) {       \
        extern __shared__ __align__(16) unsigned char raw[];                                   \
        const Team tm = Team::block();                                                         \
        const int sys = blockIdx.x;                                                            \
        const auto op = make_op<FMT, R>(P, sys, raw, tm);                                      \
        SYSTEM<FMT, R>(op, sys_io(P, sys), solve_cfg(P, sys), team_smem(raw, P.n_pad), tm);    \
    }

BBS_UNIFORM_KERNEL(bicgstab_kernel, bicgstab_system)
BBS_UNIFORM_KERNEL(cg_kernel, cg_system)
BBS_UNIFORM_KERNEL(gmres_kernel, gmres_system)
#undef BBS_UNIFORM_KERNEL

// The folded BiCGSTAB keeps six vectors in registers; at 5-6 rows per thread
// a cap of 128 registers holds them without spilling and doubles the systems
// an SM keeps resident (the FP64 pipe needs many warps to stay busy).
__host__ __device__ constexpr int folded_min_blocks(int R) { return (R == 5 || R == 6) ? 2 : 1; }

template <int FMT, int R>
__global__ void __launch_bounds__(max_threads_for(R), folded_min_blocks(R))
    bicgstab_folded_kernel(const SolveParams P) {
    extern __shared__ __align__(16) unsigned char raw[];
    const Team tm = Team::block();
    const int sys = blockIdx.x;
    const auto op = make_op<FMT, R>(P, sys, raw, tm);
    bicgstab_scaled_system<FMT, R>(op, sys_io(P, sys), solve_cfg(P, sys), team_smem(raw, P.n_pad), tm);
}
}  // namespace bbs
