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

// Shared-memory layout common to the FP64 solvers:
//   red [256] | xa [n_pad] | xb [n_pad] | extra solver space | staged values
struct Smem64 {
    double* red;
    double* xa;
    double* xb;
    double* extra;
};

__device__ __forceinline__ Smem64 smem64_layout(unsigned char* raw, int n_pad) {
    Smem64 s;
    s.red = reinterpret_cast<double*>(raw);
    s.xa = s.red + 256;
    s.xb = s.xa + n_pad;
    s.extra = s.xb + n_pad;
    return s;
}

// Residual r = b - A x (x staged through xs) and ||r||^2 for the log.
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
__device__ __forceinline__ void write_result(const SolveParams& P, int sys, const double (&x)[R],
                                             int status, int iters, double rel, int inner,
                                             const Team& tm) {
    double* xg = P.x + (size_t)sys * P.n;
#pragma unroll
    for (int q = 0; q < R; ++q) {
        const int row = tm.row(q);
        if (row < P.n) xg[row] = x[q];
    }
    if (tm.tid == 0) {
        P.iters[sys] = iters;
        P.rel_res[sys] = rel;
        P.status[sys] = status;
        if (P.inner_iters != nullptr) P.inner_iters[sys] = inner;
    }
}

template <int FMT, int R>
__device__ __forceinline__ void load_system(const SolveParams& P, int sys, double (&b)[R],
                                            double (&x)[R], const Team& tm) {
    const double* bg = P.b + (size_t)sys * P.n;
    const double* xg = P.x + (size_t)sys * P.n;
#pragma unroll
    for (int q = 0; q < R; ++q) {
        const int row = tm.row(q);
        b[q] = (row < P.n) ? bg[row] : 0.0;
        x[q] = (row < P.n) ? xg[row] : 0.0;
    }
}

// Prologue shared by the solvers: staging, b, x0, Jacobi, r0 = b - A x0 and
// (||b||^2, ||r0||^2). Returns the Op for this system.
template <int FMT, int R>
__device__ __forceinline__ Op<FMT, R, double, double> make_op(const SolveParams& P, int sys,
                                                              unsigned char* raw, size_t stage_off,
                                                              const Team& tm) {
    Mat<double> A{P.values + (size_t)sys * P.vps, P.row_ptrs, P.cols, P.n, P.k};
    const double* as = nullptr;
    if (P.stage) {
        double* s = reinterpret_cast<double*>(raw + stage_off);
        stage_values(A.vals, s, P.vps, tm);
        __syncthreads();
        as = s;
    }
    return Op<FMT, R, double, double>{A, as};
}

// ------------------------------------------------------------- BiCGSTAB

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
__global__ void __launch_bounds__(max_threads_for(R), 1) bicgstab_kernel(const SolveParams P) {
    extern __shared__ __align__(16) unsigned char raw[];
    const Team tm = Team::make();
    const int sys = blockIdx.x;
    const int n = P.n;
    const Smem64 sm = smem64_layout(raw, P.n_pad);
    const auto op = make_op<FMT, R>(P, sys, raw, P.stage_off, tm);
    int parity = 0;

    double b[R], x[R], r[R], rh[R], p[R], v[R], dinv[R], t[R];
    load_system<FMT, R>(P, sys, b, x, tm);
    jacobi_setup<FMT, R>(op.A, P.precond == 1, dinv, tm);

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
        write_result(P, sys, x, ST_NAN, 0, __longlong_as_double(0x7ff8000000000000LL), 0, tm);
        return;
    }
    if (nb2 == 0.0) {
#pragma unroll
        for (int q = 0; q < R; ++q) x[q] = 0.0;
        write_result(P, sys, x, ST_CONVERGED, 0, 0.0, 0, tm);
        return;
    }
    const double tau2 = (P.tol_type == 1) ? P.tol * P.tol * nb2 : P.tol * P.tol;
    if (!finite(rr)) {
        status = ST_NAN;
    } else if (rr <= tau2) {
        status = ST_CONVERGED;
    } else {
        double rho = rr;  // r^ = r, so r^.r = ||r||^2
        double rho_old = 1.0, alpha = 1.0, omega = 1.0;
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
            if (!finite(rho)) { status = ST_NAN; break; }
            if (rho == 0.0) { status = ST_BREAKDOWN; break; }
            const double beta = (rho * alpha) / (rho_old * omega);
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
                omega = (tt == 0.0) ? 0.0 : ts / tt;
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
                rho_old = alpha = omega = 1.0;
                continue;
            }
            if (omega == 0.0) { status = ST_BREAKDOWN; break; }
            rho_old = rho;
            rho = rho_next;
        }
        if (status < 0) status = ST_MAX_ITER;
    }
    if (!have_res) res2 = true_residual(op, b, x, r, sm.xa, sm.red, parity, tm, n);
    write_result(P, sys, x, status, iters, sqrt(res2 / nb2), 0, tm);
}

// ------------------------------------------------------------------- CG

// Alg. 1 (BatchCg) with the exit test on ||r||: t = A p ; alpha = rho/(p.t) ;
// x += alpha p ; r -= alpha t ; z = M r ; rho^ = r.z ; p = z + (rho^/rho) p.
// Two reductions per iteration: (p.t) and (r.r, r.z).
template <int FMT, int R>
__global__ void __launch_bounds__(max_threads_for(R), 1) cg_kernel(const SolveParams P) {
    extern __shared__ __align__(16) unsigned char raw[];
    const Team tm = Team::make();
    const int sys = blockIdx.x;
    const int n = P.n;
    const Smem64 sm = smem64_layout(raw, P.n_pad);
    const auto op = make_op<FMT, R>(P, sys, raw, P.stage_off, tm);
    int parity = 0;

    double b[R], x[R], r[R], z[R], p[R], t[R], dinv[R];
    load_system<FMT, R>(P, sys, b, x, tm);
    jacobi_setup<FMT, R>(op.A, P.precond == 1, dinv, tm);

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
        write_result(P, sys, x, ST_NAN, 0, __longlong_as_double(0x7ff8000000000000LL), 0, tm);
        return;
    }
    if (nb2 == 0.0) {
#pragma unroll
        for (int q = 0; q < R; ++q) x[q] = 0.0;
        write_result(P, sys, x, ST_CONVERGED, 0, 0.0, 0, tm);
        return;
    }
    const double tau2 = (P.tol_type == 1) ? P.tol * P.tol * nb2 : P.tol * P.tol;
    if (!finite(rr)) {
        status = ST_NAN;
    } else if (rr <= tau2) {
        status = ST_CONVERGED;
    } else {
        have_res = false;
        int restarts = 0;
#pragma unroll
        for (int q = 0; q < R; ++q) p[q] = z[q];
        for (int it = 1; it <= P.max_iters; ++it) {
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
    write_result(P, sys, x, status, iters, sqrt(res2 / nb2), 0, tm);
}

// ---------------------------------------------------------------- GMRES

// Restarted GMRES(m), right-preconditioned: Arnoldi with modified
// Gram-Schmidt (one reduction per basis vector), Givens rotations applied by
// thread 0 to the Hessenberg column in shared memory, residual estimate
// |g_{j+1}|; each Arnoldi step is one iteration. The basis V (m+1 vectors)
// lives in shared memory or, when it does not fit, in the workspace; each
// thread only touches its own rows of it.
template <int FMT, int R>
__global__ void __launch_bounds__(max_threads_for(R), 1) gmres_kernel(const SolveParams P) {
    extern __shared__ __align__(16) unsigned char raw[];
    const Team tm = Team::make();
    const int sys = blockIdx.x;
    const int n = P.n;
    const int m = P.restart;
    const Smem64 sm = smem64_layout(raw, P.n_pad);
    const auto op = make_op<FMT, R>(P, sys, raw, P.stage_off, tm);
    int parity = 0;
    // extra: H[(m+1)*m] | cs[m] | sn[m] | g[m+1] | y[m] | ctl[4] | V (if in smem)
    double* H = sm.extra;
    double* cs = H + (m + 1) * m;
    double* sn = cs + m;
    double* g = sn + m;
    double* y = g + m + 1;
    int* ctl = reinterpret_cast<int*>(y + m);
    double* V = (P.ws != nullptr) ? P.ws + (size_t)sys * (m + 1) * P.n_pad : y + m + 2;
    const size_t vstride = P.n_pad;

    double b[R], x[R], r[R], w[R], dinv[R];
    load_system<FMT, R>(P, sys, b, x, tm);
    jacobi_setup<FMT, R>(op.A, P.precond == 1, dinv, tm);
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
        write_result(P, sys, x, ST_NAN, 0, __longlong_as_double(0x7ff8000000000000LL), 0, tm);
        return;
    }
    if (nb2 == 0.0) {
#pragma unroll
        for (int q = 0; q < R; ++q) x[q] = 0.0;
        write_result(P, sys, x, ST_CONVERGED, 0, 0.0, 0, tm);
        return;
    }
    const double tau2 = (P.tol_type == 1) ? P.tol * P.tol * nb2 : P.tol * P.tol;
    const double tau = sqrt(tau2);
    int status = -1, it = 0, restarts = 0;
    if (!finite(beta2))
        status = ST_NAN;
    else if (beta2 <= tau2)
        status = ST_CONVERGED;
    while (status < 0) {
        if (it >= P.max_iters) { status = ST_MAX_ITER; break; }
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
            __syncthreads();
            k = ctl[0];
            singular = ctl[1];
            estimate_ok = ctl[2];
            __syncthreads();  // ctl is rewritten by thread 0 in the next step
            if (singular || estimate_ok || it >= P.max_iters) break;
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
        __syncthreads();
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
        if (it >= P.max_iters) { status = ST_MAX_ITER; break; }
        if (estimate_ok && ++restarts > kMaxRestarts) { status = ST_MAX_ITER; break; }
    }
    double res2 = beta2;
    if (status == ST_NAN) res2 = true_residual(op, b, x, r, sm.xa, sm.red, parity, tm, n);
    write_result(P, sys, x, status, it, sqrt(res2 / nb2), 0, tm);
}

}  // namespace bbs
