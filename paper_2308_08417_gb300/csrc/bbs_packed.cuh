// BiCGSTAB for small systems packed several to a warp (Sec. 3.2's one
// system per work-group, with the work-group narrowed to L lanes).
//
// On GB300 an FP64 warp-instruction costs the same pipe time whether 32 or 1
// of its lanes are active, and the FP64 pipe bounds these solvers. A system of
// n rows on a whole warp wastes the lanes of its last row group (n = 144 on
// 32 lanes: 160 slots) and pays the scalar work of every iteration (the
// divisions for alpha, omega and beta, the reduction trees) once per system.
// Here each aligned group of L lanes (L = 4, 8 or 16) owns one system, so one
// warp advances 32 / L systems with each instruction:
//   * lane l of group g owns rows l, l + L, ..., l + (R-1) L of system g;
//   * the scalar work and the reductions (group_sum over L lanes) serve all
//     the warp's systems at once;
//   * n = 144 fits 16 lanes x 9 rows exactly.
//
// The groups run in lockstep: every lane executes every instruction, and a
// system that has stopped (converged, broken down, out of restarts) keeps
// computing discarded values until the warp's last system stops. Its x~ is
// frozen by predication, and the rare per-system branches (the half-step
// exit, the true-residual confirmation) run for the whole warp when any group
// takes them, with only that group keeping the results. The method, its
// stopping rules and its results are those of the one-system-per-team kernels
// (bicgstab_scaled_system): Jacobi folded into the staged values, As = A D^-1
// on x~ = D x, squared-norm tests on the integer pipe, true-residual
// confirmation with at most kMaxRestarts restarts.
#pragma once

#include "bbs_solvers.cuh"

namespace bbs {

// Format the staged values of a packed system are multiplied in: CSR values
// are staged in the ELL layout (slot j of row r at j n + r, zero padding)
// through a column table built once per solve, so the SpMV walks fixed-width
// slots with independent loads instead of row-pointer chains.
template <int FMT>
constexpr int staged_fmt() { return FMT == FMT_CSR ? FMT_ELL : FMT; }

// A packed system's operator: A is the system in global memory (its stored
// format; diagonal lookups), S the staged copy in shared memory (format
// staged_fmt<FMT>, S.vals = the staged values).
template <int FMT, int R>
struct PackedOp {
    Mat<double> A;
    Mat<double> S;
    __device__ __forceinline__ void apply(const double* xs, double (&y)[R], const Team& tm) const {
        spmv_staged<staged_fmt<FMT>(), R>(S, S.vals, xs, y, tm);
    }
    // S = S D^-1 (Jacobi folded into the staged values)
    __device__ __forceinline__ void scale(const double (&dinv)[R], double* tmp, const Team& tm) const {
        scale_columns<staged_fmt<FMT>(), R>(S, const_cast<double*>(S.vals), dinv, tmp, tm);
    }
};

// Residual b - A x (x staged through xsm) of every group; a group with
// `take` set keeps it in r. Returns the group's ||b - A x||^2.
template <int FMT, int L, int R>
__device__ __forceinline__ double packed_residual(const PackedOp<FMT, R>& op,
                                                  const double* __restrict__ bg, const double (&x)[R],
                                                  double (&r)[R], bool take, double* xsm,
                                                  const Team& tm, int n) {
    put(xsm, x, tm, n);
    __syncwarp();
    double ax[R];
    op.apply(xsm, ax, tm);
#pragma unroll
    for (int q = 0; q < R; ++q) {
        const int row = tm.row(q);
        ax[q] = (row < n ? bg[row] : 0.0) - ax[q];
    }
    double s[1] = {pdot(ax, ax)};
    group_sum<L>(s, tm.lane);
    if (take) {
#pragma unroll
        for (int q = 0; q < R; ++q) r[q] = ax[q];
    }
    return s[0];
}

// One group's system. `valid` is false for the groups past the end of the
// batch: they read a real system (io points at one) but never write.
template <int FMT, int L, int R>
__device__ __forceinline__ void bicgstab_packed_system(const PackedOp<FMT, R>& op,
                                                       const SysIO& io, bool valid, const SolveCfg& C,
                                                       const TeamSmem& sm, const Team& tm) {
    const int n = io.n;
    const bool jac = C.precond == 1;
    // p lives in shared memory (xa, the SpMV input it is copied to anyway),
    // which leaves five register vectors
    double xs[R], r[R], rh[R], v[R], t[R];
    if (jac) {
        double dinv[R];
        jacobi_setup<FMT, R>(op.A, true, dinv, tm);
        op.scale(dinv, sm.xb, tm);
    }
#pragma unroll
    for (int q = 0; q < R; ++q) {  // x~ = D x0 (1 for a zero diagonal, D = I without Jacobi)
        const int row = tm.row(q);
        const double d = (jac && row < n) ? diag_entry<FMT>(op.A, row) : 0.0;
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
        group_sum<L>(s0, tm.lane);
        nb2 = s0[0];
    }
    // special: 1 = non-finite ||b|| (x stays x0), 2 = b = 0 (x = 0)
    const int special = !finite64(nb2) ? 1 : zero64(nb2) ? 2 : 0;
    bool active = valid && special == 0;
    int status = -1, iters = 0, restarts = 0;
    double rr = packed_residual<FMT, L, R>(op, io.b, xs, r, true, sm.xa, tm, n);
    double res2 = rr;
    bool have_res = true;
    const double tau2 = (C.tol_type == 1) ? C.tol * C.tol * nb2 : C.tol * C.tol;
    if (active) {
        if (!finite64(rr)) {
            status = ST_NAN;
            active = false;
        } else if (le_nonneg64(rr, tau2)) {
            status = ST_CONVERGED;
            active = false;
        } else {
            have_res = false;
        }
    }
    // beta = (rho alpha) / (rho_old omega): cfac holds alpha / (rho omega) of
    // the previous step, found with omega = ts / tt from one division (1
    // before the first step and after a restart, where p = 0 and v = 0 make
    // beta irrelevant)
    double rho = rr, alpha = 1.0, omega = 1.0, cfac = 1.0;
    __syncwarp();  // every lane is done reading xa
#pragma unroll
    for (int q = 0; q < R; ++q) {
        const int row = tm.row(q);
        rh[q] = r[q];
        v[q] = 0.0;
        if (row < n) sm.xa[row] = 0.0;  // p = 0
    }
    for (int it = 1; it <= C.max_iters; ++it) {
        if (!__any_sync(kFull, active)) break;
        if (active) {
            iters = it;
            if (!finite64(rho)) {
                status = ST_NAN;
                active = false;
            } else if (zero64(rho)) {
                status = ST_BREAKDOWN;
                active = false;
            }
        }
        const double beta = rho * cfac;
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const int row = tm.row(q);
            if (row < n) sm.xa[row] = fma(beta, fma(-omega, v[q], sm.xa[row]), r[q]);
        }
        __syncwarp();
        op.apply(sm.xa, v, tm);
        double s1[1] = {pdot(rh, v)};
        group_sum<L>(s1, tm.lane);
        const double sigma = s1[0];
        if (active) {
            if (!finite64(sigma)) {
                status = ST_NAN;
                active = false;
            } else if (zero64(sigma)) {
                status = ST_BREAKDOWN;
                active = false;
            }
        }
        alpha = rho / sigma;
#pragma unroll
        for (int q = 0; q < R; ++q) r[q] = fma(-alpha, v[q], r[q]);  // r holds s
        put(sm.xb, r, tm, n);
        __syncwarp();
        op.apply(sm.xb, t, tm);
        double s3[3] = {pdot(r, r), pdot(t, t), pdot(t, r)};
        group_sum<L>(s3, tm.lane);
        const double ss = s3[0], tt = s3[1], ts = s3[2];
        if (active && !finite64(ss)) {
            status = ST_NAN;
            active = false;
        }
        const bool half = active && le_nonneg64(ss, tau2);
        bool full = active && !half;
        if (half) {
#pragma unroll
            for (int q = 0; q < R; ++q) {
                const int row = tm.row(q);
                xs[q] = fma(alpha, row < n ? sm.xa[row] : 0.0, xs[q]);
            }
        }
        bool cand = half;
        double rho_next = 0.0;
        if (__any_sync(kFull, full)) {
            if (full && (!finite64(tt) || !finite64(ts))) {
                status = ST_NAN;
                active = false;
                full = false;
            }
            // omega = ts / tt and the next beta's alpha / (rho omega) =
            // alpha tt / (rho ts) from one division; where the product or a
            // quotient leaves the normal range (systems scaled far from 1),
            // plain divisions in the original form
            const double den = tt * rho * ts;
            const double inv = 1.0 / den;
            const double qs = ts * inv, qt = tt * inv;  // 1 / (tt rho), 1 / (rho ts)
            double om = qs * (rho * ts);
            double cf = qt * (alpha * tt);
            const bool fast = normal64(den) && normal64(qs) && normal64(qt) && finite64(om) && finite64(cf);
            if (__any_sync(kFull, !fast) && !fast) {
                om = zero64(tt) ? 0.0 : ts / tt;
                cf = alpha / (rho * om);
            }
            if (full) {
                omega = om;
                cfac = cf;
            }
#pragma unroll
            for (int q = 0; q < R; ++q) {
                const int row = tm.row(q);
                const double nx = fma(om, r[q], fma(alpha, row < n ? sm.xa[row] : 0.0, xs[q]));
                if (full) xs[q] = nx;
                r[q] = fma(-om, t[q], r[q]);
            }
            double s2[2] = {pdot(r, r), pdot(rh, r)};
            group_sum<L>(s2, tm.lane);
            if (full) {
                if (!finite64(s2[0])) {
                    status = ST_NAN;
                    active = false;
                } else {
                    rr = s2[0];
                    rho_next = s2[1];
                    cand = le_nonneg64(rr, tau2);
                }
            }
        }
        bool restarted = false;
        if (__any_sync(kFull, cand)) {
            // through xb (s is spent), so that xa keeps every group's p
            const double res = packed_residual<FMT, L, R>(op, io.b, xs, r, cand, sm.xb, tm, n);
            if (cand) {
                res2 = res;
                have_res = true;
                if (!finite64(res2)) {
                    status = ST_NAN;
                    active = false;
                } else if (le_nonneg64(res2, tau2)) {
                    status = ST_CONVERGED;
                    active = false;
                } else if (++restarts > kMaxRestarts) {
                    status = ST_MAX_ITER;
                    active = false;
                } else {
                    have_res = false;
#pragma unroll
                    for (int q = 0; q < R; ++q) {
                        const int row = tm.row(q);
                        rh[q] = r[q];
                        v[q] = 0.0;
                        if (row < n) sm.xa[row] = 0.0;
                    }
                    rho = res2;
                    alpha = omega = cfac = 1.0;
                    restarted = true;
                }
            }
        }
        if (active && !restarted) {
            if (zero64(omega)) {
                status = ST_BREAKDOWN;
                active = false;
            } else {
                rho = rho_next;
            }
        }
    }
    if (active) status = ST_MAX_ITER;
    const bool need = valid && special == 0 && !have_res;
    if (__any_sync(kFull, need)) {
        const double res = packed_residual<FMT, L, R>(op, io.b, xs, r, false, sm.xb, tm, n);
        if (need) res2 = res;
    }
    if (!valid) return;
    if (special == 1) {
        if (tm.tid == 0) {
            *io.iters = 0;
            *io.rel_res = quiet_nan();
            *io.status = ST_NAN;
            if (io.inner != nullptr) *io.inner = 0;
        }
        return;
    }
    if (special == 2) {
#pragma unroll
        for (int q = 0; q < R; ++q) xs[q] = 0.0;
        write_result(io, xs, ST_CONVERGED, 0, 0.0, 0, tm);
        return;
    }
    if (iters > 0) {  // x = D^-1 x~ (1 for a zero diagonal)
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const int row = tm.row(q);
            if (row >= n) continue;
            const double d = jac ? diag_entry<FMT>(op.A, row) : 0.0;
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

// ------------------------------------------------------------------- CG

// Alg. 1 (BatchCg) with Jacobi, packed like BiCGSTAB above (the exit test on
// ||r|| and the true-residual confirmation of cg_system). z = D^-1 r is formed
// on the fly from the register-resident inverse diagonal.
template <int FMT, int L, int R>
__device__ __forceinline__ void cg_packed_system(const PackedOp<FMT, R>& op, const SysIO& io,
                                                 bool valid, const SolveCfg& C, const TeamSmem& sm,
                                                 const Team& tm) {
    const int n = io.n;
    double x[R], r[R], p[R], t[R], dinv[R];
    jacobi_setup<FMT, R>(op.A, C.precond == 1, dinv, tm);
#pragma unroll
    for (int q = 0; q < R; ++q) {
        const int row = tm.row(q);
        x[q] = row < n ? io.x[row] : 0.0;
    }
    put(sm.xa, x, tm, n);
    __syncwarp();
    op.apply(sm.xa, t, tm);
    double bb = 0.0;
#pragma unroll
    for (int q = 0; q < R; ++q) {
        const int row = tm.row(q);
        const double bq = row < n ? io.b[row] : 0.0;
        r[q] = bq - t[q];
        bb = fma(bq, bq, bb);
    }
    double s0[3] = {bb, pdot(r, r), 0.0};
#pragma unroll
    for (int q = 0; q < R; ++q) s0[2] = fma(r[q], dinv[q] * r[q], s0[2]);
    group_sum<L>(s0, tm.lane);
    const double nb2 = s0[0];
    double rr = s0[1], rho = s0[2];
    const int special = !finite(nb2) ? 1 : (nb2 == 0.0) ? 2 : 0;
    bool active = valid && special == 0;
    int status = -1, iters = 0, restarts = 0;
    double res2 = rr;
    bool have_res = true;
    const double tau2 = (C.tol_type == 1) ? C.tol * C.tol * nb2 : C.tol * C.tol;
    if (active) {
        if (!finite(rr)) {
            status = ST_NAN;
            active = false;
        } else if (rr <= tau2) {
            status = ST_CONVERGED;
            active = false;
        } else {
            have_res = false;
        }
    }
#pragma unroll
    for (int q = 0; q < R; ++q) p[q] = dinv[q] * r[q];
    for (int it = 1; it <= C.max_iters; ++it) {
        if (!__any_sync(kFull, active)) break;
        if (active) {
            iters = it;
            if (!finite64(rho)) {
                status = ST_NAN;
                active = false;
            } else if (zero64(rho)) {
                status = ST_BREAKDOWN;
                active = false;
            }
        }
        put(sm.xa, p, tm, n);
        __syncwarp();
        op.apply(sm.xa, t, tm);
        double s1[1] = {pdot(p, t)};
        group_sum<L>(s1, tm.lane);
        const double pt = s1[0];
        if (active) {
            if (!finite64(pt)) {
                status = ST_NAN;
                active = false;
            } else if (zero64(pt)) {
                status = ST_BREAKDOWN;
                active = false;
            }
        }
        // alpha = rho / pt and 1 / rho (for the ratio below) from one division;
        // plain divisions where the product is not a normal number
        const double den = pt * rho;
        const double inv = 1.0 / den;
        const double qp = rho * inv;  // 1 / pt
        double alpha = qp * rho;
        double rinv = pt * inv;
        const bool fast = normal64(den) && normal64(qp) && normal64(rinv) && finite64(alpha);
        if (__any_sync(kFull, !fast) && !fast) {
            alpha = rho / pt;
            rinv = 1.0 / rho;
        }
        double s2[2] = {0.0, 0.0};
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const double nx = fma(alpha, p[q], x[q]);
            if (active) x[q] = nx;
            r[q] = fma(-alpha, t[q], r[q]);
            t[q] = dinv[q] * r[q];  // z = M r, held in t until p is updated
            s2[0] = fma(r[q], r[q], s2[0]);
            s2[1] = fma(r[q], t[q], s2[1]);
        }
        group_sum<L>(s2, tm.lane);
        bool cand = false;
        if (active) {
            rr = s2[0];
            if (!finite64(rr)) {
                status = ST_NAN;
                active = false;
            } else {
                cand = le_nonneg64(rr, tau2);
            }
        }
        // p = z + (rho_new / rho) p now, before a confirmation may reuse t;
        // a restart below replaces p with M r_true.
        const double ratio = s2[1] * rinv;
#pragma unroll
        for (int q = 0; q < R; ++q) p[q] = fma(ratio, p[q], t[q]);
        bool restarted = false;
        if (__any_sync(kFull, cand)) {
            put(sm.xa, x, tm, n);
            __syncwarp();
            op.apply(sm.xa, t, tm);
            double s3[2] = {0.0, 0.0};
#pragma unroll
            for (int q = 0; q < R; ++q) {
                const int row = tm.row(q);
                t[q] = (row < n ? io.b[row] : 0.0) - t[q];
                s3[0] = fma(t[q], t[q], s3[0]);
                s3[1] = fma(t[q], dinv[q] * t[q], s3[1]);
            }
            group_sum<L>(s3, tm.lane);
            if (cand) {
#pragma unroll
                for (int q = 0; q < R; ++q) r[q] = t[q];
                res2 = s3[0];
                have_res = true;
                if (!finite(res2)) {
                    status = ST_NAN;
                    active = false;
                } else if (res2 <= tau2) {
                    status = ST_CONVERGED;
                    active = false;
                } else if (++restarts > kMaxRestarts) {
                    status = ST_MAX_ITER;
                    active = false;
                } else {
                    have_res = false;
#pragma unroll
                    for (int q = 0; q < R; ++q) p[q] = dinv[q] * r[q];
                    rho = s3[1];
                    restarted = true;
                }
            }
        }
        // (unconditional: a stopped system's rho is never read again, and the
        // old rho is then dead once 1 / rho is known)
        if (!restarted) rho = s2[1];
    }
    if (active) status = ST_MAX_ITER;
    const bool need = valid && special == 0 && !have_res;
    if (__any_sync(kFull, need)) {
        double dummy[R];
        const double res = packed_residual<FMT, L, R>(op, io.b, x, dummy, false, sm.xa, tm, n);
        if (need) res2 = res;
    }
    if (!valid) return;
    if (special == 1) {
        write_result(io, x, ST_NAN, 0, quiet_nan(), 0, tm);
        return;
    }
    if (special == 2) {
#pragma unroll
        for (int q = 0; q < R; ++q) x[q] = 0.0;
        write_result(io, x, ST_CONVERGED, 0, 0.0, 0, tm);
        return;
    }
    write_result(io, x, status, iters, sqrt(res2 / nb2), 0, tm);
}

// ----------------------------------------------------------------- GMRES

// Right-preconditioned GMRES(m) with Jacobi folded into the staged values
// (As = A D^-1 on x~ = D x), packed like BiCGSTAB above; the method and its
// rules are those of gmres_system: Arnoldi with modified Gram-Schmidt,
// Givens rotations, the residual estimate |g_{j+1}| as the inner exit test,
// the true residual after every cycle, restarts capped like the other
// solvers' confirmations.
// Each lane keeps its rows of the system's Krylov basis V [(m+1) x n_pad] in
// the workspace (global memory, L2-resident: only the lane that writes a
// row reads it), so shared memory holds only the staged values, the SpMV
// input and the group's small arrays ext = H [(m+1) m] | cs [m] | sn [m] |
// g [m+1] | y [m] | ctl [2 doubles]. The scalar Givens and back-substitution
// work runs on the group's first lane, in lockstep with the other groups'.
template <int FMT, int L, int R>
__device__ __forceinline__ void gmres_packed_system(const PackedOp<FMT, R>& op, const SysIO& io, bool valid,
                                                    const SolveCfg& C, double* xa, double* ext, const Team& tm) {
    const int n = io.n;
    const int m = C.restart;
    const bool jac = C.precond == 1;
    const size_t vs = (size_t)((n + 1) & ~1);
    double* V = C.ws;
    // H holds the (m + 1) x m Hessenberg column by column, only rows 0..j + 1
    // of column j: entry (i, j) at j (j + 3) / 2 + i, m (m + 3) / 2 in all
    double* H = ext;
    const auto hx = [](int i, int j) { return j * (j + 3) / 2 + i; };
    double* cs = H + m * (m + 3) / 2;
    double* sn = cs + m;
    double* g = sn + m;
    double* y = g + m + 1;
    int* ctl = reinterpret_cast<int*>(y + m);
    const bool lead = tm.tid == 0;
    if (jac) {
        double dinv[R];
        jacobi_setup<FMT, R>(op.A, true, dinv, tm);
        op.scale(dinv, xa, tm);
    }
    double xs[R], w[R];
#pragma unroll
    for (int q = 0; q < R; ++q) {  // x~ = D x0
        const int row = tm.row(q);
        const double d = (jac && row < n) ? diag_entry<FMT>(op.A, row) : 0.0;
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
        group_sum<L>(s0, tm.lane);
        nb2 = s0[0];
    }
    const int special = !finite(nb2) ? 1 : (nb2 == 0.0) ? 2 : 0;
    bool active = valid && special == 0;
    double beta2 = packed_residual<FMT, L, R>(op, io.b, xs, w, true, xa, tm, n);  // w = r
    const double tau2 = (C.tol_type == 1) ? C.tol * C.tol * nb2 : C.tol * C.tol;
    const double tau = sqrt(tau2);
    int status = -1, it = 0, restarts = 0;
    if (active) {
        if (!finite(beta2)) {
            status = ST_NAN;
            active = false;
        } else if (beta2 <= tau2) {
            status = ST_CONVERGED;
            active = false;
        }
    }
    bool nan_exit = false;  // NAN inside a cycle: the log recomputes the residual
    while (__any_sync(kFull, active)) {
        if (active && it >= C.max_iters) {
            status = ST_MAX_ITER;
            active = false;
        }
        bool cyc = active;
        const double binv = 1.0 / sqrt(beta2);
        if (cyc) {
#pragma unroll
            for (int q = 0; q < R; ++q) {
                const int row = tm.row(q);
                if (row < n) V[row] = w[q] * binv;
            }
            if (lead) {
                for (int i = 0; i <= m; ++i) g[i] = 0.0;
                g[0] = sqrt(beta2);
            }
        }
        int k = 0;
        bool singular = false, estimate_ok = false;
        for (int j = 0; j < m; ++j) {
            if (!__any_sync(kFull, cyc)) break;
            if (cyc) ++it;
            {
                double u[R];
#pragma unroll
                for (int q = 0; q < R; ++q) {
                    const int row = tm.row(q);
                    u[q] = row < n ? V[(size_t)j * vs + row] : 0.0;
                }
                __syncwarp();  // every lane is done reading xa
                put(xa, u, tm, n);
            }
            __syncwarp();
            op.apply(xa, w, tm);
            bool bad = false;
            for (int i = 0; i <= j; ++i) {  // modified Gram-Schmidt
                double vr[R];
#pragma unroll
                for (int q = 0; q < R; ++q) {
                    const int row = tm.row(q);
                    vr[q] = row < n ? V[(size_t)i * vs + row] : 0.0;
                }
                double h[1] = {pdot(w, vr)};
                group_sum<L>(h, tm.lane);
                bad |= !finite64(h[0]);
#pragma unroll
                for (int q = 0; q < R; ++q) w[q] = fma(-h[0], vr[q], w[q]);
                if (cyc && lead) H[hx(i, j)] = h[0];
            }
            double hw[1] = {pdot(w, w)};
            group_sum<L>(hw, tm.lane);
            // h_{j+1,j} = ||w|| and its reciprocal from one rsqrt (every lane
            // runs this: cheaper than a square root and a division)
            const double hinv = rsqrt(hw[0]);
            const double hn = __double_as_longlong(hw[0]) > 0 ? hw[0] * hinv : hw[0];
            bad |= !finite64(hn);
            if (cyc && bad) {
                status = ST_NAN;
                active = false;
                cyc = false;
                nan_exit = true;
            }
            if (cyc && lead) {
                H[hx(j + 1, j)] = hn;
                for (int i = 0; i < j; ++i) {
                    const double a = H[hx(i, j)], c = H[hx(i + 1, j)];
                    H[hx(i, j)] = cs[i] * a + sn[i] * c;
                    H[hx(i + 1, j)] = -sn[i] * a + cs[i] * c;
                }
                const double a = H[hx(j, j)];
                const double denom = sqrt(a * a + hn * hn);
                int c0, c1 = 0, c2 = 0;
                if (denom == 0.0) {
                    c0 = j;
                    c1 = 1;
                } else {
                    const double dinv = 1.0 / denom;
                    cs[j] = a * dinv;
                    sn[j] = hn * dinv;
                    H[hx(j, j)] = denom;
                    H[hx(j + 1, j)] = 0.0;
                    g[j + 1] = -sn[j] * g[j];
                    g[j] = cs[j] * g[j];
                    c0 = j + 1;
                    c2 = (hn == 0.0 || fabs(g[j + 1]) <= tau) ? 1 : 0;
                }
                ctl[0] = c0;
                ctl[1] = c1 | (c2 << 1);
            }
            __syncwarp();
            if (cyc) {  // the group's first lane wrote its ctl
                k = ctl[0];
                singular = ctl[1] & 1;
                estimate_ok = (ctl[1] >> 1) & 1;
            }
            __syncwarp();  // ctl is rewritten in the next step
            if (cyc && (singular || estimate_ok || it >= C.max_iters)) cyc = false;
            if (cyc) {
#pragma unroll
                for (int q = 0; q < R; ++q) {
                    const int row = tm.row(q);
                    if (row < n) V[(size_t)(j + 1) * vs + row] = w[q] * hinv;
                }
            }
        }
        // y = H(0:k,0:k)^-1 g(0:k) ; x~ += V y, for the groups still solving
        const bool upd = active;
        if (upd && lead) {
            for (int i = k - 1; i >= 0; --i) {
                double sum = g[i];
                for (int l = i + 1; l < k; ++l) sum -= H[hx(i, l)] * y[l];
                y[i] = sum / H[hx(i, i)];
            }
        }
        __syncwarp();
        if (upd) {
#pragma unroll
            for (int q = 0; q < R; ++q) {
                const int row = tm.row(q);
                if (row < n) {
                    double sum = 0.0;
                    for (int i = 0; i < k; ++i) sum = fma(y[i], V[(size_t)i * vs + row], sum);
                    xs[q] += sum;
                }
            }
        }
        if (__any_sync(kFull, upd)) {
            __syncwarp();
            const double res = packed_residual<FMT, L, R>(op, io.b, xs, w, upd, xa, tm, n);
            if (upd) {
                beta2 = res;
                if (!finite(beta2)) {
                    status = ST_NAN;
                    active = false;
                } else if (beta2 <= tau2) {
                    status = ST_CONVERGED;
                    active = false;
                } else if (singular) {
                    status = ST_BREAKDOWN;
                    active = false;
                } else if (it >= C.max_iters) {
                    status = ST_MAX_ITER;
                    active = false;
                } else if (estimate_ok && ++restarts > kMaxRestarts) {
                    status = ST_MAX_ITER;
                    active = false;
                }
            }
        }
    }
    double res2 = beta2;
    if (__any_sync(kFull, valid && nan_exit)) {
        __syncwarp();
        double r[R];
        const double res = packed_residual<FMT, L, R>(op, io.b, xs, r, false, xa, tm, n);
        if (nan_exit) res2 = res;
    }
    // The basis is dead scratch from here on: drop the 128-byte lines wholly
    // inside this system's slot from L2 without writing them back (dirty lines
    // of finished systems would otherwise crowd live data out of L2 and be
    // written to DRAM when evicted).
    __syncwarp();
    if (valid && V != nullptr) {
        const uintptr_t first = (reinterpret_cast<uintptr_t>(V) + 127) & ~static_cast<uintptr_t>(127);
        const uintptr_t end = (reinterpret_cast<uintptr_t>(V) + (size_t)(m + 1) * vs * 8) & ~static_cast<uintptr_t>(127);
        for (uintptr_t a = first + (uintptr_t)tm.tid * 128; a < end; a += (uintptr_t)L * 128)
            asm volatile("discard.global.L2 [%0], 128;" ::"l"(a) : "memory");
    }
    if (!valid) return;
    if (special == 1) {
        if (tm.tid == 0) {
            *io.iters = 0;
            *io.rel_res = quiet_nan();
            *io.status = ST_NAN;
            if (io.inner != nullptr) *io.inner = 0;
        }
        return;
    }
    if (special == 2) {
#pragma unroll
        for (int q = 0; q < R; ++q) xs[q] = 0.0;
        write_result(io, xs, ST_CONVERGED, 0, 0.0, 0, tm);
        return;
    }
    if (it > 0) {  // x = D^-1 x~
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const int row = tm.row(q);
            if (row >= n) continue;
            const double d = jac ? diag_entry<FMT>(op.A, row) : 0.0;
            io.x[row] = (d != 0.0) ? xs[q] / d : xs[q];
        }
    }
    if (tm.tid == 0) {
        *io.iters = it;
        *io.rel_res = sqrt(res2 / nb2);
        *io.status = status;
        if (io.inner != nullptr) *io.inner = 0;
    }
}

// ------------------------------------------------------------- kernels

// Resident blocks an SM must hold, which sets the register cap (registers
// are split over the SM's four schedulers, so 16 one-warp blocks allow 128
// registers and 12 allow 168). Both solvers keep five R-row vectors in
// registers and fit 128 up to R = 5, 168 beyond without spilling.
__host__ __device__ constexpr int packed_min_blocks(int R) { return R <= 5 ? 16 : 12; }
__host__ __device__ constexpr int packed_cg_min_blocks(int R) { return R <= 5 ? 16 : 12; }

// The calling lane's group: team of L lanes, its shared-memory slice
// (xa [n_pad] | xb [n_pad] | staged values, P.slice bytes per group) and its
// system (groups past the end of the batch read the last system and never
// write). CSR values are gathered into the ELL layout through P.xsrc.
template <int FMT, int L, int R>
struct PackedGroup {
    Team tm;
    TeamSmem sm;
    bool valid;
    int sys;
    PackedOp<FMT, R> op;
    // blk: the batch's block of 32 / L systems this warp solves (blockIdx.x
    // unless the kernel strides over the batch)
    __device__ __forceinline__ PackedGroup(const SolveParams& P, unsigned char* raw, int blk) {
        constexpr int S = 32 / L;
        const int lane = threadIdx.x & 31, g = lane / L;
        const int s = blk * S + g;
        valid = s < P.num_batch;
        sys = valid ? s : P.num_batch - 1;
        tm.tid = lane & (L - 1);
        tm.nt = L;
        tm.lane = lane;
        tm.warp = 0;
        tm.nwarps = 1;
        tm.bar = 0;
        unsigned char* slice = raw + (size_t)g * P.slice;
        sm.red = nullptr;
        sm.xa = reinterpret_cast<double*>(slice);
        sm.xb = sm.xa + P.n_pad;
        sm.extra = nullptr;
        const double* vals = P.values + (size_t)sys * P.vps;
        double* as = reinterpret_cast<double*>(slice + P.stage_off);
        op.A = Mat<double>{vals, P.row_ptrs, P.cols, P.n, P.k};
        if constexpr (FMT == FMT_CSR) {  // gathered into ELL order by 8-byte asynchronous copies
            const int count = P.xk * P.n;
#pragma unroll 4
            for (int i = tm.tid; i < count; i += L) {
                const int src = ldg(P.xsrc + i);
                if (src >= 0)
                    cp_async8(as + i, vals + src);
                else
                    as[i] = 0.0;
            }
            cp_async_wait_all();
            op.S = Mat<double>{as, nullptr, P.xcols, P.n, P.xk};
        } else {
            stage_values(vals, as, P.vps, tm);
            op.S = Mat<double>{as, P.row_ptrs, P.cols, P.n, P.k};
        }
        __syncwarp();
    }
};

// Every system of a CSR call whose pattern has a row longer than the width
// of its column table reports NAN (the table could not hold that row).
template <int FMT, int L, int R>
__device__ __forceinline__ bool packed_reject(const SolveParams& P, const PackedGroup<FMT, L, R>& G) {
    if constexpr (FMT == FMT_CSR) {
        if (ldg(P.xflag) != 0) {
            if (G.valid && G.tm.tid == 0) {
                P.iters[G.sys] = 0;
                P.rel_res[G.sys] = quiet_nan();
                P.status[G.sys] = ST_NAN;
                if (P.inner_iters != nullptr) P.inner_iters[G.sys] = 0;
            }
            return true;
        }
    }
    return false;
}

// One warp per block, 32 / L systems per warp.
template <int FMT, int L, int R>
__global__ void __launch_bounds__(32, packed_min_blocks(R)) bicgstab_packed_kernel(const SolveParams P) {
    extern __shared__ __align__(16) unsigned char raw[];
    const PackedGroup<FMT, L, R> G(P, raw, blockIdx.x);
    if (packed_reject(P, G)) return;
    bicgstab_packed_system<FMT, L, R>(G.op, sys_io(P, G.sys), G.valid, solve_cfg(P, G.sys), G.sm, G.tm);
}

// GMRES: the group's small arrays follow its staged values in the slice.
template <int FMT, int L, int R>
__global__ void __launch_bounds__(32, packed_cg_min_blocks(R)) gmres_packed_kernel(const SolveParams P) {
    extern __shared__ __align__(16) unsigned char raw[];
    const PackedGroup<FMT, L, R> G(P, raw, blockIdx.x);
    if (packed_reject(P, G)) return;
    const size_t count = FMT == FMT_CSR ? (size_t)P.xk * P.n : P.vps;
    unsigned char* slice = raw + (size_t)((threadIdx.x & 31) / L) * P.slice;
    double* ext = reinterpret_cast<double*>(slice + P.stage_off + ((count * 8 + 15) & ~(size_t)15));
    gmres_packed_system<FMT, L, R>(G.op, sys_io(P, G.sys), G.valid, solve_cfg(P, G.sys), G.sm.xa, ext, G.tm);
}

template <int FMT, int L, int R>
__global__ void __launch_bounds__(32, packed_cg_min_blocks(R)) cg_packed_kernel(const SolveParams P) {
    extern __shared__ __align__(16) unsigned char raw[];
    const PackedGroup<FMT, L, R> G(P, raw, blockIdx.x);
    if (packed_reject(P, G)) return;
    cg_packed_system<FMT, L, R>(G.op, sys_io(P, G.sys), G.valid, solve_cfg(P, G.sys), G.sm, G.tm);
}

}  // namespace bbs
