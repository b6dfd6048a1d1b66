// BiCGSTAB + ILU(0) on BatchCsr with small systems packed several to a warp
// (the packing of bbs_packed.cuh applied to the ILU(0) path of bbs_ilu.cu).
//
// Each aligned group of L lanes owns one system and the warp runs its 32 / L
// systems in lockstep. The systems share the pattern, so they share the level
// schedule: every group factors and solves the same rows of the same level
// at the same time, and a level of up to L rows takes one pass of the group.
// Per group, shared memory holds
//   xa [n_pad] | xb [n_pad] | lu [k n] (ELL order)
// where lu starts as the system's values gathered into ELL order through the
// per-solve CSR column table (slot j of row i at j n + i) and is factored in
// place: for each stored k < i of row i, l_ik = a_ik / u_kk and
// a_ij -= l_ik u_kj for every j > k stored in rows i and k (IKJ form, rows
// level by level). A zero pivot counts as 1, as in the one-system kernel.
// As soon as row k is final its diagonal slot is overwritten with 1 / u_kk
// (later rows read u_k only right of the diagonal), so each lower entry costs
// one multiply. Once every row is final, U's off-diagonal entries are divided
// by their pivot, which takes the pivot multiply off the backward solve's
// dependent chain. M^-1 = U^-1 L^-1 is applied in place in xa / xb.
// The SpMV reads the original values from global memory through the same
// table (they stay in L1/L2). The method, its stopping rules and its log
// are those of bicgstab_ilu_kernel.
#pragma once

#include "bbs_ilu.cuh"
#include "bbs_packed.cuh"

namespace bbs {

// The pattern as the packed ILU kernels read it. The dependent steps of the
// factorisation and the triangular solves read it from a block-shared copy
// in shared memory: the ELL column table, each row's length and diagonal
// slot and the level schedule, all 8-bit (n <= 160), and each row's CSR start
// (16-bit: nnz < 2^15), from which the SpMV finds slot j of row i at CSR
// entry srp[i] + j and gathers the value from global memory.
struct IluPattern {
    const int32_t* xcols;  // global
    const int32_t* xsrc;   // global
    int n, k;
    int nlevL, nlevU;
    const uint16_t* srp;   // shared [n]: CSR start of each row (slot j of row i is entry srp[i] + j)
    const uint8_t* scols;  // shared [k n], 255 past the row end
    const uint8_t* slen;   // shared [n]
    const uint8_t* sdslot; // shared [n], 255 without a stored diagonal
    const uint8_t* slevL;  // shared [nlevL + 1]
    const uint8_t* srowsL; // shared [n]
    const uint8_t* slevU;  // shared [nlevU + 1]
    const uint8_t* srowsU; // shared [n]
    __device__ __forceinline__ int len(int i) const { return slen[i]; }
    __device__ __forceinline__ int col(int e, int i) const { return scols[e * n + i]; }  // e < len(i)
    __device__ __forceinline__ int dslot(int i) const { return sdslot[i] == 255 ? -1 : sdslot[i]; }
};

// The whole warp copies the pattern into `dst` (ilu_pattern_smem bytes).
__device__ __forceinline__ void ilu_pattern_stage(IluPattern& Pt, const IluSchedule& S, const int32_t* rp,
                                                  unsigned char* dst, int lane) {
    const int n = Pt.n, k = Pt.k;
    uint16_t* rps = reinterpret_cast<uint16_t*>(dst);
    uint8_t* cols = dst + 2 * (size_t)n;
    uint8_t* len = cols + (size_t)k * n;
    uint8_t* dsl = len + n;
    uint8_t* levL = dsl + n;
    uint8_t* rowsL = levL + n + 1;
    uint8_t* levU = rowsL + n;
    uint8_t* rowsU = levU + n + 1;
    for (int i = lane; i < k * n; i += 32) {
        const int c = ldg(Pt.xcols + i);
        cols[i] = (uint8_t)(c >= 0 ? c : 255);
    }
    for (int i = lane; i < n; i += 32) {
        const int r0 = ldg(rp + i);
        rps[i] = (uint16_t)r0;
        len[i] = (uint8_t)min(k, ldg(rp + i + 1) - r0);
        const int d = S.diag_pos[i];
        dsl[i] = (uint8_t)(d >= 0 ? d - r0 : 255);
        rowsL[i] = (uint8_t)S.rowsL[i];
        rowsU[i] = (uint8_t)S.rowsU[i];
    }
    for (int l = lane; l <= S.nlevL; l += 32) levL[l] = (uint8_t)S.levL_ptr[l];
    for (int l = lane; l <= S.nlevU; l += 32) levU[l] = (uint8_t)S.levU_ptr[l];
    __syncwarp();
    Pt.srp = rps;
    Pt.scols = cols;
    Pt.slen = len;
    Pt.sdslot = dsl;
    Pt.slevL = levL;
    Pt.srowsL = rowsL;
    Pt.slevU = levU;
    Pt.srowsU = rowsU;
    Pt.nlevL = S.nlevL;
    Pt.nlevU = S.nlevU;
}

// y = A x with A's values read from global memory in ELL order.
template <int R>
__device__ __forceinline__ void spmv_gather(const IluPattern& Pt, const double* __restrict__ vals,
                                            const double* __restrict__ xs, double (&y)[R], const Team& tm) {
#pragma unroll
    for (int q = 0; q < R; ++q) {
        const int row = tm.row(q);
        double sum = 0.0;
        if (row < Pt.n) {
            const double* vr = vals + Pt.srp[row];  // slot j of the row is CSR entry srp[row] + j
            for (int j = 0; j < Pt.k; ++j) {
                const int col = Pt.scols[j * Pt.n + row];
                if (col != 255) sum = fma(ldg(vr + j), xs[col], sum);
            }
        }
        y[q] = sum;
    }
}

// Overwrite row i's finished diagonal u_ii with 1 / u_ii (1 for a zero or
// missing pivot).
__device__ __forceinline__ void invert_pivot(const IluPattern& Pt, double* lu, int i) {
    const int d = Pt.dslot(i);
    if (d < 0) return;
    double& u = lu[(size_t)d * Pt.n + i];
    u = (u != 0.0) ? 1.0 / u : 1.0;
}

// 1 / u_ii of a finished row.
__device__ __forceinline__ double pivot_inv(const IluPattern& Pt, const double* lu, int i) {
    const int d = Pt.dslot(i);
    return d >= 0 ? lu[(size_t)d * Pt.n + i] : 1.0;
}

// In-place ILU(0) of the group's staged values, level by level.
__device__ __forceinline__ void ilu_factor_packed(const IluPattern& Pt, double* lu, const Team& tm) {
    const int n = Pt.n;
    for (int t = Pt.slevL[0] + tm.tid; t < Pt.slevL[1]; t += tm.nt) {  // rows without a lower part
        const int i = Pt.srowsL[t];
        invert_pivot(Pt, lu, i);
    }
    __syncwarp();
    for (int l = 1; l < Pt.nlevL; ++l) {
        for (int t = Pt.slevL[l] + tm.tid; t < Pt.slevL[l + 1]; t += tm.nt) {
            const int i = Pt.srowsL[t];
            const int len = Pt.len(i);
            for (int e = 0; e < len; ++e) {
                const int kk = Pt.col(e, i);
                if (kk >= i) break;
                const double lik = lu[(size_t)e * n + i] * pivot_inv(Pt, lu, kk);
                lu[(size_t)e * n + i] = lik;
                const int lenk = Pt.len(kk);
                int f = 0;
                for (int g = e + 1; g < len; ++g) {  // merge of the sorted rows i and k
                    const int j = Pt.col(g, i);
                    while (f < lenk && Pt.col(f, kk) < j) ++f;
                    if (f < lenk && Pt.col(f, kk) == j)
                        lu[(size_t)g * n + i] = fma(-lik, lu[(size_t)f * n + kk], lu[(size_t)g * n + i]);
                }
            }
            invert_pivot(Pt, lu, i);
        }
        __syncwarp();
    }
    // Every row is final: store U's off-diagonal entries divided by their
    // row's pivot, u_ij / u_ii, so that the backward solve needs no multiply
    // on its dependent chain (its right-hand side is scaled in one pass).
    for (int i = tm.tid; i < n; i += tm.nt) {
        const int d = Pt.dslot(i);
        if (d < 0) continue;
        const double pinv = lu[(size_t)d * n + i];
        const int len = Pt.len(i);
        for (int e = d + 1; e < len; ++e) lu[(size_t)e * n + i] *= pinv;
    }
    __syncwarp();
}

// buf = U^-1 L^-1 buf, in place, by the group. With the factor's U rows
// stored as u_ij / u_ii: y = L^-1 buf, then y_i / u_ii for every row in one
// pass, then x_i = y_i / u_ii - sum_j (u_ij / u_ii) x_j level by level.
// (Bounding the slot loops by the diagonal slot instead of testing columns
// measured 12 % slower.)
__device__ __forceinline__ void ilu_apply_packed(const IluPattern& Pt, const double* lu, double* buf,
                                                 const Team& tm) {
    const int n = Pt.n;
    for (int l = 1; l < Pt.nlevL; ++l) {
        for (int t = Pt.slevL[l] + tm.tid; t < Pt.slevL[l + 1]; t += tm.nt) {
            const int i = Pt.srowsL[t];
            double sum = buf[i];
            const int len = Pt.len(i);
            for (int e = 0; e < len; ++e) {
                const int kk = Pt.col(e, i);
                if (kk >= i) break;
                sum = fma(-lu[(size_t)e * n + i], buf[kk], sum);
            }
            buf[i] = sum;
        }
        __syncwarp();
    }
    for (int i = tm.tid; i < n; i += tm.nt) buf[i] *= pivot_inv(Pt, lu, i);
    __syncwarp();
    for (int l = 0; l < Pt.nlevU; ++l) {
        for (int t = Pt.slevU[l] + tm.tid; t < Pt.slevU[l + 1]; t += tm.nt) {
            const int i = Pt.srowsU[t];
            double sum = buf[i];
            for (int e = Pt.len(i) - 1; e >= 0; --e) {
                const int j = Pt.col(e, i);
                if (j <= i) break;
                sum = fma(-lu[(size_t)e * n + i], buf[j], sum);
            }
            buf[i] = sum;
        }
        __syncwarp();
    }
}

// r = b - A x through xsm for every group; groups with `take` keep r.
template <int L, int R>
__device__ __forceinline__ double ilu_packed_residual(const IluPattern& Pt, const double* vals,
                                                      const double* __restrict__ bg, const double (&x)[R],
                                                      double (&r)[R], bool take, double* xsm, const Team& tm) {
    put(xsm, x, tm, Pt.n);
    __syncwarp();
    double ax[R];
    spmv_gather<R>(Pt, vals, xsm, ax, tm);
#pragma unroll
    for (int q = 0; q < R; ++q) {
        const int row = tm.row(q);
        ax[q] = (row < Pt.n ? bg[row] : 0.0) - ax[q];
    }
    double s[1] = {pdot(ax, ax)};
    group_sum<L>(s, tm.lane);
    if (take) {
#pragma unroll
        for (int q = 0; q < R; ++q) r[q] = ax[q];
    }
    return s[0];
}

// Right-preconditioned BiCGSTAB, M = (L U)^-1, for one group's system.
template <int L, int R>
__device__ __forceinline__ void bicgstab_ilu_packed_system(const IluPattern& Pt, const double* vals,
                                                           const double* lu,
                                                           const SysIO& io, bool valid, const SolveCfg& C,
                                                           const TeamSmem& sm, const Team& tm) {
    const int n = io.n;
    double x[R], r[R], rh[R], p[R], v[R], t[R];
#pragma unroll
    for (int q = 0; q < R; ++q) {
        const int row = tm.row(q);
        x[q] = row < n ? io.x[row] : 0.0;
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
    const int special = !finite64(nb2) ? 1 : zero64(nb2) ? 2 : 0;
    bool active = valid && special == 0;
    int status = -1, iters = 0, restarts = 0;
    double rr = ilu_packed_residual<L, R>(Pt, vals, io.b, x, r, true, sm.xa, tm);
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
    double rho = rr, rho_old = 1.0, alpha = 1.0, omega = 1.0;
#pragma unroll
    for (int q = 0; q < R; ++q) {
        rh[q] = r[q];
        p[q] = 0.0;
        v[q] = 0.0;
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
        const double beta = (rho * alpha) / (rho_old * omega);
#pragma unroll
        for (int q = 0; q < R; ++q) p[q] = fma(beta, fma(-omega, v[q], p[q]), r[q]);
        put(sm.xa, p, tm, n);
        __syncwarp();
        ilu_apply_packed(Pt, lu, sm.xa, tm);  // xa = p^
        spmv_gather<R>(Pt, vals, sm.xa, v, tm);
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
        ilu_apply_packed(Pt, lu, sm.xb, tm);  // xb = s^
        spmv_gather<R>(Pt, vals, sm.xb, t, tm);
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
                if (row < n) x[q] = fma(alpha, sm.xa[row], x[q]);
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
            const double om = zero64(tt) ? 0.0 : ts / tt;
            if (full) omega = om;
#pragma unroll
            for (int q = 0; q < R; ++q) {
                const int row = tm.row(q);
                if (full && row < n) x[q] = fma(om, sm.xb[row], fma(alpha, sm.xa[row], x[q]));
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
            __syncwarp();  // x is updated from xa / xb before they are reused
            const double res = ilu_packed_residual<L, R>(Pt, vals, io.b, x, r, cand, sm.xa, tm);
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
                        rh[q] = r[q];
                        p[q] = 0.0;
                        v[q] = 0.0;
                    }
                    rho = res2;
                    rho_old = alpha = omega = 1.0;
                    restarted = true;
                }
            }
        }
        if (active && !restarted) {
            if (zero64(omega)) {
                status = ST_BREAKDOWN;
                active = false;
            } else {
                rho_old = rho;
                rho = rho_next;
            }
        }
    }
    if (active) status = ST_MAX_ITER;
    const bool need = valid && special == 0 && !have_res;
    if (__any_sync(kFull, need)) {
        __syncwarp();
        const double res = ilu_packed_residual<L, R>(Pt, vals, io.b, x, r, false, sm.xa, tm);
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

// One warp per block, 32 / L systems per warp; shared memory per group of
// P.slice bytes: xa [n_pad] | xb [n_pad] | lu at P.stage_off; after the
// 32 / L slices, the block's copy of the pattern.
template <int L, int R>
__global__ void __launch_bounds__(32, packed_cg_min_blocks(R))
    bicgstab_ilu_packed_kernel(const SolveParams P, const int* sched) {
    extern __shared__ __align__(16) unsigned char raw[];
    constexpr int S = 32 / L;
    const int lane = threadIdx.x & 31, g = lane / L;
    const int s = blockIdx.x * S + g;
    const bool valid = s < P.num_batch;
    const int sys = valid ? s : P.num_batch - 1;
    Team tm;
    tm.tid = lane & (L - 1);
    tm.nt = L;
    tm.lane = lane;
    tm.warp = 0;
    tm.nwarps = 1;
    tm.bar = 0;
    unsigned char* slice = raw + (size_t)g * P.slice;
    TeamSmem sm;
    sm.red = nullptr;
    sm.xa = reinterpret_cast<double*>(slice);
    sm.xb = sm.xa + P.n_pad;
    sm.extra = nullptr;
    double* lu = reinterpret_cast<double*>(slice + P.stage_off);
    const size_t cells = (size_t)P.xk * P.n;
    IluPattern Pt;
    Pt.xcols = P.xcols;
    Pt.xsrc = P.xsrc;
    Pt.n = P.n;
    Pt.k = P.xk;
    ilu_pattern_stage(Pt, ilu_schedule(sched, P.n), P.row_ptrs,
                      raw + (size_t)S * P.slice, lane);
    const double* vals = P.values + (size_t)sys * P.vps;
#pragma unroll 4
    for (size_t i = tm.tid; i < cells; i += L) {  // 8-byte asynchronous gathers into ELL order
        const int src = ldg(P.xsrc + i);
        if (src >= 0)
            cp_async8(lu + i, vals + src);
        else
            lu[i] = 0.0;
    }
    cp_async_wait_all();
    __syncwarp();
    const SysIO io = sys_io(P, sys);
    if (ldg(P.xflag) != 0) {  // a row longer than the table: every system reports NAN
        if (valid && tm.tid == 0) {
            *io.iters = 0;
            *io.rel_res = quiet_nan();
            *io.status = ST_NAN;
            if (io.inner != nullptr) *io.inner = 0;
        }
        return;
    }
    ilu_factor_packed(Pt, lu, tm);
    bicgstab_ilu_packed_system<L, R>(Pt, vals, lu, io, valid, solve_cfg(P, sys), sm, tm);
}

}  // namespace bbs
