/*
 * Plain FP64 CPU oracle of the batched Krylov solvers.
 *
 * TEST INFRASTRUCTURE ONLY. The test suite, the smoke check and the
 * benchmark's CPU-baseline leg are the only callers. It shares no code,
 * header, table or helper with the CUDA library, and the library never calls
 * it: there is no CPU fallback anywhere in the product.
 *
 * Every routine is a direct serial statement of the method: each system is
 * solved on its own, sums run left to right from +0.0, nothing is blocked,
 * fused or reordered, and the build forbids floating-point contraction
 * (-ffp-contract=off) so that the same source gives the same bits on x86-64
 * and AArch64.
 *
 * What it follows:
 *   Sec. 3.1     batch formats sharing one pattern (BatchCsr, BatchEll
 *                column-major with pad column -1, BatchDense row-major).
 *   Sec. 3, Table "Batched feature support": solvers BatchCg, BatchBicgstab,
 *                BatchGmres, scalar BatchJacobi, Absolute/Relative stopping.
 *   Alg. 1       BatchCg, with the exit test on the residual 2-norm.
 *   Sec. 3.2     BiCGSTAB and GMRES composed of SpMV, dot, norm and vector
 *                updates (textbook statements: van der Vorst's BiCGSTAB and
 *                Saad's restarted GMRES with modified Gram-Schmidt and Givens
 *                rotations, both right-preconditioned).
 *   Sec. 2.1     the initial guess x0 is used (x is in/out) and each system
 *                is monitored on its own (per-system iteration/residual log).
 *   Sec. 2.1     "precision format" as a parameter: the mixed mode runs the
 *                inner BiCGSTAB in FP32 inside an FP64 refinement loop.
 *   Sec. 3, Table "Batched feature support": BatchIlu / BatchTrsv, read as
 *                the incomplete LU factorisation with zero fill-in on the
 *                shared CSR pattern (ILU(0), Saad's IKJ form) applied by a
 *                forward (unit lower) and a backward (upper) triangular
 *                solve; right preconditioner of BiCGSTAB and GMRES.
 *
 * Readings where the paper is silent (all shared with the CUDA path by
 * specification, not by code):
 *   - stop when ||r||_2 <= tau, tau = tol*||b||_2 (relative) or tol
 *     (absolute); a passing recursive residual is confirmed with the true
 *     residual b - A x; a failed confirmation restarts the method from the
 *     true residual (at most OM_MAX_RESTARTS times, then MAX_ITER);
 *   - b = 0 gives x = 0 after 0 iterations;
 *   - Jacobi uses 1 for a zero or missing diagonal;
 *   - exact-zero breakdown tests only (rho, sigma, omega, p.t, Givens);
 *   - a non-finite scalar stops the system with status NAN;
 *   - rel_res logged = ||b - A x||_2 / ||b||_2 of the returned x.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { OM_CSR = 0, OM_ELL = 1, OM_DENSE = 2 };
enum { OM_BICGSTAB = 0, OM_CG = 1, OM_GMRES = 2 };
enum { OM_NOPRECOND = 0, OM_JACOBI = 1, OM_ILU0 = 2 };
enum { OM_ABSOLUTE = 0, OM_RELATIVE = 1 };
enum { OM_CONVERGED = 0, OM_MAX_ITER = 1, OM_BREAKDOWN = 2, OM_NAN = 3 };
#define OM_MAX_RESTARTS 3

typedef struct {
    int fmt, n, ell_k;
    const int32_t *row_ptrs; /* CSR */
    const int32_t *col_idxs; /* CSR: nnz; ELL: ell_k*n column-major */
    const double *vals;      /* this system's values */
} om_mat;

typedef struct {
    int fmt, n, ell_k;
    const int32_t *row_ptrs, *col_idxs;
    const float *vals;
} om_mat32;

typedef struct {
    int solver, precond, tol_type, max_iters, restart;
    double tol;
} om_opts;

typedef struct {
    int32_t iters, status;
    double rel_res;
} om_result;

/* ---------------------------------------------------------------- basics */

/* y = A x, one row at a time, entries in stored (ascending column) order. */
static void spmv(const om_mat *A, const double *x, double *y)
{
    const int n = A->n;
    for (int i = 0; i < n; ++i) {
        double sum = 0.0;
        if (A->fmt == OM_CSR) {
            for (int e = A->row_ptrs[i]; e < A->row_ptrs[i + 1]; ++e)
                sum = sum + A->vals[e] * x[A->col_idxs[e]];
        } else if (A->fmt == OM_ELL) {
            for (int j = 0; j < A->ell_k; ++j) {
                const int c = A->col_idxs[(size_t)j * n + i];
                if (c < 0)
                    continue;
                sum = sum + A->vals[(size_t)j * n + i] * x[c];
            }
        } else {
            for (int j = 0; j < n; ++j)
                sum = sum + A->vals[(size_t)i * n + j] * x[j];
        }
        y[i] = sum;
    }
}

static void spmv32(const om_mat32 *A, const float *x, float *y)
{
    const int n = A->n;
    for (int i = 0; i < n; ++i) {
        float sum = 0.0f;
        if (A->fmt == OM_CSR) {
            for (int e = A->row_ptrs[i]; e < A->row_ptrs[i + 1]; ++e)
                sum = sum + A->vals[e] * x[A->col_idxs[e]];
        } else if (A->fmt == OM_ELL) {
            for (int j = 0; j < A->ell_k; ++j) {
                const int c = A->col_idxs[(size_t)j * n + i];
                if (c < 0)
                    continue;
                sum = sum + A->vals[(size_t)j * n + i] * x[c];
            }
        } else {
            for (int j = 0; j < n; ++j)
                sum = sum + A->vals[(size_t)i * n + j] * x[j];
        }
        y[i] = sum;
    }
}

/* a_ii, or 0 when row i stores no diagonal entry */
static double diag_entry(const om_mat *A, int i)
{
    const int n = A->n;
    if (A->fmt == OM_CSR) {
        for (int e = A->row_ptrs[i]; e < A->row_ptrs[i + 1]; ++e)
            if (A->col_idxs[e] == i)
                return A->vals[e];
    } else if (A->fmt == OM_ELL) {
        for (int j = 0; j < A->ell_k; ++j)
            if (A->col_idxs[(size_t)j * n + i] == i)
                return A->vals[(size_t)j * n + i];
    } else {
        return A->vals[(size_t)i * n + i];
    }
    return 0.0;
}

static float diag_entry32(const om_mat32 *A, int i)
{
    const int n = A->n;
    if (A->fmt == OM_CSR) {
        for (int e = A->row_ptrs[i]; e < A->row_ptrs[i + 1]; ++e)
            if (A->col_idxs[e] == i)
                return A->vals[e];
    } else if (A->fmt == OM_ELL) {
        for (int j = 0; j < A->ell_k; ++j)
            if (A->col_idxs[(size_t)j * n + i] == i)
                return A->vals[(size_t)j * n + i];
    } else {
        return A->vals[(size_t)i * n + i];
    }
    return 0.0f;
}

/* Scalar Jacobi: M = D^-1, with 1 where the diagonal is zero or absent.
 * With no preconditioner M = I. */
static void precond_setup(const om_mat *A, int precond, double *dinv)
{
    for (int i = 0; i < A->n; ++i) {
        const double d = diag_entry(A, i);
        dinv[i] = (precond == OM_JACOBI && d != 0.0) ? 1.0 / d : 1.0;
    }
}

/* ILU(0) on the CSR pattern, in place in `lu` (a copy of A's values): for
 * each row i, for each k < i stored in row i (ascending), a_ik /= a_kk and
 * a_ij -= a_ik a_kj for every j > k stored in both rows i and k. The unit
 * lower factor L and the upper factor U share the pattern. A zero pivot is
 * replaced by 1 (the same rule as Jacobi's zero diagonal). */
static void ilu0_factor(const om_mat *A, double *lu)
{
    const int n = A->n;
    const int32_t *rp = A->row_ptrs, *ci = A->col_idxs;
    for (int i = 0; i < n; ++i) {
        for (int e = rp[i]; e < rp[i + 1]; ++e) {
            const int k = ci[e];
            if (k >= i)
                break;
            double pivot = 0.0; /* u_kk */
            for (int f = rp[k]; f < rp[k + 1]; ++f)
                if (ci[f] == k)
                    pivot = lu[f];
            if (pivot == 0.0)
                pivot = 1.0;
            lu[e] = lu[e] / pivot;
            for (int g = e + 1; g < rp[i + 1]; ++g) { /* j = ci[g] > k */
                const int j = ci[g];
                for (int f = rp[k]; f < rp[k + 1]; ++f)
                    if (ci[f] == j)
                        lu[g] = lu[g] - lu[e] * lu[f];
            }
        }
    }
}

/* z = U^-1 L^-1 v with the factors of ilu0_factor (L unit lower). */
static void ilu0_apply(const om_mat *A, const double *lu, const double *v, double *z)
{
    const int n = A->n;
    const int32_t *rp = A->row_ptrs, *ci = A->col_idxs;
    for (int i = 0; i < n; ++i) { /* L y = v */
        double sum = v[i];
        for (int e = rp[i]; e < rp[i + 1]; ++e)
            if (ci[e] < i)
                sum = sum - lu[e] * z[ci[e]];
        z[i] = sum;
    }
    for (int i = n - 1; i >= 0; --i) { /* U z = y */
        double sum = z[i], d = 0.0;
        for (int e = rp[i]; e < rp[i + 1]; ++e) {
            if (ci[e] > i)
                sum = sum - lu[e] * z[ci[e]];
            else if (ci[e] == i)
                d = lu[e];
        }
        z[i] = sum / (d != 0.0 ? d : 1.0);
    }
}

/* The right preconditioner M^-1 of one system: Jacobi (dinv), none, or ILU(0). */
typedef struct {
    int kind;
    const om_mat *A;
    double *dinv; /* n: Jacobi / none */
    double *lu;   /* nnz: ILU(0) factors */
} om_prec;

static int prec_init(om_prec *M, const om_mat *A, int kind)
{
    M->kind = kind;
    M->A = A;
    M->dinv = (double *)malloc(sizeof(double) * A->n);
    M->lu = NULL;
    if (kind == OM_ILU0) {
        if (A->fmt != OM_CSR)
            return 0;
        const int nnz = A->row_ptrs[A->n];
        M->lu = (double *)malloc(sizeof(double) * (nnz > 0 ? nnz : 1));
        memcpy(M->lu, A->vals, sizeof(double) * nnz);
        ilu0_factor(A, M->lu);
    }
    precond_setup(A, kind == OM_JACOBI ? OM_JACOBI : OM_NOPRECOND, M->dinv);
    return 1;
}

static void prec_free(om_prec *M)
{
    free(M->dinv);
    free(M->lu);
}

/* z = M^-1 v */
static void prec_apply(const om_prec *M, const double *v, double *z)
{
    if (M->kind == OM_ILU0) {
        ilu0_apply(M->A, M->lu, v, z);
    } else {
        for (int i = 0; i < M->A->n; ++i)
            z[i] = M->dinv[i] * v[i];
    }
}

static double dot(const double *a, const double *b, int n)
{
    double sum = 0.0;
    for (int i = 0; i < n; ++i)
        sum = sum + a[i] * b[i];
    return sum;
}

static float dot32(const float *a, const float *b, int n)
{
    float sum = 0.0f;
    for (int i = 0; i < n; ++i)
        sum = sum + a[i] * b[i];
    return sum;
}

static double norm2(const double *a, int n) { return sqrt(dot(a, a, n)); }

/* r = b - A x */
static void residual(const om_mat *A, const double *b, const double *x, double *r, double *tmp)
{
    spmv(A, x, tmp);
    for (int i = 0; i < A->n; ++i)
        r[i] = b[i] - tmp[i];
}

/* Logged relative residual of the returned x: ||b - A x|| / ||b||. */
static double true_rel_res(const om_mat *A, const double *b, const double *x, double nb,
                           double *r, double *tmp)
{
    residual(A, b, x, r, tmp);
    return norm2(r, A->n) / nb;
}

static void finish(om_result *res, int status, int iters, const om_mat *A, const double *b,
                   const double *x, double nb, double *r, double *tmp)
{
    res->status = status;
    res->iters = iters;
    res->rel_res = true_rel_res(A, b, x, nb, r, tmp);
}

/* Common entry checks. Returns 1 when the system is already decided. */
static int start(const om_mat *A, const double *b, double *x, const om_opts *o, om_result *res,
                 double *nb_out, double *tau_out)
{
    const int n = A->n;
    const double nb = norm2(b, n);
    *nb_out = nb;
    if (!isfinite(nb)) {
        res->status = OM_NAN;
        res->iters = 0;
        res->rel_res = NAN;
        return 1;
    }
    if (nb == 0.0) { /* b = 0: the solution is x = 0 */
        for (int i = 0; i < n; ++i)
            x[i] = 0.0;
        res->status = OM_CONVERGED;
        res->iters = 0;
        res->rel_res = 0.0;
        return 1;
    }
    *tau_out = (o->tol_type == OM_RELATIVE) ? o->tol * nb : o->tol;
    return 0;
}

/* ------------------------------------------------------------- BiCGSTAB */

/*
 * Right-preconditioned BiCGSTAB (van der Vorst), M = D^-1:
 *   r = b - A x, r^ = r, rho_old = alpha = omega = 1, v = p = 0
 *   loop: rho = r^.r ; beta = (rho/rho_old)(alpha/omega)
 *         p = r + beta (p - omega v) ; p^ = M p ; v = A p^
 *         alpha = rho / (r^.v) ; s = r - alpha v        [exit test on s]
 *         s^ = M s ; t = A s^ ; omega = (t.s)/(t.t)
 *         x = x + alpha p^ + omega s^ ; r = s - omega t [exit test on r]
 */
static void bicgstab(const om_mat *A, const double *b, double *x, const om_opts *o, om_result *res)
{
    const int n = A->n;
    double nb, tau;
    if (start(A, b, x, o, res, &nb, &tau))
        return;
    double *buf = (double *)calloc((size_t)11 * n, sizeof(double));
    double *r = buf + n, *rh = buf + 2 * n, *p = buf + 3 * n, *ph = buf + 4 * n;
    double *v = buf + 5 * n, *s = buf + 6 * n, *sh = buf + 7 * n, *t = buf + 8 * n;
    double *rt = buf + 9 * n, *tmp = buf + 10 * n;
    om_prec M;
    prec_init(&M, A, o->precond);

    residual(A, b, x, r, tmp);
    double rn = norm2(r, n);
    if (!isfinite(rn)) {
        finish(res, OM_NAN, 0, A, b, x, nb, rt, tmp);
        goto done;
    }
    if (rn <= tau) {
        res->status = OM_CONVERGED;
        res->iters = 0;
        res->rel_res = rn / nb;
        goto done;
    }
    memcpy(rh, r, sizeof(double) * n);
    double rho_old = 1.0, alpha = 1.0, omega = 1.0;
    int restarts = 0;
    for (int it = 1; it <= o->max_iters; ++it) {
        const double rho = dot(rh, r, n);
        if (!isfinite(rho)) {
            finish(res, OM_NAN, it, A, b, x, nb, rt, tmp);
            goto done;
        }
        if (rho == 0.0) {
            finish(res, OM_BREAKDOWN, it, A, b, x, nb, rt, tmp);
            goto done;
        }
        const double beta = (rho / rho_old) * (alpha / omega);
        for (int i = 0; i < n; ++i)
            p[i] = r[i] + beta * (p[i] - omega * v[i]);
        prec_apply(&M, p, ph);
        spmv(A, ph, v);
        const double sigma = dot(rh, v, n);
        if (!isfinite(sigma)) {
            finish(res, OM_NAN, it, A, b, x, nb, rt, tmp);
            goto done;
        }
        if (sigma == 0.0) {
            finish(res, OM_BREAKDOWN, it, A, b, x, nb, rt, tmp);
            goto done;
        }
        alpha = rho / sigma;
        for (int i = 0; i < n; ++i)
            s[i] = r[i] - alpha * v[i];
        const double sn = norm2(s, n);
        if (!isfinite(sn)) {
            finish(res, OM_NAN, it, A, b, x, nb, rt, tmp);
            goto done;
        }
        int candidate = 0;
        if (sn <= tau) { /* half-step exit: x = x + alpha p^ */
            for (int i = 0; i < n; ++i)
                x[i] = x[i] + alpha * ph[i];
            candidate = 1;
        } else {
            prec_apply(&M, s, sh);
            spmv(A, sh, t);
            const double tt = dot(t, t, n);
            const double ts = dot(t, s, n);
            if (!isfinite(tt) || !isfinite(ts)) {
                finish(res, OM_NAN, it, A, b, x, nb, rt, tmp);
                goto done;
            }
            omega = (tt == 0.0) ? 0.0 : ts / tt;
            for (int i = 0; i < n; ++i)
                x[i] = x[i] + alpha * ph[i] + omega * sh[i];
            for (int i = 0; i < n; ++i)
                r[i] = s[i] - omega * t[i];
            rn = norm2(r, n);
            if (!isfinite(rn)) {
                finish(res, OM_NAN, it, A, b, x, nb, rt, tmp);
                goto done;
            }
            candidate = (rn <= tau);
        }
        if (candidate) { /* confirm with the true residual */
            residual(A, b, x, rt, tmp);
            const double tn = norm2(rt, n);
            if (!isfinite(tn)) {
                finish(res, OM_NAN, it, A, b, x, nb, rt, tmp);
                goto done;
            }
            if (tn <= tau) {
                res->status = OM_CONVERGED;
                res->iters = it;
                res->rel_res = tn / nb;
                goto done;
            }
            if (++restarts > OM_MAX_RESTARTS) {
                res->status = OM_MAX_ITER;
                res->iters = it;
                res->rel_res = tn / nb;
                goto done;
            }
            /* restart from the true residual */
            memcpy(r, rt, sizeof(double) * n);
            memcpy(rh, rt, sizeof(double) * n);
            memset(p, 0, sizeof(double) * n);
            memset(v, 0, sizeof(double) * n);
            rho_old = alpha = omega = 1.0;
            continue;
        }
        if (omega == 0.0) {
            finish(res, OM_BREAKDOWN, it, A, b, x, nb, rt, tmp);
            goto done;
        }
        rho_old = rho;
    }
    finish(res, OM_MAX_ITER, o->max_iters, A, b, x, nb, rt, tmp);
done:
    prec_free(&M);
    free(buf);
}

/* ------------------------------------------------------------------- CG */

/*
 * Alg. 1 (BatchCg): r = b - A x, z = M r, p = z, rho = r.z
 *   loop: t = A p ; alpha = rho / (p.t) ; x = x + alpha p ; r = r - alpha t
 *         [exit test on r] ; z = M r ; rho^ = r.z ; p = z + (rho^/rho) p ;
 *         rho = rho^
 * The exit test is ||r|| <= tau (in place of Alg. 1's |rho| < tau); testing
 * after the r update is the same point as Alg. 1's test at the loop head.
 */
static void cg(const om_mat *A, const double *b, double *x, const om_opts *o, om_result *res)
{
    const int n = A->n;
    double nb, tau;
    if (start(A, b, x, o, res, &nb, &tau))
        return;
    double *buf = (double *)calloc((size_t)7 * n, sizeof(double));
    double *dinv = buf, *r = buf + n, *z = buf + 2 * n, *p = buf + 3 * n, *t = buf + 4 * n;
    double *rt = buf + 5 * n, *tmp = buf + 6 * n;
    precond_setup(A, o->precond, dinv);

    residual(A, b, x, r, tmp);
    double rn = norm2(r, n);
    if (!isfinite(rn)) {
        finish(res, OM_NAN, 0, A, b, x, nb, rt, tmp);
        goto done;
    }
    if (rn <= tau) {
        res->status = OM_CONVERGED;
        res->iters = 0;
        res->rel_res = rn / nb;
        goto done;
    }
    for (int i = 0; i < n; ++i)
        z[i] = dinv[i] * r[i];
    memcpy(p, z, sizeof(double) * n);
    double rho = dot(r, z, n);
    int restarts = 0;
    for (int it = 1; it <= o->max_iters; ++it) {
        if (!isfinite(rho)) {
            finish(res, OM_NAN, it, A, b, x, nb, rt, tmp);
            goto done;
        }
        if (rho == 0.0) {
            finish(res, OM_BREAKDOWN, it, A, b, x, nb, rt, tmp);
            goto done;
        }
        spmv(A, p, t);
        const double pt = dot(p, t, n);
        if (!isfinite(pt)) {
            finish(res, OM_NAN, it, A, b, x, nb, rt, tmp);
            goto done;
        }
        if (pt == 0.0) {
            finish(res, OM_BREAKDOWN, it, A, b, x, nb, rt, tmp);
            goto done;
        }
        const double alpha = rho / pt;
        for (int i = 0; i < n; ++i)
            x[i] = x[i] + alpha * p[i];
        for (int i = 0; i < n; ++i)
            r[i] = r[i] - alpha * t[i];
        rn = norm2(r, n);
        if (!isfinite(rn)) {
            finish(res, OM_NAN, it, A, b, x, nb, rt, tmp);
            goto done;
        }
        if (rn <= tau) {
            residual(A, b, x, rt, tmp);
            const double tn = norm2(rt, n);
            if (!isfinite(tn)) {
                finish(res, OM_NAN, it, A, b, x, nb, rt, tmp);
                goto done;
            }
            if (tn <= tau) {
                res->status = OM_CONVERGED;
                res->iters = it;
                res->rel_res = tn / nb;
                goto done;
            }
            if (++restarts > OM_MAX_RESTARTS) {
                res->status = OM_MAX_ITER;
                res->iters = it;
                res->rel_res = tn / nb;
                goto done;
            }
            memcpy(r, rt, sizeof(double) * n);
            for (int i = 0; i < n; ++i)
                z[i] = dinv[i] * r[i];
            memcpy(p, z, sizeof(double) * n);
            rho = dot(r, z, n);
            continue;
        }
        for (int i = 0; i < n; ++i)
            z[i] = dinv[i] * r[i];
        const double rho_hat = dot(r, z, n);
        const double ratio = rho_hat / rho;
        for (int i = 0; i < n; ++i)
            p[i] = z[i] + ratio * p[i];
        rho = rho_hat;
    }
    finish(res, OM_MAX_ITER, o->max_iters, A, b, x, nb, rt, tmp);
done:
    free(buf);
}

/* ---------------------------------------------------------------- GMRES */

/*
 * Restarted GMRES(m), right-preconditioned (A M u = r, x = x + M u):
 * Arnoldi with modified Gram-Schmidt, Givens rotations on the Hessenberg
 * matrix, residual estimate |g_{j+1}|. Each Arnoldi step is one iteration.
 * At the end of a cycle the (k x k) triangular system is solved, x updated
 * and the true residual taken; it decides convergence.
 */
static void gmres(const om_mat *A, const double *b, double *x, const om_opts *o, om_result *res)
{
    const int n = A->n;
    const int m = o->restart;
    double nb, tau;
    if (start(A, b, x, o, res, &nb, &tau))
        return;
    double *buf = (double *)calloc((size_t)(m + 1) * n + 6 * (size_t)n, sizeof(double));
    double *V = buf;                         /* (m+1) x n, row j = basis vector j */
    double *r = buf + (size_t)(m + 1) * n + n, *w = r + n, *u = w + n;
    double *tmp = u + n, *zz = tmp + n;
    double *H = (double *)calloc((size_t)(m + 1) * m, sizeof(double)); /* H[i*m + j] */
    double *cs = (double *)calloc((size_t)m, sizeof(double));
    double *sn = (double *)calloc((size_t)m, sizeof(double));
    double *g = (double *)calloc((size_t)m + 1, sizeof(double));
    double *y = (double *)calloc((size_t)m, sizeof(double));
    om_prec M;
    prec_init(&M, A, o->precond);

    residual(A, b, x, r, tmp);
    double beta = norm2(r, n);
    if (!isfinite(beta)) {
        finish(res, OM_NAN, 0, A, b, x, nb, w, tmp);
        goto done;
    }
    if (beta <= tau) {
        res->status = OM_CONVERGED;
        res->iters = 0;
        res->rel_res = beta / nb;
        goto done;
    }
    int it = 0, restarts = 0;
    for (;;) {
        if (it >= o->max_iters) { /* only reached with max_iters == 0 */
            res->status = OM_MAX_ITER;
            res->iters = it;
            res->rel_res = beta / nb;
            goto done;
        }
        for (int i = 0; i < n; ++i)
            V[i] = r[i] / beta;
        memset(g, 0, sizeof(double) * (m + 1));
        g[0] = beta;
        int k = 0, singular = 0, estimate_ok = 0;
        for (int j = 0; j < m; ++j) {
            ++it;
            double *vj = V + (size_t)j * n;
            prec_apply(&M, vj, u);
            spmv(A, u, w);
            for (int i = 0; i <= j; ++i) { /* modified Gram-Schmidt */
                const double *vi = V + (size_t)i * n;
                const double h = dot(w, vi, n);
                H[i * m + j] = h;
                for (int l = 0; l < n; ++l)
                    w[l] = w[l] - h * vi[l];
            }
            const double hn = norm2(w, n);
            H[(j + 1) * m + j] = hn;
            int bad = !isfinite(hn);
            for (int i = 0; i <= j; ++i)
                bad |= !isfinite(H[i * m + j]);
            if (bad) {
                finish(res, OM_NAN, it, A, b, x, nb, w, tmp);
                goto done;
            }
            for (int i = 0; i < j; ++i) { /* earlier rotations on column j */
                const double a = H[i * m + j], c = H[(i + 1) * m + j];
                H[i * m + j] = cs[i] * a + sn[i] * c;
                H[(i + 1) * m + j] = -sn[i] * a + cs[i] * c;
            }
            const double a = H[j * m + j];
            const double denom = sqrt(a * a + hn * hn);
            if (denom == 0.0) { /* singular Hessenberg: keep columns 0..j-1 */
                k = j;
                singular = 1;
                break;
            }
            cs[j] = a / denom;
            sn[j] = hn / denom;
            H[j * m + j] = denom;
            H[(j + 1) * m + j] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            k = j + 1;
            if (hn == 0.0 || fabs(g[j + 1]) <= tau) {
                estimate_ok = 1;
                break;
            }
            if (it >= o->max_iters)
                break;
            double *vn = V + (size_t)(j + 1) * n;
            for (int i = 0; i < n; ++i)
                vn[i] = w[i] / hn;
        }
        /* y = H(0:k,0:k)^-1 g(0:k) by back substitution ; x = x + M (V y) */
        for (int i = k - 1; i >= 0; --i) {
            double sum = g[i];
            for (int l = i + 1; l < k; ++l)
                sum = sum - H[i * m + l] * y[l];
            y[i] = sum / H[i * m + i];
        }
        for (int l = 0; l < n; ++l) {
            double sum = 0.0;
            for (int i = 0; i < k; ++i)
                sum = sum + y[i] * V[(size_t)i * n + l];
            zz[l] = sum;
        }
        prec_apply(&M, zz, u);
        for (int l = 0; l < n; ++l)
            x[l] = x[l] + u[l];
        residual(A, b, x, r, tmp);
        beta = norm2(r, n);
        if (!isfinite(beta)) {
            finish(res, OM_NAN, it, A, b, x, nb, w, tmp);
            goto done;
        }
        if (beta <= tau) {
            res->status = OM_CONVERGED;
            res->iters = it;
            res->rel_res = beta / nb;
            goto done;
        }
        if (singular) {
            res->status = OM_BREAKDOWN;
            res->iters = it;
            res->rel_res = beta / nb;
            goto done;
        }
        if (it >= o->max_iters) {
            res->status = OM_MAX_ITER;
            res->iters = it;
            res->rel_res = beta / nb;
            goto done;
        }
        if (estimate_ok && ++restarts > OM_MAX_RESTARTS) {
            res->status = OM_MAX_ITER;
            res->iters = it;
            res->rel_res = beta / nb;
            goto done;
        }
    }
done:
    prec_free(&M);
    free(buf);
    free(H);
    free(cs);
    free(sn);
    free(g);
    free(y);
}

static void solve_one(const om_mat *A, const double *b, double *x, const om_opts *o, om_result *res)
{
    if (o->solver == OM_CG)
        cg(A, b, x, o, res);
    else if (o->solver == OM_GMRES)
        gmres(A, b, x, o, res);
    else
        bicgstab(A, b, x, o, res);
}

/* --------------------------------------------- mixed-precision refinement */

/*
 * FP32 BiCGSTAB + Jacobi on A32 d = w from d = 0, run until the recursive
 * residual passes inner_tol*||w|| (no confirmation: the FP64 outer loop judges),
 * a breakdown, a non-finite scalar, or max_inner iterations. Returns the
 * iteration at which it stopped.
 */
static int inner_bicgstab32(const om_mat32 *A, const float *dinv, const float *w, float *d,
                            float inner_tol, int max_inner, float *buf)
{
    const int n = A->n;
    float *r = buf, *rh = buf + n, *p = buf + 2 * n, *ph = buf + 3 * n, *v = buf + 4 * n;
    float *s = buf + 5 * n, *sh = buf + 6 * n, *t = buf + 7 * n;
    for (int i = 0; i < n; ++i) {
        d[i] = 0.0f;
        r[i] = w[i]; /* r = w - A*0 */
        rh[i] = w[i];
        p[i] = 0.0f;
        v[i] = 0.0f;
    }
    const float tau = inner_tol * sqrtf(dot32(w, w, n));
    float rho_old = 1.0f, alpha = 1.0f, omega = 1.0f;
    for (int it = 1; it <= max_inner; ++it) {
        const float rho = dot32(rh, r, n);
        if (!isfinite(rho) || rho == 0.0f)
            return it;
        const float beta = (rho / rho_old) * (alpha / omega);
        for (int i = 0; i < n; ++i)
            p[i] = r[i] + beta * (p[i] - omega * v[i]);
        for (int i = 0; i < n; ++i)
            ph[i] = dinv[i] * p[i];
        spmv32(A, ph, v);
        const float sigma = dot32(rh, v, n);
        if (!isfinite(sigma) || sigma == 0.0f)
            return it;
        alpha = rho / sigma;
        for (int i = 0; i < n; ++i)
            s[i] = r[i] - alpha * v[i];
        if (sqrtf(dot32(s, s, n)) <= tau) {
            for (int i = 0; i < n; ++i)
                d[i] = d[i] + alpha * ph[i];
            return it;
        }
        for (int i = 0; i < n; ++i)
            sh[i] = dinv[i] * s[i];
        spmv32(A, sh, t);
        const float tt = dot32(t, t, n);
        const float ts = dot32(t, s, n);
        omega = (tt == 0.0f) ? 0.0f : ts / tt;
        for (int i = 0; i < n; ++i)
            d[i] = d[i] + alpha * ph[i] + omega * sh[i];
        for (int i = 0; i < n; ++i)
            r[i] = s[i] - omega * t[i];
        const float rn = sqrtf(dot32(r, r, n));
        if (!isfinite(rn) || rn <= tau || omega == 0.0f)
            return it;
        rho_old = rho;
    }
    return max_inner;
}

/*
 * Iterative refinement: the residual r = b - A x, its norm, the exit test and
 * the update x = x + ||r|| d stay in FP64; the correction d solves
 * A32 d = r/||r|| in FP32. iters = outer steps, inner = total inner iterations.
 */
static void refine(const om_mat *A, const om_mat32 *A32, const double *b, double *x,
                   const om_opts *o, double inner_tol, int max_outer, om_result *res,
                   int32_t *inner_total)
{
    const int n = A->n;
    double nb, tau;
    *inner_total = 0;
    if (start(A, b, x, o, res, &nb, &tau))
        return;
    double *r = (double *)malloc(sizeof(double) * 2 * n), *tmp = r + n;
    float *f = (float *)malloc(sizeof(float) * 11 * n);
    float *dinv32 = f, *w = f + n, *d = f + 2 * n, *work = f + 3 * n;
    for (int i = 0; i < n; ++i) {
        const float a = (o->precond == OM_JACOBI) ? diag_entry32(A32, i) : 0.0f;
        dinv32[i] = (a != 0.0f) ? 1.0f / a : 1.0f;
    }
    for (int k = 0;; ++k) {
        residual(A, b, x, r, tmp);
        const double rn = norm2(r, n);
        if (!isfinite(rn)) {
            res->status = OM_NAN;
            res->iters = k;
            res->rel_res = rn / nb;
            break;
        }
        if (rn <= tau || k == max_outer) {
            res->status = (rn <= tau) ? OM_CONVERGED : OM_MAX_ITER;
            res->iters = k;
            res->rel_res = rn / nb;
            break;
        }
        for (int i = 0; i < n; ++i)
            w[i] = (float)(r[i] / rn);
        *inner_total += inner_bicgstab32(A32, dinv32, w, d, (float)inner_tol, o->max_iters, work);
        for (int i = 0; i < n; ++i)
            x[i] = x[i] + rn * (double)d[i];
    }
    free(r);
    free(f);
}

/* ------------------------------------------------------------ batch API */

static size_t vals_per_system(int fmt, int n, int nnz, int ell_k)
{
    if (fmt == OM_CSR)
        return (size_t)nnz;
    if (fmt == OM_ELL)
        return (size_t)ell_k * n;
    return (size_t)n * n;
}

int om_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* y_i = A_i x_i for every system. */
void om_spmv_batch(int fmt, int n, int nnz, int ell_k, const int32_t *row_ptrs,
                   const int32_t *col_idxs, const double *values, int num_batch,
                   const double *x, double *y)
{
    const size_t vps = vals_per_system(fmt, n, nnz, ell_k);
    for (int bi = 0; bi < num_batch; ++bi) {
        om_mat A = {fmt, n, ell_k, row_ptrs, col_idxs, values + vps * bi};
        spmv(&A, x + (size_t)n * bi, y + (size_t)n * bi);
    }
}

/* ILU(0) factors of every system of a BatchCsr batch (test access). */
void om_ilu0_batch(int n, const int32_t *row_ptrs, const int32_t *col_idxs, const double *values,
                   int num_batch, double *lu)
{
    const int nnz = row_ptrs[n];
    for (int bi = 0; bi < num_batch; ++bi) {
        om_mat A = {OM_CSR, n, 0, row_ptrs, col_idxs, values + (size_t)nnz * bi};
        memcpy(lu + (size_t)nnz * bi, A.vals, sizeof(double) * nnz);
        ilu0_factor(&A, lu + (size_t)nnz * bi);
    }
}

/* Solve every system of a shared-pattern batch; x is in/out. */
void om_solve_batch(int solver, int precond, int fmt, int n, int nnz, int ell_k,
                    const int32_t *row_ptrs, const int32_t *col_idxs, const double *values,
                    int num_batch, const double *b, double *x, int tol_type, double tol,
                    int max_iters, int restart, int32_t *iters, double *rel_res,
                    int32_t *status, int nthreads)
{
    const size_t vps = vals_per_system(fmt, n, nnz, ell_k);
    const om_opts o = {solver, precond, tol_type, max_iters, restart, tol};
#pragma omp parallel for schedule(dynamic, 64) num_threads(nthreads > 0 ? nthreads : 1)
    for (int bi = 0; bi < num_batch; ++bi) {
        om_mat A = {fmt, n, ell_k, row_ptrs, col_idxs, values + vps * bi};
        om_result res;
        solve_one(&A, b + (size_t)n * bi, x + (size_t)n * bi, &o, &res);
        iters[bi] = res.iters;
        rel_res[bi] = res.rel_res;
        status[bi] = res.status;
    }
}

/* Mixed precision: FP32 inner BiCGSTAB inside FP64 refinement. values32 is
 * the FP32 copy of values (same layout). max_iters caps each inner solve. */
void om_refine_batch(int precond, int fmt, int n, int nnz, int ell_k, const int32_t *row_ptrs,
                     const int32_t *col_idxs, const double *values, const float *values32,
                     int num_batch, const double *b, double *x, int tol_type, double tol,
                     int max_iters, double inner_tol, int max_outer, int32_t *iters,
                     double *rel_res, int32_t *status, int32_t *inner_iters, int nthreads)
{
    const size_t vps = vals_per_system(fmt, n, nnz, ell_k);
    const om_opts o = {OM_BICGSTAB, precond, tol_type, max_iters, 0, tol};
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads > 0 ? nthreads : 1)
    for (int bi = 0; bi < num_batch; ++bi) {
        om_mat A = {fmt, n, ell_k, row_ptrs, col_idxs, values + vps * bi};
        om_mat32 A32 = {fmt, n, ell_k, row_ptrs, col_idxs, values32 + vps * bi};
        om_result res;
        int32_t inner = 0;
        refine(&A, &A32, b + (size_t)n * bi, x + (size_t)n * bi, &o, inner_tol, max_outer, &res,
               &inner);
        iters[bi] = res.iters;
        rel_res[bi] = res.rel_res;
        status[bi] = res.status;
        if (inner_iters)
            inner_iters[bi] = inner;
    }
}

/* Uneven batch in BatchCsr: system i uses pattern sys_pattern[i] from the
 * pools, values at values + val_off[i], vectors at b/x + vec_off[i]. */
void om_solve_varsize(int solver, int precond, int num_batch, const int32_t *pat_n,
                      const int64_t *pat_rp_off, const int64_t *pat_ci_off,
                      const int32_t *row_ptrs, const int32_t *col_idxs,
                      const int32_t *sys_pattern, const int64_t *val_off, const int64_t *vec_off,
                      const double *values, const double *b, double *x, int tol_type, double tol,
                      int max_iters, int restart, int32_t *iters, double *rel_res,
                      int32_t *status, int nthreads)
{
    const om_opts o = {solver, precond, tol_type, max_iters, restart, tol};
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads > 0 ? nthreads : 1)
    for (int bi = 0; bi < num_batch; ++bi) {
        const int pi = sys_pattern[bi];
        om_mat A = {OM_CSR, pat_n[pi], 0, row_ptrs + pat_rp_off[pi], col_idxs + pat_ci_off[pi],
                    values + val_off[bi]};
        om_result res;
        solve_one(&A, b + vec_off[bi], x + vec_off[bi], &o, &res);
        iters[bi] = res.iters;
        rel_res[bi] = res.rel_res;
        status[bi] = res.status;
    }
}
