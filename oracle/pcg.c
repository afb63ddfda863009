/*
 * pcg.c -- oracle: per-sample Jacobi-preconditioned conjugate gradients.
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * The ensemble solve of Section 2.3 with per-sample ("ensemble-valued") inner
 * products and norms is, as that section states, equivalent to solving each
 * sample's system of Eq. (discrete-sys) independently; so the oracle solves
 * one sample at a time.  Conventions (the paper is silent on them):
 *   - x0 = 0, r = b, z = D^{-1} r, p = z (Hestenes-Stiefel form);
 *   - convergence when ||r||_2 <= rtol ||b||_2 on the recursively updated
 *     residual, checked after each update; the iteration count is the number
 *     of products q = A p that led to an update;
 *   - the A-conjugate norm guard of Section 4: when p^T A p is not positive
 *     (or not finite) the sample stops with status OR_BREAKDOWN and its x is
 *     left as it was;
 *   - every inner product is a plain left-to-right sum.
 */
#include "oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

void or_spmv(int J, const int64_t *rowptr, const int32_t *colidx,
             const double *vals, const double *x, double *y)
{
    for (int i = 0; i < J; i++) {
        double s = 0.0;
        for (int64_t k = rowptr[i]; k < rowptr[i + 1]; k++) s = s + vals[k] * x[colidx[k]];
        y[i] = s;
    }
}

int or_jacobi(int J, const int64_t *rowptr, const int32_t *colidx,
              const double *vals, double *dinv)
{
    for (int i = 0; i < J; i++) {
        double d = 0.0;
        int found = 0;
        for (int64_t k = rowptr[i]; k < rowptr[i + 1]; k++)
            if (colidx[k] == i) { d = vals[k]; found = 1; }
        if (!found) return -1;
        dinv[i] = 1.0 / d;
    }
    return 0;
}

static double dot(int J, const double *a, const double *b)
{
    double s = 0.0;
    for (int i = 0; i < J; i++) s = s + a[i] * b[i];
    return s;
}

/* The iteration, optionally recording the relative residual ||r_k|| / ||b||
 * after every update k = 1, 2, ... in hist[k - 1] (Section 4's convergence
 * record, kept for every iteration instead of only the last). */
static int pcg_run(int J, const int64_t *rowptr, const int32_t *colidx,
                   const double *vals, const double *b, double rtol, int maxit,
                   double *x, int *iters, double *relres, double *hist)
{
    double *dinv = malloc(sizeof(double) * J), *r = malloc(sizeof(double) * J);
    double *z = malloc(sizeof(double) * J), *p = malloc(sizeof(double) * J);
    double *q = malloc(sizeof(double) * J);
    int status;
    if (or_jacobi(J, rowptr, colidx, vals, dinv)) { status = OR_BADINPUT; *iters = 0; *relres = NAN; goto done; }

    for (int i = 0; i < J; i++) {
        x[i] = 0.0;
        r[i] = b[i];
        z[i] = dinv[i] * r[i];
        p[i] = z[i];
    }
    double bb = dot(J, b, b);
    double bnorm = sqrt(bb);
    double rz = dot(J, r, z);
    double rr = bb;
    int k = 0;
    if (!isfinite(bb) || !isfinite(rz)) { status = OR_BADINPUT; *iters = 0; *relres = NAN; goto done; }
    if (bnorm == 0.0) { status = OR_CONVERGED; *iters = 0; *relres = 0.0; goto done; }

    status = OR_MAXIT;
    while (k < maxit) {
        or_spmv(J, rowptr, colidx, vals, p, q);
        double pq = dot(J, p, q);
        if (!(pq > 0.0) || !isfinite(pq)) { status = OR_BREAKDOWN; break; }
        double alpha = rz / pq;
        for (int i = 0; i < J; i++) {
            x[i] = x[i] + alpha * p[i];
            r[i] = r[i] - alpha * q[i];
        }
        k++;
        rr = dot(J, r, r);
        if (hist) hist[k - 1] = sqrt(rr) / bnorm;
        if (sqrt(rr) <= rtol * bnorm) { status = OR_CONVERGED; break; }
        for (int i = 0; i < J; i++) z[i] = dinv[i] * r[i];
        double rz_new = dot(J, r, z);
        double beta = rz_new / rz;
        for (int i = 0; i < J; i++) p[i] = z[i] + beta * p[i];
        rz = rz_new;
    }
    *iters = k;
    *relres = sqrt(rr) / bnorm;
done:
    free(dinv); free(r); free(z); free(p); free(q);
    return status;
}

int or_pcg(int J, const int64_t *rowptr, const int32_t *colidx,
           const double *vals, const double *b, double rtol, int maxit,
           double *x, int *iters, double *relres)
{
    return pcg_run(J, rowptr, colidx, vals, b, rtol, maxit, x, iters, relres, NULL);
}

int or_pcg_history(int J, const int64_t *rowptr, const int32_t *colidx,
                   const double *vals, const double *b, double rtol, int maxit,
                   double *x, int *iters, double *relres, double *hist)
{
    return pcg_run(J, rowptr, colidx, vals, b, rtol, maxit, x, iters, relres, hist);
}

/* ---- batch driver: one sample per thread at a time ----------------------- */
typedef struct {
    int kind, n, nparam, M, nthreads, tid, maxit;
    double aniso, rtol;
    const double *xi;
    int *iters, *status;
    double *relres, *G, *xout;
    const int64_t *rowptr;
    const int32_t *colidx;
    int J;
    int64_t nnz;
    int err;
} batch_arg;

static void *batch_worker(void *vp)
{
    batch_arg *a = (batch_arg *)vp;
    double *vals = malloc(sizeof(double) * a->nnz);
    double *b = malloc(sizeof(double) * a->J);
    double *x = malloc(sizeof(double) * a->J);
    for (int m = a->tid; m < a->M; m += a->nthreads) {
        const double *xi = a->xi + (int64_t)m * a->nparam;
        if (or_assemble(a->kind, a->n, a->nparam, a->aniso, xi, a->rowptr, a->colidx, vals, b)) {
            a->err = -1;
            break;
        }
        a->status[m] = or_pcg(a->J, a->rowptr, a->colidx, vals, b, a->rtol, a->maxit, x,
                              &a->iters[m], &a->relres[m]);
        a->G[m] = dot(a->J, x, x);
        if (a->xout) memcpy(a->xout + (int64_t)m * a->J, x, sizeof(double) * a->J);
    }
    free(vals); free(b); free(x);
    return NULL;
}

int or_solve_batch(int kind, int n, int nparam, double aniso, int M,
                   const double *xi, double rtol, int maxit, int nthreads,
                   int *iters, int *status, double *relres, double *G, double *xout)
{
    int J;
    int64_t nnz;
    if (or_problem_size(kind, n, &J, &nnz)) return -1;
    int64_t *rowptr = malloc(sizeof(int64_t) * (J + 1));
    int32_t *colidx = malloc(sizeof(int32_t) * nnz);
    or_pattern(kind, n, rowptr, colidx);
    if (nthreads < 1) nthreads = 1;
    if (nthreads > M) nthreads = M > 0 ? M : 1;
    pthread_t *th = malloc(sizeof(pthread_t) * nthreads);
    batch_arg *args = malloc(sizeof(batch_arg) * nthreads);
    for (int t = 0; t < nthreads; t++) {
        batch_arg a = {kind, n, nparam, M, nthreads, t, maxit, aniso, rtol, xi, iters, status,
                       relres, G, xout, rowptr, colidx, J, nnz, 0};
        args[t] = a;
        pthread_create(&th[t], NULL, batch_worker, &args[t]);
    }
    int err = 0;
    for (int t = 0; t < nthreads; t++) {
        pthread_join(th[t], NULL);
        if (args[t].err) err = args[t].err;
    }
    free(th); free(args); free(rowptr); free(colidx);
    return err;
}

/* ---- mixed precision ------------------------------------------------------
 * FP64 iterative refinement around an FP32 inner Jacobi-PCG:
 *   r = b - A64 x (FP64); stop when ||r|| <= rtol_outer ||b||;
 *   solve A32 d = r with FP32 matrix values and FP32 vectors, FP64 scalars
 *   and inner-product accumulation, to ||r - A32 d|| <= rtol_inner ||r||;
 *   x = x + d in FP64. */
int or_pcg_ir(int J, const int64_t *rowptr, const int32_t *colidx,
              const double *vals, const double *b, double rtol_outer,
              double rtol_inner, int maxit_inner, int maxit_outer,
              double *x, int *outer_its, int *inner_its, double *relres)
{
    int64_t nnz = rowptr[J];
    float *v32 = malloc(sizeof(float) * nnz);
    float *dinv32 = malloc(sizeof(float) * J), *r32 = malloc(sizeof(float) * J);
    float *p32 = malloc(sizeof(float) * J), *q32 = malloc(sizeof(float) * J);
    float *z32 = malloc(sizeof(float) * J), *d32 = malloc(sizeof(float) * J);
    double *r = malloc(sizeof(double) * J), *dinv = malloc(sizeof(double) * J);
    int status = OR_MAXIT;
    *outer_its = 0;
    *inner_its = 0;
    if (or_jacobi(J, rowptr, colidx, vals, dinv)) { status = OR_BADINPUT; goto done; }
    for (int64_t k = 0; k < nnz; k++) v32[k] = (float)vals[k];
    for (int i = 0; i < J; i++) {
        dinv32[i] = (float)dinv[i];
        x[i] = 0.0;
    }
    double bnorm = sqrt(dot(J, b, b));
    if (!isfinite(bnorm)) { status = OR_BADINPUT; goto done; }
    for (;;) {
        or_spmv(J, rowptr, colidx, vals, x, r);
        for (int i = 0; i < J; i++) r[i] = b[i] - r[i];
        double rn = sqrt(dot(J, r, r));
        *relres = (bnorm > 0.0) ? rn / bnorm : 0.0;
        if (rn <= rtol_outer * bnorm) { status = OR_CONVERGED; break; }
        if (*outer_its >= maxit_outer) { status = OR_MAXIT; break; }
        /* inner FP32 PCG on A32 d = r */
        double rr = 0.0, rz = 0.0;
        for (int i = 0; i < J; i++) {
            r32[i] = (float)r[i];
            d32[i] = 0.0f;
            z32[i] = dinv32[i] * r32[i];
            p32[i] = z32[i];
            rr = rr + (double)r32[i] * (double)r32[i];
            rz = rz + (double)r32[i] * (double)z32[i];
        }
        double r0 = sqrt(rr);
        int k = 0;
        while (k < maxit_inner) {
            double pq = 0.0;
            for (int i = 0; i < J; i++) {
                float s = 0.0f;
                for (int64_t e = rowptr[i]; e < rowptr[i + 1]; e++) s = s + v32[e] * p32[colidx[e]];
                q32[i] = s;
                pq = pq + (double)p32[i] * (double)s;
            }
            if (!(pq > 0.0) || !isfinite(pq)) break;
            double alpha = rz / pq;
            float af = (float)alpha;
            rr = 0.0;
            for (int i = 0; i < J; i++) {
                d32[i] = d32[i] + af * p32[i];
                r32[i] = r32[i] - af * q32[i];
                rr = rr + (double)r32[i] * (double)r32[i];
            }
            k++;
            if (sqrt(rr) <= rtol_inner * r0) break;
            double rz_new = 0.0;
            for (int i = 0; i < J; i++) {
                z32[i] = dinv32[i] * r32[i];
                rz_new = rz_new + (double)r32[i] * (double)z32[i];
            }
            float bf = (float)(rz_new / rz);
            for (int i = 0; i < J; i++) p32[i] = z32[i] + bf * p32[i];
            rz = rz_new;
        }
        *inner_its += k;
        (*outer_its)++;
        if (k == 0) { status = OR_BREAKDOWN; break; }
        for (int i = 0; i < J; i++) x[i] = x[i] + (double)d32[i];
    }
done:
    free(v32); free(dinv32); free(r32); free(p32); free(q32); free(z32); free(d32);
    free(r); free(dinv);
    return status;
}

/* ---- adjoint gradient ------------------------------------------------------
 * Q(xi) = w^T u with A(xi) u = b.  With A lambda = w (A symmetric),
 *   dQ/dxi_k = -lambda^T (dA/dxi_k) u.
 * For the FD flux form A = sum_f k_f a_f a_f^T / h^2 with a_f = e_p - e_nbr
 * (or e_p for a boundary face), so
 *   dQ/dxi_k = -sum_f (dk_f/dxi_k) (lambda_p - lambda_nbr)(u_p - u_nbr) / h^2,
 * the neighbour values being 0 on boundary faces.  dk_f/dxi_k follows from
 * the field's form k = exp(s(x, xi)) 10^(aniso xi_j):
 *   dk/dxi = k * d(log k)/dxi, with d(log k)/dxi linear in the sine modes. */
static double dlogk(int kind, int nparam, double aniso, int axis, int kparam, const double *x)
{
    if (kind == OR_FD5_LOGKL) {
        if (kparam == 0) return axis == 1 ? aniso * log(10.0) : 0.0;
        static const int M2[7][2] = {{1, 1}, {2, 1}, {1, 2}, {2, 2}, {3, 1}, {1, 3}, {3, 2}};
        double phi = sin(M_PI * (double)M2[kparam - 1][0] * x[0]) *
                     sin(M_PI * (double)M2[kparam - 1][1] * x[1]);
        return 0.5 * phi / (double)kparam;
    }
    if (kind == OR_FD7_AXIS) {
        if (kparam == 0) return axis == 1 ? aniso * log(10.0) : 0.0;
        if (kparam == 1) return axis == 2 ? aniso * log(10.0) : 0.0;
        static const int M3[4][3] = {{1, 1, 1}, {2, 1, 1}, {1, 2, 1}, {1, 1, 2}};
        int m = kparam - 2;
        double phi = sin(M_PI * (double)M3[m][0] * x[0]) * sin(M_PI * (double)M3[m][1] * x[1]) *
                     sin(M_PI * (double)M3[m][2] * x[2]);
        return 0.3 * phi;
    }
    (void)nparam;
    return NAN;
}

int or_adjoint_grad(int kind, int n, int nparam, double aniso, const double *xi,
                    const double *w, double rtol, int maxit,
                    double *Q, double *grad, int *iters_fwd, int *iters_adj)
{
    if (kind != OR_FD5_LOGKL && kind != OR_FD7_AXIS) return -1;
    int J;
    int64_t nnz;
    if (or_problem_size(kind, n, &J, &nnz)) return -1;
    int d = (kind == OR_FD7_AXIS) ? 3 : 2;
    int64_t *rowptr = malloc(sizeof(int64_t) * (J + 1));
    int32_t *colidx = malloc(sizeof(int32_t) * nnz);
    double *vals = malloc(sizeof(double) * nnz), *b = malloc(sizeof(double) * J);
    double *u = malloc(sizeof(double) * J), *lam = malloc(sizeof(double) * J);
    or_pattern(kind, n, rowptr, colidx);
    int st = or_assemble(kind, n, nparam, aniso, xi, rowptr, colidx, vals, b);
    double rr;
    int s1 = -1, s2 = -1;
    if (st == 0) {
        s1 = or_pcg(J, rowptr, colidx, vals, b, rtol, maxit, u, iters_fwd, &rr);
        s2 = or_pcg(J, rowptr, colidx, vals, w, rtol, maxit, lam, iters_adj, &rr);
        *Q = dot(J, w, u);
        double ih2 = (double)(n + 1) * (double)(n + 1);
        double K[9];
        for (int k = 0; k < nparam; k++) grad[k] = 0.0;
        for (int p = 0; p < J; p++) {
            int g[3] = {p % n, (p / n) % n, (d == 3) ? p / (n * n) : 0};
            int stride[3] = {1, n, n * n};
            for (int axis = 0; axis < d; axis++)
                for (int dir = -1; dir <= 1; dir += 2) {
                    int nb = g[axis] + dir;
                    /* each interior face once (from its lower node); boundary faces from their node */
                    if (nb >= 0 && nb < n && dir < 0) continue;
                    double xm[3];
                    for (int a = 0; a < d; a++) xm[a] = (double)(g[a] + 1) / (double)(n + 1);
                    xm[axis] = ((double)(g[axis] + 1) + 0.5 * dir) / (double)(n + 1);
                    or_tensor(kind, nparam, aniso, xi, xm, K);
                    double kf = K[axis * d + axis];
                    double un = 0.0, ln = 0.0;
                    if (nb >= 0 && nb < n) {
                        un = u[p + dir * stride[axis]];
                        ln = lam[p + dir * stride[axis]];
                    }
                    double prod = (lam[p] - ln) * (u[p] - un) * ih2;
                    for (int k = 0; k < nparam; k++)
                        grad[k] = grad[k] - kf * dlogk(kind, nparam, aniso, axis, k, xm) * prod;
                }
        }
    }
    free(rowptr); free(colidx); free(vals); free(b); free(u); free(lam);
    if (st) return -1;
    return (s1 != OR_CONVERGED) ? s1 : s2;
}
