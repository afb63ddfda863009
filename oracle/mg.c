/*
 * mg.c -- oracle: geometric multigrid V-cycle as the CG preconditioner of the
 * trilinear problems (OR_Q1_3D_KL / OR_Q1_3D_DISC).
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Section 4 preconditions CG with multigrid whose levels are smoothed by a
 * second-order Chebyshev polynomial and whose coarsest level is solved
 * directly.  On the structured (n + 1)^3-cell mesh the hierarchy here is the
 * nested trilinear one (written out from the definitions, slowly):
 *   - levels: n_0 = n interior nodes per axis, n_{l+1} = (n_l - 1) / 2 while
 *     n_l > 3; n must be 2^k - 1 (k >= 2).  Node c (0-based) of level l + 1 sits
 *     on node 2c + 1 of level l;
 *   - prolongation P: trilinear interpolation, P(f, c) = prod_axes w with
 *     w = 1 if f_a = 2 c_a + 1, 1/2 if |f_a - (2 c_a + 1)| = 1, else 0
 *     (Dirichlet nodes carry zero);
 *   - coarse operators A_{l+1} = P^T A_l P (Galerkin), in the 27-point pattern
 *     of level l + 1;
 *   - smoother: the degree-2 Chebyshev semi-iteration on D^-1 A over
 *     [lambda_max / 30, lambda_max], lambda_max the Gershgorin bound
 *     max_i sum_j |a_ij| / a_ii of D^-1 A;
 *   - coarsest level (n = 3, 27 unknowns): dense Cholesky;
 *   - one V-cycle per application: pre-smooth from zero, restrict the
 *     residual, recurse, add the prolonged correction, post-smooth.  Both
 *     smoothings apply the same polynomial, so the V-cycle is symmetric.
 * CG itself follows or_pcg with z = V-cycle(r) in place of D^-1 r.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define MG_RATIO 30.0

int or_mg_levels(int n, int *ns)
{
    int k = 0;
    if (n < 3) return -1;
    for (int m = n + 1; m > 1; m >>= 1) {
        if (m & 1) return -1;  /* n + 1 must be a power of two */
    }
    ns[k++] = n;
    while (ns[k - 1] > 3) {
        if (k >= OR_MG_MAXLEV) return -1;
        ns[k] = (ns[k - 1] - 1) / 2;
        k++;
    }
    return k;
}

/* Weight of fine coordinate f in the 1-D interpolation from coarse coordinate c. */
static double w1(int f, int c)
{
    int d = f - (2 * c + 1);
    if (d == 0) return 1.0;
    if (d == 1 || d == -1) return 0.5;
    return 0.0;
}

static int64_t find_col(const int64_t *rp, const int32_t *ci, int row, int col)
{
    for (int64_t k = rp[row]; k < rp[row + 1]; k++)
        if (ci[k] == col) return k;
    return -1;
}

int or_mg_galerkin(int nf, const int64_t *rpf, const int32_t *cif, const double *vf,
                   int nc, const int64_t *rpc, const int32_t *cic, double *vc)
{
    if (nf != 2 * nc + 1) return -1;
    for (int64_t k = 0; k < rpc[nc * nc * nc]; k++) vc[k] = 0.0;
    for (int I2 = 0; I2 < nc; I2++)
        for (int I1 = 0; I1 < nc; I1++)
            for (int I0 = 0; I0 < nc; I0++) {
                const int I = I0 + nc * I1 + nc * nc * I2;
                /* fine nodes i with P(i, I) != 0, in increasing index */
                for (int i2 = 2 * I2; i2 <= 2 * I2 + 2; i2++)
                    for (int i1 = 2 * I1; i1 <= 2 * I1 + 2; i1++)
                        for (int i0 = 2 * I0; i0 <= 2 * I0 + 2; i0++) {
                            const int i = i0 + nf * i1 + nf * nf * i2;
                            const double wi = w1(i0, I0) * w1(i1, I1) * w1(i2, I2);
                            for (int64_t k = rpf[i]; k < rpf[i + 1]; k++) {
                                const int j = cif[k];
                                const int j0 = j % nf, j1 = (j / nf) % nf, j2 = j / (nf * nf);
                                /* coarse J with P(j, J) != 0 */
                                for (int J2 = (j2 - 1) / 2 - 1; J2 <= (j2 + 1) / 2; J2++)
                                    for (int J1 = (j1 - 1) / 2 - 1; J1 <= (j1 + 1) / 2; J1++)
                                        for (int J0 = (j0 - 1) / 2 - 1; J0 <= (j0 + 1) / 2; J0++) {
                                            if (J0 < 0 || J0 >= nc || J1 < 0 || J1 >= nc || J2 < 0 || J2 >= nc)
                                                continue;
                                            const double wj = w1(j0, J0) * w1(j1, J1) * w1(j2, J2);
                                            if (wj == 0.0) continue;
                                            const int J = J0 + nc * J1 + nc * nc * J2;
                                            const int64_t pos = find_col(rpc, cic, I, J);
                                            if (pos < 0) return -1;
                                            const double w = wi * wj;
                                            vc[pos] = vc[pos] + w * vf[k];
                                        }
                            }
                        }
            }
    return 0;
}

void or_mg_prolong(int nf, int nc, const double *ec, double *ef)
{
    for (int f2 = 0; f2 < nf; f2++)
        for (int f1 = 0; f1 < nf; f1++)
            for (int f0 = 0; f0 < nf; f0++) {
                double s = 0.0;
                for (int c2 = (f2 - 1) / 2 - 1; c2 <= (f2 + 1) / 2; c2++)
                    for (int c1 = (f1 - 1) / 2 - 1; c1 <= (f1 + 1) / 2; c1++)
                        for (int c0 = (f0 - 1) / 2 - 1; c0 <= (f0 + 1) / 2; c0++) {
                            if (c0 < 0 || c0 >= nc || c1 < 0 || c1 >= nc || c2 < 0 || c2 >= nc) continue;
                            const double w = w1(f0, c0) * w1(f1, c1) * w1(f2, c2);
                            if (w == 0.0) continue;
                            s = s + w * ec[c0 + nc * c1 + nc * nc * c2];
                        }
                ef[f0 + nf * f1 + nf * nf * f2] = s;
            }
}

void or_mg_restrict(int nf, int nc, const double *rf, double *rc)
{
    for (int c2 = 0; c2 < nc; c2++)
        for (int c1 = 0; c1 < nc; c1++)
            for (int c0 = 0; c0 < nc; c0++) {
                double s = 0.0;
                for (int f2 = 2 * c2; f2 <= 2 * c2 + 2; f2++)
                    for (int f1 = 2 * c1; f1 <= 2 * c1 + 2; f1++)
                        for (int f0 = 2 * c0; f0 <= 2 * c0 + 2; f0++) {
                            const double w = w1(f0, c0) * w1(f1, c1) * w1(f2, c2);
                            s = s + w * rf[f0 + nf * f1 + nf * nf * f2];
                        }
                rc[c0 + nc * c1 + nc * nc * c2] = s;
            }
}

double or_gershgorin(int J, const int64_t *rp, const int32_t *ci, const double *v)
{
    /* NaN when a row's ratio is not finite and positive (zero, negative or
     * missing diagonal, non-finite values): the hierarchy is then unusable. */
    double m = 0.0;
    int bad = 0;
    for (int i = 0; i < J; i++) {
        double s = 0.0, d = 0.0;
        for (int64_t k = rp[i]; k < rp[i + 1]; k++) {
            s = s + fabs(v[k]);
            if (ci[k] == i) d = v[k];
        }
        const double r = s / d;
        if (!(r > 0.0) || !isfinite(r)) bad = 1;
        else if (r > m) m = r;
    }
    return bad ? NAN : m;
}

void or_cheb(int J, const int64_t *rp, const int32_t *ci, const double *v, const double *dinv,
             double lmax, const double *b, double *x)
{
    /* Chebyshev semi-iteration of degree 2 on [lmax / 30, lmax]: the error
     * after it is p(D^-1 A) e_0, p(t) = T_2((theta - t) / delta) / T_2(theta / delta). */
    const double lmin = lmax / MG_RATIO;
    const double theta = (lmax + lmin) / 2.0, delta = (lmax - lmin) / 2.0;
    const double sigma = theta / delta;
    const double rho0 = 1.0 / sigma;
    double *d = malloc(sizeof(double) * J), *ax = malloc(sizeof(double) * J);
    or_spmv(J, rp, ci, v, x, ax);
    for (int i = 0; i < J; i++) {
        d[i] = dinv[i] * (b[i] - ax[i]) / theta;
        x[i] = x[i] + d[i];
    }
    const double rho1 = 1.0 / (2.0 * sigma - rho0);
    const double c1 = rho1 * rho0, c2 = 2.0 * rho1 / delta;
    or_spmv(J, rp, ci, v, x, ax);
    for (int i = 0; i < J; i++) {
        d[i] = c1 * d[i] + c2 * (dinv[i] * (b[i] - ax[i]));
        x[i] = x[i] + d[i];
    }
    free(d);
    free(ax);
}

/* ---- the hierarchy ----------------------------------------------------- */
typedef struct {
    int nlev;
    int n[OR_MG_MAXLEV], J[OR_MG_MAXLEV];
    int64_t *rp[OR_MG_MAXLEV];
    int32_t *ci[OR_MG_MAXLEV];
    double *v[OR_MG_MAXLEV], *dinv[OR_MG_MAXLEV];
    double lmax[OR_MG_MAXLEV];
    double *L;  /* dense Cholesky factor of the coarsest level, row-major J x J */
} mg_t;

static void mg_free(mg_t *m)
{
    for (int l = 0; l < m->nlev; l++) {
        if (l > 0) {
            free(m->rp[l]);
            free(m->ci[l]);
            free(m->v[l]);
        }
        free(m->dinv[l]);
    }
    free(m->L);
}

/* Cholesky A = L L^T of a dense row-major matrix; -1 on a non-positive pivot. */
static int chol(int J, const double *A, double *L)
{
    for (int k = 0; k < J * J; k++) L[k] = 0.0;
    for (int j = 0; j < J; j++) {
        double s = A[j * J + j];
        for (int k = 0; k < j; k++) s = s - L[j * J + k] * L[j * J + k];
        if (!(s > 0.0)) return -1;
        const double d = sqrt(s);
        L[j * J + j] = d;
        for (int i = j + 1; i < J; i++) {
            double t = A[i * J + j];
            for (int k = 0; k < j; k++) t = t - L[i * J + k] * L[j * J + k];
            L[i * J + j] = t / d;
        }
    }
    return 0;
}

static void chol_solve(int J, const double *L, const double *r, double *e)
{
    for (int i = 0; i < J; i++) {
        double s = r[i];
        for (int k = 0; k < i; k++) s = s - L[i * J + k] * e[k];
        e[i] = s / L[i * J + i];
    }
    for (int i = J - 1; i >= 0; i--) {
        double s = e[i];
        for (int k = i + 1; k < J; k++) s = s - L[k * J + i] * e[k];
        e[i] = s / L[i * J + i];
    }
}

static int mg_build(int n, const int64_t *rp, const int32_t *ci, const double *v, mg_t *m)
{
    memset(m, 0, sizeof(*m));
    int nl = or_mg_levels(n, m->n);
    if (nl < 1) return -1;
    m->nlev = nl;
    int rc = 0;
    for (int l = 0; l < nl; l++) {
        const int nn = m->n[l];
        int J;
        int64_t nnz;
        or_problem_size(OR_Q1_3D_KL, nn, &J, &nnz);
        m->J[l] = J;
        if (l == 0) {
            m->rp[0] = (int64_t *)rp;
            m->ci[0] = (int32_t *)ci;
            m->v[0] = (double *)v;
        } else {
            m->rp[l] = malloc(sizeof(int64_t) * (J + 1));
            m->ci[l] = malloc(sizeof(int32_t) * nnz);
            m->v[l] = malloc(sizeof(double) * nnz);
            or_pattern(OR_Q1_3D_KL, nn, m->rp[l], m->ci[l]);
            if (or_mg_galerkin(m->n[l - 1], m->rp[l - 1], m->ci[l - 1], m->v[l - 1], nn, m->rp[l], m->ci[l],
                               m->v[l]))
                rc = -1;
        }
        m->dinv[l] = malloc(sizeof(double) * J);
        if (or_jacobi(J, m->rp[l], m->ci[l], m->v[l], m->dinv[l])) rc = -1;
        m->lmax[l] = or_gershgorin(J, m->rp[l], m->ci[l], m->v[l]);
        if (!isfinite(m->lmax[l])) rc = -1;
    }
    const int l = nl - 1, J = m->J[l];
    double *A = calloc((size_t)J * J, sizeof(double));
    for (int i = 0; i < J; i++)
        for (int64_t k = m->rp[l][i]; k < m->rp[l][i + 1]; k++) A[i * J + m->ci[l][k]] = m->v[l][k];
    m->L = malloc(sizeof(double) * J * J);
    if (chol(J, A, m->L)) rc = -1;
    free(A);
    return rc;
}

static void mg_vcycle(const mg_t *m, int l, const double *r, double *e)
{
    const int J = m->J[l];
    if (l == m->nlev - 1) {
        chol_solve(J, m->L, r, e);
        return;
    }
    const int Jc = m->J[l + 1];
    double *res = malloc(sizeof(double) * J), *rc = malloc(sizeof(double) * Jc);
    double *ec = malloc(sizeof(double) * Jc), *pe = malloc(sizeof(double) * J);
    for (int i = 0; i < J; i++) e[i] = 0.0;
    or_cheb(J, m->rp[l], m->ci[l], m->v[l], m->dinv[l], m->lmax[l], r, e);
    or_spmv(J, m->rp[l], m->ci[l], m->v[l], e, res);
    for (int i = 0; i < J; i++) res[i] = r[i] - res[i];
    or_mg_restrict(m->n[l], m->n[l + 1], res, rc);
    mg_vcycle(m, l + 1, rc, ec);
    or_mg_prolong(m->n[l], m->n[l + 1], ec, pe);
    for (int i = 0; i < J; i++) e[i] = e[i] + pe[i];
    or_cheb(J, m->rp[l], m->ci[l], m->v[l], m->dinv[l], m->lmax[l], r, e);
    free(res);
    free(rc);
    free(ec);
    free(pe);
}

int or_mg_coarse(int n, const int64_t *rp, const int32_t *ci, const double *v, int level, double *vc,
                 double *lmax)
{
    mg_t m;
    int rc = mg_build(n, rp, ci, v, &m);
    if (level < 0 || level >= m.nlev) rc = -1;
    if (rc == 0) {
        int J;
        int64_t nnz;
        or_problem_size(OR_Q1_3D_KL, m.n[level], &J, &nnz);
        memcpy(vc, m.v[level], sizeof(double) * nnz);
        *lmax = m.lmax[level];
    }
    mg_free(&m);
    return rc;
}

int or_mg_apply(int n, const int64_t *rp, const int32_t *ci, const double *v, const double *r, double *z)
{
    mg_t m;
    int rc = mg_build(n, rp, ci, v, &m);
    if (rc == 0) mg_vcycle(&m, 0, r, z);
    mg_free(&m);
    return rc;
}

static double dot(int J, const double *a, const double *b)
{
    double s = 0.0;
    for (int i = 0; i < J; i++) s = s + a[i] * b[i];
    return s;
}

int or_mgpcg(int n, const int64_t *rp, const int32_t *ci, const double *v, const double *b, double rtol,
             int maxit, double *x, int *iters, double *relres)
{
    mg_t m;
    int status;
    const int J = n * n * n;
    double *r = malloc(sizeof(double) * J), *z = malloc(sizeof(double) * J);
    double *p = malloc(sizeof(double) * J), *q = malloc(sizeof(double) * J);
    for (int i = 0; i < J; i++) x[i] = 0.0;
    if (mg_build(n, rp, ci, v, &m)) { status = OR_BADINPUT; *iters = 0; *relres = NAN; goto done; }
    for (int i = 0; i < J; i++) r[i] = b[i];
    mg_vcycle(&m, 0, r, z);
    for (int i = 0; i < J; i++) p[i] = z[i];
    double bb = dot(J, b, b);
    double bnorm = sqrt(bb);
    double rz = dot(J, r, z);
    double rr = bb;
    int k = 0;
    if (!isfinite(bb) || !isfinite(rz)) { status = OR_BADINPUT; *iters = 0; *relres = NAN; goto done; }
    if (bnorm == 0.0) { status = OR_CONVERGED; *iters = 0; *relres = 0.0; goto done; }
    status = OR_MAXIT;
    while (k < maxit) {
        or_spmv(J, rp, ci, v, p, q);
        double pq = dot(J, p, q);
        if (!(pq > 0.0) || !isfinite(pq)) { status = OR_BREAKDOWN; break; }
        double alpha = rz / pq;
        for (int i = 0; i < J; i++) {
            x[i] = x[i] + alpha * p[i];
            r[i] = r[i] - alpha * q[i];
        }
        k++;
        rr = dot(J, r, r);
        if (sqrt(rr) <= rtol * bnorm) { status = OR_CONVERGED; break; }
        mg_vcycle(&m, 0, r, z);
        double rz_new = dot(J, r, z);
        double beta = rz_new / rz;
        for (int i = 0; i < J; i++) p[i] = z[i] + beta * p[i];
        rz = rz_new;
    }
    *iters = k;
    *relres = sqrt(rr) / bnorm;
done:
    mg_free(&m);
    free(r); free(z); free(p); free(q);
    return status;
}

/* ---- FP32 V-cycle: the mixed-precision preconditioner ---------------------
 * The hierarchy is built in FP64 as above, then its values, inverse diagonals
 * and coarsest factor are rounded to float and one V-cycle runs entirely in
 * float (the right-hand side rounded in, the correction widened out).  The
 * Chebyshev coefficients are formed in FP64 and rounded: 1/theta, c1, c2 with
 * d0 = D^-1 (b - A x) / theta and d1 = c1 d0 + c2 D^-1 (b - A x).  CG stays in
 * FP64 (or_mgpcg32). */
typedef struct {
    float *v[OR_MG_MAXLEV], *dinv[OR_MG_MAXLEV];
    float c[OR_MG_MAXLEV][3];
    float *L;
} mg32_t;

static void mg32_from(const mg_t *m, mg32_t *f)
{
    for (int l = 0; l < m->nlev; l++) {
        const int J = m->J[l];
        const int64_t nnz = m->rp[l][J];
        f->v[l] = malloc(sizeof(float) * nnz);
        f->dinv[l] = malloc(sizeof(float) * J);
        for (int64_t k = 0; k < nnz; k++) f->v[l][k] = (float)m->v[l][k];
        for (int i = 0; i < J; i++) f->dinv[l][i] = (float)m->dinv[l][i];
        const double lmax = m->lmax[l], lmin = lmax / MG_RATIO;
        const double theta = (lmax + lmin) / 2.0, delta = (lmax - lmin) / 2.0;
        const double sigma = theta / delta, rho0 = 1.0 / sigma, rho1 = 1.0 / (2.0 * sigma - rho0);
        f->c[l][0] = (float)(1.0 / theta);
        f->c[l][1] = (float)(rho1 * rho0);
        f->c[l][2] = (float)(2.0 * rho1 / delta);
    }
    const int J = m->J[m->nlev - 1];
    f->L = malloc(sizeof(float) * J * J);
    for (int k = 0; k < J * J; k++) f->L[k] = (float)m->L[k];
}

static void mg32_free(const mg_t *m, mg32_t *f)
{
    for (int l = 0; l < m->nlev; l++) {
        free(f->v[l]);
        free(f->dinv[l]);
    }
    free(f->L);
}

static void spmv32(int J, const int64_t *rp, const int32_t *ci, const float *v, const float *x, float *y)
{
    for (int i = 0; i < J; i++) {
        float s = 0.0f;
        for (int64_t k = rp[i]; k < rp[i + 1]; k++) s = s + v[k] * x[ci[k]];
        y[i] = s;
    }
}

static void cheb32(int J, const int64_t *rp, const int32_t *ci, const float *v, const float *dinv, const float *c,
                   const float *b, float *x)
{
    float *d = malloc(sizeof(float) * J), *ax = malloc(sizeof(float) * J);
    spmv32(J, rp, ci, v, x, ax);
    for (int i = 0; i < J; i++) {
        d[i] = dinv[i] * (b[i] - ax[i]) * c[0];
        x[i] = x[i] + d[i];
    }
    spmv32(J, rp, ci, v, x, ax);
    for (int i = 0; i < J; i++) {
        d[i] = c[1] * d[i] + c[2] * (dinv[i] * (b[i] - ax[i]));
        x[i] = x[i] + d[i];
    }
    free(d);
    free(ax);
}

static void vcycle32(const mg_t *m, const mg32_t *f, int l, const float *r, float *e)
{
    const int J = m->J[l];
    if (l == m->nlev - 1) {
        for (int i = 0; i < J; i++) {
            float s = r[i];
            for (int k = 0; k < i; k++) s = s - f->L[i * J + k] * e[k];
            e[i] = s / f->L[i * J + i];
        }
        for (int i = J - 1; i >= 0; i--) {
            float s = e[i];
            for (int k = i + 1; k < J; k++) s = s - f->L[k * J + i] * e[k];
            e[i] = s / f->L[i * J + i];
        }
        return;
    }
    const int nf = m->n[l], nc = m->n[l + 1], Jc = m->J[l + 1];
    float *res = malloc(sizeof(float) * J), *rc = malloc(sizeof(float) * Jc), *ec = malloc(sizeof(float) * Jc);
    for (int i = 0; i < J; i++) e[i] = 0.0f;
    cheb32(J, m->rp[l], m->ci[l], f->v[l], f->dinv[l], f->c[l], r, e);
    spmv32(J, m->rp[l], m->ci[l], f->v[l], e, res);
    for (int i = 0; i < J; i++) res[i] = r[i] - res[i];
    for (int c2 = 0; c2 < nc; c2++)  /* rc = P^T res */
        for (int c1 = 0; c1 < nc; c1++)
            for (int c0 = 0; c0 < nc; c0++) {
                float acc = 0.0f;
                for (int f2 = 2 * c2; f2 <= 2 * c2 + 2; f2++)
                    for (int f1 = 2 * c1; f1 <= 2 * c1 + 2; f1++)
                        for (int f0 = 2 * c0; f0 <= 2 * c0 + 2; f0++)
                            acc = acc + (float)(w1(f0, c0) * w1(f1, c1) * w1(f2, c2)) * res[f0 + nf * f1 + nf * nf * f2];
                rc[c0 + nc * c1 + nc * nc * c2] = acc;
            }
    vcycle32(m, f, l + 1, rc, ec);
    for (int f2 = 0; f2 < nf; f2++)  /* e += P ec */
        for (int f1 = 0; f1 < nf; f1++)
            for (int f0 = 0; f0 < nf; f0++) {
                float acc = 0.0f;
                for (int c2 = (f2 - 1) / 2 - 1; c2 <= (f2 + 1) / 2; c2++)
                    for (int c1 = (f1 - 1) / 2 - 1; c1 <= (f1 + 1) / 2; c1++)
                        for (int c0 = (f0 - 1) / 2 - 1; c0 <= (f0 + 1) / 2; c0++) {
                            if (c0 < 0 || c0 >= nc || c1 < 0 || c1 >= nc || c2 < 0 || c2 >= nc) continue;
                            const double w = w1(f0, c0) * w1(f1, c1) * w1(f2, c2);
                            if (w == 0.0) continue;
                            acc = acc + (float)w * ec[c0 + nc * c1 + nc * nc * c2];
                        }
                e[f0 + nf * f1 + nf * nf * f2] = e[f0 + nf * f1 + nf * nf * f2] + acc;
            }
    cheb32(J, m->rp[l], m->ci[l], f->v[l], f->dinv[l], f->c[l], r, e);
    free(res);
    free(rc);
    free(ec);
}

int or_mg_apply32(int n, const int64_t *rp, const int32_t *ci, const double *v, const double *r, double *z)
{
    mg_t m;
    int rc = mg_build(n, rp, ci, v, &m);
    if (rc == 0) {
        mg32_t f;
        mg32_from(&m, &f);
        const int J = m.J[0];
        float *r32 = malloc(sizeof(float) * J), *e32 = malloc(sizeof(float) * J);
        for (int i = 0; i < J; i++) r32[i] = (float)r[i];
        vcycle32(&m, &f, 0, r32, e32);
        for (int i = 0; i < J; i++) z[i] = (double)e32[i];
        free(r32);
        free(e32);
        mg32_free(&m, &f);
    }
    mg_free(&m);
    return rc;
}

int or_mgpcg32(int n, const int64_t *rp, const int32_t *ci, const double *v, const double *b, double rtol,
               int maxit, double *x, int *iters, double *relres)
{
    mg_t m;
    mg32_t f;
    int status, built = 0;
    const int J = n * n * n;
    double *r = malloc(sizeof(double) * J), *z = malloc(sizeof(double) * J);
    double *p = malloc(sizeof(double) * J), *q = malloc(sizeof(double) * J);
    float *r32 = malloc(sizeof(float) * J), *e32 = malloc(sizeof(float) * J);
    for (int i = 0; i < J; i++) x[i] = 0.0;
    if (mg_build(n, rp, ci, v, &m)) { status = OR_BADINPUT; *iters = 0; *relres = NAN; goto done; }
    mg32_from(&m, &f);
    built = 1;
#define PREC(rv, zv)                                                  \
    do {                                                              \
        for (int i_ = 0; i_ < J; i_++) r32[i_] = (float)(rv)[i_];     \
        vcycle32(&m, &f, 0, r32, e32);                                \
        for (int i_ = 0; i_ < J; i_++) (zv)[i_] = (double)e32[i_];    \
    } while (0)
    for (int i = 0; i < J; i++) r[i] = b[i];
    PREC(r, z);
    for (int i = 0; i < J; i++) p[i] = z[i];
    double bb = dot(J, b, b);
    double bnorm = sqrt(bb);
    double rz = dot(J, r, z);
    double rr = bb;
    int k = 0;
    if (!isfinite(bb) || !isfinite(rz)) { status = OR_BADINPUT; *iters = 0; *relres = NAN; goto done; }
    if (bnorm == 0.0) { status = OR_CONVERGED; *iters = 0; *relres = 0.0; goto done; }
    status = OR_MAXIT;
    while (k < maxit) {
        or_spmv(J, rp, ci, v, p, q);
        double pq = dot(J, p, q);
        if (!(pq > 0.0) || !isfinite(pq)) { status = OR_BREAKDOWN; break; }
        double alpha = rz / pq;
        for (int i = 0; i < J; i++) {
            x[i] = x[i] + alpha * p[i];
            r[i] = r[i] - alpha * q[i];
        }
        k++;
        rr = dot(J, r, r);
        if (sqrt(rr) <= rtol * bnorm) { status = OR_CONVERGED; break; }
        PREC(r, z);
        double rz_new = dot(J, r, z);
        double beta = rz_new / rz;
        for (int i = 0; i < J; i++) p[i] = z[i] + beta * p[i];
        rz = rz_new;
    }
#undef PREC
    *iters = k;
    *relres = sqrt(rr) / bnorm;
done:
    if (built) mg32_free(&m, &f);
    mg_free(&m);
    free(r); free(z); free(p); free(q); free(r32); free(e32);
    return status;
}
