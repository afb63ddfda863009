/*
 * problem.c -- oracle: grid graph and per-sample assembly of the discrete
 * systems L_m U_m = F_m of Eq. (discrete-sys) for the stochastic elliptic
 * problem of Eq. (elliptic-SPDE).
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Grid: h = 1/(n+1); interior nodes at x = (i+1) h, i = 0..n-1 per axis;
 * unknowns in lexicographic order with x fastest.  Dirichlet neighbours are
 * zero and are dropped from the graph.
 *
 * FD (5-point 2-D, 7-point 3-D), flux form:
 *     (A u)_p = sum over the 2d faces f of p:  k_f (u_p - u_nbr) / h^2,
 * where k_f is the diagonal tensor entry for the face's axis evaluated at the
 * face midpoint; a boundary face contributes only to the diagonal.
 * Load b_p = f = 1.
 *
 * Q1 (2-D bilinear elements of side h, 9-point stencil): the tensor is
 * evaluated once per element at its centroid and the exact element stiffness
 * int grad(phi_a) . K grad(phi_b) of a constant tensor is assembled element
 * by element in lexicographic element order.  Load b_p = int f phi_p = h^2.
 *
 * Q1 3-D (trilinear elements of side h, 27-point stencil; the discretisation
 * of Section 4): as Q1 with the diagonal tensor diag(a, 1, 1) at the element
 * centroid; the exact element stiffness of a diagonal tensor is
 *   sum_d K_dd h (1-D derivative product along d) (1-D mass products across d)
 * on the reference cube; load b_p = int f phi_p = h^3.
 */
#include "oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>

/* KL-style sine modes (m_x, m_y) used by the 2-D log-coefficient fields. */
static const int MODES2[7][2] = {{1, 1}, {2, 1}, {1, 2}, {2, 2}, {3, 1}, {1, 3}, {3, 2}};
/* Tensor-sine modes (m_x, m_y, m_z) for xi_3..xi_6 of the 3-D field. */
static const int MODES3[4][3] = {{1, 1, 1}, {2, 1, 1}, {1, 2, 1}, {1, 1, 2}};

static double sinmode(int m, double x) { return sin(M_PI * (double)m * x); }

/* ---- exponential-covariance KL (Section 4) -----------------------------------
 * 1-D kernel exp(-|s - t| / delta) on [0, 1], written on [-1/2, 1/2] with
 * c = 1 / delta.  Eigenfunctions and eigenvalues (the classical closed form of
 * this integral equation):
 *   even: cos(w u) / sqrt(1/2 + sin(w) / (2 w)),  w tan(w / 2) = c,      w in (0, pi)
 *   odd:  sin(w u) / sqrt(1/2 - sin(w) / (2 w)),  c tan(w / 2) + w = 0,  w in (pi, 2 pi)
 *   lambda = 2 c / (w^2 + c^2),  u = s - 1/2.
 * The roots are found by bisection (both functions increase across their
 * bracket).  With delta = 1/4 the four largest products of three 1-D modes are
 * e1 e1 e1, o1 e1 e1, e1 o1 e1, e1 e1 o1 (the next, e1 o1 o1, is smaller than
 * all of them); sigma0 scales the eigenvalues. */
static const double KL_DELTA = 0.25;
static const double KL_SIGMA0 = 17.320508075688772;  /* sqrt(300) */
static const double KL_AMIN = 0.1;

static double kl_root(int which)
{
    double c = 1.0 / KL_DELTA;
    double lo = which ? M_PI : 0.0, hi = which ? 2.0 * M_PI : M_PI;
    for (int it = 0; it < 200; it++) {
        double mid = 0.5 * (lo + hi);
        double f = which ? c * tan(0.5 * mid) + mid : mid * tan(0.5 * mid) - c;
        if (f < 0.0)
            lo = mid;
        else
            hi = mid;
    }
    return 0.5 * (lo + hi);
}

/* the two roots, found once (the batch solver assembles from several threads) */
static double kl_roots[2];
static pthread_once_t kl_once = PTHREAD_ONCE_INIT;
static void kl_init(void)
{
    kl_roots[0] = kl_root(0);
    kl_roots[1] = kl_root(1);
}

int or_kl_1d(int which, double *w, double *lambda)
{
    if (which != 0 && which != 1) return -1;
    pthread_once(&kl_once, kl_init);
    double c = 1.0 / KL_DELTA;
    double r = kl_roots[which];
    *w = r;
    *lambda = 2.0 * c / (r * r + c * c);
    return 0;
}

static double kl_1d_mode(int which, double w, double s)
{
    double u = s - 0.5;
    if (which == 0) return cos(w * u) / sqrt(0.5 + sin(w) / (2.0 * w));
    return sin(w * u) / sqrt(0.5 - sin(w) / (2.0 * w));
}

/* parameter k = 1..4: which coordinate carries the odd factor (0 = none) */
static const int KL_ODD_AXIS[4] = {0, 1, 2, 3};

double or_kl_lambda(int k)
{
    double we, le, wo, lo;
    or_kl_1d(0, &we, &le);
    or_kl_1d(1, &wo, &lo);
    return KL_SIGMA0 * (KL_ODD_AXIS[k - 1] ? lo * le * le : le * le * le);
}

double or_kl_mode(int k, const double *x)
{
    double we, le, wo, lo;
    or_kl_1d(0, &we, &le);
    or_kl_1d(1, &wo, &lo);
    double b = 1.0;
    for (int d = 0; d < 3; d++)
        b = b * (KL_ODD_AXIS[k - 1] == d + 1 ? kl_1d_mode(1, wo, x[d]) : kl_1d_mode(0, we, x[d]));
    return b;
}

int or_problem_size(int kind, int n, int *J, int64_t *nnz)
{
    if (n < 1) return -1;
    int64_t nn = n;
    switch (kind) {
    case OR_FD5_LOGKL: *J = (int)(nn * nn); *nnz = 5 * nn * nn - 4 * nn; return 0;
    case OR_Q1_ROT:    *J = (int)(nn * nn); *nnz = (3 * nn - 2) * (3 * nn - 2); return 0;
    case OR_FD7_AXIS:  *J = (int)(nn * nn * nn); *nnz = 7 * nn * nn * nn - 6 * nn * nn; return 0;
    case OR_Q1_3D_KL:
    case OR_Q1_3D_DISC: *J = (int)(nn * nn * nn); *nnz = (3 * nn - 2) * (3 * nn - 2) * (3 * nn - 2); return 0;
    default: return -1;
    }
}

/* Graph of one row: neighbours listed in increasing column order. */
int or_pattern(int kind, int n, int64_t *rowptr, int32_t *colidx)
{
    int64_t k = 0;
    rowptr[0] = 0;
    if (kind == OR_FD5_LOGKL) {
        for (int j = 0; j < n; j++)
            for (int i = 0; i < n; i++) {
                int p = i + n * j;
                if (j > 0) colidx[k++] = p - n;
                if (i > 0) colidx[k++] = p - 1;
                colidx[k++] = p;
                if (i < n - 1) colidx[k++] = p + 1;
                if (j < n - 1) colidx[k++] = p + n;
                rowptr[p + 1] = k;
            }
        return 0;
    }
    if (kind == OR_Q1_ROT) {
        for (int j = 0; j < n; j++)
            for (int i = 0; i < n; i++) {
                int p = i + n * j;
                for (int dj = -1; dj <= 1; dj++)
                    for (int di = -1; di <= 1; di++) {
                        int ii = i + di, jj = j + dj;
                        if (ii < 0 || ii >= n || jj < 0 || jj >= n) continue;
                        colidx[k++] = ii + n * jj;
                    }
                rowptr[p + 1] = k;
            }
        return 0;
    }
    if (kind == OR_Q1_3D_KL || kind == OR_Q1_3D_DISC) {
        for (int l = 0; l < n; l++)
            for (int j = 0; j < n; j++)
                for (int i = 0; i < n; i++) {
                    int p = i + n * j + n * n * l;
                    for (int dl = -1; dl <= 1; dl++)
                        for (int dj = -1; dj <= 1; dj++)
                            for (int di = -1; di <= 1; di++) {
                                int ii = i + di, jj = j + dj, ll = l + dl;
                                if (ii < 0 || ii >= n || jj < 0 || jj >= n || ll < 0 || ll >= n) continue;
                                colidx[k++] = ii + n * jj + n * n * ll;
                            }
                    rowptr[p + 1] = k;
                }
        return 0;
    }
    if (kind == OR_FD7_AXIS) {
        int n2 = n * n;
        for (int l = 0; l < n; l++)
            for (int j = 0; j < n; j++)
                for (int i = 0; i < n; i++) {
                    int p = i + n * j + n2 * l;
                    if (l > 0) colidx[k++] = p - n2;
                    if (j > 0) colidx[k++] = p - n;
                    if (i > 0) colidx[k++] = p - 1;
                    colidx[k++] = p;
                    if (i < n - 1) colidx[k++] = p + 1;
                    if (j < n - 1) colidx[k++] = p + n;
                    if (l < n - 1) colidx[k++] = p + n2;
                    rowptr[p + 1] = k;
                }
        return 0;
    }
    return -1;
}

/* The diffusion tensor A(x, xi) (row-major d x d). */
int or_tensor(int kind, int nparam, double aniso, const double *xi, const double *x, double *K)
{
    if (kind == OR_FD5_LOGKL) {
        /* log a = 0.5 * sum_{k=1}^{N-1} xi_{k+1} phi_k(x) / k    (Eq. diff-coeff, log form) */
        if (nparam < 1 || nparam > 8) return -1;
        double s = 0.0;
        for (int k = 1; k < nparam; k++) {
            double phi = sinmode(MODES2[k - 1][0], x[0]) * sinmode(MODES2[k - 1][1], x[1]);
            s = s + (xi[k] * phi) / (double)k;
        }
        double a = exp(0.5 * s);
        K[0] = a;
        K[1] = 0.0;
        K[2] = 0.0;
        K[3] = a * pow(10.0, aniso * xi[0]);
        return 0;
    }
    if (kind == OR_Q1_ROT) {
        if (nparam != 4) return -1;
        double phi1 = sinmode(1, x[0]) * sinmode(1, x[1]);
        double phi2 = sinmode(2, x[0]) * sinmode(1, x[1]);
        double a = exp(0.5 * (xi[1] * phi1 + (xi[3] * phi2) / 2.0));
        double theta = (M_PI / 4.0) * (1.0 + xi[2]);
        double c = cos(theta), s = sin(theta);
        double d2 = pow(10.0, aniso * xi[0]);
        /* R diag(1, d2) R^T with R = [[c, -s], [s, c]] */
        K[0] = a * (c * c + s * s * d2);
        K[1] = a * (c * s * (1.0 - d2));
        K[2] = K[1];
        K[3] = a * (s * s + c * c * d2);
        return 0;
    }
    if (kind == OR_FD7_AXIS) {
        if (nparam != 6) return -1;
        double s = 0.0;
        for (int k = 0; k < 4; k++) {
            double phi = sinmode(MODES3[k][0], x[0]) * sinmode(MODES3[k][1], x[1]) *
                         sinmode(MODES3[k][2], x[2]);
            s = s + xi[2 + k] * phi;
        }
        double e = exp(0.3 * s);
        for (int q = 0; q < 9; q++) K[q] = 0.0;
        K[0] = e;
        K[4] = e * pow(10.0, aniso * xi[0]);
        K[8] = e * pow(10.0, aniso * xi[1]);
        return 0;
    }
    if (kind == OR_Q1_3D_KL || kind == OR_Q1_3D_DISC) {
        if (nparam != 4) return -1;
        double s = 0.0;
        for (int k = 1; k <= 4; k++) s = s + sqrt(or_kl_lambda(k)) * or_kl_mode(k, x) * xi[k - 1];
        double ahat = 1.0;
        if (kind == OR_Q1_3D_DISC) {
            double r = sqrt(xi[0] * xi[0] + xi[1] * xi[1] + xi[2] * xi[2] + xi[3] * xi[3]);
            double d = sqrt(3.0);
            ahat = (r < d / 4.0) ? 1.0 : (r < d / 2.0 ? 100.0 : 10.0);
        }
        for (int q = 0; q < 9; q++) K[q] = 0.0;
        K[0] = KL_AMIN + ahat * exp(s);
        K[4] = 1.0;
        K[8] = 1.0;
        return 0;
    }
    return -1;
}

static int64_t find_col(const int64_t *rowptr, const int32_t *colidx, int row, int col)
{
    for (int64_t k = rowptr[row]; k < rowptr[row + 1]; k++)
        if (colidx[k] == col) return k;
    return -1;
}

/* Coordinate of a (half-)integer grid position t, i.e. t * h. */
static double coord(double t, int n) { return t / (double)(n + 1); }

static int assemble_fd(int kind, int n, int nparam, double aniso, const double *xi,
                       const int64_t *rowptr, const int32_t *colidx, double *vals, double *b)
{
    int d = (kind == OR_FD7_AXIS) ? 3 : 2;
    double ih2 = (double)(n + 1) * (double)(n + 1);
    int J = (d == 3) ? n * n * n : n * n;
    double K[9];
    for (int p = 0; p < J; p++) {
        int g[3] = {p % n, (p / n) % n, (d == 3) ? p / (n * n) : 0};
        int stride[3] = {1, n, n * n};
        /* faces in increasing column order: -z, -y, -x, +x, +y, +z */
        double diag = 0.0;
        for (int side = 0; side < 2; side++) {
            for (int q = 0; q < d; q++) {
                int axis = (side == 0) ? d - 1 - q : q;
                int dir = (side == 0) ? -1 : 1;
                double xm[3];
                for (int a = 0; a < d; a++) xm[a] = coord((double)g[a] + 1.0, n);
                xm[axis] = coord((double)g[axis] + 1.0 + 0.5 * dir, n);
                if (or_tensor(kind, nparam, aniso, xi, xm, K)) return -1;
                double kf = K[axis * d + axis];
                diag = diag + kf;
                int nb = g[axis] + dir;
                if (nb >= 0 && nb < n) {
                    int64_t pos = find_col(rowptr, colidx, p, p + dir * stride[axis]);
                    if (pos < 0) return -2;
                    vals[pos] = -(kf * ih2);
                }
            }
        }
        int64_t pd = find_col(rowptr, colidx, p, p);
        if (pd < 0) return -2;
        vals[pd] = diag * ih2;
        b[p] = 1.0;
    }
    return 0;
}

static int assemble_q1(int n, int nparam, double aniso, const double *xi,
                       const int64_t *rowptr, const int32_t *colidx, double *vals, double *b)
{
    int J = n * n;
    for (int64_t k = 0; k < rowptr[J]; k++) vals[k] = 0.0;
    /* Reference-square integrals of products of 1-D factors:
       int (1-s)^2 = int s^2 = 1/3, int s(1-s) = 1/6, int d/ds(.) against a
       1-D factor = 1/2; the sign of d/ds is -1 for (1-s) and +1 for s. */
    double sg[2] = {-1.0, 1.0};
    double Mm[2][2] = {{1.0 / 3.0, 1.0 / 6.0}, {1.0 / 6.0, 1.0 / 3.0}};
    double K[4];
    for (int ey = 0; ey <= n; ey++)
        for (int ex = 0; ex <= n; ex++) {
            double xc[2] = {coord((double)ex + 0.5, n), coord((double)ey + 0.5, n)};
            if (or_tensor(OR_Q1_ROT, nparam, aniso, xi, xc, K)) return -1;
            for (int l = 0; l < 4; l++) {
                int al = l & 1, bl = l >> 1;
                int nxl = ex + al, nyl = ey + bl; /* node coords 0..n+1 */
                if (nxl < 1 || nxl > n || nyl < 1 || nyl > n) continue;
                int row = (nxl - 1) + n * (nyl - 1);
                for (int m = 0; m < 4; m++) {
                    int am = m & 1, bm = m >> 1;
                    int nxm = ex + am, nym = ey + bm;
                    if (nxm < 1 || nxm > n || nym < 1 || nym > n) continue;
                    int col = (nxm - 1) + n * (nym - 1);
                    double c1 = sg[al] * sg[am] * Mm[bl][bm]; /* d/dx d/dx */
                    double c2 = sg[bl] * sg[bm] * Mm[al][am]; /* d/dy d/dy */
                    double c3 = (sg[al] * sg[bm] + sg[bl] * sg[am]) / 4.0; /* mixed */
                    double ke = K[0] * c1 + K[3] * c2 + K[1] * c3;
                    int64_t pos = find_col(rowptr, colidx, row, col);
                    if (pos < 0) return -2;
                    vals[pos] = vals[pos] + ke;
                }
            }
        }
    double bh = 1.0 / ((double)(n + 1) * (double)(n + 1));
    for (int p = 0; p < J; p++) b[p] = bh;
    return 0;
}

static int assemble_q1_3d(int kind, int n, int nparam, double aniso, const double *xi,
                          const int64_t *rowptr, const int32_t *colidx, double *vals, double *b)
{
    int J = n * n * n;
    for (int64_t k = 0; k < rowptr[J]; k++) vals[k] = 0.0;
    double h = 1.0 / (double)(n + 1);
    double sg[2] = {-1.0, 1.0};
    double Mm[2][2] = {{1.0 / 3.0, 1.0 / 6.0}, {1.0 / 6.0, 1.0 / 3.0}};
    double K[9];
    for (int ez = 0; ez <= n; ez++)
        for (int ey = 0; ey <= n; ey++)
            for (int ex = 0; ex <= n; ex++) {
                double xc[3] = {coord((double)ex + 0.5, n), coord((double)ey + 0.5, n), coord((double)ez + 0.5, n)};
                if (or_tensor(kind, nparam, aniso, xi, xc, K)) return -1;
                for (int l = 0; l < 8; l++) {
                    int al = l & 1, bl = (l >> 1) & 1, cl = l >> 2;
                    int nx = ex + al, ny = ey + bl, nz = ez + cl;
                    if (nx < 1 || nx > n || ny < 1 || ny > n || nz < 1 || nz > n) continue;
                    int row = (nx - 1) + n * (ny - 1) + n * n * (nz - 1);
                    for (int m = 0; m < 8; m++) {
                        int am = m & 1, bm = (m >> 1) & 1, cm = m >> 2;
                        int mx = ex + am, my = ey + bm, mz = ez + cm;
                        if (mx < 1 || mx > n || my < 1 || my > n || mz < 1 || mz > n) continue;
                        int col = (mx - 1) + n * (my - 1) + n * n * (mz - 1);
                        double dx = sg[al] * sg[am] * Mm[bl][bm] * Mm[cl][cm];
                        double dy = Mm[al][am] * sg[bl] * sg[bm] * Mm[cl][cm];
                        double dz = Mm[al][am] * Mm[bl][bm] * sg[cl] * sg[cm];
                        double ke = h * (K[0] * dx + K[4] * dy + K[8] * dz);
                        int64_t pos = find_col(rowptr, colidx, row, col);
                        if (pos < 0) return -2;
                        vals[pos] = vals[pos] + ke;
                    }
                }
            }
    for (int p = 0; p < J; p++) b[p] = h * h * h;
    return 0;
}

int or_assemble(int kind, int n, int nparam, double aniso, const double *xi,
                const int64_t *rowptr, const int32_t *colidx, double *vals, double *b)
{
    if (kind == OR_Q1_3D_KL || kind == OR_Q1_3D_DISC)
        return assemble_q1_3d(kind, n, nparam, aniso, xi, rowptr, colidx, vals, b);
    if (kind == OR_FD5_LOGKL || kind == OR_FD7_AXIS)
        return assemble_fd(kind, n, nparam, aniso, xi, rowptr, colidx, vals, b);
    if (kind == OR_Q1_ROT)
        return assemble_q1(n, nparam, aniso, xi, rowptr, colidx, vals, b);
    return -1;
}

/* Parameter-based grouping indicator, Eq. (pb-indicator):
 *   H(xi) = max over the points where the tensor is evaluated (FD face
 *   midpoints, Q1 element centroids) of lambda_max(A) / lambda_min(A).
 * Eigenvalues of the symmetric 2x2 / 3x3 tensor: 2x2 in closed form; the 3-D
 * tensors of OR_FD7_AXIS are diagonal. */
static double ratio2(const double *K)
{
    double t = 0.5 * (K[0] + K[3]);
    double d = sqrt(0.25 * (K[0] - K[3]) * (K[0] - K[3]) + K[1] * K[2]);
    return (t + d) / (t - d);
}

double or_param_indicator(int kind, int n, int nparam, double aniso, const double *xi)
{
    double K[9], x[3], H = 0.0;
    if (kind == OR_Q1_3D_KL || kind == OR_Q1_3D_DISC) {
        /* element centroids; the tensor diag(a, 1, 1) has eigenvalues a, 1, 1 */
        for (int ez = 0; ez <= n; ez++)
            for (int ey = 0; ey <= n; ey++)
                for (int ex = 0; ex <= n; ex++) {
                    x[0] = coord((double)ex + 0.5, n);
                    x[1] = coord((double)ey + 0.5, n);
                    x[2] = coord((double)ez + 0.5, n);
                    or_tensor(kind, nparam, aniso, xi, x, K);
                    double r = K[0] > 1.0 ? K[0] : 1.0 / K[0];
                    if (r > H) H = r;
                }
        return H;
    }
    if (kind == OR_Q1_ROT) {
        for (int ey = 0; ey <= n; ey++)
            for (int ex = 0; ex <= n; ex++) {
                x[0] = coord((double)ex + 0.5, n);
                x[1] = coord((double)ey + 0.5, n);
                or_tensor(kind, nparam, aniso, xi, x, K);
                double r = ratio2(K);
                if (r > H) H = r;
            }
        return H;
    }
    int d = (kind == OR_FD7_AXIS) ? 3 : 2;
    int J = (d == 3) ? n * n * n : n * n;
    for (int p = 0; p < J; p++) {
        int g[3] = {p % n, (p / n) % n, (d == 3) ? p / (n * n) : 0};
        for (int axis = 0; axis < d; axis++)
            for (int dir = -1; dir <= 1; dir += 2) {
                for (int a = 0; a < d; a++) x[a] = coord((double)g[a] + 1.0, n);
                x[axis] = coord((double)g[axis] + 1.0 + 0.5 * dir, n);
                or_tensor(kind, nparam, aniso, xi, x, K);
                double r;
                if (d == 2) {
                    r = ratio2(K);
                } else {
                    double mx = K[0], mn = K[0];
                    if (K[4] > mx) mx = K[4];
                    if (K[8] > mx) mx = K[8];
                    if (K[4] < mn) mn = K[4];
                    if (K[8] < mn) mn = K[8];
                    r = mx / mn;
                }
                if (r > H) H = r;
            }
    }
    return H;
}
