// assemble.cu -- the shared graph and the ensemble assembly kernel (K1).
//
// Eq. (elliptic-SPDE) discretised on the unit square / cube (h = 1/(n+1),
// interior nodes, x fastest).  The values of all S samples of an ensemble are
// written interleaved, vals[e][k][s]: the commuted Kronecker layout of
// Eq. (discrete-comm-kron-sys), one CSR graph for every sample.
//
//   FD (5/7-point, flux form):  (A u)_p = sum_f k_f (u_p - u_nbr) / h^2, with
//       k_f the tensor's diagonal entry for the face axis at the face midpoint;
//       boundary faces add to the diagonal only; f = 1.
//   Q1 (9-point):  element stiffness int grad(phi_a) . K grad(phi_b) of the
//       tensor evaluated at the element centroid, summed over the (up to) four
//       elements shared by the two nodes in lexicographic element order; f = 1
//       gives b = h^2.
//
//   Q1 3-D (27-point, Section 4): element stiffness of the diagonal tensor
//       diag(a, 1, 1) at the element centroid, summed over the (up to) eight
//       elements shared by the two nodes; f = 1 gives b = h^3.
//
// One thread per (ensemble, row, lane); lanes are fastest so every store of a
// nonzero's S values is one contiguous run.
#include "ens_common.cuh"

#include <cmath>
#include <mutex>

namespace ens {

namespace {

__constant__ int kModes2[7][2] = {{1, 1}, {2, 1}, {1, 2}, {2, 2}, {3, 1}, {1, 3}, {3, 2}};
__constant__ int kModes3[4][3] = {{1, 1, 1}, {2, 1, 1}, {1, 2, 1}, {1, 1, 2}};

// ---- pattern ---------------------------------------------------------------
// rowptr by a single-block scan of the per-row neighbour counts.
__global__ void k_rowptr(int kind, int n, int J, int32_t *rowptr)
{
    __shared__ long long part[1024];
    int t = threadIdx.x;
    int chunk = (J + blockDim.x - 1) / blockDim.x;
    int r0 = t * chunk, r1 = min(J, r0 + chunk);
    int cols[27];
    long long s = 0;
    for (int r = r0; r < r1; r++) s += row_neighbours(kind, n, r, cols);
    part[t] = s;
    __syncthreads();
    if (t == 0) {
        long long acc = 0;
        for (int k = 0; k < (int)blockDim.x; k++) {
            long long v = part[k];
            part[k] = acc;
            acc += v;
        }
    }
    __syncthreads();
    long long acc = part[t];
    if (t == 0) rowptr[0] = 0;
    for (int r = r0; r < r1; r++) {
        acc += row_neighbours(kind, n, r, cols);
        rowptr[r + 1] = (int32_t)acc;
    }
}

__global__ void k_colidx(int kind, int n, int J, const int32_t *__restrict__ rowptr,
                         int32_t *__restrict__ colidx)
{
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= J) return;
    int cols[27];
    int c = row_neighbours(kind, n, r, cols);
    int32_t k0 = rowptr[r];
    for (int q = 0; q < c; q++) colidx[k0 + q] = cols[q];
}

// ---- fields ------------------------------------------------------------------
// log a for the 2-D FD field: 0.5 sum_{k=1}^{N-1} xi_k phi_k / k (xi 0-based).
__device__ double fd5_a(const double *xi, int N, double x, double y)
{
    double s = 0.0;
    for (int k = 1; k < N; k++) {
        double phi = dmul(sinpi(kModes2[k - 1][0] * x), sinpi(kModes2[k - 1][1] * y));
        s = dadd(s, dmul(xi[k], phi) / (double)k);
    }
    return exp(dmul(0.5, s));
}

__device__ double fd7_e(const double *xi, double x, double y, double z)
{
    double s = 0.0;
    for (int k = 0; k < 4; k++) {
        double phi = dmul(dmul(sinpi(kModes3[k][0] * x), sinpi(kModes3[k][1] * y)), sinpi(kModes3[k][2] * z));
        s = dadd(s, dmul(xi[2 + k], phi));
    }
    return exp(dmul(0.3, s));
}

template <typename V>
__device__ __forceinline__ void put(V *vals, long long idx, double v) { vals[idx] = (V)v; }

// ---- FD 5-point ------------------------------------------------------------
template <typename V>
__global__ void k_assemble_fd5(int n, int N, double aniso, int S, int E, const double *__restrict__ xi,
                               const int32_t *__restrict__ rowptr, V *__restrict__ vals,
                               double *__restrict__ dinv, double *__restrict__ b, long long nnz, const int32_t *__restrict__ lanes, int nlanes)
{
    const int J = n * n;
    const long long total = lanes ? (long long)nlanes * J : (long long)E * J * S;
    const double den = (double)(n + 1);
    const double ih2 = den * den;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        int s, row, e;
        if (lanes) {  // one refilled lane after another: rows of a lane are consecutive threads
            const int L = lanes[t / J];
            row = (int)(t % J);
            e = L / S;
            s = L % S;
        } else {
            s = (int)(t % S);
            long long er = t / S;
            row = (int)(er % J);
            e = (int)(er / J);
        }
        double x[8];
        const double *xs = xi + ((long long)e * S + s) * N;
        for (int k = 0; k < N; k++) x[k] = xs[k];
        int i = row % n, j = row / n;
        double d2 = exp10(dmul(aniso, x[0]));
        double xc = (double)(i + 1) / den, yc = (double)(j + 1) / den;
        double kS = dmul(fd5_a(x, N, xc, ((double)j + 0.5) / den), d2);
        double kW = fd5_a(x, N, ((double)i + 0.5) / den, yc);
        double kE = fd5_a(x, N, ((double)i + 1.5) / den, yc);
        double kN = dmul(fd5_a(x, N, xc, ((double)j + 1.5) / den), d2);
        double diag = dadd(dadd(dadd(kS, kW), kE), kN);
        long long base = (long long)e * nnz * S + s;
        long long k = rowptr[row];
        if (j > 0) put(vals, base + (k++) * S, -dmul(kS, ih2));
        if (i > 0) put(vals, base + (k++) * S, -dmul(kW, ih2));
        double dv = dmul(diag, ih2);
        put(vals, base + (k++) * S, dv);
        if (i < n - 1) put(vals, base + (k++) * S, -dmul(kE, ih2));
        if (j < n - 1) put(vals, base + (k++) * S, -dmul(kN, ih2));
        long long vi = ((long long)e * J + row) * S + s;
        if (dinv) dinv[vi] = 1.0 / dv;
        if (b) b[vi] = 1.0;
    }
}

// ---- FD 7-point ------------------------------------------------------------
template <typename V>
__global__ void k_assemble_fd7(int n, double aniso, int S, int E, const double *__restrict__ xi,
                               const int32_t *__restrict__ rowptr, V *__restrict__ vals,
                               double *__restrict__ dinv, double *__restrict__ b, long long nnz, const int32_t *__restrict__ lanes, int nlanes)
{
    const int n2 = n * n;
    const int J = n2 * n;
    const long long total = lanes ? (long long)nlanes * J : (long long)E * J * S;
    const double den = (double)(n + 1);
    const double ih2 = den * den;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        int s, row, e;
        if (lanes) {  // one refilled lane after another: rows of a lane are consecutive threads
            const int L = lanes[t / J];
            row = (int)(t % J);
            e = L / S;
            s = L % S;
        } else {
            s = (int)(t % S);
            long long er = t / S;
            row = (int)(er % J);
            e = (int)(er / J);
        }
        double x[6];
        const double *xs = xi + ((long long)e * S + s) * 6;
        for (int k = 0; k < 6; k++) x[k] = xs[k];
        int i = row % n, j = (row / n) % n, l = row / n2;
        double d2 = exp10(dmul(aniso, x[0]));
        double d3 = exp10(dmul(aniso, x[1]));
        double xc = (double)(i + 1) / den, yc = (double)(j + 1) / den, zc = (double)(l + 1) / den;
        double kB = dmul(fd7_e(x, xc, yc, ((double)l + 0.5) / den), d3);
        double kS = dmul(fd7_e(x, xc, ((double)j + 0.5) / den, zc), d2);
        double kW = fd7_e(x, ((double)i + 0.5) / den, yc, zc);
        double kE = fd7_e(x, ((double)i + 1.5) / den, yc, zc);
        double kN = dmul(fd7_e(x, xc, ((double)j + 1.5) / den, zc), d2);
        double kT = dmul(fd7_e(x, xc, yc, ((double)l + 1.5) / den), d3);
        double diag = dadd(dadd(dadd(dadd(dadd(kB, kS), kW), kE), kN), kT);
        long long base = (long long)e * nnz * S + s;
        long long k = rowptr[row];
        if (l > 0) put(vals, base + (k++) * S, -dmul(kB, ih2));
        if (j > 0) put(vals, base + (k++) * S, -dmul(kS, ih2));
        if (i > 0) put(vals, base + (k++) * S, -dmul(kW, ih2));
        double dv = dmul(diag, ih2);
        put(vals, base + (k++) * S, dv);
        if (i < n - 1) put(vals, base + (k++) * S, -dmul(kE, ih2));
        if (j < n - 1) put(vals, base + (k++) * S, -dmul(kN, ih2));
        if (l < n - 1) put(vals, base + (k++) * S, -dmul(kT, ih2));
        long long vi = ((long long)e * J + row) * S + s;
        if (dinv) dinv[vi] = 1.0 / dv;
        if (b) b[vi] = 1.0;
    }
}

// ---- Q1 9-point --------------------------------------------------------------
// Integrals on the reference square of products of the bilinear factors:
// mass-like 1/3 (same end) or 1/6 (opposite ends); derivative signs -1 / +1.
__device__ __forceinline__ double q1_mass(int u, int v) { return u == v ? 1.0 / 3.0 : 1.0 / 6.0; }
__device__ __forceinline__ double q1_sign(int u) { return u ? 1.0 : -1.0; }

template <typename V>
__global__ void k_assemble_q1(int n, double aniso, int S, int E, const double *__restrict__ xi,
                              const int32_t *__restrict__ rowptr, V *__restrict__ vals,
                              double *__restrict__ dinv, double *__restrict__ b, long long nnz, const int32_t *__restrict__ lanes, int nlanes)
{
    const int J = n * n;
    const long long total = lanes ? (long long)nlanes * J : (long long)E * J * S;
    const double den = (double)(n + 1);
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        int s, row, e;
        if (lanes) {  // one refilled lane after another: rows of a lane are consecutive threads
            const int L = lanes[t / J];
            row = (int)(t % J);
            e = L / S;
            s = L % S;
        } else {
            s = (int)(t % S);
            long long er = t / S;
            row = (int)(er % J);
            e = (int)(er / J);
        }
        const double *xs = xi + ((long long)e * S + s) * 4;
        double x0 = xs[0], x1 = xs[1], x2 = xs[2], x3 = xs[3];
        int i = row % n, j = row / n;
        // rotation and axis ratio are per sample; the log-coefficient per element
        double th = dmul(0.25, dadd(1.0, x2));  // theta / pi
        double c = cospi(th), sn = sinpi(th);
        double d2 = exp10(dmul(aniso, x0));
        double t11 = dadd(dmul(c, c), dmul(dmul(sn, sn), d2));
        double t12 = dmul(dmul(c, sn), dsub(1.0, d2));
        double t22 = dadd(dmul(sn, sn), dmul(dmul(c, c), d2));
        // the four elements around node (i+1, j+1) in lexicographic order
        double K0[4], K1[4], K3[4];
#pragma unroll
        for (int q = 0; q < 4; q++) {
            int ex = i + (q & 1), ey = j + (q >> 1);
            double xc = ((double)ex + 0.5) / den, yc = ((double)ey + 0.5) / den;
            double sy = sinpi(yc);
            double phi1 = dmul(sinpi(xc), sy);
            double phi2 = dmul(sinpi(2.0 * xc), sy);
            double a = exp(dmul(0.5, dadd(dmul(x1, phi1), dmul(x3, phi2) / 2.0)));
            K0[q] = dmul(a, t11);
            K1[q] = dmul(a, t12);
            K3[q] = dmul(a, t22);
        }
        long long base = (long long)e * nnz * S + s;
        long long k = rowptr[row];
        double dv = 1.0;
        for (int dj = -1; dj <= 1; dj++)
            for (int di = -1; di <= 1; di++) {
                int ii = i + di, jj = j + dj;
                if (ii < 0 || ii >= n || jj < 0 || jj >= n) continue;
                double v = 0.0;
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    int ex = i + (q & 1), ey = j + (q >> 1);
                    // local coordinates of the row node and the column node
                    int aR = (i + 1) - ex, bR = (j + 1) - ey;
                    int aC = (ii + 1) - ex, bC = (jj + 1) - ey;
                    if (aC < 0 || aC > 1 || bC < 0 || bC > 1) continue;
                    double c1 = q1_sign(aR) * q1_sign(aC) * q1_mass(bR, bC);
                    double c2 = q1_sign(bR) * q1_sign(bC) * q1_mass(aR, aC);
                    double c3 = (q1_sign(aR) * q1_sign(bC) + q1_sign(bR) * q1_sign(aC)) / 4.0;
                    double ke = dadd(dadd(dmul(K0[q], c1), dmul(K3[q], c2)), dmul(K1[q], c3));
                    v = dadd(v, ke);
                }
                if (di == 0 && dj == 0) dv = v;
                put(vals, base + (k++) * S, v);
            }
        long long vi = ((long long)e * J + row) * S + s;
        if (dinv) dinv[vi] = 1.0 / dv;
        if (b) b[vi] = 1.0 / (den * den);
    }
}

// ---- Section 4 field: exponential-covariance KL, Test 1 / Test 2 ---------------
// The covariance sigma0 exp(-||x - x'||_1 / delta) (delta = 1/4, sigma0 =
// sqrt(300)) is a product of 1-D kernels exp(-|s - t| / delta) on [0, 1].  With
// u = s - 1/2 and c = 1/delta the 1-D eigenfunctions are cos(w u) (w tan(w/2) = c)
// and sin(w u) (c tan(w/2) + w = 0), eigenvalue 2c / (w^2 + c^2), squared L2 norm
// 1/2 + sin(w) / (2w) and 1/2 - sin(w) / (2w).  The four largest 3-D products are
// e e e, o e e, e o e, e e o with e, o the first even and odd modes.
struct KLField {
    double we, wo;  // first even / odd roots
    double ie, io;  // 1 / L2 norm of cos(we u), sin(wo u)
    double sl[4];   // sqrt(lambda_k) of the four 3-D modes, sigma0 included
};

// Root of an increasing function on (lo, hi), halving until the bracket stops shrinking.
template <class F> double bisect(F f, double lo, double hi)
{
    for (;;) {
        const double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) return mid;
        if (f(mid) < 0.0)
            lo = mid;
        else
            hi = mid;
    }
}

const KLField &kl_field()
{
    static KLField k;
    static std::once_flag once;
    std::call_once(once, [] {
        const double c = 4.0, pi = 3.14159265358979323846;  // c = 1 / delta
        k.we = bisect([c](double w) { return w * std::tan(0.5 * w) - c; }, 0.0, pi);
        k.wo = bisect([c](double w) { return c * std::tan(0.5 * w) + w; }, pi, 2.0 * pi);
        k.ie = 1.0 / std::sqrt(0.5 + std::sin(k.we) / (2.0 * k.we));
        k.io = 1.0 / std::sqrt(0.5 - std::sin(k.wo) / (2.0 * k.wo));
        const double le = 2.0 * c / (k.we * k.we + c * c), lo = 2.0 * c / (k.wo * k.wo + c * c);
        const double sigma0 = std::sqrt(300.0);
        k.sl[0] = std::sqrt(sigma0 * le * le * le);
        for (int q = 1; q < 4; q++) k.sl[q] = std::sqrt(sigma0 * lo * le * le);
    });
    return k;
}

// ahat(xi) of Test 2 (1 for Test 1); r = ||xi||_2 summed left to right.
__device__ __forceinline__ double q13_ahat(int kind, const double *y)
{
    if (kind != ENS_Q1_3D_DISC) return 1.0;
    const double r = sqrt(dadd(dadd(dadd(dmul(y[0], y[0]), dmul(y[1], y[1])), dmul(y[2], y[2])), dmul(y[3], y[3])));
    const double d = sqrt(3.0);
    return r < d / 4.0 ? 1.0 : (r < d / 2.0 ? 100.0 : 10.0);
}

// a(x, xi) at a point: 0.1 + ahat exp(sum_k sqrt(lambda_k) b_k(x) xi_k).
__device__ __forceinline__ double q13_a(const KLField &f, const double *y, double ahat, double x0, double x1,
                                        double x2)
{
    const double e0 = f.ie * cos(f.we * (x0 - 0.5)), o0 = f.io * sin(f.wo * (x0 - 0.5));
    const double e1 = f.ie * cos(f.we * (x1 - 0.5)), o1 = f.io * sin(f.wo * (x1 - 0.5));
    const double e2 = f.ie * cos(f.we * (x2 - 0.5)), o2 = f.io * sin(f.wo * (x2 - 0.5));
    double s = f.sl[0] * (e0 * e1 * e2) * y[0];
    s += f.sl[1] * (o0 * e1 * e2) * y[1];
    s += f.sl[2] * (e0 * o1 * e2) * y[2];
    s += f.sl[3] * (e0 * e1 * o2) * y[3];
    return 0.1 + ahat * exp(s);
}

// The 1-D mode values at the element centroids (m + 1/2) h, m = 0..n, are
// the only trigonometry of the field: each block tabulates them once in
// shared memory with the expressions of q13_a, so every element coefficient
// is the same number as when evaluated directly.
constexpr int kQ13MaxCells = 401;  // n + 1 for the largest n the problem check admits

__device__ __forceinline__ double q13_a_tab(const KLField &f, const double *te, const double *to, const double *y,
                                            double ahat, int ex, int ey, int ez)
{
    const double e0 = te[ex], o0 = to[ex], e1 = te[ey], o1 = to[ey], e2 = te[ez], o2 = to[ez];
    double s = f.sl[0] * (e0 * e1 * e2) * y[0];
    s += f.sl[1] * (o0 * e1 * e2) * y[1];
    s += f.sl[2] * (e0 * o1 * e2) * y[2];
    s += f.sl[3] * (e0 * e1 * o2) * y[3];
    return 0.1 + ahat * exp(s);
}

template <typename V>
__global__ void k_assemble_q13(int n, int kind, KLField f, int S, int E, const double *__restrict__ xi,
                               const int32_t *__restrict__ rowptr, V *__restrict__ vals, double *__restrict__ dinv,
                               double *__restrict__ b, long long nnz, const int32_t *__restrict__ lanes, int nlanes)
{
    const int n2 = n * n, J = n2 * n;
    const long long total = lanes ? (long long)nlanes * J : (long long)E * J * S;
    const double h = 1.0 / (double)(n + 1);
    __shared__ double te[kQ13MaxCells], to[kQ13MaxCells];
    for (int m = threadIdx.x; m <= n && m < kQ13MaxCells; m += blockDim.x) {
        const double x = ((double)m + 0.5) * h;
        te[m] = f.ie * cos(f.we * (x - 0.5));
        to[m] = f.io * sin(f.wo * (x - 0.5));
    }
    __syncthreads();
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        int s, row, e;
        if (lanes) {
            const int L = lanes[t / J];
            row = (int)(t % J);
            e = L / S;
            s = L % S;
        } else {
            s = (int)(t % S);
            long long er = t / S;
            row = (int)(er % J);
            e = (int)(er / J);
        }
        const double *xs = xi + ((long long)e * S + s) * 4;
        const double y[4] = {xs[0], xs[1], xs[2], xs[3]};
        const double ahat = q13_ahat(kind, y);
        const int i = row % n, j = (row / n) % n, l = row / n2;
        // the eight elements around node (i+1, j+1, l+1), lower corners (i + qx, j + qy, l + qz)
        double a[8];
#pragma unroll
        for (int q = 0; q < 8; q++) {
            const int ex = i + (q & 1), ey = j + ((q >> 1) & 1), ez = l + (q >> 2);
            a[q] = q13_a_tab(f, te, to, y, ahat, ex, ey, ez);
        }
        const long long base = (long long)e * nnz * S + s;
        long long k = rowptr[row];
        double dv = 1.0;
        for (int dl = -1; dl <= 1; dl++)
            for (int dj = -1; dj <= 1; dj++)
                for (int di = -1; di <= 1; di++) {
                    const int ii = i + di, jj = j + dj, ll = l + dl;
                    if (ii < 0 || ii >= n || jj < 0 || jj >= n || ll < 0 || ll >= n) continue;
                    double v = 0.0;
#pragma unroll
                    for (int q = 0; q < 8; q++) {
                        const int ex = i + (q & 1), ey = j + ((q >> 1) & 1), ez = l + (q >> 2);
                        // local coordinates (0/1) of the row node and the column node in the element
                        const int aR = (i + 1) - ex, bR = (j + 1) - ey, cR = (l + 1) - ez;
                        const int aC = (ii + 1) - ex, bC = (jj + 1) - ey, cC = (ll + 1) - ez;
                        if (aC < 0 || aC > 1 || bC < 0 || bC > 1 || cC < 0 || cC > 1) continue;
                        const double dx = q1_sign(aR) * q1_sign(aC) * q1_mass(bR, bC) * q1_mass(cR, cC);
                        const double dy = q1_mass(aR, aC) * q1_sign(bR) * q1_sign(bC) * q1_mass(cR, cC);
                        const double dz = q1_mass(aR, aC) * q1_mass(bR, bC) * q1_sign(cR) * q1_sign(cC);
                        v += h * (a[q] * dx + dy + dz);
                    }
                    if (di == 0 && dj == 0 && dl == 0) dv = v;
                    put(vals, base + (k++) * S, v);
                }
        const long long vi = ((long long)e * J + row) * S + s;
        if (dinv) dinv[vi] = 1.0 / dv;
        if (b) b[vi] = h * h * h;
    }
}

// ---- parameter-based grouping indicator (Section 3.2, Eq. pb-indicator) -------
// H(xi) = max over the points where the tensor is evaluated (FD face
// midpoints, Q1 element centroids) of lambda_max(A) / lambda_min(A).  The
// maximum of positive doubles is taken on their bit patterns with an integer
// atomic, so the result does not depend on the order of the updates.
__device__ __forceinline__ void hmax(double *H, double v)
{
    atomicMax(reinterpret_cast<unsigned long long *>(H), (unsigned long long)__double_as_longlong(v));
}

__global__ void k_indicator(int kind, int n, int N, double aniso, int M, const double *__restrict__ xi_all,
                            double *__restrict__ H, KLField f)
{
    const int m = blockIdx.y;
    const double *xs = xi_all + (size_t)m * N;
    double x[8];
    for (int k = 0; k < N; k++) x[k] = xs[k];
    const double den = (double)(n + 1);
    double best = 0.0;
    if (kind == ENS_Q1_3D_KL || kind == ENS_Q1_3D_DISC) {
        // element centroids; diag(a, 1, 1) has eigenvalues a, 1, 1
        const int m1 = n + 1, ne = m1 * m1 * m1;
        const double ahat = q13_ahat(kind, x);
        for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < ne; q += gridDim.x * blockDim.x) {
            const int ex = q % m1, ey = (q / m1) % m1, ez = q / (m1 * m1);
            const double a = q13_a(f, x, ahat, ((double)ex + 0.5) / den, ((double)ey + 0.5) / den,
                                   ((double)ez + 0.5) / den);
            best = fmax(best, a > 1.0 ? a : 1.0 / a);
        }
    } else if (kind == ENS_Q1_ROT) {
        const int ne = (n + 1) * (n + 1);
        const double th = dmul(0.25, dadd(1.0, x[2]));
        const double c = cospi(th), sn = sinpi(th);
        const double d2 = exp10(dmul(aniso, x[0]));
        const double t11 = c * c + sn * sn * d2, t12 = c * sn * (1.0 - d2), t22 = sn * sn + c * c * d2;
        for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < ne; q += gridDim.x * blockDim.x) {
            const int ex = q % (n + 1), ey = q / (n + 1);
            const double xc = ((double)ex + 0.5) / den, yc = ((double)ey + 0.5) / den;
            const double sy = sinpi(yc);
            const double a = exp(0.5 * (x[1] * (sinpi(xc) * sy) + x[3] * (sinpi(2.0 * xc) * sy) / 2.0));
            const double k0 = a * t11, k1 = a * t12, k3 = a * t22;
            const double t = 0.5 * (k0 + k3);
            const double d = sqrt(0.25 * (k0 - k3) * (k0 - k3) + k1 * k1);
            best = fmax(best, (t + d) / (t - d));
        }
    } else {
        const int d = kind == ENS_FD7_AXIS ? 3 : 2;
        const int J = d == 3 ? n * n * n : n * n;
        const double d2 = exp10(aniso * x[0]);
        const double d3 = d == 3 ? exp10(aniso * x[1]) : 1.0;
        for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < J; p += gridDim.x * blockDim.x) {
            const int g[3] = {p % n, (p / n) % n, d == 3 ? p / (n * n) : 0};
            for (int axis = 0; axis < d; axis++)
                for (int dir = -1; dir <= 1; dir += 2) {
                    double c[3];
                    for (int q = 0; q < d; q++) c[q] = (double)(g[q] + 1) / den;
                    c[axis] = ((double)(g[axis] + 1) + 0.5 * dir) / den;
                    double e = d == 3 ? fd7_e(x, c[0], c[1], c[2]) : fd5_a(x, N, c[0], c[1]);
                    double kx = e, ky = e * d2, kz = e * d3;
                    double mx = fmax(kx, ky), mn = fmin(kx, ky);
                    if (d == 3) {
                        mx = fmax(mx, kz);
                        mn = fmin(mn, kz);
                    }
                    best = fmax(best, mx / mn);
                }
        }
    }
    // block maximum, then one atomic per block
    __shared__ double sh[256];
    sh[threadIdx.x] = best;
    __syncthreads();
    for (int off = blockDim.x / 2; off > 0; off >>= 1) {
        if (threadIdx.x < off) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + off]);
        __syncthreads();
    }
    if (threadIdx.x == 0) hmax(H + m, sh[0]);
}

unsigned grid_for(long long total, int block)
{
    long long g = (total + block - 1) / block;
    const long long cap = 152LL * 64;  // a grid-stride loop beyond ~64 blocks per SM
    return (unsigned)(g < 1 ? 1 : (g > cap ? cap : g));
}

}  // namespace

int problem_check(const ens_problem *p, int *J, int64_t *nnz, std::string *why)
{
    if (!p) { *why = "null problem"; return ENS_EINVAL; }
    long long n = p->n;
    if (n < 2) { *why = "n must be >= 2"; return ENS_EINVAL; }
    switch (p->kind) {
    case ENS_FD5_LOGKL:
        if (p->nparam < 2 || p->nparam > 8) { *why = "FD5 problem needs 2 <= nparam <= 8"; return ENS_EINVAL; }
        if (n > 40000) { *why = "n too large"; return ENS_EINVAL; }
        *J = (int)(n * n);
        *nnz = 5 * n * n - 4 * n;
        break;
    case ENS_Q1_ROT:
        if (p->nparam != 4) { *why = "Q1 problem needs nparam == 4"; return ENS_EINVAL; }
        if (n > 20000) { *why = "n too large"; return ENS_EINVAL; }
        *J = (int)(n * n);
        *nnz = (3 * n - 2) * (3 * n - 2);
        break;
    case ENS_FD7_AXIS:
        if (p->nparam != 6) { *why = "FD7 problem needs nparam == 6"; return ENS_EINVAL; }
        if (n > 1000) { *why = "n too large"; return ENS_EINVAL; }
        *J = (int)(n * n * n);
        *nnz = 7 * n * n * n - 6 * n * n;
        break;
    case ENS_Q1_3D_KL:
    case ENS_Q1_3D_DISC:
        if (p->nparam != 4) { *why = "3-D Q1 problem needs nparam == 4"; return ENS_EINVAL; }
        if (n > 400) { *why = "n too large"; return ENS_EINVAL; }
        *J = (int)(n * n * n);
        *nnz = (3 * n - 2) * (3 * n - 2) * (3 * n - 2);
        break;
    default:
        *why = "unknown problem kind";
        return ENS_EINVAL;
    }
    if (*nnz >= (1LL << 31)) { *why = "nnz does not fit int32 column indices"; return ENS_EINVAL; }
    return ENS_OK;
}

}  // namespace ens

using namespace ens;

extern "C" int ens_problem_size(const ens_problem *p, int *J, int64_t *nnz)
{
    std::string why;
    if (!J || !nnz) return ENS_EINVAL;
    return problem_check(p, J, nnz, &why);
}

extern "C" int ens_pattern(ens_handle h, const ens_problem *p, int32_t *rowptr, int32_t *colidx,
                           void *stream)
{
    if (!h) return ENS_EINVAL;
    int J;
    int64_t nnz;
    std::string why;
    int rc = problem_check(p, &J, &nnz, &why);
    if (rc) return set_error(h, rc, "ens_pattern: " + why);
    if (!rowptr || !colidx) return set_error(h, ENS_EINVAL, "ens_pattern: null output");
    cudaStream_t st = (cudaStream_t)stream;
    k_rowptr<<<1, 1024, 0, st>>>(p->kind, p->n, J, rowptr);
    ENS_LAUNCH_CHECK(h, "ens_pattern: rowptr kernel");
    k_colidx<<<(J + 255) / 256, 256, 0, st>>>(p->kind, p->n, J, rowptr, colidx);
    ENS_LAUNCH_CHECK(h, "ens_pattern: colidx kernel");
    return ENS_OK;
}

namespace ens {
int assemble_lanes(ens_ctx *h, const ens_problem *p, int S, int E, const double *xi, const int32_t *rowptr,
                   void *vals, int vals_f32, double *dinv, double *b, const int32_t *lanes, int nlanes,
                   cudaStream_t st)
{
    int J;
    int64_t nnz;
    std::string why;
    int rc = problem_check(p, &J, &nnz, &why);
    if (rc) return set_error(h, rc, "ens_assemble: " + why);
    if (lanes && nlanes <= 0) return ENS_OK;
    long long total = lanes ? (long long)nlanes * J : (long long)E * J * S;
    unsigned grid = grid_for(total, 256);
    switch (p->kind) {
    case ENS_FD5_LOGKL:
        if (vals_f32)
            k_assemble_fd5<float><<<grid, 256, 0, st>>>(p->n, p->nparam, p->aniso, S, E, xi, rowptr, (float *)vals, dinv, b, nnz, lanes, nlanes);
        else
            k_assemble_fd5<double><<<grid, 256, 0, st>>>(p->n, p->nparam, p->aniso, S, E, xi, rowptr, (double *)vals, dinv, b, nnz, lanes, nlanes);
        break;
    case ENS_Q1_ROT:
        if (vals_f32)
            k_assemble_q1<float><<<grid, 256, 0, st>>>(p->n, p->aniso, S, E, xi, rowptr, (float *)vals, dinv, b, nnz, lanes, nlanes);
        else
            k_assemble_q1<double><<<grid, 256, 0, st>>>(p->n, p->aniso, S, E, xi, rowptr, (double *)vals, dinv, b, nnz, lanes, nlanes);
        break;
    case ENS_Q1_3D_KL:
    case ENS_Q1_3D_DISC:
        if (vals_f32)
            k_assemble_q13<float><<<grid, 256, 0, st>>>(p->n, p->kind, kl_field(), S, E, xi, rowptr, (float *)vals, dinv, b, nnz, lanes, nlanes);
        else
            k_assemble_q13<double><<<grid, 256, 0, st>>>(p->n, p->kind, kl_field(), S, E, xi, rowptr, (double *)vals, dinv, b, nnz, lanes, nlanes);
        break;
    default:
        if (vals_f32)
            k_assemble_fd7<float><<<grid, 256, 0, st>>>(p->n, p->aniso, S, E, xi, rowptr, (float *)vals, dinv, b, nnz, lanes, nlanes);
        else
            k_assemble_fd7<double><<<grid, 256, 0, st>>>(p->n, p->aniso, S, E, xi, rowptr, (double *)vals, dinv, b, nnz, lanes, nlanes);
        break;
    }
    ENS_LAUNCH_CHECK(h, "ens_assemble: kernel launch");
    return ENS_OK;
}

int pattern_into(ens_ctx *h, const ens_problem *p, int32_t *rowptr, int32_t *colidx, cudaStream_t st)
{
    int J;
    int64_t nnz;
    std::string why;
    int rc = problem_check(p, &J, &nnz, &why);
    if (rc) return set_error(h, rc, "pattern: " + why);
    k_rowptr<<<1, 1024, 0, st>>>(p->kind, p->n, J, rowptr);
    ENS_LAUNCH_CHECK(h, "pattern: rowptr kernel");
    k_colidx<<<(J + 255) / 256, 256, 0, st>>>(p->kind, p->n, J, rowptr, colidx);
    ENS_LAUNCH_CHECK(h, "pattern: colidx kernel");
    return ENS_OK;
}
}  // namespace ens

extern "C" int ens_assemble(ens_handle h, const ens_problem *p, int S, int E, const double *xi,
                            const int32_t *rowptr, const int32_t *colidx, void *vals, int vals_f32,
                            double *dinv, double *b, void *stream)
{
    if (!h) return ENS_EINVAL;
    int J;
    int64_t nnz;
    std::string why;
    int rc = problem_check(p, &J, &nnz, &why);
    if (rc) return set_error(h, rc, "ens_assemble: " + why);
    if (!lane_count_ok(S)) return set_error(h, ENS_EINVAL, "ens_assemble: S must be a power of two <= 64");
    if (E < 0) return set_error(h, ENS_EINVAL, "ens_assemble: E < 0");
    if (E == 0) return ENS_OK;
    if (!xi || !rowptr || !colidx || !vals) return set_error(h, ENS_EINVAL, "ens_assemble: null pointer");
    return assemble_lanes(h, p, S, E, xi, rowptr, vals, vals_f32, dinv, b, nullptr, 0, (cudaStream_t)stream);
}

extern "C" int ens_param_indicator(ens_handle h, const ens_problem *p, int M, const double *xi, double *H,
                                   void *stream)
{
    if (!h) return ENS_EINVAL;
    int J;
    int64_t nnz;
    std::string why;
    int rc = problem_check(p, &J, &nnz, &why);
    if (rc) return set_error(h, rc, "ens_param_indicator: " + why);
    if (M < 0 || M > 65535) return set_error(h, ENS_EINVAL, "ens_param_indicator: M must be in 0..65535");
    if (M == 0) return ENS_OK;
    if (!xi || !H) return set_error(h, ENS_EINVAL, "ens_param_indicator: null pointer");
    cudaStream_t st = (cudaStream_t)stream;
    ENS_CUDA_CHECK(h, cudaMemsetAsync(H, 0, (size_t)M * sizeof(double), st));
    const long long m1 = p->n + 1;
    const long long pts = p->kind == ENS_Q1_ROT ? m1 * m1
                          : (p->kind == ENS_Q1_3D_KL || p->kind == ENS_Q1_3D_DISC ? m1 * m1 * m1 : (long long)J);
    unsigned bx = (unsigned)((pts + 255) / 256);
    if (bx > 64) bx = 64;
    dim3 grid(bx, M);
    k_indicator<<<grid, 256, 0, st>>>(p->kind, p->n, p->nparam, p->aniso, M, xi, H, kl_field());
    ENS_LAUNCH_CHECK(h, "ens_param_indicator");
    return ENS_OK;
}
