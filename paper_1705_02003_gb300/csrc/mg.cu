// mg.cu -- ensemble multigrid V-cycle preconditioner and multigrid-preconditioned
// CG for the trilinear problems (ENS_Q1_3D_KL / ENS_Q1_3D_DISC).
//
// Section 4 preconditions CG with a multigrid hierarchy whose levels are
// smoothed by a second-order Chebyshev polynomial and whose coarsest level is
// solved directly; like the rest of that solver it is instantiated on the
// ensemble scalar, so every level stores S samples per nonzero and every
// operation is per sample.  On the structured (n + 1)^3-cell mesh this
// library uses the nested trilinear hierarchy (the mesh is structured, so the
// aggregates of an algebraic method are known in advance):
//   - levels n_0 = n, n_{l+1} = (n_l - 1) / 2 down to 3 (n = 2^k - 1, k >= 2);
//     coarse node c sits on fine node 2c + 1;
//   - P = trilinear interpolation (weights 1, 1/2 per axis), R = P^T;
//   - coarse operators A_{l+1} = P^T A_l P (Galerkin), per sample;
//   - smoother: the degree-2 Chebyshev semi-iteration on D^-1 A over
//     [lambda_max / 30, lambda_max], lambda_max the per-sample Gershgorin bound
//     max_i sum_j |a_ij| / a_ii;
//   - coarsest level (27 unknowns): per-sample dense Cholesky, applied as the
//     explicit inverse built from it;
//   - one V-cycle per CG iteration (pre-smooth from 0, restrict, recurse,
//     prolong-add, post-smooth).
// The setup (Galerkin products, Gershgorin bounds, Cholesky) follows the order
// of the textbook sums and rounds each sum on its own (the Galerkin products by
// the power-of-two weights are exact), so it reproduces a plain host
// computation bit for bit; the V-cycle itself uses fused multiply-adds.  With
// `mixed` the hierarchy is also rounded once to float and the V-cycle runs in
// float (the same kernels instantiated on float); CG stays in double.  Each
// lane's input is scaled by a power of two that brings its largest entry
// below 2 before the rounding to float, and the result is scaled back: exact,
// and the V-cycle commutes with it, so lanes of any magnitude FP64 holds
// stay inside float's range.
//
// Layout: every vector of level l is [E][J_l][S] f64, every matrix
// [E][nnz_l][S] f64 (level 0 is the caller's), the coarsest operator's
// inverse [E][729][S].  Per-sample scalars are [E][S].
#include "ens_common.cuh"

#include <algorithm>
#include <cmath>

namespace ens {
namespace {

constexpr int kMgMaxLev = 8;
constexpr int kRedRows = 256;   // rows per block of the CG reduction kernels
constexpr double kRatio = 30.0;
constexpr int kCoarseJ = 27;
constexpr int kInv = kCoarseJ * kCoarseJ;

struct MgLevel {
    int n = 0, J = 0;
    int64_t nnz = 0;
    int32_t *rp = nullptr, *ci = nullptr;  // coarse levels' graph
    double *vals = nullptr;                // coarse levels' values
    double *dinv = nullptr;
    double *coef = nullptr;                // [E][S][4]: 1/theta, c1, c2, -
    unsigned long long *lmax = nullptr;    // [E][S] bits of the Gershgorin bound
    double *rhs = nullptr, *e = nullptr, *t = nullptr, *d = nullptr, *res = nullptr;
    // the float copy of the level for the mixed-precision V-cycle (level 0 included)
    float *vals32 = nullptr, *dinv32 = nullptr, *coef32 = nullptr;
    float *rhs32 = nullptr, *e32 = nullptr, *t32 = nullptr, *d32 = nullptr, *res32 = nullptr;
};

struct MgWork {
    int L = 0;
    MgLevel lv[kMgMaxLev];
    double *cinv = nullptr;  // [E][27 * 27][S]: inverse of the coarsest operator
    float *cinv32 = nullptr;
    unsigned long long *rmax = nullptr;  // [E][S] per-lane largest |r| of the float V-cycle's input
    int mixed = 0;           // the V-cycle runs in float on a float copy of the hierarchy
    int *bad = nullptr;      // [E][S]
    // CG state
    double *r = nullptr, *p = nullptr, *q = nullptr, *z = nullptr;
    double *part0 = nullptr, *part1 = nullptr;  // [E][nblk][S]
    double *rz = nullptr, *rr = nullptr, *alpha = nullptr, *beta = nullptr, *bnorm = nullptr;
    int *k = nullptr, *live = nullptr, *ens_live = nullptr, *live_total = nullptr;
    int nblk = 0;
    size_t bytes = 0;
};

bool mg_levels(int n, int *ns, int *L)
{
    if (n < 3) return false;
    for (int m = n + 1; m > 1; m >>= 1)
        if (m & 1) return false;
    int k = 0;
    ns[k++] = n;
    while (ns[k - 1] > 3) {
        if (k >= kMgMaxLev) return false;
        ns[k] = (ns[k - 1] - 1) / 2;
        k++;
    }
    *L = k;
    return true;
}

// Lay the workspace out from `base` (nullptr: only count the bytes).
bool mg_layout(const ens_problem *p, int S, int E, int mixed, char *base, MgWork *w)
{
    int ns[kMgMaxLev], L;
    if (!mg_levels(p->n, ns, &L)) return false;
    size_t off = 0;
    auto take = [&](size_t bytes) -> char * {
        char *ptr = base ? base + off : nullptr;
        off += align256(bytes);
        return ptr;
    };
    const size_t ES = (size_t)E * S;
    w->L = L;
    for (int l = 0; l < L; l++) {
        MgLevel &v = w->lv[l];
        v.n = ns[l];
        v.J = ns[l] * ns[l] * ns[l];
        v.nnz = (int64_t)(3 * ns[l] - 2) * (3 * ns[l] - 2) * (3 * ns[l] - 2);
        const size_t vec = ES * v.J * sizeof(double);
        if (l > 0) {
            v.rp = (int32_t *)take(sizeof(int32_t) * (v.J + 1));
            v.ci = (int32_t *)take(sizeof(int32_t) * v.nnz);
            v.vals = (double *)take(ES * v.nnz * sizeof(double));
            v.rhs = (double *)take(vec);
        }
        v.dinv = (double *)take(vec);
        v.coef = (double *)take(ES * 4 * sizeof(double));
        v.lmax = (unsigned long long *)take(ES * sizeof(unsigned long long));
        v.e = (double *)take(vec);
        if (l < L - 1) {
            v.t = (double *)take(vec);
            v.d = (double *)take(vec);
            v.res = (double *)take(vec);
        }
    }
    w->cinv = (double *)take(ES * kInv * sizeof(double));
    w->mixed = mixed;
    if (mixed) {
        for (int l = 0; l < L; l++) {
            MgLevel &v = w->lv[l];
            const size_t vec = ES * v.J * sizeof(float);
            v.vals32 = (float *)take(ES * v.nnz * sizeof(float));
            v.dinv32 = (float *)take(vec);
            v.coef32 = (float *)take(ES * 4 * sizeof(float));
            v.rhs32 = (float *)take(vec);
            v.e32 = (float *)take(vec);
            if (l < L - 1) {
                v.t32 = (float *)take(vec);
                v.d32 = (float *)take(vec);
                v.res32 = (float *)take(vec);
            }
        }
        w->cinv32 = (float *)take(ES * kInv * sizeof(float));
        w->rmax = (unsigned long long *)take(ES * sizeof(unsigned long long));
    }
    w->bad = (int *)take(ES * sizeof(int));
    const int J = w->lv[0].J;
    const size_t vec0 = ES * J * sizeof(double);
    w->r = (double *)take(vec0);
    w->p = (double *)take(vec0);
    w->q = (double *)take(vec0);
    w->z = w->lv[0].e;
    w->nblk = (J + kRedRows - 1) / kRedRows;
    w->part0 = (double *)take(ES * w->nblk * sizeof(double));
    w->part1 = (double *)take(ES * w->nblk * sizeof(double));
    w->rz = (double *)take(ES * sizeof(double));
    w->rr = (double *)take(ES * sizeof(double));
    w->alpha = (double *)take(ES * sizeof(double));
    w->beta = (double *)take(ES * sizeof(double));
    w->bnorm = (double *)take(ES * sizeof(double));
    w->k = (int *)take(ES * sizeof(int));
    w->live = (int *)take(ES * sizeof(int));
    w->ens_live = (int *)take((size_t)E * sizeof(int));
    w->live_total = (int *)take(sizeof(int));
    w->bytes = off;
    return true;
}

// ---- setup kernels (one row-lane per thread: lane t % S, row blockIdx.x G + t / S) ----

__device__ __forceinline__ void row_lane(int S, int *s, int *i)
{
    const int G = blockDim.x / S;
    *s = threadIdx.x % S;
    *i = blockIdx.x * G + threadIdx.x / S;
}

// D^-1 and the Gershgorin ratio sum_j |a_ij| / a_ii of every row-lane; the
// per-lane maximum by an atomic maximum on the bits (positive doubles order
// like their bit patterns); a ratio that is not finite and positive marks the
// lane unusable.
__global__ void k_mg_diag(int J, int S, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                          const double *__restrict__ vals, double *__restrict__ dinv,
                          unsigned long long *__restrict__ lmax, int *__restrict__ bad)
{
    int s, i;
    row_lane(S, &s, &i);
    const int e = blockIdx.y;
    if (i >= J) return;
    const int64_t nnz = rp[J];
    const double *v = vals + (size_t)e * nnz * S + s;
    double sum = 0.0, d = 0.0;
    for (int k = rp[i]; k < rp[i + 1]; k++) {
        const double a = v[(size_t)k * S];
        sum = dadd(sum, fabs(a));
        if (ci[k] == i) d = a;
    }
    const double ratio = __ddiv_rn(sum, d);
    dinv[((size_t)e * J + i) * S + s] = __ddiv_rn(1.0, d);
    if (!(ratio > 0.0) || !isfinite(ratio))
        bad[e * S + s] = 1;
    else
        atomicMax(lmax + e * S + s, (unsigned long long)__double_as_longlong(ratio));
}

// Chebyshev coefficients of each lane from its bound: 1/theta, and c1, c2 of the second step.
__global__ void k_mg_coef(int ES, const unsigned long long *__restrict__ lmax, double *__restrict__ coef)
{
    const int L = blockIdx.x * blockDim.x + threadIdx.x;
    if (L >= ES) return;
    const double lm = __longlong_as_double((long long)lmax[L]);
    const double lmin = lm / kRatio;
    const double theta = (lm + lmin) / 2.0, delta = (lm - lmin) / 2.0;
    const double sigma = theta / delta;
    const double rho0 = 1.0 / sigma;
    const double rho1 = 1.0 / (2.0 * sigma - rho0);
    coef[4 * L + 0] = 1.0 / theta;
    coef[4 * L + 1] = rho1 * rho0;
    coef[4 * L + 2] = 2.0 * rho1 / delta;
    coef[4 * L + 3] = 0.0;
}

// Per-axis coarse parents of fine coordinate f: (index, weight), ascending.
__device__ __forceinline__ int parents(int f, int nc, int *c, double *w)
{
    int m = 0;
    if (f & 1) {
        c[0] = (f - 1) >> 1;
        w[0] = 1.0;
        m = 1;
    } else {
        const int a = (f >> 1) - 1, b = f >> 1;
        if (a >= 0) { c[m] = a; w[m] = 0.5; m++; }
        if (b < nc) { c[m] = b; w[m] = 0.5; m++; }
    }
    return m;
}

__device__ __forceinline__ double w1(int f, int c)
{
    const int d = f - (2 * c + 1);
    return d == 0 ? 1.0 : ((d == 1 || d == -1) ? 0.5 : 0.0);
}

// 2^-m as a double (0 <= m <= 6), built from its exponent bits.
__device__ __forceinline__ double pow2_neg(int m) { return __longlong_as_double((long long)(1023 - m) << 52); }

// A_c = P^T A_f P, one thread per coarse entry (I, J) and lane: its
// contributions w_i w_j a_ij are added in the order of the triple sum (fine
// nodes i of I ascending, then the columns j of row i ascending, restricted to
// the children of J).  w_i w_j = 2^-m is exact, and so is its product with a
// (normal) value, so a fused multiply-add rounds exactly what the textbook
// triple sum with a separate product and sum rounds: the entry matches it bit
// for bit.  (The product as a separate FP64 multiply, or as an exponent shift
// with a rare-case branch, ran at half this kernel's speed or less.)  A row's columns (fine or coarse) are its 3x3x3
// neighbourhood clipped to the grid, in lexicographic order, so the position
// of a column in its row follows from the clipped box.
__global__ void k_mg_galerkin(int nf, int nc, int S, const int32_t *__restrict__ rpf, const double *__restrict__ vf,
                              const int32_t *__restrict__ rpc, double *__restrict__ vc)
{
    int s, q;
    row_lane(S, &s, &q);  // q = 27 I + slot
    const int e = blockIdx.y;
    const int Jc = nc * nc * nc, Jf = nf * nf * nf;
    if (q >= 27 * Jc) return;
    const int I = q / 27, slot = q % 27;
    const int I0 = I % nc, I1 = (I / nc) % nc, I2 = I / (nc * nc);
    const int J0 = I0 + slot % 3 - 1, J1 = I1 + (slot / 3) % 3 - 1, J2 = I2 + slot / 9 - 1;
    if (J0 < 0 || J0 >= nc || J1 < 0 || J1 >= nc || J2 < 0 || J2 >= nc) return;
    const int64_t nnzf = rpf[Jf], nnzc = rpc[Jc];
    const double *v = vf + (size_t)e * nnzf * S + s;
    double acc = 0.0;
    for (int i2 = 2 * I2; i2 <= 2 * I2 + 2; i2++)
        for (int i1 = 2 * I1; i1 <= 2 * I1 + 2; i1++)
            for (int i0 = 2 * I0; i0 <= 2 * I0 + 2; i0++) {
                // row box of i and the children box of J, per axis
                const int rb0 = max(i0 - 1, 0), rb1 = max(i1 - 1, 0), rb2 = max(i2 - 1, 0);
                const int rn0 = min(i0 + 1, nf - 1) - rb0 + 1, rn1 = min(i1 + 1, nf - 1) - rb1 + 1;
                const int lo0 = max(rb0, 2 * J0), hi0 = min(i0 + 1, min(nf - 1, 2 * J0 + 2));
                const int lo1 = max(rb1, 2 * J1), hi1 = min(i1 + 1, min(nf - 1, 2 * J1 + 2));
                const int lo2 = max(rb2, 2 * J2), hi2 = min(i2 + 1, min(nf - 1, 2 * J2 + 2));
                if (lo0 > hi0 || lo1 > hi1 || lo2 > hi2) continue;
                const int i = i0 + nf * (i1 + nf * i2);
                // half weights of i (w_i = 2^-mi) and of the j below (w_j = 2^-mj)
                const int mi = (i0 != 2 * I0 + 1) + (i1 != 2 * I1 + 1) + (i2 != 2 * I2 + 1);
                const int base = rpf[i];
                for (int j2 = lo2; j2 <= hi2; j2++)
                    for (int j1 = lo1; j1 <= hi1; j1++)
                        for (int j0 = lo0; j0 <= hi0; j0++) {
                            const int k = base + ((j2 - rb2) * rn1 + (j1 - rb1)) * rn0 + (j0 - rb0);
                            const int mj = (j0 != 2 * J0 + 1) + (j1 != 2 * J1 + 1) + (j2 != 2 * J2 + 1);
                            acc = fma(v[(size_t)k * S], pow2_neg(mi + mj), acc);
                        }
            }
    // the entry's position in coarse row I
    const int cb0 = max(I0 - 1, 0), cb1 = max(I1 - 1, 0), cb2 = max(I2 - 1, 0);
    const int cn0 = min(I0 + 1, nc - 1) - cb0 + 1, cn1 = min(I1 + 1, nc - 1) - cb1 + 1;
    const int kc = rpc[I] + ((J2 - cb2) * cn1 + (J1 - cb1)) * cn0 + (J0 - cb0);
    vc[((size_t)e * nnzc + kc) * S + s] = acc;
}

// The coarsest level (27 unknowns), one block per lane: Cholesky A = L L^T in
// shared memory by one thread in the textbook order (each product, difference,
// quotient and root rounded on its own), then thread j < 27 solves
// L L^T x = e_j for column j of A^-1.  The V-cycle's coarsest solve is then a
// 27 x 27 product.
__global__ void k_mg_chol(int S, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                          const double *__restrict__ vals, double *__restrict__ cinv, int *__restrict__ bad)
{
    __shared__ double A[kInv];
    __shared__ double Lf[kInv];
    __shared__ int fail;
    const int s = blockIdx.x, e = blockIdx.y;
    const int64_t nnz = rp[kCoarseJ];
    for (int q = threadIdx.x; q < kInv; q += blockDim.x) {
        A[q] = 0.0;
        Lf[q] = 0.0;
    }
    if (threadIdx.x == 0) fail = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < kCoarseJ; i += blockDim.x)
        for (int k = rp[i]; k < rp[i + 1]; k++) A[i * kCoarseJ + ci[k]] = vals[((size_t)e * nnz + k) * S + s];
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int j = 0; j < kCoarseJ && !fail; j++) {
            double sj = A[j * kCoarseJ + j];
            for (int k = 0; k < j; k++) sj = dsub(sj, dmul(Lf[j * kCoarseJ + k], Lf[j * kCoarseJ + k]));
            if (!(sj > 0.0)) {
                fail = 1;
                break;
            }
            const double d = __dsqrt_rn(sj);
            Lf[j * kCoarseJ + j] = d;
            for (int i = j + 1; i < kCoarseJ; i++) {
                double t = A[i * kCoarseJ + j];
                for (int k = 0; k < j; k++) t = dsub(t, dmul(Lf[i * kCoarseJ + k], Lf[j * kCoarseJ + k]));
                Lf[i * kCoarseJ + j] = __ddiv_rn(t, d);
            }
        }
        if (fail) bad[e * S + s] = 1;
    }
    __syncthreads();
    const int j = threadIdx.x;
    if (j < kCoarseJ) {
        double y[kCoarseJ];
#pragma unroll 1
        for (int i = 0; i < kCoarseJ; i++) {
            double acc = i == j ? 1.0 : 0.0;
#pragma unroll 1
            for (int k = 0; k < i; k++) acc = fma(-Lf[i * kCoarseJ + k], y[k], acc);
            y[i] = acc / Lf[i * kCoarseJ + i];
        }
#pragma unroll 1
        for (int i = kCoarseJ - 1; i >= 0; i--) {
            double acc = y[i];
#pragma unroll 1
            for (int k = i + 1; k < kCoarseJ; k++) acc = fma(-Lf[k * kCoarseJ + i], y[k], acc);
            y[i] = acc / Lf[i * kCoarseJ + i];
        }
#pragma unroll 1
        for (int i = 0; i < kCoarseJ; i++) cinv[((size_t)e * kInv + i * kCoarseJ + j) * S + s] = y[i];
    }
}

// ---- V-cycle kernels ----------------------------------------------------------

__device__ __forceinline__ bool ens_skip(const int *ens_live, int e) { return ens_live && ens_live[e] == 0; }

// The V-cycle kernels are templates on the value type T of the hierarchy's
// values, diagonals, coefficients and vectors: double for the FP64 V-cycle,
// float for the mixed-precision one (CG itself stays in double).

// One row-lane of A x, nonzeros in order.  (Reading the row in chunks of nine,
// all loads of a chunk issued before its multiply-adds, took 80 registers and
// three resident blocks per SM instead of eight and made the 31^3 solve 1.6-2x
// slower, measured: here more warps hide the latency better than more loads
// in flight per thread.)
template <typename T>
__device__ __forceinline__ T row_dot(const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                     const T *__restrict__ v, const T *__restrict__ x, int i, int S)
{
    T acc = T(0);
    for (int k = rp[i]; k < rp[i + 1]; k++) acc = fma(v[(size_t)k * S], x[(size_t)ci[k] * S], acc);
    return acc;
}

// First Chebyshev step: d = D^-1 (b - A x) / theta, x_out = x + d (x = 0 when x_in is null).
template <typename T>
__global__ void k_mg_cheb1(int J, int S, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                           const T *__restrict__ vals, const T *__restrict__ dinv, const T *__restrict__ coef,
                           const T *__restrict__ b, const T *__restrict__ x_in, T *__restrict__ d,
                           T *__restrict__ x_out, const int *__restrict__ ens_live)
{
    int s, i;
    row_lane(S, &s, &i);
    const int e = blockIdx.y;
    if (i >= J || ens_skip(ens_live, e)) return;
    const int64_t nnz = rp[J];
    const size_t vb = (size_t)e * J * S + s, o = vb + (size_t)i * S;
    T x0 = T(0), res = b[o];
    if (x_in) {
        res -= row_dot<T>(rp, ci, vals + (size_t)e * nnz * S + s, x_in + vb, i, S);
        x0 = x_in[o];
    }
    const T dd = dinv[o] * res * coef[4 * (e * S + s)];
    d[o] = dd;
    x_out[o] = x0 + dd;
}

// Second Chebyshev step: d = c1 d + c2 D^-1 (b - A x), x_out = x + d.
template <typename T>
__global__ void k_mg_cheb2(int J, int S, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                           const T *__restrict__ vals, const T *__restrict__ dinv, const T *__restrict__ coef,
                           const T *__restrict__ b, const T *__restrict__ x_in, T *__restrict__ d,
                           T *__restrict__ x_out, const int *__restrict__ ens_live)
{
    int s, i;
    row_lane(S, &s, &i);
    const int e = blockIdx.y;
    if (i >= J || ens_skip(ens_live, e)) return;
    const int64_t nnz = rp[J];
    const size_t vb = (size_t)e * J * S + s, o = vb + (size_t)i * S;
    const T res = b[o] - row_dot<T>(rp, ci, vals + (size_t)e * nnz * S + s, x_in + vb, i, S);
    const T *c = coef + 4 * (e * S + s);
    const T dd = fma(c[1], d[o], c[2] * (dinv[o] * res));
    d[o] = dd;
    x_out[o] = x_in[o] + dd;
}

// res = b - A x
template <typename T>
__global__ void k_mg_resid(int J, int S, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                           const T *__restrict__ vals, const T *__restrict__ b, const T *__restrict__ x,
                           T *__restrict__ res, const int *__restrict__ ens_live)
{
    int s, i;
    row_lane(S, &s, &i);
    const int e = blockIdx.y;
    if (i >= J || ens_skip(ens_live, e)) return;
    const int64_t nnz = rp[J];
    const size_t vb = (size_t)e * J * S + s, o = vb + (size_t)i * S;
    res[o] = b[o] - row_dot<T>(rp, ci, vals + (size_t)e * nnz * S + s, x + vb, i, S);
}

// rc = P^T rf: the 27 fine nodes of each coarse node, ascending.
template <typename T>
__global__ void k_mg_restrict(int nf, int nc, int S, const T *__restrict__ rf, T *__restrict__ rc,
                              const int *__restrict__ ens_live)
{
    int s, I;
    row_lane(S, &s, &I);
    const int e = blockIdx.y;
    const int Jc = nc * nc * nc, Jf = nf * nf * nf;
    if (I >= Jc || ens_skip(ens_live, e)) return;
    const int I0 = I % nc, I1 = (I / nc) % nc, I2 = I / (nc * nc);
    const T *r = rf + (size_t)e * Jf * S + s;
    T acc = T(0);
    for (int i2 = 2 * I2; i2 <= 2 * I2 + 2; i2++)
        for (int i1 = 2 * I1; i1 <= 2 * I1 + 2; i1++)
            for (int i0 = 2 * I0; i0 <= 2 * I0 + 2; i0++) {
                const T w = (T)(w1(i0, I0) * w1(i1, I1) * w1(i2, I2));
                acc = fma(w, r[(size_t)(i0 + nf * (i1 + nf * i2)) * S], acc);
            }
    rc[((size_t)e * Jc + I) * S + s] = acc;
}

// ef += P ec: the (up to 8) coarse parents of each fine node, ascending.
template <typename T>
__global__ void k_mg_prolong_add(int nf, int nc, int S, const T *__restrict__ ec, T *__restrict__ ef,
                                 const int *__restrict__ ens_live)
{
    int s, i;
    row_lane(S, &s, &i);
    const int e = blockIdx.y;
    const int Jc = nc * nc * nc, Jf = nf * nf * nf;
    if (i >= Jf || ens_skip(ens_live, e)) return;
    const int f0 = i % nf, f1 = (i / nf) % nf, f2 = i / (nf * nf);
    int c0[2], c1[2], c2[2];
    double u0[2], u1[2], u2[2];
    const int m0 = parents(f0, nc, c0, u0), m1 = parents(f1, nc, c1, u1), m2 = parents(f2, nc, c2, u2);
    const T *c = ec + (size_t)e * Jc * S + s;
    T acc = T(0);
    for (int b2 = 0; b2 < m2; b2++)
        for (int b1 = 0; b1 < m1; b1++)
            for (int b0 = 0; b0 < m0; b0++)
                acc = fma((T)(u0[b0] * u1[b1] * u2[b2]), c[(size_t)(c0[b0] + nc * (c1[b1] + nc * c2[b2])) * S], acc);
    const size_t o = ((size_t)e * Jf + i) * S + s;
    ef[o] = ef[o] + acc;
}

// Coarsest level: e = A^-1 r, one row-lane per thread (27 products, ascending).
template <typename T>
__global__ void k_mg_coarse_solve(int S, const T *__restrict__ cinv, const T *__restrict__ r, T *__restrict__ x,
                                  const int *__restrict__ ens_live)
{
    int s, i;
    row_lane(S, &s, &i);
    const int e = blockIdx.y;
    if (i >= kCoarseJ || ens_skip(ens_live, e)) return;
    const T *a = cinv + ((size_t)e * kInv + i * kCoarseJ) * S + s;
    const T *rv = r + (size_t)e * kCoarseJ * S + s;
    T acc = T(0);
#pragma unroll
    for (int j = 0; j < kCoarseJ; j++) acc = fma(a[(size_t)j * S], rv[(size_t)j * S], acc);
    x[((size_t)e * kCoarseJ + i) * S + s] = acc;
}

// Element-wise conversions between the CG's double vectors and the float
// V-cycle (and of the hierarchy at setup), in ensemble order; skipped
// ensembles (ens_live[e] == 0, with per_ens elements each) are left alone.
template <typename A, typename B>
__global__ void k_mg_convert(size_t n, size_t per_ens, const A *__restrict__ src, B *__restrict__ dst,
                             const int *__restrict__ ens_live)
{
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
        if (ens_live && ens_live[t / per_ens] == 0) continue;
        dst[t] = (B)src[t];
    }
}

// Per-lane largest magnitude of a double vector [E][J][S] (as the bits of a
// non-negative double, whose integer order is the numeric order), for the
// power-of-two scaling of the float V-cycle's input.  mx[E][S] starts at 0.
__global__ void k_mg_lane_max(int J, int S, const double *__restrict__ r, unsigned long long *mx,
                              const int *__restrict__ ens_live)
{
    const int e = blockIdx.y;
    if (ens_live && ens_live[e] == 0) return;
    const int s = threadIdx.x % S, g = threadIdx.x / S, G = blockDim.x / S;
    const double *re = r + (size_t)e * J * S + s;
    double m = 0.0;
    for (int j = blockIdx.x * G + g; j < J; j += gridDim.x * G) m = fmax(m, fabs(re[(size_t)j * S]));
    __shared__ double sh[kBlock];
    sh[threadIdx.x] = m;
    __syncthreads();
    if (threadIdx.x < S) {
        for (int q = 1; q < G; q++) m = fmax(m, sh[q * S + threadIdx.x]);
        // NaN compares false in fmax; a lane with a NaN residual keeps its own value
        if (m > 0.0) atomicMax(mx + (size_t)e * S + threadIdx.x, (unsigned long long)__double_as_longlong(m));
    }
}

// The power of two 2^x of a lane's scale: x = the binary exponent of its
// largest magnitude (0 for a zero or non-finite lane), so the scaled values lie
// below 2 in magnitude and their float rounding neither overflows nor leaves
// the normal range for entries within 2^-125 of the largest.
__device__ __forceinline__ int lane_exponent(const unsigned long long *mx, size_t L)
{
    const double m = __longlong_as_double((long long)mx[L]);
    return (m > 0.0 && isfinite(m)) ? ilogb(m) : 0;
}

// dst = float(src 2^-x) per lane (narrow) or dst = double(src) 2^x (widen).
// Scaling by a power of two is exact, and every operation of the V-cycle
// commutes with it, so in range the result equals the unscaled one bit for bit.
template <typename A, typename B>
__global__ void k_mg_convert_scaled(size_t n, size_t per_ens, int S, const A *__restrict__ src, B *__restrict__ dst,
                                    const unsigned long long *__restrict__ mx, int widen,
                                    const int *__restrict__ ens_live)
{
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
        const size_t e = t / per_ens;
        if (ens_live && ens_live[e] == 0) continue;
        const int x = lane_exponent(mx, e * S + t % S);
        dst[t] = (B)scalbn((double)src[t], widen ? x : -x);
    }
}

// ---- CG kernels: 256-row blocks, per-lane block partial sums ---------------------

// Per-lane sum over the block's row groups, pairwise in a fixed order; the
// result is valid in threads t < S.
__device__ __forceinline__ double block_lane_sum(double v, int S, double *sh)
{
    const int t = threadIdx.x, G = blockDim.x / S;
    sh[t] = v;
    __syncthreads();
    for (int st = G / 2; st > 0; st >>= 1) {
        if (t / S < st) sh[t] = dadd(sh[t], sh[t + st * S]);
        __syncthreads();
    }
    return sh[t];
}

// Per-lane largest magnitude over the block's row groups, atomically merged
// into mx[L] (the bits of a non-negative double order like the value).
__device__ __forceinline__ void block_lane_max(double v, int S, unsigned long long *mx, int L)
{
    __shared__ double shm[kBlock];
    const int t = threadIdx.x, G = blockDim.x / S;
    shm[t] = v;
    __syncthreads();
    if (t < S) {
        for (int q = 1; q < G; q++) v = fmax(v, shm[q * S + t]);
        if (v > 0.0) atomicMax(mx + L, (unsigned long long)__double_as_longlong(v));
    }
}

struct CgArgs {
    int J, S, E, nblk, maxit;
    double rtol;
    const uint8_t *active;
    int32_t *iters, *status;
    double *relres;
};

// x = 0, r = b; block partials of b^T b (part0).
__global__ void k_mgcg_init(int J, int S, int nblk, const double *__restrict__ b, double *__restrict__ x,
                            double *__restrict__ r, double *__restrict__ part, unsigned long long *rmax)
{
    __shared__ double sh[kBlock];
    const int e = blockIdx.y, s = threadIdx.x % S, G = blockDim.x / S;
    const int r0 = blockIdx.x * kRedRows, r1 = min(J, r0 + kRedRows);
    double acc = 0.0, m = 0.0;
    for (int i = r0 + threadIdx.x / S; i < r1; i += G) {
        const size_t o = ((size_t)e * J + i) * S + s;
        const double bv = b[o];
        x[o] = 0.0;
        r[o] = bv;
        acc = fma(bv, bv, acc);
        m = fmax(m, fabs(bv));
    }
    const double tot = block_lane_sum(acc, S, sh);
    if (threadIdx.x < S) part[((size_t)e * nblk + blockIdx.x) * S + s] = tot;
    if (rmax) block_lane_max(m, S, rmax, e * S + s);
}

// Block partials of u^T v for live lanes (all lanes when live is null).
__global__ void k_mgcg_dot(int J, int S, int nblk, const double *__restrict__ u, const double *__restrict__ v,
                           const int *__restrict__ live, const int *__restrict__ ens_live, double *__restrict__ part)
{
    __shared__ double sh[kBlock];
    const int e = blockIdx.y, s = threadIdx.x % S, G = blockDim.x / S;
    if (ens_skip(ens_live, e)) return;
    const bool on = !live || live[e * S + s];
    const int r0 = blockIdx.x * kRedRows, r1 = min(J, r0 + kRedRows);
    double acc = 0.0;
    if (on)
        for (int i = r0 + threadIdx.x / S; i < r1; i += G) {
            const size_t o = ((size_t)e * J + i) * S + s;
            acc = fma(u[o], v[o], acc);
        }
    const double tot = block_lane_sum(acc, S, sh);
    if (threadIdx.x < S) part[((size_t)e * nblk + blockIdx.x) * S + s] = tot;
}

// q = A p for live lanes, one row-lane per thread (p^T q follows in k_mgcg_dot).
__global__ void k_mgcg_spmv(int J, int S, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                            const double *__restrict__ vals, const double *__restrict__ p, double *__restrict__ q,
                            const int *__restrict__ live, const int *__restrict__ ens_live)
{
    int s, i;
    row_lane(S, &s, &i);
    const int e = blockIdx.y;
    if (i >= J || ens_skip(ens_live, e) || !live[e * S + s]) return;
    const int64_t nnz = rp[J];
    const size_t vb = (size_t)e * J * S + s;
    q[vb + (size_t)i * S] = row_dot(rp, ci, vals + (size_t)e * nnz * S + s, p + vb, i, S);
}

// x += alpha p, r -= alpha q and block partials of r^T r for live lanes.
__global__ void k_mgcg_update(int J, int S, int nblk, double *__restrict__ x, double *__restrict__ r,
                              const double *__restrict__ p, const double *__restrict__ q,
                              const double *__restrict__ alpha, const int *__restrict__ live,
                              const int *__restrict__ ens_live, double *__restrict__ part,
                              unsigned long long *rmax)
{
    __shared__ double sh[kBlock];
    const int e = blockIdx.y, s = threadIdx.x % S, G = blockDim.x / S;
    if (ens_skip(ens_live, e)) return;
    const int L = e * S + s;
    const bool on = live[L] != 0;
    const double al = on ? alpha[L] : 0.0;
    const int r0 = blockIdx.x * kRedRows, r1 = min(J, r0 + kRedRows);
    double acc = 0.0, m = 0.0;
    if (on)
        for (int i = r0 + threadIdx.x / S; i < r1; i += G) {
            const size_t o = ((size_t)e * J + i) * S + s;
            x[o] = fma(al, p[o], x[o]);
            const double rv = fma(-al, q[o], r[o]);
            r[o] = rv;
            acc = fma(rv, rv, acc);
            m = fmax(m, fabs(rv));
        }
    const double tot = block_lane_sum(acc, S, sh);
    if (threadIdx.x < S) part[((size_t)e * nblk + blockIdx.x) * S + s] = tot;
    if (rmax) block_lane_max(m, S, rmax, L);
}

// p = z + beta p for live lanes; p = z for every lane when beta is null.
__global__ void k_mgcg_dir(int J, int S, const double *__restrict__ z, double *__restrict__ p,
                           const double *__restrict__ beta, const int *__restrict__ live,
                           const int *__restrict__ ens_live)
{
    int s, i;
    row_lane(S, &s, &i);
    const int e = blockIdx.y;
    if (i >= J || ens_skip(ens_live, e)) return;
    const int L = e * S + s;
    const size_t o = ((size_t)e * J + i) * S + s;
    if (!beta)
        p[o] = z[o];
    else if (live[L])
        p[o] = fma(beta[L], p[o], z[o]);
}

// The lane totals of nblk block partials: thread group g sums partials
// g, g + G, ... in turn, then the groups combine pairwise (fixed order).
__device__ double lane_total(const double *__restrict__ part, int nblk, int S, int e, double *sh)
{
    const int t = threadIdx.x, s = t % S, g = t / S, G = blockDim.x / S;
    double v = 0.0;
    for (int b = g; b < nblk; b += G) v = dadd(v, part[((size_t)e * nblk + b) * S + s]);
    return block_lane_sum(v, S, sh);
}

__device__ __forceinline__ void mg_freeze(const CgArgs &a, int *live, int L, int st, int it, double relres,
                                          int *dead)
{
    live[L] = 0;
    a.status[L] = st;
    a.iters[L] = it;
    a.relres[L] = relres;
    atomicAdd(dead, 1);
}

// Kinds of the per-lane finishing step.
enum { FIN_INIT = 0, FIN_ALPHA = 1, FIN_CONV = 2, FIN_BETA = 3 };

__global__ void k_mgcg_final(CgArgs a, int kind, const double *__restrict__ part0, const double *__restrict__ part1,
                             MgWork w)
{
    __shared__ double sh[kBlock];
    __shared__ int dead, born;
    const int e = blockIdx.x, S = a.S;
    if (kind != FIN_INIT && w.ens_live[e] == 0) return;
    if (threadIdx.x == 0) dead = born = 0;
    const double t0 = lane_total(part0, a.nblk, S, e, sh);
    __syncthreads();
    double t1 = 0.0;
    if (kind == FIN_INIT) t1 = lane_total(part1, a.nblk, S, e, sh);
    if (threadIdx.x < S) {
        const int L = e * S + threadIdx.x;
        // the float V-cycle's lane maxima of the next r start from zero (k_mgcg_update merges into them)
        if (kind == FIN_ALPHA && w.rmax) w.rmax[L] = 0ull;
        if (kind == FIN_INIT) {
            const double bsq = t0, rz = t1;
            const int act = a.active ? (int)a.active[L] : 1;
            int lv = 0;
            w.k[L] = 0;
            if (!act) {
                a.status[L] = ENS_LANE_INACTIVE; a.iters[L] = 0; a.relres[L] = 0.0;
            } else if (w.bad[L] || !isfinite(bsq) || !isfinite(rz)) {
                a.status[L] = ENS_LANE_BADINPUT; a.iters[L] = 0;
                a.relres[L] = __longlong_as_double(0x7ff8000000000000LL);
            } else if (bsq == 0.0) {
                a.status[L] = ENS_LANE_CONVERGED; a.iters[L] = 0; a.relres[L] = 0.0;
            } else if (a.maxit <= 0) {
                a.status[L] = ENS_LANE_MAXIT; a.iters[L] = 0; a.relres[L] = 1.0;
            } else {
                lv = 1;
                w.bnorm[L] = sqrt(bsq);
                w.rz[L] = rz;
                w.rr[L] = bsq;
                a.status[L] = ENS_LANE_MAXIT; a.iters[L] = 0; a.relres[L] = 1.0;
            }
            w.live[L] = lv;
            if (lv) atomicAdd(&born, 1);
        } else if (w.live[L]) {
            if (kind == FIN_ALPHA) {
                const double pq = t0;
                if (!(pq > 0.0) || !isfinite(pq))
                    mg_freeze(a, w.live, L, ENS_LANE_BREAKDOWN, w.k[L], sqrt(w.rr[L]) / w.bnorm[L], &dead);
                else
                    w.alpha[L] = w.rz[L] / pq;
            } else if (kind == FIN_CONV) {
                const int k = w.k[L] + 1;
                w.k[L] = k;
                w.rr[L] = t0;
                const double res = sqrt(t0), bn = w.bnorm[L];
                if (res <= a.rtol * bn)
                    mg_freeze(a, w.live, L, ENS_LANE_CONVERGED, k, res / bn, &dead);
                else if (k >= a.maxit)
                    mg_freeze(a, w.live, L, ENS_LANE_MAXIT, k, res / bn, &dead);
            } else {
                const double rzn = t0;
                w.beta[L] = rzn / w.rz[L];
                w.rz[L] = rzn;
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (kind == FIN_INIT) {
            w.ens_live[e] = born;
            if (born) atomicAdd(w.live_total, born);
        } else if (dead) {
            w.ens_live[e] -= dead;
            atomicSub(w.live_total, dead);
        }
    }
}

// ---- host side ------------------------------------------------------------------

inline dim3 rl_grid(int J, int S, int E) { return dim3((unsigned)((J + kBlock / S - 1) / (kBlock / S)), (unsigned)E); }

// The workspace's set-up record on this handle (nullptr if it has none).
MgTag *mg_tag(ens_ctx *h, const void *work)
{
    for (auto &t : h->mg_tags)
        if (t.work == work) return &t;
    return nullptr;
}

void mg_record(ens_ctx *h, const ens_problem *p, int S, int E, int mixed, const void *work)
{
    MgTag *t = mg_tag(h, work);
    if (!t) {
        if (h->mg_tags.size() >= 16) h->mg_tags.erase(h->mg_tags.begin());
        h->mg_tags.push_back(MgTag());
        t = &h->mg_tags.back();
    }
    t->work = work;
    t->kind = p->kind;
    t->n = p->n;
    t->S = S;
    t->E = E;
    t->mixed = mixed;
}

int mg_check(ens_ctx *h, const char *who, const ens_problem *p, int S, int E, int mixed, const void *work,
             size_t work_bytes, MgWork *w, bool setup = false)
{
    if (!h) return ENS_EINVAL;
    if (!p) return set_error(h, ENS_EINVAL, std::string(who) + ": null problem");
    if (p->kind != ENS_Q1_3D_KL && p->kind != ENS_Q1_3D_DISC)
        return set_error(h, ENS_ENOTSUP, std::string(who) + ": the multigrid hierarchy is built for the trilinear problems only");
    int J;
    int64_t nnz;
    std::string why;
    if (problem_check(p, &J, &nnz, &why)) return set_error(h, ENS_EINVAL, std::string(who) + ": " + why);
    if (!lane_count_ok(S) || E < 0) return set_error(h, ENS_EINVAL, std::string(who) + ": bad S / E");
    if (mixed != 0 && mixed != 1) return set_error(h, ENS_EINVAL, std::string(who) + ": mixed must be 0 or 1");
    if (!mg_layout(p, S, E, mixed, nullptr, w))
        return set_error(h, ENS_EINVAL, std::string(who) + ": n must be 2^k - 1 (k >= 2)");
    if (E > 0 && (!work || work_bytes < w->bytes)) return set_error(h, ENS_EINVAL, std::string(who) + ": workspace too small");
    if (!setup && E > 0) {
        const MgTag *t = mg_tag(h, work);
        if (t && (t->kind != p->kind || t->n != p->n || t->S != S || t->E != E || t->mixed != mixed))
            return set_error(h, ENS_EINVAL, std::string(who) + ": the workspace was set up (ens_mg_setup) with another "
                                            "problem, S, E or mixed flag");
    }
    mg_layout(p, S, E, mixed, (char *)work, w);
    return ENS_OK;
}

// The arrays of one level in the V-cycle's precision.
template <typename T> struct LevelView {
    const T *vals, *dinv, *coef;
    T *rhs, *e, *t, *d, *res;
};
template <typename T> LevelView<T> level_view(const MgLevel &v);
template <> LevelView<double> level_view<double>(const MgLevel &v)
{
    return {v.vals, v.dinv, v.coef, v.rhs, v.e, v.t, v.d, v.res};
}
template <> LevelView<float> level_view<float>(const MgLevel &v)
{
    return {v.vals32, v.dinv32, v.coef32, v.rhs32, v.e32, v.t32, v.d32, v.res32};
}
inline const double *coarse_inverse(const MgWork &w, double *) { return w.cinv; }
inline const float *coarse_inverse(const MgWork &w, float *) { return w.cinv32; }

// One V-cycle in precision T: e0 = M rhs0 on level 0 (vals0: level 0's values in T).
template <typename T>
int mg_vcycle(ens_ctx *h, const MgWork &w, const int32_t *rp0, const int32_t *ci0, const T *vals0, int S, int E,
              const T *rhs0, T *e0, const int *ens_live, cudaStream_t st)
{
    const int L = w.L;
    for (int l = 0; l < L - 1; l++) {
        const MgLevel &v = w.lv[l];
        const LevelView<T> a = level_view<T>(v);
        const int32_t *rp = l ? v.rp : rp0, *ci = l ? v.ci : ci0;
        const T *vals = l ? a.vals : vals0;
        const T *rhs = l ? a.rhs : rhs0;
        T *e = l ? a.e : e0;
        const dim3 g = rl_grid(v.J, S, E);
        k_mg_cheb1<T><<<g, kBlock, 0, st>>>(v.J, S, rp, ci, vals, a.dinv, a.coef, rhs, nullptr, a.d, a.t, ens_live);
        k_mg_cheb2<T><<<g, kBlock, 0, st>>>(v.J, S, rp, ci, vals, a.dinv, a.coef, rhs, a.t, a.d, e, ens_live);
        k_mg_resid<T><<<g, kBlock, 0, st>>>(v.J, S, rp, ci, vals, rhs, e, a.res, ens_live);
        k_mg_restrict<T><<<rl_grid(w.lv[l + 1].J, S, E), kBlock, 0, st>>>(v.n, w.lv[l + 1].n, S, a.res,
                                                                         level_view<T>(w.lv[l + 1]).rhs, ens_live);
    }
    {
        const LevelView<T> a = level_view<T>(w.lv[L - 1]);
        const T *rhs = L > 1 ? a.rhs : rhs0;
        T *e = L > 1 ? a.e : e0;
        k_mg_coarse_solve<T><<<rl_grid(kCoarseJ, S, E), kBlock, 0, st>>>(S, coarse_inverse(w, (T *)nullptr), rhs,
                                                                          e, ens_live);
    }
    for (int l = L - 2; l >= 0; l--) {
        const MgLevel &v = w.lv[l];
        const LevelView<T> a = level_view<T>(v);
        const int32_t *rp = l ? v.rp : rp0, *ci = l ? v.ci : ci0;
        const T *vals = l ? a.vals : vals0;
        const T *rhs = l ? a.rhs : rhs0;
        T *e = l ? a.e : e0;
        const T *ec = level_view<T>(w.lv[l + 1]).e;  // l + 1 >= 1: a coarse level's correction
        const dim3 g = rl_grid(v.J, S, E);
        k_mg_prolong_add<T><<<g, kBlock, 0, st>>>(v.n, w.lv[l + 1].n, S, ec, e, ens_live);
        k_mg_cheb1<T><<<g, kBlock, 0, st>>>(v.J, S, rp, ci, vals, a.dinv, a.coef, rhs, e, a.d, a.t, ens_live);
        k_mg_cheb2<T><<<g, kBlock, 0, st>>>(v.J, S, rp, ci, vals, a.dinv, a.coef, rhs, a.t, a.d, e, ens_live);
    }
    ENS_LAUNCH_CHECK(h, "multigrid V-cycle");
    return ENS_OK;
}

inline unsigned convert_blocks(size_t n)
{
    const size_t b = (n + kBlock - 1) / kBlock;
    return (unsigned)(b < 152 * 16 ? (b ? b : 1) : 152 * 16);
}

// z = M r with the work's V-cycle: in double, or r rounded to float, the float
// V-cycle, and its result widened to double.  rmax_ready: the CG kernel that
// wrote r already left each lane's largest |r| in w.rmax.
int mg_precond(ens_ctx *h, const MgWork &w, const int32_t *rp0, const int32_t *ci0, const double *vals0, int S,
               int E, const double *r, double *z, const int *ens_live, cudaStream_t st, bool rmax_ready = false)
{
    if (!w.mixed) return mg_vcycle<double>(h, w, rp0, ci0, vals0, S, E, r, z, ens_live, st);
    const int J = w.lv[0].J;
    const size_t per = (size_t)J * S, n = per * E;
    if (!rmax_ready) {
        ENS_CUDA_CHECK(h, cudaMemsetAsync(w.rmax, 0, sizeof(unsigned long long) * E * S, st));
        const unsigned nb = (unsigned)std::min<int>((J + kBlock / S - 1) / (kBlock / S), 64);
        k_mg_lane_max<<<dim3(nb, (unsigned)E), kBlock, 0, st>>>(J, S, r, w.rmax, ens_live);
    }
    k_mg_convert_scaled<double, float><<<convert_blocks(n), kBlock, 0, st>>>(n, per, S, r, w.lv[0].rhs32, w.rmax, 0,
                                                                             ens_live);
    const int rc = mg_vcycle<float>(h, w, rp0, ci0, w.lv[0].vals32, S, E, w.lv[0].rhs32, w.lv[0].e32, ens_live, st);
    if (rc) return rc;
    k_mg_convert_scaled<float, double><<<convert_blocks(n), kBlock, 0, st>>>(n, per, S, w.lv[0].e32, z, w.rmax, 1,
                                                                             ens_live);
    ENS_LAUNCH_CHECK(h, "multigrid V-cycle (float)");
    return ENS_OK;
}

}  // namespace
}  // namespace ens

using namespace ens;

extern "C" size_t ens_mg_workspace_size(const ens_problem *p, int S, int E, int mixed)
{
    if (!p || (p->kind != ENS_Q1_3D_KL && p->kind != ENS_Q1_3D_DISC) || !lane_count_ok(S) || E < 0) return 0;
    if (mixed != 0 && mixed != 1) return 0;
    int J;
    int64_t nnz;
    std::string why;
    if (problem_check(p, &J, &nnz, &why)) return 0;
    MgWork w;
    if (!mg_layout(p, S, E, mixed, nullptr, &w)) return 0;
    return w.bytes;
}

extern "C" int ens_mg_setup(ens_handle h, const ens_problem *p, int S, int E, int mixed, const int32_t *rowptr,
                            const int32_t *colidx, const double *vals, void *work, size_t work_bytes, void *stream)
{
    MgWork w;
    int rc = mg_check(h, "ens_mg_setup", p, S, E, mixed, work, work_bytes, &w, true);
    if (rc) return rc;
    if (E == 0) return ENS_OK;
    if (!rowptr || !colidx || !vals) return set_error(h, ENS_EINVAL, "ens_mg_setup: null pointer");
    mg_record(h, p, S, E, mixed, work);
    cudaStream_t st = (cudaStream_t)stream;
    const int ES = E * S;
    for (int l = 1; l < w.L; l++) {
        ens_problem pc = *p;
        pc.n = w.lv[l].n;
        rc = pattern_into(h, &pc, w.lv[l].rp, w.lv[l].ci, st);
        if (rc) return rc;
    }
    ENS_CUDA_CHECK(h, cudaMemsetAsync(w.bad, 0, sizeof(int) * ES, st));
    for (int l = 0; l < w.L; l++) {
        MgLevel &v = w.lv[l];
        const int32_t *rp = l ? v.rp : rowptr, *ci = l ? v.ci : colidx;
        const double *vl = l ? v.vals : vals;
        if (l > 0) {
            const MgLevel &f = w.lv[l - 1];
            k_mg_galerkin<<<rl_grid(27 * v.J, S, E), kBlock, 0, st>>>(f.n, v.n, S, l - 1 ? f.rp : rowptr,
                                                                      l - 1 ? f.vals : vals, v.rp, v.vals);
        }
        ENS_CUDA_CHECK(h, cudaMemsetAsync(v.lmax, 0, sizeof(unsigned long long) * ES, st));
        k_mg_diag<<<rl_grid(v.J, S, E), kBlock, 0, st>>>(v.J, S, rp, ci, vl, v.dinv, v.lmax, w.bad);
        k_mg_coef<<<(ES + kBlock - 1) / kBlock, kBlock, 0, st>>>(ES, v.lmax, v.coef);
    }
    {
        const MgLevel &c = w.lv[w.L - 1];
        k_mg_chol<<<dim3((unsigned)S, (unsigned)E), 32, 0, st>>>(S, w.L > 1 ? c.rp : rowptr, w.L > 1 ? c.ci : colidx,
                                                                  w.L > 1 ? c.vals : vals, w.cinv, w.bad);
    }
    if (mixed) {  // the float copy of the whole hierarchy, each value rounded once
        auto cvt = [&](const double *src, float *dst, size_t n) {
            k_mg_convert<double, float><<<convert_blocks(n), kBlock, 0, st>>>(n, n, src, dst, nullptr);
        };
        for (int l = 0; l < w.L; l++) {
            MgLevel &v = w.lv[l];
            cvt(l ? v.vals : vals, v.vals32, (size_t)ES * v.nnz);
            cvt(v.dinv, v.dinv32, (size_t)ES * v.J);
            cvt(v.coef, v.coef32, (size_t)ES * 4);
        }
        cvt(w.cinv, w.cinv32, (size_t)ES * kInv);
    }
    ENS_LAUNCH_CHECK(h, "ens_mg_setup");
    return ENS_OK;
}

extern "C" int ens_mg_level(ens_handle h, const ens_problem *p, int S, int E, int mixed, int level,
                            double *vals_out, double *lmax_out, const void *work, size_t work_bytes, void *stream)
{
    MgWork w;
    int rc = mg_check(h, "ens_mg_level", p, S, E, mixed, work, work_bytes, &w);
    if (rc) return rc;
    if (level < 0 || level >= w.L) return set_error(h, ENS_EINVAL, "ens_mg_level: no such level");
    if (E == 0) return ENS_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const MgLevel &v = w.lv[level];
    const size_t ES = (size_t)E * S;
    if (vals_out && level > 0)
        ENS_CUDA_CHECK(h, cudaMemcpyAsync(vals_out, v.vals, ES * v.nnz * sizeof(double), cudaMemcpyDeviceToDevice, st));
    if (lmax_out)
        ENS_CUDA_CHECK(h, cudaMemcpyAsync(lmax_out, v.lmax, ES * sizeof(double), cudaMemcpyDeviceToDevice, st));
    return ENS_OK;
}

extern "C" int ens_mg_apply(ens_handle h, const ens_problem *p, int S, int E, int mixed, const int32_t *rowptr,
                            const int32_t *colidx, const double *vals, const double *r, double *z, void *work,
                            size_t work_bytes, void *stream)
{
    MgWork w;
    int rc = mg_check(h, "ens_mg_apply", p, S, E, mixed, work, work_bytes, &w);
    if (rc) return rc;
    if (E == 0) return ENS_OK;
    if (!rowptr || !colidx || !vals || !r || !z) return set_error(h, ENS_EINVAL, "ens_mg_apply: null pointer");
    return mg_precond(h, w, rowptr, colidx, vals, S, E, r, z, nullptr, (cudaStream_t)stream);
}

extern "C" int ens_mgpcg_solve(ens_handle h, const ens_problem *p, int S, int E, int mixed, const int32_t *rowptr,
                               const int32_t *colidx, const double *vals, const double *b, double *x,
                               const uint8_t *active, double rtol, int maxit, int32_t *iters, double *relres,
                               int32_t *status, void *work, size_t work_bytes, void *stream)
{
    MgWork w;
    int rc = mg_check(h, "ens_mgpcg_solve", p, S, E, mixed, work, work_bytes, &w);
    if (rc) return rc;
    if (E == 0) return ENS_OK;
    if (!rowptr || !colidx || !vals || !b || !x || !iters || !relres || !status)
        return set_error(h, ENS_EINVAL, "ens_mgpcg_solve: null pointer");
    if (!(rtol >= 0.0)) return set_error(h, ENS_EINVAL, "ens_mgpcg_solve: rtol must be >= 0");
    cudaStream_t st = (cudaStream_t)stream;
    const int J = w.lv[0].J;
    CgArgs a;
    a.J = J; a.S = S; a.E = E; a.nblk = w.nblk; a.maxit = maxit; a.rtol = rtol;
    a.active = active; a.iters = iters; a.status = status; a.relres = relres;
    const dim3 gred((unsigned)w.nblk, (unsigned)E), grl = rl_grid(J, S, E);
    ENS_CUDA_CHECK(h, cudaMemsetAsync(w.live_total, 0, sizeof(int), st));
    // x = 0, r = b, z = M r, p = z; b^T b and r^T z decide each lane's start
    if (w.mixed) ENS_CUDA_CHECK(h, cudaMemsetAsync(w.rmax, 0, sizeof(unsigned long long) * E * S, st));
    k_mgcg_init<<<gred, kBlock, 0, st>>>(J, S, w.nblk, b, x, w.r, w.part0, w.mixed ? w.rmax : nullptr);
    rc = mg_precond(h, w, rowptr, colidx, vals, S, E, w.r, w.z, nullptr, st, true);
    if (rc) return rc;
    k_mgcg_dot<<<gred, kBlock, 0, st>>>(J, S, w.nblk, w.r, w.z, nullptr, nullptr, w.part1);
    k_mgcg_final<<<E, kBlock, 0, st>>>(a, FIN_INIT, w.part0, w.part1, w);
    k_mgcg_dir<<<grl, kBlock, 0, st>>>(J, S, w.z, w.p, nullptr, w.live, nullptr);
    ENS_LAUNCH_CHECK(h, "ens_mgpcg_solve: init");
    int left = 0;
    ENS_CUDA_CHECK(h, cudaMemcpyAsync(&left, w.live_total, sizeof(int), cudaMemcpyDeviceToHost, st));
    ENS_CUDA_CHECK(h, cudaStreamSynchronize(st));
    int trips = 0;
    while (left > 0 && trips < maxit) {
        // a few iterations per look at the live count: a lane freezes at its
        // own iteration, so the count only decides when launching can stop
        const int chunk = trips < 8 ? 2 : 4;
        for (int c = 0; c < chunk && trips < maxit; c++, trips++) {
            k_mgcg_spmv<<<grl, kBlock, 0, st>>>(J, S, rowptr, colidx, vals, w.p, w.q, w.live, w.ens_live);
            k_mgcg_dot<<<gred, kBlock, 0, st>>>(J, S, w.nblk, w.p, w.q, w.live, w.ens_live, w.part0);
            k_mgcg_final<<<E, kBlock, 0, st>>>(a, FIN_ALPHA, w.part0, nullptr, w);
            k_mgcg_update<<<gred, kBlock, 0, st>>>(J, S, w.nblk, x, w.r, w.p, w.q, w.alpha, w.live, w.ens_live,
                                                   w.part0, w.mixed ? w.rmax : nullptr);
            k_mgcg_final<<<E, kBlock, 0, st>>>(a, FIN_CONV, w.part0, nullptr, w);
            rc = mg_precond(h, w, rowptr, colidx, vals, S, E, w.r, w.z, w.ens_live, st, true);
            if (rc) return rc;
            k_mgcg_dot<<<gred, kBlock, 0, st>>>(J, S, w.nblk, w.r, w.z, w.live, w.ens_live, w.part0);
            k_mgcg_final<<<E, kBlock, 0, st>>>(a, FIN_BETA, w.part0, nullptr, w);
            k_mgcg_dir<<<grl, kBlock, 0, st>>>(J, S, w.z, w.p, w.beta, w.live, w.ens_live);
        }
        ENS_LAUNCH_CHECK(h, "ens_mgpcg_solve: iteration");
        ENS_CUDA_CHECK(h, cudaMemcpyAsync(&left, w.live_total, sizeof(int), cudaMemcpyDeviceToHost, st));
        ENS_CUDA_CHECK(h, cudaStreamSynchronize(st));
    }
    return ENS_OK;
}
