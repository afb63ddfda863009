// adjoint.cu -- gradient of a linear quantity of interest through the ensemble
// solve (K8, the differentiation layer).
//
// For Q(xi) = w^T u with A(xi) u = b, b independent of xi, and the adjoint
// A lambda = w (A is symmetric), dQ/dxi_k = -lambda^T (dA/dxi_k) u.  The FD
// operators of Eq. (elliptic-SPDE) are sums over faces, A = sum_f k_f a_f a_f^T / h^2
// with a_f = e_p - e_nbr (or e_p for a boundary face), so
//   dQ/dxi_k = -sum_f (dk_f/dxi_k) (lambda_p - lambda_nbr)(u_p - u_nbr) / h^2,
// the neighbour values being 0 on boundary faces.  The face coefficient is
// k_f = exp(s(x_f, xi)) 10^(aniso xi_j) (the log form of Eq. diff-coeff), so
// dk_f/dxi_k = k_f d(s + aniso ln10 xi_j)/dxi_k, linear in the sine modes.
//
// One thread per (ensemble, row, lane) takes the faces its row owns (the +x,
// +y, +z faces and every boundary face of the row); the N per-lane sums are
// reduced per block and the last block of each ensemble adds the block
// partials in block order (deterministic).
#include "ens_common.cuh"

#include <algorithm>
#include <cmath>

namespace ens {
namespace {

constexpr int kAdjBlock = 256;

__constant__ int kM2[7][2] = {{1, 1}, {2, 1}, {1, 2}, {2, 2}, {3, 1}, {1, 3}, {3, 2}};
__constant__ int kM3[4][3] = {{1, 1, 1}, {2, 1, 1}, {1, 2, 1}, {1, 1, 2}};

// log k_f and d(log k_f)/dxi_k for one face of the given axis at point x.
template <int D>
__device__ double face_dlog(int N, double aniso, const double *xi, int axis, const double *x, double *dl)
{
    double s = 0.0;
    if (D == 2) {
        for (int k = 1; k < N; k++) {
            double phi = sinpi(kM2[k - 1][0] * x[0]) * sinpi(kM2[k - 1][1] * x[1]);
            s = fma(xi[k], phi / (double)k, s);
            dl[k] = 0.5 * phi / (double)k;
        }
        s = 0.5 * s;
        dl[0] = axis == 1 ? aniso * M_LN10 : 0.0;
        if (axis == 1) s = fma(aniso * M_LN10, xi[0], s);
    } else {
        for (int k = 0; k < 4; k++) {
            double phi = sinpi(kM3[k][0] * x[0]) * sinpi(kM3[k][1] * x[1]) * sinpi(kM3[k][2] * x[2]);
            s = fma(xi[2 + k], phi, s);
            dl[2 + k] = 0.3 * phi;
        }
        s = 0.3 * s;
        dl[0] = axis == 1 ? aniso * M_LN10 : 0.0;
        dl[1] = axis == 2 ? aniso * M_LN10 : 0.0;
        if (axis == 1) s = fma(aniso * M_LN10, xi[0], s);
        if (axis == 2) s = fma(aniso * M_LN10, xi[1], s);
    }
    return s;
}

template <int D, int NMAX>
__global__ void __launch_bounds__(kAdjBlock) k_adjoint(int n, int N, double aniso, int S, int E, int RT,
                                                       const double *__restrict__ xi_all,
                                                       const double *__restrict__ u_all,
                                                       const double *__restrict__ lam_all,
                                                       double *__restrict__ part, int *counter,
                                                       double *__restrict__ grad)
{
    const int J = D == 2 ? n * n : n * n * n;
    const int e = blockIdx.y;
    const int nblk = gridDim.x;
    const double den = (double)(n + 1);
    const double ih2 = den * den;
    double acc[NMAX];
#pragma unroll
    for (int k = 0; k < NMAX; k++) acc[k] = 0.0;
    // thread t: lane t % S, rows t / S, t / S + blockDim / S, ... within the block's tile
    const int s = threadIdx.x % S, g = threadIdx.x / S, G = blockDim.x / S;
    const int r0 = blockIdx.x * RT, r1 = min(J, r0 + RT);
    double xs[8];
    const double *xsrc = xi_all + ((size_t)e * S + s) * N;
    for (int k = 0; k < N; k++) xs[k] = xsrc[k];
    const double *u = u_all + (size_t)e * J * S + s;
    const double *lam = lam_all + (size_t)e * J * S + s;
    const int stride[3] = {1, n, n * n};
    for (int p = r0 + g; p < r1; p += G) {
        const int gi[3] = {p % n, (p / n) % n, D == 3 ? p / (n * n) : 0};
        const double up = u[(size_t)p * S], lp = lam[(size_t)p * S];
        for (int axis = 0; axis < D; axis++)
            for (int dir = -1; dir <= 1; dir += 2) {
                const int nb = gi[axis] + dir;
                const bool interior = nb >= 0 && nb < n;
                if (interior && dir < 0) continue;  // interior faces are owned by their lower node
                double x[3];
                for (int a = 0; a < D; a++) x[a] = (double)(gi[a] + 1) / den;
                x[axis] = ((double)(gi[axis] + 1) + 0.5 * dir) / den;
                double dl[NMAX];
                const double lk = face_dlog<D>(N, aniso, xs, axis, x, dl);
                const double kf = exp(lk);
                double un = 0.0, ln = 0.0;
                if (interior) {
                    un = u[(size_t)(p + dir * stride[axis]) * S];
                    ln = lam[(size_t)(p + dir * stride[axis]) * S];
                }
                const double prod = kf * (lp - ln) * (up - un) * ih2;
#pragma unroll
                for (int k = 0; k < NMAX; k++)
                    if (k < N) acc[k] = fma(-dl[k], prod, acc[k]);
            }
    }
    // per-lane block sums in a fixed order: thread groups g = 0..G-1 of lane s
    __shared__ double sh[kAdjBlock];
    __shared__ int s_last;
    for (int k = 0; k < N; k++) {
        sh[threadIdx.x] = acc[k];
        __syncthreads();
        if (threadIdx.x < S) {
            double v = 0.0;
            for (int q = 0; q < G; q++) v = dadd(v, sh[q * S + threadIdx.x]);
            part[(((size_t)e * nblk + blockIdx.x) * N + k) * S + threadIdx.x] = v;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(counter + e, 1) == nblk - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    for (int t = threadIdx.x; t < N * S; t += blockDim.x) {
        const int k = t / S, l = t % S;
        double v = 0.0;
        for (int b = 0; b < nblk; b++) v = dadd(v, __ldcg(part + (((size_t)e * nblk + b) * N + k) * S + l));
        grad[((size_t)e * S + l) * N + k] = v;
    }
    if (threadIdx.x == 0) counter[e] = 0;
}

int adj_geometry(int J, int *RT)
{
    int rt = (J + 152 * 4 - 1) / (152 * 4);
    if (rt < 64) rt = 64;
    *RT = rt;
    return (J + rt - 1) / rt;
}

}  // namespace
}  // namespace ens

using namespace ens;

extern "C" size_t ens_adjoint_workspace_size(const ens_problem *p, int S, int E)
{
    int J;
    int64_t nnz;
    std::string why;
    if (problem_check(p, &J, &nnz, &why) || !lane_count_ok(S) || E <= 0) return 0;
    int RT;
    int nblk = adj_geometry(J, &RT);
    return align256((size_t)E * nblk * p->nparam * S * sizeof(double)) + align256((size_t)E * sizeof(int));
}

extern "C" int ens_adjoint_grad(ens_handle h, const ens_problem *p, int S, int E, const double *xi,
                                const double *u, const double *lam, double *grad, void *work, size_t work_bytes,
                                void *stream)
{
    if (!h) return ENS_EINVAL;
    int J;
    int64_t nnz;
    std::string why;
    int rc = problem_check(p, &J, &nnz, &why);
    if (rc) return set_error(h, rc, "ens_adjoint_grad: " + why);
    if (p->kind != ENS_FD5_LOGKL && p->kind != ENS_FD7_AXIS)
        return set_error(h, ENS_ENOTSUP, "ens_adjoint_grad: only the FD problems have an adjoint gradient here");
    if (!lane_count_ok(S) || E < 0 || E > 65535) return set_error(h, ENS_EINVAL, "ens_adjoint_grad: bad S / E");
    if (E == 0) return ENS_OK;
    if (!xi || !u || !lam || !grad || !work) return set_error(h, ENS_EINVAL, "ens_adjoint_grad: null pointer");
    const size_t need = ens_adjoint_workspace_size(p, S, E);
    if (work_bytes < need) return set_error(h, ENS_ENOMEM, "ens_adjoint_grad: workspace too small");
    int RT;
    const int nblk = adj_geometry(J, &RT);
    double *part = (double *)work;
    int *counter = (int *)((char *)work + align256((size_t)E * nblk * p->nparam * S * sizeof(double)));
    cudaStream_t st = (cudaStream_t)stream;
    ENS_CUDA_CHECK(h, cudaMemsetAsync(counter, 0, (size_t)E * sizeof(int), st));
    dim3 grid(nblk, E);
    if (p->kind == ENS_FD5_LOGKL)
        k_adjoint<2, 8><<<grid, kAdjBlock, 0, st>>>(p->n, p->nparam, p->aniso, S, E, RT, xi, u, lam, part, counter,
                                                    grad);
    else
        k_adjoint<3, 8><<<grid, kAdjBlock, 0, st>>>(p->n, p->nparam, p->aniso, S, E, RT, xi, u, lam, part, counter,
                                                    grad);
    ENS_LAUNCH_CHECK(h, "ens_adjoint_grad");
    return ENS_OK;
}

namespace ens {
namespace {

// b[e][j][s] = w[j]: the adjoint right-hand side of every lane.
__global__ void k_broadcast_w(int J, int S, int E, const double *__restrict__ w, double *__restrict__ b)
{
    const size_t n = (size_t)E * J * S;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        b[i] = w[(i / S) % J];
}

struct AdjWs {
    double *vals, *dinv, *b;
    void *pcg, *grad;
    size_t pcg_bytes, grad_bytes, total;
};

AdjWs adj_layout(const ens_problem *p, int J, int64_t nnz, int S, int E, char *base)
{
    AdjWs w;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        void *ptr = base ? base + off : nullptr;
        off = align256(off + bytes);
        return ptr;
    };
    w.vals = (double *)take((size_t)E * nnz * S * sizeof(double));
    w.dinv = (double *)take((size_t)E * J * S * sizeof(double));
    w.b = (double *)take((size_t)E * J * S * sizeof(double));
    w.pcg_bytes = ens_pcg_workspace_size(J, nnz, S, E);
    w.pcg = take(w.pcg_bytes);
    w.grad_bytes = ens_adjoint_workspace_size(p, S, E);
    w.grad = take(w.grad_bytes);
    w.total = off;
    return w;
}

}  // namespace
}  // namespace ens

extern "C" size_t ens_adjoint_solve_workspace_size(const ens_problem *p, int S, int E)
{
    int J;
    int64_t nnz;
    std::string why;
    if (problem_check(p, &J, &nnz, &why) || !lane_count_ok(S) || E <= 0) return 0;
    if (p->kind != ENS_FD5_LOGKL && p->kind != ENS_FD7_AXIS) return 0;
    return adj_layout(p, J, nnz, S, E, nullptr).total;
}

extern "C" int ens_adjoint_solve_grad(ens_handle h, const ens_problem *p, int S, int E, const double *xi,
                                      const int32_t *rowptr, const int32_t *colidx, const double *u,
                                      const double *w, const uint8_t *active, double rtol, int maxit, double *Q,
                                      double *grad, double *lam, int32_t *iters, double *relres, int32_t *status,
                                      void *work, size_t work_bytes, void *stream)
{
    if (!h) return ENS_EINVAL;
    int J;
    int64_t nnz;
    std::string why;
    int rc = problem_check(p, &J, &nnz, &why);
    if (rc) return set_error(h, rc, "ens_adjoint_solve_grad: " + why);
    if (p->kind != ENS_FD5_LOGKL && p->kind != ENS_FD7_AXIS)
        return set_error(h, ENS_ENOTSUP, "ens_adjoint_solve_grad: only the FD problems have an adjoint gradient here");
    if (!lane_count_ok(S) || E < 0 || E > 65535) return set_error(h, ENS_EINVAL, "ens_adjoint_solve_grad: bad S / E");
    if (E == 0) return ENS_OK;
    if (!xi || !rowptr || !colidx || !u || !w || !Q || !grad || !lam || !iters || !relres || !status || !work)
        return set_error(h, ENS_EINVAL, "ens_adjoint_solve_grad: null pointer");
    if (work_bytes < ens_adjoint_solve_workspace_size(p, S, E))
        return set_error(h, ENS_ENOMEM, "ens_adjoint_solve_grad: workspace too small");
    AdjWs ws = adj_layout(p, J, nnz, S, E, (char *)work);
    cudaStream_t st = (cudaStream_t)stream;
    rc = ens_assemble(h, p, S, E, xi, rowptr, colidx, ws.vals, 0, ws.dinv, nullptr, stream);
    if (rc) return rc;
    const size_t n = (size_t)E * J * S;
    const int blocks = (int)std::min<size_t>((n + 255) / 256, (size_t)152 * 16);
    k_broadcast_w<<<blocks, 256, 0, st>>>(J, S, E, w, ws.b);
    ENS_LAUNCH_CHECK(h, "ens_adjoint_solve_grad (right-hand side)");
    rc = ens_pcg_solve(h, J, nnz, S, E, rowptr, colidx, ws.vals, ws.dinv, ws.b, lam, active, rtol, maxit, iters,
                       relres, status, ws.pcg, ws.pcg_bytes, stream);
    if (rc) return rc;
    rc = ens_qoi(h, J, S, E, u, w, Q, stream);
    if (rc) return rc;
    return ens_adjoint_grad(h, p, S, E, xi, u, lam, grad, ws.grad, ws.grad_bytes, stream);
}
