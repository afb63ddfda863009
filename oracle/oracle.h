/*
 * oracle.h -- plain CPU FP64 restatement of the ensemble-grouping method of
 * D'Elia, Phipps, Rushdi, Ebeida, "Surrogate-based Ensemble Grouping Strategies
 * for Embedded Sampling-based UQ" (arXiv 1705.02003).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, includes or
 * calls this code; only the tests, __graft_entry__.smoke() and the bench's
 * cpu_baseline / reference arm use it.  It shares no header, helper, table or
 * constant with the CUDA path.
 *
 * Everything here is deliberately slow and obvious: per-sample loops, plain
 * left-to-right sums, no blocking, no fused multiply-add (built with
 * -ffp-contract=off).
 *
 * Problem kinds (the spatial discretisation of Eq. (elliptic-SPDE),
 * -div(A grad u) = f on the unit square/cube, u = 0 on the boundary):
 *   OR_FD5_LOGKL   2-D 5-point finite differences, n x n interior nodes,
 *                  A = exp(0.5 * sum_{k=1}^{N-1} xi_{k+1} phi_k / k) diag(1, 10^(aniso xi_1)),
 *                  f = 1.  N = nparam in 2..8.
 *   OR_Q1_ROT      2-D bilinear (Q1) finite elements, 9-point stencil,
 *                  A = a R(theta) diag(1, 10^(aniso xi_1)) R(theta)^T,
 *                  theta = pi/4 (1 + xi_3), log a = 0.5 (xi_2 phi_1 + xi_4 phi_2 / 2),
 *                  f = 1.  N = 4.
 *   OR_FD7_AXIS    3-D 7-point finite differences,
 *                  A = diag(1, 10^(aniso xi_1), 10^(aniso xi_2)) exp(0.3 sum_{k=3}^{6} xi_k phi_k),
 *                  f = 1.  N = 6.
 *   OR_Q1_3D_KL    3-D trilinear (Q1) finite elements on (n+1)^3 cells, 27-point
 *                  stencil, the field of Section 4 (Test 1):
 *                  A = diag(a, 1, 1), a = a_min + ahat exp(sum_{k=1}^{4} sqrt(lambda_k) b_k(x) xi_k)
 *                  (Eq. diff-coeff), (lambda_k, b_k) the four largest eigenpairs of the
 *                  exponential covariance sigma0 exp(-||x - x'||_1 / delta), delta = 1/4,
 *                  sigma0 = sqrt(300); ahat = 1, a_min = 0.1.  f = 1.  N = 4.
 *   OR_Q1_3D_DISC  the same with Test 2's discontinuous ahat(xi) = 1, 100, 10 for
 *                  r < d/4, d/4 <= r < d/2, r >= d/2 (r = ||xi||_2, d = sqrt(3)).
 * phi_k are products of sines sin(m pi x_d); the mode lists are in problem.c.
 * The log-coefficient form follows Eq. (diff-coeff); the tensor forms are the
 * anisotropic A(x, y) of Section 2.1 / Section 4.
 */
#ifndef ORACLE_H
#define ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { OR_FD5_LOGKL = 1, OR_Q1_ROT = 2, OR_FD7_AXIS = 3, OR_Q1_3D_KL = 4, OR_Q1_3D_DISC = 5 };

/* Per-sample PCG outcome codes. */
enum { OR_CONVERGED = 0, OR_MAXIT = 1, OR_BREAKDOWN = 2, OR_BADINPUT = 3 };

/* ---- problem.c ---------------------------------------------------------- */
int  or_problem_size(int kind, int n, int *J, int64_t *nnz);
int  or_pattern(int kind, int n, int64_t *rowptr, int32_t *colidx);
/* One sample: matrix values in the pattern's order and the load vector. */
int  or_assemble(int kind, int n, int nparam, double aniso, const double *xi,
                 const int64_t *rowptr, const int32_t *colidx,
                 double *vals, double *b);
/* The diffusion tensor at one point (row-major d x d); used by the tests'
 * manufactured-solution and eigenvalue checks through its effect only. */
int  or_tensor(int kind, int nparam, double aniso, const double *xi,
               const double *x, double *K);
double or_param_indicator(int kind, int n, int nparam, double aniso, const double *xi);
/* The exponential-covariance KL eigenpairs of OR_Q1_3D_*: the 1-D root w and
 * eigenvalue of the first even (which = 0) or odd (which = 1) mode of
 * exp(-|s - t| / delta) on [0, 1]; the 3-D eigenvalue lambda_k and mode b_k(x)
 * of parameter k = 1..4 (covariance scale sigma0 included). */
int    or_kl_1d(int which, double *w, double *lambda);
double or_kl_lambda(int k);
double or_kl_mode(int k, const double *x);

/* ---- mg.c: multigrid V-cycle preconditioner of the trilinear problems ---- */
#define OR_MG_MAXLEV 8
/* Levels of the hierarchy for n interior nodes per axis (n = 2^k - 1, k >= 2):
 * writes ns[0..L-1] (n, (n-1)/2, ..., 3) and returns L, or -1. */
int    or_mg_levels(int n, int *ns);
/* A_c = P^T A_f P in the 27-point pattern of the coarse level (nf = 2 nc + 1). */
int    or_mg_galerkin(int nf, const int64_t *rpf, const int32_t *cif, const double *vf,
                      int nc, const int64_t *rpc, const int32_t *cic, double *vc);
void   or_mg_prolong(int nf, int nc, const double *ec, double *ef);   /* ef = P ec */
void   or_mg_restrict(int nf, int nc, const double *rf, double *rc);  /* rc = P^T rf */
/* Gershgorin bound max_i sum_j |a_ij| / a_ii of D^-1 A; NaN if a row's ratio
 * is not finite and positive. */
double or_gershgorin(int J, const int64_t *rp, const int32_t *ci, const double *v);
/* Degree-2 Chebyshev smoothing of A x = b from the x given, on [lmax/30, lmax]. */
void   or_cheb(int J, const int64_t *rp, const int32_t *ci, const double *v, const double *dinv,
               double lmax, const double *b, double *x);
/* Level `level`'s Galerkin values and Gershgorin bound of the hierarchy built
 * from the fine matrix (n per axis, the OR_Q1_3D pattern). */
int    or_mg_coarse(int n, const int64_t *rp, const int32_t *ci, const double *v, int level,
                    double *vc, double *lmax);
/* z = one V-cycle applied to r. */
int    or_mg_apply(int n, const int64_t *rp, const int32_t *ci, const double *v, const double *r,
                   double *z);
/* CG preconditioned by one V-cycle per iteration; conventions of or_pcg. */
int    or_mgpcg(int n, const int64_t *rp, const int32_t *ci, const double *v, const double *b,
                double rtol, int maxit, double *x, int *iters, double *relres);

/* The same V-cycle run in float on the hierarchy rounded to float (r rounded
 * in, z widened out), and CG (in FP64) preconditioned by it. */
int    or_mg_apply32(int n, const int64_t *rp, const int32_t *ci, const double *v, const double *r,
                     double *z);
int    or_mgpcg32(int n, const int64_t *rp, const int32_t *ci, const double *v, const double *b,
                  double rtol, int maxit, double *x, int *iters, double *relres);

/* ---- pcg.c -------------------------------------------------------------- */
void or_spmv(int J, const int64_t *rowptr, const int32_t *colidx,
             const double *vals, const double *x, double *y);
int  or_jacobi(int J, const int64_t *rowptr, const int32_t *colidx,
               const double *vals, double *dinv);
int  or_pcg(int J, const int64_t *rowptr, const int32_t *colidx,
            const double *vals, const double *b, double rtol, int maxit,
            double *x, int *iters, double *relres);
/* or_pcg that also records ||r_k|| / ||b|| after every update k in hist[k - 1]
 * (hist holds maxit entries; rtol = 0 runs all maxit iterations). */
int  or_pcg_history(int J, const int64_t *rowptr, const int32_t *colidx,
                    const double *vals, const double *b, double rtol, int maxit,
                    double *x, int *iters, double *relres, double *hist);
/* Assemble + solve M samples, one sample per thread at a time. */
int  or_solve_batch(int kind, int n, int nparam, double aniso, int M,
                    const double *xi, double rtol, int maxit, int nthreads,
                    int *iters, int *status, double *relres, double *G,
                    double *xout /* [M][J] or NULL */);
/* Mixed precision: FP32 inner Jacobi-PCG inside FP64 iterative refinement. */
int  or_pcg_ir(int J, const int64_t *rowptr, const int32_t *colidx,
               const double *vals, const double *b, double rtol_outer,
               double rtol_inner, int maxit_inner, int maxit_outer,
               double *x, int *outer_its, int *inner_its, double *relres);
/* Adjoint gradient of Q = w^T u for the FD kinds. */
int  or_adjoint_grad(int kind, int n, int nparam, double aniso, const double *xi,
                     const double *w, double rtol, int maxit,
                     double *Q, double *grad, int *iters_fwd, int *iters_adj);

/* ---- sgrid.c ------------------------------------------------------------ */
double or_sg_coord(int l, int64_t i);
double or_hat(int l, int64_t i, double y);
void   or_sg_points(int N, int M, const int8_t *lvl, const int32_t *idx, double *y);
void   or_sg_eval(int N, int M, const int8_t *lvl, const int32_t *idx,
                  const double *surplus, int Q, const double *yq, double *out);
int    or_sg_initial(int N, int level, int max_out, int8_t *lvl, int32_t *idx);
int    or_sg_refine(int N, int M, const int8_t *lvl, const int32_t *idx,
                    int first, const double *surplus, double tau, int max_level,
                    int max_out, int8_t *out_lvl, int32_t *out_idx);
void   or_sort_perm(int M, const double *keys, int32_t *perm);
double or_work_ratio(int S, int M, const int32_t *perm, const double *iters);

#ifdef __cplusplus
}
#endif
#endif
