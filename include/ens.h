/*
 * ens.h -- C ABI of libens: ensemble Jacobi-PCG for parametrised anisotropic
 * diffusion on one GB300 (sm_103a), with surrogate-based ensemble grouping;
 * for the 3-D trilinear problems also a multigrid-preconditioned ensemble CG.
 *
 * Method: D'Elia, Phipps, Rushdi, Ebeida, "Surrogate-based Ensemble Grouping
 * Strategies for Embedded Sampling-based Uncertainty Quantification"
 * (arXiv 1705.02003).  Each entry point cites the passage that defines what it
 * computes.
 *
 * Conventions for every call
 *   - Pointers are DEVICE memory owned by the caller unless marked (host).
 *     The library never frees or keeps caller memory beyond the call.
 *   - `stream` is a cudaStream_t (passed as void*); work is queued on it and the
 *     call returns without waiting unless the entry point says otherwise.
 *   - Layout of ensemble data ("commuted Kronecker" order, Eq. discrete-comm-kron-sys):
 *       matrix values  vals[E][nnz][S]   -- lane (sample) index fastest
 *       vectors        v[E][J][S]
 *       per-lane data  a[E][S]
 *     E ensembles of S samples share one CSR graph (rowptr[J+1], colidx[nnz],
 *     int32, rows sorted by column).  S must be 1, 2, 4, 8, 16, 32 or 64.
 *   - Return value: ENS_OK (0) or a negative ENS_E* code; the handle keeps a
 *     message (ens_last_error).  No entry point aborts, traps or spins without
 *     a bound.  Per-sample outcomes are reported in status[] (ENS_LANE_*).
 */
#ifndef ENS_H
#define ENS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ENS_VERSION 1

enum {
    ENS_OK = 0,
    ENS_EINVAL = -1,   /* bad argument: null pointer, size, S not supported, ... */
    ENS_ECUDA = -2,    /* a CUDA runtime error; message in ens_last_error */
    ENS_ENOMEM = -3,   /* caller workspace smaller than the *_workspace_size answer */
    ENS_ETIMEOUT = -4, /* a bounded device-side wait gave up */
    ENS_ENOTSUP = -5   /* combination not implemented (e.g. adjoint of a finite-element problem) */
};

/* Per-sample ("lane") outcome of a solve. */
enum {
    ENS_LANE_CONVERGED = 0, /* ||r||_2 <= rtol ||b||_2 reached */
    ENS_LANE_MAXIT = 1,     /* maxit iterations without convergence */
    ENS_LANE_BREAKDOWN = 2, /* p^T A p <= 0 or not finite: lane frozen, x kept */
    ENS_LANE_BADINPUT = 3,  /* b^T b or r^T D^-1 r not finite at the start */
    ENS_LANE_INACTIVE = 4   /* lane masked out by the caller (padding) */
};

/* Spatial problems: -div(A(x, xi) grad u) = f on the unit square/cube,
 * u = 0 on the boundary (Eq. elliptic-SPDE), with the tensor A built from
 * the log-form coefficient of Eq. (diff-coeff).  h = 1/(n+1); unknowns are
 * the n^d interior nodes in lexicographic order, x fastest.
 *   ENS_FD5_LOGKL  2-D 5-point FD, A = exp(0.5 sum_{k=1}^{N-1} xi_{k+1} phi_k / k)
 *                  diag(1, 10^(aniso xi_1)), f = 1; 2 <= N <= 8.
 *                  phi_k = sin(a pi x) sin(b pi y), (a,b) = (1,1), (2,1), (1,2),
 *                  (2,2), (3,1), (1,3), (3,2).  Face coefficients at face midpoints.
 *   ENS_Q1_ROT     2-D bilinear FEM (9-point), A = a R(t) diag(1, 10^(aniso xi_1)) R(t)^T,
 *                  t = pi/4 (1 + xi_3), log a = 0.5 (xi_2 phi_1 + xi_4 phi_2 / 2), f = 1;
 *                  N = 4.  Tensor at element centroids, exact element stiffness.
 *   ENS_FD7_AXIS   3-D 7-point FD, A = diag(1, 10^(aniso xi_1), 10^(aniso xi_2))
 *                  exp(0.3 sum_{k=3}^{6} xi_k phi_k), phi = sin(a pi x) sin(b pi y) sin(c pi z),
 *                  (a,b,c) = (1,1,1), (2,1,1), (1,2,1), (1,1,2); f = 1; N = 6.
 *   ENS_Q1_3D_KL   the problem of Section 4, Test 1: 3-D trilinear FEM (27-point) on
 *                  (n+1)^3 cells, A = diag(a, 1, 1) at element centroids,
 *                  a = 0.1 + exp(sum_{k=1}^{4} sqrt(lambda_k) b_k(x) xi_k) (Eq. diff-coeff),
 *                  (lambda_k, b_k) the four largest eigenpairs of the exponential
 *                  covariance sqrt(300) exp(-||x - x'||_1 / (1/4)) on [0,1]^3 (products of
 *                  the first even 1-D mode e and odd mode o: eee, oee, eoe, eeo);
 *                  f = 1 (b = h^3); N = 4; aniso unused.
 *   ENS_Q1_3D_DISC Section 4, Test 2: the same with ahat(xi) exp(...) in place of
 *                  exp(...), ahat = 1, 100, 10 for ||xi||_2 < sqrt(3)/4, < sqrt(3)/2, >=. */
enum { ENS_FD5_LOGKL = 1, ENS_Q1_ROT = 2, ENS_FD7_AXIS = 3, ENS_Q1_3D_KL = 4, ENS_Q1_3D_DISC = 5 };

typedef struct {
    int kind;     /* ENS_FD5_LOGKL | ENS_Q1_ROT | ENS_FD7_AXIS | ENS_Q1_3D_KL | ENS_Q1_3D_DISC */
    int n;        /* interior nodes per axis, >= 2 */
    int nparam;   /* N, random parameters per sample */
    double aniso; /* exponent scale of the axis anisotropy */
} ens_problem;

typedef struct ens_ctx *ens_handle;

/* Create a handle bound to CUDA device `device` (it becomes current for the
 * calling thread).  The handle owns a private capture stream, one device word
 * for the graph check (ens_check_pattern), the scratch of the device-wide sort
 * (allocated only when a grouping has more than 16384 points) and a cache of
 * at most 32 instantiated CUDA graphs (keyed by every pointer and size of a
 * solve, least recently used evicted first); it is not thread-safe.
 * ens_destroy releases all of them.  Environment variables read here: ENS_PCG_HOST_LOOP,
 * ENS_PCG_BRANCHES, ENS_PCG_FUSED, ENS_CHECK (see ens_pcg_solve,
 * ens_pcg_branches, ens_pcg_cluster_size, ens_check_pattern). */
int ens_create(ens_handle *h, int device);
int ens_destroy(ens_handle h);
/* (host) message of the last failed call on this handle; never NULL. */
const char *ens_last_error(ens_handle h);

/* (host) J and nnz of the problem's graph.  No device work. */
int ens_problem_size(const ens_problem *p, int *J, int64_t *nnz);

/* The shared sparsity graph of Eqs. (discrete-sys)/(discrete-comm-kron-sys):
 * writes rowptr[J+1] and colidx[nnz] (device, int32). */
int ens_pattern(ens_handle h, const ens_problem *p, int32_t *rowptr, int32_t *colidx,
                void *stream);

/* Ensemble assembly (Section 2.3, "storing each nonzero entry as a length-S
 * array"): for E ensembles of S samples with parameters xi[E][S][nparam]
 * (device, f64), writes the sample-interleaved values vals[E][nnz][S]
 * (f64, or f32 when vals_f32 != 0), the Jacobi inverse diagonal dinv[E][J][S]
 * and the load b[E][J][S] (both f64; either may be NULL).  A NaN parameter
 * gives NaN values in its lane only. */
int ens_assemble(ens_handle h, const ens_problem *p, int S, int E, const double *xi,
                 const int32_t *rowptr, const int32_t *colidx, void *vals, int vals_f32,
                 double *dinv, double *b, void *stream);

/* Parameter-based grouping indicator (Section 3.2, Eq. pb-indicator), the
 * comparator of the surrogate grouping: for M samples xi[M][nparam] (device),
 * H[m] = max over the points where the tensor is evaluated (FD face midpoints,
 * Q1 element centroids) of lambda_max(A(x, xi_m)) / lambda_min(A(x, xi_m)).
 * Sorting by H (ens_sort_chunk) gives the "par" grouping. */
int ens_param_indicator(ens_handle h, const ens_problem *p, int M, const double *xi, double *H,
                        void *stream);

/* Validate a CSR graph (no counterpart in the paper: a guard of this
 * library).  Checks rowptr[0] == 0, rowptr[J] == nnz, rowptr non-decreasing
 * with every entry in [0, nnz], and every colidx entry in [0, J); reads only
 * rowptr[0..J] and colidx[0..nnz).  Returns ENS_OK, or ENS_EINVAL with the
 * failed checks in ens_last_error.  Synchronises `stream`.  With the
 * environment variable ENS_CHECK=1 at ens_create, ens_pcg_solve,
 * ens_pcg_solve_ir, ens_pcg_solve_static and ens_spmv run this check on their
 * graph first and return its error without launching anything else. */
int ens_check_pattern(ens_handle h, int J, int64_t nnz, const int32_t *rowptr, const int32_t *colidx,
                      void *stream);

/* Number of independent loop branches ens_pcg_solve runs for E ensembles
 * (no counterpart in the paper: a scheduling choice of this library): one per
 * ensemble up to 16, or the value of the environment variable
 * ENS_PCG_BRANCHES (n >= 1, capped at 16 and at E) read at ens_create; 1 in
 * the host-loop mode.  Returns 0 for a NULL handle or E <= 0. */
int ens_pcg_branches(ens_handle h, int E);

/* Thread-block cluster size of the one-launch schedule ens_pcg_solve uses for
 * this problem, or 0 where it runs the graph loop described there (no
 * counterpart in the paper: a scheduling choice of this library).  Problems of
 * at most 1024 unknowns (16 row tiles of 64) with S <= 32 take the one-launch
 * schedule when the device holds all E clusters at once and a CTA's FP64 work
 * per CG trip, 64 S (nnz/J + 7) multiply-adds, is at most 26000: one cluster of
 * one CTA per row tile runs the start, every CG trip and the finish of its
 * ensemble in a single kernel, with cluster barriers instead of kernel
 * boundaries.  The environment variable ENS_PCG_FUSED at ens_create selects 0
 * (never) or 2 (also past the work bound); it is not used in the host-loop
 * mode.  May query the device (cluster occupancy, once per kernel and layout);
 * no device work.  Returns 0 for a NULL handle or invalid sizes. */
int ens_pcg_cluster_size(ens_handle h, int J, int64_t nnz, int S, int E);

/* Bytes of caller workspace ens_pcg_solve needs (device memory, 256-byte aligned). */
size_t ens_pcg_workspace_size(int J, int64_t nnz, int S, int E);

/* Ensemble Jacobi-PCG with per-sample inner products and norms (Section 2.3:
 * the ensemble inner product is taken per component so each sample converges
 * at its own rate; Section 4: per-sample convergence record and the zero
 * A-conjugate-norm guard).  Solves A_s x_s = b_s for every active lane s of
 * every ensemble, from x = 0, to ||r_s||_2 <= rtol ||b_s||_2 on the
 * recursively updated residual; a converged, broken-down or maxit lane is
 * frozen (no further updates) while the others continue.
 *   active[E][S]  (device u8, may be NULL = all active) 0 marks a padding lane.
 *   x[E][J][S]    output (written for every lane; 0 for inactive lanes).
 *   iters[E][S], relres[E][S], status[E][S]  outputs (relres = ||r||/||b||).
 *   work          caller scratch of at least ens_pcg_workspace_size bytes.
 * The iteration runs inside one CUDA graph of ens_pcg_branches(h, E) device-
 * evaluated while loops side by side, each over a contiguous range of the
 * ensembles and at most maxit trips, so the call does not synchronise the
 * stream and each range of ensembles stops on its own.  With the environment
 * variable ENS_PCG_HOST_LOOP=1 at ens_create, the same kernels are instead
 * launched from the host, which reads the live-lane count back every 16 trips
 * (a profiling aid: kernel profilers do not see kernels inside a conditional
 * graph body).  Problems of at most 1024 unknowns instead run as one kernel
 * launch (ens_pcg_cluster_size).  Results do not depend on any of these
 * choices, bit for bit: every schedule performs the same operations in the
 * same order.  A lane's results do not depend on E, on its position or on the
 * other lanes either, with one exception: for one-lane ensembles (S = 1) on
 * problems of more than 4096 unknowns, a call with E J >= 1,867,776 (three
 * 4096-row blocks per SM of 152) uses 4096-row tiles instead of 256-row ones,
 * so a sample's rounding then depends on the size of its batch (the tile
 * sets the order of its inner-product sums). */
int ens_pcg_solve(ens_handle h, int J, int64_t nnz, int S, int E,
                  const int32_t *rowptr, const int32_t *colidx, const double *vals,
                  const double *dinv, const double *b, double *x, const uint8_t *active,
                  double rtol, int maxit, int32_t *iters, double *relres, int32_t *status,
                  void *work, size_t work_bytes, void *stream);

/* ---- Multigrid-preconditioned ensemble CG (the trilinear problems) --------
 * Section 4 preconditions CG with multigrid (a Chebyshev-smoothed hierarchy,
 * coarsest level solved directly), instantiated on the ensemble scalar.  For
 * ENS_Q1_3D_KL / ENS_Q1_3D_DISC with n = 2^k - 1 (k >= 2) interior nodes per
 * axis this library builds the nested trilinear hierarchy per sample:
 * levels n, (n-1)/2, ..., 3; P = trilinear interpolation; coarse operators
 * P^T A P (Galerkin); a degree-2 Chebyshev smoother on D^-1 A over
 * [lambda/30, lambda], lambda the sample's Gershgorin bound
 * max_i sum_j |a_ij| / a_ii; a dense Cholesky solve on the 27-unknown coarsest
 * level; one V-cycle (pre-smooth, coarse correction, post-smooth) per CG
 * iteration.  Other kinds or sizes: ENS_ENOTSUP / ENS_EINVAL. */

/* Mixed precision (`mixed` = 1; 0 = FP64 throughout): the hierarchy is built
 * in FP64 as described, then rounded once to float, and every V-cycle runs in
 * float (r rounded in, z widened out); CG, its inner products, residual test
 * and iterate stay FP64.  Each lane's r is scaled by a power of two that puts
 * its largest entry in [1, 2) before the rounding and z is scaled back (exact,
 * and the V-cycle commutes with it), so any lane magnitude FP64 represents
 * stays inside float's range; entries more than 2^125 below a lane's largest
 * round to zero.  The preconditioner only approximates A^-1, so its
 * rounding changes the iteration counts little (the FP32 and FP64 V-cycles
 * differ by ~2e-7 relative).  Every call on one workspace uses the same p, S,
 * E and `mixed` (the layout depends on them): the handle records them at
 * ens_mg_setup (for its last 16 workspaces), and ens_mg_level, ens_mg_apply and
 * ens_mgpcg_solve on such a workspace with other values return ENS_EINVAL.
 *
 * Bytes of caller workspace the calls below need (0 when unsupported). */
size_t ens_mg_workspace_size(const ens_problem *p, int S, int E, int mixed);

/* Build the hierarchy of E ensembles from the fine values vals[E][nnz][S]
 * (device f64; rowptr/colidx the problem's graph from ens_pattern) into work:
 * coarse graphs and Galerkin values, inverse diagonals, Gershgorin bounds and
 * Chebyshev coefficients of every level, the coarsest level's factor.  A lane
 * whose row ratios are not all finite and positive, or whose coarsest
 * factorisation meets a non-positive pivot, is marked unusable (its solve
 * reports ENS_LANE_BADINPUT).  The products, sums and roots of the setup are
 * each rounded on their own, in the order of the definitions, so the coarse
 * values match a plain host computation bit for bit.  No synchronisation. */
int ens_mg_setup(ens_handle h, const ens_problem *p, int S, int E, int mixed, const int32_t *rowptr,
                 const int32_t *colidx, const double *vals, void *work, size_t work_bytes,
                 void *stream);

/* Copy level `level` of the hierarchy in `work` out (device, f64): its Galerkin
 * values vals_out[E][nnz_l][S] (levels >= 1; level 0 is the caller's own) and
 * the Gershgorin bounds lmax_out[E][S] (0 for an unusable lane).  Either may
 * be NULL.  An inspection aid (no counterpart in the paper). */
int ens_mg_level(ens_handle h, const ens_problem *p, int S, int E, int mixed, int level,
                 double *vals_out, double *lmax_out, const void *work, size_t work_bytes, void *stream);

/* z[E][J][S] = one V-cycle applied to r[E][J][S] (device f64) with the
 * hierarchy of the last ens_mg_setup on `work` (same p, S, E and vals: the
 * workspace layout depends on them).  Lanes marked unusable get undefined
 * values.  No synchronisation. */
int ens_mg_apply(ens_handle h, const ens_problem *p, int S, int E, int mixed, const int32_t *rowptr,
                 const int32_t *colidx, const double *vals, const double *r, double *z,
                 void *work, size_t work_bytes, void *stream);

/* CG preconditioned by one V-cycle per iteration, with the conventions and
 * outputs of ens_pcg_solve (x = 0 start, per-sample inner products, the
 * unpreconditioned ||r_s|| <= rtol ||b_s|| test after each update, frozen lanes,
 * status codes; active may be NULL).  Needs ens_mg_setup on `work` with the
 * same p, S, E and vals first.  The host launches the iterations and reads the live-lane
 * count back every two to four of them (the call synchronises the stream);
 * each lane still stops at its own iteration, so results do not depend on that
 * cadence.  Deterministic: per-lane results depend only on the lane's data, S
 * and J. */
int ens_mgpcg_solve(ens_handle h, const ens_problem *p, int S, int E, int mixed, const int32_t *rowptr,
                    const int32_t *colidx, const double *vals, const double *b, double *x,
                    const uint8_t *active, double rtol, int maxit, int32_t *iters, double *relres,
                    int32_t *status, void *work, size_t work_bytes, void *stream);

/* Bytes of caller workspace ens_solve_stream needs (0 for bad arguments). */
size_t ens_stream_workspace_size(const ens_problem *p, int S, int E);

/* Continuous ensemble batching (the batching layer; the paper solves fixed
 * ensembles one after another, Section 4).  M samples xi[M][nparam] (device)
 * run through a pool of E ensembles of S lanes, in the queue order order[M]
 * (device int32 permutation; NULL = 0, 1, ...).  The device while loop runs
 * `chunk` trips at a time; after each chunk every lane that has frozen
 * (converged, maxit, breakdown) returns its outcome by sample index and takes
 * the next queued sample: only that lane's values are assembled and only its
 * CG state restarts, while the other lanes keep iterating.  When the queue is
 * empty the live lanes are re-packed into as few ensembles as hold them.
 * Each sample's iteration and result are those of ens_pcg_solve for it.
 * Outputs by sample: iters[M], status[M], relres[M], and qoi[M] (may be NULL)
 * = ||u||_2^2, or w^T u when w[J] (device) is given.  The graph, values,
 * vectors and lane state live in the caller's workspace
 * (ens_stream_workspace_size).  Synchronises `stream` once per chunk. */
int ens_solve_stream(ens_handle h, const ens_problem *p, int S, int E, int M, const double *xi,
                     const int32_t *order, const double *w, double rtol, int maxit, int chunk,
                     int32_t *iters, int32_t *status, double *relres, double *qoi, void *work,
                     size_t work_bytes, void *stream);

/* Bytes of caller workspace ens_adjoint_grad needs (0 for bad arguments). */
size_t ens_adjoint_workspace_size(const ens_problem *p, int S, int E);

/* Adjoint gradient of a linear quantity of interest (the differentiation
 * layer; the paper's QoI G_u of Section 2.1 is such a functional).  With
 * u[E][J][S] the solutions of A(xi) u = b and lam[E][J][S] those of the adjoint
 * A(xi) lam = w (A is symmetric; b does not depend on xi), writes
 *   grad[E][S][nparam] = dQ/dxi = -lam^T (dA/dxi) u,   Q = w^T u,
 * summed face by face over the FD operator (FD5 and FD7 problems only;
 * ENS_ENOTSUP for the finite-element problems).  xi[E][S][nparam] as for ens_assemble.  Deterministic:
 * fixed per-lane summation order. */
int ens_adjoint_grad(ens_handle h, const ens_problem *p, int S, int E, const double *xi,
                     const double *u, const double *lam, double *grad, void *work,
                     size_t work_bytes, void *stream);

/* Bytes of caller workspace ens_adjoint_solve_grad needs (0 for bad arguments
 * or a finite-element problem). */
size_t ens_adjoint_solve_workspace_size(const ens_problem *p, int S, int E);

/* The adjoint solve and the gradient in one call: given the forward solutions
 * u[E][J][S] of A(xi) u = b (ens_pcg_solve), assembles A(xi) (ens_assemble),
 * solves the adjoint systems A(xi) lam = w for every active lane by the
 * ensemble Jacobi-PCG of ens_pcg_solve (x = 0 start, rtol, maxit, frozen lanes,
 * per-lane status), and writes
 *   Q[E][S] = w^T u (ens_qoi with weights),
 *   grad[E][S][nparam] = dQ/dxi = -lam^T (dA/dxi) u (ens_adjoint_grad),
 *   lam[E][J][S], iters[E][S], relres[E][S], status[E][S] of the adjoint solve.
 * w[J] (device) is the functional's weight vector; active as for ens_pcg_solve
 * (NULL = all lanes).  The assembled values, the adjoint right-hand side and
 * the solver's scratch live in work (ens_adjoint_solve_workspace_size bytes).
 * FD5 and FD7 problems only (ENS_ENOTSUP otherwise).  No synchronisation. */
int ens_adjoint_solve_grad(ens_handle h, const ens_problem *p, int S, int E, const double *xi,
                           const int32_t *rowptr, const int32_t *colidx, const double *u,
                           const double *w, const uint8_t *active, double rtol, int maxit, double *Q,
                           double *grad, double *lam, int32_t *iters, double *relres, int32_t *status,
                           void *work, size_t work_bytes, void *stream);

/* Bytes of caller workspace ens_pcg_solve_ir needs. */
size_t ens_pcg_ir_workspace_size(int J, int64_t nnz, int S, int E);

/* Mixed precision: FP32 matrix values and inner Jacobi-PCG inside FP64
 * iterative refinement (the precision layer; the paper solves in FP64
 * throughout, Section 4).  Per lane: x = 0; then repeatedly
 *   r = b - A x with the FP64 values `vals` (FP64 residual and norm);
 *   stop when ||r||_2 <= rtol ||b||_2 (status CONVERGED), or after maxit_outer
 *   corrections (MAXIT);
 *   solve A32 d = r with the FP32 values `vals32` (ens_assemble with
 *   vals_f32 = 1) by the same ensemble Jacobi-PCG, FP32 vectors but FP64 inner
 *   products, norms and CG scalars, to ||r - A32 d|| <= rtol_inner ||r|| or
 *   maxit_inner iterations;
 *   x = x + d in FP64.
 * A lane whose inner solve cannot make progress (breakdown before its first
 * update, or a non-finite residual) stops with status BREAKDOWN.
 * Outputs: x[E][J][S], iters[E][S] = inner iterations summed over the
 * corrections, outer_its[E][S] = corrections applied, relres[E][S] = the FP64
 * relative residual ||b - A x|| / ||b|| of the returned x, status[E][S].
 * The host reads the live-lane count back once per correction, so the call
 * synchronises `stream`. */
int ens_pcg_solve_ir(ens_handle h, int J, int64_t nnz, int S, int E,
                     const int32_t *rowptr, const int32_t *colidx, const double *vals,
                     const float *vals32, const double *dinv, const double *b, double *x,
                     const uint8_t *active, double rtol, double rtol_inner, int maxit_inner,
                     int maxit_outer, int32_t *iters, int32_t *outer_its, double *relres,
                     int32_t *status, void *work, size_t work_bytes, void *stream);

/* The same solve for callers that cannot allocate device memory.  The paper
 * has no counterpart: this exists for code that must not call cudaMalloc --
 * for example code running under an allocator that owns all device memory, or
 * a plug-in that may not create or grow device allocations -- and so cannot
 * provide the `work` buffer of ens_pcg_solve.  Its scratch is a file-scope
 * device array of ENS_PCG_STATIC_SCRATCH_BYTES (8 MiB), which every GPU that
 * loads the library holds until the process exits; a problem whose workspace
 * (ens_pcg_workspace_size) exceeds it is rejected with ENS_EINVAL and a message.
 * The caller still provides every input and output, as for ens_pcg_solve.
 *   - It runs on the calling thread's current device.  Its first call on a
 *     device looks up the array's device address there (once per device);
 *     make that first call before any stream capture.  The address is kept
 *     for the life of the process: after cudaDeviceReset on a device (which
 *     unloads the library's device code there) this entry point must not be
 *     called on that device again.
 *   - It calls no cudaMalloc, cudaFree or allocating library routine, and
 *     instantiates no CUDA graph: the iteration is launched from the host,
 *     which reads the live-lane count back every 16 trips (so the call
 *     synchronises `stream`).
 *   - Every call shares the one array: calls that overlap on the GPU (other
 *     streams, other threads) race and must not be issued; the array keeps the
 *     previous call's contents, and the call clears what must start at zero.
 *   - h may be NULL (then no message is kept). */
#define ENS_PCG_STATIC_SCRATCH_BYTES ((size_t)8 << 20)
int ens_pcg_solve_static(ens_handle h, int J, int64_t nnz, int S, int E,
                         const int32_t *rowptr, const int32_t *colidx, const double *vals,
                         const double *dinv, const double *b, double *x, const uint8_t *active,
                         double rtol, int maxit, int32_t *iters, double *relres, int32_t *status,
                         void *stream);

/* Ensemble SpMV (Section 2.3: the matrix-vector product of the commuted
 * Kronecker system, each nonzero's S values applied to the S lanes of its
 * column): q[E][J][S] = A_s p_s for every lane, and pq[E][S] = p_s^T q_s
 * (device, may be NULL).  This is the same kernel the PCG loop runs (K2),
 * launched alone; work as for ens_pcg_solve. */
int ens_spmv(ens_handle h, int J, int64_t nnz, int S, int E, const int32_t *rowptr,
             const int32_t *colidx, const double *vals, const double *p, double *q, double *pq,
             void *work, size_t work_bytes, void *stream);

/* Surrogate-based grouping (Section 3.1, "SGS-based grouping", Eq. SGSiterations):
 * evaluates the hierarchical piecewise-linear sparse-grid surrogate
 *   pred[q] = sum_{m<M} surplus[m] prod_n psi_{lvl[m][n], idx[m][n]}(yq[q][n])
 * (hat basis of Section 2.2, summed in m order) at Mq points yq[Mq][N], then
 * returns perm[Mq], the stable ascending order of pred (ties keep index order),
 * which cut into consecutive runs of S forms the ensembles; *n_ens (host) =
 * ceil(Mq / S), the last ensemble padded.  M may be 0 (pred = 0, identity).
 * lvl[M][N] int8, idx[M][N] int32, surplus[M] f64: device.  Mq <= 2^26.  Up to
 * 16384 points the sort runs in one thread block; above that it runs over the
 * whole GPU on scratch the handle owns, allocated (or grown) on first use,
 * which synchronises `stream` once.  Both give the same permutation. */
int ens_group(ens_handle h, int N, int M, const int8_t *lvl, const int32_t *idx,
              const double *surplus, int Mq, const double *yq, int S, double *pred,
              int32_t *perm, int *n_ens, void *stream);

/* The surrogate alone (Eq. SGSiterations / SGSoutput), same arithmetic as
 * ens_group: out[q] = sum_m surplus[m] psi_m(yq[q]).  When values[Mq]
 * (device) is given, out[q] = values[q] - that sum instead: the hierarchical
 * surplus of Eq. (hierSGint) of a new point, because every basis function of a
 * point at the same or a finer level vanishes there (the triangularity noted
 * beside the hierarchisation system). */
int ens_sg_eval(ens_handle h, int N, int M, const int8_t *lvl, const int32_t *idx,
                const double *surplus, int Mq, const double *yq, const double *values,
                double *out, void *stream);

/* Per-sample quantity of interest of a solution x[E][J][S] (device):
 *   w == NULL:  out[e][s] = sum_j x[e][j][s]^2      (G = ||u||_l2^2, Section 4)
 *   w != NULL:  out[e][s] = sum_j w[j] x[e][j][s]   (a weighted mean, e.g. G_u of
 *                                                   Section 2.1 over a region)
 * Each ensemble is summed by one block in a fixed order (deterministic). */
int ens_qoi(ens_handle h, int J, int S, int E, const double *x, const double *w, double *out,
            void *stream);

/* The sort-and-chunk step of ens_group alone, on caller keys[Mq] (device):
 * used for the natural (identity keys), random and iteration-sorted groupings.
 * Numbers ascend, NaN keys come last, ties keep index order; Mq <= 2^26, with
 * the same one-block / device-wide split as ens_group. */
int ens_sort_chunk(ens_handle h, int Mq, const double *keys, int S, int32_t *perm, int *n_ens,
                   void *stream);

/* (host) Classic adaptive refinement (Section 2.2, "Adaptivity"): every point
 * m in [first, M) with |surplus[m]| >= tau gets its children -- per dimension
 * n, (0,i) -> (1,1) and (l,i) -> (l+1, 2i-1), (l+1, 2i+1) for l >= 1 -- unless
 * the child is already in the grid or already listed, or its level sum
 * exceeds max_level.  Writes up to max_out children to out_lvl/out_idx (host,
 * [.][N]) in generation order and returns their count, or a negative code.
 * All arrays host memory. */
int ens_sg_refine(int N, int M, const int8_t *lvl, const int32_t *idx, int first,
                  const double *surplus, double tau, int max_level, int max_out,
                  int8_t *out_lvl, int32_t *out_idx);

/* (host) The full sparse grid of levels 0..level (Section 2.2, Z_l with
 * alpha(l) = |l|): the 2^N corners (corner c has i_n = bit n of c), then
 * `level` refinement rounds of every newest point.  Returns the count. */
int ens_sg_initial(int N, int level, int max_out, int8_t *lvl, int32_t *idx);

/* (host) Coordinates of M grid points (Section 2.2, the 1-D points
 * y_{l,i} = i 2^(1-l) - 1 of the hierarchical basis, taken per dimension):
 * y[m][n] = idx[m][n] 2^(1 - lvl[m][n]) - 1, exact (dyadic).  lvl[M][N],
 * idx[M][N] and y[M][N] are host memory; ENS_EINVAL for a level outside
 * [0, 62] or a NULL array with M > 0. */
int ens_sg_points(int N, int M, const int8_t *lvl, const int32_t *idx, double *y);

/* Measurement aid (no counterpart in the paper): the FP64 issue rate, which
 * bounds the ensemble SpMV and the PCG vector kernels on GB300.  Launches
 * `blocks` blocks of 256 threads, each thread running eight independent FP64
 * fused multiply-add recurrences for `iters` steps, on `stream`; sink[blocks]
 * (device f64) is written only in a case that never occurs (it keeps the
 * work from being optimised away).  Time the launch with events on `stream`;
 * ens_fp64_peak_flops gives its floating-point operations (2 per fused
 * multiply-add). */
int ens_fp64_peak(ens_handle h, int blocks, int iters, double *sink, void *stream);
double ens_fp64_peak_flops(int blocks, int iters);

#ifdef __cplusplus
}
#endif
#endif /* ENS_H */
