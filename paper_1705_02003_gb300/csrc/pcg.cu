// pcg.cu -- ensemble Jacobi-PCG with per-sample inner products (K2, K3, K4),
// its FP32-in-FP64 iterative-refinement form, and the stand-alone SpMV.
//
// Section 2.3: the S samples of an ensemble share one graph; their values are
// interleaved [nnz][S] and their vectors [J][S].  Inner products and norms are
// taken per sample ("ensemble inner product"), so each sample follows its own
// CG recurrence and converges at its own rate; Section 4 records when each
// sample converges and replaces the update by zero when p^T A p vanishes.
// Here a sample that converges, breaks down or reaches maxit is frozen: its
// lane is skipped by every later kernel, so its x is final and the ensemble
// result equals S independent solves.
//
// One CG iteration is three kernels, each followed by a per-lane reduction
// finished by the last block of the ensemble to arrive (fixed block order, so
// results are deterministic and independent of E and of the other lanes):
//   K2  q = A p (CSR, one column index per nonzero for all S lanes), p^T q  -> alpha
//   K3  x += alpha p, r -= alpha q, r^T r, r^T D^-1 r                       -> convergence, beta
//   K4  p = D^-1 r + beta p; block (0,0) also drives the graph's while loop.
// The kernels are templates over the value type T of the matrix and vectors:
// T = double is the FP64 method; T = float is the inner solve of the
// mixed-precision form, whose inner products, norms and CG scalars stay FP64.
//
// Arithmetic: GB300 issues about two FP64 operations per clock per SM, which
// is the binding limit of these kernels before HBM is, so every
// multiply-accumulate is one fused multiply-add (the per-row sums keep the
// oracle's column order; only the rounding of each step differs from it).
//
// The loop is one CUDA graph: a conditional WHILE node whose body holds K2-K4
// and whose condition K4 sets to (live lanes > 0 && trips < maxit), so the
// host launches one graph per solve and never waits inside it.
#include "pcg_core.cuh"

#include <cmath>
#include <cstring>
#include <mutex>

namespace ens {

using namespace pcgi;

namespace {

// Per-lane block reduction of NS sums, then the cross-block sum in the last
// block of the ensemble.  Returns true in that block, with tot[ns * S + s]
// holding the totals (shared memory).
template <class LG, int S, int NS>
__device__ bool reduce_lanes(double (&acc)[NS][LG::V], double *part_base[NS], int e, int nblk,
                             int *counter, double *tot)
{
    constexpr int V = LG::V, TPR = LG::TPR;
    __shared__ double warp_part[kBlock / 32][NS][S];
    __shared__ double grp[LG::G][NS][S];
    __shared__ int s_last;
    const int tid = threadIdx.x, wid = tid >> 5, lid = tid & 31;
#pragma unroll
    for (int ns = 0; ns < NS; ns++)
#pragma unroll
        for (int v = 0; v < V; v++)
            for (int off = 16; off >= TPR; off >>= 1)
                acc[ns][v] = dadd(acc[ns][v], __shfl_xor_sync(0xffffffffu, acc[ns][v], off));
    if (lid < TPR) {
#pragma unroll
        for (int ns = 0; ns < NS; ns++)
#pragma unroll
            for (int v = 0; v < V; v++) warp_part[wid][ns][lid * V + v] = acc[ns][v];
    }
    __syncthreads();
    if (tid < S) {
#pragma unroll
        for (int ns = 0; ns < NS; ns++) {
            double s = 0.0;
            for (int w = 0; w < kBlock / 32; w++) s = dadd(s, warp_part[w][ns][tid]);
            part_base[ns][((size_t)e * nblk + blockIdx.x) * S + tid] = s;
        }
    }
    // The barrier orders the partial writes before thread 0's fence, and the
    // fence is cumulative, so one fence publishes the whole block's partials.
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        s_last = (atomicAdd(counter, 1) == nblk - 1);
    }
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
    {
        // Partials b = g, g + G, g + 2G, ... summed in that order; the loads
        // are issued eight at a time so the tail is not one L2 round trip per term.
        constexpr int U = 8;
        const int g = tid / S, s = tid % S;
#pragma unroll
        for (int ns = 0; ns < NS; ns++) {
            double v = 0.0;
            const double *pb = part_base[ns] + (size_t)e * nblk * S + s;
            for (int b0 = g; b0 < nblk; b0 += U * LG::G) {
                double t[U];
#pragma unroll
                for (int u = 0; u < U; u++) {
                    const int b = b0 + u * LG::G;
                    t[u] = b < nblk ? __ldcg(pb + (size_t)b * S) : 0.0;
                }
#pragma unroll
                for (int u = 0; u < U; u++)
                    if (b0 + u * LG::G < nblk) v = dadd(v, t[u]);
            }
            grp[g][ns][s] = v;
        }
    }
    __syncthreads();
    {
        // The G group sums of a lane are combined pairwise, group g with
        // g + st for st = G/2, ..., 1: a fixed order with log2 G dependent
        // additions.  (One thread adding the G sums in turn cost about 50 ns
        // per addition at S = 1, where G = 256.)
        const int g = tid / S, s = tid % S;
        for (int st = LG::G / 2; st > 0; st >>= 1) {
            if (g < st) {
#pragma unroll
                for (int ns = 0; ns < NS; ns++) grp[g][ns][s] = dadd(grp[g][ns][s], grp[g + st][ns][s]);
            }
            __syncthreads();
        }
    }
    if (tid < S) {
#pragma unroll
        for (int ns = 0; ns < NS; ns++) tot[ns * S + tid] = grp[0][ns][tid];
    }
    if (tid == 0) *counter = 0;
    __syncthreads();
    return true;
}

// Freeze lane L with an outcome; called by the single thread owning L.
__device__ __forceinline__ void freeze(const Args &a, int L, int st, int iters, double relres, int *dead)
{
    a.w.live[L] = 0;
    a.status[L] = st;
    a.iters[L] = iters;
    a.relres[L] = relres;
    atomicAdd(dead, 1);
}

// Streamed arrays are passed as kernel parameters: read out of the by-value
// Args struct instead, their loads were measured to lose half of the kernel's
// memory-level parallelism on sm_103a.

// ---- K0: x = 0, r = b, p = D^-1 b; r^T r and r^T D^-1 r per lane ------------
template <typename T, int S>
__global__ void __launch_bounds__(kBlock) k_init(Args a, const double *__restrict__ bb, const T *__restrict__ dinv,
                                                 T *__restrict__ xx, T *__restrict__ rr, T *__restrict__ pp)
{
    using LG = VecGeo<T, S>;
    constexpr int V = LG::V, TPR = LG::TPR, RPP = LG::RPP;
    const int e = blockIdx.y;
    const int lane0 = (threadIdx.x % TPR) * V;
    const size_t vbase = (size_t)e * a.J * S;
    double acc[2][V] = {};
    const int r0 = blockIdx.x * a.g.RT, r1 = min(a.J, r0 + a.g.RT);
    bool rf[V], any = false, all = true;
#pragma unroll
    for (int v = 0; v < V; v++) {
        rf[v] = a.refill ? a.refill[e * S + lane0 + v] != 0 : true;
        any = any || rf[v];
        all = all && rf[v];
    }
    for (int r = r0 + threadIdx.x / TPR; any && r < r1; r += RPP) {
        size_t o = vbase + (size_t)r * S + lane0;
        Vec<T, V> dv, xv, rv, pv;
        dv.load_ro(dinv + o);
        if (!all) {  // lanes that keep running share this access: keep their values
            xv.load(xx + o);
            rv.load(rr + o);
            pv.load(pp + o);
        }
#pragma unroll
        for (int v = 0; v < V; v++) {
            if (!rf[v]) continue;
            xv.v[v] = T(0);
            rv.v[v] = (T)__ldg(bb + o + v);
            pv.v[v] = dv.v[v] * rv.v[v];
            acc[0][v] = fma(wide(rv.v[v]), wide(rv.v[v]), acc[0][v]);
            acc[1][v] = fma(wide(rv.v[v]), wide(pv.v[v]), acc[1][v]);
        }
        xv.store(xx + o);
        rv.store(rr + o);
        pv.store(pp + o);
    }
    __shared__ double tot[2 * S];
    __shared__ int live_cnt;
    if (threadIdx.x == 0) live_cnt = 0;
    double *parts[2] = {a.w.part0, a.w.part1};
    if (!reduce_lanes<LG, S, 2>(acc, parts, e, a.g.nblk, a.w.counter + e * CNT_KINDS + CNT_INIT, tot)) return;
    if (threadIdx.x < S && (!a.refill || a.refill[e * S + threadIdx.x])) {
        const int s = threadIdx.x, L = e * S + s;
        const double bsq = tot[s], rz = tot[S + s];
        const int act = a.active ? (int)a.active[L] : 1;
        a.w.k[L] = 0;
        int live = 0;
        if (!act) {
            a.status[L] = ENS_LANE_INACTIVE; a.iters[L] = 0; a.relres[L] = 0.0;
        } else if (!isfinite(bsq) || !isfinite(rz)) {
            a.status[L] = ENS_LANE_BADINPUT; a.iters[L] = 0; a.relres[L] = __longlong_as_double(0x7ff8000000000000LL);
        } else if (bsq == 0.0) {
            a.status[L] = ENS_LANE_CONVERGED; a.iters[L] = 0; a.relres[L] = 0.0;
        } else if (a.maxit <= 0) {
            a.status[L] = ENS_LANE_MAXIT; a.iters[L] = 0; a.relres[L] = 1.0;
        } else {
            live = 1;
            a.w.bnorm[L] = sqrt(bsq);
            a.w.rz[L] = rz;
            a.w.rr[L] = bsq;
            a.status[L] = ENS_LANE_MAXIT;
            a.iters[L] = 0;
            a.relres[L] = 1.0;
        }
        a.w.live[L] = live;
        if (live) atomicAdd(&live_cnt, 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (a.refill)
            a.w.ens_live[e] += live_cnt;
        else
            a.w.ens_live[e] = live_cnt;
        atomicAdd(a.w.ctl + CTL_NLIVE, live_cnt);
    }
}

// ---- K2: q = A p and p^T q per lane -> alpha -----------------------------------
constexpr int kChunk = 9;  // nonzeros loaded together per row in the refinement's FP64 residual


// CYC: the block's rows are 256-row chunks dealt in turn (block b takes chunks
// b, b + nblk, ...) instead of one run of RT rows, so the blocks resident at
// any moment cover one contiguous band of rows.  It is used for 7-point rows
// with tiles longer than one chunk: their +-n^2 neighbours then stay in L2
// (measured on 128^3: 1.20 -> 1.13 ms per launch of one ensemble).  With
// RT = 256 both mappings are the same.  The mapping is a function of J and the
// pattern only, so results still do not depend on E or on lane position.
template <typename T, int S, int V_, int KC, bool CYC = false>
__global__ void __launch_bounds__(kBlock, (SpmvOcc<S, V_, KC>::value))
    k_spmv(Args a, const int32_t *__restrict__ rowptr, const int32_t *__restrict__ colidx,
           const T *__restrict__ vals_all, const T *__restrict__ p_all, T *__restrict__ q_all)
{
    using LG = LaneGeo<S, V_>;
    constexpr int V = LG::V, TPR = LG::TPR, RPP = LG::RPP;
    const int e = blockIdx.y;
    if (a.w.ens_live[e] == 0) return;
    const int lane0 = (threadIdx.x % TPR) * V;
    const int L0 = e * S + lane0;
    bool mine = a.w.live[L0] != 0;
    if (V == 2) mine = mine || a.w.live[L0 + 1] != 0;
    double acc[1][V] = {};
    if (mine) {
        const T *__restrict__ vals = vals_all + (size_t)e * a.nnz * S + lane0;
        const T *__restrict__ p = p_all + (size_t)e * a.J * S + lane0;
        T *__restrict__ q = q_all + (size_t)e * a.J * S + lane0;
        if constexpr (CYC) {
            for (int t = threadIdx.x / TPR; t < a.g.RT; t += RPP) {
                const int r = (blockIdx.x + (t >> 8) * a.g.nblk) * 256 + (t & 255);
                if (r >= a.J) break;
                spmv_row<T, S, V, KC>(r, rowptr, colidx, vals, p, q, acc);
            }
        } else {
            const int r0 = blockIdx.x * a.g.RT, r1 = min(a.J, r0 + a.g.RT);
            for (int r = r0 + threadIdx.x / TPR; r < r1; r += RPP)
                spmv_row<T, S, V, KC>(r, rowptr, colidx, vals, p, q, acc);
        }
    }
    __shared__ double tot[S];
    __shared__ int dead;
    if (threadIdx.x == 0) dead = 0;
    double *parts[1] = {a.w.part0};
    if (!reduce_lanes<LG, S, 1>(acc, parts, e, a.g.nblk, a.w.counter + e * CNT_KINDS + CNT_SPMV, tot)) return;
    if (threadIdx.x < S && a.pq_out) {
        a.pq_out[e * S + threadIdx.x] = tot[threadIdx.x];
    } else if (threadIdx.x < S) {
        const int L = e * S + threadIdx.x;
        if (a.w.live[L]) {
            const double pq = tot[threadIdx.x];
            if (!(pq > 0.0) || !isfinite(pq)) {
                // zero (or invalid) A-conjugate norm: freeze, x stays as it is
                freeze(a, L, ENS_LANE_BREAKDOWN, a.w.k[L], sqrt(a.w.rr[L]) / a.w.bnorm[L], &dead);
            } else {
                a.w.alpha[L] = a.w.rz[L] / pq;
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && dead) {
        a.w.ens_live[e] -= dead;
        atomicSub(a.w.ctl + CTL_NLIVE, dead);
    }
}

// ---- K3: x += alpha p, r -= alpha q, z = D^-1 r; r^T r and r^T z -> convergence, beta ----
template <typename T, int S>
__global__ void __launch_bounds__(kBlock) k_update(Args a, T *__restrict__ xx, T *__restrict__ rr,
                                                   const T *__restrict__ pp, const T *__restrict__ qq,
                                                   const T *__restrict__ dinv, T *__restrict__ zz)
{
    using LG = VecGeo<T, S>;
    constexpr int V = LG::V, TPR = LG::TPR, RPP = LG::RPP;
    const int e = blockIdx.y;
    if (a.w.ens_live[e] == 0) return;
    const int lane0 = (threadIdx.x % TPR) * V;
    const int L0 = e * S + lane0;
    int lv[V];
    T al[V];
    bool mine = false;
#pragma unroll
    for (int v = 0; v < V; v++) {
        lv[v] = a.w.live[L0 + v];
        al[v] = lv[v] ? (T)a.w.alpha[L0 + v] : T(0);
        mine = mine || lv[v];
    }
    double acc[2][V] = {};
    if (mine) {
        const size_t vb = (size_t)e * a.J * S + lane0;
        const int r0 = blockIdx.x * a.g.RT, r1 = min(a.J, r0 + a.g.RT);
        for (int r = r0 + threadIdx.x / TPR; r < r1; r += RPP) {
            const size_t o = vb + (size_t)r * S;
            Vec<T, V> xv, rv, pv, qv, dv, zv;
            xv.load(xx + o);
            rv.load(rr + o);
            pv.load_ro(pp + o);
            qv.load_ro(qq + o);
            dv.load_ro(dinv + o);
#pragma unroll
            for (int v = 0; v < V; v++) {
                zv.v[v] = T(0);
                if (!lv[v]) continue;  // frozen lane: keep x and r
                xv.v[v] = fma(al[v], pv.v[v], xv.v[v]);
                rv.v[v] = fma(-al[v], qv.v[v], rv.v[v]);
                zv.v[v] = dv.v[v] * rv.v[v];
                acc[0][v] = fma(wide(rv.v[v]), wide(rv.v[v]), acc[0][v]);
                acc[1][v] = fma(wide(rv.v[v]), wide(zv.v[v]), acc[1][v]);
            }
            xv.store(xx + o);
            rv.store(rr + o);
            zv.store(zz + o);
        }
    }
    __shared__ double tot[2 * S];
    __shared__ int dead;
    if (threadIdx.x == 0) dead = 0;
    double *parts[2] = {a.w.part0, a.w.part1};
    if (!reduce_lanes<LG, S, 2>(acc, parts, e, a.g.nblk, a.w.counter + e * CNT_KINDS + CNT_UPD, tot)) return;
    if (threadIdx.x < S) {
        const int L = e * S + threadIdx.x;
        if (a.w.live[L]) {
            const int k = a.w.k[L] + 1;
            a.w.k[L] = k;
            const double rsq = tot[threadIdx.x], rzn = tot[S + threadIdx.x];
            a.w.rr[L] = rsq;
            const double res = sqrt(rsq);
            const double bn = a.w.bnorm[L];
            if (res <= a.rtol * bn) {
                freeze(a, L, ENS_LANE_CONVERGED, k, res / bn, &dead);
            } else if (k >= a.maxit) {
                freeze(a, L, ENS_LANE_MAXIT, k, res / bn, &dead);
            } else {
                a.w.beta[L] = rzn / a.w.rz[L];
                a.w.rz[L] = rzn;
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && dead) {
        a.w.ens_live[e] -= dead;
        atomicSub(a.w.ctl + CTL_NLIVE, dead);
    }
}

// ---- K4: p = z + beta p (z = D^-1 r from K3); loop control ----------------------
template <typename T, int S>
__global__ void __launch_bounds__(kBlock) k_direction(Args a, const T *__restrict__ zz, T *__restrict__ pp)
{
    using LG = VecGeo<T, S>;
    constexpr int V = LG::V, TPR = LG::TPR, RPP = LG::RPP;
    const int e = blockIdx.y;
    if (blockIdx.x == 0 && blockIdx.y == 0) {
        // K3 has finished for every ensemble of this branch, so their live
        // counts are final here: loop again while one of them has a live lane.
        int any = 0;
        for (int i = threadIdx.x; i < a.E; i += kBlock) any |= a.w.ens_live[i] > 0;
        any = __syncthreads_or(any);
        if (threadIdx.x == 0) {
            int *trip = a.w.ctl + a.branch * CTL_WORDS + CTL_TRIPS;
            const int trips = *trip + 1;
            *trip = trips;
            if (a.in_graph) cudaGraphSetConditional(a.cond, (any && trips < a.trip_cap) ? 1u : 0u);
        }
    }
    if (a.w.ens_live[e] == 0) return;
    const int lane0 = (threadIdx.x % TPR) * V;
    const int L0 = e * S + lane0;
    int lv[V];
    T be[V];
    bool mine = false;
#pragma unroll
    for (int v = 0; v < V; v++) {
        lv[v] = a.w.live[L0 + v];
        be[v] = lv[v] ? (T)a.w.beta[L0 + v] : T(0);
        mine = mine || lv[v];
    }
    if (!mine) return;
    const size_t vb = (size_t)e * a.J * S + lane0;
    const int r0 = blockIdx.x * a.g.RT, r1 = min(a.J, r0 + a.g.RT);
    for (int r = r0 + threadIdx.x / TPR; r < r1; r += RPP) {
        const size_t o = vb + (size_t)r * S;
        Vec<T, V> zv, pv;
        zv.load_ro(zz + o);
        pv.load(pp + o);
#pragma unroll
        for (int v = 0; v < V; v++)
            if (lv[v]) pv.v[v] = fma(be[v], pv.v[v], zv.v[v]);
        pv.store(pp + o);
    }
}

// Lanes still live when the loop stopped (only possible through the trip cap).
__global__ void k_finish(Args a)
{
    int L = blockIdx.x * blockDim.x + threadIdx.x;
    if (L >= a.E * a.S) return;
    if (a.w.live[L]) {
        a.w.live[L] = 0;
        a.status[L] = ENS_LANE_MAXIT;
        a.iters[L] = a.w.k[L];
        a.relres[L] = sqrt(a.w.rr[L]) / a.w.bnorm[L];
    }
}

// ens_spmv: every lane live, every ensemble live.
__global__ void k_spmv_prep(Args a)
{
    int L = blockIdx.x * blockDim.x + threadIdx.x;
    if (L < a.E * a.S) a.w.live[L] = 1;
    if (L < a.E) a.w.ens_live[L] = a.S;
}

// The K2 variant for S and the pattern's mean row length (see k_spmv): the
// chunk matches the stencil (5, 7 or 9 nonzeros), because a chunk slot past the
// end of a row is an FP64 multiply-add the whole warp skips but still issues
// (measured on the 7-point rows with KC = 9: the FP64 pipe busy 27 % longer
// than the real multiply-adds need).
template <typename T, int S>
void launch_k2(const Args &a, cudaStream_t st)
{
    dim3 grid(a.g.nblk, a.E);
    const double row = (double)a.nnz / a.J;
    const T *vals = (const T *)a.vals, *p = (const T *)a.w.p;
    T *q = (T *)a.w.q;
    constexpr int V1 = SpmvGeo<S>::V;
    if (row <= 5.5) {
        if constexpr (sizeof(T) == 8 && (S == 16 || S == 32))
            k_spmv<T, S, 2, 5><<<grid, kBlock, 0, st>>>(a, a.rowptr, a.colidx, vals, p, q);
        else
            k_spmv<T, S, V1, 5><<<grid, kBlock, 0, st>>>(a, a.rowptr, a.colidx, vals, p, q);
    } else if (row <= 7.5) {
        const bool cyc = a.g.RT > 256;
        if constexpr (sizeof(T) == 8 && S == 32) {
            if (cyc)
                k_spmv<T, S, 2, 7, true><<<grid, kBlock, 0, st>>>(a, a.rowptr, a.colidx, vals, p, q);
            else
                k_spmv<T, S, 2, 7><<<grid, kBlock, 0, st>>>(a, a.rowptr, a.colidx, vals, p, q);
        } else {
            if (cyc)
                k_spmv<T, S, V1, 7, true><<<grid, kBlock, 0, st>>>(a, a.rowptr, a.colidx, vals, p, q);
            else
                k_spmv<T, S, V1, 7><<<grid, kBlock, 0, st>>>(a, a.rowptr, a.colidx, vals, p, q);
        }
    } else {
        k_spmv<T, S, V1, 9><<<grid, kBlock, 0, st>>>(a, a.rowptr, a.colidx, vals, p, q);
    }
}

template <typename T, int S>
void launch_spmv(const Args &a, cudaStream_t st)
{
    launch_k2<T, S>(a, st);
}

template <typename T, int S>
void launch_body(const Args &a, cudaStream_t st)
{
    dim3 grid(a.g.nblk, a.E);
    launch_k2<T, S>(a, st);
    k_update<T, S><<<grid, kBlock, 0, st>>>(a, (T *)a.x, (T *)a.w.r, (const T *)a.w.p, (const T *)a.w.q,
                                           (const T *)a.dinv, (T *)a.w.z);
    k_direction<T, S><<<grid, kBlock, 0, st>>>(a, (const T *)a.w.z, (T *)a.w.p);
}

template <typename T, int S>
void launch_init(const Args &a, cudaStream_t st)
{
    dim3 grid(a.g.nblk, a.E);
    k_init<T, S><<<grid, kBlock, 0, st>>>(a, a.b, (const T *)a.dinv, (T *)a.x, (T *)a.w.r, (T *)a.w.p);
}

#define ENS_DISPATCH_S(FN, T, a, st)          \
    switch ((a).S) {                          \
    case 1: FN<T, 1>(a, st); break;           \
    case 2: FN<T, 2>(a, st); break;           \
    case 4: FN<T, 4>(a, st); break;           \
    case 8: FN<T, 8>(a, st); break;           \
    case 16: FN<T, 16>(a, st); break;         \
    case 32: FN<T, 32>(a, st); break;         \
    default: FN<T, 64>(a, st); break;         \
    }

template <typename T> void dispatch_body(const Args &a, cudaStream_t st) { ENS_DISPATCH_S(launch_body, T, a, st) }
template <typename T> void dispatch_init(const Args &a, cudaStream_t st) { ENS_DISPATCH_S(launch_init, T, a, st) }
template <typename T> void dispatch_spmv(const Args &a, cudaStream_t st) { ENS_DISPATCH_S(launch_spmv, T, a, st) }

uint64_t bits(const void *p) { return (uint64_t)(uintptr_t)p; }
uint64_t bits(double d)
{
    uint64_t u;
    memcpy(&u, &d, 8);
    return u;
}

// The arguments of the ensembles [e0, e0 + Eb) alone: every per-ensemble and
// per-lane array offset to e0, run as graph branch `branch`.
template <typename T>
Args sub_args(const Args &a, int e0, int Eb, int branch)
{
    Args s = a;
    const size_t ev = (size_t)e0 * a.J * a.S, en = (size_t)e0 * a.nnz * a.S, el = (size_t)e0 * a.S;
    s.E = Eb;
    s.branch = branch;
    s.vals = (const T *)a.vals + en;
    s.dinv = (const T *)a.dinv + ev;
    s.b = a.b + ev;
    s.x = (T *)a.x + ev;
    if (a.active) s.active = a.active + el;
    s.iters = a.iters + el;
    s.status = a.status + el;
    s.relres = a.relres + el;
    if (a.pq_out) s.pq_out = a.pq_out + el;
    if (a.refill) s.refill = a.refill + el;
    s.w.r = (T *)a.w.r + ev;
    s.w.p = (T *)a.w.p + ev;
    s.w.q = (T *)a.w.q + ev;
    s.w.z = (T *)a.w.z + ev;
    s.w.part0 = a.w.part0 + (size_t)e0 * a.g.nblk * a.S;
    s.w.part1 = a.w.part1 + (size_t)e0 * a.g.nblk * a.S;
    s.w.bnorm = a.w.bnorm + el;
    s.w.rz = a.w.rz + el;
    s.w.alpha = a.w.alpha + el;
    s.w.beta = a.w.beta + el;
    s.w.rr = a.w.rr + el;
    s.w.k = a.w.k + el;
    s.w.live = a.w.live + el;
    s.w.ens_live = a.w.ens_live + e0;
    s.w.counter = a.w.counter + (size_t)e0 * CNT_KINDS;
    return s;  // w.ctl stays shared: CTL_NLIVE counts every branch's lanes
}

// Graph branches for E ensembles: one per ensemble up to kMaxBranches.  Each
// branch runs its own while loop, so ensembles advance independently: the
// SpMV (FP64-bound) of one overlaps the vector updates (HBM-bound) of another,
// no kernel waits for the slowest ensemble of the solve, and ensembles that
// have finished launch nothing.  The kernels and the per-ensemble reduction
// order are the same as with one branch, so the results are identical.
int loop_branches(const ens_ctx *h, int E)
{
    int b = h->branches > 0 ? h->branches : kMaxBranches;
    if (b > kMaxBranches) b = kMaxBranches;
    return b < E ? b : (E > 0 ? E : 1);
}

// Instantiate (or reuse) the while-loop graph for these arguments: `branches`
// conditional WHILE nodes side by side, branch b over the ensembles
// [b E / branches, (b + 1) E / branches).
template <typename T>
int loop_graph(ens_ctx *h, Args a, int branches, cudaGraphExec_t *out)
{
    std::vector<uint64_t> key = {bits(a.rowptr), bits(a.colidx), bits(a.vals), bits(a.dinv), bits(a.b),
                                 bits(a.x), bits(a.active), bits(a.iters), bits(a.status), bits(a.relres),
                                 bits(a.w.r), bits(a.w.part0), bits(a.w.live), (uint64_t)a.J, (uint64_t)a.S,
                                 (uint64_t)a.E, (uint64_t)a.maxit, (uint64_t)a.nnz, bits(a.rtol),
                                 (uint64_t)a.g.nblk, (uint64_t)a.g.RT, (uint64_t)sizeof(T), (uint64_t)a.trip_cap,
                                 bits(a.refill), (uint64_t)branches};
    h->clock++;
    for (auto &ge : h->graphs)
        if (ge.key == key) {
            ge.last_use = h->clock;
            *out = ge.exec;
            return ENS_OK;
        }
    cudaGraph_t g = nullptr;
    ENS_CUDA_CHECK(h, cudaGraphCreate(&g, 0));
    for (int br = 0; br < branches; br++) {
        const int e0 = (int)((long long)br * a.E / branches), e1 = (int)((long long)(br + 1) * a.E / branches);
        Args ab = sub_args<T>(a, e0, e1 - e0, br);
        cudaGraphConditionalHandle cond;
        cudaError_t e = cudaGraphConditionalHandleCreate(&cond, g, 1, cudaGraphCondAssignDefault);
        if (e != cudaSuccess) {
            cudaGraphDestroy(g);
            return cuda_error(h, e, "cudaGraphConditionalHandleCreate");
        }
        cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
        cp.conditional.handle = cond;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t node;
        e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp);
        if (e != cudaSuccess) {
            cudaGraphDestroy(g);
            return cuda_error(h, e, "cudaGraphAddNode(conditional)");
        }
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        ab.cond = cond;
        ab.in_graph = 1;
        e = cudaStreamBeginCaptureToGraph(h->capture, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) {
            cudaGraphDestroy(g);
            return cuda_error(h, e, "cudaStreamBeginCaptureToGraph");
        }
        dispatch_body<T>(ab, h->capture);
        cudaError_t le = cudaGetLastError();
        cudaGraph_t captured = nullptr;
        e = cudaStreamEndCapture(h->capture, &captured);
        if (le != cudaSuccess || e != cudaSuccess) {
            cudaGraphDestroy(g);
            return cuda_error(h, le != cudaSuccess ? le : e, "capturing the PCG loop body");
        }
    }
    cudaGraphExec_t exec = nullptr;
    cudaError_t e = cudaGraphInstantiate(&exec, g, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return cuda_error(h, e, "cudaGraphInstantiate");
    }
    const size_t kMaxGraphs = 32;
    if (h->graphs.size() >= kMaxGraphs) {
        size_t old = 0;
        for (size_t i = 1; i < h->graphs.size(); i++)
            if (h->graphs[i].last_use < h->graphs[old].last_use) old = i;
        cudaGraphExecDestroy(h->graphs[old].exec);
        cudaGraphDestroy(h->graphs[old].graph);
        h->graphs.erase(h->graphs.begin() + old);
    }
    GraphEntry ge;
    ge.key = key;
    ge.graph = g;
    ge.exec = exec;
    ge.last_use = h->clock;
    h->graphs.push_back(ge);
    *out = exec;
    return ENS_OK;
}

// Run the whole PCG (init, loop, finish) for prepared arguments.
template <typename T>
int run_solve(ens_ctx *h, const Args &a, cudaStream_t st, bool host_loop, int branches = 1)
{
    if (host_loop) branches = 1;
    ENS_CUDA_CHECK(h, cudaMemsetAsync(a.w.counter, 0, (size_t)a.E * CNT_KINDS * sizeof(int), st));
    ENS_CUDA_CHECK(h, cudaMemsetAsync(a.w.ctl, 0, 2 * sizeof(int), st));
    for (int br = 1; br < branches; br++)
        ENS_CUDA_CHECK(h, cudaMemsetAsync(a.w.ctl + br * CTL_WORDS + CTL_TRIPS, 0, sizeof(int), st));
    dispatch_init<T>(a, st);
    ENS_LAUNCH_CHECK(h, "PCG init kernel");
    if (host_loop) {
        // Same kernels launched from the host, with the live count read back
        // every 16 trips (profilers see each launch; the graph path does not
        // expose kernels inside a conditional body to them).
        int ctl[2] = {1, 0};
        while (ctl[0] > 0 && ctl[1] < a.trip_cap) {
            for (int t = 0; t < 16; t++) dispatch_body<T>(a, st);
            ENS_LAUNCH_CHECK(h, "PCG loop kernels");
            ENS_CUDA_CHECK(h, cudaMemcpyAsync(ctl, a.w.ctl, sizeof(ctl), cudaMemcpyDeviceToHost, st));
            ENS_CUDA_CHECK(h, cudaStreamSynchronize(st));
        }
    } else {
        cudaGraphExec_t exec;
        int rc = loop_graph<T>(h, a, branches, &exec);
        if (rc) return rc;
        ENS_CUDA_CHECK(h, cudaGraphLaunch(exec, st));
    }
    k_finish<<<(a.E * a.S + 255) / 256, 256, 0, st>>>(a);
    ENS_LAUNCH_CHECK(h, "PCG finish kernel");
    return ENS_OK;
}

int check_solve_args(ens_ctx *h, const char *who, int J, int64_t nnz, int S, int E, double rtol, int maxit)
{
    if (!lane_count_ok(S)) return set_error(h, ENS_EINVAL, std::string(who) + ": S must be 1,2,4,...,64");
    if (J <= 0 || nnz <= 0 || E < 0 || nnz >= (1LL << 31))
        return set_error(h, ENS_EINVAL, std::string(who) + ": bad J / nnz / E");
    if (E > 65535) return set_error(h, ENS_EINVAL, std::string(who) + ": E > 65535");
    if (!(rtol >= 0.0) || maxit < 0) return set_error(h, ENS_EINVAL, std::string(who) + ": bad rtol / maxit");
    return ENS_OK;
}

}  // namespace
}  // namespace ens

using namespace ens;

extern "C" int ens_pcg_branches(ens_handle h, int E)
{
    if (!h || E <= 0) return 0;
    return h->host_loop ? 1 : loop_branches(h, E);
}

extern "C" int ens_pcg_cluster_size(ens_handle h, int J, int64_t nnz, int S, int E)
{
    return fused_cluster_size(h, J, nnz, S, E);
}

extern "C" size_t ens_pcg_workspace_size(int J, int64_t nnz, int S, int E)
{
    (void)nnz;
    if (J <= 0 || E <= 0 || !lane_count_ok(S)) return 0;
    return layout(J, S, E, geometry(J, S, E), nullptr, nullptr);
}

extern "C" int ens_pcg_solve(ens_handle h, int J, int64_t nnz, int S, int E, const int32_t *rowptr,
                             const int32_t *colidx, const double *vals, const double *dinv, const double *b,
                             double *x, const uint8_t *active, double rtol, int maxit, int32_t *iters,
                             double *relres, int32_t *status, void *work, size_t work_bytes, void *stream)
{
    if (!h) return ENS_EINVAL;
    int rc = check_solve_args(h, "ens_pcg_solve", J, nnz, S, E, rtol, maxit);
    if (rc) return rc;
    if (E == 0) return ENS_OK;
    if (!rowptr || !colidx || !vals || !dinv || !b || !x || !iters || !relres || !status || !work)
        return set_error(h, ENS_EINVAL, "ens_pcg_solve: null pointer");
    if (((uintptr_t)vals | (uintptr_t)dinv | (uintptr_t)b | (uintptr_t)x | (uintptr_t)work) & 15)
        return set_error(h, ENS_EINVAL, "ens_pcg_solve: arrays must be 16-byte aligned");
    if (h->check) {
        int crc = check_pattern(h, "ens_pcg_solve", J, nnz, rowptr, colidx, (cudaStream_t)stream);
        if (crc) return crc;
    }
    Geo g = geometry(J, S, E);
    const size_t need = layout(J, S, E, g, nullptr, nullptr);
    if (work_bytes < need)
        return set_error(h, ENS_ENOMEM, "ens_pcg_solve: workspace too small (need " + std::to_string(need) + " bytes)");
    Args a;
    memset(&a, 0, sizeof(a));
    a.J = J; a.S = S; a.E = E; a.maxit = maxit; a.nnz = nnz; a.rtol = rtol; a.g = g;
    a.rowptr = rowptr; a.colidx = colidx; a.vals = vals; a.dinv = dinv; a.b = b; a.x = x;
    a.active = active; a.iters = iters; a.status = status; a.relres = relres;
    a.trip_cap = maxit;
    layout(J, S, E, g, &a.w, (char *)work);
    const int C = fused_cluster_size(h, J, nnz, S, E);
    if (C > 0) return fused_solve(h, a, C, (cudaStream_t)stream);
    return run_solve<double>(h, a, (cudaStream_t)stream, h->host_loop != 0, loop_branches(h, E));
}

// ---- mixed precision: FP32 inner PCG inside FP64 iterative refinement ---------
// r = b - A64 x in FP64; stop a lane when ||r|| <= rtol ||b||; else solve
// A32 d = r with the FP32 form of the loop above (to ||r - A32 d|| <= rtol_inner ||r||,
// FP64 inner products and scalars) and update x += d in FP64.
namespace ens {
namespace {

struct IrWs {
    Ws inner;            // FP32 loop workspace
    double *r64;         // [E][J][S] outer residual
    float *dinv32, *d32; // [E][J][S]
    double *bnorm;       // [E][S] ||b||
    int *olive, *oits, *inner_tot;  // [E][S]
    uint8_t *iactive;    // [E][S] lanes the next inner solve works on
    int32_t *istatus, *iiters;  // [E][S] inner outcome
    double *irelres;     // [E][S]
};

size_t ir_layout(int J, int S, int E, const Geo &g, IrWs *w, char *base)
{
    Bump m(base);
    IrWs t;
    lay_loop(m, J, S, E, g, sizeof(float), &t.inner);
    size_t vec = (size_t)E * J * S;
    size_t lane = (size_t)E * S;
    t.r64 = (double *)m.take(vec * 8);
    t.dinv32 = (float *)m.take(vec * 4);
    t.d32 = (float *)m.take(vec * 4);
    t.bnorm = (double *)m.take(lane * 8);
    t.olive = (int *)m.take(lane * 4);
    t.oits = (int *)m.take(lane * 4);
    t.inner_tot = (int *)m.take(lane * 4);
    t.iactive = (uint8_t *)m.take(lane);
    t.istatus = (int32_t *)m.take(lane * 4);
    t.iiters = (int32_t *)m.take(lane * 4);
    t.irelres = (double *)m.take(lane * 8);
    if (w) *w = t;
    return m.off;
}

struct IrArgs {
    int J, S, E, maxit_outer;
    long long nnz;
    double rtol;
    Geo g;
    const uint8_t *active;
    int32_t *iters, *outer_its, *status;
    double *relres;
    IrWs w;
};

// x = 0, D^-1 in FP32, outer lane state.
__global__ void k_ir_prep(IrArgs a, const double *__restrict__ dinv, double *__restrict__ x)
{
    const size_t n = (size_t)a.E * a.J * a.S;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        x[i] = 0.0;
        a.w.dinv32[i] = (float)dinv[i];
    }
    const int lanes = a.E * a.S;
    for (int L = blockIdx.x * blockDim.x + threadIdx.x; L < lanes; L += gridDim.x * blockDim.x) {
        const int act = a.active ? (int)a.active[L] : 1;
        a.w.olive[L] = act;
        a.w.oits[L] = 0;
        a.w.inner_tot[L] = 0;
        a.status[L] = act ? ENS_LANE_MAXIT : ENS_LANE_INACTIVE;
        a.iters[L] = 0;
        a.outer_its[L] = 0;
        a.relres[L] = act ? 1.0 : 0.0;
    }
}

// r = b - A64 x (FP64) and ||r||^2 per lane -> outer convergence.
template <int S>
__global__ void __launch_bounds__(kBlock, (S >= 64 ? 2 : (S == 1 ? 3 : 4)))
    k_residual(IrArgs a, Args sa, const int32_t *__restrict__ rowptr, const int32_t *__restrict__ colidx,
               const double *__restrict__ vals_all, const double *__restrict__ x_all,
               const double *__restrict__ b_all, double *__restrict__ r_all)
{
    using LG = SpmvGeo<S>;
    constexpr int V = LG::V, TPR = LG::TPR, RPP = LG::RPP;
    const int e = blockIdx.y;
    const int lane0 = (threadIdx.x % TPR) * V;
    const int L0 = e * S + lane0;
    bool mine = a.w.olive[L0] != 0;
    if (V == 2) mine = mine || a.w.olive[L0 + 1] != 0;
    double acc[1][V] = {};
    if (mine) {
        const double *__restrict__ vals = vals_all + (size_t)e * a.nnz * S + lane0;
        const double *__restrict__ x = x_all + (size_t)e * a.J * S + lane0;
        const double *__restrict__ bb = b_all + (size_t)e * a.J * S + lane0;
        double *__restrict__ r = r_all + (size_t)e * a.J * S + lane0;
        const int r0 = blockIdx.x * a.g.RT, r1 = min(a.J, r0 + a.g.RT);
        for (int row = r0 + threadIdx.x / TPR; row < r1; row += RPP) {
            const int k0 = __ldg(rowptr + row), k1 = __ldg(rowptr + row + 1);
            double s[V];
#pragma unroll
            for (int v = 0; v < V; v++) s[v] = 0.0;
            for (int kb = k0; kb < k1; kb += kChunk) {
                int c[kChunk];
                Vec<double, V> av[kChunk], xv[kChunk];
#pragma unroll
                for (int u = 0; u < kChunk; u++)
                    if (kb + u < k1) c[u] = __ldg(colidx + kb + u);
#pragma unroll
                for (int u = 0; u < kChunk; u++)
                    if (kb + u < k1) {
                        av[u].load_stream(vals + (size_t)(kb + u) * S);
                        xv[u].load_ro(x + (size_t)c[u] * S);
                    }
#pragma unroll
                for (int u = 0; u < kChunk; u++)
                    if (kb + u < k1) {
#pragma unroll
                        for (int v = 0; v < V; v++) s[v] = fma(av[u].v[v], xv[u].v[v], s[v]);
                    }
            }
            Vec<double, V> bv, rv;
            bv.load_ro(bb + (size_t)row * S);
#pragma unroll
            for (int v = 0; v < V; v++) {
                rv.v[v] = bv.v[v] - s[v];
                acc[0][v] = fma(rv.v[v], rv.v[v], acc[0][v]);
            }
            rv.store(r + (size_t)row * S);
        }
    }
    __shared__ double tot[S];
    __shared__ int live_cnt;
    if (threadIdx.x == 0) live_cnt = 0;
    double *parts[1] = {sa.w.part0};
    if (!reduce_lanes<LG, S, 1>(acc, parts, e, a.g.nblk, sa.w.counter + e * CNT_KINDS + CNT_RES, tot)) return;
    if (threadIdx.x < S) {
        const int L = e * S + threadIdx.x;
        int go = 0;
        if (a.w.olive[L]) {
            const double rn = sqrt(tot[threadIdx.x]);
            const int it = a.w.oits[L];
            if (it == 0) a.w.bnorm[L] = rn;  // x = 0 on the first pass: r = b
            const double bn = a.w.bnorm[L];
            a.iters[L] = a.w.inner_tot[L];
            a.outer_its[L] = it;
            if (!isfinite(rn)) {
                a.w.olive[L] = 0;
                a.status[L] = it == 0 ? ENS_LANE_BADINPUT : ENS_LANE_BREAKDOWN;
                a.relres[L] = __longlong_as_double(0x7ff8000000000000LL);
            } else if (bn == 0.0) {
                a.w.olive[L] = 0;
                a.status[L] = ENS_LANE_CONVERGED;
                a.relres[L] = 0.0;
            } else if (rn <= a.rtol * bn) {
                a.w.olive[L] = 0;
                a.status[L] = ENS_LANE_CONVERGED;
                a.relres[L] = rn / bn;
            } else if (it >= a.maxit_outer) {
                a.w.olive[L] = 0;
                a.status[L] = ENS_LANE_MAXIT;
                a.relres[L] = rn / bn;
            } else {
                a.relres[L] = rn / bn;
                go = 1;
            }
        }
        a.w.iactive[L] = (uint8_t)go;
        if (go) atomicAdd(&live_cnt, 1);
    }
    __syncthreads();
    if (threadIdx.x == 0 && live_cnt) atomicAdd(sa.w.ctl + CTL_OUTER_LIVE, live_cnt);
}

// x += d (FP64) for the lanes of the inner solve.
template <int S>
__global__ void k_ir_update(IrArgs a, double *__restrict__ x, const float *__restrict__ d)
{
    const size_t n = (size_t)a.E * a.J * S;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int L = (int)((i / ((size_t)a.J * S)) * S + i % S);
        if (a.w.iactive[L]) x[i] = x[i] + (double)d[i];
    }
}

// Outer bookkeeping after an inner solve.
__global__ void k_ir_lanes(IrArgs a)
{
    const int lanes = a.E * a.S;
    for (int L = blockIdx.x * blockDim.x + threadIdx.x; L < lanes; L += gridDim.x * blockDim.x) {
        if (!a.w.iactive[L]) continue;
        a.w.oits[L] += 1;
        a.w.inner_tot[L] += a.w.iiters[L];
        const int st = a.w.istatus[L];
        if ((st == ENS_LANE_BREAKDOWN && a.w.iiters[L] == 0) || st == ENS_LANE_BADINPUT) {
            a.w.olive[L] = 0;  // no progress possible: keep x
            a.status[L] = ENS_LANE_BREAKDOWN;
            a.iters[L] = a.w.inner_tot[L];
            a.outer_its[L] = a.w.oits[L];
        }
    }
}

template <int S>
void launch_residual(const IrArgs &ia, const Args &sa, const double *vals, const double *x, const double *b,
                     cudaStream_t st)
{
    dim3 grid(ia.g.nblk, ia.E);
    k_residual<S><<<grid, kBlock, 0, st>>>(ia, sa, sa.rowptr, sa.colidx, vals, x, b, ia.w.r64);
}

template <int S>
void launch_ir_update(const IrArgs &ia, double *x, cudaStream_t st)
{
    k_ir_update<S><<<152 * 4, 256, 0, st>>>(ia, x, ia.w.d32);
}

}  // namespace
}  // namespace ens

extern "C" size_t ens_pcg_ir_workspace_size(int J, int64_t nnz, int S, int E)
{
    (void)nnz;
    if (J <= 0 || E <= 0 || !lane_count_ok(S)) return 0;
    return ir_layout(J, S, E, geometry(J, S, E), nullptr, nullptr);
}

extern "C" int ens_pcg_solve_ir(ens_handle h, int J, int64_t nnz, int S, int E, const int32_t *rowptr,
                                const int32_t *colidx, const double *vals, const float *vals32, const double *dinv,
                                const double *b, double *x, const uint8_t *active, double rtol, double rtol_inner,
                                int maxit_inner, int maxit_outer, int32_t *iters, int32_t *outer_its,
                                double *relres, int32_t *status, void *work, size_t work_bytes, void *stream)
{
    if (!h) return ENS_EINVAL;
    int rc = check_solve_args(h, "ens_pcg_solve_ir", J, nnz, S, E, rtol, maxit_inner);
    if (rc) return rc;
    if (!(rtol_inner > 0.0 && rtol_inner < 1.0) || maxit_outer < 0)
        return set_error(h, ENS_EINVAL, "ens_pcg_solve_ir: need 0 < rtol_inner < 1 and maxit_outer >= 0");
    if (E == 0) return ENS_OK;
    if (!rowptr || !colidx || !vals || !vals32 || !dinv || !b || !x || !iters || !outer_its || !relres || !status ||
        !work)
        return set_error(h, ENS_EINVAL, "ens_pcg_solve_ir: null pointer");
    if (((uintptr_t)vals | (uintptr_t)vals32 | (uintptr_t)dinv | (uintptr_t)b | (uintptr_t)x | (uintptr_t)work) & 15)
        return set_error(h, ENS_EINVAL, "ens_pcg_solve_ir: arrays must be 16-byte aligned");
    if (h->check) {
        int crc = check_pattern(h, "ens_pcg_solve_ir", J, nnz, rowptr, colidx, (cudaStream_t)stream);
        if (crc) return crc;
    }
    Geo g = geometry(J, S, E);
    const size_t need = ir_layout(J, S, E, g, nullptr, nullptr);
    if (work_bytes < need)
        return set_error(h, ENS_ENOMEM, "ens_pcg_solve_ir: workspace too small (need " + std::to_string(need) + " bytes)");
    cudaStream_t st = (cudaStream_t)stream;
    IrArgs ia;
    memset(&ia, 0, sizeof(ia));
    ia.J = J; ia.S = S; ia.E = E; ia.maxit_outer = maxit_outer; ia.nnz = nnz; ia.rtol = rtol; ia.g = g;
    ia.active = active; ia.iters = iters; ia.outer_its = outer_its; ia.status = status; ia.relres = relres;
    ir_layout(J, S, E, g, &ia.w, (char *)work);
    // the inner FP32 solve: b = the FP64 residual, x = the FP32 correction
    Args sa;
    memset(&sa, 0, sizeof(sa));
    sa.J = J; sa.S = S; sa.E = E; sa.maxit = maxit_inner; sa.nnz = nnz; sa.rtol = rtol_inner; sa.g = g;
    sa.rowptr = rowptr; sa.colidx = colidx; sa.vals = vals32; sa.dinv = ia.w.dinv32; sa.b = ia.w.r64;
    sa.x = ia.w.d32; sa.active = ia.w.iactive; sa.iters = ia.w.iiters; sa.status = ia.w.istatus;
    sa.relres = ia.w.irelres; sa.w = ia.w.inner; sa.trip_cap = maxit_inner;
    ENS_CUDA_CHECK(h, cudaMemsetAsync(sa.w.counter, 0, (size_t)E * CNT_KINDS * sizeof(int), st));
    k_ir_prep<<<152 * 4, 256, 0, st>>>(ia, dinv, x);
    ENS_LAUNCH_CHECK(h, "ens_pcg_solve_ir: prep");
    for (int it = 0; it <= maxit_outer; it++) {
        ENS_CUDA_CHECK(h, cudaMemsetAsync(sa.w.ctl + CTL_OUTER_LIVE, 0, sizeof(int), st));
        switch (S) {
        case 1: launch_residual<1>(ia, sa, vals, x, b, st); break;
        case 2: launch_residual<2>(ia, sa, vals, x, b, st); break;
        case 4: launch_residual<4>(ia, sa, vals, x, b, st); break;
        case 8: launch_residual<8>(ia, sa, vals, x, b, st); break;
        case 16: launch_residual<16>(ia, sa, vals, x, b, st); break;
        case 32: launch_residual<32>(ia, sa, vals, x, b, st); break;
        default: launch_residual<64>(ia, sa, vals, x, b, st); break;
        }
        ENS_LAUNCH_CHECK(h, "ens_pcg_solve_ir: residual");
        int olive = 0;
        ENS_CUDA_CHECK(h, cudaMemcpyAsync(&olive, sa.w.ctl + CTL_OUTER_LIVE, sizeof(int), cudaMemcpyDeviceToHost, st));
        ENS_CUDA_CHECK(h, cudaStreamSynchronize(st));
        if (olive == 0) break;
        rc = run_solve<float>(h, sa, st, h->host_loop != 0, loop_branches(h, E));
        if (rc) return rc;
        switch (S) {
        case 1: launch_ir_update<1>(ia, x, st); break;
        case 2: launch_ir_update<2>(ia, x, st); break;
        case 4: launch_ir_update<4>(ia, x, st); break;
        case 8: launch_ir_update<8>(ia, x, st); break;
        case 16: launch_ir_update<16>(ia, x, st); break;
        case 32: launch_ir_update<32>(ia, x, st); break;
        default: launch_ir_update<64>(ia, x, st); break;
        }
        k_ir_lanes<<<(E * S + 255) / 256, 256, 0, st>>>(ia);
        ENS_LAUNCH_CHECK(h, "ens_pcg_solve_ir: update");
    }
    return ENS_OK;
}

// ---- continuous ensemble batching (the batching layer) ---------------------------
// M samples run through a pool of E ensembles of S lanes.  The device loop runs
// a chunk of trips; then every lane that froze gives its outcome back (by
// sample index) and takes the next queued sample: its values are assembled
// into that lane alone and its CG state restarts, while the other lanes keep
// iterating.  Once the queue is empty, the live lanes are re-packed into as
// few ensembles as hold them, so drained ensembles cost nothing.
namespace ens {
namespace {

struct StreamWs {
    int32_t *rowptr, *colidx;
    double *vals, *dinv, *b, *x;  // [E][nnz][S], [E][J][S]
    double *lane_xi;              // [E][S][N]
    int32_t *lane_sample;         // [E][S], -1 = empty
    int32_t *lane_iters, *lane_status;
    double *lane_relres;
    uint8_t *active, *refill;     // [E][S]
    int32_t *list;                // [2 E S] harvest lanes / re-pack moves
    Ws loop;
};

size_t stream_layout(int J, int64_t nnz, int S, int E, int N, const Geo &g, StreamWs *w, char *base)
{
    Bump m(base);
    StreamWs t;
    const size_t lanes = (size_t)E * S;
    t.rowptr = (int32_t *)m.take((size_t)(J + 1) * 4);
    t.colidx = (int32_t *)m.take((size_t)nnz * 4);
    t.vals = (double *)m.take((size_t)E * nnz * S * 8);
    t.dinv = (double *)m.take((size_t)E * J * S * 8);
    t.b = (double *)m.take((size_t)E * J * S * 8);
    t.x = (double *)m.take((size_t)E * J * S * 8);
    t.lane_xi = (double *)m.take(lanes * N * 8);
    t.lane_sample = (int32_t *)m.take(lanes * 4);
    t.lane_iters = (int32_t *)m.take(lanes * 4);
    t.lane_status = (int32_t *)m.take(lanes * 4);
    t.lane_relres = (double *)m.take(lanes * 8);
    t.active = (uint8_t *)m.take(lanes);
    t.refill = (uint8_t *)m.take(lanes);
    t.list = (int32_t *)m.take(lanes * 2 * 4);
    lay_loop(m, J, S, E, g, sizeof(double), &t.loop);
    if (w) *w = t;
    return m.off;
}

// lane_xi of the refilled lanes from the caller's samples.
__global__ void k_gather_xi(int lanes, int N, const uint8_t *__restrict__ refill, const int32_t *__restrict__ sample,
                            const double *__restrict__ xi, double *__restrict__ lane_xi)
{
    int L = blockIdx.x * blockDim.x + threadIdx.x;
    if (L >= lanes || !refill[L] || sample[L] < 0) return;
    for (int k = 0; k < N; k++) lane_xi[(size_t)L * N + k] = xi[(size_t)sample[L] * N + k];
}

// Outcome of finished lanes (list of lane ids) to their samples; QoI by one
// block per lane (fixed order: thread t sums rows t, t + 256, ..., then a tree).
__global__ void k_harvest(int nh, const int32_t *__restrict__ list, int J, int S, const int32_t *__restrict__ sample,
                          const double *__restrict__ x, const double *__restrict__ w,
                          const int32_t *__restrict__ lane_iters, const int32_t *__restrict__ lane_status,
                          const double *__restrict__ lane_relres, int32_t *iters, int32_t *status, double *relres,
                          double *qoi)
{
    __shared__ double sh[256];
    if ((int)blockIdx.x >= nh) return;
    const int L = list[blockIdx.x];
    const int e = L / S, s = L % S;
    const double *xe = x + (size_t)e * J * S + s;
    double acc = 0.0;
    for (int j = threadIdx.x; j < J; j += blockDim.x) {
        const double v = xe[(size_t)j * S];
        acc = fma(w ? w[j] : v, v, acc);
    }
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int off = blockDim.x / 2; off > 0; off >>= 1) {
        if ((int)threadIdx.x < off) sh[threadIdx.x] = dadd(sh[threadIdx.x], sh[threadIdx.x + off]);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const int m = sample[L];
        iters[m] = lane_iters[L];
        status[m] = lane_status[L];
        relres[m] = lane_relres[L];
        if (qoi) qoi[m] = sh[0];
    }
}

// Re-pack: move live lanes (list of (src, dst) pairs) -- their values, vectors
// and CG state -- so the drained ensembles go idle.  Grid: (chunks, moves).
__global__ void k_repack(int nm, const int32_t *__restrict__ moves, int J, long long nnz, int S, int N,
                         StreamWs w)
{
    const int mv = blockIdx.y;
    if (mv >= nm) return;
    const int src = moves[2 * mv], dst = moves[2 * mv + 1];
    const int es = src / S, ss = src % S, ed = dst / S, sd = dst % S;
    const size_t vs = (size_t)es * nnz * S + ss, vd = (size_t)ed * nnz * S + sd;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < nnz; k += (long long)gridDim.x * blockDim.x)
        w.vals[vd + (size_t)k * S] = w.vals[vs + (size_t)k * S];
    const size_t xs = (size_t)es * J * S + ss, xd = (size_t)ed * J * S + sd;
    double *r = (double *)w.loop.r, *p = (double *)w.loop.p;
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < J; j += (long long)gridDim.x * blockDim.x) {
        const size_t a = xs + (size_t)j * S, c = xd + (size_t)j * S;
        w.x[c] = w.x[a];
        w.dinv[c] = w.dinv[a];
        w.b[c] = w.b[a];
        r[c] = r[a];
        p[c] = p[a];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        w.loop.bnorm[dst] = w.loop.bnorm[src];
        w.loop.rz[dst] = w.loop.rz[src];
        w.loop.rr[dst] = w.loop.rr[src];
        w.loop.k[dst] = w.loop.k[src];
        w.loop.live[dst] = w.loop.live[src];
        w.loop.live[src] = 0;
        w.lane_sample[dst] = w.lane_sample[src];
        w.lane_sample[src] = -1;
        w.lane_status[dst] = w.lane_status[src];
        w.lane_iters[dst] = w.lane_iters[src];
        w.lane_relres[dst] = w.lane_relres[src];
        for (int k = 0; k < N; k++) w.lane_xi[(size_t)dst * N + k] = w.lane_xi[(size_t)src * N + k];
    }
}

__global__ void k_count_live(int E, int S, const int *__restrict__ live, int *__restrict__ ens_live)
{
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E) return;
    int c = 0;
    for (int s = 0; s < S; s++) c += live[e * S + s];
    ens_live[e] = c;
}

}  // namespace
}  // namespace ens

extern "C" size_t ens_stream_workspace_size(const ens_problem *p, int S, int E)
{
    int J;
    int64_t nnz;
    std::string why;
    if (problem_check(p, &J, &nnz, &why) || !lane_count_ok(S) || E <= 0) return 0;
    return stream_layout(J, nnz, S, E, p->nparam, geometry(J, S, E), nullptr, nullptr);
}

extern "C" int ens_solve_stream(ens_handle h, const ens_problem *p, int S, int E, int M, const double *xi,
                                const int32_t *order, const double *w, double rtol, int maxit, int chunk,
                                int32_t *iters, int32_t *status, double *relres, double *qoi, void *work,
                                size_t work_bytes, void *stream)
{
    if (!h) return ENS_EINVAL;
    int J;
    int64_t nnz;
    std::string why;
    int rc = problem_check(p, &J, &nnz, &why);
    if (rc) return set_error(h, rc, "ens_solve_stream: " + why);
    rc = check_solve_args(h, "ens_solve_stream", J, nnz, S, E, rtol, maxit);
    if (rc) return rc;
    if (E < 1 || M < 0 || chunk < 1) return set_error(h, ENS_EINVAL, "ens_solve_stream: need E >= 1, M >= 0, chunk >= 1");
    if (M == 0) return ENS_OK;
    if (!xi || !iters || !status || !relres || !work) return set_error(h, ENS_EINVAL, "ens_solve_stream: null pointer");
    Geo g = geometry(J, S, E);
    const size_t need = stream_layout(J, nnz, S, E, p->nparam, g, nullptr, nullptr);
    if (work_bytes < need)
        return set_error(h, ENS_ENOMEM, "ens_solve_stream: workspace too small (need " + std::to_string(need) + " bytes)");
    cudaStream_t st = (cudaStream_t)stream;
    StreamWs sw;
    stream_layout(J, nnz, S, E, p->nparam, g, &sw, (char *)work);
    const int N = p->nparam, lanes = E * S;
    rc = pattern_into(h, p, sw.rowptr, sw.colidx, st);
    if (rc) return rc;

    // the queue, in the caller's order
    std::vector<int32_t> queue(M);
    if (order) {
        ENS_CUDA_CHECK(h, cudaMemcpyAsync(queue.data(), order, (size_t)M * 4, cudaMemcpyDeviceToHost, st));
        ENS_CUDA_CHECK(h, cudaStreamSynchronize(st));
        std::vector<char> seen(M, 0);
        for (int i = 0; i < M; i++) {
            if (queue[i] < 0 || queue[i] >= M || seen[queue[i]])
                return set_error(h, ENS_EINVAL, "ens_solve_stream: order is not a permutation of 0..M-1");
            seen[queue[i]] = 1;
        }
    } else {
        for (int i = 0; i < M; i++) queue[i] = i;
    }
    int next = 0;
    std::vector<int32_t> lane_sample(lanes, -1);
    std::vector<uint8_t> refill(lanes, 0);
    std::vector<int> live(lanes, 0);
    std::vector<int32_t> list;

    Args a;
    memset(&a, 0, sizeof(a));
    a.J = J; a.S = S; a.E = E; a.maxit = maxit; a.nnz = nnz; a.rtol = rtol; a.g = g;
    a.rowptr = sw.rowptr; a.colidx = sw.colidx; a.vals = sw.vals; a.dinv = sw.dinv; a.b = sw.b; a.x = sw.x;
    a.active = sw.active; a.iters = sw.lane_iters; a.status = sw.lane_status; a.relres = sw.lane_relres;
    a.w = sw.loop;
    a.trip_cap = chunk;

    // first fill: every lane gets a sample while the queue lasts; empty lanes
    // carry a copy of sample queue[0] so their (unused) values stay finite
    for (int L = 0; L < lanes; L++) {
        if (next < M) lane_sample[L] = queue[next++];
        refill[L] = 1;
    }
    {
        std::vector<int32_t> fill_sample(lane_sample);
        std::vector<uint8_t> act(lanes);
        for (int L = 0; L < lanes; L++) {
            act[L] = lane_sample[L] >= 0;
            if (fill_sample[L] < 0) fill_sample[L] = queue[0];
        }
        ENS_CUDA_CHECK(h, cudaMemcpyAsync(sw.lane_sample, fill_sample.data(), lanes * 4, cudaMemcpyHostToDevice, st));
        ENS_CUDA_CHECK(h, cudaMemcpyAsync(sw.refill, refill.data(), lanes, cudaMemcpyHostToDevice, st));
        ENS_CUDA_CHECK(h, cudaMemcpyAsync(sw.active, act.data(), lanes, cudaMemcpyHostToDevice, st));
        k_gather_xi<<<(lanes + 255) / 256, 256, 0, st>>>(lanes, N, sw.refill, sw.lane_sample, xi, sw.lane_xi);
        ENS_CUDA_CHECK(h, cudaMemcpyAsync(sw.lane_sample, lane_sample.data(), lanes * 4, cudaMemcpyHostToDevice, st));
        rc = assemble_lanes(h, p, S, E, sw.lane_xi, sw.rowptr, sw.vals, 0, sw.dinv, sw.b, nullptr, 0, st);
        if (rc) return rc;
        ENS_CUDA_CHECK(h, cudaMemsetAsync(a.w.counter, 0, (size_t)E * CNT_KINDS * sizeof(int), st));
        ENS_CUDA_CHECK(h, cudaMemsetAsync(a.w.ctl, 0, 2 * sizeof(int), st));
        dispatch_init<double>(a, st);
        ENS_LAUNCH_CHECK(h, "ens_solve_stream: first fill");
    }
    cudaGraphExec_t exec = nullptr;
    const int branches = h->host_loop ? 1 : loop_branches(h, E);
    if (!h->host_loop) {
        rc = loop_graph<double>(h, a, branches, &exec);
        if (rc) return rc;
    }
    bool repacked_all = false;
    const long long max_rounds = ((long long)M / lanes + 2) * ((long long)maxit / chunk + 2) + 16;
    for (long long round = 0; round < max_rounds; round++) {
        // a chunk of trips
        for (int br = 0; br < branches; br++)
            ENS_CUDA_CHECK(h, cudaMemsetAsync(a.w.ctl + br * CTL_WORDS + CTL_TRIPS, 0, sizeof(int), st));
        if (exec) {
            ENS_CUDA_CHECK(h, cudaGraphLaunch(exec, st));
        } else {
            for (int t = 0; t < chunk; t++) dispatch_body<double>(a, st);
            ENS_LAUNCH_CHECK(h, "ens_solve_stream: loop kernels");
        }
        ENS_CUDA_CHECK(h, cudaMemcpyAsync(live.data(), a.w.live, lanes * sizeof(int), cudaMemcpyDeviceToHost, st));
        ENS_CUDA_CHECK(h, cudaStreamSynchronize(st));
        // finished lanes give their outcome back and take the next samples
        list.clear();
        for (int L = 0; L < lanes; L++)
            if (lane_sample[L] >= 0 && !live[L]) list.push_back(L);
        const int nh = (int)list.size();
        if (nh) {
            ENS_CUDA_CHECK(h, cudaMemcpyAsync(sw.list, list.data(), nh * 4, cudaMemcpyHostToDevice, st));
            k_harvest<<<nh, 256, 0, st>>>(nh, sw.list, J, S, sw.lane_sample, sw.x, w, sw.lane_iters, sw.lane_status,
                                          sw.lane_relres, iters, status, relres, qoi);
            ENS_LAUNCH_CHECK(h, "ens_solve_stream: harvest");
        }
        int nref = 0;
        std::fill(refill.begin(), refill.end(), 0);
        for (int i = 0; i < nh; i++) {
            const int L = list[i];
            if (next < M) {
                lane_sample[L] = queue[next++];
                refill[L] = 1;
                nref++;
            } else {
                lane_sample[L] = -1;
            }
        }
        int nlive = 0;
        for (int L = 0; L < lanes; L++) nlive += (lane_sample[L] >= 0);
        if (nlive == 0) break;
        // the harvest kernel reads lane_sample: update it only after the harvest is queued
        ENS_CUDA_CHECK(h, cudaMemcpyAsync(sw.lane_sample, lane_sample.data(), lanes * 4, cudaMemcpyHostToDevice, st));
        if (nref) {
            std::vector<int32_t> rl;
            for (int L = 0; L < lanes; L++)
                if (refill[L]) rl.push_back(L);
            ENS_CUDA_CHECK(h, cudaMemcpyAsync(sw.refill, refill.data(), lanes, cudaMemcpyHostToDevice, st));
            ENS_CUDA_CHECK(h, cudaMemcpyAsync(sw.active, refill.data(), lanes, cudaMemcpyHostToDevice, st));
            ENS_CUDA_CHECK(h, cudaMemcpyAsync(sw.list, rl.data(), rl.size() * 4, cudaMemcpyHostToDevice, st));
            k_gather_xi<<<(lanes + 255) / 256, 256, 0, st>>>(lanes, N, sw.refill, sw.lane_sample, xi, sw.lane_xi);
            rc = assemble_lanes(h, p, S, E, sw.lane_xi, sw.rowptr, sw.vals, 0, sw.dinv, sw.b, sw.list, (int)rl.size(),
                                st);
            if (rc) return rc;
            Args ra = a;
            ra.refill = sw.refill;
            dispatch_init<double>(ra, st);
            ENS_LAUNCH_CHECK(h, "ens_solve_stream: refill");
        }
        // queue drained: gather the live lanes into the first ensembles
        if (next >= M && !repacked_all) {
            const int target = (nlive + S - 1) / S;
            std::vector<int> src, dst;
            for (int L = target * S; L < lanes; L++)
                if (lane_sample[L] >= 0) src.push_back(L);
            for (int L = 0; L < target * S && dst.size() < src.size(); L++)
                if (lane_sample[L] < 0) dst.push_back(L);
            if (!src.empty() && dst.size() == src.size()) {
                list.clear();
                for (size_t i = 0; i < src.size(); i++) {
                    list.push_back(src[i]);
                    list.push_back(dst[i]);
                    lane_sample[dst[i]] = lane_sample[src[i]];
                    lane_sample[src[i]] = -1;
                }
                const int nm = (int)src.size();
                ENS_CUDA_CHECK(h, cudaMemcpyAsync(sw.list, list.data(), nm * 8, cudaMemcpyHostToDevice, st));
                dim3 grid(64, nm);
                k_repack<<<grid, 256, 0, st>>>(nm, sw.list, J, nnz, S, N, sw);
                k_count_live<<<(E + 127) / 128, 128, 0, st>>>(E, S, a.w.live, a.w.ens_live);
                ENS_LAUNCH_CHECK(h, "ens_solve_stream: re-pack");
            }
            if (target <= 1) repacked_all = true;
        }
    }
    return ENS_OK;
}

// ---- the solve for callers that cannot allocate device memory ------------------
// Some callers cannot call cudaMalloc at all: code running under an allocator
// that owns all device memory, or plug-ins that may not create or grow device
// allocations.  For them ens_pcg_solve_static takes its scratch from this
// file-scope array instead of a caller workspace.  It is small on purpose, as
// every GPU that loads the library holds it until the process exits.
constexpr size_t kStaticScratchBytes = ENS_PCG_STATIC_SCRATCH_BYTES;  // 8 MiB
static __device__ __align__(256) unsigned char g_pcg_scratch[kStaticScratchBytes];

namespace ens {
namespace {
std::mutex g_scratch_mu;
void *g_scratch_addr[128] = {};  // device address of g_pcg_scratch, per device

// The symbol's name is a host-side stand-in; the device address is looked up
// once per device, with that device current.
int scratch_address(ens_ctx *h, void **out)
{
    int dev = 0;
    ENS_CUDA_CHECK(h, cudaGetDevice(&dev));
    if (dev < 0 || dev >= 128) return set_error(h, ENS_EINVAL, "ens_pcg_solve_static: device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        ENS_CUDA_CHECK(h, cudaGetSymbolAddress(&p, g_pcg_scratch));
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return ENS_OK;
}
}  // namespace
}  // namespace ens

extern "C" int ens_pcg_solve_static(ens_handle h, int J, int64_t nnz, int S, int E, const int32_t *rowptr,
                                    const int32_t *colidx, const double *vals, const double *dinv,
                                    const double *b, double *x, const uint8_t *active, double rtol, int maxit,
                                    int32_t *iters, double *relres, int32_t *status, void *stream)
{
    int rc = check_solve_args(h, "ens_pcg_solve_static", J, nnz, S, E, rtol, maxit);
    if (rc) return rc;
    if (E == 0) return ENS_OK;
    if (!rowptr || !colidx || !vals || !dinv || !b || !x || !iters || !relres || !status)
        return set_error(h, ENS_EINVAL, "ens_pcg_solve_static: null pointer");
    if (((uintptr_t)vals | (uintptr_t)dinv | (uintptr_t)b | (uintptr_t)x) & 15)
        return set_error(h, ENS_EINVAL, "ens_pcg_solve_static: arrays must be 16-byte aligned");
    if (h && h->check) {  // h may be NULL here
        int crc = check_pattern(h, "ens_pcg_solve_static", J, nnz, rowptr, colidx, (cudaStream_t)stream);
        if (crc) return crc;
    }
    Geo g = geometry(J, S, E);
    const size_t need = layout(J, S, E, g, nullptr, nullptr);
    if (need > kStaticScratchBytes)
        return set_error(h, ENS_EINVAL, "ens_pcg_solve_static: this problem needs " + std::to_string(need) +
                                            " bytes of scratch; the static scratch holds " +
                                            std::to_string(kStaticScratchBytes) + " (use ens_pcg_solve)");
    void *scratch = nullptr;
    rc = scratch_address(h, &scratch);
    if (rc) return rc;
    Args a;
    memset(&a, 0, sizeof(a));
    a.J = J; a.S = S; a.E = E; a.maxit = maxit; a.nnz = nnz; a.rtol = rtol; a.g = g;
    a.rowptr = rowptr; a.colidx = colidx; a.vals = vals; a.dinv = dinv; a.b = b; a.x = x;
    a.active = active; a.iters = iters; a.status = status; a.relres = relres;
    a.trip_cap = maxit;
    layout(J, S, E, g, &a.w, (char *)scratch);
    // The array keeps the previous call's contents: run_solve clears the
    // counters and the loop control; everything else is written before it is read.
    return run_solve<double>(h, a, (cudaStream_t)stream, true);
}

extern "C" int ens_spmv(ens_handle h, int J, int64_t nnz, int S, int E, const int32_t *rowptr,
                        const int32_t *colidx, const double *vals, const double *p, double *q, double *pq,
                        void *work, size_t work_bytes, void *stream)
{
    if (!h) return ENS_EINVAL;
    if (!lane_count_ok(S)) return set_error(h, ENS_EINVAL, "ens_spmv: S must be 1,2,4,...,64");
    if (J <= 0 || nnz <= 0 || E < 0 || E > 65535 || nnz >= (1LL << 31))
        return set_error(h, ENS_EINVAL, "ens_spmv: bad sizes");
    if (E == 0) return ENS_OK;
    if (!rowptr || !colidx || !vals || !p || !q || !work) return set_error(h, ENS_EINVAL, "ens_spmv: null pointer");
    if (((uintptr_t)vals | (uintptr_t)p | (uintptr_t)q | (uintptr_t)work) & 15)
        return set_error(h, ENS_EINVAL, "ens_spmv: arrays must be 16-byte aligned");
    if (h->check) {
        int crc = check_pattern(h, "ens_spmv", J, nnz, rowptr, colidx, (cudaStream_t)stream);
        if (crc) return crc;
    }
    Geo g = geometry(J, S, E);
    const size_t need = layout(J, S, E, g, nullptr, nullptr);
    if (work_bytes < need) return set_error(h, ENS_ENOMEM, "ens_spmv: workspace too small");
    Args a;
    memset(&a, 0, sizeof(a));
    a.J = J; a.S = S; a.E = E; a.nnz = nnz; a.g = g;
    a.rowptr = rowptr; a.colidx = colidx; a.vals = vals;
    layout(J, S, E, g, &a.w, (char *)work);
    a.w.p = const_cast<double *>(p);
    a.w.q = q;
    a.pq_out = pq ? pq : a.w.alpha;
    cudaStream_t st = (cudaStream_t)stream;
    ENS_CUDA_CHECK(h, cudaMemsetAsync(a.w.counter, 0, (size_t)E * CNT_KINDS * sizeof(int), st));
    k_spmv_prep<<<(E * S + 255) / 256, 256, 0, st>>>(a);
    ENS_LAUNCH_CHECK(h, "ens_spmv: prep");
    dispatch_spmv<double>(a, st);
    ENS_LAUNCH_CHECK(h, "ens_spmv: kernel");
    return ENS_OK;
}

// ---- per-sample quantity of interest ---------------------------------------------
// One block per ensemble; thread t owns lane t % S and rows t / S, t / S + 1024 / S, ...
// so the per-lane sum has a fixed order (rows in stride, then the threads of a lane
// pairwise: thread group g with g + st for st = G/2, ..., 1).
namespace ens {
namespace {
__global__ void __launch_bounds__(1024) k_qoi(int J, int S, const double *__restrict__ x,
                                              const double *__restrict__ w, double *__restrict__ out)
{
    extern __shared__ double sh[];
    const int e = blockIdx.x, t = threadIdx.x;
    const int s = t % S, g = t / S, G = blockDim.x / S;
    const double *xe = x + (size_t)e * J * S;
    double acc = 0.0;
    for (int j = g; j < J; j += G) {
        double v = xe[(size_t)j * S + s];
        acc = fma(w ? w[j] : v, v, acc);
    }
    sh[t] = acc;
    __syncthreads();
    for (int st = G / 2; st > 0; st >>= 1) {
        if (g < st) sh[t] = dadd(sh[t], sh[t + st * S]);
        __syncthreads();
    }
    if (t < S) out[(size_t)e * S + t] = sh[t];
}
}  // namespace
}  // namespace ens

extern "C" int ens_qoi(ens_handle h, int J, int S, int E, const double *x, const double *w, double *out,
                       void *stream)
{
    if (!h) return ENS_EINVAL;
    if (!lane_count_ok(S) || J <= 0 || E < 0) return set_error(h, ENS_EINVAL, "ens_qoi: bad J / S / E");
    if (E == 0) return ENS_OK;
    if (!x || !out) return set_error(h, ENS_EINVAL, "ens_qoi: null pointer");
    k_qoi<<<E, 1024, 1024 * sizeof(double), (cudaStream_t)stream>>>(J, S, x, w, out);
    ENS_LAUNCH_CHECK(h, "ens_qoi");
    return ENS_OK;
}
