// pcg.cu -- ensemble Jacobi-PCG with per-sample inner products (K2, K3, K4).
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
//   K2  q = A p (CSR, one column index per nonzero for all S lanes, the S
//       values as 16-byte vector loads), partial p^T q       -> alpha
//   K3  x += alpha p, r -= alpha q, partial r^T r, r^T D^-1 r  -> convergence, beta
//   K4  p = D^-1 r + beta p; block (0,0) also drives the graph's while loop.
// Arithmetic: GB300 issues about two FP64 operations per clock per SM, which
// is the binding limit of these kernels before HBM is, so every
// multiply-accumulate is one fused multiply-add (the per-row sums keep the
// oracle's column order; only the rounding of each step differs from it).
//
// The loop is one CUDA graph: a conditional WHILE node whose body holds K2-K4
// and whose condition K4 sets to (live lanes > 0 && trips < maxit), so the
// host launches one graph per solve and never waits inside it.
#include "ens_common.cuh"

#include <cmath>
#include <cstring>
#include <mutex>

namespace ens {

namespace {

enum { CTL_NLIVE = 0, CTL_TRIPS = 1, CTL_WORDS = 16 };
enum { CNT_INIT = 0, CNT_SPMV = 1, CNT_UPD = 2, CNT_KINDS = 4 };

struct Ws {
    double *r, *p, *q;      // [E][J][S]
    double *part0, *part1;  // [E][nblk][S]
    double *bnorm, *rz, *alpha, *beta, *rr;  // [E][S]
    int *k, *live;          // [E][S]
    int *ens_live;          // [E]
    int *counter;           // [E][CNT_KINDS]
    int *ctl;               // [CTL_WORDS]
};

struct Geo {
    int nblk;  // blocks per ensemble
    int RT;    // rows per block
};

struct Args {
    int J, S, E, maxit;
    long long nnz;
    double rtol;
    Geo g;
    const int32_t *rowptr, *colidx;
    const double *vals, *dinv, *b;
    double *x;
    const uint8_t *active;
    int32_t *iters, *status;
    double *relres;
    Ws w;
    double *pq_out;  // ens_spmv: write p^T q per lane here instead of alpha
    int in_graph;    // K4 drives the graph's while loop (else the host loops)
    cudaGraphConditionalHandle cond;
};

// Rows per block: at least 256 (so the per-block reduction tail is amortised
// over enough rows) and enough to give about four blocks per SM for one
// ensemble; a multiple of 256, so every kernel's row pass divides it.  The
// geometry depends on J only, so a lane's reduction order is the same for any
// E and any lane position.
Geo geometry(int J, int S)
{
    (void)S;
    const long long target = 152LL * 4;
    long long RT = ((long long)J + target - 1) / target;
    if (RT < 256) RT = 256;
    RT = (RT + 255) / 256 * 256;
    Geo g;
    g.RT = (int)RT;
    g.nblk = (int)((J + RT - 1) / RT);
    return g;
}

size_t layout(int J, int S, int E, const Geo &g, Ws *w, char *base)
{
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align256(off + bytes);
        return base ? (void *)(base + o) : nullptr;
    };
    size_t vec = (size_t)E * J * S * sizeof(double);
    size_t part = (size_t)E * g.nblk * S * sizeof(double);
    size_t lane = (size_t)E * S;
    Ws t;
    t.r = (double *)take(vec);
    t.p = (double *)take(vec);
    t.q = (double *)take(vec);
    t.part0 = (double *)take(part);
    t.part1 = (double *)take(part);
    t.bnorm = (double *)take(lane * 8);
    t.rz = (double *)take(lane * 8);
    t.alpha = (double *)take(lane * 8);
    t.beta = (double *)take(lane * 8);
    t.rr = (double *)take(lane * 8);
    t.k = (int *)take(lane * 4);
    t.live = (int *)take(lane * 4);
    t.ens_live = (int *)take((size_t)E * 4);
    t.counter = (int *)take((size_t)E * CNT_KINDS * 4);
    t.ctl = (int *)take(CTL_WORDS * 4);
    if (w) *w = t;
    return off;
}

// ---- lane vectors: V = 2 consecutive lanes per thread as one 16-byte access --
template <int V> struct Vec;
template <> struct Vec<1> {
    double v[1];
    __device__ __forceinline__ void load(const double *p) { v[0] = *p; }
    __device__ __forceinline__ void load_ro(const double *p) { v[0] = __ldg(p); }
    __device__ __forceinline__ void load_stream(const double *p) { v[0] = __ldcs(p); }
    __device__ __forceinline__ void store(double *p) const { *p = v[0]; }
};
template <> struct Vec<2> {
    double v[2];
    __device__ __forceinline__ void load(const double *p)
    {
        double2 t = *reinterpret_cast<const double2 *>(p);
        v[0] = t.x;
        v[1] = t.y;
    }
    __device__ __forceinline__ void load_stream(const double *p)
    {
        double2 t = __ldcs(reinterpret_cast<const double2 *>(p));
        v[0] = t.x;
        v[1] = t.y;
    }
    __device__ __forceinline__ void load_ro(const double *p)
    {
        double2 t = __ldg(reinterpret_cast<const double2 *>(p));
        v[0] = t.x;
        v[1] = t.y;
    }
    __device__ __forceinline__ void store(double *p) const
    {
        *reinterpret_cast<double2 *>(p) = make_double2(v[0], v[1]);
    }
};

// V lanes per thread.  The vector kernels (K0, K3, K4) take two lanes per
// thread as one 16-byte access; the SpMV (K2) takes one lane per thread, which
// halves its registers and doubles its resident warps -- it is bound by the
// FP64 issue rate, and more independent multiply-add chains per SM keep that
// pipe busier (two lanes per thread are kept only for S = 64, so a row stays
// within one warp).
template <int S, int V_> struct LaneGeo {
    static constexpr int V = V_;
    static constexpr int TPR = S / V;          // threads per row
    static constexpr int RPP = kBlock / TPR;   // rows per block pass
    static constexpr int G = kBlock / S;       // groups in the final cross-block sum
};
template <int S> using VecGeo = LaneGeo<S, (S >= 2 ? 2 : 1)>;
template <int S> using SpmvGeo = LaneGeo<S, (S >= 64 ? 2 : 1)>;

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
        const int g = tid / S, s = tid % S;
#pragma unroll
        for (int ns = 0; ns < NS; ns++) {
            double v = 0.0;
            const double *pb = part_base[ns] + (size_t)e * nblk * S;
            for (int b = g; b < nblk; b += LG::G) v = dadd(v, __ldcg(pb + (size_t)b * S + s));
            grp[g][ns][s] = v;
        }
    }
    __syncthreads();
    if (tid < S) {
#pragma unroll
        for (int ns = 0; ns < NS; ns++) {
            double v = 0.0;
            for (int g = 0; g < LG::G; g++) v = dadd(v, grp[g][ns][tid]);
            tot[ns * S + tid] = v;
        }
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

// ---- K0: x = 0, r = b, p = D^-1 b; b^T b and r^T D^-1 r per lane ------------
// Streamed arrays are passed as kernel parameters: read out of the by-value
// Args struct instead, their loads were measured to lose half of the kernel's
// memory-level parallelism on sm_103a.
template <int S>
__global__ void __launch_bounds__(kBlock) k_init(Args a, const double *__restrict__ bb, const double *__restrict__ dinv,
                                                 double *__restrict__ xx, double *__restrict__ rr,
                                                 double *__restrict__ pp)
{
    using LG = VecGeo<S>;
    constexpr int V = LG::V, TPR = LG::TPR, RPP = LG::RPP;
    const int e = blockIdx.y;
    const int lane0 = (threadIdx.x % TPR) * V;
    const size_t vbase = (size_t)e * a.J * S;
    double acc[2][V] = {};
    const int r0 = blockIdx.x * a.g.RT, r1 = min(a.J, r0 + a.g.RT);
    for (int r = r0 + threadIdx.x / TPR; r < r1; r += RPP) {
        size_t o = vbase + (size_t)r * S + lane0;
        Vec<V> bv, dv, xv, pv;
        bv.load_ro(bb + o);
        dv.load_ro(dinv + o);
#pragma unroll
        for (int v = 0; v < V; v++) {
            xv.v[v] = 0.0;
            pv.v[v] = dv.v[v] * bv.v[v];
            acc[0][v] = fma(bv.v[v], bv.v[v], acc[0][v]);
            acc[1][v] = fma(bv.v[v], pv.v[v], acc[1][v]);
        }
        xv.store(xx + o);
        bv.store(rr + o);
        pv.store(pp + o);
    }
    __shared__ double tot[2 * S];
    __shared__ int dead;
    if (threadIdx.x == 0) dead = 0;
    double *parts[2] = {a.w.part0, a.w.part1};
    if (!reduce_lanes<LG, S, 2>(acc, parts, e, a.g.nblk, a.w.counter + e * CNT_KINDS + CNT_INIT, tot)) return;
    int *live_cnt = &dead;  // counts live lanes here
    if (threadIdx.x < S) {
        const int s = threadIdx.x, L = e * S + s;
        const double bb = tot[s], rz = tot[S + s];
        const int act = a.active ? (int)a.active[L] : 1;
        a.w.k[L] = 0;
        int live = 0;
        if (!act) {
            a.status[L] = ENS_LANE_INACTIVE; a.iters[L] = 0; a.relres[L] = 0.0;
        } else if (!isfinite(bb) || !isfinite(rz)) {
            a.status[L] = ENS_LANE_BADINPUT; a.iters[L] = 0; a.relres[L] = __longlong_as_double(0x7ff8000000000000LL);
        } else if (bb == 0.0) {
            a.status[L] = ENS_LANE_CONVERGED; a.iters[L] = 0; a.relres[L] = 0.0;
        } else if (a.maxit <= 0) {
            a.status[L] = ENS_LANE_MAXIT; a.iters[L] = 0; a.relres[L] = 1.0;
        } else {
            live = 1;
            a.w.bnorm[L] = sqrt(bb);
            a.w.rz[L] = rz;
            a.w.rr[L] = bb;
            a.status[L] = ENS_LANE_MAXIT;
            a.iters[L] = 0;
            a.relres[L] = 1.0;
        }
        a.w.live[L] = live;
        if (live) atomicAdd(live_cnt, 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        a.w.ens_live[e] = *live_cnt;
        atomicAdd(a.w.ctl + CTL_NLIVE, *live_cnt);
    }
}

// ---- K2: q = A p and p^T q per lane -> alpha -----------------------------------
constexpr int kChunk = 9;  // nonzeros loaded together per row (covers the 5/7/9-point rows)

template <int S>
__global__ void __launch_bounds__(kBlock, (S >= 64 ? 2 : (S == 1 ? 3 : 4)))
    k_spmv(Args a, const int32_t *__restrict__ rowptr, const int32_t *__restrict__ colidx,
           const double *__restrict__ vals_all, const double *__restrict__ p_all, double *__restrict__ q_all)
{
    using LG = SpmvGeo<S>;
    constexpr int V = LG::V, TPR = LG::TPR, RPP = LG::RPP;
    const int e = blockIdx.y;
    if (a.w.ens_live[e] == 0) return;
    const int lane0 = (threadIdx.x % TPR) * V;
    const int L0 = e * S + lane0;
    bool mine = a.w.live[L0] != 0;
    if (V == 2) mine = mine || a.w.live[L0 + 1] != 0;
    double acc[1][V] = {};
    if (mine) {
        const double *__restrict__ vals = vals_all + (size_t)e * a.nnz * S + lane0;
        const double *__restrict__ p = p_all + (size_t)e * a.J * S + lane0;
        double *__restrict__ q = q_all + (size_t)e * a.J * S + lane0;
        const int r0 = blockIdx.x * a.g.RT, r1 = min(a.J, r0 + a.g.RT);
        for (int r = r0 + threadIdx.x / TPR; r < r1; r += RPP) {
            const int k0 = __ldg(rowptr + r), k1 = __ldg(rowptr + r + 1);
            double s[V];
#pragma unroll
            for (int v = 0; v < V; v++) s[v] = 0.0;
            for (int kb = k0; kb < k1; kb += kChunk) {
                int c[kChunk];
                Vec<V> av[kChunk], xv[kChunk];
#pragma unroll
                for (int u = 0; u < kChunk; u++)
                    if (kb + u < k1) c[u] = __ldg(colidx + kb + u);
#pragma unroll
                for (int u = 0; u < kChunk; u++)
                    if (kb + u < k1) {
                        av[u].load_stream(vals + (size_t)(kb + u) * S);
                        xv[u].load_ro(p + (size_t)c[u] * S);
                    }
#pragma unroll
                for (int u = 0; u < kChunk; u++)
                    if (kb + u < k1) {
#pragma unroll
                        for (int v = 0; v < V; v++) s[v] = fma(av[u].v[v], xv[u].v[v], s[v]);
                    }
            }
            Vec<V> qv, pr;
#pragma unroll
            for (int v = 0; v < V; v++) qv.v[v] = s[v];
            qv.store(q + (size_t)r * S);
            pr.load_ro(p + (size_t)r * S);
#pragma unroll
            for (int v = 0; v < V; v++) acc[0][v] = fma(pr.v[v], s[v], acc[0][v]);
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

// ---- K3: x += alpha p, r -= alpha q; r^T r and r^T D^-1 r -> convergence, beta ----
template <int S>
__global__ void __launch_bounds__(kBlock) k_update(Args a, double *__restrict__ xx, double *__restrict__ rr,
                                                   const double *__restrict__ pp, const double *__restrict__ qq,
                                                   const double *__restrict__ dinv)
{
    using LG = VecGeo<S>;
    constexpr int V = LG::V, TPR = LG::TPR, RPP = LG::RPP;
    const int e = blockIdx.y;
    if (a.w.ens_live[e] == 0) return;
    const int lane0 = (threadIdx.x % TPR) * V;
    const int L0 = e * S + lane0;
    int lv[V];
    double al[V];
    bool mine = false;
#pragma unroll
    for (int v = 0; v < V; v++) {
        lv[v] = a.w.live[L0 + v];
        al[v] = lv[v] ? a.w.alpha[L0 + v] : 0.0;
        mine = mine || lv[v];
    }
    double acc[2][V] = {};
    if (mine) {
        const size_t vb = (size_t)e * a.J * S + lane0;
        const int r0 = blockIdx.x * a.g.RT, r1 = min(a.J, r0 + a.g.RT);
        for (int r = r0 + threadIdx.x / TPR; r < r1; r += RPP) {
            const size_t o = vb + (size_t)r * S;
            Vec<V> xv, rv, pv, qv, dv;
            xv.load(xx + o);
            rv.load(rr + o);
            pv.load_ro(pp + o);
            qv.load_ro(qq + o);
            dv.load_ro(dinv + o);
#pragma unroll
            for (int v = 0; v < V; v++) {
                if (!lv[v]) continue;  // frozen lane: keep x and r
                xv.v[v] = fma(al[v], pv.v[v], xv.v[v]);
                rv.v[v] = fma(-al[v], qv.v[v], rv.v[v]);
                acc[0][v] = fma(rv.v[v], rv.v[v], acc[0][v]);
                acc[1][v] = fma(rv.v[v], dv.v[v] * rv.v[v], acc[1][v]);
            }
            xv.store(xx + o);
            rv.store(rr + o);
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
            const double rr = tot[threadIdx.x], rzn = tot[S + threadIdx.x];
            a.w.rr[L] = rr;
            const double res = sqrt(rr);
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

// ---- K4: p = D^-1 r + beta p; loop control -------------------------------------
template <int S>
__global__ void __launch_bounds__(kBlock) k_direction(Args a, const double *__restrict__ rr,
                                                      const double *__restrict__ dinv, double *__restrict__ pp)
{
    using LG = VecGeo<S>;
    constexpr int V = LG::V, TPR = LG::TPR, RPP = LG::RPP;
    const int e = blockIdx.y;
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) {
        // K3 has finished for every ensemble, so the live count is final here.
        const int trips = a.w.ctl[CTL_TRIPS] + 1;
        a.w.ctl[CTL_TRIPS] = trips;
        const int more = (a.w.ctl[CTL_NLIVE] > 0) && (trips < a.maxit);
        if (a.in_graph) cudaGraphSetConditional(a.cond, more ? 1u : 0u);
    }
    if (a.w.ens_live[e] == 0) return;
    const int lane0 = (threadIdx.x % TPR) * V;
    const int L0 = e * S + lane0;
    int lv[V];
    double be[V];
    bool mine = false;
#pragma unroll
    for (int v = 0; v < V; v++) {
        lv[v] = a.w.live[L0 + v];
        be[v] = lv[v] ? a.w.beta[L0 + v] : 0.0;
        mine = mine || lv[v];
    }
    if (!mine) return;
    const size_t vb = (size_t)e * a.J * S + lane0;
    const int r0 = blockIdx.x * a.g.RT, r1 = min(a.J, r0 + a.g.RT);
    for (int r = r0 + threadIdx.x / TPR; r < r1; r += RPP) {
        const size_t o = vb + (size_t)r * S;
        Vec<V> rv, dv, pv;
        rv.load_ro(rr + o);
        dv.load_ro(dinv + o);
        pv.load(pp + o);
#pragma unroll
        for (int v = 0; v < V; v++)
            if (lv[v]) pv.v[v] = fma(be[v], pv.v[v], dv.v[v] * rv.v[v]);
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

template <int S>
void launch_spmv(const Args &a, cudaStream_t st)
{
    dim3 grid(a.g.nblk, a.E);
    k_spmv<S><<<grid, kBlock, 0, st>>>(a, a.rowptr, a.colidx, a.vals, a.w.p, a.w.q);
}

void dispatch_spmv(const Args &a, cudaStream_t st)
{
    switch (a.S) {
    case 1: launch_spmv<1>(a, st); break;
    case 2: launch_spmv<2>(a, st); break;
    case 4: launch_spmv<4>(a, st); break;
    case 8: launch_spmv<8>(a, st); break;
    case 16: launch_spmv<16>(a, st); break;
    case 32: launch_spmv<32>(a, st); break;
    default: launch_spmv<64>(a, st); break;
    }
}

template <int S>
void launch_body(const Args &a, cudaStream_t st)
{
    dim3 grid(a.g.nblk, a.E);
    k_spmv<S><<<grid, kBlock, 0, st>>>(a, a.rowptr, a.colidx, a.vals, a.w.p, a.w.q);
    k_update<S><<<grid, kBlock, 0, st>>>(a, a.x, a.w.r, a.w.p, a.w.q, a.dinv);
    k_direction<S><<<grid, kBlock, 0, st>>>(a, a.w.r, a.dinv, a.w.p);
}

template <int S>
void launch_init(const Args &a, cudaStream_t st)
{
    dim3 grid(a.g.nblk, a.E);
    k_init<S><<<grid, kBlock, 0, st>>>(a, a.b, a.dinv, a.x, a.w.r, a.w.p);
}

void dispatch_body(const Args &a, cudaStream_t st)
{
    switch (a.S) {
    case 1: launch_body<1>(a, st); break;
    case 2: launch_body<2>(a, st); break;
    case 4: launch_body<4>(a, st); break;
    case 8: launch_body<8>(a, st); break;
    case 16: launch_body<16>(a, st); break;
    case 32: launch_body<32>(a, st); break;
    default: launch_body<64>(a, st); break;
    }
}

void dispatch_init(const Args &a, cudaStream_t st)
{
    switch (a.S) {
    case 1: launch_init<1>(a, st); break;
    case 2: launch_init<2>(a, st); break;
    case 4: launch_init<4>(a, st); break;
    case 8: launch_init<8>(a, st); break;
    case 16: launch_init<16>(a, st); break;
    case 32: launch_init<32>(a, st); break;
    default: launch_init<64>(a, st); break;
    }
}

uint64_t bits(const void *p) { return (uint64_t)(uintptr_t)p; }
uint64_t bits(double d)
{
    uint64_t u;
    memcpy(&u, &d, 8);
    return u;
}

// Instantiate (or reuse) the while-loop graph for these arguments.
int loop_graph(ens_ctx *h, Args a, cudaGraphExec_t *out)
{
    std::vector<uint64_t> key = {bits(a.rowptr), bits(a.colidx), bits(a.vals), bits(a.dinv), bits(a.b),
                                 bits(a.x), bits(a.active), bits(a.iters), bits(a.status), bits(a.relres),
                                 bits(a.w.r), (uint64_t)a.J, (uint64_t)a.S, (uint64_t)a.E,
                                 (uint64_t)a.maxit, (uint64_t)a.nnz, bits(a.rtol),
                                 (uint64_t)a.g.nblk, (uint64_t)a.g.RT};
    h->clock++;
    for (auto &ge : h->graphs)
        if (ge.key == key) {
            ge.last_use = h->clock;
            *out = ge.exec;
            return ENS_OK;
        }
    cudaGraph_t g = nullptr;
    ENS_CUDA_CHECK(h, cudaGraphCreate(&g, 0));
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
    a.cond = cond;
    a.in_graph = 1;
    e = cudaStreamBeginCaptureToGraph(h->capture, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return cuda_error(h, e, "cudaStreamBeginCaptureToGraph");
    }
    dispatch_body(a, h->capture);
    cudaError_t le = cudaGetLastError();
    cudaGraph_t captured = nullptr;
    e = cudaStreamEndCapture(h->capture, &captured);
    if (le != cudaSuccess || e != cudaSuccess) {
        cudaGraphDestroy(g);
        return cuda_error(h, le != cudaSuccess ? le : e, "capturing the PCG loop body");
    }
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, g, 0);
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

}  // namespace
}  // namespace ens

using namespace ens;

extern "C" size_t ens_pcg_workspace_size(int J, int64_t nnz, int S, int E)
{
    (void)nnz;
    if (J <= 0 || E <= 0 || !lane_count_ok(S)) return 0;
    return layout(J, S, E, geometry(J, S), nullptr, nullptr);
}

extern "C" int ens_pcg_solve(ens_handle h, int J, int64_t nnz, int S, int E, const int32_t *rowptr,
                             const int32_t *colidx, const double *vals, const double *dinv, const double *b,
                             double *x, const uint8_t *active, double rtol, int maxit, int32_t *iters,
                             double *relres, int32_t *status, void *work, size_t work_bytes, void *stream)
{
    if (!h) return ENS_EINVAL;
    if (!lane_count_ok(S)) return set_error(h, ENS_EINVAL, "ens_pcg_solve: S must be 1,2,4,...,64");
    if (J <= 0 || nnz <= 0 || E < 0 || nnz >= (1LL << 31))
        return set_error(h, ENS_EINVAL, "ens_pcg_solve: bad J / nnz / E");
    if (E == 0) return ENS_OK;
    if (!(rtol >= 0.0) || maxit < 0) return set_error(h, ENS_EINVAL, "ens_pcg_solve: bad rtol / maxit");
    if (!rowptr || !colidx || !vals || !dinv || !b || !x || !iters || !relres || !status || !work)
        return set_error(h, ENS_EINVAL, "ens_pcg_solve: null pointer");
    if (((uintptr_t)vals | (uintptr_t)dinv | (uintptr_t)b | (uintptr_t)x | (uintptr_t)work) & 15)
        return set_error(h, ENS_EINVAL, "ens_pcg_solve: arrays must be 16-byte aligned");
    Geo g = geometry(J, S);
    const size_t need = layout(J, S, E, g, nullptr, nullptr);
    if (work_bytes < need)
        return set_error(h, ENS_ENOMEM, "ens_pcg_solve: workspace too small (need " + std::to_string(need) + " bytes)");
    Args a;
    memset(&a, 0, sizeof(a));
    a.J = J; a.S = S; a.E = E; a.maxit = maxit; a.nnz = nnz; a.rtol = rtol; a.g = g;
    a.rowptr = rowptr; a.colidx = colidx; a.vals = vals; a.dinv = dinv; a.b = b; a.x = x;
    a.active = active; a.iters = iters; a.status = status; a.relres = relres;
    layout(J, S, E, g, &a.w, (char *)work);
    cudaStream_t st = (cudaStream_t)stream;
    ENS_CUDA_CHECK(h, cudaMemsetAsync(a.w.counter, 0, (size_t)E * CNT_KINDS * sizeof(int), st));
    ENS_CUDA_CHECK(h, cudaMemsetAsync(a.w.ctl, 0, CTL_WORDS * sizeof(int), st));
    dispatch_init(a, st);
    ENS_LAUNCH_CHECK(h, "ens_pcg_solve: init kernel");
    if (h->host_loop) {
        // Same kernels launched from the host, with the live count read back
        // every 16 trips (profilers see each launch; the graph path does not
        // expose kernels inside a conditional body to them).
        int ctl[2] = {1, 0};
        while (ctl[0] > 0 && ctl[1] < maxit) {
            for (int t = 0; t < 16; t++) dispatch_body(a, st);
            ENS_LAUNCH_CHECK(h, "ens_pcg_solve: loop kernels");
            ENS_CUDA_CHECK(h, cudaMemcpyAsync(ctl, a.w.ctl, sizeof(ctl), cudaMemcpyDeviceToHost, st));
            ENS_CUDA_CHECK(h, cudaStreamSynchronize(st));
        }
    } else {
        cudaGraphExec_t exec;
        int rc = loop_graph(h, a, &exec);
        if (rc) return rc;
        ENS_CUDA_CHECK(h, cudaGraphLaunch(exec, st));
    }
    k_finish<<<(E * S + 255) / 256, 256, 0, st>>>(a);
    ENS_LAUNCH_CHECK(h, "ens_pcg_solve: finish kernel");
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
    if (!lane_count_ok(S)) return set_error(h, ENS_EINVAL, "ens_pcg_solve_static: S must be 1,2,4,...,64");
    if (J <= 0 || nnz <= 0 || E < 0 || nnz >= (1LL << 31))
        return set_error(h, ENS_EINVAL, "ens_pcg_solve_static: bad J / nnz / E");
    if (E == 0) return ENS_OK;
    if (!(rtol >= 0.0) || maxit < 0) return set_error(h, ENS_EINVAL, "ens_pcg_solve_static: bad rtol / maxit");
    if (!rowptr || !colidx || !vals || !dinv || !b || !x || !iters || !relres || !status)
        return set_error(h, ENS_EINVAL, "ens_pcg_solve_static: null pointer");
    if (((uintptr_t)vals | (uintptr_t)dinv | (uintptr_t)b | (uintptr_t)x) & 15)
        return set_error(h, ENS_EINVAL, "ens_pcg_solve_static: arrays must be 16-byte aligned");
    Geo g = geometry(J, S);
    const size_t need = layout(J, S, E, g, nullptr, nullptr);
    if (need > kStaticScratchBytes)
        return set_error(h, ENS_EINVAL, "ens_pcg_solve_static: this problem needs " + std::to_string(need) +
                                            " bytes of scratch; the static scratch holds " +
                                            std::to_string(kStaticScratchBytes) + " (use ens_pcg_solve)");
    void *scratch = nullptr;
    int rc = scratch_address(h, &scratch);
    if (rc) return rc;
    Args a;
    memset(&a, 0, sizeof(a));
    a.J = J; a.S = S; a.E = E; a.maxit = maxit; a.nnz = nnz; a.rtol = rtol; a.g = g;
    a.rowptr = rowptr; a.colidx = colidx; a.vals = vals; a.dinv = dinv; a.b = b; a.x = x;
    a.active = active; a.iters = iters; a.status = status; a.relres = relres;
    layout(J, S, E, g, &a.w, (char *)scratch);
    cudaStream_t st = (cudaStream_t)stream;
    // The array keeps the previous call's contents: the counters and the loop
    // control start from zero here; everything else is written before it is read.
    ENS_CUDA_CHECK(h, cudaMemsetAsync(a.w.counter, 0, (size_t)E * CNT_KINDS * sizeof(int), st));
    ENS_CUDA_CHECK(h, cudaMemsetAsync(a.w.ctl, 0, CTL_WORDS * sizeof(int), st));
    dispatch_init(a, st);
    ENS_LAUNCH_CHECK(h, "ens_pcg_solve_static: init kernel");
    int ctl[2] = {1, 0};
    while (ctl[0] > 0 && ctl[1] < maxit) {
        for (int t = 0; t < 16; t++) dispatch_body(a, st);
        ENS_LAUNCH_CHECK(h, "ens_pcg_solve_static: loop kernels");
        ENS_CUDA_CHECK(h, cudaMemcpyAsync(ctl, a.w.ctl, sizeof(ctl), cudaMemcpyDeviceToHost, st));
        ENS_CUDA_CHECK(h, cudaStreamSynchronize(st));
    }
    k_finish<<<(E * S + 255) / 256, 256, 0, st>>>(a);
    ENS_LAUNCH_CHECK(h, "ens_pcg_solve_static: finish kernel");
    return ENS_OK;
}

extern "C" int ens_spmv(ens_handle h, int J, int64_t nnz, int S, int E, const int32_t *rowptr,
                        const int32_t *colidx, const double *vals, const double *p, double *q, double *pq,
                        void *work, size_t work_bytes, void *stream)
{
    if (!h) return ENS_EINVAL;
    if (!lane_count_ok(S)) return set_error(h, ENS_EINVAL, "ens_spmv: S must be 1,2,4,...,64");
    if (J <= 0 || nnz <= 0 || E < 0 || nnz >= (1LL << 31)) return set_error(h, ENS_EINVAL, "ens_spmv: bad sizes");
    if (E == 0) return ENS_OK;
    if (!rowptr || !colidx || !vals || !p || !q || !work) return set_error(h, ENS_EINVAL, "ens_spmv: null pointer");
    if (((uintptr_t)vals | (uintptr_t)p | (uintptr_t)q | (uintptr_t)work) & 15)
        return set_error(h, ENS_EINVAL, "ens_spmv: arrays must be 16-byte aligned");
    Geo g = geometry(J, S);
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
    dispatch_spmv(a, st);
    ENS_LAUNCH_CHECK(h, "ens_spmv: kernel");
    return ENS_OK;
}

// ---- per-sample quantity of interest ---------------------------------------------
// One block per ensemble; thread t owns lane t % S and rows t / S, t / S + 1024 / S, ...
// so the per-lane sum has a fixed order (rows in stride, then the threads of a lane).
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
    if (t < S) {
        double v = 0.0;
        for (int q = 0; q < G; q++) v = dadd(v, sh[q * S + t]);
        out[(size_t)e * S + t] = v;
    }
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
