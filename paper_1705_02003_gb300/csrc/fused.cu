// fused.cu -- the ensemble Jacobi-PCG of a small problem as one launch.
//
// On a problem of at most 1024 unknowns, one trip of the three-kernel loop
// (pcg.cu) holds well under a microsecond of work per ensemble.  The three
// kernel launches and two grid-wide reductions around that work take about
// 20 us, so the trip's time is launch and memory latency.  Here one
// thread-block cluster per ensemble runs the whole solve in one launch: the
// start, every CG trip and the finish.  CTA c of the cluster owns row tile c of
// the loop's geometry (the same 64-row tiles), and the kernel boundaries become
// cluster barriers.
//
// The state stays on chip.  A CTA keeps its tile's rows of x, r and q, and its
// tile's pattern, values and D^-1 when they fit, in shared memory, with windows
// of p and z that cover every column its rows touch.  K3 stores each new row of
// z into the z window of every CTA that holds the row, through distributed
// shared memory, and after the barrier that closes K3 every CTA forms the new p
// over its whole window itself.  A trip then takes two cluster barriers.  When
// some CTA's window would not fit, p lives in global memory instead and a third
// barrier follows the direction update.
//
// The results are bit-identical to the three-kernel loop's.  The arithmetic is
// that of Section 2.3's per-sample recurrences, performed the same way:
//   - every row and vector update is the same sequence of fused multiply-adds,
//     with the same thread-to-row mapping;
//   - a tile's partial of each per-lane sum is formed exactly as a block of the
//     loop forms it;
//   - the cross-tile stage adds the partials in the loop's order.
// The partials also travel through distributed shared memory.  Each CTA writes
// its tile's partials into every CTA of the cluster.  After the barrier every
// CTA forms the same totals, so each CTA holds an identical copy of the CG
// scalars and of every lane's state.  Decisions (freeze a lane, stop) therefore
// need no further exchange, and every CTA takes the same number of barriers.
#include "pcg_core.cuh"

#include <cmath>
#include <cstring>

namespace ens {
namespace pcgi {
namespace {

constexpr int kMaxCluster = 16;  // CTAs per ensemble (above 8 the cluster size is non-portable)
constexpr int kTile = 64;        // rows per tile (the loop's geometry for J <= 4096)
constexpr int kWindow = 256;     // rows of the p and z windows (the tile and up to 96 rows each side)

__device__ __forceinline__ void cluster_barrier()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ int cluster_rank()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return (int)r;
}

// The address of the shared-memory word `local` in CTA `rank` of this cluster.
__device__ __forceinline__ unsigned remote(const void *local, int rank)
{
    const unsigned la = (unsigned)__cvta_generic_to_shared(local);
    unsigned ra;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(la), "r"((unsigned)rank));
    return ra;
}

__device__ __forceinline__ void store_remote(double *local, int rank, double v)
{
    asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(remote(local, rank)), "d"(v) : "memory");
}

__device__ __forceinline__ void store_remote(int *local, int rank, int v)
{
    asm volatile("st.shared::cluster.s32 [%0], %1;" ::"r"(remote(local, rank)), "r"(v) : "memory");
}

// V consecutive lanes of one row into CTA `rank`'s copy of `local`.
template <int V>
__device__ __forceinline__ void store_remote_lanes(double *local, int rank, const double *v)
{
    if constexpr (V == 2)
        asm volatile("st.shared::cluster.v2.f64 [%0], {%1, %2};" ::"r"(remote(local, rank)), "d"(v[0]), "d"(v[1])
                     : "memory");
    else
        store_remote(local, rank, v[0]);
}

// One tile's partial of NS per-lane sums from the threads' accumulators.  The
// warp-shuffle sum and then the sum over warps in warp order are the first stage
// of the loop's block reduction.  The partial of lane s goes into slot `blk` of
// the exchange array xch[NS][nblk][S] of every CTA of the cluster; warp 0 forms
// the sums (thread s for lane s) and spreads the stores over its 32 threads.
// The caller's next cluster barrier orders these reads of wp before its next use.
template <class LG, int S, int NS>
__device__ __forceinline__ void publish_tile(double (&acc)[NS][LG::V], double (*wp)[2][S], double *xch, int nblk,
                                             int blk, int C)
{
    constexpr int V = LG::V, TPR = LG::TPR;
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
            for (int v = 0; v < V; v++) wp[wid][ns][lid * V + v] = acc[ns][v];
    }
    __syncthreads();
    if (wid == 0) {
        double sum[NS];
#pragma unroll
        for (int ns = 0; ns < NS; ns++) {
            double t = 0.0;
            if (lid < S)
                for (int w = 0; w < kBlock / 32; w++) t = dadd(t, wp[w][ns][lid]);
            sum[ns] = t;
        }
        for (int i0 = 0; i0 < C * S; i0 += 32) {
            const int i = i0 + lid, rank = i / S, s = i % S;
#pragma unroll
            for (int ns = 0; ns < NS; ns++) {
                const double v = __shfl_sync(0xffffffffu, sum[ns], s);
                if (i < C * S) store_remote(xch + ((size_t)ns * nblk + blk) * S + s, rank, v);
            }
        }
    }
}

// The totals from the exchanged partials, in the order of the loop's last
// block: with G = kBlock / S groups per lane, group g adds the partials
// g, g + G, ... in turn (starting from 0.0), and the G group sums are combined
// pairwise, g with g + G/2, ..., g with g + 1.  Here nblk <= 16, so for S <= 16
// (G >= 16) a group holds one partial at most, and every step with a partner
// at or past nblk adds +0.0 to a value that is not -0.0 (the first stage adds
// to +0.0, and sums of such values are never -0.0), which leaves it unchanged:
// those steps are skipped, leaving the pairwise tree over 16 groups.  For
// S = 32 (G = 8) the groups hold partials g and g + 8.  Thread t handles group
// g = t % GS of lane s = t / GS (GS = min(G, 16) consecutive threads per lane);
// on return thread g = 0 holds lane s's totals.  Only the warps that hold
// groups add (an FP64 warp instruction occupies the pipe for its whole warp on
// this part), but every thread must call it.
template <int S, int NS>
__device__ __forceinline__ void combine(const double *xch, int nblk, double (&tot)[NS])
{
    constexpr int G = kBlock / S, GS = G < 16 ? G : 16;
    constexpr int WORK = S * GS < 32 ? 32 : S * GS;  // threads of the warps that hold groups
    const int tid = threadIdx.x, g = tid % GS, s = tid / GS;
    const bool mine = s < S;
#pragma unroll
    for (int ns = 0; ns < NS; ns++) {
        double v = 0.0;
        if (mine)
            for (int b = g; b < nblk; b += G) v = dadd(v, xch[((size_t)ns * nblk + b) * S + s]);
        tot[ns] = v;
    }
    if (tid >= WORK) return;
#pragma unroll
    for (int st = GS / 2; st > 0; st >>= 1) {
#pragma unroll
        for (int ns = 0; ns < NS; ns++) {
            const double o = __shfl_down_sync(0xffffffffu, tot[ns], st);
            if (g < st) tot[ns] = dadd(tot[ns], o);
        }
    }
}

// With PACK, the totals that combine left in thread ls * GS (lead) move to
// thread ls, through shared memory; without it they stay where they are.
// Every thread must call it.
template <int S, int NS, bool PACK>
__device__ __forceinline__ void to_lane_threads(double (&t)[NS], bool lead, int ls, double (*ttot)[S])
{
    if constexpr (PACK) {
        if (lead) {
#pragma unroll
            for (int ns = 0; ns < NS; ns++) ttot[ns][ls] = t[ns];
        }
        __syncthreads();
        if (threadIdx.x < S) {
#pragma unroll
            for (int ns = 0; ns < NS; ns++) t[ns] = ttot[ns][threadIdx.x];
        }
    }
}

// A row of a windowed vector (V lanes from lane0) into this CTA's window and
// into the window of every other CTA that holds the row.  w is the window
// array (the same offset in every CTA); CTA k's window holds rows
// [wlo[k], whi[k]).
template <int S, int V>
__device__ __forceinline__ void put_row(int row, int lane0, const double *val, int c, int C, const int *wlo,
                                        const int *whi, double *w)
{
    for (int k = 0; k < C; k++) {
        if (row < wlo[k] || row >= whi[k]) continue;
        double *d = w + (size_t)(row - wlo[k]) * S + lane0;
        if (k == c) {
#pragma unroll
            for (int v = 0; v < V; v++) d[v] = val[v];
        } else {
            store_remote_lanes<V>(d, k, val);
        }
    }
}

// One row of K2 on the on-chip state: q_r = sum_k a_k p_{c_k} in column order
// (the fused multiply-adds of spmv_row), q_r into the tile's rows of q, and
// p_r q_r into the lane's partial.  The row's nonzeros are rp[row - r0] - kofs
// up to rp[row - r0 + 1] - kofs in cp (columns) and vp (values, offset to the
// thread's first lane): the tile's copy in shared memory, or global memory.  p
// comes from the window (pw, whose first row is lo), or from global memory
// through L2 when pw is null.  Vector pointers are offset to the first lane.
template <int S, int V, int KC>
__device__ __forceinline__ void fused_row(int row, int r0, const int *rp, int kofs, const int *cp,
                                          const double *vp, const double *pw, int lo, const double *pg, double *oq,
                                          double (&acc)[1][V])
{
    const int k0 = rp[row - r0] - kofs, k1 = rp[row - r0 + 1] - kofs;
    double s[V];
#pragma unroll
    for (int v = 0; v < V; v++) s[v] = 0.0;
    for (int kb = k0; kb < k1; kb += KC) {
        int c[KC];
        Vec<double, V> av[KC], xv[KC];
#pragma unroll
        for (int u = 0; u < KC; u++)
            if (kb + u < k1) c[u] = cp[kb + u];
#pragma unroll
        for (int u = 0; u < KC; u++)
            if (kb + u < k1) {
                av[u].load(vp + (size_t)(kb + u) * S);
                if (pw)
                    xv[u].load(pw + (size_t)(c[u] - lo) * S);
                else
                    xv[u].load_cg(pg + (size_t)c[u] * S);
            }
#pragma unroll
        for (int u = 0; u < KC; u++)
            if (kb + u < k1) {
#pragma unroll
                for (int v = 0; v < V; v++) s[v] = fma(av[u].v[v], xv[u].v[v], s[v]);
            }
    }
    Vec<double, V> qv, pr;
#pragma unroll
    for (int v = 0; v < V; v++) qv.v[v] = s[v];
    qv.store(oq + (size_t)(row - r0) * S);
    if (pw)
        pr.load(pw + (size_t)(row - lo) * S);
    else
        pr.load_cg(pg + (size_t)row * S);
#pragma unroll
    for (int v = 0; v < V; v++) acc[0][v] = fma(pr.v[v], s[v], acc[0][v]);
}

// The solve of ensemble blockIdx.y by one cluster of nblk CTAs; CTA c owns
// tile c.  K2's lane geometry is LaneGeo<S, V2> with KC-nonzero chunks, the
// variant the loop's launch_k2 picks for this pattern.  Dynamic shared memory
// (doubles): the exchange arrays xa[nblk][S] (p^T q) and xb[2][nblk][S] (the
// two-sum stages), the tile's rows of x, r and q ([kTile][S] each), the
// windows of p and z ([W][S] each), and, when vcap > 0, the tile's copy of its
// values and D^-1 ([vcap][S], [kTile][S]) followed by its column indices and
// row pointers (ints [vcap], [kTile + 1]); a tile with more than vcap nonzeros
// reads them from global memory.
//
// When every CTA's window fits (W rows), a trip takes two cluster barriers: K3
// stores each new row of z into every window that holds it before the second,
// and after it every CTA forms p = z + beta p over its whole window itself (the
// owner of a row and its neighbours compute the same fused multiply-add from
// the same values).  Otherwise p lives in global memory, z in the first rows of
// the z window, and a third barrier follows the direction update.
template <int S, int V2, int KC>
__global__ void __launch_bounds__(kBlock, 2) k_pcg_cluster(Args a, int W, int vcap)
{
    using SG = LaneGeo<S, V2>;
    using VG = VecGeo<double, S>;
    constexpr int GS = kBlock / S < 16 ? kBlock / S : 16;  // threads per lane in combine
    extern __shared__ __align__(16) double dyn[];
    __shared__ double wp[kBlock / 32][2][S];
    __shared__ double alpha[S], beta[S], rz[S], rr[S], bnorm[S];
    __shared__ int kk[S], live[S];
    __shared__ int wlo[kMaxCluster], whi[kMaxCluster];  // each CTA's window [wlo, whi); whi = 0: none
    __shared__ int s_cmin, s_cmax;

    const int e = blockIdx.y, c = cluster_rank(), nblk = a.g.nblk, C = nblk, J = a.J;
    const int r0 = c * kTile, r1 = min(J, r0 + kTile);
    const int tid = threadIdx.x, ls = tid / GS;
    const bool lead = tid % GS == 0 && ls < S;  // the thread that holds lane ls's totals after combine
    // Each lane's scalar work (divides, square roots) runs in one thread.  When
    // the combine leaves the totals in more than one warp, they first move to
    // threads 0..S-1 of warp 0: on this part an FP64 warp instruction occupies
    // the pipe for the whole warp, so eight warps dividing for two lanes each
    // cost four times one warp dividing for eight.
    constexpr bool kPack = S * GS > 32;
    __shared__ double ttot[2][S];
    const bool lt = kPack ? tid < S : lead;  // the thread that runs lane ln's logic
    const int ln = kPack ? tid : ls;
    double *xa = dyn, *xb = xa + (size_t)nblk * S;
    double *ox = xb + (size_t)2 * nblk * S, *orr = ox + kTile * S, *oq = orr + kTile * S;
    double *pwin = oq + kTile * S, *zwin = pwin + (size_t)W * S;
    double *cval = zwin + (size_t)W * S, *cdinv = cval + (size_t)vcap * S;
    int *ccol = (int *)(cdinv + (size_t)kTile * S), *crow = ccol + vcap;
    const size_t vb = (size_t)e * J * S;
    const double *__restrict__ bb = a.b + vb;
    const double *__restrict__ dinv = (const double *)a.dinv + vb;
    const double *__restrict__ vals = (const double *)a.vals + (size_t)e * a.nnz * S;
    double *pg = (double *)a.w.p + vb;
    const bool out = c == 0;  // CTA 0 writes each lane's outcome

    // ---- the windows: every column the tile's rows touch, and the tile ----
    cluster_barrier();  // every CTA of the cluster has started before any writes into another
    if (tid == 0) {
        s_cmin = r0;
        s_cmax = r1 - 1;
    }
    __syncthreads();
    {
        int mn = r0, mx = r1 - 1;
        for (int k = __ldg(a.rowptr + r0) + tid; k < __ldg(a.rowptr + r1); k += kBlock) {
            const int cc = __ldg(a.colidx + k);
            mn = min(mn, cc);
            mx = max(mx, cc);
        }
        atomicMin(&s_cmin, mn);
        atomicMax(&s_cmax, mx);
    }
    // the tile's pattern, values and D^-1 into shared memory, when they fit
    const int kb0 = __ldg(a.rowptr + r0), nt = __ldg(a.rowptr + r1) - kb0;
    const bool staged = vcap > 0 && nt <= vcap;
    if (staged) {
        for (int i = tid; i <= r1 - r0; i += kBlock) crow[i] = __ldg(a.rowptr + r0 + i) - kb0;
        for (int k = tid; k < nt; k += kBlock) ccol[k] = __ldg(a.colidx + kb0 + k);
        for (int i = tid; i < nt * S; i += kBlock) cval[i] = __ldg(vals + (size_t)kb0 * S + i);
        for (int i = tid; i < (r1 - r0) * S; i += kBlock) cdinv[i] = __ldg(dinv + (size_t)r0 * S + i);
    }
    // where the rows read their pattern, values and D^-1 from
    const int *rp = staged ? crow : a.rowptr + r0, *cp = staged ? ccol : a.colidx + kb0;
    const int kofs = staged ? 0 : kb0;
    const double *vp = staged ? cval : vals + (size_t)kb0 * S, *dp = staged ? cdinv : dinv + (size_t)r0 * S;
    __syncthreads();
    if (tid < C) {
        const bool fits = s_cmax + 1 - s_cmin <= W;
        store_remote(&wlo[c], tid, s_cmin);
        store_remote(&whi[c], tid, fits ? s_cmax + 1 : 0);
    }
    cluster_barrier();
    bool allwin = true;
    for (int k = 0; k < C; k++) allwin = allwin && whi[k] > 0;
    const int lo = allwin ? wlo[c] : r0, hi = allwin ? whi[c] : r1;  // this CTA's rows of z in zwin start at lo
    const double *pw = allwin ? pwin : nullptr;

    // ---- start: x = 0, r = b, p = D^-1 b; r^T r and r^T D^-1 r (K0) ----
    {
        constexpr int V = VG::V, TPR = VG::TPR, RPP = VG::RPP;
        const int lane0 = (tid % TPR) * V;
        double acc[2][V] = {};
        for (int row = r0 + tid / TPR; row < r1; row += RPP) {
            const size_t o = (size_t)row * S + lane0, ol = (size_t)(row - r0) * S + lane0;
            Vec<double, V> dv, xv, rv, pv;
            dv.load(dp + ol);
#pragma unroll
            for (int v = 0; v < V; v++) {
                xv.v[v] = 0.0;
                rv.v[v] = __ldg(bb + o + v);
                pv.v[v] = dv.v[v] * rv.v[v];
                acc[0][v] = fma(rv.v[v], rv.v[v], acc[0][v]);
                acc[1][v] = fma(rv.v[v], pv.v[v], acc[1][v]);
            }
            xv.store(ox + ol);
            rv.store(orr + ol);
            if (allwin)
                put_row<S, V>(row, lane0, pv.v, c, C, wlo, whi, pwin);
            else
                pv.store(pg + o);
        }
        publish_tile<VG, S, 2>(acc, wp, xb, nblk, c, C);
    }
    cluster_barrier();
    {
        double t[2];
        combine<S, 2>(xb, nblk, t);
        to_lane_threads<S, 2, kPack>(t, lead, ls, ttot);
        if (lt) {
            const int s = ln, L = e * S + s;
            const double bsq = t[0], rzs = t[1];
            const int act = a.active ? (int)a.active[L] : 1;
            int lv = 0, st;
            double rel;
            if (!act) {
                st = ENS_LANE_INACTIVE; rel = 0.0;
            } else if (!isfinite(bsq) || !isfinite(rzs)) {
                st = ENS_LANE_BADINPUT; rel = __longlong_as_double(0x7ff8000000000000LL);
            } else if (bsq == 0.0) {
                st = ENS_LANE_CONVERGED; rel = 0.0;
            } else if (a.maxit <= 0) {
                st = ENS_LANE_MAXIT; rel = 1.0;
            } else {
                lv = 1;
                bnorm[s] = sqrt(bsq);
                rz[s] = rzs;
                rr[s] = bsq;
                st = ENS_LANE_MAXIT; rel = 1.0;
            }
            kk[s] = 0;
            live[s] = lv;
            if (out) {
                a.status[L] = st;
                a.iters[L] = 0;
                a.relres[L] = rel;
            }
        }
    }
    int nl = __syncthreads_count(lt && live[ln]);

    int trips = 0;
    while (nl > 0 && trips < a.trip_cap) {
        // ---- K2: q = A p and p^T q -> alpha ----
        {
            constexpr int V = SG::V, TPR = SG::TPR, RPP = SG::RPP;
            const int lane0 = (tid % TPR) * V;
            bool mine = live[lane0] != 0;
            if (V == 2) mine = mine || live[lane0 + 1] != 0;
            double acc[1][V] = {};
            if (mine) {
                const double *pwl = pw ? pw + lane0 : nullptr;
                for (int row = r0 + tid / TPR; row < r1; row += RPP)
                    fused_row<S, V, KC>(row, r0, rp, kofs, cp, vp + lane0, pwl, lo, pg + lane0, oq + lane0, acc);
            }
            publish_tile<SG, S, 1>(acc, wp, xa, nblk, c, C);
        }
        cluster_barrier();
        {
            double t[1];
            combine<S, 1>(xa, nblk, t);
            to_lane_threads<S, 1, kPack>(t, lead, ls, ttot);
            if (lt && live[ln]) {
                const int s = ln, L = e * S + s;
                const double pq = t[0];
                if (!(pq > 0.0) || !isfinite(pq)) {
                    // zero (or invalid) A-conjugate norm: freeze, x stays as it is
                    live[s] = 0;
                    if (out) {
                        a.status[L] = ENS_LANE_BREAKDOWN;
                        a.iters[L] = kk[s];
                        a.relres[L] = sqrt(rr[s]) / bnorm[s];
                    }
                } else {
                    alpha[s] = rz[s] / pq;
                }
            }
        }
        __syncthreads();

        // ---- K3: x += alpha p, r -= alpha q, z = D^-1 r; r^T r, r^T z ----
        {
            constexpr int V = VG::V, TPR = VG::TPR, RPP = VG::RPP;
            const int lane0 = (tid % TPR) * V;
            int lv[V];
            double al[V];
            bool mine = false;
#pragma unroll
            for (int v = 0; v < V; v++) {
                lv[v] = live[lane0 + v];
                al[v] = lv[v] ? alpha[lane0 + v] : 0.0;
                mine = mine || lv[v];
            }
            double acc[2][V] = {};
            if (mine) {
                for (int row = r0 + tid / TPR; row < r1; row += RPP) {
                    const size_t ol = (size_t)(row - r0) * S + lane0;
                    Vec<double, V> xv, rv, pv, qv, dv, zv;
                    xv.load(ox + ol);
                    rv.load(orr + ol);
                    qv.load(oq + ol);
                    dv.load(dp + ol);
                    if (pw)
                        pv.load(pw + (size_t)(row - lo) * S + lane0);
                    else
                        pv.load_cg(pg + (size_t)row * S + lane0);
#pragma unroll
                    for (int v = 0; v < V; v++) {
                        zv.v[v] = 0.0;
                        if (!lv[v]) continue;  // frozen lane: keep x and r
                        xv.v[v] = fma(al[v], pv.v[v], xv.v[v]);
                        rv.v[v] = fma(-al[v], qv.v[v], rv.v[v]);
                        zv.v[v] = dv.v[v] * rv.v[v];
                        acc[0][v] = fma(rv.v[v], rv.v[v], acc[0][v]);
                        acc[1][v] = fma(rv.v[v], zv.v[v], acc[1][v]);
                    }
                    xv.store(ox + ol);
                    rv.store(orr + ol);
                    if (allwin)
                        put_row<S, V>(row, lane0, zv.v, c, C, wlo, whi, zwin);
                    else
                        zv.store(zwin + (size_t)(row - lo) * S + lane0);
                }
            }
            publish_tile<VG, S, 2>(acc, wp, xb, nblk, c, C);
        }
        cluster_barrier();  // partials of r^T r and r^T z, and (windows) the new z, are in place
        {
            double t[2];
            combine<S, 2>(xb, nblk, t);
            to_lane_threads<S, 2, kPack>(t, lead, ls, ttot);
            if (lt && live[ln]) {
                const int s = ln, L = e * S + s;
                const int k = kk[s] + 1;
                kk[s] = k;
                const double rsq = t[0], rzn = t[1];
                rr[s] = rsq;
                const double bnext = rzn / rz[s], res = sqrt(rsq), bn = bnorm[s];  // independent: overlapped
                const bool conv = res <= a.rtol * bn;
                if (conv || k >= a.maxit) {
                    live[s] = 0;
                    if (out) {
                        a.status[L] = conv ? ENS_LANE_CONVERGED : ENS_LANE_MAXIT;
                        a.iters[L] = k;
                        a.relres[L] = res / bn;
                    }
                } else {
                    beta[s] = bnext;
                    rz[s] = rzn;
                }
            }
        }
        nl = __syncthreads_count(lt && live[ln]);
        trips++;
        if (nl == 0 || trips >= a.trip_cap) break;

        // ---- K4: p = z + beta p ----
        {
            constexpr int V = VG::V, TPR = VG::TPR, RPP = VG::RPP;
            const int lane0 = (tid % TPR) * V;
            int lv[V];
            double be[V];
            bool mine = false;
#pragma unroll
            for (int v = 0; v < V; v++) {
                lv[v] = live[lane0 + v];
                be[v] = lv[v] ? beta[lane0 + v] : 0.0;
                mine = mine || lv[v];
            }
            // windows: every row of this CTA's window; else the tile's rows, in global memory
            const int w0 = allwin ? lo : r0, w1 = allwin ? hi : r1;
            if (mine) {
                for (int row = w0 + tid / TPR; row < w1; row += RPP) {
                    const size_t ow = (size_t)(row - lo) * S + lane0;
                    Vec<double, V> zv, pv;
                    zv.load(zwin + ow);
                    if (allwin)
                        pv.load(pwin + ow);
                    else
                        pv.load_cg(pg + (size_t)row * S + lane0);
#pragma unroll
                    for (int v = 0; v < V; v++)
                        if (lv[v]) pv.v[v] = fma(be[v], pv.v[v], zv.v[v]);
                    if (allwin)
                        pv.store(pwin + ow);
                    else
                        pv.store(pg + (size_t)row * S + lane0);
                }
            }
        }
        if (allwin)
            __syncthreads();  // the window's new p before this CTA's next K2
        else
            cluster_barrier();  // the new p in global memory before every CTA's next K2
    }

    // lanes still live when the trip cap stopped the loop
    if (out && lt && live[ln]) {
        const int L = e * S + ln;
        a.status[L] = ENS_LANE_MAXIT;
        a.iters[L] = kk[ln];
        a.relres[L] = sqrt(rr[ln]) / bnorm[ln];
    }
    {
        constexpr int V = VG::V, TPR = VG::TPR, RPP = VG::RPP;
        const int lane0 = (tid % TPR) * V;
        double *xg = (double *)a.x + vb;
        for (int row = r0 + tid / TPR; row < r1; row += RPP) {
            Vec<double, V> xv;
            xv.load(ox + (size_t)(row - r0) * S + lane0);
            xv.store(xg + (size_t)row * S + lane0);
        }
    }
    // no CTA leaves while another may still address its shared memory
    cluster_barrier();
}

using FusedKernel = void (*)(Args, int, int);

// The K2 variant of launch_k2 (pcg.cu) for this pattern and S, as a fused kernel.
template <int S>
FusedKernel pick_s(double row)
{
    constexpr int V1 = SpmvGeo<S>::V;
    if (row <= 5.5) {
        if constexpr (S == 16 || S == 32) return k_pcg_cluster<S, 2, 5>;
        else return k_pcg_cluster<S, V1, 5>;
    }
    if (row <= 7.5) {
        if constexpr (S == 32) return k_pcg_cluster<S, 2, 7>;
        else return k_pcg_cluster<S, V1, 7>;
    }
    return k_pcg_cluster<S, V1, 9>;
}

FusedKernel pick(int S, double row)
{
    switch (S) {
    case 1: return pick_s<1>(row);
    case 2: return pick_s<2>(row);
    case 4: return pick_s<4>(row);
    case 8: return pick_s<8>(row);
    case 16: return pick_s<16>(row);
    default: return pick_s<32>(row);
    }
}

// The layout of one launch: window rows W (the whole vector when it is shorter
// than kWindow), the staging capacity vcap in nonzeros (0: none) and the
// dynamic shared memory.  vcap allows the mean row length of the pattern over
// a tile plus four nonzeros per row; it is dropped when the total would pass
// kSmemBudget.
struct Plan {
    int W, vcap;
    size_t smem;
};
constexpr size_t kSmemBudget = 200 * 1024;

size_t fused_smem(int nblk, int S, int W, int vcap)
{
    size_t b = (size_t)(3 * nblk + 3 * kTile + 2 * W) * S * sizeof(double);
    if (vcap > 0) b += (size_t)(vcap + kTile) * S * sizeof(double) + (size_t)(vcap + kTile + 1) * sizeof(int);
    return (b + 15) & ~size_t(15);
}

Plan plan(int J, long long nnz, int S, int nblk)
{
    Plan pl;
    pl.W = J < kWindow ? J : kWindow;
    long long want = (nnz * kTile + J - 1) / J + 4 * kTile;
    if (want > nnz) want = nnz;
    pl.vcap = (int)want;
    pl.smem = fused_smem(nblk, S, pl.W, pl.vcap);
    if (pl.smem > kSmemBudget) {
        pl.vcap = 0;
        pl.smem = fused_smem(nblk, S, pl.W, 0);
    }
    return pl;
}

cudaLaunchConfig_t fused_config(int nblk, int E, const Plan &pl, cudaStream_t st, cudaLaunchAttribute *attr)
{
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3(nblk, E, 1);
    cfg.blockDim = dim3(kBlock, 1, 1);
    cfg.dynamicSmemBytes = pl.smem;
    cfg.stream = st;
    attr->id = cudaLaunchAttributeClusterDimension;
    attr->val.clusterDim.x = nblk;
    attr->val.clusterDim.y = 1;
    attr->val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

// Prepare the kernel for clusters of nblk CTAs with this layout and return how
// many such clusters the device holds at once (0: none fit); cached on the handle.
int clusters_resident(ens_ctx *h, FusedKernel k, int nblk, const Plan &pl)
{
    const void *key = (const void *)k;
    for (const auto &f : h->cluster_fit)
        if (f.kernel == key && f.C == nblk && f.smem == pl.smem) return f.resident;
    int n = 0;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess &&
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBudget) == cudaSuccess) {
        cudaLaunchAttribute attr;
        cudaLaunchConfig_t cfg = fused_config(nblk, 1, pl, nullptr, &attr);
        if (cudaOccupancyMaxActiveClusters(&n, k, &cfg) != cudaSuccess) n = 0;
    }
    cudaGetLastError();  // a refused query only means the graph loop runs instead
    h->cluster_fit.push_back({key, nblk, pl.smem, n});
    return n;
}

}  // namespace

// The one-launch schedule is taken where it was measured to win: every CTA owns
// one tile (J <= 16 x 64 rows), S <= 32 (the on-chip state of S = 64 does not
// fit), all E clusters are resident at once, and a CTA's FP64 work per trip,
// 64 S (nnz/J + 7) fused multiply-adds, is at most kMaxTripWork.  With four
// tiles per CTA (4096 unknowns, one tile after another) it was 1.0-2.5x slower
// than the graph loop; with more ensembles than resident clusters the clusters
// run in waves (E = 32 at 1024 unknowns, S = 8: 39 against 26 us per trip);
// and with much FP64 work per CTA the few SMs of a cluster are slower than the
// whole GPU (27-point rows on 343 unknowns at S = 16, 27600 multiply-adds: 36
// against 32 us; 9-point rows at S = 32, 32000: 33 against 31 us).  Below
// 26000 every measured case gained, 1.2-3.1x (the 7-point 10^3 problem at
// S = 32, 27400, gained 1.23x but is left to the loop).  With h->fused == 2
// (ENS_PCG_FUSED=2) the work bound is not applied.  Results are the same
// either way.
constexpr double kMaxTripWork = 26000.0;

int fused_cluster_size(ens_ctx *h, int J, long long nnz, int S, int E)
{
    if (!h || h->host_loop || !h->fused || J <= 0 || E <= 0 || !lane_count_ok(S) || S > 32) return 0;
    const Geo g = geometry(J, S, E);
    if (g.nblk > kMaxCluster || g.RT != kTile) return 0;
    if (h->fused != 2 && (double)kTile * S * ((double)nnz / J + 7.0) > kMaxTripWork) return 0;
    FusedKernel k = pick(S, (double)nnz / J);
    return clusters_resident(h, k, g.nblk, plan(J, nnz, S, g.nblk)) >= E ? g.nblk : 0;
}

int fused_solve(ens_ctx *h, const Args &a, int C, cudaStream_t st)
{
    if (C != a.g.nblk || a.g.RT != kTile || a.S > 32)
        return set_error(h, ENS_EINVAL, "fused_solve: not a one-launch problem");
    FusedKernel k = pick(a.S, (double)a.nnz / a.J);
    const Plan pl = plan(a.J, a.nnz, a.S, a.g.nblk);
    cudaLaunchAttribute attr;
    cudaLaunchConfig_t cfg = fused_config(a.g.nblk, a.E, pl, st, &attr);
    ENS_CUDA_CHECK(h, cudaLaunchKernelEx(&cfg, k, a, pl.W, pl.vcap));
    return ENS_OK;
}

}  // namespace pcgi
}  // namespace ens
