// pcg_core.cuh -- the pieces of the ensemble Jacobi-PCG shared by its two
// schedules: the three-kernel loop of pcg.cu (any size; one CUDA graph) and the
// one-launch cluster solve of fused.cu (small problems).  Both use the same
// workspace layout, lane geometry and per-row arithmetic, so they give
// bit-identical results.
#pragma once

#include "ens_common.cuh"

namespace ens {
namespace pcgi {

enum { CTL_NLIVE = 0, CTL_TRIPS = 1, CTL_OUTER_LIVE = 2, CTL_WORDS = 16 };
// The PCG loop of a solve may run as several independent graph branches, each
// over a contiguous range of ensembles with its own trip counter (the words
// b * CTL_WORDS + CTL_TRIPS); CTL_NLIVE counts the live lanes of all of them.
constexpr int kMaxBranches = 16;
enum { CNT_INIT = 0, CNT_SPMV = 1, CNT_UPD = 2, CNT_RES = 3, CNT_KINDS = 4 };

struct Ws {
    void *r, *p, *q, *z;    // [E][J][S] of the loop's value type (z = D^-1 r)
    double *part0, *part1;  // [E][nblk][S]
    double *bnorm, *rz, *alpha, *beta, *rr;  // [E][S]
    int *k, *live;          // [E][S]
    int *ens_live;          // [E]
    int *counter;           // [E][CNT_KINDS]
    int *ctl;               // [kMaxBranches][CTL_WORDS]
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
    const void *vals, *dinv;  // value type of the loop
    const double *b;          // right-hand side (FP64 in both forms)
    void *x;                  // value type of the loop
    const uint8_t *active;
    int32_t *iters, *status;
    double *relres;
    Ws w;
    double *pq_out;  // ens_spmv: write p^T q per lane here instead of alpha
    int in_graph;    // K4 drives the graph's while loop (else the host loops)
    int trip_cap;    // trips per launch of the loop (maxit, or the chunk of a streamed solve)
    int branch;      // graph branch running these ensembles (its trip counter)
    const uint8_t *refill;  // K0: restart only these lanes, keep the others (NULL: all lanes)
    cudaGraphConditionalHandle cond;
};

// Rows per block: at least 256 (so the per-block reduction tail is amortised
// over enough rows) and enough to give about four blocks per SM for one
// ensemble; a multiple of 256, so every kernel's row pass divides it (with the
// 64-row tiles below, the threads of a 256-row pass beyond the tile stay idle
// at S = 1 and 2).  Tiny
// problems (J <= 4096, a handful of blocks per ensemble whatever the tile) take
// 64-row tiles instead: a thread then walks 4 rows, not 16, per kernel, which
// shortens the latency chain of an iteration (32^2 workload: 1.29x; on 31^3,
// where 64-row tiles make 466 blocks per ensemble, they were 10 % slower).
//
// Small ensembles (S = 2, 4, 8; J > 4096) take tiles of 256 x 16 / S rows, so
// that a K2 thread walks 16 rows per tile as it does at S = 16 (with 256-row
// tiles an S = 4 thread had 4 rows: little independent work to hide the FP64
// latency chain).  Measured on the Q1 256^2 loop with surrogate grouping:
// S = 4 230 -> 299 sample-solves/s, S = 8 279 -> 294; on Section 4's Test 1
// S = 4 +10 %, S = 8 unchanged.  A single small ensemble then runs on fewer
// blocks (64 at S = 4 on 65536 unknowns).
//
// For S >= 2 the geometry depends on J and S only, so a lane's reduction order
// is the same for any E and any lane position.  One-lane ensembles (S = 1) are
// the exception: with 256-row tiles a thread owns one row of a 256-row tile, which
// leaves it no independent rows to hide the FP64 latency chain and pays a
// block reduction per 256 row-lanes.  When the call's one-lane ensembles fill
// the GPU (E J >= kOneLaneBatch row-lanes, three 4096-row blocks per SM) their
// tiles are kOneLaneTile rows, 16 rows per thread as at S = 16: measured on
// Q1 256^2 with 48-159 one-lane ensembles, 324 against 138 sample-solves/s.  A
// single one-lane ensemble keeps the small tiles (it would run on 16 blocks:
// 18 against 33 sample-solves/s).  So at S = 1 a sample's rounding depends on
// whether its call holds a full batch.
constexpr int kOneLaneTile = 4096;
constexpr long long kOneLaneBatch = 152LL * 3 * kOneLaneTile;

inline Geo geometry(int J, int S, int E)
{
    const long long target = 152LL * 4;
    long long RT = ((long long)J + target - 1) / target;
    const long long tile = J <= 4096 ? 64 : 256;
    if (RT < tile) RT = tile;
    RT = (RT + tile - 1) / tile * tile;
    if (S >= 2 && S <= 8 && J > 4096 && RT < 4096LL / S) RT = 4096LL / S;
    if (S == 1 && J > 4096 && (long long)E * J >= kOneLaneBatch && RT < kOneLaneTile) RT = kOneLaneTile;
    Geo g;
    g.RT = (int)RT;
    g.nblk = (int)((J + RT - 1) / RT);
    return g;
}

struct Bump {
    size_t off = 0;
    char *base;
    explicit Bump(char *b) : base(b) {}
    void *take(size_t bytes)
    {
        size_t o = off;
        off = align256(off + bytes);
        return base ? (void *)(base + o) : nullptr;
    }
};

inline void lay_loop(Bump &m, int J, int S, int E, const Geo &g, size_t tsize, Ws *w)
{
    size_t vec = (size_t)E * J * S * tsize;
    size_t part = (size_t)E * g.nblk * S * sizeof(double);
    size_t lane = (size_t)E * S;
    w->r = m.take(vec);
    w->p = m.take(vec);
    w->q = m.take(vec);
    w->z = m.take(vec);
    w->part0 = (double *)m.take(part);
    w->part1 = (double *)m.take(part);
    w->bnorm = (double *)m.take(lane * 8);
    w->rz = (double *)m.take(lane * 8);
    w->alpha = (double *)m.take(lane * 8);
    w->beta = (double *)m.take(lane * 8);
    w->rr = (double *)m.take(lane * 8);
    w->k = (int *)m.take(lane * 4);
    w->live = (int *)m.take(lane * 4);
    w->ens_live = (int *)m.take((size_t)E * 4);
    w->counter = (int *)m.take((size_t)E * CNT_KINDS * 4);
    w->ctl = (int *)m.take(kMaxBranches * CTL_WORDS * 4);
}

inline size_t layout(int J, int S, int E, const Geo &g, Ws *w, char *base)
{
    Bump m(base);
    Ws t;
    lay_loop(m, J, S, E, g, sizeof(double), &t);
    if (w) *w = t;
    return m.off;
}

// ---- lane vectors: V consecutive lanes per thread as one access --------------
template <typename T, int V> struct VT;
template <> struct VT<double, 1> {
    using R = double;
    __device__ __forceinline__ static void get(double *v, R t) { v[0] = t; }
    __device__ __forceinline__ static R put(const double *v) { return v[0]; }
};
template <> struct VT<double, 2> {
    using R = double2;
    __device__ __forceinline__ static void get(double *v, R t) { v[0] = t.x; v[1] = t.y; }
    __device__ __forceinline__ static R put(const double *v) { return make_double2(v[0], v[1]); }
};
template <> struct VT<float, 1> {
    using R = float;
    __device__ __forceinline__ static void get(float *v, R t) { v[0] = t; }
    __device__ __forceinline__ static R put(const float *v) { return v[0]; }
};
template <> struct VT<float, 2> {
    using R = float2;
    __device__ __forceinline__ static void get(float *v, R t) { v[0] = t.x; v[1] = t.y; }
    __device__ __forceinline__ static R put(const float *v) { return make_float2(v[0], v[1]); }
};
template <> struct VT<float, 4> {
    using R = float4;
    __device__ __forceinline__ static void get(float *v, R t) { v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w; }
    __device__ __forceinline__ static R put(const float *v) { return make_float4(v[0], v[1], v[2], v[3]); }
};

template <typename T, int V> struct Vec {
    using W = VT<T, V>;
    using R = typename W::R;
    T v[V];
    __device__ __forceinline__ void load(const T *p) { W::get(v, *reinterpret_cast<const R *>(p)); }
    __device__ __forceinline__ void load_ro(const T *p) { W::get(v, __ldg(reinterpret_cast<const R *>(p))); }
    __device__ __forceinline__ void load_stream(const T *p) { W::get(v, __ldcs(reinterpret_cast<const R *>(p))); }
    // through L2 only: for data that other blocks of a cluster wrote earlier in the same launch
    __device__ __forceinline__ void load_cg(const T *p) { W::get(v, __ldcg(reinterpret_cast<const R *>(p))); }
    __device__ __forceinline__ void store(T *p) const { *reinterpret_cast<R *>(p) = W::put(v); }
};

// V lanes per thread.  The vector kernels (K0, K3, K4) move 16 bytes per
// access (two FP64 or four FP32 lanes); the SpMV (K2) by default takes one
// lane per thread, which halves its registers and doubles its resident warps
// -- in FP64 it is bound by the FP64 issue rate, and more independent
// multiply-add chains per SM keep that pipe busier (S = 64 keeps two lanes
// per thread so a row stays within one warp; see k_spmv for the 5-point
// variant).
template <int S, int V_> struct LaneGeo {
    static constexpr int V = V_;
    static constexpr int TPR = S / V;          // threads per row
    static constexpr int RPP = kBlock / TPR;   // rows per block pass
    static constexpr int G = kBlock / S;       // groups in the final cross-block sum
};
template <typename T, int S>
using VecGeo = LaneGeo<S, (S >= (int)(16 / sizeof(T)) ? (int)(16 / sizeof(T)) : S)>;
template <int S> using SpmvGeo = LaneGeo<S, (S >= 64 ? 2 : 1)>;

__device__ __forceinline__ double wide(double v) { return v; }
__device__ __forceinline__ double wide(float v) { return (double)v; }

// K2 variants: V_ lanes per thread, KC nonzeros of a row loaded at once (longer
// rows continue chunk by chunk; launch_k2 sizes KC to the stencil).  One lane
// per thread suits the 9-point rows, where the FP64 pipe is the limit and more
// warps keep it fed; for shorter FP64 rows two lanes per thread put twice the
// bytes of a row in flight for the same column indices (measured per launch:
// 5-point rows at S = 16/32 0.70 -> 0.45 ms; 7-point rows at S = 32 0.64 ->
// 0.61 ms with four ensembles and 1.36 -> 1.20 ms with one; at S = 16 and in
// FP32 one lane per thread stayed faster).  The variant is a function of the
// pattern, T and S only, so the results still do not depend on E, on lane
// position or on the other lanes.
template <int S, int V_, int KC> struct SpmvOcc {
    static constexpr int value = S == 1 ? 3 : (S >= 64 ? 2 : (V_ == 1 ? 4 : (KC <= 5 ? 3 : 2)));
};

// One row of K2 for the thread's V lanes: q_r = sum_k a_k p_{c_k} in column
// order, then p_r q_r added to the lane's partial of p^T q.
template <typename T, int S, int V, int KC>
__device__ __forceinline__ void spmv_row(int r, const int32_t *__restrict__ rowptr,
                                         const int32_t *__restrict__ colidx, const T *__restrict__ vals,
                                         const T *__restrict__ p, T *__restrict__ q, double (&acc)[1][V])
{
    constexpr int kChunk = KC;
    const int k0 = __ldg(rowptr + r), k1 = __ldg(rowptr + r + 1);
    T s[V];
#pragma unroll
    for (int v = 0; v < V; v++) s[v] = T(0);
    for (int kb = k0; kb < k1; kb += kChunk) {
        int c[kChunk];
        Vec<T, V> av[kChunk], xv[kChunk];
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
    Vec<T, V> qv, pr;
#pragma unroll
    for (int v = 0; v < V; v++) qv.v[v] = s[v];
    qv.store(q + (size_t)r * S);
    pr.load_ro(p + (size_t)r * S);
#pragma unroll
    for (int v = 0; v < V; v++) acc[0][v] = fma(wide(pr.v[v]), wide(s[v]), acc[0][v]);
}

// The one-launch cluster solve of fused.cu (FP64, no refill, no p^T q output).
// fused_cluster_size returns the CTAs per ensemble it would use for this
// problem, or 0 where the three-kernel loop runs instead; fused_solve launches it.
int fused_cluster_size(ens_ctx *h, int J, long long nnz, int S, int E);
int fused_solve(ens_ctx *h, const Args &a, int C, cudaStream_t st);

}  // namespace pcgi
}  // namespace ens
