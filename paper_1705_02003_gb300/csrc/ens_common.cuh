// ens_common.cuh -- internal declarations shared by the libens translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "ens.h"

namespace ens {

struct GraphEntry {
    std::vector<uint64_t> key;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    uint64_t last_use = 0;
};

// The problem, S, E and precision a multigrid workspace was set up with (its
// layout depends on them).
struct MgTag {
    const void *work = nullptr;
    int kind = 0, n = 0, S = 0, E = 0, mixed = 0;
};

// How many clusters of C CTAs of a one-launch PCG kernel (smem bytes of
// dynamic shared memory each) the device holds at once.
struct ClusterFit {
    const void *kernel;
    int C;
    size_t smem;
    int resident;
};

}  // namespace ens

struct ens_ctx {
    int device = 0;
    std::string last_error;
    cudaStream_t capture = nullptr;          // private stream used only to capture graphs
    std::vector<ens::GraphEntry> graphs;     // small LRU cache of instantiated loops
    uint64_t clock = 0;
    int host_loop = 0;                       // ENS_PCG_HOST_LOOP=1: launch the PCG loop from the host
    int branches = 0;                        // ENS_PCG_BRANCHES=n: graph branches of a PCG loop (0: one per ensemble, at most 16)
    int check = 0;                           // ENS_CHECK=1: validate the caller's CSR graph before a solve
    int fused = 1;                           // ENS_PCG_FUSED: 0 never the one-launch schedule, 2 wherever it fits
    std::vector<ens::ClusterFit> cluster_fit;  // answers of the cluster-occupancy query, per kernel and layout
    int *check_flag = nullptr;               // device word for the graph check
    void *sort_scratch = nullptr;            // device-wide sort of more than 16384 keys (grown on demand)
    size_t sort_scratch_bytes = 0;
    std::vector<ens::MgTag> mg_tags;         // multigrid workspaces set up on this handle (the last 16)
};

namespace ens {

constexpr int kBlock = 256;  // threads per block of every vector/SpMV kernel

inline int set_error(ens_ctx *h, int code, const std::string &msg)
{
    if (h) h->last_error = msg;
    return code;
}

inline int cuda_error(ens_ctx *h, cudaError_t e, const char *where)
{
    std::string m = std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return set_error(h, ENS_ECUDA, m);
}

#define ENS_CUDA_CHECK(h, expr)                                             \
    do {                                                                    \
        cudaError_t e_ = (expr);                                            \
        if (e_ != cudaSuccess) return ens::cuda_error((h), e_, #expr);      \
    } while (0)

#define ENS_LAUNCH_CHECK(h, what)                                           \
    do {                                                                    \
        cudaError_t e_ = cudaGetLastError();                                \
        if (e_ != cudaSuccess) return ens::cuda_error((h), e_, what);       \
    } while (0)

inline bool lane_count_ok(int S)
{
    return S == 1 || S == 2 || S == 4 || S == 8 || S == 16 || S == 32 || S == 64;
}

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Rounding-explicit FP64 helpers: each product and sum is rounded on its own
// (no fused multiply-add), so a sum of products follows the same operation
// sequence as a plain left-to-right host loop.
__device__ __forceinline__ double dmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double dadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double dsub(double a, double b) { return __dsub_rn(a, b); }

// Neighbours of `row` in increasing column order; returns the count (<= 9).
// cols must hold 27 entries (the 3-D trilinear stencil).
__device__ __host__ inline int row_neighbours(int kind, int n, int row, int *cols)
{
    int c = 0;
    if (kind == ENS_FD5_LOGKL) {
        int i = row % n, j = row / n;
        if (j > 0) cols[c++] = row - n;
        if (i > 0) cols[c++] = row - 1;
        cols[c++] = row;
        if (i < n - 1) cols[c++] = row + 1;
        if (j < n - 1) cols[c++] = row + n;
    } else if (kind == ENS_Q1_ROT) {
        int i = row % n, j = row / n;
        for (int dj = -1; dj <= 1; dj++)
            for (int di = -1; di <= 1; di++) {
                int ii = i + di, jj = j + dj;
                if (ii >= 0 && ii < n && jj >= 0 && jj < n) cols[c++] = ii + n * jj;
            }
    } else if (kind == ENS_Q1_3D_KL || kind == ENS_Q1_3D_DISC) {
        int n2 = n * n;
        int i = row % n, j = (row / n) % n, l = row / n2;
        for (int dl = -1; dl <= 1; dl++)
            for (int dj = -1; dj <= 1; dj++)
                for (int di = -1; di <= 1; di++) {
                    int ii = i + di, jj = j + dj, ll = l + dl;
                    if (ii >= 0 && ii < n && jj >= 0 && jj < n && ll >= 0 && ll < n) cols[c++] = ii + n * jj + n2 * ll;
                }
    } else {
        int n2 = n * n;
        int i = row % n, j = (row / n) % n, l = row / n2;
        if (l > 0) cols[c++] = row - n2;
        if (j > 0) cols[c++] = row - n;
        if (i > 0) cols[c++] = row - 1;
        cols[c++] = row;
        if (i < n - 1) cols[c++] = row + 1;
        if (j < n - 1) cols[c++] = row + n;
        if (l < n - 1) cols[c++] = row + n2;
    }
    return c;
}

int check_pattern(ens_ctx *h, const char *who, int J, int64_t nnz, const int32_t *rowptr, const int32_t *colidx,
                  cudaStream_t st);
int problem_check(const ens_problem *p, int *J, int64_t *nnz, std::string *why);
// Assembly of the lanes listed in lanes[nlanes] (lane = e * S + s; all lanes when NULL).
int assemble_lanes(ens_ctx *h, const ens_problem *p, int S, int E, const double *xi, const int32_t *rowptr,
                   void *vals, int vals_f32, double *dinv, double *b, const int32_t *lanes, int nlanes,
                   cudaStream_t st);
// The problem's graph into caller memory (rowptr[J+1], colidx[nnz]).
int pattern_into(ens_ctx *h, const ens_problem *p, int32_t *rowptr, int32_t *colidx, cudaStream_t st);

}  // namespace ens
