// group.cu -- surrogate-based grouping: the iteration surrogate (K6) and the
// stable sort-and-chunk (K7).
//
// Section 2.2: hat basis psi_{l,i}(y) = max(0, 1 - |(y + 1 - i h_l) / h_l|),
// h_l = 2^(1-l); N-D basis = product over dimensions.  Section 3.1, Eq.
// (SGSiterations): the iteration surrogate is sum_m c_m psi_m(y) over the grid
// points of the earlier levels; the new points are ordered by increasing
// prediction and cut into ensembles of S.
//
// K6 keeps the sum in generation order m = 0, 1, ... with every product and
// sum rounded separately, and evaluates (y + 1) * 2^(l-1) - i, which equals
// (y + 1 - i h_l) / h_l bit for bit because h_l is a power of two; so the
// prediction is the same double a plain host loop gives.  Terms whose basis
// value is zero are skipped (adding +-0 leaves a sum unchanged).
//
// K7 is a bitonic sort over (key, index) pairs: the index breaks ties, which
// makes the order total and therefore equal to a stable sort.  Up to 16384
// keys it runs in one CTA in shared memory; beyond that the same network runs
// over the whole GPU, one launch per compare-exchange stage, on scratch the
// handle owns (the order of a total order is unique, so both give the same
// permutation).
#include "ens_common.cuh"

#include <algorithm>

namespace ens {
namespace {

constexpr int kMaxSort = 16384;           // one CTA
constexpr int kMaxSortGlobal = 1 << 26;   // device-wide network

__global__ void k_sg_eval(int N, int M, const int8_t *__restrict__ lvl, const int32_t *__restrict__ idx,
                          const double *__restrict__ surplus, int Mq, const double *__restrict__ yq,
                          const double *__restrict__ values, double *__restrict__ pred)
{
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= Mq) return;
    double y[16];
    for (int n = 0; n < N; n++) y[n] = dadd(yq[(size_t)q * N + n], 1.0);  // y + 1
    double acc = 0.0;
    for (int m = 0; m < M; m++) {
        double prod = 1.0;
        for (int n = 0; n < N; n++) {
            int l = lvl[(size_t)m * N + n];
            double t = dsub(dmul(y[n], ldexp(1.0, l - 1)), (double)idx[(size_t)m * N + n]);
            double psi = dsub(1.0, fabs(t));
            if (!(psi > 0.0)) { prod = 0.0; break; }
            prod = dmul(prod, psi);
        }
        if (prod != 0.0) acc = dadd(acc, dmul(surplus[m], prod));
    }
    pred[q] = values ? dsub(values[q], acc) : acc;
}

__device__ __forceinline__ bool before(double ka, int ia, double kb, int ib)
{
    // total order: numbers ascending, NaN after every number, index breaks ties
    bool na = isnan(ka), nb = isnan(kb);
    if (na != nb) return nb;
    if (!na && ka != kb) return ka < kb;
    return ia < ib;
}

__global__ void k_sort(int Mq, const double *__restrict__ keys, int32_t *__restrict__ perm, int P)
{
    extern __shared__ unsigned char smem[];
    double *k = reinterpret_cast<double *>(smem);
    int *ix = reinterpret_cast<int *>(k + P);
    for (int t = threadIdx.x; t < P; t += blockDim.x) {
        if (t < Mq) {
            k[t] = keys ? keys[t] : 0.0;
            ix[t] = t;
        } else {
            k[t] = __longlong_as_double(0x7ff8000000000000LL);  // pads sort last
            ix[t] = t;
        }
    }
    __syncthreads();
    for (int size = 2; size <= P; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = threadIdx.x; t < P; t += blockDim.x) {
                int o = t ^ stride;
                if (o > t) {
                    bool up = (t & size) == 0;
                    bool swap = up ? before(k[o], ix[o], k[t], ix[t]) : before(k[t], ix[t], k[o], ix[o]);
                    if (swap) {
                        double tk = k[t];
                        k[t] = k[o];
                        k[o] = tk;
                        int ti = ix[t];
                        ix[t] = ix[o];
                        ix[o] = ti;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int t = threadIdx.x; t < Mq; t += blockDim.x) perm[t] = ix[t];
}

// Device-wide form: pairs in handle scratch, padded to a power of two with
// NaN keys whose indices follow every real one (so they sort last).
__global__ void k_sort_init(int Mq, int P, const double *__restrict__ keys, double *k, int *ix)
{
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < P; t += (long long)gridDim.x * blockDim.x) {
        k[t] = t < Mq ? (keys ? keys[t] : 0.0) : __longlong_as_double(0x7ff8000000000000LL);
        ix[t] = (int)t;
    }
}

__global__ void k_sort_stage(int P, int size, int stride, double *k, int *ix)
{
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < P; t += (long long)gridDim.x * blockDim.x) {
        const long long o = t ^ stride;
        if (o <= t) continue;
        const bool up = (t & size) == 0;
        const double kt = k[t], ko = k[o];
        const int it = ix[t], io = ix[o];
        if (up ? before(ko, io, kt, it) : before(kt, it, ko, io)) {
            k[t] = ko;
            k[o] = kt;
            ix[t] = io;
            ix[o] = it;
        }
    }
}

__global__ void k_sort_out(int Mq, const int *__restrict__ ix, int32_t *__restrict__ perm)
{
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < Mq; t += (long long)gridDim.x * blockDim.x)
        perm[t] = ix[t];
}

int sort_global(ens_ctx *h, int Mq, const double *keys, int32_t *perm, cudaStream_t st)
{
    int P = 1;
    while (P < Mq) P <<= 1;
    const size_t need = (size_t)P * (sizeof(double) + sizeof(int));
    if (h->sort_scratch_bytes < need) {
        // grow the handle's scratch; the old buffer may still be read by queued work
        ENS_CUDA_CHECK(h, cudaStreamSynchronize(st));
        if (h->sort_scratch) cudaFree(h->sort_scratch);
        h->sort_scratch = nullptr;
        h->sort_scratch_bytes = 0;
        ENS_CUDA_CHECK(h, cudaMalloc(&h->sort_scratch, need));
        h->sort_scratch_bytes = need;
    }
    double *k = (double *)h->sort_scratch;
    int *ix = (int *)(k + P);
    const int grid = (int)std::min<long long>(((long long)P + 255) / 256, 152LL * 16);
    k_sort_init<<<grid, 256, 0, st>>>(Mq, P, keys, k, ix);
    for (int size = 2; size <= P; size <<= 1)
        for (int stride = size >> 1; stride > 0; stride >>= 1) k_sort_stage<<<grid, 256, 0, st>>>(P, size, stride, k, ix);
    k_sort_out<<<grid, 256, 0, st>>>(Mq, ix, perm);
    ENS_LAUNCH_CHECK(h, "device-wide sort");
    return ENS_OK;
}

int sort_launch(ens_ctx *h, int Mq, const double *keys, int32_t *perm, cudaStream_t st)
{
    if (Mq > kMaxSort) return sort_global(h, Mq, keys, perm, st);
    int P = 1;
    while (P < Mq) P <<= 1;
    if (P < 2) P = 2;
    size_t bytes = (size_t)P * (sizeof(double) + sizeof(int));
    if (bytes > 48 * 1024)
        ENS_CUDA_CHECK(h, cudaFuncSetAttribute(k_sort, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    k_sort<<<1, 1024, bytes, st>>>(Mq, keys, perm, P);
    ENS_LAUNCH_CHECK(h, "k_sort");
    return ENS_OK;
}

}  // namespace
}  // namespace ens

using namespace ens;

extern "C" int ens_sort_chunk(ens_handle h, int Mq, const double *keys, int S, int32_t *perm, int *n_ens,
                              void *stream)
{
    if (!h) return ENS_EINVAL;
    if (S < 1) return set_error(h, ENS_EINVAL, "ens_sort_chunk: S < 1");
    if (Mq < 0 || Mq > kMaxSortGlobal) return set_error(h, ENS_EINVAL, "ens_sort_chunk: Mq out of range (0..2^26)");
    if (n_ens) *n_ens = (Mq + S - 1) / S;
    if (Mq == 0) return ENS_OK;
    if (!perm) return set_error(h, ENS_EINVAL, "ens_sort_chunk: null perm");
    return sort_launch(h, Mq, keys, perm, (cudaStream_t)stream);
}

extern "C" int ens_group(ens_handle h, int N, int M, const int8_t *lvl, const int32_t *idx,
                         const double *surplus, int Mq, const double *yq, int S, double *pred, int32_t *perm,
                         int *n_ens, void *stream)
{
    if (!h) return ENS_EINVAL;
    if (N < 1 || N > 16) return set_error(h, ENS_EINVAL, "ens_group: N must be in 1..16");
    if (M < 0 || Mq < 0 || Mq > kMaxSortGlobal) return set_error(h, ENS_EINVAL, "ens_group: bad M / Mq (Mq <= 2^26)");
    if (S < 1) return set_error(h, ENS_EINVAL, "ens_group: S < 1");
    if (n_ens) *n_ens = (Mq + S - 1) / S;
    if (Mq == 0) return ENS_OK;
    if (!pred || !perm || !yq || (M > 0 && (!lvl || !idx || !surplus)))
        return set_error(h, ENS_EINVAL, "ens_group: null pointer");
    cudaStream_t st = (cudaStream_t)stream;
    k_sg_eval<<<(Mq + 127) / 128, 128, 0, st>>>(N, M, lvl, idx, surplus, Mq, yq, nullptr, pred);
    ENS_LAUNCH_CHECK(h, "k_sg_eval");
    return sort_launch(h, Mq, pred, perm, st);
}

extern "C" int ens_sg_eval(ens_handle h, int N, int M, const int8_t *lvl, const int32_t *idx,
                           const double *surplus, int Mq, const double *yq, const double *values, double *out,
                           void *stream)
{
    if (!h) return ENS_EINVAL;
    if (N < 1 || N > 16) return set_error(h, ENS_EINVAL, "ens_sg_eval: N must be in 1..16");
    if (M < 0 || Mq < 0) return set_error(h, ENS_EINVAL, "ens_sg_eval: bad M / Mq");
    if (Mq == 0) return ENS_OK;
    if (!out || !yq || (M > 0 && (!lvl || !idx || !surplus)))
        return set_error(h, ENS_EINVAL, "ens_sg_eval: null pointer");
    cudaStream_t st = (cudaStream_t)stream;
    k_sg_eval<<<(Mq + 127) / 128, 128, 0, st>>>(N, M, lvl, idx, surplus, Mq, yq, values, out);
    ENS_LAUNCH_CHECK(h, "k_sg_eval");
    return ENS_OK;
}
