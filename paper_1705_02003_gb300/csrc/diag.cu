// diag.cu -- a measurement aid: the FP64 fused multiply-add rate of this GPU.
//
// The ensemble SpMV and the PCG vector kernels issue about one FP64 fused
// multiply-add per 8 to 11 bytes they move, and GB300 retires far fewer FP64
// operations per clock than it moves bytes, so the roofline of these kernels
// is the FP64 issue rate rather than HBM.  k_dfma_peak measures that rate:
// every thread runs kChains independent multiply-add recurrences, enough to
// cover the FP64 latency with the resident warps, and nothing else.
#include "ens_common.cuh"

namespace ens {
namespace {

constexpr int kChains = 8;

__global__ void __launch_bounds__(kBlock) k_dfma_peak(int iters, double seed, double *sink)
{
    double a[kChains];
#pragma unroll
    for (int u = 0; u < kChains; u++) a[u] = seed + 1e-3 * threadIdx.x + u;
    const double m = 0.9999999999, c = 1e-12;
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int u = 0; u < kChains; u++) a[u] = fma(a[u], m, c);
    }
    double s = 0.0;
#pragma unroll
    for (int u = 0; u < kChains; u++) s += a[u];
    // never true for the seeds used, but the compiler cannot know that, so
    // every chain is computed
    if (s == -1.0) sink[blockIdx.x] = s;
}

}  // namespace
}  // namespace ens

extern "C" int ens_fp64_peak(ens_handle h, int blocks, int iters, double *sink, void *stream)
{
    if (blocks <= 0 || iters <= 0 || !sink) return ens::set_error(h, ENS_EINVAL, "ens_fp64_peak: bad arguments");
    ens::k_dfma_peak<<<blocks, ens::kBlock, 0, (cudaStream_t)stream>>>(iters, 1.0, sink);
    ENS_LAUNCH_CHECK(h, "k_dfma_peak");
    return ENS_OK;
}

extern "C" double ens_fp64_peak_flops(int blocks, int iters)
{
    return 2.0 * ens::kChains * (double)iters * (double)blocks * ens::kBlock;
}
