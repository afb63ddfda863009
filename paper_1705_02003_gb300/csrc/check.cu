// check.cu -- validation of a caller's CSR graph before any kernel reads
// through it (no counterpart in the paper: a guard of this library).  Every
// kernel of the solve indexes vals, p and q through rowptr and colidx; a graph
// with an entry out of range would make them read outside the caller's arrays.
// With ENS_CHECK=1 at ens_create the solve entry points run this check first
// and return ENS_EINVAL instead of launching; ens_check_pattern runs it alone.
#include "ens_common.cuh"

#include <algorithm>

namespace ens {
namespace {

enum {
    BAD_ENDS = 1,       // rowptr[0] != 0 or rowptr[J] != nnz
    BAD_ORDER = 2,      // rowptr decreases somewhere
    BAD_ROWPTR = 4,     // a rowptr entry outside [0, nnz]
    BAD_COLIDX = 8,     // a column index outside [0, J)
};

// Reads rowptr[0..J] and colidx[0..nnz) only, whatever their contents.
__global__ void k_check_pattern(int J, long long nnz, const int32_t *__restrict__ rowptr,
                                const int32_t *__restrict__ colidx, int *flags)
{
    int bad = 0;
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long stride = (long long)gridDim.x * blockDim.x;
    if (tid == 0 && (rowptr[0] != 0 || rowptr[J] != nnz)) bad |= BAD_ENDS;
    for (long long r = tid; r < J; r += stride) {
        const int a = rowptr[r], b = rowptr[r + 1];
        if (a > b) bad |= BAD_ORDER;
        if (a < 0 || (long long)a > nnz || b < 0 || (long long)b > nnz) bad |= BAD_ROWPTR;
    }
    for (long long k = tid; k < nnz; k += stride) {
        const int c = colidx[k];
        if (c < 0 || c >= J) bad |= BAD_COLIDX;
    }
    if (bad) atomicOr(flags, bad);
}

}  // namespace

int check_pattern(ens_ctx *h, const char *who, int J, int64_t nnz, const int32_t *rowptr, const int32_t *colidx,
                  cudaStream_t st)
{
    if (J <= 0 || nnz <= 0 || nnz >= (1LL << 31) || !rowptr || !colidx)
        return set_error(h, ENS_EINVAL, std::string(who) + ": bad graph sizes or null pointer");
    if (!h->check_flag) return set_error(h, ENS_ECUDA, std::string(who) + ": no check buffer on this handle");
    ENS_CUDA_CHECK(h, cudaMemsetAsync(h->check_flag, 0, sizeof(int), st));
    const long long work = nnz > J ? nnz : J;
    const int grid = (int)std::min<long long>((work + 255) / 256, 152LL * 8);
    k_check_pattern<<<grid, 256, 0, st>>>(J, nnz, rowptr, colidx, h->check_flag);
    ENS_LAUNCH_CHECK(h, "graph check kernel");
    int flags = 0;
    ENS_CUDA_CHECK(h, cudaMemcpyAsync(&flags, h->check_flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    ENS_CUDA_CHECK(h, cudaStreamSynchronize(st));
    if (!flags) return ENS_OK;
    std::string m = std::string(who) + ": invalid CSR graph:";
    if (flags & BAD_ENDS) m += " rowptr[0] != 0 or rowptr[J] != nnz;";
    if (flags & BAD_ORDER) m += " rowptr decreases;";
    if (flags & BAD_ROWPTR) m += " rowptr entry outside [0, nnz];";
    if (flags & BAD_COLIDX) m += " column index outside [0, J);";
    return set_error(h, ENS_EINVAL, m);
}

}  // namespace ens

extern "C" int ens_check_pattern(ens_handle h, int J, int64_t nnz, const int32_t *rowptr, const int32_t *colidx,
                                 void *stream)
{
    if (!h) return ENS_EINVAL;
    return ens::check_pattern(h, "ens_check_pattern", J, nnz, rowptr, colidx, (cudaStream_t)stream);
}
