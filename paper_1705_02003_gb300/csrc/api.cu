// api.cu -- handle management and the host-side sparse-grid bookkeeping.
//
// ens_sg_refine implements classic refinement (Section 2.2, "Adaptivity"):
// each point whose surplus magnitude is at least tau contributes its children,
// one dimension at a time -- a level-0 coordinate (y = -1 or +1) has the single
// child y = 0 at level 1, a level-l coordinate (l >= 1) the two children
// (l+1, 2i-1) and (l+1, 2i+1) -- skipping children already in the grid or
// already listed.  ens_sg_initial builds the full sparse grid of levels
// 0..level (Section 2.2, Z_l with alpha(l) = |l|) by refining every point of
// the newest level, starting from the 2^N corners of level 0.
#include "ens_common.cuh"

#include <cmath>
#include <cstdlib>
#include <cstring>
#include <unordered_set>

extern "C" int ens_create(ens_handle *out, int device)
{
    if (!out) return ENS_EINVAL;
    *out = nullptr;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess) return ENS_ECUDA;
    if (device < 0 || device >= ndev) return ENS_EINVAL;
    if (cudaSetDevice(device) != cudaSuccess) return ENS_ECUDA;
    ens_ctx *h = new ens_ctx();
    h->device = device;
    const char *hl = getenv("ENS_PCG_HOST_LOOP");
    h->host_loop = (hl && hl[0] == '1') ? 1 : 0;
    const char *nb = getenv("ENS_PCG_BRANCHES");
    h->branches = nb ? atoi(nb) : 0;
    if (h->branches < 0) h->branches = 0;
    const char *ck = getenv("ENS_CHECK");
    h->check = (ck && ck[0] == '1') ? 1 : 0;
    const char *fu = getenv("ENS_PCG_FUSED");
    h->fused = !fu ? 1 : fu[0] == '0' ? 0 : fu[0] == '2' ? 2 : 1;
    if (cudaStreamCreateWithFlags(&h->capture, cudaStreamNonBlocking) != cudaSuccess) {
        delete h;
        return ENS_ECUDA;
    }
    if (cudaMalloc(&h->check_flag, sizeof(int)) != cudaSuccess) {
        cudaStreamDestroy(h->capture);
        delete h;
        return ENS_ECUDA;
    }
    *out = h;
    return ENS_OK;
}

extern "C" int ens_destroy(ens_handle h)
{
    if (!h) return ENS_EINVAL;
    for (auto &g : h->graphs) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        if (g.graph) cudaGraphDestroy(g.graph);
    }
    if (h->capture) cudaStreamDestroy(h->capture);
    if (h->check_flag) cudaFree(h->check_flag);
    if (h->sort_scratch) cudaFree(h->sort_scratch);
    delete h;
    return ENS_OK;
}

extern "C" const char *ens_last_error(ens_handle h)
{
    if (!h) return "null handle";
    return h->last_error.c_str();
}

namespace {

// A grid point as a byte string of (level, index) pairs, for hashing.
std::string point_key(int N, const int8_t *l, const int32_t *i)
{
    std::string k((size_t)N * 5, '\0');
    for (int n = 0; n < N; n++) {
        k[n * 5] = (char)l[n];
        memcpy(&k[n * 5 + 1], &i[n], 4);
    }
    return k;
}

}  // namespace

extern "C" int ens_sg_refine(int N, int M, const int8_t *lvl, const int32_t *idx, int first,
                             const double *surplus, double tau, int max_level, int max_out,
                             int8_t *out_lvl, int32_t *out_idx)
{
    if (N < 1 || N > 64 || M < 0 || first < 0 || first > M || max_out < 0) return ENS_EINVAL;
    if (M > 0 && (!lvl || !idx || !surplus)) return ENS_EINVAL;
    std::unordered_set<std::string> seen;
    seen.reserve((size_t)M * 2 + 16);
    for (int m = 0; m < M; m++) seen.insert(point_key(N, lvl + (size_t)m * N, idx + (size_t)m * N));
    std::vector<int8_t> cl(N);
    std::vector<int32_t> ci(N);
    int cnt = 0;
    for (int m = first; m < M; m++) {
        if (!(std::fabs(surplus[m]) >= tau)) continue;
        const int8_t *pl = lvl + (size_t)m * N;
        const int32_t *pi = idx + (size_t)m * N;
        int lsum = 0;
        for (int n = 0; n < N; n++) lsum += pl[n];
        if (lsum + 1 > max_level) continue;
        for (int n = 0; n < N; n++) {
            const int nch = pl[n] == 0 ? 1 : 2;
            for (int c = 0; c < nch; c++) {
                for (int a = 0; a < N; a++) {
                    cl[a] = pl[a];
                    ci[a] = pi[a];
                }
                if (pl[n] == 0) {
                    cl[n] = 1;
                    ci[n] = 1;
                } else {
                    if (pl[n] >= 30) return ENS_EINVAL;  // index would overflow int32
                    cl[n] = (int8_t)(pl[n] + 1);
                    ci[n] = 2 * pi[n] + (c == 0 ? -1 : 1);
                }
                std::string key = point_key(N, cl.data(), ci.data());
                if (!seen.insert(key).second) continue;
                if (cnt >= max_out) return ENS_ENOMEM;
                memcpy(out_lvl + (size_t)cnt * N, cl.data(), N);
                memcpy(out_idx + (size_t)cnt * N, ci.data(), (size_t)N * 4);
                cnt++;
            }
        }
    }
    return cnt;
}

extern "C" int ens_sg_initial(int N, int level, int max_out, int8_t *lvl, int32_t *idx)
{
    if (N < 1 || N > 30 || level < 0 || !lvl || !idx) return ENS_EINVAL;
    int M = 1 << N;
    if (M > max_out) return ENS_ENOMEM;
    for (int c = 0; c < M; c++)
        for (int n = 0; n < N; n++) {
            lvl[(size_t)c * N + n] = 0;
            idx[(size_t)c * N + n] = (c >> n) & 1;
        }
    std::vector<double> ones(max_out, 1.0);
    int first = 0;
    for (int L = 1; L <= level; L++) {
        int add = ens_sg_refine(N, M, lvl, idx, first, ones.data(), 0.0, L, max_out - M,
                                lvl + (size_t)M * N, idx + (size_t)M * N);
        if (add < 0) return add;
        first = M;
        M += add;
    }
    return M;
}

extern "C" int ens_sg_points(int N, int M, const int8_t *lvl, const int32_t *idx, double *y)
{
    if (N < 1 || M < 0) return ENS_EINVAL;
    if (M > 0 && (!lvl || !idx || !y)) return ENS_EINVAL;
    for (size_t k = 0; k < (size_t)M * N; k++) {
        const int l = lvl[k];
        if (l < 0 || l > 62) return ENS_EINVAL;
        // y = i 2^(1-l) - 1: the product is a power-of-two scaling and the
        // difference of two dyadic numbers of at most 63 bits, so both are exact
        y[k] = std::ldexp((double)idx[k], 1 - l) - 1.0;
    }
    return ENS_OK;
}
