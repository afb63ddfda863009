/*
 * sgrid.c -- oracle: hierarchical piecewise-linear sparse grids, the
 * iteration surrogate and the sort-and-chunk grouping.
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Section 2.2 (hierarchical basis):
 *   h_l = 2^(1-l), y_{l,i} = i h_l - 1;
 *   psi_{l,i}(y) = psi((y + 1 - i h_l) / h_l),  psi(t) = max(0, 1 - |t|);
 *   level 0 holds i in {0, 1} (y = -1, +1); level l >= 1 holds odd i < 2^l.
 * N-D basis: psi_{l,i}(y) = prod_n psi_{l_n,i_n}(y_n); the point's level is |l|.
 * Surrogates, Eqs. (SGSoutput)/(SGSiterations): sum over grid points of
 *   c_m psi_m(y), summed in generation order m = 0, 1, ...
 * Surpluses (Eq. hierSGint): c = v(y) - (interpolant of the coarser points)(y);
 *   because psi_{l,i}(y_{l',i'}) = 0 whenever l' <= l (the triangularity noted
 *   beside the hierarchisation system), the interpolant over ALL points already
 *   in the grid gives the same value at a new point of the next level.
 * Classic refinement (Adaptivity paragraph): a point with |c| >= tau gets its
 *   children, one dimension at a time: (0, i) -> (1, 1); (l, i) -> (l+1, 2i-1),
 *   (l+1, 2i+1) for l >= 1.  A child already present is not added again.
 * Grouping (SGS-based grouping paragraph): order the new points by increasing
 *   predicted iterations and cut the list into ensembles of S consecutive
 *   points.  Equal predictions keep generation order (stable sort).
 * Work increase, Eqs. (Rl)/(R): R = S * sum_k max_{i in k} I_i / sum_i I_i over
 *   the real samples; lanes that pad the last ensemble count only through S.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>

double or_sg_coord(int l, int64_t i)
{
    double h = ldexp(1.0, 1 - l);
    return (double)i * h - 1.0;
}

double or_hat(int l, int64_t i, double y)
{
    double h = ldexp(1.0, 1 - l);
    double t = (y + 1.0 - (double)i * h) / h;
    double v = 1.0 - fabs(t);
    return v > 0.0 ? v : 0.0;
}

void or_sg_points(int N, int M, const int8_t *lvl, const int32_t *idx, double *y)
{
    for (int m = 0; m < M; m++)
        for (int n = 0; n < N; n++) y[m * N + n] = or_sg_coord(lvl[m * N + n], idx[m * N + n]);
}

void or_sg_eval(int N, int M, const int8_t *lvl, const int32_t *idx,
                const double *surplus, int Q, const double *yq, double *out)
{
    for (int q = 0; q < Q; q++) {
        double acc = 0.0;
        for (int m = 0; m < M; m++) {
            double prod = 1.0;
            for (int n = 0; n < N; n++) prod = prod * or_hat(lvl[m * N + n], idx[m * N + n], yq[q * N + n]);
            acc = acc + surplus[m] * prod;
        }
        out[q] = acc;
    }
}

static int same_point(int N, const int8_t *la, const int32_t *ia, const int8_t *lb, const int32_t *ib)
{
    for (int n = 0; n < N; n++)
        if (la[n] != lb[n] || ia[n] != ib[n]) return 0;
    return 1;
}

static int level_sum(int N, const int8_t *l)
{
    int s = 0;
    for (int n = 0; n < N; n++) s += l[n];
    return s;
}

/* Children of points first..M-1 whose |surplus| >= tau; returns how many were
 * written (or -1 if more than max_out would be needed). */
int or_sg_refine(int N, int M, const int8_t *lvl, const int32_t *idx,
                 int first, const double *surplus, double tau, int max_level,
                 int max_out, int8_t *out_lvl, int32_t *out_idx)
{
    int cnt = 0;
    int8_t cl[64];
    int32_t ci[64];
    if (N > 64) return -1;
    for (int m = first; m < M; m++) {
        if (!(fabs(surplus[m]) >= tau)) continue;
        if (level_sum(N, lvl + m * N) + 1 > max_level) continue;
        for (int n = 0; n < N; n++) {
            int nch = (lvl[m * N + n] == 0) ? 1 : 2;
            for (int c = 0; c < nch; c++) {
                for (int a = 0; a < N; a++) {
                    cl[a] = lvl[m * N + a];
                    ci[a] = idx[m * N + a];
                }
                if (lvl[m * N + n] == 0) {
                    cl[n] = 1;
                    ci[n] = 1;
                } else {
                    cl[n] = (int8_t)(lvl[m * N + n] + 1);
                    ci[n] = 2 * idx[m * N + n] + (c == 0 ? -1 : 1);
                }
                int dup = 0;
                for (int k = 0; k < M && !dup; k++) dup = same_point(N, cl, ci, lvl + k * N, idx + k * N);
                for (int k = 0; k < cnt && !dup; k++)
                    dup = same_point(N, cl, ci, out_lvl + k * N, out_idx + k * N);
                if (dup) continue;
                if (cnt >= max_out) return -1;
                for (int a = 0; a < N; a++) {
                    out_lvl[cnt * N + a] = cl[a];
                    out_idx[cnt * N + a] = ci[a];
                }
                cnt++;
            }
        }
    }
    return cnt;
}

/* The full grid of levels 0..level: the 2^N corners (corner c has i_n = bit n
 * of c), then `level` rounds in which every point of the newest level is
 * refined. */
int or_sg_initial(int N, int level, int max_out, int8_t *lvl, int32_t *idx)
{
    if (N < 1 || N > 30 || (1 << N) > max_out) return -1;
    int M = 1 << N;
    for (int c = 0; c < M; c++)
        for (int n = 0; n < N; n++) {
            lvl[c * N + n] = 0;
            idx[c * N + n] = (c >> n) & 1;
        }
    int first = 0;
    double *ones = malloc(sizeof(double) * max_out);
    for (int k = 0; k < max_out; k++) ones[k] = 1.0;
    for (int L = 1; L <= level; L++) {
        int add = or_sg_refine(N, M, lvl, idx, first, ones, 0.0, L, max_out - M,
                               lvl + M * N, idx + M * N);
        if (add < 0) { free(ones); return -1; }
        first = M;
        M += add;
    }
    free(ones);
    return M;
}

/* Stable ascending sort (insertion sort) of indices 0..M-1 by key. */
void or_sort_perm(int M, const double *keys, int32_t *perm)
{
    for (int i = 0; i < M; i++) perm[i] = i;
    for (int i = 1; i < M; i++) {
        int32_t v = perm[i];
        int j = i - 1;
        while (j >= 0 && keys[perm[j]] > keys[v]) {
            perm[j + 1] = perm[j];
            j--;
        }
        perm[j + 1] = v;
    }
}

double or_work_ratio(int S, int M, const int32_t *perm, const double *iters)
{
    double num = 0.0, den = 0.0;
    for (int k = 0; k * S < M; k++) {
        double mx = 0.0;
        for (int s = 0; s < S && k * S + s < M; s++) {
            double v = iters[perm[k * S + s]];
            if (v > mx) mx = v;
        }
        num = num + mx;
    }
    for (int i = 0; i < M; i++) den = den + iters[i];
    return (double)S * num / den;
}
