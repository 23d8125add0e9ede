/*
 * gen.c - seeded synthetic inputs (graphs, bytes, index draws) for the
 * Founsure GF(2) gather-XOR path. Definitions are stated in include/fs_gen.h.
 * No coding arithmetic lives here: this file only draws inputs.
 */
#include "fs_gen.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define FSG_GAMMA 0x9E3779B97F4A7C15ULL

static uint64_t fsg_mix(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

uint64_t fsg_next(uint64_t *state)
{
    *state += FSG_GAMMA;
    return fsg_mix(*state);
}

uint64_t fsg_at(uint64_t seed, uint64_t w)
{
    return fsg_mix(seed + (w + 1ULL) * FSG_GAMMA);
}

uint64_t fsg_uniform_int(uint64_t *state, uint64_t r)
{
    unsigned __int128 p = (unsigned __int128)fsg_next(state) * (unsigned __int128)r;
    return (uint64_t)(p >> 64);
}

double fsg_uniform_double(uint64_t *state)
{
    return (double)(fsg_next(state) >> 11) * 0x1.0p-53;
}

int fsg_fill_bytes(uint64_t seed, uint64_t offset, uint64_t nbytes, uint8_t *out)
{
    if (nbytes && !out) return -1;
    uint64_t i = 0;
    /* leading partial word */
    while (i < nbytes && ((offset + i) & 7ULL)) {
        uint64_t pos = offset + i;
        out[i] = (uint8_t)(fsg_at(seed, pos >> 3) >> (8 * (pos & 7ULL)));
        i++;
    }
    /* whole words, little-endian byte order */
    while (i + 8 <= nbytes) {
        uint64_t v = fsg_at(seed, (offset + i) >> 3);
        for (int q = 0; q < 8; q++) out[i + q] = (uint8_t)(v >> (8 * q));
        i += 8;
    }
    while (i < nbytes) {
        uint64_t pos = offset + i;
        out[i] = (uint8_t)(fsg_at(seed, pos >> 3) >> (8 * (pos & 7ULL)));
        i++;
    }
    return 0;
}

/* Omega_d of the Raptor distribution printed in Section 2.2. */
static const int32_t k_omega_deg[10] = {1, 2, 3, 4, 5, 8, 9, 19, 64, 65};
static const double k_omega_val[10] = {0.007969, 0.49357, 0.16622, 0.072646, 0.082558,
                                       0.056058, 0.037229, 0.05559, 0.025023, 0.003135};

int fsg_pmf(int32_t kind, int32_t k, double c, double delta,
            double *mu, int32_t len, double *info)
{
    if (!mu) return -1;
    if (kind == FSG_DIST_RSD) {
        if (k < 1 || len < k + 1 || !(c > 0.0) || !(delta > 0.0) || !(delta < 1.0)) return -2;
        double kd = (double)k;
        double R = c * log(kd / delta) * sqrt(kd);
        int32_t s = (R > 0.0) ? (int32_t)floor(kd / R) : k;
        if (s < 1) s = 1;
        if (s > k) s = k;
        double beta = 0.0;
        mu[0] = 0.0;
        for (int32_t d = 1; d <= k; d++) {
            double rho = (d == 1) ? 1.0 / kd : 1.0 / ((double)d * (double)(d - 1));
            double tau = 0.0;
            if (d < s) tau = R / ((double)d * kd);
            else if (d == s) {
                tau = R * log(R / delta) / kd;
                if (tau < 0.0) tau = 0.0;
            }
            mu[d] = rho + tau;
            beta += mu[d];
        }
        double mean = 0.0;
        for (int32_t d = 1; d <= k; d++) {
            mu[d] /= beta;
            mean += (double)d * mu[d];
        }
        for (int32_t d = k + 1; d < len; d++) mu[d] = 0.0;
        if (info) {
            info[0] = R;
            info[1] = (double)s;
            info[2] = beta;
            info[3] = mean;
        }
        return k;
    }
    if (kind == FSG_DIST_FINITE65 || kind == FSG_DIST_FINITE40 || kind == FSG_DIST_FINITE40F) {
        if (len < 66) return -2;
        for (int32_t d = 0; d < len; d++) mu[d] = 0.0;
        double raw = 0.0;
        for (int q = 0; q < 10; q++) raw += k_omega_val[q];
        for (int q = 0; q < 10; q++) {
            int32_t d = k_omega_deg[q];
            if (kind == FSG_DIST_FINITE40 && d > 40) continue;
            if (kind == FSG_DIST_FINITE40F && d > 40) d = 40;
            mu[d] += k_omega_val[q];
        }
        double tot = 0.0;
        int32_t dmax = 0;
        for (int32_t d = 1; d < len; d++) {
            tot += mu[d];
            if (mu[d] > 0.0) dmax = d;
        }
        double mean = 0.0;
        for (int32_t d = 1; d < len; d++) {
            mu[d] /= tot;
            mean += (double)d * mu[d];
        }
        if (info) {
            info[0] = 0.0;
            info[1] = 0.0;
            info[2] = raw;
            info[3] = mean;
        }
        return dmax;
    }
    return -3;
}

/* Degree draw from a pmf mu[0..dmax] (cumulative sum in fp64, ascending). */
static int32_t draw_degree(const double *cdf, int32_t dmax, uint64_t *st)
{
    double u = fsg_uniform_double(st);
    /* smallest d with u < cdf[d]; cdf is non-decreasing so the answer is a
     * support degree (cdf only rises where mu > 0) */
    int32_t lo = 1, hi = dmax;
    if (!(u < cdf[dmax])) {
        /* rounding left the total below u: largest support degree */
        int32_t d = dmax;
        while (d > 1 && cdf[d] == cdf[d - 1]) d--;
        return d;
    }
    while (lo < hi) {
        int32_t mid = lo + (hi - lo) / 2;
        if (u < cdf[mid]) hi = mid;
        else lo = mid + 1;
    }
    return lo;
}

static double *make_cdf(const double *mu, int32_t dmax)
{
    double *cdf = (double *)malloc(sizeof(double) * (size_t)(dmax + 1));
    if (!cdf) return NULL;
    double acc = 0.0;
    cdf[0] = 0.0;
    for (int32_t d = 1; d <= dmax; d++) {
        acc += mu[d];
        cdf[d] = acc;
    }
    return cdf;
}

static int cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* Floyd's algorithm: d distinct values of [0,K) into out (then sorted).
 * stamp[] has K entries; a value v is taken iff stamp[v] == tag. */
static void floyd(int32_t K, int32_t d, uint64_t *st, int32_t *out, int32_t *stamp, int32_t tag)
{
    int32_t cnt = 0;
    for (int32_t j = K - d; j < K; j++) {
        int32_t r = (int32_t)fsg_uniform_int(st, (uint64_t)j + 1ULL);
        int32_t v = (stamp[r] == tag) ? j : r;
        stamp[v] = tag;
        out[cnt++] = v;
    }
    if (d <= 32) {
        for (int32_t a = 1; a < d; a++) {
            int32_t x = out[a], q = a - 1;
            while (q >= 0 && out[q] > x) {
                out[q + 1] = out[q];
                q--;
            }
            out[q + 1] = x;
        }
    } else {
        qsort(out, (size_t)d, sizeof(int32_t), cmp_i32);
    }
}

int64_t fsg_lt_graph_nnz(int32_t k_int, int32_t n, const double *mu, int32_t dmax, uint64_t seed)
{
    if (k_int < 1 || n < 0 || !mu || dmax < 1) return -1;
    double *cdf = make_cdf(mu, dmax);
    if (!cdf) return -4;
    uint64_t st = seed;
    int64_t nnz = 0;
    for (int32_t j = 0; j < n; j++) {
        int32_t d = draw_degree(cdf, dmax, &st);
        if (d > k_int) d = k_int;
        nnz += d;
        st += (uint64_t)d * FSG_GAMMA; /* Floyd consumes exactly d outputs */
    }
    free(cdf);
    return nnz;
}

int64_t fsg_lt_graph(int32_t k_int, int32_t n, const double *mu, int32_t dmax,
                     uint64_t seed, int32_t *row_ptr, int32_t *col_idx, int64_t cap)
{
    if (k_int < 1 || n < 0 || !mu || dmax < 1 || !row_ptr || (cap > 0 && !col_idx)) return -1;
    double *cdf = make_cdf(mu, dmax);
    int32_t *stamp = (int32_t *)malloc(sizeof(int32_t) * (size_t)k_int);
    if (!cdf || !stamp) {
        free(cdf);
        free(stamp);
        return -4;
    }
    for (int32_t i = 0; i < k_int; i++) stamp[i] = -1;
    uint64_t st = seed;
    int64_t nnz = 0;
    row_ptr[0] = 0;
    for (int32_t j = 0; j < n; j++) {
        int32_t d = draw_degree(cdf, dmax, &st);
        if (d > k_int) d = k_int;
        if (nnz + d > cap || nnz + d > INT32_MAX) {
            free(cdf);
            free(stamp);
            return -5;
        }
        floyd(k_int, d, &st, col_idx + nnz, stamp, j);
        nnz += d;
        row_ptr[j + 1] = (int32_t)nnz;
    }
    free(cdf);
    free(stamp);
    return nnz;
}

int64_t fsg_precode_graph(int32_t b, int32_t m, int32_t q, uint64_t seed,
                          int32_t *row_ptr, int32_t *col_idx, int64_t cap)
{
    if (b < 0 || m < 0 || q < 0 || !row_ptr) return -1;
    int32_t qq = q < m ? q : m;
    int64_t nnz = (int64_t)b * qq;
    if (nnz > cap || nnz > INT32_MAX || (nnz > 0 && !col_idx)) return -5;
    for (int32_t j = 0; j <= m; j++) row_ptr[j] = 0;
    if (m == 0) return 0;
    int32_t *pick = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
    int32_t *stamp = (int32_t *)malloc(sizeof(int32_t) * (size_t)m);
    int32_t *fill = (int32_t *)malloc(sizeof(int32_t) * (size_t)m);
    if (!pick || !stamp || !fill) {
        free(pick);
        free(stamp);
        free(fill);
        return -4;
    }
    for (int32_t j = 0; j < m; j++) stamp[j] = -1;
    uint64_t st = seed;
    for (int32_t i = 0; i < b; i++) floyd(m, qq, &st, pick + (int64_t)i * qq, stamp, i);
    /* per-check counts, then members in ascending data order */
    for (int64_t e = 0; e < nnz; e++) row_ptr[pick[e] + 1]++;
    for (int32_t j = 0; j < m; j++) row_ptr[j + 1] += row_ptr[j];
    for (int32_t j = 0; j < m; j++) fill[j] = row_ptr[j];
    for (int32_t i = 0; i < b; i++)
        for (int32_t r = 0; r < qq; r++) {
            int32_t j = pick[(int64_t)i * qq + r];
            col_idx[fill[j]++] = i;
        }
    free(pick);
    free(stamp);
    free(fill);
    return nnz;
}

int fsg_sample_indices(int32_t n, int32_t count, uint64_t seed, int32_t *out)
{
    if (n < 0 || count < 0 || count > n || (count > 0 && !out)) return -1;
    if (count == 0) return 0;
    int32_t *a = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    if (!a) return -4;
    for (int32_t i = 0; i < n; i++) a[i] = i;
    uint64_t st = seed;
    for (int32_t i = 0; i < count; i++) {
        int32_t j = i + (int32_t)fsg_uniform_int(&st, (uint64_t)(n - i));
        int32_t tmp = a[i];
        a[i] = a[j];
        a[j] = tmp;
        out[i] = a[i];
    }
    free(a);
    return 0;
}

int32_t fsg_round_count(double fraction, int32_t n)
{
    double v = floor(fraction * (double)n + 0.5);
    if (v < 0.0) v = 0.0;
    if (v > (double)n) v = (double)n;
    return (int32_t)v;
}
