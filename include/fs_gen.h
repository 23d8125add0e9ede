/*
 * fs_gen.h - seeded synthetic inputs for the Founsure GF(2) gather-XOR path.
 *
 * This library produces INPUTS only: the bytes of data blocks, the bipartite
 * graphs (precode and LT/LDGM generator in CSR form), erasure patterns and
 * index draws. It performs none of the coding arithmetic (no XOR of blocks,
 * no peeling); both the CUDA library and the CPU oracle receive its arrays.
 *
 * Pseudo-random source: splitmix64 (S. Vigna, public domain), used here in
 * place of the paper's unspecified linear congruential generator (Section 1
 * mentions an LCG keyed by the seed; Section 2.2 footnote gives the default
 * graph seed 1389488782).
 *   state s; next(): s += 0x9E3779B97F4A7C15; return mix(s)
 *   mix(z): z = (z ^ z>>30) * 0xBF58476D1CE4E5B9
 *           z = (z ^ z>>27) * 0x94D049BB133111EB; return z ^ z>>31
 * Output number w (0-based) of a stream seeded with s0 is mix(s0 + (w+1)*g),
 * so byte streams can be produced out of order.
 *   uniform integer in [0,r): high 64 bits of next() * r (no rejection)
 *   uniform double in [0,1):  (next() >> 11) * 2^-53
 *
 * Degree distributions (Section 2.2):
 *   Robust Soliton (Luby, cited in Section 1), k inputs, parameters c, delta:
 *     R = c ln(k/delta) sqrt(k); rho(1) = 1/k, rho(d) = 1/(d(d-1)) for d>=2;
 *     s = floor(k/R) clamped to [1,k]; tau(d) = R/(d k) for d < s,
 *     tau(s) = max(0, R ln(R/delta) / k), tau(d) = 0 for d > s;
 *     beta = sum(rho + tau); mu = (rho + tau) / beta.
 *   FiniteDist Omega(x) printed in Section 2.2 (Raptor distribution, degrees
 *     1,2,3,4,5,8,9,19,64,65), renormalised because its coefficients sum to
 *     0.999998. Max-degree-40 readings: DROP removes degrees 64 and 65 and
 *     renormalises; FOLD moves their mass to degree 40.
 *   Degree draw: u = uniform double; d = smallest degree whose cumulative
 *     probability (fp64, ascending d) exceeds u, else the largest support
 *     degree; clamped to the number of inputs.
 *   Neighbours: d distinct inputs by Floyd's algorithm (for j = K-d..K-1:
 *     r = uniform in [0,j]; take j if r is already taken, else r), stored
 *     ascending. One stream per graph; each coded row draws its degree then
 *     its neighbours.
 *   Precode: each data block i, in order, joins min(q, m) distinct checks
 *     drawn by Floyd's algorithm; the CSR lists each check's members
 *     ascending. An empty check defines a zero parity block.
 *   Index draws (erasures, updates, losses): partial Fisher-Yates, the first
 *     `count` entries of a shuffled [0,n) in draw order.
 *
 * Every function returns 0 on success and a negative value on bad arguments
 * or a too-small output capacity; it never aborts. Buffers are caller-owned
 * host memory.
 */
#ifndef FS_GEN_H
#define FS_GEN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Seeds. Graph seed is the paper's default; the others are stated choices. */
#define FSG_SEED_GRAPH   1389488782ULL
#define FSG_SEED_PRECODE (FSG_SEED_GRAPH + 1ULL)
#define FSG_SEED_DATA    1ULL
#define FSG_SEED_ERASE   2ULL
#define FSG_SEED_UPDATE  3ULL
#define FSG_SEED_REPAIR  4ULL
#define FSG_SEED_NEWDATA 5ULL
/* Stripe s adds s << 32 to every seed; round r of a repeated draw adds r << 20. */
#define FSG_STRIPE_SHIFT 32
#define FSG_ROUND_SHIFT  20

/* Distribution kinds for fsg_pmf(). */
#define FSG_DIST_RSD        0  /* params: c, delta */
#define FSG_DIST_FINITE65   1  /* the printed Omega, renormalised */
#define FSG_DIST_FINITE40   2  /* max-degree-40, DROP reading (default) */
#define FSG_DIST_FINITE40F  3  /* max-degree-40, FOLD reading */

/* One splitmix64 step: advances *state and returns the output. */
uint64_t fsg_next(uint64_t *state);
/* Output number w of a stream seeded with seed (counter form). */
uint64_t fsg_at(uint64_t seed, uint64_t w);
uint64_t fsg_uniform_int(uint64_t *state, uint64_t r);
double   fsg_uniform_double(uint64_t *state);

/* nbytes of the byte stream of `seed` starting at byte `offset`:
 * byte i is little-endian byte (i mod 8) of output number floor(i/8). */
int fsg_fill_bytes(uint64_t seed, uint64_t offset, uint64_t nbytes, uint8_t *out);

/* Probability mass function of a degree distribution over inputs 0..k:
 * writes mu[0..k_or_max] (mu[0] = 0). For FSG_DIST_RSD `len` must be >= k+1;
 * for the finite kinds len >= 66. info (may be NULL) receives
 * {R, s, beta, mean degree} for RSD and {0, 0, raw sum, mean} otherwise.
 * Returns the largest support degree (>0) or a negative error. */
int fsg_pmf(int32_t kind, int32_t k, double c, double delta,
            double *mu, int32_t len, double *info);

/* Number of LT edges fsg_lt_graph() will produce (runs the stream without
 * drawing neighbours). Returns nnz >= 0 or a negative error. */
int64_t fsg_lt_graph_nnz(int32_t k_int, int32_t n, const double *mu, int32_t dmax,
                         uint64_t seed);
/* LT/LDGM generator: n rows over k_int inputs. row_ptr has n+1 entries,
 * col_idx capacity `cap`. Returns nnz or a negative error. */
int64_t fsg_lt_graph(int32_t k_int, int32_t n, const double *mu, int32_t dmax,
                     uint64_t seed, int32_t *row_ptr, int32_t *col_idx, int64_t cap);
/* Random left-q-regular precode: m checks over b data blocks. row_ptr has
 * m+1 entries, col_idx capacity b*min(q,m). Returns nnz or a negative error. */
int64_t fsg_precode_graph(int32_t b, int32_t m, int32_t q, uint64_t seed,
                          int32_t *row_ptr, int32_t *col_idx, int64_t cap);

/* First `count` entries of a Fisher-Yates shuffle of [0,n), in draw order. */
int fsg_sample_indices(int32_t n, int32_t count, uint64_t seed, int32_t *out);
/* round-half-up(fraction * n) clamped to [0,n]. */
int32_t fsg_round_count(double fraction, int32_t n);

#ifdef __cplusplus
}
#endif
#endif
