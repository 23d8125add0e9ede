/*
 * oracle.c - plain CPU oracle for the Founsure GF(2) gather-XOR path.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may call, link or
 * load this file: only tests/, __graft_entry__.smoke() and the CPU-baseline
 * leg of bench.py use it. It shares no code, header or helper with the CUDA
 * library; both receive the same seeded inputs (graphs, bytes, erasures)
 * from the input generator, which holds no coding arithmetic.
 *
 * Everything here is written for a reader checking it against the paper by
 * eye: plain byte loops, no blocking, no fusion, no reordering.
 *
 * Notation (Section 2.2): b data blocks, m = k - b precode parities
 * (check #1), k_int = b + m intermediate blocks (data 0..b-1, then parities
 * b..b+m-1), n coded blocks, t bytes per block. Blocks are stored
 * block-major: block i is bytes [i*t, (i+1)*t).
 *
 * Graphs arrive in CSR form:
 *   precode: m rows (checks), row j lists the data blocks of check j;
 *   lt:      n rows (coded blocks), row j lists the intermediates that coded
 *            block j is the XOR of (the neighbours drawn from Omega(x)).
 *
 * Functions and the passage each follows:
 *   or_encode  - Section 2.2, encoding steps (1) precode and (2) LDGM;
 *                the region XOR of Section 2.2 (first paragraph).
 *   or_dpg     - Algorithm 5 (Decoding Path Generation), Section 3.2, with
 *                the two rules of Section 3.1 (a level uses only symbols
 *                decoded in earlier levels; each source symbol is decoded by
 *                one lowest-degree coded symbol). Two-pass mode follows the
 *                Section 2.2 description of founsureDec (BP on the LT code,
 *                then BP on the precode).
 *   or_peel    - the payload of the decoding path: x_f is the XOR of the
 *                payload of g and of every other neighbour of g.
 *   or_peel_immediate - Algorithm 1 (BP skeleton) with immediate use of
 *                decoded symbols and constraints visited in a caller-given
 *                order; used only by tests to show the recovered set does
 *                not depend on the schedule.
 *
 * Readings of the paper taken here (the paper is silent or ambiguous):
 *   - maxit of Algorithms 1 and 5 is unbounded: iterate until a level
 *     finds no degree-1 constraint.
 *   - The G_i and G-bar_i of Algorithm 5 name the same set.
 *   - "g_d is minimum" means the ORIGINAL degree of g (its neighbour count);
 *     ties go to the smallest constraint index.
 *   - Joint decoding (default): surviving coded blocks and precode checks
 *     are peeled together. A precode check j is a constraint over its data
 *     members and parity b+j with payload zero. Constraint index space:
 *     coded rows 0..n-1, then checks n..n+m-1.
 *   - Unrecovered data blocks are returned as zero bytes.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_MODE_JOINT    0
#define OR_MODE_TWO_PASS 1

/* dst ^= src over t bytes (the region XOR of Section 2.2). */
static void xor_into(uint8_t *dst, const uint8_t *src, int64_t t)
{
    for (int64_t i = 0; i < t; i++) dst[i] ^= src[i];
}

/*
 * Encoding, Section 2.2:
 *   (1) parity p_j = XOR of the data blocks of check j   (j < m)
 *   (2) coded c_j  = XOR of the intermediates of row j   (j < n)
 * parity may be NULL when m == 0. Returns 0, or -1 on a bad index.
 */
int or_encode(int32_t b, int32_t m, int32_t n,
              const int32_t *pre_ptr, const int32_t *pre_idx,
              const int32_t *lt_ptr, const int32_t *lt_idx,
              int64_t t, const uint8_t *data, uint8_t *parity, uint8_t *coded)
{
    int32_t k_int = b + m;
    for (int32_t j = 0; j < m; j++) {
        uint8_t *p = parity + (int64_t)j * t;
        memset(p, 0, (size_t)t);
        for (int32_t e = pre_ptr[j]; e < pre_ptr[j + 1]; e++) {
            int32_t i = pre_idx[e];
            if (i < 0 || i >= b) return -1;
            xor_into(p, data + (int64_t)i * t, t);
        }
    }
    for (int32_t j = 0; j < n; j++) {
        uint8_t *c = coded + (int64_t)j * t;
        memset(c, 0, (size_t)t);
        for (int32_t e = lt_ptr[j]; e < lt_ptr[j + 1]; e++) {
            int32_t v = lt_idx[e];
            if (v < 0 || v >= k_int) return -1;
            const uint8_t *x = (v < b) ? data + (int64_t)v * t : parity + (int64_t)(v - b) * t;
            xor_into(c, x, t);
        }
    }
    return 0;
}

/* Constraint g of the joint graph: its neighbour count and neighbour e. */
static int32_t con_degree(int32_t g, int32_t n, const int32_t *pre_ptr, const int32_t *lt_ptr)
{
    if (g < n) return lt_ptr[g + 1] - lt_ptr[g];
    int32_t j = g - n;
    return pre_ptr[j + 1] - pre_ptr[j] + 1; /* members plus the parity itself */
}

static int32_t con_var(int32_t g, int32_t e, int32_t b, int32_t n,
                       const int32_t *pre_ptr, const int32_t *pre_idx,
                       const int32_t *lt_ptr, const int32_t *lt_idx)
{
    if (g < n) return lt_idx[lt_ptr[g] + e];
    int32_t j = g - n;
    int32_t deg = pre_ptr[j + 1] - pre_ptr[j];
    return (e < deg) ? pre_idx[pre_ptr[j] + e] : b + j;
}

/*
 * Algorithm 5 (DPG). Outputs the decoding path DP as pairs (f, g) in level
 * order, ascending f inside a level; level_of[p] is the level of pair p.
 * unrecovered[v] = 1 for every intermediate left in F.
 * Returns the number of pairs (= k_int on full recovery, i.e. |DP| = 2k
 * counting both members of each pair), or a negative value on error.
 */
int32_t or_dpg(int32_t b, int32_t m, int32_t n,
               const int32_t *pre_ptr, const int32_t *pre_idx,
               const int32_t *lt_ptr, const int32_t *lt_idx,
               const uint8_t *erased, int32_t mode,
               int32_t *pair_f, int32_t *pair_g, int32_t *level_of,
               uint8_t *unrecovered, int32_t *n_levels)
{
    int32_t k_int = b + m;
    int32_t n_con = n + m;
    uint8_t *in_F = (uint8_t *)malloc((size_t)k_int + 1);   /* F: unrecovered set */
    int32_t *best = (int32_t *)malloc(sizeof(int32_t) * ((size_t)k_int + 1));
    if (!in_F || !best) {
        free(in_F);
        free(best);
        return -4;
    }
    for (int32_t v = 0; v < k_int; v++) in_F[v] = 1; /* F <- K */

    int32_t npairs = 0, level = 0;
    int32_t n_stages = (mode == OR_MODE_TWO_PASS) ? 2 : 1;
    for (int32_t stage = 0; stage < n_stages; stage++) {
        for (;;) {
            /* survival matrix C: coded rows not in E, plus precode checks */
            for (int32_t v = 0; v < k_int; v++) best[v] = -1;
            int32_t found = 0;
            for (int32_t g = 0; g < n_con; g++) {
                int usable;
                if (g < n) usable = !erased[g] && (mode == OR_MODE_JOINT || stage == 0);
                else usable = (mode == OR_MODE_JOINT || stage == 1);
                if (!usable) continue;
                /* weight of column g after zeroing the rows of decoded symbols */
                int32_t deg = con_degree(g, n, pre_ptr, lt_ptr);
                int32_t weight = 0, f = -1;
                for (int32_t e = 0; e < deg; e++) {
                    int32_t v = con_var(g, e, b, n, pre_ptr, pre_idx, lt_ptr, lt_idx);
                    if (in_F[v]) {
                        weight++;
                        f = v;
                    }
                }
                if (weight != 1) continue;
                /* g is in G-bar_i; keep the lowest-degree g for f (ties: first g) */
                if (best[f] < 0 || deg < con_degree(best[f], n, pre_ptr, lt_ptr)) best[f] = g;
                found = 1;
            }
            if (!found) break;
            for (int32_t f = 0; f < k_int; f++) {
                if (best[f] < 0) continue;
                pair_f[npairs] = f;
                pair_g[npairs] = best[f];
                level_of[npairs] = level;
                npairs++;
            }
            /* F <- F minus the symbols decoded in this level (delayed update) */
            for (int32_t f = 0; f < k_int; f++)
                if (best[f] >= 0) in_F[f] = 0;
            level++;
        }
    }
    for (int32_t v = 0; v < k_int; v++) unrecovered[v] = in_F[v];
    if (n_levels) *n_levels = level;
    free(in_F);
    free(best);
    return npairs;
}

/*
 * Payload of the decoding path: for each pair (f, g) in DP order,
 *   x_f = payload(g) XOR (XOR of x_h for every other neighbour h of g),
 * payload(g) = coded block g for g < n, zero for a precode check.
 * data_out receives the b data blocks; unrecovered ones are zero.
 * parity_out (may be NULL) receives the m parity intermediates.
 */
int or_peel(int32_t b, int32_t m, int32_t n,
            const int32_t *pre_ptr, const int32_t *pre_idx,
            const int32_t *lt_ptr, const int32_t *lt_idx,
            int64_t t, const uint8_t *coded,
            int32_t npairs, const int32_t *pair_f, const int32_t *pair_g,
            uint8_t *data_out, uint8_t *parity_out)
{
    int32_t k_int = b + m;
    uint8_t *x = (uint8_t *)calloc((size_t)k_int * (size_t)t + 1, 1);
    if (!x) return -4;
    for (int32_t p = 0; p < npairs; p++) {
        int32_t f = pair_f[p], g = pair_g[p];
        uint8_t *dst = x + (int64_t)f * t;
        if (g < n) memcpy(dst, coded + (int64_t)g * t, (size_t)t);
        else memset(dst, 0, (size_t)t);
        int32_t deg = con_degree(g, n, pre_ptr, lt_ptr);
        for (int32_t e = 0; e < deg; e++) {
            int32_t h = con_var(g, e, b, n, pre_ptr, pre_idx, lt_ptr, lt_idx);
            if (h != f) xor_into(dst, x + (int64_t)h * t, t);
        }
    }
    memcpy(data_out, x, (size_t)b * (size_t)t);
    if (parity_out && m > 0) memcpy(parity_out, x + (int64_t)b * t, (size_t)m * (size_t)t);
    free(x);
    return 0;
}

/*
 * Algorithm 1 (BP skeleton) with immediate use of each decoded symbol:
 * sweep the usable constraints in the order `order` (a permutation of
 * 0..n+m-1), decode whenever a constraint has exactly one unknown, repeat
 * sweeps until one changes nothing. Writes unrecovered[v] like or_dpg and
 * returns the number of recovered intermediates. Symbolic only.
 */
int32_t or_peel_immediate(int32_t b, int32_t m, int32_t n,
                          const int32_t *pre_ptr, const int32_t *pre_idx,
                          const int32_t *lt_ptr, const int32_t *lt_idx,
                          const uint8_t *erased, const int32_t *order,
                          uint8_t *unrecovered)
{
    int32_t k_int = b + m, n_con = n + m, recovered = 0;
    for (int32_t v = 0; v < k_int; v++) unrecovered[v] = 1;
    int changed = 1;
    while (changed) {
        changed = 0;
        for (int32_t q = 0; q < n_con; q++) {
            int32_t g = order[q];
            if (g < n && erased[g]) continue;
            int32_t deg = con_degree(g, n, pre_ptr, lt_ptr);
            int32_t weight = 0, f = -1;
            for (int32_t e = 0; e < deg; e++) {
                int32_t v = con_var(g, e, b, n, pre_ptr, pre_idx, lt_ptr, lt_idx);
                if (unrecovered[v]) {
                    weight++;
                    f = v;
                }
            }
            if (weight == 1) {
                unrecovered[f] = 0;
                recovered++;
                changed = 1;
            }
        }
    }
    return recovered;
}
