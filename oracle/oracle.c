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
 *   or_cga     - Algorithm 4 (Check Generation Algorithm): check #2 and
 *                check #3 equations from the LT generator matrix.
 *   or_local_dpg / or_local_peel - repair of lost coded blocks by peeling
 *                over check #3 groups, scheduled like Algorithm 5.
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
 *   - Algorithm 4: zero_columns(B) counts the all-zero columns of B (the
 *     loop's comment; the text says "nonzero"); k is the number of rows of
 *     B, the k_int intermediates; an index listed twice in an LT row cancels.
 *   - Repair from check #3 groups: the smallest offering group repairs a
 *     block (the paper orders groups by cardinality so the smallest is used
 *     first); ties go to the lowest group index; unrepaired lost blocks are
 *     returned as zero bytes.
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
 *   (1) parity p_j = XOR of the members of check j, in order j = 0..m-1
 *       (members are data blocks; in a chained precode such as the array
 *       LDPC code of Algorithm 2 a member may also be an earlier parity
 *       b + i, i < j, which is final by then)
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
            if (i < 0 || i >= b + j) return -1;
            xor_into(p, i < b ? data + (int64_t)i * t : parity + (int64_t)(i - b) * t, t);
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
 * *n_sweeps (may be NULL) receives the number of sweeps that decoded at
 * least one symbol: the iteration count t_m of Section 3.1, to set beside
 * the level count of the delayed schedule of Algorithm 5.
 */
int32_t or_peel_immediate(int32_t b, int32_t m, int32_t n,
                          const int32_t *pre_ptr, const int32_t *pre_idx,
                          const int32_t *lt_ptr, const int32_t *lt_idx,
                          const uint8_t *erased, const int32_t *order,
                          uint8_t *unrecovered, int32_t *n_sweeps)
{
    int32_t k_int = b + m, n_con = n + m, recovered = 0, sweeps = 0;
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
        if (changed) sweeps++;
    }
    if (n_sweeps) *n_sweeps = sweeps;
    return recovered;
}

/* ---------------------------------------------------------------------------
 * Local recovery groups (check #2 and check #3 equations) and repair from
 * them.
 *
 * Sets of indices are sorted int32 arrays; the XOR of two GF(2) columns is
 * the symmetric difference of their sets, and the weight w of a column is the
 * size of its set.
 */
typedef struct {
    int32_t *v;
    int32_t len, cap;
} or_set;

static int set_reserve(or_set *s, int32_t cap)
{
    if (cap <= s->cap) return 0;
    int32_t c = s->cap ? s->cap : 8;
    while (c < cap) c *= 2;
    int32_t *p = (int32_t *)realloc(s->v, (size_t)c * sizeof(int32_t));
    if (!p) return -1;
    s->v = p;
    s->cap = c;
    return 0;
}

static int cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* w(a XOR b): elements in exactly one of the two sets. */
static int32_t set_xor_size(const or_set *a, const or_set *b)
{
    int32_t i = 0, j = 0, w = 0;
    while (i < a->len && j < b->len) {
        if (a->v[i] == b->v[j]) { i++; j++; }
        else if (a->v[i] < b->v[j]) { i++; w++; }
        else { j++; w++; }
    }
    return w + (a->len - i) + (b->len - j);
}

/* a = a XOR b, through tmp (which then holds the old a). */
static int set_xor_into(or_set *a, const or_set *b, or_set *tmp)
{
    if (set_reserve(tmp, a->len + b->len + 1)) return -1;
    int32_t i = 0, j = 0, w = 0;
    while (i < a->len && j < b->len) {
        if (a->v[i] == b->v[j]) { i++; j++; }
        else if (a->v[i] < b->v[j]) tmp->v[w++] = a->v[i++];
        else tmp->v[w++] = b->v[j++];
    }
    while (i < a->len) tmp->v[w++] = a->v[i++];
    while (j < b->len) tmp->v[w++] = b->v[j++];
    tmp->len = w;
    or_set t = *a;
    *a = *tmp;
    *tmp = t;
    return 0;
}

void or_free(void *p) { free(p); }

/*
 * Check Generation Algorithm (Algorithm 4, CGA; Section "Algorithm for
 * Jointly Generating Check #2 and Check #3 Equations").
 *
 * B is the k x n generator matrix of the LT layer: column j is the set of
 * intermediates of coded block j (row j of the lt CSR; an index listed twice
 * cancels). L starts as the n x n identity (column j = {j}). A sweep takes
 * j = 0..n-1 and, inside it, i = 0..n-1: when i != j, 2 w(b_j) > w(b_i) and
 * w(b_j XOR b_i) < w(b_j), it sets b_j = b_j XOR b_i and l_j = l_j XOR l_i.
 * Sweeps repeat while fewer than n - k columns of B are zero (the reading of
 * zero_columns(B): the number of all-zero columns) and stop after a sweep
 * that changed nothing, or after max_sweeps sweeps when max_sweeps > 0.
 *
 * Throughout, b_j is the XOR of the original columns named by l_j, so the
 * coded blocks of l_j XOR to zero when b_j = 0 (a check #3 group) and to
 * intermediate e when b_j = {e} (a check #2 equation).
 *
 * *out (malloc'ed; free with or_free) receives, for each column j in order,
 * the record [w(b_j), e, |l_j|, l_j ...] with e the single member of b_j when
 * w(b_j) == 1 and -1 otherwise; *out_len its length in ints. Returns the
 * number of sweeps run, or -1 when memory runs out.
 */
int32_t or_cga(int32_t k, int32_t n, const int32_t *lt_ptr, const int32_t *lt_idx,
               int32_t max_sweeps, int32_t **out, int64_t *out_len)
{
    *out = NULL;
    *out_len = 0;
    or_set *B = (or_set *)calloc((size_t)n + 1, sizeof(or_set));
    or_set *L = (or_set *)calloc((size_t)n + 1, sizeof(or_set));
    or_set tmp = {0}, row = {0};
    int32_t sweeps = -1;
    if (!B || !L) goto done;
    for (int32_t j = 0; j < n; j++) {
        int32_t d = lt_ptr[j + 1] - lt_ptr[j];
        if (set_reserve(&row, d + 1) || set_reserve(&L[j], 1)) goto done;
        memcpy(row.v, lt_idx + lt_ptr[j], (size_t)d * sizeof(int32_t));
        qsort(row.v, (size_t)d, sizeof(int32_t), cmp_i32);
        if (set_reserve(&B[j], d + 1)) goto done;
        B[j].len = 0;
        for (int32_t e = 0; e < d;) {  /* pairs of equal entries cancel */
            int32_t c = 1;
            while (e + c < d && row.v[e + c] == row.v[e]) c++;
            if (c & 1) B[j].v[B[j].len++] = row.v[e];
            e += c;
        }
        L[j].v[0] = j;
        L[j].len = 1;
    }
    sweeps = 0;
    for (;;) {
        int32_t zero = 0;
        for (int32_t j = 0; j < n; j++) zero += B[j].len == 0;
        if (zero >= n - k) break;
        if (max_sweeps > 0 && sweeps >= max_sweeps) break;
        int changed = 0;
        for (int32_t j = 0; j < n; j++) {
            for (int32_t i = 0; i < n; i++) {
                if (i == j || !(2 * B[j].len > B[i].len)) continue;
                if (set_xor_size(&B[j], &B[i]) < B[j].len) {
                    if (set_xor_into(&B[j], &B[i], &tmp) || set_xor_into(&L[j], &L[i], &tmp)) {
                        sweeps = -1;
                        goto done;
                    }
                    changed = 1;
                }
            }
        }
        sweeps++;
        if (!changed) break;
    }
    int64_t len = 0;
    for (int32_t j = 0; j < n; j++) len += 3 + L[j].len;
    *out = (int32_t *)malloc((size_t)(len + 1) * sizeof(int32_t));
    if (!*out) { sweeps = -1; goto done; }
    int64_t o = 0;
    for (int32_t j = 0; j < n; j++) {
        (*out)[o++] = B[j].len;
        (*out)[o++] = B[j].len == 1 ? B[j].v[0] : -1;
        (*out)[o++] = L[j].len;
        memcpy(*out + o, L[j].v, (size_t)L[j].len * sizeof(int32_t));
        o += L[j].len;
    }
    *out_len = o;
done:
    if (B) for (int32_t j = 0; j < n; j++) free(B[j].v);
    if (L) for (int32_t j = 0; j < n; j++) free(L[j].v);
    free(B);
    free(L);
    free(tmp.v);
    free(row.v);
    return sweeps;
}

/*
 * Repair of lost coded blocks from check #3 groups (the coded-only local
 * groups; repair, like decoding, is BP, Section "Reading/Formating" and
 * "Update Process"), scheduled like Algorithm 5: level by level, every group
 * with exactly one lost and not yet repaired member f (counted against the
 * state at the level start) offers f; each offered f takes the offering group
 * of smallest cardinality, ties to the lowest group index; then every f of
 * the level counts as repaired. It stops at a level with no offer.
 * groups: G rows over coded block indices (0..n-1). Writes the pairs in level
 * order (ascending f inside a level), their levels, the unrepaired flags (lost
 * and not repaired), *n_levels; returns the number of pairs (-1: no memory).
 */
int32_t or_local_dpg(int32_t n, int32_t G, const int32_t *g_ptr, const int32_t *g_idx,
                     const uint8_t *lost, int32_t *pair_f, int32_t *pair_g, int32_t *level_of,
                     uint8_t *unrepaired, int32_t *n_levels)
{
    uint8_t *unknown = (uint8_t *)malloc((size_t)n + 1);
    int32_t *best = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
    if (!unknown || !best) { free(unknown); free(best); return -1; }
    for (int32_t s = 0; s < n; s++) unknown[s] = lost[s] ? 1 : 0;
    int32_t np = 0, level = 0;
    for (;;) {
        for (int32_t s = 0; s < n; s++) best[s] = -1;
        for (int32_t g = 0; g < G; g++) {
            int32_t cnt = 0, f = -1;
            for (int32_t e = g_ptr[g]; e < g_ptr[g + 1]; e++)
                if (unknown[g_idx[e]]) { cnt++; f = g_idx[e]; }
            if (cnt != 1) continue;
            int32_t card = g_ptr[g + 1] - g_ptr[g];
            int32_t cur = best[f];
            if (cur < 0 || card < g_ptr[cur + 1] - g_ptr[cur] ||
                (card == g_ptr[cur + 1] - g_ptr[cur] && g < cur))
                best[f] = g;
        }
        int32_t found = 0;
        for (int32_t s = 0; s < n; s++) {
            if (best[s] < 0) continue;
            pair_f[np] = s;
            pair_g[np] = best[s];
            level_of[np] = level;
            np++;
            found++;
        }
        if (!found) break;
        for (int32_t s = 0; s < n; s++)
            if (best[s] >= 0) unknown[s] = 0;
        level++;
    }
    for (int32_t s = 0; s < n; s++) unrepaired[s] = unknown[s];
    *n_levels = level;
    free(unknown);
    free(best);
    return np;
}

/*
 * The payload of a repair path: for each pair (f, g) in order, coded block f
 * becomes the XOR of the other members of group g (all known by then).
 * coded is updated in place.
 */
int or_local_peel(int32_t n, const int32_t *g_ptr, const int32_t *g_idx, int64_t t,
                  uint8_t *coded, int32_t npairs, const int32_t *pair_f, const int32_t *pair_g)
{
    (void)n;
    for (int32_t p = 0; p < npairs; p++) {
        int32_t f = pair_f[p], g = pair_g[p];
        uint8_t *dst = coded + (int64_t)f * t;
        memset(dst, 0, (size_t)t);
        for (int32_t e = g_ptr[g]; e < g_ptr[g + 1]; e++) {
            int32_t h = g_idx[e];
            if (h != f) xor_into(dst, coded + (int64_t)h * t, t);
        }
    }
    return 0;
}
