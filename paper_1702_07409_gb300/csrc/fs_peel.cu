// fs_peel.cu - peeling decode split into a symbolic pass and a payload pass.
//
// k_dpg / k_dpg_compact: Decoding Path Generation (Algorithm 5, Section 3.2)
//   on one CTA. Per constraint g the pass keeps res[g], the number of its
//   variables still unknown, and xs[g], the XOR of their indices: when
//   res[g] == 1, xs[g] IS the one unknown, so no row is scanned. A level is:
//     A. every frontier constraint g (res 1 at the level start) bids
//        key = (degree(g), g) for its unknown f with an atomicMin: the lowest
//        original degree wins, ties go to the lowest constraint index
//        (Section 3.1, second rule);
//     B. each f with a bid becomes a pair (f, g) of the path; one block-wide
//        scan places its recipe (the padded row of g), its gather segments,
//        its accumulator slot and the adjacency slots of f;
//     C. the constraints containing each newly decoded f are updated
//        (res -= 1, xs ^= f); a constraint whose count goes 2 -> 1 joins the
//        next frontier.
//   res/xs only change in C, after every bid of the level was placed, so a
//   level uses only symbols decoded in earlier levels (Section 3.1, first
//   rule). Appends to the shared lists are warp-aggregated.
//   k_dpg_compact (graphs with at most 65536 intermediates and constraints)
//   keeps every per-level access in shared memory: 16-bit indices, 32-bit
//   keys, a shared copy of the transposed graph, and per constraint one word
//   (sum << 16 | res) where sum is the SUM of the unknown indices mod 2^16
//   instead of their XOR: decoding member f subtracts (f << 16) + 1 in one
//   atomic (res >= 1 before it, so the low field never borrows into sum), and
//   the value it returns is the constraint's state just before that update.
//   The one update that takes res from 2 to 1 therefore knows the last
//   unknown (sum - f, indices below 2^16) and bids for it at once, unless
//   that unknown is decoded in the same level (then res reaches 0 in this
//   step C too). Step C is one pass with S threads per pair (S = 2^k <=
//   T / pairs of the level), each taking every S-th constraint of its
//   pair, so no scan places the level's adjacency slots; step A of a level
//   is done by the previous level's step C: two block barriers per level.
//   k_dpg is the general form, with its state spilled to the workspace when
//   needed.
//
// k_peel: the payload. Each CTA owns one slice of L 16-byte words of every
//   block (about one CTA per SM, so every slice is in flight at once) and
//   walks all levels; pairs of a level are independent (no intermediate is
//   written twice and none is read in the level that writes it), so a
//   __syncthreads between levels is the only ordering needed: no grid-wide
//   synchronisation and no per-level launch. The path is staged ahead: the
//   pair records and segment list of level l+2 with two bulk copies
//   (cp.async.bulk, completion on an mbarrier; each range is 16-byte
//   aligned), the padded graph rows (recipes) of level l+1 with 16-byte
//   cp.async copies spread over all threads (a chunk list names the pair of
//   each 16-byte chunk), plus an L2 prefetch of level l+1's coded payloads. A recipe is gathered in segments of kRecipeSeg
//   entries, one thread per (segment, word), all loads of a segment in
//   flight at once; pairs with several segments combine them in
//   shared-memory accumulators, and the segment whose count completes a
//   word's sum writes it out (no second barrier in the level). 1024 threads
//   of at most 64 registers: twice the warps of 2-word items, which need more.
#include <cooperative_groups.h>

#include <algorithm>
#include <vector>

#include "fs_internal.cuh"

namespace cg = cooperative_groups;

namespace {

constexpr int kDpgThreads = 1024;  // fills an SM's registers: no other kernel's CTA shares it
static_assert((kDpgThreads & (kDpgThreads - 1)) == 0, "the compact schedule splits the CTA in powers of two");
constexpr int kPeelThreads = 1024;  // 64 registers a thread: one item (segment, word) each
constexpr int kPeelLmax = 64;       // largest slice (words) of one payload CTA
constexpr int kStagePairs = 256;    // pairs of one level held in shared memory
constexpr int kStageRecipe = 4096;  // recipe entries of one level held in shared memory
constexpr int kStageLevels = 1024;  // level table entries held in shared memory
constexpr int kStageSegs = 512;     // gather segments of one level
constexpr int kStageMulti = 32;     // pairs with several segments in one level
constexpr int kRec = 8;             // ints per pair record
constexpr long long kWaitLimit = 1ll << 22;  // bounded mbarrier waits
constexpr unsigned long long kEmpty = ~0ull;

// ---------------------------------------------------------------------------
// shared helpers

// Position of the calling thread in a shared list: one atomicAdd per group
// of converged threads.
__device__ __forceinline__ int append_slot(int *counter) {
    cg::coalesced_group grp = cg::coalesced_threads();
    int base = 0;
    if (grp.thread_rank() == 0) base = atomicAdd(counter, (int)grp.size());
    return grp.shfl(base, 0) + (int)grp.thread_rank();
}

// Exclusive prefix sum of four counters over the first nw warps of the block
// (the warps holding items); *total receives the sums. Only those warps call
// it; they meet on named barrier 1. Every warp scans its own lanes,
// publishes its total in s_warp[buf], and after the barrier sums the totals
// of the warps before it. Consecutive calls must alternate buf (the other
// buffer may still be read by slow warps).
__device__ int4 warps_excl_scan4(int4 x, int4 *total, int4 (*s_warp)[32], int buf, int nw) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int4 v = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int a = __shfl_up_sync(0xffffffffu, v.x, o);
        const int b = __shfl_up_sync(0xffffffffu, v.y, o);
        const int c = __shfl_up_sync(0xffffffffu, v.z, o);
        const int d = __shfl_up_sync(0xffffffffu, v.w, o);
        if (lane >= o) {
            v.x += a;
            v.y += b;
            v.z += c;
            v.w += d;
        }
    }
    if (nw == 1) {
        *total = make_int4(__shfl_sync(0xffffffffu, v.x, 31), __shfl_sync(0xffffffffu, v.y, 31),
                           __shfl_sync(0xffffffffu, v.z, 31), __shfl_sync(0xffffffffu, v.w, 31));
        return make_int4(v.x - x.x, v.y - x.y, v.z - x.z, v.w - x.w);
    }
    if (lane == 31) s_warp[buf][wid] = v;
    asm volatile("bar.sync 1, %0;\n" ::"r"(nw * 32) : "memory");
    // lane j holds warp j's total; before = sum over j < wid, all = sum over j < nw
    const int4 t = lane < nw ? s_warp[buf][lane] : make_int4(0, 0, 0, 0);
    int4 b = lane < wid ? t : make_int4(0, 0, 0, 0);
    int4 all = t;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        b.x += __shfl_xor_sync(0xffffffffu, b.x, o);
        b.y += __shfl_xor_sync(0xffffffffu, b.y, o);
        b.z += __shfl_xor_sync(0xffffffffu, b.z, o);
        b.w += __shfl_xor_sync(0xffffffffu, b.w, o);
        all.x += __shfl_xor_sync(0xffffffffu, all.x, o);
        all.y += __shfl_xor_sync(0xffffffffu, all.y, o);
        all.z += __shfl_xor_sync(0xffffffffu, all.z, o);
        all.w += __shfl_xor_sync(0xffffffffu, all.w, o);
    }
    *total = all;
    return make_int4(b.x + v.x - x.x, b.y + v.y - x.y, b.z + v.z - x.z, b.w + v.w - x.w);
}

template <typename T>
__device__ __forceinline__ T *place(unsigned char *smem, int32_t off, T *global) {
    return off >= 0 ? reinterpret_cast<T *>(smem + off) : global;
}

// ---------------------------------------------------------------------------
// symbolic pass

}  // namespace

bool flow_applies(const fs_code *c);

namespace {

// flow_hdr word set to 1 by the compact schedule when it wrote flow_list
constexpr int kFlowHdrList = 8;
// constraints whose members the compact schedule lists in recovery order:
// those a pair of which can have more than 8 loads (kFlowSeg)
constexpr int kListDeg = 9;

struct DpgArgs {
    const int32_t *con_ptr, *con_ptr4, *con_xs, *con_sum, *var_ptr, *var_idx;
    const uint8_t *erased;
    int32_t b, n, k_int, n_con;
    int two_pass;
    // workspace copies of the general form's state
    int32_t *res, *xs;
    unsigned long long *best;
    uint8_t *known;
    int32_t *front_a, *front_b, *touched;
    // outputs
    int32_t *pair_f, *pair_g, *level_off, *seg_pair, *chunk_pair, *unrec_list, *hdr;
    int4 *pair_rec, *level_tab;
    uint8_t *unrecovered;
    int32_t *n_unrecovered;
    // the dataflow plan: header (a new path has no plan yet), the level of
    // every recovered intermediate, units per key (cleared)
    int32_t *flow_hdr;
    uint16_t *flow_lvl;
    int32_t *flow_hist;
    // the key walk's plan: members of every constraint of degree >=
    // kListDeg in the order they were recovered, and every pair's level and
    // constraint degree; or null
    uint16_t *flow_list;
    uint32_t *flow_pinfo;
};

// stage: -1 joint (every surviving coded row and every check), 0 coded rows
// only, 1 checks only (two-pass mode, Section 2.2). ok: survival flags in
// shared memory, or null to read the erasure flags.
__device__ __forceinline__ bool usable(const DpgArgs &a, const uint8_t *ok, int32_t g, int stage) {
    if (g < a.n) return stage <= 0 && (ok ? ok[g] != 0 : a.erased[g] == 0);
    return stage != 0;
}

// Per-level bookkeeping shared by both forms of the symbolic pass.
struct LevelCursor {
    int32_t np = 0, level = 0, rb = 0, sb = 0, cb = 0, maxp = 0, maxr = 0, maxs = 0, maxm = 0;
    int scan_buf = 0;
};

// Step B of a level in the general form: writes the pairs i < nt (pair_of(i)
// gives f and g) with their payload records, and stores the level's totals in
// *s_len (read them after the next block barrier). Called by every thread;
// only the warps holding pairs scan.
template <typename PairOf>
__device__ void emit_level(const DpgArgs &a, LevelCursor &cur, int nt, PairOf pair_of,
                           const int32_t *cptr4, int4 (*s_warp4)[32], int4 *s_len) {
    int4 len = make_int4(0, 0, 0, 0);
    const int32_t sb = cur.sb;
    for (int base = 0; base < nt; base += blockDim.x) {
        const int nw = (min(nt - base, (int)blockDim.x) + 31) >> 5;  // warps holding pairs
        const int buf = cur.scan_buf;
        cur.scan_buf ^= 1;
        if ((int)(threadIdx.x >> 5) >= nw) continue;
        const int i = base + threadIdx.x;
        int4 cnt = make_int4(0, 0, 0, 0);  // recipe, segments, multi (w unused)
        int32_t f = -1, g = -1;
        if (i < nt) {
            pair_of(i, &f, &g);
            cnt.x = cptr4[g + 1] - cptr4[g];  // padded row length (multiple of 4)
            cnt.y = (cnt.x + kRecipeSeg - 1) / kRecipeSeg;
            cnt.z = cnt.y > 1 ? 1 : 0;
        }
        int4 total;
        const int4 off = warps_excl_scan4(cnt, &total, s_warp4, buf, nw);
        if (i < nt) {
            const int32_t p = cur.np + i;
            a.pair_f[p] = f;
            a.pair_g[p] = g;
            a.flow_lvl[f] = (uint16_t)cur.level;
            const int32_t so = len.y + off.y;
            a.pair_rec[2 * (size_t)p] = make_int4(f, g, len.x + off.x, cnt.z ? len.z + off.z : -1);
            a.pair_rec[2 * (size_t)p + 1] = make_int4(cptr4[g], cnt.x, so, cnt.y);
            for (int k = 0; k < cnt.y; ++k) a.seg_pair[sb + so + k] = i;
            const int32_t c0 = cur.cb + ((len.x + off.x) >> 2);
            for (int k = 0; k < (cnt.x >> 2); ++k) a.chunk_pair[c0 + k] = i;
        }
        len.x += total.x;
        len.y += total.y;
        len.z += total.z;
        len.w += total.w;
    }
    if (threadIdx.x == 0) {  // warp 0 holds pairs whenever nt > 0
        a.level_off[cur.level] = cur.np;
        a.level_tab[2 * cur.level] = make_int4(cur.np, nt, sb, len.y);
        a.level_tab[2 * cur.level + 1] = make_int4(cur.cb, len.x >> 2, 0, 0);
        *s_len = len;
    }
}

__device__ __forceinline__ void advance(LevelCursor &cur, int nt, const int4 &len) {
    cur.maxp = max(cur.maxp, nt);
    cur.maxr = max(cur.maxr, len.x);
    cur.maxs = max(cur.maxs, len.y);
    cur.maxm = max(cur.maxm, len.z);
    cur.np += nt;
    cur.rb += len.x;
    cur.sb += (len.y + 3) & ~3;  // each level's segment list starts 16-byte aligned
    cur.cb += ((len.x >> 2) + 3) & ~3;  // ... and its chunk list
    ++cur.level;
}

// Block-wide exclusive scan of two counters (x, y); *tot receives the sums.
// Every thread calls it; s_w holds 32 int2 of scratch.
__device__ int2 block_excl_scan2(int2 c, int2 *tot, int2 *s_w) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (int)(blockDim.x >> 5);
    int2 v = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int a = __shfl_up_sync(0xffffffffu, v.x, o);
        const int b = __shfl_up_sync(0xffffffffu, v.y, o);
        if (lane >= o) {
            v.x += a;
            v.y += b;
        }
    }
    if (lane == 31) s_w[wid] = v;
    __syncthreads();
    int2 before = make_int2(0, 0), all = make_int2(0, 0);
    for (int j = 0; j < nw; ++j) {
        const int2 t = s_w[j];
        if (j < wid) {
            before.x += t.x;
            before.y += t.y;
        }
        all.x += t.x;
        all.y += t.y;
    }
    __syncthreads();
    *tot = all;
    return make_int2(before.x + v.x - c.x, before.y + v.y - c.y);
}

// The compact form's view of its pairs after the walk, all in shared memory:
// pair p decodes pf[p] at level plv[p] with the constraint whose winning
// bid is still in best[pf[p]] (low 16 bits); level l's pairs are
// lvo[l] .. lvo[l + 1] - 1. px / py / pz / lsb / lcb are scratch for
// format_path (over arrays the walk no longer needs).
struct CompactPairs {
    const uint32_t *best;
    const uint16_t *pf, *plv, *deg;
    const int32_t *cptr4;
    int32_t *lvo, *px, *py, *pz, *lsb, *lcb;
};

// After the walk of the compact form: the payload's records from the pair
// list (levels are contiguous ranges of pairs, so the level-relative offsets
// are differences of prefix sums over the whole list). Per pair x = padded
// row length (its recipe), y = its segments of kRecipeSeg entries, z = 1 when
// it has several (a multi-segment pair takes an accumulator). Writes
// pair_rec, seg_pair, chunk_pair, level_tab and flow_pinfo exactly as
// emit_level does level by level, and fills cur's totals and maxima for
// finish_dpg. Reads only shared memory.
__device__ void format_path(const DpgArgs &a, LevelCursor &cur, const CompactPairs &q, int2 *s_w2,
                            int *s_max) {
    const int tid = threadIdx.x, T = blockDim.x;
    const int32_t P = cur.np, NL = cur.level;
    auto g_of = [&](int32_t p) { return (int32_t)(q.best[q.pf[p]] & 0xffffu); };
    auto sizes = [&](int32_t g, int *x, int *y, int *z) {
        *x = q.cptr4[g + 1] - q.cptr4[g];
        *y = (*x + kRecipeSeg - 1) / kRecipeSeg;
        *z = *y > 1 ? 1 : 0;
    };
    if (tid < 4) s_max[tid] = 0;
    if (tid == 0) q.lvo[NL] = P;
    // A: prefixes in pair order
    const int per = (P + T - 1) / T;
    const int p0 = min(P, tid * per), p1 = min(P, p0 + per);
    int2 cxy = make_int2(0, 0);
    int cz = 0;
    for (int32_t p = p0; p < p1; ++p) {
        int x, y, z;
        sizes(g_of(p), &x, &y, &z);
        cxy.x += x;
        cxy.y += y;
        cz += z;
    }
    int2 txy, tz2;
    int2 oxy = block_excl_scan2(cxy, &txy, s_w2);
    int2 oz = block_excl_scan2(make_int2(cz, 0), &tz2, s_w2);
    for (int32_t p = p0; p < p1; ++p) {
        int x, y, z;
        sizes(g_of(p), &x, &y, &z);
        q.px[p] = oxy.x;
        q.py[p] = oxy.y;
        q.pz[p] = oz.x;
        oxy.x += x;
        oxy.y += y;
        oz.x += z;
    }
    __syncthreads();
    // B: per level its totals, and its segment and chunk list bases (each
    // level's lists start on multiples of 4)
    const int perl = (NL + T - 1) / T;
    const int l0 = min(NL, tid * perl), l1 = min(NL, l0 + perl);
    auto level_sizes = [&](int32_t l, int32_t *first, int32_t *next, int *recipes, int *segs, int *multi) {
        *first = q.lvo[l];
        *next = q.lvo[l + 1];
        const int nx = *next < P ? q.px[*next] : txy.x, ny = *next < P ? q.py[*next] : txy.y;
        const int nz = *next < P ? q.pz[*next] : tz2.x;
        *recipes = nx - q.px[*first];
        *segs = ny - q.py[*first];
        *multi = nz - q.pz[*first];
    };
    int2 c4 = make_int2(0, 0);
    for (int32_t l = l0; l < l1; ++l) {
        int32_t first, next;
        int recipes, segs, multi;
        level_sizes(l, &first, &next, &recipes, &segs, &multi);
        c4.x += (segs + 3) & ~3;
        c4.y += ((recipes >> 2) + 3) & ~3;
        atomicMax(s_max + 0, next - first);
        atomicMax(s_max + 1, recipes);
        atomicMax(s_max + 2, segs);
        atomicMax(s_max + 3, multi);
    }
    int2 t4;
    int2 base = block_excl_scan2(c4, &t4, s_w2);
    for (int32_t l = l0; l < l1; ++l) {
        int32_t first, next;
        int recipes, segs, multi;
        level_sizes(l, &first, &next, &recipes, &segs, &multi);
        a.level_tab[2 * l] = make_int4(first, next - first, base.x, segs);
        a.level_tab[2 * l + 1] = make_int4(base.y, recipes >> 2, 0, 0);
        q.lsb[l] = base.x;
        q.lcb[l] = base.y;
        base.x += (segs + 3) & ~3;
        base.y += ((recipes >> 2) + 3) & ~3;
    }
    __syncthreads();
    // C: the records and the segment / chunk lists
    for (int32_t p = p0; p < p1; ++p) {
        const int32_t l = q.plv[p], first = q.lvo[l], i = p - first;
        const int32_t f = q.pf[p], g = g_of(p);
        int x, y, z;
        sizes(g, &x, &y, &z);
        const int ro = q.px[p] - q.px[first], so = q.py[p] - q.py[first];
        const int mslot = z ? q.pz[p] - q.pz[first] : -1;
        a.pair_rec[2 * (size_t)p] = make_int4(f, g, ro, mslot);
        a.pair_rec[2 * (size_t)p + 1] = make_int4(q.cptr4[g], x, so, y);
        const int32_t sb = q.lsb[l] + so, cb = q.lcb[l] + (ro >> 2);
        for (int k = 0; k < y; ++k) a.seg_pair[sb + k] = i;
        for (int k = 0; k < (x >> 2); ++k) a.chunk_pair[cb + k] = i;
        if (a.flow_pinfo) a.flow_pinfo[p] = (uint32_t)l | ((uint32_t)q.deg[g] << 16);
    }
    __syncthreads();
    cur.maxp = s_max[0];
    cur.maxr = s_max[1];
    cur.maxs = s_max[2];
    cur.maxm = s_max[3];
    cur.sb = t4.x;
    cur.cb = t4.y;
}

// End of the pass: totals, the staged flag, unrecovered flags and list.
__device__ void finish_dpg(const DpgArgs &a, const LevelCursor &cur, const uint8_t *known,
                           int *s_cnt, int *s_cnt_data) {
    if (threadIdx.x == 0) {
        a.level_off[cur.level] = cur.np;
        a.level_tab[2 * cur.level] = make_int4(cur.np, 0, cur.sb, 0);
        a.level_tab[2 * cur.level + 1] = make_int4(cur.cb, 0, 0, 0);
        a.hdr[WS_N_LEVELS] = cur.level;
        a.hdr[WS_N_PAIRS] = cur.np;
        a.hdr[WS_STAGED] = (cur.maxp <= kStagePairs && cur.maxr <= kStageRecipe &&
                            cur.maxs <= kStageSegs && cur.maxm <= kStageMulti &&
                            cur.level <= kStageLevels)
                               ? 1
                               : 0;
        *s_cnt = 0;
        *s_cnt_data = 0;
    }
    for (int32_t l = threadIdx.x; l <= cur.level + 1; l += blockDim.x) a.flow_hist[l] = 0;
    __syncthreads();
    for (int32_t v = threadIdx.x; v < a.k_int; v += blockDim.x) {
        const uint8_t u = known[v] ? 0 : 1;
        a.unrecovered[v] = u;
        if (u) {
            atomicAdd(s_cnt, 1);
            if (v < a.b) a.unrec_list[append_slot(s_cnt_data)] = v;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        *a.n_unrecovered = *s_cnt;
        a.hdr[WS_N_UNREC_DATA] = *s_cnt_data;
        a.hdr[WS_COL_STEPS] = -1;  // no column payload plan for this path (yet)
        for (int i = 0; i <= kFlowHdrList; ++i) a.flow_hdr[i] = 0;  // ... and no dataflow plan
    }
}

// Shared-memory placement of the general form: byte offsets into dynamic
// shared memory, or -1 for the workspace copy.
struct DpgPlace {
    int32_t res, xs, best, known, front, next, touched, cptr, cptr4, vptr, ok;
    int32_t bytes;
};

__device__ __forceinline__ void dpg_body(const DpgArgs &a, const DpgPlace &pl) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int4 s_warp4[2][32];
    __shared__ int4 s_len;
    __shared__ int s_nf, s_nt, s_nnext, s_cnt, s_cnt_data;

    const int tid = threadIdx.x, T = blockDim.x;
    const int32_t K = a.k_int, G = a.n_con;

    int32_t *res = place(smem, pl.res, a.res);
    int32_t *xs = place(smem, pl.xs, a.xs);
    unsigned long long *best = place(smem, pl.best, a.best);
    uint8_t *known = place(smem, pl.known, a.known);
    int32_t *front = place(smem, pl.front, a.front_a);
    int32_t *next = place(smem, pl.next, a.front_b);
    int32_t *touched = place(smem, pl.touched, a.touched);
    const int32_t *cptr = place(smem, pl.cptr, const_cast<int32_t *>(a.con_ptr));
    const int32_t *cptr4 = place(smem, pl.cptr4, const_cast<int32_t *>(a.con_ptr4));
    const int32_t *vptr = place(smem, pl.vptr, const_cast<int32_t *>(a.var_ptr));
    uint8_t *ok = pl.ok >= 0 ? smem + pl.ok : nullptr;

    if (tid == 0) a.hdr[WS_STATUS] = FS_OK;
    if (pl.cptr >= 0)
        for (int32_t g = tid; g <= G; g += T)
            reinterpret_cast<int32_t *>(smem + pl.cptr)[g] = __ldg(a.con_ptr + g);
    if (pl.cptr4 >= 0)
        for (int32_t g = tid; g <= G; g += T)
            reinterpret_cast<int32_t *>(smem + pl.cptr4)[g] = __ldg(a.con_ptr4 + g);
    if (pl.vptr >= 0)
        for (int32_t v = tid; v <= K; v += T)
            reinterpret_cast<int32_t *>(smem + pl.vptr)[v] = __ldg(a.var_ptr + v);
    if (ok)
        for (int32_t g = tid; g < G; g += T) ok[g] = (g < a.n) ? (a.erased[g] == 0) : 1;
    for (int32_t v = tid; v < K; v += T) {
        known[v] = 0;
        best[v] = kEmpty;
    }
    for (int32_t g = tid; g < G; g += T) {
        res[g] = __ldg(a.con_ptr + g + 1) - __ldg(a.con_ptr + g);
        xs[g] = __ldg(a.con_xs + g);
    }
    int stage = a.two_pass ? 0 : -1;
    if (tid == 0) s_nf = 0;
    __syncthreads();
    for (int32_t g = tid; g < G; g += T)
        if (usable(a, ok, g, stage) && res[g] == 1) front[append_slot(&s_nf)] = g;
    __syncthreads();

    LevelCursor cur;
    for (;;) {
        const int nf = s_nf;
        if (tid == 0) {
            s_nt = 0;
            s_nnext = 0;
        }
        __syncthreads();
        // A: frontier constraints bid for their single unknown
        for (int i = tid; i < nf; i += T) {
            const int32_t g = front[i];
            if (res[g] != 1) continue;  // its unknown was decoded by another constraint
            const int32_t f = xs[g];
            const unsigned long long key =
                ((unsigned long long)(cptr[g + 1] - cptr[g]) << 32) | (uint32_t)g;
            if (atomicMin(best + f, key) == kEmpty) touched[append_slot(&s_nt)] = f;
        }
        __syncthreads();
        const int nt = s_nt;
        if (nt == 0) {
            if (stage != 0) break;
            // two-pass: the coded rows reached their fixpoint; peel the checks
            stage = 1;
            if (tid == 0) s_nf = 0;
            __syncthreads();
            for (int32_t g = a.n + tid; g < G; g += T)
                if (res[g] == 1) front[append_slot(&s_nf)] = g;
            __syncthreads();
            continue;
        }
        // B: pairs of the level
        emit_level(
            a, cur, nt,
            [&](int i, int32_t *f, int32_t *g) {
                *f = touched[i];
                *g = (int32_t)(best[*f] & 0xffffffffull);
            },
            cptr4, s_warp4, &s_len);
        for (int i = tid; i < nt; i += T) {
            const int32_t f = touched[i];
            best[f] = kEmpty;
            known[f] = 1;
        }
        __syncthreads();
        const int4 len = s_len;
        // C: one thread per pair updates the constraints containing its symbol
        for (int i = tid; i < nt; i += T) {
            const int32_t f = touched[i];
            const int32_t v1 = vptr[f + 1];
            for (int32_t e = vptr[f]; e < v1; ++e) {
                const int32_t c = __ldg(a.var_idx + e);
                atomicXor(xs + c, f);
                if (atomicSub(res + c, 1) == 2 && usable(a, ok, c, stage))
                    next[append_slot(&s_nnext)] = c;
            }
        }
        __syncthreads();
        if (tid == 0) s_nf = s_nnext;
        advance(cur, nt, len);
        int32_t *tmp = front;
        front = next;
        next = tmp;
        __syncthreads();
    }
    finish_dpg(a, cur, known, &s_cnt, &s_cnt_data);
}

__global__ void __launch_bounds__(kDpgThreads, 1) k_dpg(DpgArgs a, DpgPlace pl) { dpg_body(a, pl); }

// one CTA per stripe of a batch
__global__ void __launch_bounds__(kDpgThreads, 1) k_dpg_batch(const DpgArgs *as, const DpgPlace *ps) {
    const DpgArgs a = as[blockIdx.x];
    const DpgPlace pl = ps[blockIdx.x];
    dpg_body(a, pl);
}

DpgPlace plan_dpg(const fs_code *c) {
    DpgPlace p;
    const int64_t K = c->k_int + 1, G = c->n_con + 1;
    const int64_t budget = (int64_t)c->smem_optin - 1024;  // static shared memory of k_dpg
    int64_t o = 0;
    auto take = [&](int64_t bytes) {
        const int64_t at = o;
        o = (o + bytes + 15) & ~(int64_t)15;
        return (int32_t)at;
    };
    // the peel state: all in shared memory or all in the workspace
    const int64_t state = 8 * K + 4 * G * 4 + 4 * K + K + 16 * 8;
    if (state <= budget) {
        p.best = take(8 * K);
        p.res = take(4 * G);
        p.xs = take(4 * G);
        p.front = take(4 * G);
        p.next = take(4 * G);
        p.touched = take(4 * K);
        p.known = take(K);
    } else {
        p.best = p.res = p.xs = p.front = p.next = p.touched = p.known = -1;
    }
    // graph row pointers and survival flags, each where room is left
    p.cptr = (o + 4 * G <= budget) ? take(4 * G) : -1;
    p.cptr4 = (o + 4 * G <= budget) ? take(4 * G) : -1;
    p.vptr = (o + 4 * K <= budget) ? take(4 * K) : -1;
    p.ok = (o + G <= budget) ? take(G) : -1;
    p.bytes = (int32_t)o;
    return p;
}

struct DpgCompactPlace {
    // through the walk and the formatting
    int32_t best, cptr4, deg, known, pf, plv, lvo;
    // the walk only
    int32_t pk, vptr, front, vidx, ok;
    // the formatting only, over the walk's arrays
    int32_t px, py, pz, lsb, lcb;
    int32_t bytes;
};

__device__ __forceinline__ void dpg_compact_body(const DpgArgs &a, const DpgCompactPlace &pl) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int2 s_w2[32];
    __shared__ int s_max[4];
    // symbols of the next level, by level parity (a level reads one list
    // while its step C fills the other)
    __shared__ int s_nt[2], s_cnt, s_cnt_data;
    constexpr uint32_t kE = 0xffffffffu;

    const int tid = threadIdx.x, T = blockDim.x;
    const int32_t K = a.k_int, G = a.n_con;
    uint32_t *best = reinterpret_cast<uint32_t *>(smem + pl.best);
    uint32_t *pk = reinterpret_cast<uint32_t *>(smem + pl.pk);  // sum << 16 | res
    uint16_t *touched2 = reinterpret_cast<uint16_t *>(smem + pl.front);  // [2][K + 1]
    uint8_t *known = smem + pl.known;
    int32_t *cptr4 = reinterpret_cast<int32_t *>(smem + pl.cptr4);
    int32_t *vptr = reinterpret_cast<int32_t *>(smem + pl.vptr);
    uint16_t *vidx = reinterpret_cast<uint16_t *>(smem + pl.vidx);
    uint16_t *deg = reinterpret_cast<uint16_t *>(smem + pl.deg);
    uint8_t *ok = smem + pl.ok;
    uint16_t *pf = reinterpret_cast<uint16_t *>(smem + pl.pf);    // [K + 1] f of pair p
    uint16_t *plv = reinterpret_cast<uint16_t *>(smem + pl.plv);  // [K + 1] level of pair p
    int32_t *lvo = reinterpret_cast<int32_t *>(smem + pl.lvo);    // [K + 2] first pair of level l

    // Constraint c, left with the one unknown f, bids key = (degree, c) for
    // it; the first bid for f lists f for the level.
    auto bid = [&](int32_t c, uint32_t f, int list) {
        const uint32_t key = ((uint32_t)deg[c] << 16) | (uint32_t)c;
        if (atomicMin(best + f, key) == kE)
            touched2[(size_t)list * (K + 1) + append_slot(&s_nt[list])] = (uint16_t)f;
    };

    if (tid == 0) a.hdr[WS_STATUS] = FS_OK;
    for (int32_t g = tid; g <= G; g += T) cptr4[g] = __ldg(a.con_ptr4 + g);
    for (int32_t v = tid; v <= K; v += T) vptr[v] = __ldg(a.var_ptr + v);
    const int32_t e_con = __ldg(a.var_ptr + K);
    for (int32_t e = tid; e < e_con; e += T) vidx[e] = (uint16_t)__ldg(a.var_idx + e);
    for (int32_t v = tid; v < K; v += T) {
        known[v] = 0;
        best[v] = kE;
    }
    for (int32_t g = tid; g < G; g += T) {
        const uint32_t d = (uint32_t)(__ldg(a.con_ptr + g + 1) - __ldg(a.con_ptr + g));
        deg[g] = (uint16_t)d;
        pk[g] = ((uint32_t)__ldg(a.con_sum + g) << 16) | d;
        ok[g] = (g < a.n) ? (a.erased[g] == 0) : 1;
    }
    int stage = a.two_pass ? 0 : -1;
    if (tid == 0) s_nt[0] = s_nt[1] = 0;
    __syncthreads();
    for (int32_t g = tid; g < G; g += T)
        if (usable(a, ok, g, stage) && (pk[g] & 0xffffu) == 1) bid(g, pk[g] >> 16, 0);
    __syncthreads();

    LevelCursor cur;
    for (;;) {
        const int par = cur.level & 1;
        const int nt = s_nt[par];
        const uint16_t *touched = touched2 + (size_t)par * (K + 1);
        if (nt == 0) {
            if (stage != 0) break;
            // two-pass: the coded rows reached their fixpoint; peel the checks
            // (those left with one unknown during the first stage bid now)
            stage = 1;
            __syncthreads();  // every thread has read the empty count
            for (int32_t g = a.n + tid; g < G; g += T)
                if ((pk[g] & 0xffffu) == 1) bid(g, pk[g] >> 16, par);
            __syncthreads();
            continue;
        }
        // B: pairs of the level, kept in shared memory (f and level per pair;
        // g stays in f's winning bid: a decoded symbol gets no further bid)
        // for the payload's records, formatted after the walk; f's level goes
        // to the dataflow plan
        for (int i = tid; i < nt; i += T) {
            const int32_t f = touched[i];
            const int32_t g = (int32_t)(best[f] & 0xffffu);
            const int32_t p = cur.np + i;
            a.pair_f[p] = f;
            a.pair_g[p] = g;
            a.flow_lvl[f] = (uint16_t)cur.level;
            pf[p] = (uint16_t)f;
            plv[p] = (uint16_t)cur.level;
            known[f] = 1;
        }
        if (tid == 0) {
            a.level_off[cur.level] = cur.np;
            lvo[cur.level] = cur.np;
            s_nt[par ^ 1] = 0;  // the list the next level's bids fill
        }
        __syncthreads();
        // C (and step A of the next level): S threads per pair, thread j of
        // a pair takes its adjacency slots j, j + S, ... and removes f from
        // each constraint c there; the update that leaves c one unknown bids
        // for it, unless that unknown is decoded in this level too
        auto update = [&](int32_t c, uint32_t f, uint32_t old) {
            const uint32_t res = old & 0xffffu;
            // f is the (deg - res)-th member of c to be recovered
            if (a.flow_list && deg[c] >= kListDeg)
                a.flow_list[cptr4[c] + (int)deg[c] - (int)res] = (uint16_t)f;
            if (res == 2) {
                const uint32_t last = ((old >> 16) - f) & 0xffffu;
                if (!known[last] && usable(a, ok, c, stage)) bid(c, last, par ^ 1);
            }
        };
        // S = 2^k threads per pair, the largest with S * nt <= T (T is a
        // power of two, so S divides T and the rounds of R = T / S pairs
        // give every slot to exactly one thread); uniform, no division
        const int k = max(0, (31 - __clz(T)) - (32 - __clz(nt - 1)));
        const int S = 1 << k, R = T >> k;
        for (int i = tid >> k; i < nt; i += R) {
            const uint32_t f = touched[i];
            const uint32_t dec = 0u - ((f << 16) + 1u);
            const int32_t e1 = vptr[f + 1];
            // two slots per round trip: both atomics in flight before either
            // result is tested
            for (int32_t e = vptr[f] + (tid & (S - 1)); e < e1; e += 2 * S) {
                const int32_t c0 = vidx[e];
                const bool two = e + S < e1;
                const int32_t c1 = two ? (int32_t)vidx[e + S] : c0;
                const uint32_t o0 = atomicAdd(pk + c0, dec);
                const uint32_t o1 = two ? atomicAdd(pk + c1, dec) : 0u;
                update(c0, f, o0);
                if (two) update(c1, f, o1);
            }
        }
        __syncthreads();
        cur.np += nt;
        ++cur.level;
    }
    CompactPairs q;
    q.best = best;
    q.pf = pf;
    q.plv = plv;
    q.deg = deg;
    q.cptr4 = cptr4;
    q.lvo = lvo;
    q.px = reinterpret_cast<int32_t *>(smem + pl.px);
    q.py = reinterpret_cast<int32_t *>(smem + pl.py);
    q.pz = reinterpret_cast<int32_t *>(smem + pl.pz);
    q.lsb = reinterpret_cast<int32_t *>(smem + pl.lsb);
    q.lcb = reinterpret_cast<int32_t *>(smem + pl.lcb);
    format_path(a, cur, q, s_w2, s_max);
    finish_dpg(a, cur, known, &s_cnt, &s_cnt_data);
    if (tid == 0 && a.flow_list) a.flow_hdr[kFlowHdrList] = 1;  // after finish_dpg's clear
}

__global__ void __launch_bounds__(kDpgThreads, 1) k_dpg_compact(DpgArgs a, DpgCompactPlace pl) {
    dpg_compact_body(a, pl);
}

// one CTA per stripe of a batch
__global__ void __launch_bounds__(kDpgThreads, 1)
    k_dpg_compact_batch(const DpgArgs *as, const DpgCompactPlace *ps) {
    const DpgArgs a = as[blockIdx.x];
    const DpgCompactPlace pl = ps[blockIdx.x];
    dpg_compact_body(a, pl);
}

// Shared-memory layout of k_dpg_compact, or bytes = -1 when the code does not
// qualify (sizes beyond 16-bit indices, or more than the shared memory).
DpgCompactPlace plan_dpg_compact(const fs_code *c) {
    DpgCompactPlace p;
    p.bytes = -1;
    const int64_t K = c->k_int, G = c->n_con;
    // 16-bit indices; degrees below 2^16 (the res field of the packed word)
    if (K > 65536 || G > 65536 || c->max_con_deg > 65535) return p;
    int64_t o = 0;
    auto take = [&](int64_t bytes) {
        const int64_t at = o;
        o = (o + bytes + 15) & ~(int64_t)15;
        return (int32_t)at;
    };
    // through the walk and the formatting (levels <= pairs <= K)
    p.best = take(4 * (K + 1));
    p.cptr4 = take(4 * (G + 1));
    p.deg = take(2 * (G + 1));
    p.known = take(K + 1);
    p.pf = take(2 * (K + 1));
    p.plv = take(2 * (K + 1));
    p.lvo = take(4 * (K + 2));
    const int64_t live = o;
    // the walk only
    p.pk = take(4 * (G + 1));
    p.vptr = take(4 * (K + 1));
    p.front = take(2 * 2 * (K + 1));  // the two symbol lists
    p.vidx = take(2 * (c->e_con + 1));
    p.ok = take(G + 1);
    const int64_t walk = o;
    // the formatting only, over the walk's arrays
    o = live;
    p.px = take(4 * (K + 1));
    p.py = take(4 * (K + 1));
    p.pz = take(4 * (K + 1));
    p.lsb = take(4 * (K + 2));
    p.lcb = take(4 * (K + 2));
    o = std::max(o, walk);
    if (o > (int64_t)c->smem_optin - 1024) return p;
    p.bytes = (int32_t)o;
    return p;
}

// ---------------------------------------------------------------------------
// payload

struct PeelArgs {
    const uint4 *coded;
    uint4 *data;    // intermediates v < b
    uint4 *parity;  // intermediates v >= b (workspace)
    const int32_t *con_idx4, *seg_pair, *chunk_pair, *unrec_list, *hdr;
    const int4 *pair_rec, *level_tab;
    int32_t b, n;
    int64_t tw;
    int32_t L;  // words of every block per CTA
    int32_t hints;  // 1: gathered / recovered blocks evict-last, coded payloads evict-first
    int32_t *status;
    // dataflow walk (flow_body, on the plan of k_flow_units / k_flow_place)
    // when 1, key walk (keys_body, on the plan of k_key_plan) when 2
    int32_t flow;
    int32_t k_int;
    const int32_t *fhdr, *fslot;
    const uint2 *funits;
    const uint4 *fbatch;
    const uint16_t *fmem;
    const int4 *fktab;  // the key walk's table (keys_body)
};

__device__ __forceinline__ void xor4(uint4 &a, const uint4 &b) {
    a.x ^= b.x;
    a.y ^= b.y;
    a.z ^= b.z;
    a.w ^= b.w;
}

__device__ __forceinline__ uint4 *block_ptr(const PeelArgs &a, int32_t v) {
    return (v < a.b) ? a.data + (int64_t)v * a.tw : a.parity + (int64_t)(v - a.b) * a.tw;
}

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

// Waits for the phase with the given parity; false after `rounds` x
// kWaitLimit polls.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, int rounds = 1) {
    const uint32_t addr = smem_addr(bar);
    for (long long i = 0; i < kWaitLimit * rounds; ++i) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(addr), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// Bulk copy of `bytes` (a multiple of 16) from global to shared memory,
// completing on bar.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes,
                                         uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::
            "r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ void xor_shared(uint4 *d, const uint4 &v) {
    uint32_t *w = reinterpret_cast<uint32_t *>(d);
    atomicXor(w + 0, v.x);
    atomicXor(w + 1, v.y);
    atomicXor(w + 2, v.z);
    atomicXor(w + 3, v.w);
}

// Levels read straight from global memory (used when a level does not fit
// the shared-memory stages): one thread per (pair, word).
__device__ void peel_direct(const PeelArgs &a, int64_t w0, int lanes) {
    const int32_t n_levels = a.hdr[WS_N_LEVELS];
    for (int32_t l = 0; l < n_levels; ++l) {
        const int4 lt = a.level_tab[2 * l];
        const int32_t items = lt.y * lanes;
        for (int32_t it = threadIdx.x; it < items; it += blockDim.x) {
            const int32_t q = it / lanes, lane = it - q * lanes;
            const int4 r0 = a.pair_rec[2 * (size_t)(lt.x + q)];
            const int4 r1 = a.pair_rec[2 * (size_t)(lt.x + q) + 1];
            const int32_t f = r0.x, g = r0.y;
            const int64_t w = w0 + lane;
            uint4 acc = make_uint4(0, 0, 0, 0);
            if (g < a.n) acc = __ldg(a.coded + (int64_t)g * a.tw + w);
            for (int32_t r = 0; r < r1.y; ++r) {
                const int32_t h = __ldg(a.con_idx4 + r1.x + r);
                if (h >= 0 && h != f) xor4(acc, block_ptr(a, h)[w]);
            }
            block_ptr(a, f)[w] = acc;
        }
        __syncthreads();
    }
}

// One thread: bulk copies of level l's pair records, segment list and chunk
// list into their slots (one mbarrier phase).
__device__ __forceinline__ void issue_pairs(const PeelArgs &a, const int4 *ltab, int l,
                                            int32_t *pairs_slot, int32_t *segs_slot,
                                            int32_t *chunks_slot, uint64_t *bar) {
    const int4 lt = ltab[2 * l], lc = ltab[2 * l + 1];
    const uint32_t pb = (uint32_t)lt.y * kRec * 4;
    const uint32_t sbytes = (uint32_t)((lt.w + 3) & ~3) * 4;
    const uint32_t cbytes = (uint32_t)((lc.y + 3) & ~3) * 4;
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    mbar_expect_tx(bar, pb + sbytes + cbytes);
    bulk_g2s(pairs_slot, a.pair_rec + 2 * (size_t)lt.x, pb, bar);
    if (sbytes) bulk_g2s(segs_slot, a.seg_pair + lt.z, sbytes, bar);
    if (cbytes) bulk_g2s(chunks_slot, a.chunk_pair + lc.x, cbytes, bar);
}

__device__ __forceinline__ void cp_async16(void *sdst, const void *gsrc) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_addr(sdst)), "l"(gsrc)
                 : "memory");
}

// All threads: level l's recipes (its padded graph rows, 16 bytes per copy)
// into rows_slot from its staged pair records and chunk list, and an L2
// prefetch of its coded payload slices.
__device__ __forceinline__ void stage_rows(const PeelArgs &a, const int4 *ltab, int l,
                                           const int32_t *prec, const int32_t *chunks,
                                           int32_t *rows_slot, int64_t w0, int lanes) {
    const int np = ltab[2 * l].y, nc = ltab[2 * l + 1].y;
    for (int c = threadIdx.x; c < nc; c += blockDim.x) {
        const int32_t *r = prec + (size_t)chunks[c] * kRec;
        cp_async16(rows_slot + 4 * c, a.con_idx4 + r[4] + (4 * c - r[2]));
    }
    const int lines = (lanes * 16 + 127) >> 7;
    for (int i = threadIdx.x; i < np * lines; i += blockDim.x) {
        const int q = i / lines, k = i - q * lines;
        const int32_t g = prec[(size_t)q * kRec + 1];
        if (g < a.n) {
            const char *p = reinterpret_cast<const char *>(a.coded + (int64_t)g * a.tw + w0) + 128 * k;
            asm volatile("prefetch.global.L2 [%0];\n" ::"l"(p));
        }
    }
}

__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}

__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// kHints: L2 eviction hints on the gathers and stores (FS_TUNE_L2_HINTS), a
// template parameter so the default path carries no branch and no policy
// registers for them (the key walk measured 10% faster without them).
template <bool kHints>
__device__ __forceinline__ void peel_body(const PeelArgs &a, int64_t slice) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ __align__(8) uint64_t mb_pairs[3];
    __shared__ int s_ok;
    const int L = a.L;
    const int64_t w0 = slice * L;
    const int lanes = (int)min((int64_t)L, a.tw - w0);
    const int32_t nl = a.hdr[WS_N_LEVELS];

    if (!a.hdr[WS_STAGED]) {
        peel_direct(a, w0, lanes);
    } else {
        int4 *ltab = reinterpret_cast<int4 *>(smem);                  // [2 (levels + 1)]
        int32_t *pairs = reinterpret_cast<int32_t *>(ltab + 2 * (kStageLevels + 1));  // [3][P*kRec]
        int32_t *segs = pairs + 3 * kStagePairs * kRec;                // [3][S]
        int32_t *chunks = segs + 3 * kStageSegs;                       // [3][R / 4]
        int32_t *rows = chunks + 3 * (kStageRecipe / 4);               // [2][R]
        uint4 *accs = reinterpret_cast<uint4 *>(rows + 2 * kStageRecipe);  // [kStageMulti][L]
        // segments of each (multi-segment pair, word) summed so far: the
        // segment that completes a sum writes it out
        int32_t *done = reinterpret_cast<int32_t *>(accs + (size_t)kStageMulti * L);  // [kStageMulti][L]
        for (int i = threadIdx.x; i < 2 * (nl + 1); i += blockDim.x) ltab[i] = a.level_tab[i];
        for (int i = threadIdx.x; i < kStageMulti * L; i += blockDim.x)
            accs[i] = make_uint4(0, 0, 0, 0);
        for (int i = threadIdx.x; i < kStageMulti * L; i += blockDim.x) done[i] = 0;
        if (threadIdx.x == 0) {
            for (int k = 0; k < 3; ++k) mbar_init(&mb_pairs[k]);
            asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
            s_ok = 1;
        }
        __syncthreads();
        // prologue: pairs of levels 0 and 1 (bulk), rows of level 0
        if (threadIdx.x == 0) {
            for (int l = 0; l < 2 && l < nl; ++l)
                issue_pairs(a, ltab, l, pairs + l * kStagePairs * kRec, segs + l * kStageSegs,
                            chunks + l * (kStageRecipe / 4), &mb_pairs[l]);
            s_ok = (nl == 0 || mbar_wait(&mb_pairs[0], 0)) ? 1 : 0;
            if (!s_ok) {
                // give up, but first wait longer (8 bounds) for the copies of
                // levels 0 and 1 still in flight
                mbar_wait(&mb_pairs[0], 0, 8);
                if (nl > 1) mbar_wait(&mb_pairs[1], 0, 8);
            }
        }
        __syncthreads();
        if (s_ok && nl > 0) stage_rows(a, ltab, 0, pairs, chunks, rows, w0, lanes);
        cp_async_commit();
        // thread 0 alone reads and writes fail (a failed prologue stops the
        // walk at its first level); every thread reads s_ok only after the
        // barrier that follows thread 0's write
        int fail = (threadIdx.x == 0 && !s_ok) ? 1 : 0;
        // every thread keeps one word k of the slice and takes segments srow,
        // srow + nrows, ... of each level (no division per item); counted from
        // the highest thread, so the lowest blockDim.x mod lanes threads take
        // none and the staging below (thread 0's bulk copies, the low
        // threads' row copies) overlaps the gathers
        const int rt0 = (int)blockDim.x - 1 - (int)threadIdx.x;
        const int k = rt0 % lanes, srow = rt0 / lanes, nrows = (int)blockDim.x / lanes;
        for (int32_t l = 0; l < nl; ++l) {
            const int ps = l % 3, rslot = l & 1;
            // level l's pairs (bulk) and rows (this thread's copies) are in;
            // so are level l+1's pairs, which step 2 reads
            cp_async_wait_all();
            if (threadIdx.x == 0 && fail) s_ok = 0;
            if (threadIdx.x == 0 && !fail) {
                const uint32_t ph0 = (uint32_t)((l / 3) & 1), ph1 = (uint32_t)(((l + 1) / 3) & 1);
                const bool in0 = mbar_wait(&mb_pairs[ps], ph0);
                const bool in1 = in0 && (l + 1 >= nl || mbar_wait(&mb_pairs[(l + 1) % 3], ph1));
                s_ok = in1 ? 1 : 0;
                if (!in1) {
                    // give up, but first wait longer (8 bounds) for each copy not
                    // yet seen to land (levels l and l+1; l+2's is not issued
                    // yet); only if that wait expires too does the CTA leave with
                    // a copy possibly still landing in its shared memory
                    if (!in0) mbar_wait(&mb_pairs[ps], ph0, 8);
                    if (l + 1 < nl) mbar_wait(&mb_pairs[(l + 1) % 3], ph1, 8);
                }
            }
            __syncthreads();  // level l-1 is written; level l's stages are in
            if (!s_ok) break;
            const int32_t *pc = pairs + ps * kStagePairs * kRec;
            const int32_t *sp = segs + ps * kStageSegs;
            const int32_t *hs = rows + rslot * kStageRecipe;
            // stage ahead into the slots level l-1 used: pairs of l+2 (bulk),
            // rows of l+1 (every thread)
            if (threadIdx.x == 0 && l + 2 < nl)
                issue_pairs(a, ltab, l + 2, pairs + ((l + 2) % 3) * kStagePairs * kRec,
                            segs + ((l + 2) % 3) * kStageSegs,
                            chunks + ((l + 2) % 3) * (kStageRecipe / 4), &mb_pairs[(l + 2) % 3]);
            if (l + 1 < nl)
                stage_rows(a, ltab, l + 1, pairs + ((l + 1) % 3) * kStagePairs * kRec,
                           chunks + ((l + 1) % 3) * (kStageRecipe / 4),
                           rows + ((l + 1) & 1) * kStageRecipe, w0, lanes);
            cp_async_commit();
            const int ns = ltab[2 * l].w;
            const uint64_t pol_last = kHints ? l2_policy_last() : 0, pol_first = kHints ? l2_policy_first() : 0;
            // every (segment, word): one gather of at most kRecipeSeg blocks
            for (int s = (srow < nrows ? srow : ns); s < ns; s += nrows) {
                const int32_t *rec = pc + (size_t)sp[s] * kRec;
                const int32_t f = rec[0], g = rec[1], slot = rec[3];
                const int sidx = s - rec[6];
                const int32_t rs = rec[2] + sidx * kRecipeSeg;
                const int32_t cnt = min(kRecipeSeg, rec[2] + rec[5] - rs);
                const int64_t w = w0 + k;
                uint4 acc = make_uint4(0, 0, 0, 0);
                if (sidx == 0 && g < a.n) {
                    const uint4 *src = a.coded + (int64_t)g * a.tw + w;
                    acc = kHints ? ld_nc_hint(src, pol_first) : src[0];
                }
                uint4 x[kRecipeSeg];  // every load of the segment in flight at once
#pragma unroll
                for (int j = 0; j < kRecipeSeg; ++j) {
                    const int32_t h = j < cnt ? hs[rs + j] : -1;
                    x[j] = make_uint4(0, 0, 0, 0);
                    if (h >= 0 && h != f) {
                        const uint4 *src = block_ptr(a, h) + w;
                        x[j] = kHints ? ld_hint(src, pol_last) : src[0];
                    }
                }
#pragma unroll
                for (int j = 0; j < kRecipeSeg; ++j) xor4(acc, x[j]);
                if (slot < 0) {
                    uint4 *dst = block_ptr(a, f) + w;
                    if (kHints) st_hint(dst, acc, pol_last);
                    else dst[0] = acc;
                } else {  // one of several segments: combine in shared memory
                    uint4 *sa = accs + slot * L + k;
                    xor_shared(sa, acc);
                    __threadfence_block();  // the sum holds this segment before it counts
                    if (atomicAdd(&done[slot * L + k], 1) == rec[7] - 1) {
                        // the last segment of this word: every other one is in
                        __threadfence_block();
                        block_ptr(a, f)[w] = sa[0];
                        sa[0] = make_uint4(0, 0, 0, 0);
                        done[slot * L + k] = 0;  // the slot is free for a later level
                    }
                }
            }
        }
        cp_async_wait_all();
        __syncthreads();
        if (threadIdx.x == 0 && !s_ok) atomicExch(a.status, FS_ERR_TIMEOUT);
    }
    // unrecovered data blocks read as zero
    const int32_t nu = a.hdr[WS_N_UNREC_DATA];
    for (int32_t it = threadIdx.x; it < nu * lanes; it += blockDim.x) {
        const int32_t q = it / lanes, lane = it - q * lanes;
        a.data[(int64_t)a.unrec_list[q] * a.tw + w0 + lane] = make_uint4(0, 0, 0, 0);
    }
}

// ---------------------------------------------------------------------------
// dataflow payload
//
// The level walk above waits for a whole level at a barrier, and its gathers
// reach far back: a decoder of degree 19, or a precode check with ~97
// members, reads blocks recovered dozens of levels earlier, which L2 no
// longer holds (at the precoded stripe 45% of the coded-row gathers and 75%
// of the check gathers reach back past more than 62 MB of newer output).
// The dataflow walk gathers the members of such heavy pairs while they are
// fresh, and packs small gathers into full rounds of loads. Its plan:
//   - a light pair (at most 8 loads: c_g when g is a coded row, then the
//     other members of g) is one whole unit; its key is its level;
//   - a heavy pair has its members sorted by the level that recovered them
//     (up to kFlowSortMax) and cut into segments of at least 8 loads (the
//     first one starting with c_g); a segment's key is 1 + the highest
//     level among its members, so it can run as soon as they exist:
//       * a precode check sums its segments into a shared-memory
//         accumulator of its own (kFlowSlots of them); the segment that
//         completes the count writes x_f;
//       * any other heavy pair chains its segments through x_f itself:
//         segment r > 0 loads the partial sum the previous one wrote, adds
//         its members and writes it back. Keys are made non-decreasing and
//         segments with equal keys merged, so the keys of a chain rise
//         strictly;
//   - units are put in key order and consecutive units of one key packed
//     into batches of at most 8 loads (one round of loads in flight).
// Every unit reads only pairs whose units all have smaller keys (a pair of
// level l has its members in levels below l, hence keys at most l), and a
// chain segment also reads its predecessor, which has a smaller key; units
// of one key never read each other. In the payload (flow_body) warp w takes
// batches w, w + 32, ... and waits, on shared-memory ready flags, for what
// each batch reads. The batch at the lowest position not yet done reads only
// finished work and its warp is working on it (a warp takes its batches in
// order), so the walk always advances; every wait is bounded all the same
// and an expired wait stops the CTA with FS_ERR_TIMEOUT. Each (pair, word) of
// the result is the XOR of the same terms as in the level walk.

constexpr int kFlowSeg = 8;           // loads of one segment (at least); of one batch (at most)
constexpr int kFlowSortMax = 256;     // heavy members sorted by level up to this count
constexpr int kFlowChain = 120;       // chain segments of one pair at most
constexpr int kFlowMaxDeg = 4000;     // largest constraint degree (12-bit load counts)
constexpr int kFlowUnitThreads = 256;
constexpr long long kFlowWaitLimit = 1ll << 22;  // polls of a ready flag

// unit record: x = f | hasg << 16 | kind << 17 | aux << 19 | last << 27,
//              y = first load | member loads << 20
// (k_flow_units writes the first load's place in flow_raw, k_flow_place its
// place in flow_mem)
enum { kUnitWhole = 0, kUnitSlot = 1, kUnitChain = 2 };
constexpr uint32_t kMoffMask = (1u << 20) - 1;
constexpr uint8_t kReadyFinal = 0x80;  // ready flag: x_f is final; low bits: chain segments done
enum { kFhUnits = 0, kFhLoads = 1, kFhOk = 2, kFhSlots = 3, kFhBatches = 4, kFhSlotCtr = 5,
       kFhOverflow = 6, kFhKeyFit = 7 };
// the key walk's shared-memory stages (one key each): units (from an even
// index) and loads (from a multiple of 8), and the key table
constexpr int kKeyUnits = 1024;
constexpr int kKeyMem = 4096;
constexpr int kKeyMax = 1024;  // 80 KiB of stages in all: the rest of the SM's
                               // shared memory serves as L1 for the gathers

// Loads of a unit: c_g, the chain's partial sum, its members; a unit with
// none (a check of no members decoding its parity: the zero block) keeps one
// slot that loads nothing.
__device__ __forceinline__ int unit_slots(uint2 r) {
    const int hasg = (int)((r.x >> 16) & 1u), kind = (int)((r.x >> 17) & 3u);
    const int aux = (int)((r.x >> 19) & 0xffu);
    const int sl = hasg + ((kind == kUnitChain && aux > 0) ? 1 : 0) + (int)(r.y >> 20);
    return sl > 0 ? sl : 1;
}

struct FlowUnitArgs {
    const int32_t *hdr;
    const int4 *pair_rec;
    const int32_t *con_ptr, *con_idx4;
    const uint16_t *lvl;
    int32_t n, slot_cap;
    int32_t *fhdr, *hist, *ucnt, *slot_nseg;
    uint2 *uarea;
    uint16_t *ukey, *raw;
};

// Every pair of the path into units, one warp per pair (a light pair is
// done by lane 0; a heavy one by the whole warp, which sorts its members).
__global__ void __launch_bounds__(kFlowUnitThreads) k_flow_units(FlowUnitArgs a) {
    __shared__ int s_key[kFlowUnitThreads / 32][128];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int32_t P = a.hdr[WS_N_PAIRS], NL = a.hdr[WS_N_LEVELS];
    const int32_t p = blockIdx.x * (kFlowUnitThreads / 32) + wid;
    if (p >= P) return;  // whole warps leave; no block barrier below
    int *skey = s_key[wid];
    {
        const int4 r0 = a.pair_rec[2 * (size_t)p];
        const int32_t f = r0.x, g = r0.y, e4 = a.pair_rec[2 * (size_t)p + 1].x;
        const int32_t deg = __ldg(a.con_ptr + g + 1) - __ldg(a.con_ptr + g);
        const int hasg = g < a.n ? 1 : 0, loads = hasg + deg - 1;
        if (loads <= kFlowSeg) {
            // light: its loads in row order (g first) and one whole unit
            if (lane == 0) {
                int w = e4;
                if (hasg) a.raw[w++] = (uint16_t)g;
                const int4 *row = reinterpret_cast<const int4 *>(a.con_idx4 + e4);
                int4 q4[3];
#pragma unroll
                for (int i = 0; i < 3; ++i) q4[i] = 4 * i < deg ? __ldg(row + i) : make_int4(-1, -1, -1, -1);
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    const int32_t hv[4] = {q4[i].x, q4[i].y, q4[i].z, q4[i].w};
#pragma unroll
                    for (int t = 0; t < 4; ++t)
                        if (4 * i + t < deg && hv[t] != f) a.raw[w++] = (uint16_t)hv[t];
                }
                const int key = min((int)a.lvl[f], NL);
                a.uarea[e4 >> 2] = make_uint2((uint32_t)f | ((uint32_t)hasg << 16),
                                              (uint32_t)e4 | ((uint32_t)(deg - 1) << 20));
                a.ukey[e4 >> 2] = (uint16_t)key;
                a.ucnt[p] = 1;
                atomicAdd(a.hist + key, 1);
            }
            return;
        }
    }
    {
        const int4 r0 = a.pair_rec[2 * (size_t)p];
        const int32_t f = r0.x, g = r0.y, e4 = a.pair_rec[2 * (size_t)p + 1].x;
        const int32_t deg = __ldg(a.con_ptr + g + 1) - __ldg(a.con_ptr + g);
        const int hasg = g < a.n ? 1 : 0, d = deg - 1, loads = hasg + d;
        // a check sums into a slot while slots last; the rest chain
        int slot = -1;
        if (!hasg) {
            if (lane == 0) slot = atomicAdd(a.fhdr + kFhSlotCtr, 1);
            slot = __shfl_sync(0xffffffffu, slot, 0);
            if (slot >= a.slot_cap) slot = -1;
        }
        int S = kFlowSeg;
        if (slot < 0) S = max(S, (loads + kFlowChain - 1) / kFlowChain);
        const int nseg = (loads + S - 1) / S;
        if (hasg && lane == 0) a.raw[e4] = (uint16_t)g;
        for (int s = lane; s < 128; s += 32) skey[s] = 0;
        __syncwarp();
        // the member at load position q belongs to segment q / S, whose key
        // is 1 + the highest level among its members
        if (deg <= kFlowSortMax) {
            // element i of this lane is row entry lane + 32 i; its key
            // (level, index) ranks it among the d members (keys are distinct;
            // the f entry and lanes past the row hold the largest key)
            uint32_t key[kFlowSortMax / 32];
#pragma unroll
            for (int i = 0; i < kFlowSortMax / 32; ++i) {
                const int j = lane + 32 * i;
                key[i] = 0xFFFFFFFFu;
                if (j < deg) {
                    const int32_t h = __ldg(a.con_idx4 + e4 + j);
                    if (h != f) key[i] = ((uint32_t)a.lvl[h] << 16) | (uint32_t)h;
                }
            }
            int rk[kFlowSortMax / 32];
#pragma unroll
            for (int i = 0; i < kFlowSortMax / 32; ++i) rk[i] = 0;
#pragma unroll
            for (int i2 = 0; i2 < kFlowSortMax / 32; ++i2) {
                if (32 * i2 >= deg) break;
                for (int q = 0; q < 32; ++q) {
                    const uint32_t kq = __shfl_sync(0xffffffffu, key[i2], q);
#pragma unroll
                    for (int i = 0; i < kFlowSortMax / 32; ++i) rk[i] += kq < key[i] ? 1 : 0;
                }
            }
#pragma unroll
            for (int i = 0; i < kFlowSortMax / 32; ++i) {
                if (key[i] == 0xFFFFFFFFu) continue;
                const int q = hasg + rk[i];
                a.raw[e4 + q] = (uint16_t)(key[i] & 0xffffu);
                if (q / S < 128) atomicMax(skey + q / S, min((int)(key[i] >> 16) + 1, NL));
            }
        } else {
            // row order, compacted by ballot
            int w = 0;
            for (int32_t j0 = 0; j0 < deg; j0 += 32) {
                const int32_t h = j0 + lane < deg ? __ldg(a.con_idx4 + e4 + j0 + lane) : f;
                const unsigned keep = __ballot_sync(0xffffffffu, h != f);
                if (h != f) {
                    const int q = hasg + w + __popc(keep & ((1u << lane) - 1));
                    a.raw[e4 + q] = (uint16_t)h;
                    if (q / S < 128) atomicMax(skey + q / S, min((int)a.lvl[h] + 1, NL));
                }
                w += __popc(keep);
            }
        }
        __syncwarp();
        if (lane == 0) {
            const int ub = e4 >> 2;
            if (nseg > 128) {
                atomicExch(a.fhdr + kFhOverflow, 1);  // more segments than the key table
                a.ucnt[p] = 0;
            } else if (slot >= 0) {
                for (int s = 0; s < nseg; ++s) {
                    const int s0 = s * S, s1 = min(loads, s0 + S);
                    const int hg = (s == 0) ? hasg : 0;
                    a.uarea[ub + s] = make_uint2((uint32_t)f | ((uint32_t)hg << 16) |
                                                     ((uint32_t)kUnitSlot << 17) | ((uint32_t)slot << 19),
                                                 (uint32_t)(e4 + s0) | ((uint32_t)(s1 - s0 - hg) << 20));
                    a.ukey[ub + s] = (uint16_t)skey[s];
                    atomicAdd(a.hist + skey[s], 1);
                }
                a.slot_nseg[slot] = nseg;
                a.ucnt[p] = nseg;
            } else {
                // chain: keys made non-decreasing (a later key is still at
                // most the pair's level), runs of equal keys merged
                for (int s = 1; s < nseg; ++s) skey[s] = max(skey[s], skey[s - 1]);
                int runs = 0;
                for (int s = 0; s < nseg; ++s) runs += (s == 0 || skey[s] != skey[s - 1]) ? 1 : 0;
                int r = -1;
                for (int s = 0; s < nseg; ++s) {
                    if (s > 0 && skey[s] == skey[s - 1]) continue;
                    ++r;
                    int e = s;
                    while (e + 1 < nseg && skey[e + 1] == skey[s]) ++e;
                    const int s0 = s * S, s1 = min(loads, (e + 1) * S);
                    const int hg = (s == 0) ? hasg : 0;
                    a.uarea[ub + r] = make_uint2((uint32_t)f | ((uint32_t)hg << 16) |
                                                     ((uint32_t)kUnitChain << 17) | ((uint32_t)r << 19) |
                                                     ((r == runs - 1) ? (1u << 27) : 0u),
                                                 (uint32_t)(e4 + s0) | ((uint32_t)(s1 - s0 - hg) << 20));
                    a.ukey[ub + r] = (uint16_t)skey[s];
                    atomicAdd(a.hist + skey[s], 1);
                }
                a.ucnt[p] = runs;
            }
        }
        __syncwarp();
    }
}

struct FlowPlaceArgs {
    const int32_t *hdr, *hist, *ucnt;
    const int4 *pair_rec;
    const uint2 *uarea;
    const uint16_t *ukey, *raw;  // read-only here (written by k_flow_units)
    int32_t *fhdr;
    uint2 *units;
    uint4 *batches;
    uint16_t *mem;
    int32_t cap_bytes;   // shared memory the payload has for units, batches and loads
    int32_t slot_cap;
    int32_t smem_bytes;  // dynamic shared memory of this kernel
};

// Block-wide exclusive scan of one counter; *tot receives the sum. Every
// thread calls it; s_w holds 32 ints of scratch.
__device__ int flow_block_scan(int x, int *tot, int *s_w) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (int)(blockDim.x >> 5);
    int v = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    if (lane == 31) s_w[wid] = v;
    __syncthreads();
    int before = 0, all = 0;
    for (int j = 0; j < nw; ++j) {
        const int t = s_w[j];
        before += j < wid ? t : 0;
        all += t;
    }
    __syncthreads();  // s_w may be reused after this
    *tot = all;
    return before + v - x;
}

// The units in key order, their batches and their loads in batch order.
__global__ void __launch_bounds__(1024, 1) k_flow_place(FlowPlaceArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_w[32];
    const int tid = threadIdx.x, T = blockDim.x;
    const int32_t P = a.hdr[WS_N_PAIRS], NL = a.hdr[WS_N_LEVELS];
    if (a.fhdr[kFhOverflow]) return;  // no plan: the payload walks level by level
    auto up16 = [](int x) { return (x + 15) & ~15; };
    // keys 0..NL: their first unit (kst), a placement cursor (kcur), their
    // batch count then first batch (kb)
    const int nk = NL + 1;
    int *kst = reinterpret_cast<int *>(smem);
    int *kcur = kst + nk + 1;
    int *kb = kcur + nk + 1;
    const int per = (nk + T - 1) / T;
    int c = 0;
    for (int k = tid * per; k < min(nk, (tid + 1) * per); ++k) c += a.hist[k];
    int U;
    int run = flow_block_scan(c, &U, s_w);
    for (int k = tid * per; k < min(nk, (tid + 1) * per); ++k) {
        kst[k] = run;
        kcur[k] = 0;
        run += a.hist[k];
    }
    if (tid == 0) kst[nk] = U;
    const int o_srec = up16(4 * 3 * (nk + 1));
    const int o_uoff = o_srec + up16(8 * U);
    if (o_uoff + up16(4 * (U + 1)) > a.smem_bytes) return;
    uint2 *srec = reinterpret_cast<uint2 *>(smem + o_srec);
    int *uoff = reinterpret_cast<int *>(smem + o_uoff);
    __syncthreads();
    // every unit at its key's place (any order inside a key)
    for (int32_t p = tid; p < P; p += T) {
        const int32_t ub = __ldg(&a.pair_rec[2 * (size_t)p + 1].x) >> 2;
        const int cu = __ldg(a.ucnt + p);
        for (int i = 0; i < cu; ++i) {
            const int k = __ldg(a.ukey + ub + i);
            srec[kst[k] + atomicAdd(kcur + k, 1)] = __ldg(a.uarea + ub + i);
        }
    }
    __syncthreads();
    // the loads of the units in this order
    const int upt = (U + T - 1) / T;
    c = 0;
    for (int u = tid * upt; u < min(U, (tid + 1) * upt); ++u) c += unit_slots(srec[u]);
    int M;
    run = flow_block_scan(c, &M, s_w);
    for (int u = tid * upt; u < min(U, (tid + 1) * upt); ++u) {
        uoff[u] = run;
        run += unit_slots(srec[u]);
    }
    if (tid == 0) uoff[U] = M;
    __syncthreads();
    // batches: consecutive units of one key, at most kFlowSeg loads and
    // units each (a unit of more loads alone)
    c = 0;
    for (int k = tid * per; k < min(nk, (tid + 1) * per); ++k) {
        int nb = 0, load = kFlowSeg + 1, cnt = kFlowSeg;
        for (int u = kst[k]; u < kst[k + 1]; ++u) {
            const int sl = unit_slots(srec[u]);
            if (load + sl > kFlowSeg || cnt == kFlowSeg) {
                ++nb;
                load = 0;
                cnt = 0;
            }
            load += sl;
            ++cnt;
        }
        kb[k] = nb;
        c += nb;
    }
    int NB;
    run = flow_block_scan(c, &NB, s_w);
    const bool fits = up16(8 * U) + up16(16 * NB) + up16(2 * M) <= a.cap_bytes && M <= (int)kMoffMask &&
                      U < 65536;
    for (int k = tid * per; k < min(nk, (tid + 1) * per); ++k) {
        const int nb = kb[k];
        kb[k] = run;
        run += nb;
    }
    __syncthreads();
    if (!fits) return;
    // batch record: {u0 | units << 16 | loads << 20, first load, masks over
    // its loads (a batch of at most kFlowSeg): c_g | partial sum << 8 | last
    // load of a unit << 16 (a dummy load of a unit without loads has both of
    // the first two bits), 0}
    auto put_batch = [&](int b, int u0, int cnt, int load) {
        uint32_t cm = 0, pm = 0, em = 0;
        if (load <= kFlowSeg) {
            int j = 0;
            for (int u = u0; u < u0 + cnt; ++u) {
                const uint2 r = srec[u];
                const int hasg = (int)((r.x >> 16) & 1u), kind = (int)((r.x >> 17) & 3u);
                const int aux = (int)((r.x >> 19) & 0xffu);
                const int sl = unit_slots(r);
                if (hasg + ((kind == kUnitChain && aux > 0) ? 1 : 0) + (int)(r.y >> 20) == 0) {
                    cm |= 1u << j;
                    pm |= 1u << j;
                } else {
                    if (hasg) cm |= 1u << j;
                    if (kind == kUnitChain && aux > 0) pm |= 1u << (j + hasg);
                }
                j += sl;
                em |= 1u << (j - 1);
            }
        }
        a.batches[b] = make_uint4((uint32_t)u0 | ((uint32_t)cnt << 16) | ((uint32_t)load << 20),
                                  (uint32_t)uoff[u0], cm | (pm << 8) | (em << 16), 0u);
    };
    for (int k = tid * per; k < min(nk, (tid + 1) * per); ++k) {
        int b = kb[k] - 1, load = kFlowSeg + 1, cnt = kFlowSeg, u0 = 0;
        for (int u = kst[k]; u < kst[k + 1]; ++u) {
            const int sl = unit_slots(srec[u]);
            if (load + sl > kFlowSeg || cnt == kFlowSeg) {
                if (b >= kb[k]) put_batch(b, u0, cnt, load);
                ++b;
                load = 0;
                cnt = 0;
                u0 = u;
            }
            load += sl;
            ++cnt;
        }
        if (b >= kb[k]) put_batch(b, u0, cnt, load);
    }
    // the units with their loads' new place; the loads: c_g, the chain's
    // partial sum (x_f), then the members
    for (int u = tid; u < U; u += T) {
        const uint2 r = srec[u];
        const int hasg = (int)((r.x >> 16) & 1u), kind = (int)((r.x >> 17) & 3u);
        const int aux = (int)((r.x >> 19) & 0xffu), cnt = (int)(r.y >> 20);
        const int from = (int)(r.y & kMoffMask);
        int o = uoff[u];
        if (hasg + ((kind == kUnitChain && aux > 0) ? 1 : 0) + cnt == 0) a.mem[o] = 0;  // dummy
        if (hasg) a.mem[o++] = __ldg(a.raw + from);
        if (kind == kUnitChain && aux > 0) a.mem[o++] = (uint16_t)(r.x & 0xffffu);
        for (int j0 = 0; j0 < cnt; j0 += 8) {
            uint16_t v[8];  // loads issued together
#pragma unroll
            for (int j = 0; j < 8; ++j) v[j] = j0 + j < cnt ? __ldg(a.raw + from + hasg + j0 + j) : 0;
#pragma unroll
            for (int j = 0; j < 8; ++j)
                if (j0 + j < cnt) a.mem[o + j0 + j] = v[j];
        }
        a.units[u] = make_uint2(r.x, (uint32_t)uoff[u] | (r.y & ~kMoffMask));
    }
    __syncthreads();
    if (tid == 0) {
        a.fhdr[kFhUnits] = U;
        a.fhdr[kFhLoads] = M;
        a.fhdr[kFhBatches] = NB;
        a.fhdr[kFhSlots] = min(a.fhdr[kFhSlotCtr], a.slot_cap);
        __threadfence();
        a.fhdr[kFhOk] = 1;
    }
}

// The key walk's plan: one CTA (it runs beside the encode on the one SM the
// encode leaves free, right after the schedule), every counter in shared
// memory. From the path's pairs, the level of every recovered intermediate
// (flow_lvl) and every heavy constraint's members in the order the schedule
// recovered them, that is by ascending level (flow_list):
//   A. a light pair (at most kFlowSeg loads) is one whole unit keyed by its
//      level; a heavy pair is listed for B;
//   B. a heavy pair's loads (c_g, then its members in that order) are cut
//      into segments of S; a segment's key is 1 + the level of its last
//      member (its highest); runs of equal keys are merged into chain links
//      (link r > 0 also loads x_f);
//   C. prefix sums over keys give each key's range of units and loads;
//   D. every unit and its loads are placed in its key's range: whole pairs
//      from the front, chain links from the back (the links then run in the
//      key's last rounds, which measured faster than any mix).
// A path that does not fit (more keys, heavy pairs or segments than the
// tables, a key larger than the payload's stages), or whose schedule kept
// no member order, gets no plan: the header stays zero and the payload walks
// level by level.
constexpr int kPlanThreads = 1024;
constexpr int kPlanHeavy = 1024;  // heavy pairs
constexpr int kPlanSegs = 4096;   // their segments
constexpr int kPlanUnits = 8192;  // units, staged in shared memory
constexpr int kPlanMem = 40960;   // loads, staged in shared memory

struct KeyPlanArgs {
    const int32_t *hdr;
    const int4 *pair_rec;
    const int32_t *con_idx4;
    const uint16_t *lvl, *list;
    const uint32_t *pinfo;
    int32_t n;
    int32_t *fhdr;
    int4 *ktab;
    uint2 *units;
    uint16_t *mem;
};

size_t key_plan_smem() {
    auto up16 = [](size_t x) { return (x + 15) & ~(size_t)15; };
    return up16((size_t)6 * 4 * (kKeyMax + 1)) + up16((size_t)kPlanHeavy * (16 + 8)) +
           up16((size_t)kPlanSegs * (4 + 2)) + up16((size_t)kPlanUnits * 8) + up16((size_t)kPlanMem * 2);
}

// S (loads per segment) of a heavy pair of `loads` loads: 8, or more when a
// chain would have more than kFlowChain links.
__device__ __forceinline__ int plan_seg(int loads) {
    return max(kFlowSeg, (loads + kFlowChain - 1) / kFlowChain);
}

// Five pairs of one thread (p0, p0 + T, ...): records, degrees and levels
// (from flow_pinfo: reads of consecutive words, not scattered ones), all
// loads in flight together.
struct PlanPairs {
    int4 r0[5];
    int32_t e4[5], deg[5];
    int lv[5];
};

__device__ __forceinline__ void plan_pairs(const KeyPlanArgs &a, int32_t p0, int32_t P, int T, PlanPairs &q) {
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        const int32_t p = p0 + i * T;
        if (p < P) {
            q.r0[i] = __ldg(&a.pair_rec[2 * (size_t)p]);
            q.e4[i] = __ldg(&a.pair_rec[2 * (size_t)p + 1].x);
        }
    }
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        const int32_t p = p0 + i * T;
        if (p < P) {
            const uint32_t w = a.pinfo[p];
            q.deg[i] = (int32_t)(w >> 16);
            q.lv[i] = (int)(w & 0xffffu);
        }
    }
}

// Whether segment j (of the heavy pair whose segments x = {first, count}
// holds) starts a chain link; if so, the link's last segment *e (relative to
// the pair) and its index *r among the pair's links (the key changes before
// it).
__device__ __forceinline__ bool plan_link(const uint32_t *segk, int2 x, int j, int *e, int *r) {
    const int s = j - x.x;
    if (s > 0 && segk[j - 1] == segk[j]) return false;  // not the first segment of its run
    int ee = s;
    while (ee + 1 < x.y && segk[x.x + ee + 1] == segk[j]) ++ee;
    int rr = 0;
    for (int t = 1; t <= s; ++t) rr += segk[x.x + t] != segk[x.x + t - 1] ? 1 : 0;
    *e = ee;
    *r = rr;
    return true;
}

__global__ void __launch_bounds__(kPlanThreads, 1) k_key_plan(KeyPlanArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_w[32];
    __shared__ int s_nh, s_ns, s_bad, s_u, s_m;
    const int tid = threadIdx.x, T = blockDim.x;
    const int32_t P = a.hdr[WS_N_PAIRS], NL = a.hdr[WS_N_LEVELS];
    const int nk = NL + 1;
    if (nk > kKeyMax || a.fhdr[kFlowHdrList] != 1) return;  // no plan (every thread)
    auto up16 = [](size_t x) { return (x + 15) & ~(size_t)15; };
    int *hu = reinterpret_cast<int *>(smem);  // units per key
    int *hl = hu + (kKeyMax + 1);             // loads per key
    int *cu = hl + (kKeyMax + 1);             // units placed (whole pairs low 16 bits, links high 16)
    int *cl = cu + (kKeyMax + 1);             // loads placed
    int *bu = cl + (kKeyMax + 1);             // first unit
    int *bl = bu + (kKeyMax + 1);             // first load
    size_t o = up16((size_t)6 * 4 * (kKeyMax + 1));
    int4 *hrec = reinterpret_cast<int4 *>(smem + o);  // heavy pair: {f, g, e4, deg}
    int2 *hx = reinterpret_cast<int2 *>(hrec + kPlanHeavy);  // {first segment, segments}
    o += up16((size_t)kPlanHeavy * (16 + 8));
    uint32_t *segk = reinterpret_cast<uint32_t *>(smem + o);  // segment keys
    uint16_t *segh = reinterpret_cast<uint16_t *>(segk + kPlanSegs);  // segment: its heavy pair
    o += up16((size_t)kPlanSegs * (4 + 2));
    // the units and their loads, built here and written out in 16-byte
    // pieces at the end (scattered 2- and 8-byte stores to global memory
    // were the plan's largest cost)
    uint2 *sunit = reinterpret_cast<uint2 *>(smem + o);
    o += up16((size_t)kPlanUnits * 8);
    uint16_t *smm = reinterpret_cast<uint16_t *>(smem + o);
    for (int i = tid; i < 4 * (kKeyMax + 1); i += T) hu[i] = 0;  // hu, hl, cu, cl
    if (tid == 0) {
        s_nh = 0;
        s_ns = 0;
        s_bad = 0;
    }
    __syncthreads();

    // A: five pairs a thread at a time (their loads in flight together)
    for (int32_t p0 = tid; p0 < P; p0 += 5 * T) {
        PlanPairs q;
        plan_pairs(a, p0, P, T, q);
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            if (p0 + i * T >= P) continue;
            const int32_t g = q.r0[i].y, deg = q.deg[i];
            const int hasg = g < a.n ? 1 : 0, loads = hasg + deg - 1;
            if (loads <= kFlowSeg) {
                const int k = min(q.lv[i], (int)NL);
                atomicAdd(hu + k, 1);
                atomicAdd(hl + k, max(loads, 1));
            } else {
                const int S = plan_seg(loads), nseg = (loads + S - 1) / S;
                const int h = atomicAdd(&s_nh, 1);
                const int sg = atomicAdd(&s_ns, nseg);
                if (h >= kPlanHeavy || sg + nseg > kPlanSegs || deg < kListDeg) {
                    s_bad = 1;
                    continue;
                }
                hrec[h] = make_int4(q.r0[i].x, g, q.e4[i], deg);
                hx[h] = make_int2(sg, nseg);
                for (int j = 0; j < nseg; ++j) segh[sg + j] = (uint16_t)h;
            }
        }
    }
    __syncthreads();
    if (s_bad) return;  // no plan (every thread)
    const int NS = s_ns;

    // B: segment keys, one thread a segment: the level of the segment's last
    // member (its highest: the members come by ascending level) + 1
    for (int j0 = tid; j0 < NS; j0 += 4 * T) {
        uint16_t m4[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int j = j0 + i * T;
            m4[i] = 0;
            if (j < NS) {
                const int h = segh[j];
                const int4 hr = hrec[h];
                const int hasg = hr.y < a.n ? 1 : 0, loads = hasg + hr.w - 1;
                const int s = j - hx[h].x;
                m4[i] = a.list[hr.z + min(loads, (s + 1) * plan_seg(loads)) - 1 - hasg];
            }
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int j = j0 + i * T;
            if (j < NS) segk[j] = (uint32_t)min((int)a.lvl[m4[i]] + 1, (int)NL);
        }
    }
    __syncthreads();
    // ... and the chain links (runs of equal keys) counted per key
    for (int j = tid; j < NS; j += T) {
        const int h = segh[j];
        const int2 x = hx[h];
        int e, r;
        if (!plan_link(segk, x, j, &e, &r)) continue;
        const int4 hr = hrec[h];
        const int hasg = hr.y < a.n ? 1 : 0, loads = hasg + hr.w - 1;
        const int S = plan_seg(loads);
        const int s0 = (j - x.x) * S, s1 = min(loads, (e + 1) * S);
        atomicAdd(hu + segk[j], 1);
        atomicAdd(hl + segk[j], (s1 - s0) + (r > 0 ? 1 : 0));
    }
    __syncthreads();

    // C: the keys' ranges
    {
        const int c0 = tid < nk ? hu[tid] : 0, c1 = tid < nk ? hl[tid] : 0;
        int U, M;
        const int ub = flow_block_scan(c0, &U, s_w);
        const int lb = flow_block_scan(c1, &M, s_w);
        if (tid < nk) {
            bu[tid] = ub;
            bl[tid] = lb;
            const int u0 = ub & ~1, u1 = (ub + c0 + 1) & ~1, m0 = lb & ~7, m1 = (lb + c1 + 7) & ~7;
            a.ktab[2 * tid] = make_int4(ub, c0, u0, u1 - u0);
            a.ktab[2 * tid + 1] = make_int4(m0, m1 - m0, 0, 0);
            if (u1 - u0 > kKeyUnits || m1 - m0 > kKeyMem) s_bad = 1;
        }
        if (tid == 0) {
            if (M > (int)kMoffMask || M > kPlanMem || U > kPlanUnits) s_bad = 1;
            s_u = U;
            s_m = M;
        }
        __syncthreads();
        if (s_bad) return;  // no plan (every thread)
        if (tid == 0) {
            a.fhdr[kFhUnits] = U;
            a.fhdr[kFhLoads] = M;
        }
    }

    // D: whole pairs from the front of their key's range ...
    for (int32_t p0 = tid; p0 < P; p0 += 5 * T) {
        PlanPairs q;
        plan_pairs(a, p0, P, T, q);
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            if (p0 + i * T >= P) continue;
            const int32_t f = q.r0[i].x, g = q.r0[i].y, deg = q.deg[i];
            const int hasg = g < a.n ? 1 : 0, loads = hasg + deg - 1;
            if (loads > kFlowSeg) continue;
            const int k = min(q.lv[i], (int)NL);
            const int pos = bu[k] + (atomicAdd(cu + k, 1) & 0xffff);
            const int lpos = bl[k] + atomicAdd(cl + k, max(loads, 1));
            const int4 *row = reinterpret_cast<const int4 *>(a.con_idx4 + q.e4[i]);
            int4 q4[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) q4[c] = 4 * c < deg ? __ldg(row + c) : make_int4(-1, -1, -1, -1);
            int w = lpos;
            if (loads == 0) smm[w] = 0;  // a unit without loads keeps one slot
            if (hasg) smm[w++] = (uint16_t)g;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const int32_t hv[4] = {q4[c].x, q4[c].y, q4[c].z, q4[c].w};
#pragma unroll
                for (int t = 0; t < 4; ++t)
                    if (4 * c + t < deg && hv[t] != f) smm[w++] = (uint16_t)hv[t];
            }
            sunit[pos] = make_uint2((uint32_t)f | ((uint32_t)hasg << 16) | ((uint32_t)kUnitWhole << 17),
                                      (uint32_t)lpos | ((uint32_t)(deg - 1) << 20));
        }
    }
    // ... chain links from the back, one thread a link
    for (int j = tid; j < NS; j += T) {
        const int h = segh[j];
        const int2 x = hx[h];
        int e, r;
        if (!plan_link(segk, x, j, &e, &r)) continue;
        const int4 hr = hrec[h];
        const int32_t f = hr.x, g = hr.y;
        const int hasg = g < a.n ? 1 : 0, loads = hasg + hr.w - 1;
        const int S = plan_seg(loads);
        const int s = j - x.x, key = (int)segk[j];
        const int s0 = s * S, s1 = min(loads, (e + 1) * S);
        const int hg = s == 0 ? hasg : 0, cnt = s1 - s0 - hg, last = e == x.y - 1 ? 1 : 0;
        const int old = atomicAdd(cu + key, 0x10000);
        const int pos = bu[key] + hu[key] - 1 - (old >> 16);
        const int lpos = bl[key] + atomicAdd(cl + key, hg + (r > 0 ? 1 : 0) + cnt);
        const uint16_t *ml = a.list + hr.z;
        int w = lpos;
        if (hg) smm[w++] = (uint16_t)g;
        if (r > 0) smm[w++] = (uint16_t)f;
        for (int qq = s0 + hg; qq < s1; qq += 8) {
            uint16_t v[8];  // members loaded together
#pragma unroll
            for (int t = 0; t < 8; ++t) v[t] = qq + t < s1 ? ml[qq + t - hasg] : 0;
#pragma unroll
            for (int t = 0; t < 8; ++t)
                if (qq + t < s1) smm[w + t] = v[t];
            w += min(8, s1 - qq);
        }
        sunit[pos] = make_uint2((uint32_t)f | ((uint32_t)hg << 16) | ((uint32_t)kUnitChain << 17) |
                                      ((uint32_t)r << 19) | ((uint32_t)last << 27),
                                  (uint32_t)lpos | ((uint32_t)cnt << 20));
    }
    __syncthreads();
    // E: units and loads out in 16-byte pieces (both arrays have room past
    // the last piece)
    {
        const int4 *su = reinterpret_cast<const int4 *>(sunit);
        int4 *du = reinterpret_cast<int4 *>(a.units);
        for (int i = tid; i < (s_u + 1) / 2; i += T) du[i] = su[i];
        const int4 *sm = reinterpret_cast<const int4 *>(smm);
        int4 *dm = reinterpret_cast<int4 *>(a.mem);
        for (int i = tid; i < (s_m + 7) / 8; i += T) dm[i] = sm[i];
    }
    __syncthreads();
    if (tid == 0) {
        a.fhdr[kFhKeyFit] = 1;
        __threadfence();
        a.fhdr[kFhOk] = 1;
    }
}

// Writes x_f of a finished check from its accumulator and marks it final
// (the whole warp; every segment fenced before counting).
__device__ __forceinline__ void flow_finish_slot(const PeelArgs &a, uint2 r, uint4 *accs, uint8_t *ready,
                                                 int64_t w0, int lanes, int L) {
    const int lane = threadIdx.x & 31;
    const int32_t f = (int32_t)(r.x & 0xffffu);
    __threadfence_block();
    const volatile uint4 *sa = accs + (size_t)((r.x >> 19) & 0xffu) * L;
    for (int k = lane; k < lanes; k += 32) {
        const uint4 v = make_uint4(sa[k].x, sa[k].y, sa[k].z, sa[k].w);
        block_ptr(a, f)[w0 + k] = v;
    }
    __syncwarp();
    if (lane == 0) {
        __threadfence_block();
        *(volatile uint8_t *)(ready + f) = kReadyFinal;
    }
}

// One unit of ns > kFlowSeg loads (ml[0..ns): c_g, the chain's partial sum,
// members), gathered kFlowSeg at a time. Returns false when its wait expired
// (the CTA stops).
__device__ bool flow_big_unit(const PeelArgs &a, uint2 r, const uint16_t *ml, int ns,
                              const volatile uint8_t *rdy, uint8_t *ready, uint4 *accs, int32_t *done,
                              int64_t w0, int lanes, int L, int *s_abort) {
    const int lane = threadIdx.x & 31;
    const int32_t f = (int32_t)(r.x & 0xffffu);
    const int hasg = (int)((r.x >> 16) & 1u), kind = (int)((r.x >> 17) & 3u);
    const int aux = (int)((r.x >> 19) & 0xffu);
    const int part = (kind == kUnitChain && aux > 0) ? 1 : 0;  // load hasg is the partial sum
    bool ok = false;
    for (long long it = 0; it < kFlowWaitLimit; ++it) {
        bool mine = true;
        for (int j = lane; j < ns; j += 32) {
            if (hasg && j == 0) continue;
            if (part && j == hasg) mine = mine && (rdy[f] & 0x7f) == aux;
            else mine = mine && (rdy[ml[j]] & kReadyFinal) != 0;
        }
        ok = __all_sync(0xffffffffu, mine);
        if (ok || __any_sync(0xffffffffu, *(volatile int *)s_abort != 0)) break;  // warp-uniform exit
        __nanosleep(32);
    }
    if (!ok) {
        if (lane == 0) {
            atomicExch(a.status, FS_ERR_TIMEOUT);
            *s_abort = 1;
        }
        return false;
    }
    __syncwarp();
    __threadfence_block();
    for (int k = lane; k < lanes; k += 32) {
        const int64_t w = w0 + k;
        uint4 acc = make_uint4(0, 0, 0, 0);
        for (int j0 = 0; j0 < ns; j0 += kFlowSeg) {
            uint4 x[kFlowSeg];
#pragma unroll
            for (int j = 0; j < kFlowSeg; ++j) {
                const int jj = j0 + j;
                x[j] = make_uint4(0, 0, 0, 0);
                if (jj < ns) {
                    if (hasg && jj == 0) x[j] = __ldg(a.coded + (int64_t)ml[0] * a.tw + w);
                    else x[j] = block_ptr(a, ml[jj])[w];
                }
            }
#pragma unroll
            for (int j = 0; j < kFlowSeg; ++j) xor4(acc, x[j]);
        }
        if (kind == kUnitSlot) xor_shared(accs + (size_t)aux * L + k, acc);
        else block_ptr(a, f)[w] = acc;
    }
    __syncwarp();
    int fin = 0;
    if (lane == 0) {
        __threadfence_block();
        if (kind == kUnitWhole) *(volatile uint8_t *)(ready + f) = kReadyFinal;
        else if (kind == kUnitChain)
            *(volatile uint8_t *)(ready + f) = ((r.x >> 27) & 1u) ? kReadyFinal : (uint8_t)(aux + 1);
        else fin = atomicSub(done + aux, 1) == 1 ? 1 : 0;
    }
    if (__shfl_sync(0xffffffffu, fin, 0)) flow_finish_slot(a, r, accs, ready, w0, lanes, L);
    return true;
}

// Runs the payload on the plan; returns false (the same answer in every
// thread, before anything is written to global memory) when there is no
// plan, and the caller walks level by level.
__device__ bool flow_body(const PeelArgs &a, int64_t slice) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_abort;
    const int32_t *fh = a.fhdr;
    if (fh[kFhOk] != 1) return false;
    const int tid = threadIdx.x, T = blockDim.x, lane = tid & 31, wid = tid >> 5, nw = T >> 5;
    const int32_t K = a.k_int, U = fh[kFhUnits], M = fh[kFhLoads], NS = fh[kFhSlots];
    const int32_t NB = fh[kFhBatches];
    const int L = a.L;
    const int64_t w0 = slice * L;
    const int lanes = (int)min((int64_t)L, a.tw - w0);
    auto up16 = [](int x) { return (x + 15) & ~15; };
    // shared layout: ready[K], units[U], batches[NB], mem[M], done[NS], accs[NS][L]
    uint8_t *ready = smem;
    const int o_units = up16(K);
    const int o_batch = o_units + up16(8 * U);
    const int o_mem = o_batch + up16(16 * NB);
    const int o_done = o_mem + up16(2 * M);
    const int o_acc = o_done + up16(4 * NS);
    uint2 *units = reinterpret_cast<uint2 *>(smem + o_units);
    uint4 *batches = reinterpret_cast<uint4 *>(smem + o_batch);
    uint16_t *mem = reinterpret_cast<uint16_t *>(smem + o_mem);
    int32_t *done = reinterpret_cast<int32_t *>(smem + o_done);
    uint4 *accs = reinterpret_cast<uint4 *>(smem + o_acc);
    // the plan into shared memory (16-byte copies; the arrays are padded)
    {
        const int4 *su = reinterpret_cast<const int4 *>(a.funits);
        for (int i = tid; i < up16(8 * U) / 16; i += T) reinterpret_cast<int4 *>(units)[i] = su[i];
        for (int i = tid; i < NB; i += T) batches[i] = a.fbatch[i];
        const int4 *sm = reinterpret_cast<const int4 *>(a.fmem);
        for (int i = tid; i < up16(2 * M) / 16; i += T) reinterpret_cast<int4 *>(mem)[i] = sm[i];
    }
    for (int i = tid; i < up16(K) / 16; i += T) reinterpret_cast<int4 *>(ready)[i] = make_int4(0, 0, 0, 0);
    for (int i = tid; i < NS; i += T) done[i] = a.fslot[i];
    for (int i = tid; i < NS * L; i += T) accs[i] = make_uint4(0, 0, 0, 0);
    if (tid == 0) s_abort = 0;
    __syncthreads();

    const volatile uint8_t *rdy = ready;
    for (int b = wid; b < NB; b += nw) {
        if (__any_sync(0xffffffffu, *(volatile int *)&s_abort != 0)) break;  // warp-uniform
        const uint4 br = batches[b];
        const int u0 = (int)(br.x & 0xffffu), nu = (int)((br.x >> 16) & 15u);
        const int ns = (int)((br.x >> 20) & 0xfffu), mo = (int)br.y;
        if (ns > kFlowSeg) {
            // one unit of more loads than a round (alone in its batch)
            if (!flow_big_unit(a, units[u0], mem + mo, ns, rdy, ready, accs, done, w0, lanes, L,
                               &s_abort))
                break;
            continue;
        }
        // lane j < ns owns load j of the batch: its block, its kind (0 member,
        // 1 coded row, 2 the chain's partial sum, 3 nothing), its unit and
        // whether it is its unit's last load (from the batch's masks)
        int id = 0, typ = 0, ui = 0, endu = 0, need = 0;
        if (lane < ns) {
            const uint32_t bit = 1u << lane, em = (br.z >> 16) & 0xffu;
            id = mem[mo + lane];
            typ = ((br.z & bit) ? 1 : 0) | (((br.z >> 8) & bit) ? 2 : 0);
            endu = (em & bit) ? 1 : 0;
            ui = __popc(em & (bit - 1));
            if (typ == 2) need = (int)((units[u0 + ui].x >> 19) & 0xffu);
        }
        // wait for every block the batch reads
        bool ok = false;
        for (long long it = 0; it < kFlowWaitLimit; ++it) {
            bool mine = true;
            if (lane < ns) {
                if (typ == 0) mine = (rdy[id] & kReadyFinal) != 0;
                else if (typ == 2) mine = (rdy[id] & 0x7f) == need;
            }
            ok = __all_sync(0xffffffffu, mine);
            if (ok || __any_sync(0xffffffffu, *(volatile int *)&s_abort != 0)) break;  // warp-uniform
            __nanosleep(32);
        }
        if (!ok) {
            if (lane == 0) {
                atomicExch(a.status, FS_ERR_TIMEOUT);
                s_abort = 1;
            }
            break;
        }
        __syncwarp();  // the watchers' reads come before every lane's loads
        __threadfence_block();
        // every lane learns every load of the batch (all 32 lanes here:
        // the word loop below leaves out the lanes past the slice)
        // load j: block | kind << 16 | last of its unit << 18 | unit << 19
        uint32_t jl[kFlowSeg];
#pragma unroll
        for (int j = 0; j < kFlowSeg; ++j)
            jl[j] = __shfl_sync(0xffffffffu,
                                (uint32_t)id | ((uint32_t)typ << 16) | ((uint32_t)endu << 18) |
                                    ((uint32_t)ui << 19),
                                j);
        for (int k = lane; k < lanes; k += 32) {
            const int64_t w = w0 + k;
            uint4 x[kFlowSeg];  // the batch's loads, all in flight at once
#pragma unroll
            for (int j = 0; j < kFlowSeg; ++j) {
                x[j] = make_uint4(0, 0, 0, 0);
                if (j < ns) {
                    const int t = (int)((jl[j] >> 16) & 3u), jid = (int)(jl[j] & 0xffffu);
                    if (t == 1) x[j] = __ldg(a.coded + (int64_t)jid * a.tw + w);
                    else if (t != 3) x[j] = block_ptr(a, jid)[w];
                }
            }
            uint4 acc = make_uint4(0, 0, 0, 0);
#pragma unroll
            for (int j = 0; j < kFlowSeg; ++j) {
                const int je = (int)((jl[j] >> 18) & 1u);
                const int jui = (int)(jl[j] >> 19);
                if (j < ns) {
                    xor4(acc, x[j]);
                    if (je) {
                        const uint2 r = units[u0 + jui];
                        const int32_t f = (int32_t)(r.x & 0xffffu);
                        if (((r.x >> 17) & 3u) == kUnitSlot)
                            xor_shared(accs + (size_t)((r.x >> 19) & 0xffu) * L + k, acc);
                        else
                            block_ptr(a, f)[w] = acc;
                        acc = make_uint4(0, 0, 0, 0);
                    }
                }
            }
        }
        // release: every lane's writes come before the fences and flags
        __syncwarp();
        int fin = 0;
        if (lane < nu) {
            const uint2 r = units[u0 + lane];
            const int32_t f = (int32_t)(r.x & 0xffffu);
            const int kind = (int)((r.x >> 17) & 3u), aux = (int)((r.x >> 19) & 0xffu);
            __threadfence_block();
            if (kind == kUnitWhole) *(volatile uint8_t *)(ready + f) = kReadyFinal;
            else if (kind == kUnitChain)
                *(volatile uint8_t *)(ready + f) = ((r.x >> 27) & 1u) ? kReadyFinal : (uint8_t)(aux + 1);
            else fin = atomicSub(done + aux, 1) == 1 ? 1 : 0;
        }
        // a check whose last segment this was: its sum is complete (every
        // other segment fenced before counting)
        unsigned fins = __ballot_sync(0xffffffffu, fin != 0);
        while (fins) {
            const int i = __ffs(fins) - 1;
            fins &= fins - 1;
            flow_finish_slot(a, units[u0 + i], accs, ready, w0, lanes, L);
        }
    }
    __syncthreads();
    // unrecovered data blocks read as zero
    const int32_t nu = a.hdr[WS_N_UNREC_DATA];
    for (int32_t it = tid; it < nu * lanes; it += T) {
        const int32_t q = it / lanes, lane2 = it - q * lanes;
        a.data[(int64_t)a.unrec_list[q] * a.tw + w0 + lane2] = make_uint4(0, 0, 0, 0);
    }
    return true;
}

// ---------------------------------------------------------------------------
// key walk
//
// The units of the key walk's plan (k_key_plan below: every heavy pair
// chained, units keyed like the dataflow plan's) walked with one block
// barrier per key (= level). Key k's units read only blocks that units of
// smaller keys finished, so after the barrier that ends key k - 1 every unit
// of key k may run at once, one item per (unit, word) as in the level walk:
// its loads (c_g, the chain's partial sum, its members) all in flight, then
// one store. The heavy gathers run while their members are fresh in L2.
// Stages: key k's units and loads are bulk-copied into slot k % 3 two keys
// ahead (one mbarrier phase each), and key k + 1's coded rows are prefetched
// into L2 while key k runs.

constexpr int kKeyRound = 9;  // loads in flight per item (a chain link: its partial sum and 8 members)

size_t keys_smem_bytes() {
    return (size_t)kKeyMax * 32 + (size_t)3 * (kKeyUnits * 8 + kKeyMem * 2);
}

// One thread: bulk copies of key k's units and loads into slot k % 3.
__device__ __forceinline__ void issue_key(const PeelArgs &a, const int4 *kt, int k, uint2 *sun,
                                          uint16_t *smm, uint64_t *bar) {
    const int4 t0 = kt[2 * k], t1 = kt[2 * k + 1];
    const int sl = k % 3;
    const uint32_t ub = (uint32_t)t0.w * 8, mb = (uint32_t)t1.y * 2;
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    mbar_expect_tx(bar, ub + mb);
    if (ub) bulk_g2s(sun + sl * kKeyUnits, a.funits + t0.z, ub, bar);
    if (mb) bulk_g2s(smm + sl * kKeyMem, a.fmem + t1.x, mb, bar);
}

// Returns false (the same answer in every thread, before anything is written
// to global memory) when the path has no key-walk plan; the level walk then
// runs in the launch that follows (k_peel).
template <bool kHints>
__device__ bool keys_body(const PeelArgs &a, int64_t slice) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ __align__(8) uint64_t mb_keys[3];
    __shared__ int s_ok[2];  // by key parity: thread 0 writes the next while others read this one
    const int32_t *fh = a.fhdr;
    if (fh[kFhOk] != 1 || fh[kFhKeyFit] != 1) return false;
    const int tid = threadIdx.x, T = blockDim.x;
    const int L = a.L;
    const int64_t w0 = slice * L;
    const int lanes = (int)min((int64_t)L, a.tw - w0);
    const int nk = a.hdr[WS_N_LEVELS] + 1;
    int4 *kt = reinterpret_cast<int4 *>(smem);                        // [2 kKeyMax]
    uint2 *sun = reinterpret_cast<uint2 *>(kt + 2 * kKeyMax);          // [3][kKeyUnits]
    uint16_t *smm = reinterpret_cast<uint16_t *>(sun + 3 * kKeyUnits);  // [3][kKeyMem]
    for (int i = tid; i < 2 * nk; i += T) kt[i] = a.fktab[i];
    if (tid == 0) {
        for (int k = 0; k < 3; ++k) mbar_init(&mb_keys[k]);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        s_ok[0] = s_ok[1] = 1;
    }
    __syncthreads();
    if (tid == 0)
        for (int k = 0; k < 2 && k < nk; ++k) issue_key(a, kt, k, sun, smm, &mb_keys[k]);
    const int lines = (lanes * 16 + 127) >> 7;
    // every thread keeps one word kk and takes units srow, srow + nrows, ...
    // of each key, counted from the highest thread (as in the level walk)
    const int rt0 = T - 1 - tid;
    const int kk = rt0 % lanes, srow = rt0 / lanes, nrows = T / lanes;
    bool ok = true;
    for (int k = 0; k < nk; ++k) {
        const int ps = k % 3;
        if (tid == 0) {
            // key k's stages are in; so are key k + 1's, whose coded rows are
            // prefetched below
            const uint32_t ph0 = (uint32_t)((k / 3) & 1), ph1 = (uint32_t)(((k + 1) / 3) & 1);
            const bool in0 = mbar_wait(&mb_keys[ps], ph0);
            const bool in1 = in0 && (k + 1 >= nk || mbar_wait(&mb_keys[(k + 1) % 3], ph1));
            s_ok[k & 1] = in1 ? 1 : 0;
            if (!in1) {
                // give up, but first wait longer (8 bounds) for the copies
                // not yet seen to land (keys k and k + 1; k + 2's is not
                // issued yet)
                if (!in0) mbar_wait(&mb_keys[ps], ph0, 8);
                if (k + 1 < nk) mbar_wait(&mb_keys[(k + 1) % 3], ph1, 8);
            }
        }
        __syncthreads();  // key k - 1 is written; key k's stages are in
        if (!s_ok[k & 1]) {
            ok = false;
            break;
        }
        if (tid == 0 && k + 2 < nk) issue_key(a, kt, k + 2, sun, smm, &mb_keys[(k + 2) % 3]);
        if (k + 1 < nk) {
            // L2 prefetch of the coded rows key k + 1 reads (low threads; the
            // items below start from the high ones)
            const int q = (k + 1) % 3;
            const int4 n0 = kt[2 * (k + 1)], n1 = kt[2 * (k + 1) + 1];
            const uint2 *un = sun + q * kKeyUnits + (n0.x - n0.z);
            for (int i = tid; i < n0.y * lines; i += T) {
                const int j = i / lines, ln = i - j * lines;
                const uint2 r = un[j];
                if ((r.x >> 16) & 1u) {
                    const int32_t g = smm[q * kKeyMem + (int)(r.y & kMoffMask) - n1.x];
                    const char *p = reinterpret_cast<const char *>(a.coded + (int64_t)g * a.tw + w0) + 128 * ln;
                    asm volatile("prefetch.global.L2 [%0];\n" ::"l"(p));
                }
            }
        }
        const int4 t0 = kt[2 * k], t1 = kt[2 * k + 1];
        const uint2 *ut = sun + ps * kKeyUnits + (t0.x - t0.z);
        const uint16_t *mt = smm + ps * kKeyMem;
        const uint64_t pol_last = kHints ? l2_policy_last() : 0, pol_first = kHints ? l2_policy_first() : 0;
        for (int j = (srow < nrows ? srow : t0.y); j < t0.y; j += nrows) {
            const int64_t w = w0 + kk;
            const uint2 r = ut[j];
            // loads: c_g (hasg), the chain's partial sum (a link after the
            // first), the members; none for a check without members (x_f = 0)
            const int hasg = (int)((r.x >> 16) & 1u);
            const int part = (((r.x >> 17) & 3u) == kUnitChain && ((r.x >> 19) & 0xffu) > 0) ? 1 : 0;
            const int nl = hasg + part + (int)(r.y >> 20);
            const int mo = (int)(r.y & kMoffMask) - t1.x;  // its first load in the stage
            uint4 x[kKeyRound];  // the round's loads, all in flight at once
#pragma unroll
            for (int i = 0; i < kKeyRound; ++i) {
                x[i] = make_uint4(0, 0, 0, 0);
                if (i < nl) {
                    const int32_t h = mt[mo + i];
                    if (i == 0 && hasg) {
                        const uint4 *src = a.coded + (int64_t)h * a.tw + w;
                        x[i] = kHints ? ld_nc_hint(src, pol_first) : src[0];
                    } else {
                        const uint4 *src = block_ptr(a, h) + w;
                        x[i] = kHints ? ld_hint(src, pol_last) : src[0];
                    }
                }
            }
            uint4 acc = x[0];
#pragma unroll
            for (int i = 1; i < kKeyRound; ++i) xor4(acc, x[i]);
            // a link of more loads (equal keys merged): further rounds of 8
            for (int j0 = kKeyRound; j0 < nl; j0 += 8) {
                uint4 y[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    y[i] = make_uint4(0, 0, 0, 0);
                    if (j0 + i < nl) y[i] = block_ptr(a, mt[mo + j0 + i])[w];
                }
#pragma unroll
                for (int i = 0; i < 8; ++i) xor4(acc, y[i]);
            }
            uint4 *dst = block_ptr(a, (int32_t)(r.x & 0xffffu)) + w;
            if (kHints) st_hint(dst, acc, pol_last);
            else dst[0] = acc;
        }
    }
    __syncthreads();
    if (tid == 0 && !ok) atomicExch(a.status, FS_ERR_TIMEOUT);
    // unrecovered data blocks read as zero
    const int32_t nu = a.hdr[WS_N_UNREC_DATA];
    for (int32_t it = tid; it < nu * lanes; it += T) {
        const int32_t q = it / lanes, lane2 = it - q * lanes;
        a.data[(int64_t)a.unrec_list[q] * a.tw + w0 + lane2] = make_uint4(0, 0, 0, 0);
    }
    return true;
}

// The level walk alone; k_peel_flow is the dataflow walk (its own kernel, so
// its registers do not weigh on the level walk), which falls back to the
// level walk when the path has no plan.
// The level walk; after k_peel_keys (a.flow == 2) it runs only where the key
// walk had no plan (the same answer in every thread).
template <bool kHints>
__global__ void __launch_bounds__(kPeelThreads, 1) k_peel(PeelArgs a) {
    if (a.flow == 2 && a.fhdr[kFhOk] == 1 && a.fhdr[kFhKeyFit] == 1) return;
    peel_body<kHints>(a, blockIdx.x);
}

template <bool kHints>
__global__ void __launch_bounds__(kPeelThreads, 1) k_peel_flow(PeelArgs a) {
    if (flow_body(a, blockIdx.x)) return;
    peel_body<kHints>(a, blockIdx.x);
}

// the key walk; where its plan is missing it does nothing, and k_peel,
// launched right after it, walks level by level (the level walk's stages
// would make this launch's shared memory, and so take L1 from the gathers)
template <bool kHints>
__global__ void __launch_bounds__(kPeelThreads, 1) k_peel_keys(PeelArgs a) {
    keys_body<kHints>(a, blockIdx.x);
}

// one CTA per (stripe, slice) item of a batch
template <bool kHints>
__global__ void __launch_bounds__(kPeelThreads, 1) k_peel_batch(const PeelArgs *as, const int2 *items) {
    const int2 it = items[blockIdx.x];
    const PeelArgs a = as[it.x];
    peel_body<kHints>(a, it.y);
}

size_t peel_smem_bytes(int64_t L) {
    return (size_t)(kStageLevels + 1) * 32 + (size_t)3 * kStagePairs * kRec * 4 +
           (size_t)3 * kStageSegs * 4 + (size_t)3 * (kStageRecipe / 4) * 4 +
           (size_t)2 * kStageRecipe * 4 +
           (size_t)kStageMulti * L * 16 + (size_t)kStageMulti * L * 4;
}

}  // namespace

namespace {

DpgArgs dpg_args(const fs_code *c, const uint8_t *erased, uint8_t *ws, uint8_t *unrecovered,
                 int32_t *n_unrecovered) {
    const DecodeLayout L = decode_layout(c);
    DpgArgs a;
    a.con_ptr = c->con_ptr;
    a.con_ptr4 = c->con_ptr4;
    a.con_xs = c->con_xs;
    a.con_sum = c->con_sum;
    a.var_ptr = c->var_ptr;
    a.var_idx = c->var_idx;
    a.erased = erased;
    a.b = c->b;
    a.n = c->n;
    a.k_int = c->k_int;
    a.n_con = c->n_con;
    a.two_pass = (c->flags & FS_DECODE_TWO_PASS) ? 1 : 0;
    a.res = reinterpret_cast<int32_t *>(ws + L.res);
    a.xs = reinterpret_cast<int32_t *>(ws + L.xs);
    a.best = reinterpret_cast<unsigned long long *>(ws + L.best);
    a.known = ws + L.known;
    a.front_a = reinterpret_cast<int32_t *>(ws + L.front_a);
    a.front_b = reinterpret_cast<int32_t *>(ws + L.front_b);
    a.touched = reinterpret_cast<int32_t *>(ws + L.touched);
    a.pair_f = reinterpret_cast<int32_t *>(ws + L.pair_f);
    a.pair_g = reinterpret_cast<int32_t *>(ws + L.pair_g);
    a.pair_rec = reinterpret_cast<int4 *>(ws + L.pair_rec);
    a.level_off = reinterpret_cast<int32_t *>(ws + L.level_off);
    a.level_tab = reinterpret_cast<int4 *>(ws + L.level_tab);
    a.seg_pair = reinterpret_cast<int32_t *>(ws + L.seg_pair);
    a.chunk_pair = reinterpret_cast<int32_t *>(ws + L.chunk_pair);
    a.unrec_list = reinterpret_cast<int32_t *>(ws + L.unrec_list);
    a.hdr = reinterpret_cast<int32_t *>(ws);
    a.unrecovered = unrecovered;
    a.n_unrecovered = n_unrecovered;
    a.flow_hdr = reinterpret_cast<int32_t *>(ws + L.flow_hdr);
    a.flow_lvl = reinterpret_cast<uint16_t *>(ws + L.flow_lvl);
    a.flow_hist = reinterpret_cast<int32_t *>(ws + L.flow_hist);
    const bool keys = c->peel_flow >= 2 && !(c->peel_columns && col_fits(c)) && flow_applies(c);
    a.flow_list = keys ? reinterpret_cast<uint16_t *>(ws + L.flow_list) : nullptr;
    a.flow_pinfo = keys ? reinterpret_cast<uint32_t *>(ws + L.flow_pinfo) : nullptr;
    return a;
}

}  // namespace

namespace {

cudaError_t launch_dpg_only(const fs_code *c, const uint8_t *erased, uint8_t *ws,
                            uint8_t *unrecovered, int32_t *n_unrecovered, cudaStream_t s) {
    const DpgArgs a = dpg_args(c, erased, ws, unrecovered, n_unrecovered);
    const DpgCompactPlace cp = plan_dpg_compact(c);
    if (c->dpg_compact && cp.bytes >= 0) {
        if (cp.bytes > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(
                k_dpg_compact, cudaFuncAttributeMaxDynamicSharedMemorySize, cp.bytes);
            if (e != cudaSuccess) return e;
        }
        k_dpg_compact<<<1, kDpgThreads, (size_t)cp.bytes, s>>>(a, cp);
        return cudaGetLastError();
    }
    const DpgPlace pl = plan_dpg(c);
    if (pl.bytes > 48 * 1024) {
        cudaError_t e =
            cudaFuncSetAttribute(k_dpg, cudaFuncAttributeMaxDynamicSharedMemorySize, pl.bytes);
        if (e != cudaSuccess) return e;
    }
    k_dpg<<<1, kDpgThreads, (size_t)pl.bytes, s>>>(a, pl);
    return cudaGetLastError();
}

}  // namespace

bool flow_applies(const fs_code *c);
namespace {
cudaError_t launch_flow_plan(const fs_code *c, uint8_t *ws, cudaStream_t s);
}  // namespace

// The symbolic pass, then the plan of the payload that will run: the column
// payload's when it is selected and the code fits it, else the dataflow
// walk's where it applies.
cudaError_t launch_dpg(const fs_code *c, const uint8_t *erased, uint8_t *ws, uint8_t *unrecovered,
                       int32_t *n_unrecovered, cudaStream_t s) {
    cudaError_t e = launch_dpg_only(c, erased, ws, unrecovered, n_unrecovered, s);
    if (e == cudaSuccess && c->peel_columns && col_fits(c)) e = launch_col_plan(c, ws, s);
    if (e == cudaSuccess && !(c->peel_columns && col_fits(c)) && flow_applies(c))
        e = launch_flow_plan(c, ws, s);
    return e;
}

namespace {

// slice width: every slice in flight at once (peel_ctas CTAs per SM), at
// most kPeelLmax words
int64_t peel_slice_words(const fs_code *c) {
    const int64_t ctas = (int64_t)c->num_sms * c->peel_ctas;
    int64_t Lw = (c->tw + ctas - 1) / ctas;
    if (Lw > kPeelLmax) Lw = kPeelLmax;
    if (Lw < 1) Lw = 1;
    return Lw;
}

PeelArgs peel_args(const fs_code *c, const uint4 *coded, uint4 *data_out, uint8_t *ws) {
    const DecodeLayout L = decode_layout(c);
    PeelArgs a;
    a.coded = coded;
    a.data = data_out;
    a.parity = reinterpret_cast<uint4 *>(ws + L.parity);
    a.con_idx4 = c->con_idx4;
    a.seg_pair = reinterpret_cast<const int32_t *>(ws + L.seg_pair);
    a.chunk_pair = reinterpret_cast<const int32_t *>(ws + L.chunk_pair);
    a.unrec_list = reinterpret_cast<const int32_t *>(ws + L.unrec_list);
    a.hdr = reinterpret_cast<const int32_t *>(ws);
    a.pair_rec = reinterpret_cast<const int4 *>(ws + L.pair_rec);
    a.level_tab = reinterpret_cast<const int4 *>(ws + L.level_tab);
    a.b = c->b;
    a.n = c->n;
    a.tw = c->tw;
    a.hints = c->l2_hints;
    a.status = reinterpret_cast<int32_t *>(ws) + WS_STATUS;
    a.L = (int32_t)peel_slice_words(c);
    a.flow = 0;  // the launcher turns the dataflow walk on where it applies
    a.k_int = c->k_int;
    a.fhdr = reinterpret_cast<const int32_t *>(ws + L.flow_hdr);
    a.funits = reinterpret_cast<const uint2 *>(ws + L.flow_units);
    a.fbatch = reinterpret_cast<const uint4 *>(ws + L.flow_batch);
    a.fmem = reinterpret_cast<const uint16_t *>(ws + L.flow_mem);
    a.fslot = reinterpret_cast<const int32_t *>(ws + L.flow_slot);
    a.fktab = reinterpret_cast<const int4 *>(ws + L.flow_ktab);
    return a;
}

}  // namespace

// The key walk by default (FS_TUNE_PEEL_FLOW = 2) only where the
// intermediates reach 64 MiB: below that the recovered blocks stay in L2 for
// the level walk too, and the schedule's member order and the plan kernel
// (~10-40 us) would not pay; 3 takes it at any size.
constexpr int64_t kKeyWalkMinBytes = (int64_t)64 << 20;

// The dataflow walks apply to one 1024-thread CTA per SM, 16-bit block ids
// and levels, rows of at most kFlowMaxDeg and padded graphs whose offsets fit
// 20 bits (and the key walk to a device with room for its stages and its plan).
bool flow_applies(const fs_code *c) {
    const bool keys = c->peel_flow >= 2;
    return c->peel_flow && c->peel_ctas == 1 && c->k_int <= 65535 && c->n_con <= 65535 &&
           c->max_con_deg <= kFlowMaxDeg && c->e_con4 < (int64_t)kMoffMask &&
           (!keys || (keys_smem_bytes() <= c->smem_optin && key_plan_smem() <= c->smem_optin)) &&
           (c->peel_flow != 2 || (int64_t)c->k_int * c->t >= kKeyWalkMinBytes);
}

namespace {

// Check accumulator slots of the payload: at most kFlowSlots, and at most
// 64 KiB of shared memory.
int flow_slot_cap(int64_t L) { return (int)std::min<int64_t>(kFlowSlots, 65536 / (16 * L)); }

size_t flow_smem(const fs_code *c) { return c->smem_optin & ~(size_t)15; }

cudaError_t launch_flow_plan(const fs_code *c, uint8_t *ws, cudaStream_t s) {
    const DecodeLayout L = decode_layout(c);
    const int64_t Lw = peel_slice_words(c);
    if (c->peel_flow >= 2) {
        // the key walk's plan: one CTA
        KeyPlanArgs k;
        k.hdr = reinterpret_cast<const int32_t *>(ws);
        k.pair_rec = reinterpret_cast<const int4 *>(ws + L.pair_rec);
        k.con_idx4 = c->con_idx4;
        k.lvl = reinterpret_cast<const uint16_t *>(ws + L.flow_lvl);
        k.list = reinterpret_cast<const uint16_t *>(ws + L.flow_list);
        k.pinfo = reinterpret_cast<const uint32_t *>(ws + L.flow_pinfo);
        k.n = c->n;
        k.fhdr = reinterpret_cast<int32_t *>(ws + L.flow_hdr);
        k.ktab = reinterpret_cast<int4 *>(ws + L.flow_ktab);
        k.units = reinterpret_cast<uint2 *>(ws + L.flow_units);
        k.mem = reinterpret_cast<uint16_t *>(ws + L.flow_mem);
        const size_t ksm = key_plan_smem();
        cudaError_t e = cudaFuncSetAttribute(k_key_plan, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ksm);
        if (e != cudaSuccess) return e;
        k_key_plan<<<1, kPlanThreads, ksm, s>>>(k);
        return cudaGetLastError();
    }
    const int slots = flow_slot_cap(Lw);
    const size_t smem = flow_smem(c);
    FlowUnitArgs u;
    u.hdr = reinterpret_cast<const int32_t *>(ws);
    u.pair_rec = reinterpret_cast<const int4 *>(ws + L.pair_rec);
    u.con_ptr = c->con_ptr;
    u.con_idx4 = c->con_idx4;
    u.lvl = reinterpret_cast<const uint16_t *>(ws + L.flow_lvl);
    u.n = c->n;
    u.slot_cap = slots;
    u.fhdr = reinterpret_cast<int32_t *>(ws + L.flow_hdr);
    u.hist = reinterpret_cast<int32_t *>(ws + L.flow_hist);
    u.ucnt = reinterpret_cast<int32_t *>(ws + L.flow_ucnt);
    u.slot_nseg = reinterpret_cast<int32_t *>(ws + L.flow_slot);
    u.uarea = reinterpret_cast<uint2 *>(ws + L.flow_uarea);
    u.ukey = reinterpret_cast<uint16_t *>(ws + L.flow_ukey);
    u.raw = reinterpret_cast<uint16_t *>(ws + L.flow_raw);
    // a warp for every possible pair; those past the path's pairs return
    const int ctas = (c->k_int + kFlowUnitThreads / 32 - 1) / (kFlowUnitThreads / 32);
    k_flow_units<<<std::max(ctas, 1), kFlowUnitThreads, 0, s>>>(u);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    FlowPlaceArgs a;
    a.hdr = u.hdr;
    a.hist = u.hist;
    a.ucnt = u.ucnt;
    a.pair_rec = u.pair_rec;
    a.uarea = u.uarea;
    a.ukey = u.ukey;
    a.raw = u.raw;
    a.fhdr = u.fhdr;
    a.units = reinterpret_cast<uint2 *>(ws + L.flow_units);
    a.batches = reinterpret_cast<uint4 *>(ws + L.flow_batch);
    a.mem = reinterpret_cast<uint16_t *>(ws + L.flow_mem);
    // the payload's shared memory less its ready flags, counters and accumulators
    const int64_t rest = (int64_t)smem - ((c->k_int + 15) & ~15) - ((4 * slots + 15) & ~15) -
                         (int64_t)slots * Lw * 16;
    a.cap_bytes = (int32_t)std::max<int64_t>(rest, 0);
    a.slot_cap = slots;
    a.smem_bytes = (int32_t)smem;
    e = cudaFuncSetAttribute(k_flow_place, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_flow_place<<<1, 1024, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_peel(const fs_code *c, const uint4 *coded, uint4 *data_out, uint8_t *ws,
                        cudaStream_t s) {
    if (c->peel_columns && col_fits(c)) return launch_peel_col(c, coded, data_out, ws, s);
    PeelArgs a = peel_args(c, coded, data_out, ws);
    const int64_t Lw = a.L;
    size_t smem = peel_smem_bytes(Lw);
    if (flow_applies(c)) {
        // the dataflow walk: all the shared memory the CTA may have (the
        // plan's size depends on the path, which only the device knows;
        // k_flow_place checks it)
        a.flow = std::min(c->peel_flow, 2);  // 3: the key walk at any size
        if (a.flow == 1) smem = std::max(smem, flow_smem(c));
    }
    const bool h = a.hints != 0;
    // one CTA per SM: 1024 threads; several: the SM's threads split between them
    const int threads =
        c->peel_ctas >= 4 ? kPeelThreads / 4 : (c->peel_ctas >= 2 ? kPeelThreads / 2 : kPeelThreads);
    const int64_t n_slices = (c->tw + Lw - 1) / Lw;
    cudaError_t e;
    if (a.flow == 2) {
        // the key walk on its own stages, then the level walk where it had
        // no plan (an empty launch where it had one)
        const auto kk = h ? k_peel_keys<true> : k_peel_keys<false>;
        const size_t ks = keys_smem_bytes();
        e = cudaFuncSetAttribute(kk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ks);
        if (e != cudaSuccess) return e;
        kk<<<(unsigned)n_slices, threads, ks, s>>>(a);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    const auto kern = a.flow == 1 ? (h ? k_peel_flow<true> : k_peel_flow<false>) : (h ? k_peel<true> : k_peel<false>);
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)n_slices, threads, smem, s>>>(a);
    return cudaGetLastError();
}

// ---- batched decode ----------------------------------------------------------
// The symbolic pass of every stripe (one CTA each, compact form where it fits)
// in one launch per form, then the payload of every (stripe, byte slice) item
// in one launch; each item walks all levels of its stripe's path for its slice.

struct DecodeBatch {
    DpgArgs *d_dc = nullptr;
    DpgCompactPlace *d_pc = nullptr;
    int n_c = 0, smem_c = 0;
    DpgArgs *d_dg = nullptr;
    DpgPlace *d_pg = nullptr;
    int n_g = 0, smem_g = 0;
    PeelArgs *d_peel = nullptr;
    int2 *d_items = nullptr;
    int n_items = 0;
    size_t smem_p = 0;
    bool hints = false;  // a stripe's code asks for L2 hints: the payload takes them for all
};

namespace {

template <typename T>
cudaError_t upload_vec(T **dst, const std::vector<T> &v) {
    return plan_upload(dst, v.data(), v.size());
}

}  // namespace

cudaError_t decode_batch_plan(const fs_code *const *codes, const void *const *coded,
                              const uint8_t *const *erased, void *const *data_out,
                              uint8_t *const *unrecovered, int32_t *const *n_unrecovered,
                              void *const *ws, int32_t n, bool schedule_only, DecodeBatch **out) {
    *out = nullptr;
    std::vector<DpgArgs> dc, dg;
    std::vector<DpgCompactPlace> pc;
    std::vector<DpgPlace> pg;
    std::vector<PeelArgs> peel;
    std::vector<int2> items;
    DecodeBatch *b = new DecodeBatch();
    for (int32_t i = 0; i < n; ++i) {
        const fs_code *c = codes[i];
        uint8_t *w = static_cast<uint8_t *>(ws[i]);
        DpgArgs a = dpg_args(c, erased[i], w, unrecovered[i], n_unrecovered[i]);
        a.flow_list = nullptr;  // the batch's payload walks level by level: no member order
        a.flow_pinfo = nullptr;
        const DpgCompactPlace cp = plan_dpg_compact(c);
        if (c->dpg_compact && cp.bytes >= 0) {
            dc.push_back(a);
            pc.push_back(cp);
            b->smem_c = std::max(b->smem_c, (int)cp.bytes);
        } else {
            const DpgPlace pl = plan_dpg(c);
            dg.push_back(a);
            pg.push_back(pl);
            b->smem_g = std::max(b->smem_g, (int)pl.bytes);
        }
        if (schedule_only) continue;  // the symbolic pass alone
        const PeelArgs pa = peel_args(c, static_cast<const uint4 *>(coded[i]),
                                      static_cast<uint4 *>(data_out[i]), w);
        peel.push_back(pa);
        b->hints = b->hints || pa.hints != 0;
        const int64_t slices = (c->tw + pa.L - 1) / pa.L;
        if ((int64_t)items.size() + slices >= INT32_MAX) {
            decode_batch_free(b);
            return cudaErrorInvalidValue;
        }
        for (int64_t k = 0; k < slices; ++k) items.push_back(make_int2(i, (int)k));
        b->smem_p = std::max(b->smem_p, peel_smem_bytes(pa.L));
    }
    b->n_c = (int)dc.size();
    b->n_g = (int)dg.size();
    b->n_items = (int)items.size();
    cudaError_t e = upload_vec(&b->d_dc, dc);
    if (e == cudaSuccess) e = upload_vec(&b->d_pc, pc);
    if (e == cudaSuccess) e = upload_vec(&b->d_dg, dg);
    if (e == cudaSuccess) e = upload_vec(&b->d_pg, pg);
    if (e == cudaSuccess) e = upload_vec(&b->d_peel, peel);
    if (e == cudaSuccess) e = upload_vec(&b->d_items, items);
    if (e == cudaSuccess && b->smem_c > 48 * 1024)
        e = cudaFuncSetAttribute(k_dpg_compact_batch, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 b->smem_c);
    if (e == cudaSuccess && b->smem_g > 48 * 1024)
        e = cudaFuncSetAttribute(k_dpg_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, b->smem_g);
    if (e == cudaSuccess && b->n_items > 0)
        e = cudaFuncSetAttribute(b->hints ? k_peel_batch<true> : k_peel_batch<false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem_p);
    if (e != cudaSuccess) {
        decode_batch_free(b);
        return e;
    }
    *out = b;
    return cudaSuccess;
}

cudaError_t decode_batch_run(const DecodeBatch *b, cudaStream_t s) {
    if (b->n_c > 0) k_dpg_compact_batch<<<b->n_c, kDpgThreads, (size_t)b->smem_c, s>>>(b->d_dc, b->d_pc);
    if (b->n_g > 0) k_dpg_batch<<<b->n_g, kDpgThreads, (size_t)b->smem_g, s>>>(b->d_dg, b->d_pg);
    if (b->n_items > 0) {
        const auto kern = b->hints ? k_peel_batch<true> : k_peel_batch<false>;
        kern<<<b->n_items, kPeelThreads, b->smem_p, s>>>(b->d_peel, b->d_items);
    }
    return cudaGetLastError();
}

void decode_batch_free(DecodeBatch *b) {
    if (!b) return;
    plan_free(b->d_dc);
    plan_free(b->d_pc);
    plan_free(b->d_dg);
    plan_free(b->d_pg);
    plan_free(b->d_peel);
    plan_free(b->d_items);
    delete b;
}
