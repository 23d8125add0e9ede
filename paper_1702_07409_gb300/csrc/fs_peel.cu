// fs_peel.cu - peeling decode split into a symbolic pass and a payload pass.
//
// k_dpg: Decoding Path Generation (Algorithm 5, Section 3.2) on one CTA.
//   Per constraint g the pass keeps res[g], the number of its variables still
//   unknown, and xs[g], the XOR of their indices: when res[g] == 1, xs[g] IS
//   the one unknown, so no row is scanned. The state lives in shared memory
//   when it fits, else in the workspace. A level is:
//     A. every frontier constraint g (res 1 at the level start) bids
//        key = (degree(g) << 32 | g) for its unknown f with an atomicMin: the
//        lowest original degree wins, ties go to the lowest constraint index
//        (Section 3.1, second rule);
//     B. each f with a bid becomes a pair (f, g) of the path; one block-wide
//        scan places the recipe of g (its whole row), its gather segments,
//        its accumulator slot and the adjacency slots of f;
//     C. slot-parallel: every recipe slot copies one entry of the row of g,
//        and every adjacency slot updates one constraint that contains f
//        (res -= 1, xs ^= f); a constraint whose count goes 2 -> 1 joins the
//        next frontier. Each thread finds its pair by binary search over the
//        level's scan offsets, so all loads of the step are independent.
//   res/xs only change in C, after every bid of the level was placed, so a
//   level uses only symbols decoded in earlier levels (Section 3.1, first
//   rule). Appends to the shared lists are warp-aggregated.
//
// k_peel: the payload. Each CTA owns one slice of L 16-byte words of every
//   block (about one CTA per SM, so every slice is in flight at once) and
//   walks all levels; pairs of a level are independent (no intermediate is
//   written twice and none is read in the level that writes it), so a
//   __syncthreads between levels is the only ordering needed: no grid-wide
//   synchronisation and no per-level launch. The level's metadata is staged
//   into shared memory two levels ahead with cp.async, and the coded
//   payloads and gathered blocks of the next level are bulk-prefetched into
//   L2 one level ahead. A recipe is gathered in segments of at most
//   kRecipeSeg blocks, one thread per (segment, word pair), all loads of a
//   segment in flight at once; pairs with several segments combine them in
//   shared-memory accumulators with XOR atomics before the block is written.
#include <cooperative_groups.h>

#include "fs_internal.cuh"

namespace cg = cooperative_groups;

namespace {

constexpr int kDpgThreads = 1024;
constexpr int kPeelThreads = 512;
constexpr int kPeelV = 2;           // 16-byte words per payload item
constexpr int kPeelLmax = 64;       // largest slice (words) of one payload CTA
constexpr int kStagePairs = 256;    // pairs of one level held in shared memory
constexpr int kStageRecipe = 2048;  // recipe entries of one level held in shared memory
constexpr int kStageLevels = 1024;  // level bounds held in shared memory
constexpr int kStageSegs = 512;     // gather segments of one level
constexpr int kStageMulti = 32;     // pairs with several segments in one level
// one metadata stage: f[P], g[P], ro[P+1], so[P+1], slot[P], sp[S], h[R]
constexpr int kMF = 0, kMG = kStagePairs, kMRO = 2 * kStagePairs, kMSO = 3 * kStagePairs + 1,
              kMSL = 4 * kStagePairs + 2, kMSP = 5 * kStagePairs + 2,
              kMH = 5 * kStagePairs + 2 + kStageSegs;
constexpr int kMetaInts = kMH + kStageRecipe;
constexpr unsigned long long kEmpty = ~0ull;

// Shared-memory placement of the DPG arrays: byte offsets into dynamic shared
// memory, or -1 for the workspace (global) copy.
struct DpgPlace {
    int32_t res, xs, best, known, front, next, touched, lvl_o, lvl_v, cptr, vptr;
    int32_t bytes;
};

struct DpgArgs {
    const int32_t *con_ptr, *con_idx, *con_xs, *var_ptr, *var_idx;
    const uint8_t *erased;
    int32_t b, n, k_int, n_con;
    int two_pass;
    DpgPlace pl;
    // workspace copies of the state (used where pl.* == -1)
    int32_t *res, *xs;
    unsigned long long *best;
    uint8_t *known;
    int32_t *front_a, *front_b, *touched, *lvl_o, *lvl_v;
    // outputs
    int32_t *pair_f, *pair_g, *level_off, *level_r0, *level_s0, *recipe_off, *seg_off, *acc_slot,
        *seg_pair, *recipe_h, *unrec_list, *hdr;
    uint8_t *unrecovered;
    int32_t *n_unrecovered;
};

// stage: -1 joint (every surviving coded row and every check), 0 coded rows
// only, 1 checks only (two-pass mode, Section 2.2)
__device__ __forceinline__ bool usable(const DpgArgs &a, int32_t g, int stage) {
    if (g < a.n) return stage <= 0 && a.erased[g] == 0;
    return stage != 0;
}

// Position of the calling thread in a shared list: one atomicAdd per group
// of converged threads.
__device__ __forceinline__ int append_slot(int *counter) {
    cg::coalesced_group grp = cg::coalesced_threads();
    int base = 0;
    if (grp.thread_rank() == 0) base = atomicAdd(counter, (int)grp.size());
    return grp.shfl(base, 0) + (int)grp.thread_rank();
}

// Block-wide exclusive prefix sum of four counters at once; *total receives
// the sums. All threads of the block must call it.
__device__ int4 block_excl_scan4(int4 x, int4 *total, int4 *s_warp) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
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
    if (lane == 31) s_warp[wid] = v;
    __syncthreads();
    if (wid == 0) {
        int4 s = lane < nw ? s_warp[lane] : make_int4(0, 0, 0, 0);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int a = __shfl_up_sync(0xffffffffu, s.x, o);
            const int b = __shfl_up_sync(0xffffffffu, s.y, o);
            const int c = __shfl_up_sync(0xffffffffu, s.z, o);
            const int d = __shfl_up_sync(0xffffffffu, s.w, o);
            if (lane >= o) {
                s.x += a;
                s.y += b;
                s.z += c;
                s.w += d;
            }
        }
        s_warp[lane] = s;  // inclusive warp totals
    }
    __syncthreads();
    const int4 before = wid > 0 ? s_warp[wid - 1] : make_int4(0, 0, 0, 0);
    *total = s_warp[nw - 1];
    __syncthreads();
    return make_int4(before.x + v.x - x.x, before.y + v.y - x.y, before.z + v.z - x.z,
                     before.w + v.w - x.w);
}

// Largest i in [0, n) with off[i] <= x, for ascending off[0] <= x.
__device__ __forceinline__ int find_slot(const int32_t *off, int n, int32_t x) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= x) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <typename T>
__device__ __forceinline__ T *place(unsigned char *smem, int32_t off, T *global) {
    return off >= 0 ? reinterpret_cast<T *>(smem + off) : global;
}

__global__ void __launch_bounds__(kDpgThreads, 1) k_dpg(DpgArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int4 s_warp4[32];
    __shared__ int s_nf, s_nt, s_nnext, s_cnt, s_cnt_data;

    const int tid = threadIdx.x, T = blockDim.x;
    const int32_t K = a.k_int, G = a.n_con;

    int32_t *res = place(smem, a.pl.res, a.res);
    int32_t *xs = place(smem, a.pl.xs, a.xs);
    unsigned long long *best = place(smem, a.pl.best, a.best);
    uint8_t *known = place(smem, a.pl.known, a.known);
    int32_t *front = place(smem, a.pl.front, a.front_a);
    int32_t *next = place(smem, a.pl.next, a.front_b);
    int32_t *touched = place(smem, a.pl.touched, a.touched);
    int32_t *lvl_o = place(smem, a.pl.lvl_o, a.lvl_o);
    int32_t *lvl_v = place(smem, a.pl.lvl_v, a.lvl_v);
    const int32_t *cptr = place(smem, a.pl.cptr, const_cast<int32_t *>(a.con_ptr));
    const int32_t *vptr = place(smem, a.pl.vptr, const_cast<int32_t *>(a.var_ptr));

    if (tid == 0) a.hdr[WS_STATUS] = FS_OK;
    if (a.pl.cptr >= 0)
        for (int32_t g = tid; g <= G; g += T)
            reinterpret_cast<int32_t *>(smem + a.pl.cptr)[g] = __ldg(a.con_ptr + g);
    if (a.pl.vptr >= 0)
        for (int32_t v = tid; v <= K; v += T)
            reinterpret_cast<int32_t *>(smem + a.pl.vptr)[v] = __ldg(a.var_ptr + v);
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
        if (usable(a, g, stage) && res[g] == 1) front[append_slot(&s_nf)] = g;
    __syncthreads();

    int32_t np = 0, level = 0, rb = 0, sb = 0, maxp = 0, maxr = 0, maxs = 0, maxm = 0;
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
        if (tid == 0) {
            a.level_off[level] = np;
            a.level_r0[level] = rb;
            a.level_s0[level] = sb;
        }
        // B: pairs of the level; one scan places recipes (x), gather
        // segments (y), adjacency slots (z) and accumulator slots (w). The
        // consumed frontier array holds g of pair i for step C.
        int32_t *lvl_g = front;
        int4 len = make_int4(0, 0, 0, 0);
        for (int base = 0; base < nt; base += T) {
            const int i = base + tid;
            int4 cnt = make_int4(0, 0, 0, 0);
            int32_t f = -1, g = -1;
            if (i < nt) {
                f = touched[i];
                const unsigned long long key = best[f];
                g = (int32_t)(key & 0xffffffffull);
                cnt.x = (int32_t)(key >> 32);
                cnt.y = (cnt.x + kRecipeSeg - 1) / kRecipeSeg;
                cnt.z = vptr[f + 1] - vptr[f];
                cnt.w = cnt.y > 1 ? 1 : 0;
                best[f] = kEmpty;
                known[f] = 1;
                a.pair_f[np + i] = f;
                a.pair_g[np + i] = g;
            }
            int4 total;
            const int4 off = block_excl_scan4(cnt, &total, s_warp4);
            if (i < nt) {
                a.recipe_off[np + i] = rb + len.x + off.x;
                a.seg_off[np + i] = sb + len.y + off.y;
                a.acc_slot[np + i] = cnt.w ? len.w + off.w : -1;
                for (int k = 0; k < cnt.y; ++k) a.seg_pair[sb + len.y + off.y + k] = i;
                lvl_g[i] = g;
                lvl_o[i] = len.x + off.x;
                lvl_v[i] = len.z + off.z;
            }
            len.x += total.x;
            len.y += total.y;
            len.z += total.z;
            len.w += total.w;
        }
        if (tid == 0) {
            lvl_o[nt] = len.x;
            lvl_v[nt] = len.z;
        }
        __syncthreads();
        // C: slot-parallel recipe copy and constraint updates
        for (int32_t r = tid; r < len.x; r += T) {
            const int i = find_slot(lvl_o, nt, r);
            a.recipe_h[rb + r] = __ldg(a.con_idx + cptr[lvl_g[i]] + (r - lvl_o[i]));
        }
        for (int32_t u = tid; u < len.z; u += T) {
            const int i = find_slot(lvl_v, nt, u);
            const int32_t f = touched[i];
            const int32_t c = __ldg(a.var_idx + vptr[f] + (u - lvl_v[i]));
            atomicXor(xs + c, f);
            if (atomicSub(res + c, 1) == 2 && usable(a, c, stage)) next[append_slot(&s_nnext)] = c;
        }
        __syncthreads();
        if (tid == 0) {
            s_nf = s_nnext;
            maxp = max(maxp, nt);
            maxr = max(maxr, len.x);
            maxs = max(maxs, len.y);
            maxm = max(maxm, len.w);
        }
        int32_t *tmp = front;
        front = next;
        next = tmp;
        np += nt;
        rb += len.x;
        sb += len.y;
        ++level;
        __syncthreads();
    }
    if (tid == 0) {
        a.level_off[level] = np;
        a.level_r0[level] = rb;
        a.level_s0[level] = sb;
        a.recipe_off[np] = rb;
        a.seg_off[np] = sb;
        a.hdr[WS_N_LEVELS] = level;
        a.hdr[WS_N_PAIRS] = np;
        a.hdr[WS_STAGED] = (maxp <= kStagePairs && maxr <= kStageRecipe && maxs <= kStageSegs &&
                            maxm <= kStageMulti && level <= kStageLevels)
                               ? 1
                               : 0;
        s_cnt = 0;
        s_cnt_data = 0;
    }
    __syncthreads();
    for (int32_t v = tid; v < K; v += T) {
        const uint8_t u = known[v] ? 0 : 1;
        a.unrecovered[v] = u;
        if (u) {
            atomicAdd(&s_cnt, 1);
            if (v < a.b) a.unrec_list[append_slot(&s_cnt_data)] = v;
        }
    }
    __syncthreads();
    if (tid == 0) {
        *a.n_unrecovered = s_cnt;
        a.hdr[WS_N_UNREC_DATA] = s_cnt_data;
    }
}

// ---------------------------------------------------------------------------
// payload

struct PeelArgs {
    const uint4 *coded;
    uint4 *data;    // intermediates v < b
    uint4 *parity;  // intermediates v >= b (workspace)
    const int32_t *pair_f, *pair_g, *level_off, *level_r0, *level_s0, *recipe_off, *seg_off,
        *acc_slot, *seg_pair, *recipe_h, *unrec_list, *hdr;
    int32_t b, n;
    int64_t tw;
    int32_t L;  // words of every block per CTA
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

__device__ __forceinline__ void cp_async4(void *sdst, const void *gsrc) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gsrc) : "memory");
}

__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}

__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// Bulk prefetch of bytes [p, p + bytes) into L2 (16-byte aligned, multiple of 16).
__device__ __forceinline__ void prefetch_l2(const void *p, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(p), "r"(bytes) : "memory");
}

// XOR of x_h[w] over recipe entries hs[rs .. re) other than f, into acc.
__device__ __forceinline__ uint4 gather_recipe(const PeelArgs &a, const int32_t *hs, int32_t rs,
                                               int32_t re, int32_t f, int64_t w, uint4 acc) {
    const uint4 zero = make_uint4(0, 0, 0, 0);
    int32_t r = rs;
    for (; r + 4 <= re; r += 4) {
        const int32_t h0 = hs[r], h1 = hs[r + 1], h2 = hs[r + 2], h3 = hs[r + 3];
        const uint4 x0 = block_ptr(a, h0)[w];
        const uint4 x1 = block_ptr(a, h1)[w];
        const uint4 x2 = block_ptr(a, h2)[w];
        const uint4 x3 = block_ptr(a, h3)[w];
        xor4(acc, h0 != f ? x0 : zero);
        xor4(acc, h1 != f ? x1 : zero);
        xor4(acc, h2 != f ? x2 : zero);
        xor4(acc, h3 != f ? x3 : zero);
    }
    for (; r < re; ++r) {
        const int32_t h = hs[r];
        if (h != f) xor4(acc, block_ptr(a, h)[w]);
    }
    return acc;
}

// Levels read straight from global memory (used when a level does not fit
// the shared-memory stages).
__device__ void peel_direct(const PeelArgs &a, int64_t w0, int lanes) {
    const int32_t n_levels = a.hdr[WS_N_LEVELS];
    for (int32_t l = 0; l < n_levels; ++l) {
        const int32_t p0 = a.level_off[l], p1 = a.level_off[l + 1];
        const int32_t items = (p1 - p0) * lanes;
        for (int32_t it = threadIdx.x; it < items; it += blockDim.x) {
            const int32_t q = it / lanes, lane = it - q * lanes;
            const int32_t p = p0 + q;
            const int32_t f = a.pair_f[p], g = a.pair_g[p];
            const int64_t w = w0 + lane;
            uint4 acc = make_uint4(0, 0, 0, 0);
            if (g < a.n) acc = __ldg(a.coded + (int64_t)g * a.tw + w);
            acc = gather_recipe(a, a.recipe_h, a.recipe_off[p], a.recipe_off[p + 1], f, w, acc);
            block_ptr(a, f)[w] = acc;
        }
        __syncthreads();
    }
}

__device__ __forceinline__ void stage_meta(const PeelArgs &a, int32_t *mb, const int32_t *lv_p,
                                           const int32_t *lv_r, const int32_t *lv_s, int l) {
    const int32_t p0 = lv_p[l], np = lv_p[l + 1] - p0;
    const int32_t r0 = lv_r[l], nr = lv_r[l + 1] - r0;
    const int32_t s0 = lv_s[l], ns = lv_s[l + 1] - s0;
    for (int i = threadIdx.x; i < np; i += blockDim.x) {
        cp_async4(mb + kMF + i, a.pair_f + p0 + i);
        cp_async4(mb + kMG + i, a.pair_g + p0 + i);
        cp_async4(mb + kMSL + i, a.acc_slot + p0 + i);
    }
    for (int i = threadIdx.x; i <= np; i += blockDim.x) {
        cp_async4(mb + kMRO + i, a.recipe_off + p0 + i);
        cp_async4(mb + kMSO + i, a.seg_off + p0 + i);
    }
    for (int i = threadIdx.x; i < ns; i += blockDim.x) cp_async4(mb + kMSP + i, a.seg_pair + s0 + i);
    for (int i = threadIdx.x; i < nr; i += blockDim.x) cp_async4(mb + kMH + i, a.recipe_h + r0 + i);
}

// L2 prefetch of what level l reads from global memory: the coded payload
// slices and the slices of every recipe block (staged metadata mb).
__device__ __forceinline__ void prefetch_level(const PeelArgs &a, const int32_t *mb, int np,
                                               int nr, int64_t w0, int lanes) {
    const uint32_t bytes = (uint32_t)lanes * 16u;
    for (int i = threadIdx.x; i < np + nr; i += blockDim.x) {
        if (i < np) {
            const int32_t g = mb[kMG + i];
            if (g < a.n) prefetch_l2(a.coded + (int64_t)g * a.tw + w0, bytes);
        } else {
            prefetch_l2(block_ptr(a, mb[kMH + (i - np)]) + w0, bytes);
        }
    }
}

__global__ void __launch_bounds__(kPeelThreads, 1) k_peel(PeelArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int L = a.L;
    const int64_t w0 = (int64_t)blockIdx.x * L;
    const int lanes = (int)min((int64_t)L, a.tw - w0);
    const int nv = (lanes + kPeelV - 1) / kPeelV;  // word pairs of this slice
    const int32_t nl = a.hdr[WS_N_LEVELS];

    if (!a.hdr[WS_STAGED]) {
        peel_direct(a, w0, lanes);
    } else {
        uint4 *accs = reinterpret_cast<uint4 *>(smem);  // [kStageMulti][L]
        uint32_t *accw = reinterpret_cast<uint32_t *>(accs);
        int32_t *lv_p = reinterpret_cast<int32_t *>(accs + kStageMulti * kPeelLmax);
        int32_t *lv_r = lv_p + kStageLevels + 1;
        int32_t *lv_s = lv_r + kStageLevels + 1;
        int32_t *meta = lv_s + kStageLevels + 1;  // [3][kMetaInts]
        for (int i = threadIdx.x; i <= nl; i += blockDim.x) {
            lv_p[i] = a.level_off[i];
            lv_r[i] = a.level_r0[i];
            lv_s[i] = a.level_s0[i];
        }
        for (int i = threadIdx.x; i < kStageMulti * L; i += blockDim.x)
            accs[i] = make_uint4(0, 0, 0, 0);
        __syncthreads();
        if (nl > 0) stage_meta(a, meta, lv_p, lv_r, lv_s, 0);
        cp_async_commit();
        cp_async_wait_all();
        __syncthreads();
        if (nl > 0) prefetch_level(a, meta, lv_p[1] - lv_p[0], lv_r[1] - lv_r[0], w0, lanes);
        if (nl > 1) stage_meta(a, meta + kMetaInts, lv_p, lv_r, lv_s, 1);
        cp_async_commit();
        cp_async_wait_all();
        __syncthreads();
        for (int32_t l = 0; l < nl; ++l) {
            const int32_t *mc = meta + (l % 3) * kMetaInts;
            // prefetch: level l+1 into L2, metadata of level l+2 into shared memory
            if (l + 1 < nl)
                prefetch_level(a, meta + ((l + 1) % 3) * kMetaInts, lv_p[l + 2] - lv_p[l + 1],
                               lv_r[l + 2] - lv_r[l + 1], w0, lanes);
            if (l + 2 < nl) stage_meta(a, meta + ((l + 2) % 3) * kMetaInts, lv_p, lv_r, lv_s, l + 2);
            cp_async_commit();
            const int np = lv_p[l + 1] - lv_p[l];
            const int ns = lv_s[l + 1] - lv_s[l];
            const int32_t r0 = lv_r[l], s0 = lv_s[l];
            const int32_t *hs = mc + kMH;
            // every (segment, word pair): one gather of at most kRecipeSeg blocks
            for (int it = threadIdx.x; it < ns * nv; it += blockDim.x) {
                const int s = it / nv, k = it - s * nv;
                const int q = mc[kMSP + s];
                const int32_t f = mc[kMF + q], g = mc[kMG + q];
                const int sidx = s - (mc[kMSO + q] - s0);
                const int32_t rs = mc[kMRO + q] - r0 + sidx * kRecipeSeg;
                const int32_t cnt = min(kRecipeSeg, mc[kMRO + q + 1] - r0 - rs);
                const int64_t w = w0 + k * kPeelV;
                const bool two = k * kPeelV + 1 < lanes;
                uint4 acc0 = make_uint4(0, 0, 0, 0), acc1 = acc0;
                if (sidx == 0 && g < a.n) {
                    const uint4 *src = a.coded + (int64_t)g * a.tw + w;
                    acc0 = src[0];
                    if (two) acc1 = src[1];
                }
                uint4 x0[kRecipeSeg], x1[kRecipeSeg];
#pragma unroll
                for (int j = 0; j < kRecipeSeg; ++j) {
                    const int32_t h = j < cnt ? hs[rs + j] : f;
                    x0[j] = x1[j] = make_uint4(0, 0, 0, 0);
                    if (h != f) {
                        const uint4 *src = block_ptr(a, h) + w;
                        x0[j] = src[0];
                        if (two) x1[j] = src[1];
                    }
                }
#pragma unroll
                for (int j = 0; j < kRecipeSeg; ++j) {
                    xor4(acc0, x0[j]);
                    xor4(acc1, x1[j]);
                }
                const int slot = mc[kMSL + q];
                if (slot < 0) {
                    uint4 *dst = block_ptr(a, f) + w;
                    dst[0] = acc0;
                    if (two) dst[1] = acc1;
                } else {
                    uint32_t *d = accw + 4 * (slot * L + k * kPeelV);
                    atomicXor(d + 0, acc0.x);
                    atomicXor(d + 1, acc0.y);
                    atomicXor(d + 2, acc0.z);
                    atomicXor(d + 3, acc0.w);
                    if (two) {
                        atomicXor(d + 4, acc1.x);
                        atomicXor(d + 5, acc1.y);
                        atomicXor(d + 6, acc1.z);
                        atomicXor(d + 7, acc1.w);
                    }
                }
            }
            if (ns > np) {  // some pair has several segments: write their sums
                __syncthreads();
                for (int it = threadIdx.x; it < np * lanes; it += blockDim.x) {
                    const int q = it / lanes, lane = it - q * lanes;
                    const int slot = mc[kMSL + q];
                    if (slot < 0) continue;
                    block_ptr(a, mc[kMF + q])[w0 + lane] = accs[slot * L + lane];
                    accs[slot * L + lane] = make_uint4(0, 0, 0, 0);
                }
            }
            cp_async_wait_all();
            __syncthreads();
        }
    }
    // unrecovered data blocks read as zero
    const int32_t nu = a.hdr[WS_N_UNREC_DATA];
    for (int32_t it = threadIdx.x; it < nu * lanes; it += blockDim.x) {
        const int32_t q = it / lanes, lane = it - q * lanes;
        a.data[(int64_t)a.unrec_list[q] * a.tw + w0 + lane] = make_uint4(0, 0, 0, 0);
    }
}

constexpr size_t kPeelSmem = (size_t)kStageMulti * kPeelLmax * 16 +
                             (size_t)3 * (kStageLevels + 1) * 4 + (size_t)3 * kMetaInts * 4;

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
    const int64_t state = 8 * K + 4 * G * 4 + 4 * K * 3 + K + 16 * 10;
    if (state <= budget) {
        p.best = take(8 * K);
        p.res = take(4 * G);
        p.xs = take(4 * G);
        p.front = take(4 * G);
        p.next = take(4 * G);
        p.touched = take(4 * K);
        p.lvl_o = take(4 * K);
        p.lvl_v = take(4 * K);
        p.known = take(K);
    } else {
        p.best = p.res = p.xs = p.front = p.next = p.touched = p.lvl_o = p.lvl_v = p.known = -1;
    }
    // graph row pointers, each where room is left
    p.cptr = (o + 4 * G <= budget) ? take(4 * G) : -1;
    p.vptr = (o + 4 * K <= budget) ? take(4 * K) : -1;
    p.bytes = (int32_t)o;
    return p;
}

}  // namespace

cudaError_t launch_dpg(const fs_code *c, const uint8_t *erased, uint8_t *ws, uint8_t *unrecovered,
                       int32_t *n_unrecovered, cudaStream_t s) {
    const DecodeLayout L = decode_layout(c);
    DpgArgs a;
    a.con_ptr = c->con_ptr;
    a.con_idx = c->con_idx;
    a.con_xs = c->con_xs;
    a.var_ptr = c->var_ptr;
    a.var_idx = c->var_idx;
    a.erased = erased;
    a.b = c->b;
    a.n = c->n;
    a.k_int = c->k_int;
    a.n_con = c->n_con;
    a.two_pass = (c->flags & FS_DECODE_TWO_PASS) ? 1 : 0;
    a.pl = plan_dpg(c);
    a.res = reinterpret_cast<int32_t *>(ws + L.res);
    a.xs = reinterpret_cast<int32_t *>(ws + L.xs);
    a.best = reinterpret_cast<unsigned long long *>(ws + L.best);
    a.known = ws + L.known;
    a.front_a = reinterpret_cast<int32_t *>(ws + L.front_a);
    a.front_b = reinterpret_cast<int32_t *>(ws + L.front_b);
    a.touched = reinterpret_cast<int32_t *>(ws + L.touched);
    a.lvl_o = reinterpret_cast<int32_t *>(ws + L.lvl_o);
    a.lvl_v = reinterpret_cast<int32_t *>(ws + L.lvl_v);
    a.pair_f = reinterpret_cast<int32_t *>(ws + L.pair_f);
    a.pair_g = reinterpret_cast<int32_t *>(ws + L.pair_g);
    a.level_off = reinterpret_cast<int32_t *>(ws + L.level_off);
    a.level_r0 = reinterpret_cast<int32_t *>(ws + L.level_r0);
    a.level_s0 = reinterpret_cast<int32_t *>(ws + L.level_s0);
    a.recipe_off = reinterpret_cast<int32_t *>(ws + L.recipe_off);
    a.seg_off = reinterpret_cast<int32_t *>(ws + L.seg_off);
    a.acc_slot = reinterpret_cast<int32_t *>(ws + L.acc_slot);
    a.seg_pair = reinterpret_cast<int32_t *>(ws + L.seg_pair);
    a.recipe_h = reinterpret_cast<int32_t *>(ws + L.recipe_h);
    a.unrec_list = reinterpret_cast<int32_t *>(ws + L.unrec_list);
    a.hdr = reinterpret_cast<int32_t *>(ws);
    a.unrecovered = unrecovered;
    a.n_unrecovered = n_unrecovered;
    const size_t dyn = (size_t)a.pl.bytes;
    if (dyn > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_dpg, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)dyn);
        if (e != cudaSuccess) return e;
    }
    k_dpg<<<1, kDpgThreads, dyn, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_peel(const fs_code *c, const uint4 *coded, uint4 *data_out, uint8_t *ws,
                        cudaStream_t s) {
    const DecodeLayout L = decode_layout(c);
    PeelArgs a;
    a.coded = coded;
    a.data = data_out;
    a.parity = reinterpret_cast<uint4 *>(ws + L.parity);
    a.pair_f = reinterpret_cast<const int32_t *>(ws + L.pair_f);
    a.pair_g = reinterpret_cast<const int32_t *>(ws + L.pair_g);
    a.level_off = reinterpret_cast<const int32_t *>(ws + L.level_off);
    a.level_r0 = reinterpret_cast<const int32_t *>(ws + L.level_r0);
    a.level_s0 = reinterpret_cast<const int32_t *>(ws + L.level_s0);
    a.recipe_off = reinterpret_cast<const int32_t *>(ws + L.recipe_off);
    a.seg_off = reinterpret_cast<const int32_t *>(ws + L.seg_off);
    a.acc_slot = reinterpret_cast<const int32_t *>(ws + L.acc_slot);
    a.seg_pair = reinterpret_cast<const int32_t *>(ws + L.seg_pair);
    a.recipe_h = reinterpret_cast<const int32_t *>(ws + L.recipe_h);
    a.unrec_list = reinterpret_cast<const int32_t *>(ws + L.unrec_list);
    a.hdr = reinterpret_cast<const int32_t *>(ws);
    a.b = c->b;
    a.n = c->n;
    a.tw = c->tw;
    // slice width: every slice in flight at once (peel_ctas CTAs per SM),
    // a whole number of word pairs, at most kPeelLmax words
    const int64_t ctas = (int64_t)c->num_sms * c->peel_ctas;
    int64_t Lw = (c->tw + ctas - 1) / ctas;
    Lw = (Lw + kPeelV - 1) / kPeelV * kPeelV;
    if (Lw > kPeelLmax) Lw = kPeelLmax;
    if (Lw < kPeelV) Lw = kPeelV;
    a.L = (int32_t)Lw;
    cudaError_t e =
        cudaFuncSetAttribute(k_peel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPeelSmem);
    if (e != cudaSuccess) return e;
    const int64_t n_slices = (c->tw + Lw - 1) / Lw;
    k_peel<<<(unsigned)n_slices, kPeelThreads, kPeelSmem, s>>>(a);
    return cudaGetLastError();
}
