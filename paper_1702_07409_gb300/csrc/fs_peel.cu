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
//        scan places its recipe (the row of g), its gather segments and its
//        accumulator slot;
//     C. one thread per new pair walks the constraints that contain f
//        (res -= 1, xs ^= f); a constraint whose count goes 2 -> 1 joins the
//        next frontier.
//   res/xs only change in C, after every bid of the level was placed, so a
//   level uses only symbols decoded in earlier levels (Section 3.1, first
//   rule). Appends to the shared lists are warp-aggregated.
//
// k_peel: the payload. Each CTA owns one slice of L 16-byte words of every
//   block (about one CTA per SM, so every slice is in flight at once) and
//   walks all levels; pairs of a level are independent (no intermediate is
//   written twice and none is read in the level that writes it), so a
//   __syncthreads between levels is the only ordering needed: no grid-wide
//   synchronisation and no per-level launch. Pair metadata is staged into
//   shared memory three levels ahead and recipes (rows of the joint graph)
//   two levels ahead with cp.async; the coded payloads and gathered blocks of
//   the next level are bulk-prefetched into L2 one level ahead. A recipe is
//   gathered in segments of at most kRecipeSeg blocks, one thread per
//   (segment, word pair), all loads of a segment in flight at once; pairs
//   with several segments combine them in shared-memory accumulators.
//   Precode checks are not gathered at all when their slices fit in shared
//   memory: each CTA keeps, per check j, S_j = XOR of the members of j
//   recovered so far (a recovered block is XORed into the accumulators of its
//   checks as soon as it is produced). When check j decodes f, every other
//   member is known, so x_f = S_j: one shared-memory read instead of a
//   gather of the whole row. Within a level no accumulator is both read and
//   updated: a member recovered in the level would be a second unknown of the
//   check that reads it.

#include <cooperative_groups.h>

#include "fs_internal.cuh"

namespace cg = cooperative_groups;

namespace {

constexpr int kDpgThreads = 256;
constexpr int kPeelThreads = 512;
constexpr int kPeelV = 2;           // 16-byte words per payload item
constexpr int kPeelLmax = 64;       // largest slice (words) of one payload CTA
constexpr int kStagePairs = 256;    // pairs of one level held in shared memory
constexpr int kStageRecipe = 2048;  // recipe entries of one level held in shared memory
constexpr int kStageLevels = 1024;  // level bounds held in shared memory
constexpr int kStageSegs = 512;     // gather segments of one level
constexpr int kStageMulti = 32;     // pairs with several segments in one level
constexpr size_t kChkAccBytes = 96 * 1024;  // largest shared-memory check accumulator
// one pair stage: f[P], g[P], e0[P], slot[P], ro[P+1], so[P+1], sp[S]
constexpr int kMF = 0, kMG = kStagePairs, kME = 2 * kStagePairs, kMSL = 3 * kStagePairs,
              kMRO = 4 * kStagePairs, kMSO = 5 * kStagePairs + 1, kMSP = 6 * kStagePairs + 2;
constexpr int kPairInts = kMSP + kStageSegs;
constexpr unsigned long long kEmpty = ~0ull;

// Shared-memory placement of the DPG arrays: byte offsets into dynamic shared
// memory, or -1 for the workspace (global) copy.
struct DpgPlace {
    int32_t res, xs, best, known, front, next, touched, cptr, vptr, ok;
    int32_t bytes;
};

struct DpgArgs {
    const int32_t *con_ptr, *con_xs, *var_ptr, *var_idx;
    const uint8_t *erased;
    int32_t b, n, k_int, n_con;
    int two_pass;
    DpgPlace pl;
    // workspace copies of the state (used where pl.* == -1)
    int32_t *res, *xs;
    unsigned long long *best;
    uint8_t *known;
    int32_t *front_a, *front_b, *touched;
    // outputs
    int32_t *pair_f, *pair_g, *pair_e0, *level_off, *level_r0, *level_s0, *recipe_off, *seg_off,
        *acc_slot, *seg_pair, *unrec_list, *hdr;
    uint8_t *unrecovered;
    int32_t *n_unrecovered;
};

// stage: -1 joint (every surviving coded row and every check), 0 coded rows
// only, 1 checks only (two-pass mode, Section 2.2). ok: survival flags in
// shared memory, or null to read the erasure flags.
__device__ __forceinline__ bool usable(const DpgArgs &a, const uint8_t *ok, int32_t g, int stage) {
    if (g < a.n) return stage <= 0 && (ok ? ok[g] != 0 : a.erased[g] == 0);
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

// Block-wide exclusive prefix sum of three counters at once; *total receives
// the sums. All threads of the block must call it.
__device__ int3 block_excl_scan3(int3 x, int3 *total, int3 *s_warp) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    int3 v = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int a = __shfl_up_sync(0xffffffffu, v.x, o);
        const int b = __shfl_up_sync(0xffffffffu, v.y, o);
        const int c = __shfl_up_sync(0xffffffffu, v.z, o);
        if (lane >= o) {
            v.x += a;
            v.y += b;
            v.z += c;
        }
    }
    if (lane == 31) s_warp[wid] = v;
    __syncthreads();
    if (wid == 0) {
        int3 s = lane < nw ? s_warp[lane] : make_int3(0, 0, 0);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int a = __shfl_up_sync(0xffffffffu, s.x, o);
            const int b = __shfl_up_sync(0xffffffffu, s.y, o);
            const int c = __shfl_up_sync(0xffffffffu, s.z, o);
            if (lane >= o) {
                s.x += a;
                s.y += b;
                s.z += c;
            }
        }
        s_warp[lane] = s;  // inclusive warp totals
    }
    __syncthreads();
    const int3 before = wid > 0 ? s_warp[wid - 1] : make_int3(0, 0, 0);
    *total = s_warp[nw - 1];
    __syncthreads();
    return make_int3(before.x + v.x - x.x, before.y + v.y - x.y, before.z + v.z - x.z);
}

// Block-wide exclusive prefix sum of four counters at once.
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
    __shared__ int3 s_warp3[32];
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
    const int32_t *cptr = place(smem, a.pl.cptr, const_cast<int32_t *>(a.con_ptr));
    const int32_t *vptr = place(smem, a.pl.vptr, const_cast<int32_t *>(a.var_ptr));
    // ok[g]: coded row g survived (erasure flags copied once; checks always 1)
    uint8_t *ok = a.pl.ok >= 0 ? smem + a.pl.ok : nullptr;

    if (tid == 0) a.hdr[WS_STATUS] = FS_OK;
    // the transposed graph is read once per decoded symbol: warm L2 with it
    {
        const char *p0 = reinterpret_cast<const char *>(a.var_idx);
        const int64_t bytes = (int64_t)__ldg(a.var_ptr + K) * 4;
        for (int64_t o = (int64_t)tid * 4096; o < bytes; o += (int64_t)T * 4096) {
            const int64_t len = min((int64_t)4096, bytes - o) & ~(int64_t)15;
            if (len > 0 && ((reinterpret_cast<uintptr_t>(p0 + o) & 15) == 0))
                asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(p0 + o),
                             "r"((uint32_t)len)
                             : "memory");
        }
    }
    if (ok)
        for (int32_t g = tid; g < G; g += T) ok[g] = (g < a.n) ? (a.erased[g] == 0) : 1;
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
        if (usable(a, ok, g, stage) && res[g] == 1) front[append_slot(&s_nf)] = g;
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
        // segments (y) and accumulator slots (z)
        int3 len = make_int3(0, 0, 0);
        for (int base = 0; base < nt; base += T) {
            const int i = base + tid;
            int3 cnt = make_int3(0, 0, 0);
            int32_t f = -1, g = -1;
            if (i < nt) {
                f = touched[i];
                const unsigned long long key = best[f];
                g = (int32_t)(key & 0xffffffffull);
                cnt.x = (int32_t)(key >> 32);
                cnt.y = (cnt.x + kRecipeSeg - 1) / kRecipeSeg;
                cnt.z = cnt.y > 1 ? 1 : 0;
                best[f] = kEmpty;
                known[f] = 1;
            }
            int3 total;
            const int3 off = block_excl_scan3(cnt, &total, s_warp3);
            if (i < nt) {
                const int32_t p = np + i;
                a.pair_f[p] = f;
                a.pair_g[p] = g;
                a.pair_e0[p] = cptr[g];
                a.recipe_off[p] = rb + len.x + off.x;
                a.seg_off[p] = sb + len.y + off.y;
                a.acc_slot[p] = cnt.z ? len.z + off.z : -1;
                for (int k = 0; k < cnt.y; ++k) a.seg_pair[sb + len.y + off.y + k] = i;
            }
            len.x += total.x;
            len.y += total.y;
            len.z += total.z;
        }
        // C: one thread per pair updates the constraints containing its symbol
        for (int i = tid; i < nt; i += T) {
            const int32_t f = touched[i];
            const int32_t v1 = vptr[f + 1];
            int32_t e = vptr[f];
            for (; e + 4 <= v1; e += 4) {
                int32_t c[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) c[j] = __ldg(a.var_idx + e + j);
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    atomicXor(xs + c[j], f);
                    if (atomicSub(res + c[j], 1) == 2 && usable(a, ok, c[j], stage))
                        next[append_slot(&s_nnext)] = c[j];
                }
            }
            for (; e < v1; ++e) {
                const int32_t c = __ldg(a.var_idx + e);
                atomicXor(xs + c, f);
                if (atomicSub(res + c, 1) == 2 && usable(a, ok, c, stage)) next[append_slot(&s_nnext)] = c;
            }
        }
        __syncthreads();
        if (tid == 0) {
            s_nf = s_nnext;
            maxp = max(maxp, nt);
            maxr = max(maxr, len.x);
            maxs = max(maxs, len.y);
            maxm = max(maxm, len.z);
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

// Compact DPG for graphs with at most 65536 intermediates and constraints:
// the same algorithm with every per-level access in shared memory. Indices
// are 16-bit, res and xs share one word (res << 16 | xs: a decrement touches
// only the high half, the XOR only the low half), keys are 32-bit
// (degree << 16 | g), and the transposed graph is copied to shared memory, so
// a level makes no global load. Step C runs one thread per adjacency slot
// (the slots of the level's symbols are placed by the same scan as the
// recipes), so no thread walks a whole adjacency list.
struct DpgCompactPlace {
    int32_t best, pk, front, next, touched, known, cptr, vptr, vidx, ok, lvl_v, bytes;
};

__global__ void __launch_bounds__(kDpgThreads, 1) k_dpg_compact(DpgArgs a, DpgCompactPlace pl) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int4 s_warp4[32];
    __shared__ int s_nf, s_nt, s_nnext, s_cnt, s_cnt_data;
    constexpr uint32_t kE = 0xffffffffu;

    const int tid = threadIdx.x, T = blockDim.x;
    const int32_t K = a.k_int, G = a.n_con;
    uint32_t *best = reinterpret_cast<uint32_t *>(smem + pl.best);
    uint32_t *pk = reinterpret_cast<uint32_t *>(smem + pl.pk);
    uint16_t *front = reinterpret_cast<uint16_t *>(smem + pl.front);
    uint16_t *next = reinterpret_cast<uint16_t *>(smem + pl.next);
    uint16_t *touched = reinterpret_cast<uint16_t *>(smem + pl.touched);
    uint8_t *known = smem + pl.known;
    int32_t *cptr = reinterpret_cast<int32_t *>(smem + pl.cptr);
    int32_t *vptr = reinterpret_cast<int32_t *>(smem + pl.vptr);
    uint16_t *vidx = reinterpret_cast<uint16_t *>(smem + pl.vidx);
    uint8_t *ok = smem + pl.ok;
    int32_t *lvl_v = reinterpret_cast<int32_t *>(smem + pl.lvl_v);  // adjacency slots per pair

    if (tid == 0) a.hdr[WS_STATUS] = FS_OK;
    for (int32_t g = tid; g <= G; g += T) cptr[g] = __ldg(a.con_ptr + g);
    for (int32_t v = tid; v <= K; v += T) vptr[v] = __ldg(a.var_ptr + v);
    const int32_t e_con = __ldg(a.var_ptr + K);
    for (int32_t e = tid; e < e_con; e += T) vidx[e] = (uint16_t)__ldg(a.var_idx + e);
    for (int32_t v = tid; v < K; v += T) {
        known[v] = 0;
        best[v] = kE;
    }
    for (int32_t g = tid; g < G; g += T) {
        const uint32_t deg = (uint32_t)(__ldg(a.con_ptr + g + 1) - __ldg(a.con_ptr + g));
        pk[g] = (deg << 16) | ((uint32_t)__ldg(a.con_xs + g) & 0xffffu);
        ok[g] = (g < a.n) ? (a.erased[g] == 0) : 1;
    }
    int stage = a.two_pass ? 0 : -1;
    if (tid == 0) s_nf = 0;
    __syncthreads();
    for (int32_t g = tid; g < G; g += T)
        if (usable(a, ok, g, stage) && (pk[g] >> 16) == 1) front[append_slot(&s_nf)] = (uint16_t)g;
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
            const uint32_t w = pk[g];
            if ((w >> 16) != 1) continue;  // its unknown was decoded by another constraint
            const int32_t f = (int32_t)(w & 0xffffu);
            const uint32_t key = ((uint32_t)(cptr[g + 1] - cptr[g]) << 16) | (uint32_t)g;
            if (atomicMin(best + f, key) == kE) touched[append_slot(&s_nt)] = (uint16_t)f;
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
                if ((pk[g] >> 16) == 1) front[append_slot(&s_nf)] = (uint16_t)g;
            __syncthreads();
            continue;
        }
        if (tid == 0) {
            a.level_off[level] = np;
            a.level_r0[level] = rb;
            a.level_s0[level] = sb;
        }
        // B: pairs of the level; one scan places recipes (x), gather
        // segments (y), accumulator slots (z) and adjacency slots (w)
        int4 len = make_int4(0, 0, 0, 0);
        for (int base = 0; base < nt; base += T) {
            const int i = base + tid;
            int4 cnt = make_int4(0, 0, 0, 0);
            int32_t f = -1, g = -1;
            if (i < nt) {
                f = touched[i];
                const uint32_t key = best[f];
                g = (int32_t)(key & 0xffffu);
                cnt.x = (int32_t)(key >> 16);
                cnt.y = (cnt.x + kRecipeSeg - 1) / kRecipeSeg;
                cnt.z = cnt.y > 1 ? 1 : 0;
                cnt.w = vptr[f + 1] - vptr[f];
                best[f] = kE;
                known[f] = 1;
            }
            int4 total;
            const int4 off = block_excl_scan4(cnt, &total, s_warp4);
            if (i < nt) {
                const int32_t p = np + i;
                a.pair_f[p] = f;
                a.pair_g[p] = g;
                a.pair_e0[p] = cptr[g];
                a.recipe_off[p] = rb + len.x + off.x;
                a.seg_off[p] = sb + len.y + off.y;
                a.acc_slot[p] = cnt.z ? len.z + off.z : -1;
                for (int k = 0; k < cnt.y; ++k) a.seg_pair[sb + len.y + off.y + k] = i;
                lvl_v[i] = len.w + off.w;
            }
            len.x += total.x;
            len.y += total.y;
            len.z += total.z;
            len.w += total.w;
        }
        if (tid == 0) lvl_v[nt] = len.w;
        __syncthreads();
        // C: one thread per adjacency slot (its pair found by binary search)
        // updates one constraint containing a newly decoded symbol
        for (int32_t u = tid; u < len.w; u += T) {
            const int i = find_slot(lvl_v, nt, u);
            const int32_t f = touched[i];
            const int32_t c = vidx[vptr[f] + (u - lvl_v[i])];
            atomicXor(pk + c, (uint32_t)f);
            if ((atomicSub(pk + c, 1u << 16) >> 16) == 2 && usable(a, ok, c, stage))
                next[append_slot(&s_nnext)] = (uint16_t)c;
        }
        __syncthreads();
        if (tid == 0) {
            s_nf = s_nnext;
            maxp = max(maxp, nt);
            maxr = max(maxr, len.x);
            maxs = max(maxs, len.y);
            maxm = max(maxm, len.z);
        }
        uint16_t *tmp = front;
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

// Shared-memory layout of k_dpg_compact, or bytes = -1 when the code does not
// qualify (sizes beyond 16-bit indices, or more than the shared memory).
DpgCompactPlace plan_dpg_compact(const fs_code *c) {
    DpgCompactPlace p;
    p.bytes = -1;
    const int64_t K = c->k_int, G = c->n_con;
    if (K > 65536 || G > 65536 || c->max_con_deg > 65535) return p;
    int64_t o = 0;
    auto take = [&](int64_t bytes) {
        const int64_t at = o;
        o = (o + bytes + 15) & ~(int64_t)15;
        return (int32_t)at;
    };
    p.best = take(4 * (K + 1));
    p.pk = take(4 * (G + 1));
    p.cptr = take(4 * (G + 1));
    p.vptr = take(4 * (K + 1));
    p.lvl_v = take(4 * (K + 1));
    p.front = take(2 * (G + 1));
    p.next = take(2 * (G + 1));
    p.touched = take(2 * (K + 1));
    p.vidx = take(2 * (c->e_con + 1));
    p.known = take(K + 1);
    p.ok = take(G + 1);
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
    const int32_t *con_idx, *chk_ptr, *chk_idx;
    const int32_t *pair_f, *pair_g, *pair_e0, *level_off, *level_r0, *level_s0, *recipe_off,
        *seg_off, *acc_slot, *seg_pair, *unrec_list, *hdr;
    int32_t b, m, n;
    int64_t tw;
    int32_t L;        // words of every block per CTA
    int32_t chk_acc;  // 1: checks decode from shared-memory accumulators
    int32_t chk_smem; // 1: the check lists are copied to shared memory
    int32_t pf_gather; // 1: gathered blocks of the next level are prefetched into L2
    int32_t k_int, e_chk;
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

__device__ __forceinline__ void xor_shared(uint4 *d, const uint4 &v) {
    uint32_t *w = reinterpret_cast<uint32_t *>(d);
    atomicXor(w + 0, v.x);
    atomicXor(w + 1, v.y);
    atomicXor(w + 2, v.z);
    atomicXor(w + 3, v.w);
}

// XORs word `word` of a recovered block f into the accumulators of its
// checks (cptr / cidx: the check lists, in shared or global memory).
__device__ __forceinline__ void add_to_checks(const PeelArgs &a, const int32_t *cptr,
                                              const int32_t *cidx, uint4 *sacc, int32_t f,
                                              int word, const uint4 &v0, const uint4 &v1,
                                              bool two) {
    const int32_t e1 = cptr[f + 1];
    for (int32_t e = cptr[f]; e < e1; ++e) {
        uint4 *d = sacc + (int64_t)cidx[e] * a.L + word;
        xor_shared(d, v0);
        if (two) xor_shared(d + 1, v1);
    }
}

// Largest q in [0, n) with off[q] - base <= x, for off[0] - base <= x.
__device__ __forceinline__ int find_pair(const int32_t *off, int n, int32_t base, int32_t x) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] - base <= x) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Levels read straight from global memory (used when a level does not fit
// the shared-memory stages): one thread per (pair, word).
__device__ void peel_direct(const PeelArgs &a, int64_t w0, int lanes) {
    const int32_t n_levels = a.hdr[WS_N_LEVELS];
    for (int32_t l = 0; l < n_levels; ++l) {
        const int32_t p0 = a.level_off[l], p1 = a.level_off[l + 1];
        const int32_t items = (p1 - p0) * lanes;
        for (int32_t it = threadIdx.x; it < items; it += blockDim.x) {
            const int32_t q = it / lanes, lane = it - q * lanes;
            const int32_t p = p0 + q;
            const int32_t f = a.pair_f[p], g = a.pair_g[p];
            const int32_t e0 = a.pair_e0[p], deg = a.recipe_off[p + 1] - a.recipe_off[p];
            const int64_t w = w0 + lane;
            uint4 acc = make_uint4(0, 0, 0, 0);
            if (g < a.n) acc = __ldg(a.coded + (int64_t)g * a.tw + w);
            for (int32_t r = 0; r < deg; ++r) {
                const int32_t h = __ldg(a.con_idx + e0 + r);
                if (h != f) xor4(acc, block_ptr(a, h)[w]);
            }
            block_ptr(a, f)[w] = acc;
        }
        __syncthreads();
    }
}

__device__ __forceinline__ void stage_pairs(const PeelArgs &a, int32_t *pb, const int32_t *lv_p,
                                            const int32_t *lv_s, int l) {
    const int32_t p0 = lv_p[l], np = lv_p[l + 1] - p0;
    const int32_t s0 = lv_s[l], ns = lv_s[l + 1] - s0;
    for (int i = threadIdx.x; i < np; i += blockDim.x) {
        cp_async4(pb + kMF + i, a.pair_f + p0 + i);
        cp_async4(pb + kMG + i, a.pair_g + p0 + i);
        cp_async4(pb + kME + i, a.pair_e0 + p0 + i);
        cp_async4(pb + kMSL + i, a.acc_slot + p0 + i);
    }
    for (int i = threadIdx.x; i <= np; i += blockDim.x) {
        cp_async4(pb + kMRO + i, a.recipe_off + p0 + i);
        cp_async4(pb + kMSO + i, a.seg_off + p0 + i);
    }
    for (int i = threadIdx.x; i < ns; i += blockDim.x) cp_async4(pb + kMSP + i, a.seg_pair + s0 + i);
}

// Rows of the level's constraints into rb (pair metadata pb already staged),
// one thread per entry. With check accumulators, check rows are not needed.
__device__ __forceinline__ void stage_recipes(const PeelArgs &a, int32_t *rb, const int32_t *pb,
                                              int np, int32_t r0, int32_t nr) {
    for (int r = threadIdx.x; r < nr; r += blockDim.x) {
        const int q = find_pair(pb + kMRO, np, r0, r);
        if (a.chk_acc && pb[kMG + q] >= a.n) continue;
        cp_async4(rb + r, a.con_idx + pb[kME + q] + (r - (pb[kMRO + q] - r0)));
    }
}

// L2 prefetch of what a level reads from global memory: its coded payload
// slices and the slices of its recipe blocks (one thread per entry).
__device__ __forceinline__ void prefetch_level(const PeelArgs &a, const int32_t *pb,
                                               const int32_t *rb, int np, int32_t r0, int32_t nr,
                                               int64_t w0, int lanes) {
    const uint32_t bytes = (uint32_t)lanes * 16u;
    const int n_items = a.pf_gather ? np + nr : np;
    for (int i = threadIdx.x; i < n_items; i += blockDim.x) {
        if (i < np) {
            const int32_t g = pb[kMG + i];
            if (g < a.n) prefetch_l2(a.coded + (int64_t)g * a.tw + w0, bytes);
            continue;
        }
        const int r = i - np;
        const int q = find_pair(pb + kMRO, np, r0, r);
        if (a.chk_acc && pb[kMG + q] >= a.n) continue;
        const int32_t h = rb[r];
        if (h != pb[kMF + q]) prefetch_l2(block_ptr(a, h) + w0, bytes);
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
        uint4 *accs = reinterpret_cast<uint4 *>(smem);      // [kStageMulti][L]
        uint4 *sacc = accs + kStageMulti * L;               // [m][L] when chk_acc
        int32_t *lv_p = reinterpret_cast<int32_t *>(sacc + (a.chk_acc ? (int64_t)a.m * L : 0));
        int32_t *lv_r = lv_p + kStageLevels + 1;
        int32_t *lv_s = lv_r + kStageLevels + 1;
        int32_t *pairs = lv_s + kStageLevels + 1;  // [4][kPairInts]
        int32_t *recs = pairs + 4 * kPairInts;     // [3][kStageRecipe]
        int32_t *s_cptr = recs + 3 * kStageRecipe;  // [k_int + 1] when chk_smem
        int32_t *s_cidx = s_cptr + a.k_int + 1;     // [e_chk]
        const int32_t *cptr = a.chk_ptr, *cidx = a.chk_idx;
        if (a.chk_smem) {
            for (int i = threadIdx.x; i <= a.k_int; i += blockDim.x) s_cptr[i] = __ldg(a.chk_ptr + i);
            for (int i = threadIdx.x; i < a.e_chk; i += blockDim.x) s_cidx[i] = __ldg(a.chk_idx + i);
            cptr = s_cptr;
            cidx = s_cidx;
        }
        for (int i = threadIdx.x; i <= nl; i += blockDim.x) {
            lv_p[i] = a.level_off[i];
            lv_r[i] = a.level_r0[i];
            lv_s[i] = a.level_s0[i];
        }
        for (int i = threadIdx.x; i < kStageMulti * L; i += blockDim.x)
            accs[i] = make_uint4(0, 0, 0, 0);
        if (a.chk_acc)
            for (int64_t i = threadIdx.x; i < (int64_t)a.m * L; i += blockDim.x)
                sacc[i] = make_uint4(0, 0, 0, 0);
        __syncthreads();
        // prologue: pairs of levels 0..2, recipes of levels 0..1, prefetch of level 0
        for (int l = 0; l < 3 && l < nl; ++l) stage_pairs(a, pairs + l * kPairInts, lv_p, lv_s, l);
        cp_async_commit();
        cp_async_wait_all();
        __syncthreads();
        for (int l = 0; l < 2 && l < nl; ++l)
            stage_recipes(a, recs + l * kStageRecipe, pairs + l * kPairInts, lv_p[l + 1] - lv_p[l],
                          lv_r[l], lv_r[l + 1] - lv_r[l]);
        cp_async_commit();
        cp_async_wait_all();
        __syncthreads();
        if (nl > 0)
            prefetch_level(a, pairs, recs, lv_p[1] - lv_p[0], lv_r[0], lv_r[1] - lv_r[0], w0, lanes);
        for (int32_t l = 0; l < nl; ++l) {
            const int32_t *pc = pairs + (l & 3) * kPairInts;
            const int32_t *hs = recs + (l % 3) * kStageRecipe;
            // pipeline: pairs of l+3, recipes of l+2, L2 prefetch of l+1
            if (l + 3 < nl) stage_pairs(a, pairs + ((l + 3) & 3) * kPairInts, lv_p, lv_s, l + 3);
            if (l + 2 < nl)
                stage_recipes(a, recs + ((l + 2) % 3) * kStageRecipe,
                              pairs + ((l + 2) & 3) * kPairInts, lv_p[l + 3] - lv_p[l + 2],
                              lv_r[l + 2], lv_r[l + 3] - lv_r[l + 2]);
            cp_async_commit();
            if (l + 1 < nl)
                prefetch_level(a, pairs + ((l + 1) & 3) * kPairInts,
                               recs + ((l + 1) % 3) * kStageRecipe, lv_p[l + 2] - lv_p[l + 1],
                               lv_r[l + 1], lv_r[l + 2] - lv_r[l + 1], w0, lanes);
            const int np = lv_p[l + 1] - lv_p[l];
            const int ns = lv_s[l + 1] - lv_s[l];
            const int32_t r0 = lv_r[l], s0 = lv_s[l];
            // every (segment, word pair): one gather of at most kRecipeSeg blocks
            for (int it = threadIdx.x; it < ns * nv; it += blockDim.x) {
                const int s = it / nv, k = it - s * nv;
                const int q = pc[kMSP + s];
                const int32_t f = pc[kMF + q], g = pc[kMG + q];
                const int sidx = s - (pc[kMSO + q] - s0);
                const int64_t w = w0 + k * kPeelV;
                const bool two = k * kPeelV + 1 < lanes;
                uint4 acc0 = make_uint4(0, 0, 0, 0), acc1 = acc0;
                if (a.chk_acc && g >= a.n) {
                    // check g - n decodes f: every other member is in its accumulator
                    if (sidx != 0) continue;
                    const uint4 *src = sacc + (int64_t)(g - a.n) * L + k * kPeelV;
                    acc0 = src[0];
                    if (two) acc1 = src[1];
                } else {
                    const int32_t rs = pc[kMRO + q] - r0 + sidx * kRecipeSeg;
                    const int32_t cnt = min(kRecipeSeg, pc[kMRO + q + 1] - r0 - rs);
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
                    const int slot = pc[kMSL + q];
                    if (slot >= 0) {  // one of several segments: combine in shared memory
                        xor_shared(accs + slot * L + k * kPeelV, acc0);
                        if (two) xor_shared(accs + slot * L + k * kPeelV + 1, acc1);
                        continue;
                    }
                }
                uint4 *dst = block_ptr(a, f) + w;
                dst[0] = acc0;
                if (two) dst[1] = acc1;
                if (a.chk_acc) add_to_checks(a, cptr, cidx, sacc, f, k * kPeelV, acc0, acc1, two);
            }
            if (ns > np) {  // some pair has several segments: write their sums
                __syncthreads();
                for (int it = threadIdx.x; it < np * lanes; it += blockDim.x) {
                    const int q = it / lanes, lane = it - q * lanes;
                    const int slot = pc[kMSL + q];
                    if (slot < 0 || (a.chk_acc && pc[kMG + q] >= a.n)) continue;
                    const int32_t f = pc[kMF + q];
                    const uint4 v = accs[slot * L + lane];
                    block_ptr(a, f)[w0 + lane] = v;
                    accs[slot * L + lane] = make_uint4(0, 0, 0, 0);
                    if (a.chk_acc) add_to_checks(a, cptr, cidx, sacc, f, lane, v, v, false);
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

size_t peel_smem_bytes(int64_t L, int64_t chk_acc_bytes, int64_t chk_list_bytes) {
    return (size_t)kStageMulti * L * 16 + (size_t)chk_acc_bytes +
           (size_t)3 * (kStageLevels + 1) * 4 + (size_t)4 * kPairInts * 4 +
           (size_t)3 * kStageRecipe * 4 + (size_t)chk_list_bytes;
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
    // graph row pointers, each where room is left
    p.cptr = (o + 4 * G <= budget) ? take(4 * G) : -1;
    p.vptr = (o + 4 * K <= budget) ? take(4 * K) : -1;
    p.ok = (o + G <= budget) ? take(G) : -1;
    p.bytes = (int32_t)o;
    return p;
}

}  // namespace

cudaError_t launch_dpg(const fs_code *c, const uint8_t *erased, uint8_t *ws, uint8_t *unrecovered,
                       int32_t *n_unrecovered, cudaStream_t s) {
    const DecodeLayout L = decode_layout(c);
    DpgArgs a;
    a.con_ptr = c->con_ptr;
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
    a.pair_f = reinterpret_cast<int32_t *>(ws + L.pair_f);
    a.pair_g = reinterpret_cast<int32_t *>(ws + L.pair_g);
    a.pair_e0 = reinterpret_cast<int32_t *>(ws + L.pair_e0);
    a.level_off = reinterpret_cast<int32_t *>(ws + L.level_off);
    a.level_r0 = reinterpret_cast<int32_t *>(ws + L.level_r0);
    a.level_s0 = reinterpret_cast<int32_t *>(ws + L.level_s0);
    a.recipe_off = reinterpret_cast<int32_t *>(ws + L.recipe_off);
    a.seg_off = reinterpret_cast<int32_t *>(ws + L.seg_off);
    a.acc_slot = reinterpret_cast<int32_t *>(ws + L.acc_slot);
    a.seg_pair = reinterpret_cast<int32_t *>(ws + L.seg_pair);
    a.unrec_list = reinterpret_cast<int32_t *>(ws + L.unrec_list);
    a.hdr = reinterpret_cast<int32_t *>(ws);
    a.unrecovered = unrecovered;
    a.n_unrecovered = n_unrecovered;
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
    a.con_idx = c->con_idx;
    a.chk_ptr = c->chk_ptr;
    a.chk_idx = c->chk_idx;
    a.pair_f = reinterpret_cast<const int32_t *>(ws + L.pair_f);
    a.pair_g = reinterpret_cast<const int32_t *>(ws + L.pair_g);
    a.pair_e0 = reinterpret_cast<const int32_t *>(ws + L.pair_e0);
    a.level_off = reinterpret_cast<const int32_t *>(ws + L.level_off);
    a.level_r0 = reinterpret_cast<const int32_t *>(ws + L.level_r0);
    a.level_s0 = reinterpret_cast<const int32_t *>(ws + L.level_s0);
    a.recipe_off = reinterpret_cast<const int32_t *>(ws + L.recipe_off);
    a.seg_off = reinterpret_cast<const int32_t *>(ws + L.seg_off);
    a.acc_slot = reinterpret_cast<const int32_t *>(ws + L.acc_slot);
    a.seg_pair = reinterpret_cast<const int32_t *>(ws + L.seg_pair);
    a.unrec_list = reinterpret_cast<const int32_t *>(ws + L.unrec_list);
    a.hdr = reinterpret_cast<const int32_t *>(ws);
    a.b = c->b;
    a.m = c->m;
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
    const int64_t acc_bytes = (int64_t)c->m * Lw * 16;
    a.chk_acc = (c->m > 0 && c->peel_chk_acc && (size_t)acc_bytes <= kChkAccBytes) ? 1 : 0;
    a.pf_gather = c->peel_prefetch;
    a.k_int = c->k_int;
    a.e_chk = (int32_t)(c->e_pre + c->m);
    const int64_t list_bytes = 4 * ((int64_t)c->k_int + 1 + a.e_chk);
    // shared memory of one CTA: its share when peel_ctas CTAs sit on an SM
    const size_t share = c->smem_optin / (size_t)c->peel_ctas - (c->peel_ctas > 1 ? 1024 : 0);
    const size_t base = peel_smem_bytes(Lw, a.chk_acc ? acc_bytes : 0, 0);
    a.chk_smem = (a.chk_acc && base + (size_t)list_bytes <= share) ? 1 : 0;
    const size_t smem =
        peel_smem_bytes(Lw, a.chk_acc ? acc_bytes : 0, a.chk_smem ? list_bytes : 0);
    // one CTA per SM: 512 threads; several: the SM's threads split between them
    const int threads = c->peel_ctas >= 4 ? 128 : (c->peel_ctas >= 2 ? 256 : kPeelThreads);
    cudaError_t e =
        cudaFuncSetAttribute(k_peel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t n_slices = (c->tw + Lw - 1) / Lw;
    k_peel<<<(unsigned)n_slices, threads, smem, s>>>(a);
    return cudaGetLastError();
}
