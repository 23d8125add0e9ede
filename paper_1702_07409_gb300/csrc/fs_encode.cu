// fs_encode.cu - encoding (Section 2.2, steps (1) precode and (2) LDGM).
//
// k_slices (the default when the code fits): one persistent CTA per SM takes
// byte slices of the stripe (16 or 32 bytes of every block) from a ticket
// counter. For a slice it loads that slice of every data block into
// shared-memory slots with 2-D TMA copies (a box is 16 or 32 bytes x up to
// 256 blocks) and computes every output row of the slice from the slots,
// one lane per row: first the m parity rows together with the coded rows
// that read no parity, then the coded rows that read one. Rows are packed
// into warp groups whose quarter warps (8 lanes) always read 8 distinct
// bank groups (rows chosen so their inputs spread over the groups, each
// quarter's inputs placed by an edge colouring), with the index tables in
// shared memory. Every gathered operand comes from shared memory: each
// input byte crosses DRAM once. Two slot buffers let the TMA copies of the
// next slice run under the arithmetic of the current one.
//
// k_rows (fallback for codes whose slice does not fit) in two launches:
// first the m precode rows (parities, over the data blocks), then the n LT
// rows (coded blocks, over the data blocks and parities). Stream order makes
// every parity final before an LT row reads it.
//
// Work is taken in tickets (byte chunk, batch of consecutive rows: one check
// row for the precode, kRows coded rows for LT),
// chunk-major, from a counter in the workspace, so the resident CTAs work on
// about one byte range of every block at a time (its inputs stay in L2 while
// the rows that share them are computed) and a CTA that starts late simply
// takes fewer tickets. A CTA stages the row pointers and the neighbour list
// of its tickets in shared memory with cp.async, two tickets ahead for the
// pointers and one for the lists, and walks the ticket's neighbour list
// eight entries at a time across row boundaries: every thread keeps 8
// neighbours x kEncV words of loads in flight whatever the row degrees, and
// a finished row is stored as soon as the walk passes its end. Coded rows
// are written with evict-first stores so L2 keeps the inputs.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <numeric>
#include <vector>

#include "fs_internal.cuh"

namespace {

constexpr int kEncThreads = 256;
constexpr int kEncV = 1;                      // words per thread per chunk
constexpr int kChunkW = kEncV * kEncThreads;  // 16-byte words per chunk (4 KiB)
constexpr int kRows = 16;                     // rows per ticket
constexpr int kStage = 2048;                  // neighbour entries of one ticket staged
constexpr int kCtasPerSm = 4;

}  // namespace

// One job of the row kernel: the rows of one CSR (one stripe's precode or
// LT rows) over its inputs; a launch runs one job or a batch of them.
struct RowArgs {
    const int32_t *ptr, *idx;  // CSR rows
    const uint4 *inA, *inB;    // input block v: inA + v*tw (v < split), else inB
    int32_t split;
    uint4 *out;
    int32_t n_rows;
    int64_t tw;
    int32_t n_chunks;
    int stream_out;       // 1: evict-first stores
    int32_t rows;         // rows per ticket (at most kRows)
    int hints;            // 1: inputs evict-last, outputs evict-first in L2
    int32_t t0;           // first ticket of this job in the launch's ticket order
};

namespace {

__device__ __forceinline__ void xor4(uint4 &a, const uint4 &b) {
    a.x ^= b.x;
    a.y ^= b.y;
    a.z ^= b.z;
    a.w ^= b.w;
}

__device__ __forceinline__ void cp_async4(void *sdst, const void *gsrc) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gsrc) : "memory");
}

__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}

// wait until at most N committed groups are still in flight
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

struct Ticket {
    int32_t chunk, r0, nr;  // byte chunk, first row, rows
};

__device__ __forceinline__ Ticket ticket_of(const RowArgs &a, int32_t t, int32_t batches) {
    Ticket k;
    k.chunk = t / batches;
    k.r0 = (t - k.chunk * batches) * a.rows;
    k.nr = min(a.rows, a.n_rows - k.r0);
    return k;
}

template <bool kHints>
__device__ __forceinline__ void store_row(const RowArgs &a, int32_t row, int64_t w0, int64_t w1,
                                          const uint4 *acc, uint64_t pol_out) {
    uint4 *out = a.out + (int64_t)row * a.tw;
#pragma unroll
    for (int v = 0; v < kEncV; ++v) {
        const int64_t w = w0 + threadIdx.x + (int64_t)v * kEncThreads;
        if (w >= w1) continue;
        if (kHints) st_hint(out + w, acc[v], pol_out);
        else if (a.stream_out) __stcs(out + w, acc[v]);
        else __stcg(out + w, acc[v]);
    }
}

// job of global ticket t: the last job whose first ticket is <= t
__device__ __forceinline__ int find_job(const RowArgs *jobs, int n_jobs, int32_t t) {
    int lo = 0, hi = n_jobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (jobs[mid].t0 <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Tickets run job by job (a stripe's chunks one after the other), so the
// resident CTAs work on one stripe's byte range at a time. kHints: L2
// eviction hints (FS_TUNE_L2_HINTS), a template parameter so the default
// path carries no per-load branch or policy registers for them.
template <bool kHints>
__device__ __forceinline__ void rows_body(const RowArgs *jobs, int n_jobs, int32_t n_tickets,
                                          int32_t *ticket_ctr) {
    // ring of 3 pointer stages (two tickets ahead), 2 neighbour stages, 4 tickets
    __shared__ int32_t s_ptr[3][kRows + 1];
    __shared__ int32_t s_idx[2][kStage];
    __shared__ int32_t s_tk[4], s_jb[4];

    auto take = [&](int slot, int32_t t) {  // thread 0: ticket t and its job into a slot
        s_tk[slot] = t;
        s_jb[slot] = t < n_tickets ? find_job(jobs, n_jobs, t) : 0;
    };
    auto stage_ptr = [&](int k, int slot) {
        const int32_t t = s_tk[k];
        if (t >= n_tickets) return;
        const RowArgs &a = jobs[s_jb[k]];
        const int32_t batches = (a.n_rows + a.rows - 1) / a.rows;
        const Ticket tk = ticket_of(a, t - a.t0, batches);
        for (int i = threadIdx.x; i <= tk.nr; i += blockDim.x)
            cp_async4(&s_ptr[slot][i], a.ptr + tk.r0 + i);
    };
    auto stage_idx = [&](int k, int pslot, int islot) {
        const int32_t t = s_tk[k];
        if (t >= n_tickets) return;
        const RowArgs &a = jobs[s_jb[k]];
        const int32_t batches = (a.n_rows + a.rows - 1) / a.rows;
        const int32_t e0 = s_ptr[pslot][0];
        const int32_t ne = s_ptr[pslot][ticket_of(a, t - a.t0, batches).nr] - e0;
        if (ne > kStage) return;  // read straight from global memory instead
        for (int i = threadIdx.x; i < ne; i += blockDim.x)
            cp_async4(&s_idx[islot][i], a.idx + e0 + i);
    };

    // prologue: three consecutive tickets, pointers of the first two, list of the first
    if (threadIdx.x == 0) {
        const int32_t t = atomicAdd(ticket_ctr, 3);
        for (int k = 0; k < 3; ++k) take(k, t + k);
    }
    __syncthreads();
    stage_ptr(0, 0);
    cp_async_commit();
    stage_ptr(1, 1);
    cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();
    stage_idx(0, 0, 0);
    cp_async_commit();
    for (int it = 0;; ++it) {
        // ticket it's list and ticket it+1's pointers are in
        cp_async_wait<0>();
        __syncthreads();
        const int32_t t = s_tk[it & 3];
        if (t >= n_tickets) break;  // this CTA's tickets increase: no later one is below the end
        const RowArgs &a = jobs[s_jb[it & 3]];
        const int ps = it % 3, is = it & 1;
        if (threadIdx.x == 0) take((it + 3) & 3, atomicAdd(ticket_ctr, 1));
        stage_ptr((it + 2) & 3, (it + 2) % 3);
        stage_idx((it + 1) & 3, (it + 1) % 3, (it + 1) & 1);
        cp_async_commit();

        const int32_t batches = (a.n_rows + a.rows - 1) / a.rows;
        const Ticket k = ticket_of(a, t - a.t0, batches);
        const int32_t *rp = s_ptr[ps];
        const int32_t e_base = rp[0], e_end = rp[k.nr];
        const int32_t *idx = (e_end - e_base <= kStage) ? s_idx[is] : a.idx + e_base;
        const int64_t w0 = (int64_t)k.chunk * kChunkW, w1 = min(w0 + kChunkW, a.tw);
        int64_t w[kEncV];
        bool ok[kEncV];
        uint4 acc[kEncV];
#pragma unroll
        for (int v = 0; v < kEncV; ++v) {
            w[v] = w0 + threadIdx.x + (int64_t)v * kEncThreads;
            ok[v] = w[v] < w1;
            acc[v] = make_uint4(0, 0, 0, 0);
        }
        const uint64_t pol_in = kHints ? l2_policy_last() : 0;
        const uint64_t pol_out = kHints ? (a.stream_out ? l2_policy_first() : l2_policy_last()) : 0;
        int r = 0;  // row being accumulated; entries [rp[r], rp[r + 1])
        for (int32_t e = e_base; e < e_end; e += 8) {
            uint4 x[8][kEncV];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const bool on = e + j < e_end;
                const int32_t v = on ? idx[e + j - e_base] : 0;
                const uint4 *src = v < a.split ? a.inA + (int64_t)v * a.tw
                                               : a.inB + (int64_t)(v - a.split) * a.tw;
#pragma unroll
                for (int q = 0; q < kEncV; ++q)
                    x[j][q] = (on && ok[q]) ? (kHints ? ld_nc_hint(src + w[q], pol_in)
                                                      : __ldg(src + w[q]))
                                            : make_uint4(0, 0, 0, 0);
            }
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                if (e + j >= e_end) break;
                while (e + j >= rp[r + 1]) {  // row r is complete (rows may be empty)
                    store_row<kHints>(a, k.r0 + r, w0, w1, acc, pol_out);
#pragma unroll
                    for (int v = 0; v < kEncV; ++v) acc[v] = make_uint4(0, 0, 0, 0);
                    ++r;
                }
#pragma unroll
                for (int q = 0; q < kEncV; ++q) xor4(acc[q], x[j][q]);
            }
        }
        for (; r < k.nr; ++r) {  // the last row with entries, then empty rows
            store_row<kHints>(a, k.r0 + r, w0, w1, acc, pol_out);
#pragma unroll
            for (int v = 0; v < kEncV; ++v) acc[v] = make_uint4(0, 0, 0, 0);
        }
    }
    cp_async_wait<0>();
}

// one job, passed by value
template <bool kHints>
__global__ void __launch_bounds__(kEncThreads, kCtasPerSm)
    k_rows(const __grid_constant__ RowArgs a, int32_t n_tickets, int32_t *ticket_ctr) {
    rows_body<kHints>(&a, 1, n_tickets, ticket_ctr);
}

// a batch of jobs (stripes) in device memory (batches take no L2 hints)
__global__ void __launch_bounds__(kEncThreads, kCtasPerSm)
    k_rows_batch(const RowArgs *jobs, int n_jobs, int32_t n_tickets, int32_t *ticket_ctr) {
    rows_body<false>(jobs, n_jobs, n_tickets, ticket_ctr);
}

// ---- shared-memory slice encode --------------------------------------------

constexpr int kSliceThreads = 1024;
constexpr long long kSliceWait = 1ll << 22;  // bounded mbarrier waits
constexpr uint16_t kNoSlot = 0xFFFF;
constexpr int32_t kPieceMax = 24;  // members of one precode row one lane sums
constexpr uint32_t kSlotAlign = 256;  // alignment of the slot buffers in shared memory

struct SliceArgs {
    const uint4 *tab;         // tables (copied to shared memory at start)
    int32_t tab_words;        // 16-byte words of tab
    int32_t off_row, off_idx; // byte offsets inside tab
    uint4 *parity, *coded;
    int32_t m, n_grp, n_grp_p, n_grp_a, bpad, zbase, slots, box_rows, n_boxes, nbuf;
    int32_t write_parity;     // 1: this part writes the parities out (the first part)
    int32_t st32;             // 1: coded rows 32-byte aligned: 32-byte slices store each row's
                              // piece with one 256-bit store
    int32_t n_xphase;         // chained precode: parity levels after the first, and the
    int32_t xphase_end[kSliceXPhases];  // end group of each (they start at n_grp_a)
    int32_t par_hi;           // end of those levels' groups (n_grp_a when there are none)
    int64_t tw;               // 16-byte words per block
    int32_t n_slices;         // byte slices of the stripe
    int32_t *ticket;          // workspace counter, zero at launch
    int32_t *status;
};

__device__ __forceinline__ uint32_t saddr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void xor_in(uint4 &a, const uint4 &b) {
    a.x ^= b.x;
    a.y ^= b.y;
    a.z ^= b.z;
    a.w ^= b.w;
}

// 16-byte word h of slot s. With 32-byte slots the TMA copies use the 32B
// swizzle (address bit 4 ^= bit 7), so the halves of slot s trade places
// when bit 2 of s is set; either way the 8 slots s with distinct s & 7 lie
// in 8 distinct bank groups for a fixed h.
template <int V>
__device__ __forceinline__ int32_t unit_of(int32_t s, int h) {
    return V == 1 ? s : 2 * s + (h ^ ((s >> 2) & 1));
}

// Issues the TMA copies of slice `tk` (all data blocks) into `buf`.
template <int V>
__device__ __forceinline__ void issue_slice(const CUtensorMap *map, const SliceArgs &a, int32_t tk,
                                            uint4 *buf, uint64_t *bar) {
    const uint32_t bytes = (uint32_t)a.n_boxes * (uint32_t)a.box_rows * 16u * V;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(saddr(bar)),
                 "r"(bytes)
                 : "memory");
    const int32_t x = tk * 16 * V;  // byte offset of the slice inside a block
    for (int i = 0; i < a.n_boxes; ++i) {
        const int32_t y = i * a.box_rows;
        asm volatile(
            "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
            " [%0], [%1, {%2, %3}], [%4];\n" ::"r"(saddr(buf + (size_t)y * V)),
            "l"(map), "r"(x), "r"(y), "r"(saddr(bar))
            : "memory");
    }
}

// Waits for the phase with the given parity; false after `rounds` x
// kSliceWait polls.
__device__ __forceinline__ bool wait_phase(uint64_t *bar, uint32_t parity, int rounds = 1) {
    const uint32_t addr = saddr(bar);
    for (long long i = 0; i < kSliceWait * rounds; ++i) {
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

// Views of the tables once they sit in shared memory.
struct SliceTables {
    const int2 *grp;
    const uint16_t *grow, *gidx;
};

template <int V>
__device__ __forceinline__ void gather(uint4 *acc, const uint4 *slot, uint16_t s) {
#pragma unroll
    for (int h = 0; h < V; ++h) xor_in(acc[h], slot[unit_of<V>(s, h)]);
}

// d ^= v in shared memory, fire-and-forget
__device__ __forceinline__ void red_xor16(uint4 *d, const uint4 &v) {
    const uint32_t p = saddr(d);
    asm volatile("red.shared.xor.b32 [%0], %1;\n" ::"r"(p), "r"(v.x) : "memory");
    asm volatile("red.shared.xor.b32 [%0], %1;\n" ::"r"(p + 4), "r"(v.y) : "memory");
    asm volatile("red.shared.xor.b32 [%0], %1;\n" ::"r"(p + 8), "r"(v.z) : "memory");
    asm volatile("red.shared.xor.b32 [%0], %1;\n" ::"r"(p + 12), "r"(v.w) : "memory");
}

// Zeroes the m parity slots of one slot buffer.
template <int V>
__device__ __forceinline__ void zero_parities(const SliceArgs &a, uint4 *buf) {
    for (int i = threadIdx.x; i < a.m * V; i += blockDim.x) buf[(size_t)a.bpad * V + i] = make_uint4(0, 0, 0, 0);
}

// One warp group: 32 output rows, one per lane (pieces of parity rows in
// the first n_grp_p groups, coded rows after); column c of the group's entries holds
// each lane's c-th input slot (padding names a zero slot in a bank group the
// column leaves free). Indices are fetched a step ahead.
template <int V>
__device__ __forceinline__ void row_group(const SliceArgs &a, const SliceTables &tb, uint4 *slot,
                                          int q, int64_t w0) {
    const int lane = threadIdx.x & 31;
    const int2 gq = tb.grp[q];
    const uint16_t *ix = tb.gidx + gq.x + lane;
    uint4 acc[V];
#pragma unroll
    for (int h = 0; h < V; ++h) acc[h] = make_uint4(0, 0, 0, 0);
    const uint16_t z = (uint16_t)(a.zbase + (lane & 7));
    uint16_t cur[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) cur[u] = u < gq.y ? ix[u * 32] : z;
    for (int j = 0; j < gq.y; j += 4) {
        uint16_t nxt[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) nxt[u] = j + 4 + u < gq.y ? ix[(j + 4 + u) * 32] : z;
#pragma unroll
        for (int u = 0; u < 4; ++u) gather<V>(acc, slot, cur[u]);
#pragma unroll
        for (int u = 0; u < 4; ++u) cur[u] = nxt[u];
    }
    const uint16_t row = tb.grow[q * 32 + lane];
    if (row == kNoSlot) return;
    const bool piece = q < a.n_grp_p || (q >= a.n_grp_a && q < a.par_hi);
    if (piece) {  // a piece of a parity row: XOR it into the parity's slot
#pragma unroll
        for (int h = 0; h < V; ++h) red_xor16(slot + unit_of<V>(a.bpad + row, h), acc[h]);
    } else if (V == 2 && a.st32 && w0 + 1 < a.tw) {
        // both words in one 256-bit store: half the scattered store requests
        // (w0 is even, the rows 32-byte aligned)
        const uint4 &lo = acc[0], &hi = acc[V - 1];
        asm volatile("st.global.cs.v8.u32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};\n" ::"l"(
                         a.coded + (int64_t)row * a.tw + w0),
                     "r"(lo.x), "r"(lo.y), "r"(lo.z), "r"(lo.w), "r"(hi.x), "r"(hi.y), "r"(hi.z), "r"(hi.w)
                     : "memory");
    } else {
#pragma unroll
        for (int h = 0; h < V; ++h)
            if (w0 + h < a.tw) __stcs(a.coded + (int64_t)row * a.tw + w0 + h, acc[h]);
    }
}

// Warps take the n items of a phase from a shared counter (largest first in
// table order), lane 0 drawing for the warp.
template <typename Item>
__device__ __forceinline__ void drain(int *ctr, int n, Item item) {
    const int lane = threadIdx.x & 31;
    for (;;) {
        int i = 0;
        if (lane == 0) i = atomicAdd(ctr, 1);
        i = __shfl_sync(0xffffffffu, i, 0);
        if (i >= n) break;
        item(i);
    }
}

// V 16-byte words per slot (slices of 16 V bytes), data slices by 2-D TMA
// boxes (one thread issues, an mbarrier completes), nbuf slot buffers. A
// slice takes two phases: the parities together with the coded rows that
// read no parity, then (after a barrier) the coded rows that read one.
template <int V>
__global__ void __launch_bounds__(kSliceThreads, 1)
    k_slices(const __grid_constant__ CUtensorMap map, SliceArgs a) {
    extern __shared__ __align__(256) unsigned char s_raw[];
    // 256-byte aligned slots (the 32B swizzle pattern repeats every 256 bytes);
    // offset from s_raw (not integer casts) so every access stays a shared-space load
    uint4 *slot0 = reinterpret_cast<uint4 *>(s_raw + ((kSlotAlign - (saddr(s_raw) & (kSlotAlign - 1))) & (kSlotAlign - 1)));
    const size_t buf_words = (size_t)a.slots * V;
    uint4 *s_tab = slot0 + (size_t)a.nbuf * buf_words;
    const unsigned char *tp = reinterpret_cast<const unsigned char *>(s_tab);
    SliceTables tb;
    tb.grp = reinterpret_cast<const int2 *>(tp);
    tb.grow = reinterpret_cast<const uint16_t *>(tp + a.off_row);
    tb.gidx = reinterpret_cast<const uint16_t *>(tp + a.off_idx);
    __shared__ uint64_t s_bar[2];
    __shared__ int32_t s_tk[2];
    __shared__ int32_t s_ok;
    __shared__ int s_ctr[2];  // work counters of the two phases
    const int32_t n_slices = a.n_slices;
    // groups of the two phases (a chained precode's further parity levels run
    // as extra phases between them)
    const int hi_p = a.par_hi;
    const int n_one = a.n_grp_a, n_two = a.n_grp - hi_p;

    if (threadIdx.x == 0) {
        for (int i = 0; i < 2; ++i)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(saddr(&s_bar[i])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        s_tk[0] = atomicAdd(a.ticket, 1);
        if (s_tk[0] < n_slices) issue_slice<V>(&map, a, s_tk[0], slot0, &s_bar[0]);
        s_ctr[0] = 0;
        s_ctr[1] = 0;
    }
    // the tables, once per CTA, under the first slice's copies; the zero slots
    for (int32_t i = threadIdx.x; i < a.tab_words; i += blockDim.x) s_tab[i] = __ldg(a.tab + i);
    for (int i = threadIdx.x; i < 2 * 8 * V; i += blockDim.x) {
        const int bb = i / (8 * V), r = i % (8 * V);
        if (bb < a.nbuf) slot0[(size_t)bb * buf_words + (size_t)a.zbase * V + r] = make_uint4(0, 0, 0, 0);
    }
    for (int bb = 0; bb < a.nbuf; ++bb) zero_parities<V>(a, slot0 + (size_t)bb * buf_words);

    uint32_t uses0 = 0, uses1 = 0;  // completed phases of each buffer's barrier
    for (int it = 0;; ++it) {
        const int b = a.nbuf == 2 ? (it & 1) : 0;
        uint4 *slot = slot0 + (size_t)b * buf_words;
        if (threadIdx.x == 0) {
            const int32_t t = s_tk[it & 1];
            int ok = 1;
            if (t < n_slices) {
                ok = wait_phase(&s_bar[b], (b ? uses1 : uses0) & 1) ? 1 : 0;
                if (!ok) {
                    // give up, but first wait longer (8 bounds) for the copies in
                    // flight into this buffer; only if that wait expires too does
                    // the CTA leave with a copy possibly still landing
                    atomicExch(a.status, (int32_t)FS_ERR_TIMEOUT);
                    wait_phase(&s_bar[b], (b ? uses1 : uses0) & 1, 8);
                }
            }
            s_ok = ok;
        }
        // slice t is in; every warp has left the previous slice (its buffer is free)
        __syncthreads();
        const int32_t t = s_tk[it & 1];
        // a slice past the end issued no copy; a failed wait was drained above
        // (as far as its longer bound allows); the next copy is issued below
        if (t >= n_slices || !s_ok) break;
        if (b) ++uses1;
        else ++uses0;
        if (threadIdx.x == 0) {
            s_ctr[1] = 0;
            if (a.nbuf == 2) {  // next slice into the other buffer
                const int32_t nx = atomicAdd(a.ticket, 1);
                s_tk[(it + 1) & 1] = nx;
                if (nx < n_slices)
                    issue_slice<V>(&map, a, nx, slot0 + (size_t)(b ^ 1) * buf_words, &s_bar[b ^ 1]);
            }
        }
        // the other buffer's parity slots (last read by the previous slice) for the next slice
        if (a.nbuf == 2) zero_parities<V>(a, slot0 + (size_t)(b ^ 1) * buf_words);
        const int64_t w0 = (int64_t)t * V;  // first 16-byte word of the slice
        drain(&s_ctr[0], n_one, [&](int i) { row_group<V>(a, tb, slot, i, w0); });
        __syncthreads();  // the parity slots are complete
        if (threadIdx.x == 0) s_ctr[0] = 0;
        for (int ph = 0; ph < a.n_xphase; ++ph) {  // chained: the next level reads these
            const int lo = ph == 0 ? a.n_grp_a : a.xphase_end[ph - 1], hi = a.xphase_end[ph];
            __syncthreads();  // the counter is reset
            drain(&s_ctr[0], hi - lo, [&](int i) { row_group<V>(a, tb, slot, lo + i, w0); });
            __syncthreads();  // this level's parity slots are complete
            if (threadIdx.x == 0) s_ctr[0] = 0;
        }
        for (int i = threadIdx.x; a.write_parity && i < a.m * V; i += blockDim.x) {
            const int j = i / V, h = i - j * V;
            if (w0 + h < a.tw) a.parity[(int64_t)j * a.tw + w0 + h] = slot[unit_of<V>(a.bpad + j, h)];
        }
        drain(&s_ctr[1], n_two, [&](int i) { row_group<V>(a, tb, slot, hi_p + i, w0); });
        if (a.nbuf == 1) {
            __syncthreads();  // the only buffer is free
            zero_parities<V>(a, slot0);
            if (threadIdx.x == 0) {
                const int32_t nx = atomicAdd(a.ticket, 1);
                s_tk[(it + 1) & 1] = nx;
                if (nx < n_slices) issue_slice<V>(&map, a, nx, slot0, &s_bar[0]);
            }
        }
    }
}

// Batch form: persistent CTAs take items (stripe, slices [s0, s1)) from a
// counter. A CTA reloads the stripe's tables and zero slots only when its
// item's stripe differs from the previous one; within an item the copies of
// the next slice land under the arithmetic of the current one. 16-byte slots,
// two buffers; buffers start at the same place for every stripe (the largest
// stripe's buffer size apart), the tables after them.
__global__ void __launch_bounds__(kSliceThreads, 1)
    k_slices_batch(const SliceArgs *as, const CUtensorMap *maps, const int4 *items, int n_items,
                   int32_t *item_ctr, int32_t *status) {
    constexpr int V = 1;
    extern __shared__ __align__(256) unsigned char s_raw[];
    // per stripe: its tables first, then its two slot buffers (256-byte aligned)
    uint4 *s_tab = reinterpret_cast<uint4 *>(s_raw + ((kSlotAlign - (saddr(s_raw) & (kSlotAlign - 1))) & (kSlotAlign - 1)));
    __shared__ uint64_t s_bar[2];
    __shared__ int32_t s_item, s_ok;
    __shared__ int s_ctr[2];
    if (threadIdx.x == 0) {
        for (int i = 0; i < 2; ++i)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(saddr(&s_bar[i])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        s_ctr[0] = 0;
        s_ctr[1] = 0;
    }
    uint32_t uses0 = 0, uses1 = 0;  // completed phases of each buffer's barrier (thread 0)
    int cur = -1;                   // stripe whose tables are loaded
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(item_ctr, 1);
        __syncthreads();  // also: every warp is done with the previous item
        const int it = s_item;
        if (it >= n_items) break;
        const int4 item = items[it];
        const SliceArgs a = as[item.x];
        const CUtensorMap *map = maps + item.x;
        uint4 *slot0 = s_tab + (((size_t)a.tab_words + 15) & ~(size_t)15);
        const size_t buf_words = (size_t)a.slots * V;
        const unsigned char *tp = reinterpret_cast<const unsigned char *>(s_tab);
        SliceTables tb;
        tb.grp = reinterpret_cast<const int2 *>(tp);
        tb.grow = reinterpret_cast<const uint16_t *>(tp + a.off_row);
        tb.gidx = reinterpret_cast<const uint16_t *>(tp + a.off_idx);
        if (item.x != cur) {  // this stripe's tables, zero slots and zeroed parity slots
            for (int32_t i = threadIdx.x; i < a.tab_words; i += blockDim.x) s_tab[i] = __ldg(a.tab + i);
            for (int i = threadIdx.x; i < 2 * 8 * V; i += blockDim.x)
                slot0[(size_t)(i / (8 * V)) * buf_words + (size_t)a.zbase * V + i % (8 * V)] =
                    make_uint4(0, 0, 0, 0);
            for (int bb = 0; bb < 2; ++bb) zero_parities<V>(a, slot0 + (size_t)bb * buf_words);
            cur = item.x;
        }
        const int n_one = a.n_grp_a, n_two = a.n_grp - a.n_grp_a;
        if (threadIdx.x == 0) issue_slice<V>(map, a, item.y, slot0, &s_bar[0]);
        __syncthreads();  // tables and zero slots in place
        for (int32_t t = item.y, j = 0; t < item.z; ++t, ++j) {
            const int b = j & 1;
            uint4 *slot = slot0 + (size_t)b * buf_words;
            if (threadIdx.x == 0) {
                int ok = wait_phase(&s_bar[b], (b ? uses1 : uses0) & 1) ? 1 : 0;
                if (!ok) {  // give up after a longer wait (8 bounds) for the copies in flight
                    atomicExch(status, (int32_t)FS_ERR_TIMEOUT);
                    wait_phase(&s_bar[b], (b ? uses1 : uses0) & 1, 8);
                }
                s_ok = ok;
            }
            __syncthreads();  // slice t is in; every warp has left slice t - 1
            if (!s_ok) return;
            if (b) ++uses1;
            else ++uses0;
            if (threadIdx.x == 0) {
                s_ctr[1] = 0;
                if (t + 1 < item.z) issue_slice<V>(map, a, t + 1, slot0 + (size_t)(b ^ 1) * buf_words, &s_bar[b ^ 1]);
            }
            zero_parities<V>(a, slot0 + (size_t)(b ^ 1) * buf_words);
            const int64_t w0 = (int64_t)t * V;
            drain(&s_ctr[0], n_one, [&](int i) { row_group<V>(a, tb, slot, i, w0); });
            __syncthreads();  // the parity slots are complete
            if (threadIdx.x == 0) s_ctr[0] = 0;
            for (int i = threadIdx.x; a.write_parity && i < a.m * V; i += blockDim.x) {
                const int jj = i / V, h = i - jj * V;
                if (w0 + h < a.tw) a.parity[(int64_t)jj * a.tw + w0 + h] = slot[unit_of<V>(a.bpad + jj, h)];
            }
            drain(&s_ctr[1], n_two, [&](int i) { row_group<V>(a, tb, slot, a.n_grp_a + i, w0); });
        }
    }
}

using EncodeTiledFn = PFN_cuTensorMapEncodeTiled_v12000;

EncodeTiledFn tensor_map_encoder() {
    static std::once_flag once;
    static EncodeTiledFn fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

size_t slice_smem_bytes(const fs_code *c, int v, int nbuf) {
    // slot buffers, the largest part's tables, alignment slack
    int32_t tab = 0;
    for (int q = 0; q < c->sl_parts; ++q) tab = std::max(tab, c->sl_part[q].tab_bytes);
    return (size_t)nbuf * (size_t)c->sl_slots * 16 * v + (size_t)tab + kSlotAlign;
}

int grid_for(int64_t n_tiles, int num_sms, int ctas_per_sm) {
    const int64_t cap = (int64_t)num_sms * ctas_per_sm;
    const int64_t g = n_tiles < cap ? n_tiles : cap;
    return (int)(g < 1 ? 1 : g);
}

}  // namespace

int32_t encode_chunks(const fs_code *c) {
    return (int32_t)((c->tw + kChunkW - 1) / kChunkW);
}

// status word + one ticket counter per launch (header words WS_COUNT_A/B)
size_t encode_ws_bytes(const fs_code *) { return WS_HDR_BYTES; }

namespace {

// Shared memory serves a warp's 16-byte loads a quarter-warp (8 lanes) at a
// time, and slot s lies in bank group s & 7: 8 lanes that read 8 different
// groups take one pass, two lanes in the same group take two. The tables
// below order the work so that every quarter-warp reads distinct groups.
inline int bank_group(uint16_t slot) { return slot & 7; }

// Colours the edges of a bipartite multigraph (8 rows x 8 bank groups) with
// delta colours, no two edges of one colour sharing an end (Koenig's theorem;
// a clash is cleared by swapping the two colours along an alternating path).
// edges: (row position, group); returns the colour of each edge.
std::vector<int> colour_edges(const std::vector<std::pair<int, int>> &edges, int delta) {
    std::vector<int> at_r(8 * (size_t)delta, -1), at_g(8 * (size_t)delta, -1);
    std::vector<int> col(edges.size(), -1);
    std::vector<int> path;
    for (size_t e = 0; e < edges.size(); ++e) {
        const int r = edges[e].first, g = edges[e].second;
        int a = 0, b = 0;
        while (at_r[r * delta + a] >= 0) ++a;  // free at the row
        while (at_g[g * delta + b] >= 0) ++b;  // free at the group
        if (at_g[g * delta + a] >= 0) {
            // path from g along colours a, b, a, ...; it cannot reach r (a is free there)
            path.clear();
            int v = g, x = a, y = b;
            bool at_group = true;
            for (;;) {
                const int f = at_group ? at_g[v * delta + x] : at_r[v * delta + x];
                if (f < 0) break;
                path.push_back(f);
                v = at_group ? edges[f].first : edges[f].second;
                at_group = !at_group;
                std::swap(x, y);
            }
            for (int f : path) {
                at_r[edges[f].first * delta + col[f]] = -1;
                at_g[edges[f].second * delta + col[f]] = -1;
            }
            for (int f : path) {
                col[f] = col[f] == a ? b : a;
                at_r[edges[f].first * delta + col[f]] = f;
                at_g[edges[f].second * delta + col[f]] = f;
            }
        }
        col[e] = a;
        at_r[r * delta + a] = (int)e;
        at_g[g * delta + a] = (int)e;
    }
    return col;
}

}  // namespace

cudaError_t build_slice_tables(fs_code *c, const int32_t *con_ptr, const int32_t *con_idx) {
    c->sl_slots = 0;
    c->sl_parts = 0;
    // a chained precode (parities over earlier parities) runs its levels as
    // phases of their own: at most 1 + kSliceXPhases levels
    if (c->b < 1 || c->n < 1 || c->n >= kNoSlot || c->m >= kNoSlot) return cudaSuccess;
    if (c->chained && c->n_pre_levels - 1 > kSliceXPhases) return cudaSuccess;
    const int32_t box_rows = c->b < 256 ? c->b : 256;
    const int64_t bpad = ((int64_t)c->b + box_rows - 1) / box_rows * box_rows;
    // data slots, parity slots, then 8 zero slots (one per bank group)
    const int64_t zbase = (bpad + c->m + 7) & ~(int64_t)7;
    const int64_t slots = zbase + 8;
    if (slots >= kNoSlot) return cudaSuccess;
    auto slot_of = [&](int32_t v) -> uint16_t {
        return (uint16_t)(v < c->b ? v : bpad + (v - c->b));
    };
    const int32_t n = c->n, m = c->m;
    // every output row as a list of slots: the precode rows (members only;
    // the joint graph's check row n + j ends with its own parity), each cut
    // into ks pieces of at most kPieceMax members that different lanes sum
    // (long rows would otherwise hold one warp far longer than the others),
    // then the n coded rows
    int32_t max_pre = 0;
    for (int32_t j = 0; j < m; ++j) max_pre = std::max(max_pre, con_ptr[n + j + 1] - con_ptr[n + j] - 1);
    const int32_t ks = std::max<int32_t>(1, (max_pre + kPieceMax - 1) / kPieceMax);
    const int32_t mp = m * ks;  // parity pieces: piece p belongs to parity p / ks
    if (mp >= kNoSlot) return cudaSuccess;
    std::vector<std::vector<uint16_t>> in((size_t)mp + n);
    for (int32_t j = 0; j < m; ++j) {
        const int32_t e0 = con_ptr[n + j], len = con_ptr[n + j + 1] - 1 - e0;
        for (int32_t k = 0; k < ks; ++k)
            for (int32_t e = e0 + (int32_t)((int64_t)len * k / ks); e < e0 + (int32_t)((int64_t)len * (k + 1) / ks); ++e)
                in[(size_t)j * ks + k].push_back(slot_of(con_idx[e]));
    }
    for (int32_t r = 0; r < n; ++r)
        for (int32_t e = con_ptr[r]; e < con_ptr[r + 1]; ++e) in[(size_t)mp + r].push_back(slot_of(con_idx[e]));
    auto deg = [&](int32_t id) { return (int)in[id].size(); };

    // Builds the tables of one part: the parity pieces (every part computes
    // the parities its coded rows read) and coded rows [r_lo, r_hi): rows
    // into quarters of 8 (rows of about the same length, largest first, whose
    // inputs spread evenly over the bank groups), quarters sorted by width
    // and padded to whole warp groups, then each quarter's inputs placed by
    // an edge colouring. Returns false when the tables grow too large.
    struct Quarter {
        int32_t row[8];
        int delta;
    };
    struct HostPart {
        std::vector<unsigned char> tab;
        int32_t n_grp = 0, n_grp_p = 0, n_grp_a = 0, off_row = 0, off_idx = 0;
        int32_t n_xphase = 0;
        int32_t xphase_end[kSliceXPhases] = {};
    };
    // precode level of parity j (0 unless chained: its checks come in level order)
    std::vector<int32_t> plevel(m, 0);
    for (int32_t l = 0; c->chained && l < c->n_pre_levels; ++l)
        for (int32_t j = c->pre_level_off[l]; j < c->pre_level_off[l + 1]; ++j) plevel[j] = l;
    std::vector<char> used((size_t)mp + n, 0);
    auto make_part = [&](int32_t r_lo, int32_t r_hi, HostPart &hp) -> bool {
        std::vector<Quarter> quarters;
        for (int32_t p = 0; p < mp; ++p) used[p] = 0;
        for (int32_t r = r_lo; r < r_hi; ++r) used[(size_t)mp + r] = 0;
        auto build_quarters = [&](std::vector<int32_t> order) {
            std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) { return deg(x) > deg(y); });
            std::vector<Quarter> qs;
            constexpr int kWindow = 64;  // candidates looked at for each place
            size_t pos = 0;
            for (;;) {
                while (pos < order.size() && used[order[pos]]) ++pos;
                if (pos >= order.size()) break;
                Quarter q;
                std::fill(q.row, q.row + 8, -1);
                int cnt[8] = {0};
                const int dmax = deg(order[pos]);
                for (int k = 0; k < 8; ++k) {
                    int32_t best = -1;
                    int best_key = 0, best_deg = 0;
                    int seen = 0;
                    for (size_t i = pos; i < order.size() && seen < (k == 0 ? 1 : kWindow); ++i) {
                        const int32_t r = order[i];
                        if (used[r]) continue;
                        ++seen;
                        int c2[8];
                        std::copy(cnt, cnt + 8, c2);
                        for (uint16_t sl : in[r]) ++c2[bank_group(sl)];
                        const int key = std::max(*std::max_element(c2, c2 + 8), dmax);
                        if (best < 0 || key < best_key || (key == best_key && deg(r) > best_deg)) {
                            best = r;
                            best_key = key;
                            best_deg = deg(r);
                        }
                    }
                    if (best < 0) break;
                    used[best] = 1;
                    q.row[k] = best;
                    for (uint16_t sl : in[best]) ++cnt[bank_group(sl)];
                }
                q.delta = std::max(*std::max_element(cnt, cnt + 8), dmax);
                qs.push_back(q);
            }
            std::stable_sort(qs.begin(), qs.end(), [](const Quarter &x, const Quarter &y) { return x.delta > y.delta; });
            while (qs.size() % 4) {  // empty quarters complete the last warp group
                Quarter e;
                std::fill(e.row, e.row + 8, -1);
                e.delta = 0;
                qs.push_back(e);
            }
            quarters.insert(quarters.end(), qs.begin(), qs.end());
        };
        // parity rows; coded rows that read no parity (computed beside the
        // parities); coded rows that read one (after them)
        std::vector<int32_t> set_p, set_a, set_b;
        std::vector<std::vector<int32_t>> set_x(c->chained ? c->n_pre_levels - 1 : 0);
        for (int32_t p = 0; p < mp; ++p) {
            const int32_t l = plevel[p / ks];
            (l == 0 ? set_p : set_x[l - 1]).push_back(p);
        }
        for (int32_t r = r_lo; r < r_hi; ++r) {
            bool par = false;
            for (int32_t e = con_ptr[r]; e < con_ptr[r + 1]; ++e) par |= con_idx[e] >= c->b;
            (par ? set_b : set_a).push_back(mp + r);
        }
        build_quarters(set_p);
        hp.n_grp_p = (int32_t)(quarters.size() / 4);
        build_quarters(set_a);
        hp.n_grp_a = (int32_t)(quarters.size() / 4);
        hp.n_xphase = (int32_t)set_x.size();
        for (size_t l = 0; l < set_x.size(); ++l) {  // one phase per further level
            build_quarters(set_x[l]);
            hp.xphase_end[l] = (int32_t)(quarters.size() / 4);
        }
        build_quarters(set_b);
        const int32_t n_grp = (int32_t)(quarters.size() / 4);
        hp.n_grp = n_grp;
        std::vector<int2> grp(n_grp);
        int64_t total = 0;
        for (int32_t gq = 0; gq < n_grp; ++gq) {
            const int cols = quarters[(size_t)gq * 4].delta;  // sorted: the first is the widest
            grp[gq] = make_int2((int32_t)total, cols);
            total += 32 * (int64_t)cols;
            if (total > (int64_t)1 << 24) return false;
        }
        auto al16 = [](int64_t x) { return (x + 15) & ~(int64_t)15; };
        const int64_t off_row = al16((int64_t)sizeof(int2) * n_grp);
        const int64_t off_idx = al16(off_row + 2 * 32 * (int64_t)n_grp);
        const int64_t bytes = al16(off_idx + 2 * total);
        if (bytes > INT32_MAX / 2) return false;
        hp.off_row = (int32_t)off_row;
        hp.off_idx = (int32_t)off_idx;
        hp.tab.assign((size_t)bytes, 0);
        memcpy(hp.tab.data(), grp.data(), sizeof(int2) * n_grp);
        uint16_t *row = reinterpret_cast<uint16_t *>(hp.tab.data() + off_row);
        uint16_t *idx = reinterpret_cast<uint16_t *>(hp.tab.data() + off_idx);
        std::fill(row, row + 32 * (size_t)n_grp, kNoSlot);
        std::fill(idx, idx + total, kNoSlot);
        std::vector<std::pair<int, int>> edges;
        std::vector<uint16_t> eslot;
        for (size_t qi = 0; qi < quarters.size(); ++qi) {
            const Quarter &q = quarters[qi];
            const int32_t gq = (int32_t)(qi / 4), lane0 = 8 * (int32_t)(qi % 4);
            edges.clear();
            eslot.clear();
            for (int p = 0; p < 8; ++p) {
                if (q.row[p] < 0) continue;
                // output id: the parity index, or the coded row
                row[(size_t)gq * 32 + lane0 + p] = (uint16_t)(q.row[p] < mp ? q.row[p] / ks : q.row[p] - mp);
                for (uint16_t sl : in[q.row[p]]) {
                    edges.emplace_back(p, bank_group(sl));
                    eslot.push_back(sl);
                }
            }
            const std::vector<int> col = colour_edges(edges, std::max(q.delta, 1));
            for (size_t e = 0; e < edges.size(); ++e)
                idx[(size_t)grp[gq].x + (size_t)col[e] * 32 + lane0 + edges[e].first] = eslot[e];
            // empty cells of each column: the zero slot of a group the column leaves free
            for (int cc = 0; cc < grp[gq].y; ++cc) {
                uint16_t *cell = idx + (size_t)grp[gq].x + (size_t)cc * 32 + lane0;
                bool taken[8] = {false};
                for (int p = 0; p < 8; ++p)
                    if (cell[p] != kNoSlot) taken[bank_group(cell[p])] = true;
                int k = 0;
                for (int p = 0; p < 8; ++p) {
                    if (cell[p] != kNoSlot) continue;
                    while (k < 7 && taken[k]) ++k;
                    cell[p] = (uint16_t)(zbase + k);
                }
            }
        }
        return true;
    };

    // as few parts as let every part run with two slot buffers of 16 bytes;
    // one part with one buffer when no split up to kSliceParts does
    const size_t budget = c->smem_optin;
    // the same rule as the batch layout: tables rounded to 256 bytes, then the buffers
    auto fits = [&](const HostPart &hp, int nbuf) {
        return (size_t)nbuf * (size_t)slots * 16 + ((hp.tab.size() + 255) & ~(size_t)255) + kSlotAlign <=
               budget;
    };
    std::vector<HostPart> parts;
    for (int P = 1; P <= kSliceParts && parts.empty(); ++P) {
        // coded rows into P ranges of about equal entries
        std::vector<int32_t> cut(P + 1, n);
        cut[0] = 0;
        const int64_t per = ((int64_t)con_ptr[n] + P - 1) / P;
        for (int q = 1, r = 0; q < P; ++q) {
            while (r < n && con_ptr[r] < per * q) ++r;
            cut[q] = r;
        }
        std::vector<HostPart> cand(P);
        bool ok = true;
        for (int q = 0; q < P && ok; ++q) ok = make_part(cut[q], cut[q + 1], cand[q]) && fits(cand[q], 2);
        if (ok) parts = std::move(cand);
    }
    if (parts.empty()) {  // one part, one buffer
        HostPart hp;
        if (!make_part(0, n, hp) || !fits(hp, 1)) return cudaSuccess;
        parts.push_back(std::move(hp));
    }
    for (size_t q = 0; q < parts.size(); ++q) {
        SlicePart &sp = c->sl_part[q];
        const HostPart &hp = parts[q];
        cudaError_t e = cudaMalloc(&sp.tab, hp.tab.size());
        if (e == cudaSuccess) e = cudaMemcpy(sp.tab, hp.tab.data(), hp.tab.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return e;
        sp.tab_bytes = (int32_t)hp.tab.size();
        sp.n_grp = hp.n_grp;
        sp.n_grp_p = hp.n_grp_p;
        sp.n_grp_a = hp.n_grp_a;
        sp.off_row = hp.off_row;
        sp.off_idx = hp.off_idx;
        sp.n_xphase = hp.n_xphase;
        for (int l = 0; l < kSliceXPhases; ++l) sp.xphase_end[l] = hp.xphase_end[l];
    }
    c->sl_parts = (int32_t)parts.size();
    c->sl_box_rows = box_rows;
    c->sl_bpad = (int32_t)bpad;
    c->sl_zbase = (int32_t)zbase;
    c->sl_slots = (int32_t)slots;
    return cudaSuccess;
}

void free_slice_tables(fs_code *c) {
    for (int q = 0; q < kSliceParts; ++q) cudaFree(c->sl_part[q].tab);
}

namespace {

// Slice encode of the whole code; false (nothing launched) when it does not apply.
// Two slot buffers (the next slice's copies land under the current slice's
// arithmetic) matter more than the slot width, so: 32-byte slots (full-sector
// copies and stores) when two buffers of them fit, else 16-byte slots, with
// two buffers when they fit.
// The launch arguments of a code's slice encode with v words per slot and
// nbuf buffers; false when no tensor map can be made.
bool slice_setup(const fs_code *c, int part, const void *data, void *parity, void *coded, int v,
                 int nbuf, SliceArgs *a, CUtensorMap *map) {
    EncodeTiledFn encode = tensor_map_encoder();
    if (!encode) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)c->t, (cuuint64_t)c->b};
    const cuuint64_t strides[1] = {(cuuint64_t)c->t};
    const cuuint32_t box[2] = {(cuuint32_t)(16 * v), (cuuint32_t)c->sl_box_rows};
    const cuuint32_t estr[2] = {1, 1};
    if (encode(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void *>(data), dims, strides, box,
               estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               v == 2 ? CU_TENSOR_MAP_SWIZZLE_32B : CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    const SlicePart &sp = c->sl_part[part];
    a->tab = reinterpret_cast<const uint4 *>(sp.tab);
    a->tab_words = sp.tab_bytes / 16;
    a->off_row = sp.off_row;
    a->off_idx = sp.off_idx;
    a->write_parity = part == 0 ? 1 : 0;
    a->st32 = (v == 2 && (reinterpret_cast<uintptr_t>(coded) & 31) == 0 && (c->tw & 1) == 0) ? 1 : 0;
    a->parity = static_cast<uint4 *>(parity);
    a->coded = static_cast<uint4 *>(coded);
    a->m = c->m;
    a->n_grp = sp.n_grp;
    a->n_grp_p = sp.n_grp_p;
    a->n_grp_a = sp.n_grp_a;
    a->n_xphase = sp.n_xphase;
    for (int l = 0; l < kSliceXPhases; ++l) a->xphase_end[l] = sp.xphase_end[l];
    a->par_hi = sp.n_xphase > 0 ? sp.xphase_end[sp.n_xphase - 1] : sp.n_grp_a;
    a->bpad = c->sl_bpad;
    a->zbase = c->sl_zbase;
    a->slots = c->sl_slots;
    a->box_rows = c->sl_box_rows;
    a->n_boxes = c->sl_bpad / c->sl_box_rows;
    a->nbuf = nbuf;
    a->tw = c->tw;
    a->n_slices = (int32_t)((c->tw + v - 1) / v);
    a->ticket = nullptr;
    a->status = nullptr;
    return true;
}

// Slice encode of the whole code; false (nothing launched) when it does not apply.
// Two slot buffers (the next slice's copies land under the current slice's
// arithmetic) matter more than the slot width, so: 32-byte slots (full-sector
// copies and stores) when two buffers of them fit, else 16-byte slots, with
// two buffers when they fit.
// Whether the automatic policy picks slices for c: a code whose tables fit in
// one part always (each input byte crosses DRAM once); a code split into
// parts only for blocks up to 16 KiB, because every part re-reads the data
// and, for the long rows such codes have, the shared-memory gathers then cost
// as much as the row-gather encode at large blocks (measured).
bool slices_pay(const fs_code *c) {
    if (c->sl_slots == 0 || c->t >= ((int64_t)1 << 31)) return false;
    return c->encode_slices >= 2 || c->sl_parts == 1 || c->t <= 16384;
}

bool launch_slices(const fs_code *c, const void *data, void *parity, void *coded, int32_t *hdr,
                   cudaStream_t s, cudaError_t *err) {
    *err = cudaSuccess;
    if (!c->encode_slices || !slices_pay(c)) return false;
    // 32-byte slices by default when two buffers of them fit, or when the
    // coded rows take 256-bit stores and the stripe has slices enough (at
    // least 8 per SM): one buffer of them then beats two of 16-byte slices
    // (4096 x 64 KiB: 0.287 against 0.302 ms)
    const bool st32 = (reinterpret_cast<uintptr_t>(coded) & 31) == 0 && (c->tw & 1) == 0;
    const bool many = c->tw / 2 >= 8 * (int64_t)c->num_sms;
    int v = c->encode_slices == 2   ? 1
            : c->encode_slices == 3 ? 2
            : (c->tw >= 2 && (slice_smem_bytes(c, 2, 2) <= c->smem_optin || (st32 && many)) ? 2 : 1);
    if (slice_smem_bytes(c, v, 1) > c->smem_optin) v = 1;
    const int nbuf = slice_smem_bytes(c, v, 2) <= c->smem_optin ? 2 : 1;
    const size_t smem = slice_smem_bytes(c, v, nbuf);
    auto kern = v == 2 ? k_slices<2> : k_slices<1>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    for (int q = 0; q < c->sl_parts && e == cudaSuccess; ++q) {  // one launch per part
        CUtensorMap map;
        SliceArgs a;
        if (!slice_setup(c, q, data, parity, coded, v, nbuf, &a, &map)) {
            if (q == 0) return false;
            e = cudaErrorInvalidValue;
            break;
        }
        a.ticket = hdr + WS_ENC_TICKETS + q;
        a.status = hdr + WS_STATUS;
        // one CTA per SM but one: each CTA fills its SM's shared memory, so a
        // one-CTA decoding schedule launched beside the encode on another
        // stream would otherwise wait for the whole encode
        const int64_t sms = c->num_sms > 1 ? c->num_sms - 1 : 1;
        const int64_t g = a.n_slices < sms ? a.n_slices : sms;
        kern<<<(int)(g < 1 ? 1 : g), kSliceThreads, smem, s>>>(map, a);
        e = cudaGetLastError();
    }
    *err = e;
    return true;
}

}  // namespace

cudaError_t launch_encode(const fs_code *c, const void *data, void *parity, void *coded, uint8_t *ws,
                          cudaStream_t s) {
    int32_t *hdr = reinterpret_cast<int32_t *>(ws);
    // status and the ticket counters
    cudaError_t e = cudaMemsetAsync(ws, 0, WS_HDR_BYTES, s);
    if (e != cudaSuccess) return e;
    if (launch_slices(c, data, parity, coded, hdr, s, &e)) return e;
    const int32_t n_chunks = encode_chunks(c);
    const int ctas = c->gather_ctas < kCtasPerSm ? c->gather_ctas : kCtasPerSm;
    RowArgs a;
    a.tw = c->tw;
    a.n_chunks = n_chunks;
    a.hints = c->l2_hints;
    if (c->m > 0) {  // step (1): parities over the data blocks
        // a chained precode runs level by level: the checks of a level read
        // parities of earlier levels only (one launch each, in stream order)
        a.idx = c->pre_idx;
        a.inA = static_cast<const uint4 *>(data);
        a.inB = c->chained ? static_cast<const uint4 *>(parity) : nullptr;
        a.split = c->b;
        a.stream_out = 0;
        a.rows = 1;  // check rows are long: one per ticket keeps every SM busy
        a.t0 = 0;
        for (int32_t l = 0; l < c->n_pre_levels; ++l) {
            const int32_t r0 = c->chained ? c->pre_level_off[l] : 0;
            const int32_t r1 = c->chained ? c->pre_level_off[l + 1] : c->m;
            a.ptr = c->pre_ptr + r0;  // row pointers stay absolute into pre_idx
            a.out = static_cast<uint4 *>(parity) + (int64_t)r0 * c->tw;
            a.n_rows = r1 - r0;
            if (l > 0) e = cudaMemsetAsync(hdr + WS_COUNT_A, 0, sizeof(int32_t), s);
            if (e != cudaSuccess) return e;
            const int64_t tickets = (int64_t)n_chunks * a.n_rows;
            (c->l2_hints ? k_rows<true> : k_rows<false>)<<<grid_for(tickets, c->num_sms, ctas), kEncThreads,
                                                             0, s>>>(a, (int32_t)tickets, hdr + WS_COUNT_A);
            e = cudaGetLastError();
            if (e != cudaSuccess) return e;
        }
    }
    if (c->n > 0) {  // step (2): coded rows over data blocks and parities
        a.ptr = c->con_ptr;
        a.idx = c->con_idx;
        a.inA = static_cast<const uint4 *>(data);
        a.inB = static_cast<const uint4 *>(parity);
        a.split = c->b;
        a.out = static_cast<uint4 *>(coded);
        a.n_rows = c->n;
        a.stream_out = 1;
        a.rows = c->rows_per_ticket;
        a.t0 = 0;
        const int64_t tickets = (int64_t)n_chunks * ((c->n + a.rows - 1) / a.rows);
        (c->l2_hints ? k_rows<true> : k_rows<false>)<<<grid_for(tickets, c->num_sms, ctas), kEncThreads, 0,
                                                         s>>>(a, (int32_t)tickets, hdr + WS_COUNT_B);
        e = cudaGetLastError();
    }
    return e;
}

// ---- batched encode ----------------------------------------------------------
// Every stripe of a batch becomes two row jobs (its precode rows, its LT rows);
// one launch runs all precode jobs, a second all LT jobs (stream order makes
// every parity final before an LT row reads it). Tickets run stripe by stripe.

struct EncodeBatch {
    // device job arrays of the row-gather stripes: precode rows one launch per
    // precode level (a chained precode's level reads earlier levels' parities),
    // then the LT rows
    std::vector<RowArgs *> d_pre;
    std::vector<int> n_pre;
    std::vector<int32_t> t_pre;  // tickets of each precode launch
    RowArgs *d_lt = nullptr;
    int n_lt = 0;
    int32_t t_lt = 0;
    SliceArgs *d_sl = nullptr;    // slice stripes: arguments, tensor maps, items
    CUtensorMap *d_maps = nullptr;
    int4 *d_items = nullptr;
    int n_items = 0;
    size_t smem_sl = 0;
    int32_t *d_ctr = nullptr;     // ticket counters (precode, LT), item counter, status
    int num_sms = 1, ctas = 1;
};

int32_t encode_batch_status_word(const EncodeBatch *b, int32_t *out) {
    return cudaMemcpy(out, b->d_ctr + 3, sizeof(int32_t), cudaMemcpyDeviceToHost) == cudaSuccess ? 0 : -1;
}

cudaError_t encode_batch_plan(const fs_code *const *codes, const void *const *data,
                              void *const *parity, void *const *coded, int32_t n,
                              EncodeBatch **out) {
    *out = nullptr;
    std::vector<std::vector<RowArgs>> pre;  // per precode level
    std::vector<int64_t> tp;
    std::vector<RowArgs> lt;
    int64_t tl = 0;
    // stripes whose slice layout fits (16-byte slots, two buffers) go to the
    // batch slice kernel; the layout of a launch is the largest buffers and
    // the largest tables of its stripes, so stripes are added while that fits
    const size_t budget = n > 0 ? codes[0]->smem_optin : 0;
    auto tab_of = [&](int32_t i) {
        int32_t t = 0;
        for (int q = 0; q < codes[i]->sl_parts; ++q) t = std::max(t, codes[i]->sl_part[q].tab_bytes);
        return t;
    };
    std::vector<int32_t> order;
    // (in a batch only single-part codes: beside many other stripes the
    // row-gather kernel overlaps the large ones better than a split would)
    for (int32_t i = 0; i < n; ++i)
        if (codes[i]->encode_slices && slices_pay(codes[i]) && codes[i]->sl_parts == 1 &&
            !codes[i]->chained)  // the batch slice kernel runs two phases only
            order.push_back(i);
    std::sort(order.begin(), order.end(), [&](int32_t x, int32_t y) { return tab_of(x) < tab_of(y); });
    // every stripe lays out its own tables and two buffers, so a stripe
    // qualifies when its own layout fits
    std::vector<char> sliced(n, 0);
    size_t smem_sl = 0;
    for (int32_t i : order) {
        const size_t need = (size_t)2 * codes[i]->sl_slots * 16 + (((size_t)tab_of(i) + 255) & ~(size_t)255) + kSlotAlign;
        if (need > budget) continue;
        smem_sl = std::max(smem_sl, need);
        sliced[i] = 1;
    }
    std::vector<SliceArgs> sl;
    std::vector<CUtensorMap> maps;
    std::vector<int4> items;
    constexpr int32_t kItemSlices = 32;
    for (int32_t i = 0; i < n; ++i) {
        if (!sliced[i]) continue;
        for (int q = 0; q < codes[i]->sl_parts; ++q) {  // every part of the stripe
            SliceArgs a;
            CUtensorMap map;
            if (!slice_setup(codes[i], q, data[i], parity[i], coded[i], 1, 2, &a, &map))
                return cudaErrorInvalidValue;
            for (int32_t s0 = 0; s0 < a.n_slices; s0 += kItemSlices)
                items.push_back(make_int4((int)sl.size(), s0, std::min(a.n_slices, s0 + kItemSlices), 0));
            sl.push_back(a);
            maps.push_back(map);
        }
    }
    for (int32_t i = 0; i < n; ++i) {
        if (sliced[i]) continue;
        const fs_code *c = codes[i];
        const int32_t n_chunks = encode_chunks(c);
        RowArgs a{};
        a.tw = c->tw;
        a.n_chunks = n_chunks;
        a.hints = 0;
        for (int32_t l = 0; c->m > 0 && l < c->n_pre_levels; ++l) {
            const int32_t r0 = c->chained ? c->pre_level_off[l] : 0;
            const int32_t r1 = c->chained ? c->pre_level_off[l + 1] : c->m;
            if ((int32_t)pre.size() <= l) {
                pre.emplace_back();
                tp.push_back(0);
            }
            a.ptr = c->pre_ptr + r0;
            a.idx = c->pre_idx;
            a.inA = static_cast<const uint4 *>(data[i]);
            a.inB = c->chained ? static_cast<const uint4 *>(parity[i]) : nullptr;
            a.split = c->b;
            a.out = static_cast<uint4 *>(parity[i]) + (int64_t)r0 * c->tw;
            a.n_rows = r1 - r0;
            a.stream_out = 0;
            a.rows = 1;
            a.t0 = (int32_t)tp[l];
            tp[l] += (int64_t)n_chunks * a.n_rows;
            pre[l].push_back(a);
            if (tp[l] >= INT32_MAX - 4096) return cudaErrorInvalidValue;
        }
        if (c->n > 0) {
            a.ptr = c->con_ptr;
            a.idx = c->con_idx;
            a.inA = static_cast<const uint4 *>(data[i]);
            a.inB = static_cast<const uint4 *>(parity[i]);
            a.split = c->b;
            a.out = static_cast<uint4 *>(coded[i]);
            a.n_rows = c->n;
            a.stream_out = 1;
            a.rows = c->rows_per_ticket;
            a.t0 = (int32_t)tl;
            tl += (int64_t)n_chunks * ((c->n + a.rows - 1) / a.rows);
            lt.push_back(a);
        }
        if (tl >= INT32_MAX - 4096) return cudaErrorInvalidValue;
    }
    EncodeBatch *b = new EncodeBatch();
    b->d_pre.assign(pre.size(), nullptr);
    for (size_t l = 0; l < pre.size(); ++l) {
        b->n_pre.push_back((int)pre[l].size());
        b->t_pre.push_back((int32_t)tp[l]);
    }
    b->n_lt = (int)lt.size();
    b->t_lt = (int32_t)tl;
    b->num_sms = n > 0 ? codes[0]->num_sms : 1;
    b->ctas = n > 0 ? std::min(codes[0]->gather_ctas, kCtasPerSm) : 1;
    const int32_t zero[4] = {0, 0, 0, 0};
    b->n_items = (int)items.size();
    b->smem_sl = smem_sl;
    cudaError_t e = plan_upload(&b->d_ctr, zero, 4);
    for (size_t l = 0; l < pre.size() && e == cudaSuccess; ++l)
        e = plan_upload(&b->d_pre[l], pre[l].data(), pre[l].size());
    if (e == cudaSuccess) e = plan_upload(&b->d_lt, lt.data(), lt.size());
    if (e == cudaSuccess) e = plan_upload(&b->d_sl, sl.data(), sl.size());
    if (e == cudaSuccess) e = plan_upload(&b->d_maps, maps.data(), maps.size());
    if (e == cudaSuccess) e = plan_upload(&b->d_items, items.data(), items.size());
    if (e == cudaSuccess && b->n_items > 0)
        e = cudaFuncSetAttribute(k_slices_batch, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)b->smem_sl);
    if (e != cudaSuccess) {
        encode_batch_free(b);
        return e;
    }
    *out = b;
    return cudaSuccess;
}

cudaError_t encode_batch_run(const EncodeBatch *b, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(b->d_ctr, 0, 4 * sizeof(int32_t), s);
    if (e == cudaSuccess && b->n_items > 0) {
        const int g = b->n_items < b->num_sms ? b->n_items : b->num_sms;
        k_slices_batch<<<g, kSliceThreads, b->smem_sl, s>>>(b->d_sl, b->d_maps, b->d_items, b->n_items,
                                                           b->d_ctr + 2, b->d_ctr + 3);
        e = cudaGetLastError();
    }
    for (size_t l = 0; l < b->d_pre.size() && e == cudaSuccess; ++l) {
        if (b->t_pre[l] <= 0) continue;
        if (l > 0) e = cudaMemsetAsync(b->d_ctr, 0, sizeof(int32_t), s);  // fresh tickets
        if (e != cudaSuccess) break;
        k_rows_batch<<<grid_for(b->t_pre[l], b->num_sms, b->ctas), kEncThreads, 0, s>>>(
            b->d_pre[l], b->n_pre[l], b->t_pre[l], b->d_ctr);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && b->t_lt > 0) {
        k_rows_batch<<<grid_for(b->t_lt, b->num_sms, b->ctas), kEncThreads, 0, s>>>(
            b->d_lt, b->n_lt, b->t_lt, b->d_ctr + 1);
        e = cudaGetLastError();
    }
    return e;
}

void encode_batch_free(EncodeBatch *b) {
    if (!b) return;
    for (RowArgs *p : b->d_pre) plan_free(p);
    plan_free(b->d_lt);
    plan_free(b->d_sl);
    plan_free(b->d_maps);
    plan_free(b->d_items);
    plan_free(b->d_ctr);
    delete b;
}
