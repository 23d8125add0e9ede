// fs_peel_col.cu - the payload of the decoding path, one 16-byte byte column
// of every block at a time.
//
// The payload (Sections 3.1-3.2) sets x_f, for each pair (f, g) of the path in
// level order, to the payload of constraint g (a coded block, or zero for a
// precode check) XORed with every other intermediate of g. The slice payload
// (k_peel) keeps the recovered blocks in HBM; its gathers reach back over
// many levels, so with more recovered bytes than L2 holds most of them come
// from DRAM again. Here one CTA holds a 16-byte column of EVERY intermediate
// in shared memory (k_int + 1 slots: 67.6 KB for k_int = 4224), so one column
// is: load the coded payload that starts each recovered intermediate, walk
// every level inside shared memory, store the column of every intermediate.
// HBM then moves only the algorithmic bytes: one read of each coded payload
// the path uses and one write of each output block.
//
// k_col_plan (one CTA, right after the symbolic pass) turns the path into
//   col_src  per intermediate v, the coded row its slot starts from (-1: a
//            check's zero payload, an unrecovered v, and the zero slot k_int);
//   col_seg  16-byte records {e0..e6, f} (uint16): segment j of pair (f, g)
//            covers positions 7j .. 7j+6 of the row of g, with f itself and the
//            positions past the row's end naming the zero slot, so a record
//            needs no count and a long row splits into independent records;
//   col_step steps of at most kColSegMax segments, each inside one level (the
//            pairs of a level are independent, so a level may be cut
//            anywhere); a level whose pairs have no other neighbour has none.
// k_peel_col: persistent CTAs (as many per SM as shared memory allows) take
//   columns in turn. A column: 16-byte cp.async of every slot (zero fill for
//   -1; the source rows read in batches so their loads overlap), then the
//   steps, one thread per segment: seven slot loads, their XOR folded into
//   slot f with 32-bit shared-memory XOR reductions (segments of one pair may
//   share a step), a __syncthreads between steps; then 16-byte stores of
//   every slot. Each thread keeps its records of the next kColAhead steps in
//   registers (plain loads, issued that many steps early).
//
// Measured on one GB300 (b = 4096, m = 128, n = 5400, 64 KiB blocks, 20%
// erased): DRAM traffic falls to the algorithmic bytes (0.52 GB against the
// slice payload's 1.32 GB), but the kernel takes 0.59 ms against 0.41 ms.
// Each column moves 16 bytes per block, and those scattered 16-byte requests
// alone take 0.31 ms (32-byte columns halve that, but two columns of 4224
// slots leave one CTA per SM); the 98 steps of every column are each a
// barrier-separated round of shared-memory latency. It is therefore opt-in
// (FS_TUNE_PEEL_COLUMNS).
#include "fs_internal.cuh"

namespace {

constexpr int kPlanThreads = 1024;
constexpr int kColThreads = kColSegMax;  // one segment per thread
constexpr int kColAhead = 4;             // steps whose records a thread holds
constexpr int kColStepCap = 1024;        // step bounds kept in shared memory
constexpr int kColBatch = 8;             // source rows read before their copies
constexpr size_t kColHdr = ((size_t)4 * (kColStepCap + 1) + 127) & ~(size_t)127;

size_t col_smem_bytes(int32_t k_int) { return kColHdr + (size_t)(k_int + 1) * 16; }

size_t plan_smem_bytes(int32_t k_int) { return 4 * (2 * (size_t)k_int + 3); }

// ---------------------------------------------------------------------------
// plan

struct ColPlanArgs {
    const int32_t *con_ptr, *con_idx;
    const int32_t *pair_f, *pair_g, *level_off;
    int32_t *hdr;
    int32_t *status;
    int32_t *src, *step;
    uint4 *seg;
    int32_t k_int, n, n_con;
    int64_t max_segs, max_steps;
};

// In-place exclusive prefix sum of v[0, n) (shared memory) by the whole
// block; returns the total to every thread. s_warp holds 33 ints.
__device__ int32_t block_excl_scan(int32_t *v, int32_t n, int32_t *s_warp) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int32_t carry = 0;
    for (int32_t base = 0; base < n; base += blockDim.x) {
        const int32_t i = base + threadIdx.x;
        const int32_t x = i < n ? v[i] : 0;
        int32_t inc = x;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, inc, d);
            if (lane >= d) inc += y;
        }
        if (lane == 31) s_warp[warp] = inc;
        __syncthreads();
        if (warp == 0) {
            const int32_t t = lane < nw ? s_warp[lane] : 0;
            int32_t ti = t;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int32_t y = __shfl_up_sync(0xffffffffu, ti, d);
                if (lane >= d) ti += y;
            }
            s_warp[lane] = ti - t;
            if (lane == 31) s_warp[32] = ti;
        }
        __syncthreads();
        if (i < n) v[i] = carry + s_warp[warp] + inc - x;
        carry += s_warp[32];
        __syncthreads();  // s_warp is rewritten by the next chunk
    }
    return carry;
}

__global__ void __launch_bounds__(kPlanThreads) k_col_plan(ColPlanArgs a) {
    extern __shared__ int32_t s_cnt[];  // [K + 1] per pair: segments, then first segment
    __shared__ int32_t s_warp[33];
    __shared__ int32_t s_bad;
    const int32_t K = a.k_int;
    const int32_t np = a.hdr[WS_N_PAIRS], nl = a.hdr[WS_N_LEVELS];
    int32_t *s_lv = s_cnt + (K + 1);  // [K + 2] per level: steps, then first step
    if (threadIdx.x == 0) s_bad = (np < 0 || np > K || nl < 0 || nl > K) ? 1 : 0;
    __syncthreads();
    if (s_bad) {
        if (threadIdx.x == 0) {
            a.hdr[WS_COL_STEPS] = -1;
            atomicCAS(a.status, FS_OK, FS_ERR_INVALID);
        }
        return;
    }
    // sources and segments per pair
    for (int32_t v = threadIdx.x; v <= K; v += blockDim.x) a.src[v] = -1;
    __syncthreads();
    for (int32_t p = threadIdx.x; p < np; p += blockDim.x) {
        const int32_t f = a.pair_f[p], g = a.pair_g[p];
        int32_t cnt = 0;
        if (f >= 0 && f < K && g >= 0 && g < a.n_con) {
            a.src[f] = g < a.n ? g : -1;
            const int32_t d = a.con_ptr[g + 1] - a.con_ptr[g];
            cnt = d > 1 ? (d + kColSegEntries - 1) / kColSegEntries : 0;
        } else {
            s_bad = 1;
        }
        s_cnt[p] = cnt;
    }
    __syncthreads();
    const int32_t n_segs = block_excl_scan(s_cnt, np, s_warp);
    if (threadIdx.x == 0) s_cnt[np] = n_segs;
    // steps per level: the level's segments in runs of kColSegMax
    for (int32_t l = threadIdx.x; l < nl; l += blockDim.x) {
        const int32_t p0 = a.level_off[l], p1 = a.level_off[l + 1];
        int32_t ns = 0;
        if (p0 >= 0 && p0 <= p1 && p1 <= np) {
            const int32_t s0 = p0 < np ? s_cnt[p0] : n_segs, s1 = p1 < np ? s_cnt[p1] : n_segs;
            ns = (s1 - s0 + kColSegMax - 1) / kColSegMax;
        } else {
            s_bad = 1;
        }
        s_lv[l] = ns;
    }
    __syncthreads();
    const int32_t n_steps = block_excl_scan(s_lv, nl, s_warp);
    if (s_bad || n_segs > a.max_segs || n_steps > a.max_steps) {  // uniform: read after a barrier
        if (threadIdx.x == 0) {
            a.hdr[WS_COL_STEPS] = -1;
            atomicCAS(a.status, FS_OK, FS_ERR_INVALID);
        }
        return;
    }
    for (int32_t l = threadIdx.x; l < nl; l += blockDim.x) {
        const int32_t s0 = s_cnt[a.level_off[l]], s1 = s_cnt[a.level_off[l + 1]];
        int32_t q = s_lv[l];
        for (int32_t x = s0; x < s1; x += kColSegMax) a.step[q++] = x;
    }
    // records: one thread per segment; its pair is the last one whose first
    // segment is <= it (pairs without segments share the next pair's start)
    for (int32_t sg = threadIdx.x; sg < n_segs; sg += blockDim.x) {
        int32_t lo = 0, hi = np - 1;
        while (lo < hi) {
            const int32_t mid = (lo + hi + 1) >> 1;
            if (s_cnt[mid] <= sg)
                lo = mid;
            else
                hi = mid - 1;
        }
        const int32_t j = sg - s_cnt[lo];
        const int32_t f = a.pair_f[lo], g = a.pair_g[lo];
        const int32_t r0 = a.con_ptr[g] + j * kColSegEntries, r1 = a.con_ptr[g + 1];
        uint32_t e[kColSegEntries];
#pragma unroll
        for (int i = 0; i < kColSegEntries; ++i) {
            int32_t h = r0 + i < r1 ? a.con_idx[r0 + i] : -1;
            if (h == f || h < 0 || h >= K) h = K;
            e[i] = (uint32_t)h;
        }
        a.seg[sg] = make_uint4(e[0] | e[1] << 16, e[2] | e[3] << 16, e[4] | e[5] << 16,
                               e[6] | (uint32_t)f << 16);
    }
    if (threadIdx.x == 0) {
        a.step[n_steps] = n_segs;
        a.hdr[WS_COL_STEPS] = n_steps;
    }
}

// ---------------------------------------------------------------------------
// payload

struct ColArgs {
    const uint4 *coded;
    uint4 *data;    // intermediates v < b
    uint4 *parity;  // intermediates v >= b (workspace)
    const int32_t *src, *step;
    const uint4 *seg;
    const int32_t *hdr;
    int32_t *status;
    int32_t k_int, b;
    int64_t tw;
    int64_t max_segs, max_steps;
};

__device__ __forceinline__ uint32_t saddr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// 16-byte copy to shared memory; src_bytes 0 fills zeros (src is not read).
// Ordered against the slot reads by the wait_all + barrier that follow.
__device__ __forceinline__ void cp16_zfill(void *dst, const void *src, uint32_t src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(saddr(dst)), "l"(src),
                 "r"(src_bytes));
}

__device__ __forceinline__ void xor16(uint4 &a, const uint4 &b) {
    a.x ^= b.x;
    a.y ^= b.y;
    a.z ^= b.z;
    a.w ^= b.w;
}

__device__ __forceinline__ void red_xor16(uint4 *d, const uint4 &v) {
    const uint32_t p = saddr(d);
    asm volatile("red.shared.xor.b32 [%0], %1;\n" ::"r"(p), "r"(v.x) : "memory");
    asm volatile("red.shared.xor.b32 [%0], %1;\n" ::"r"(p + 4), "r"(v.y) : "memory");
    asm volatile("red.shared.xor.b32 [%0], %1;\n" ::"r"(p + 8), "r"(v.z) : "memory");
    asm volatile("red.shared.xor.b32 [%0], %1;\n" ::"r"(p + 12), "r"(v.w) : "memory");
}

__device__ __forceinline__ int32_t step_at(const ColArgs &a, const int32_t *s_step, int32_t i) {
    return i <= kColStepCap ? s_step[i] : __ldg(a.step + i);
}

// This thread's record of step j (zero when it has none in that step).
__device__ __forceinline__ uint4 record(const ColArgs &a, const int32_t *s_step, int32_t j,
                                        int32_t n_steps) {
    uint4 r = make_uint4(0, 0, 0, 0);
    if (j < n_steps) {
        const int32_t lo = step_at(a, s_step, j), hi = step_at(a, s_step, j + 1);
        if ((int32_t)threadIdx.x < hi - lo) r = __ldg(a.seg + lo + threadIdx.x);
    }
    return r;
}

__global__ void __launch_bounds__(kColThreads) k_peel_col(ColArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    int32_t *s_step = reinterpret_cast<int32_t *>(smem);
    uint4 *slot = reinterpret_cast<uint4 *>(smem + kColHdr);
    __shared__ int32_t s_bad;
    const int32_t K = a.k_int;
    const int32_t n_steps = a.hdr[WS_COL_STEPS];
    if (n_steps < 0 || n_steps > a.max_steps) {  // no plan for this path
        if (threadIdx.x == 0 && blockIdx.x == 0) atomicCAS(a.status, FS_OK, FS_ERR_INVALID);
        return;
    }
    if (threadIdx.x == 0) s_bad = 0;
    for (int32_t i = threadIdx.x; i <= n_steps && i <= kColStepCap; i += blockDim.x)
        s_step[i] = a.step[i];
    __syncthreads();
    for (int32_t i = threadIdx.x; i < n_steps; i += blockDim.x) {
        const int32_t lo = step_at(a, s_step, i), hi = step_at(a, s_step, i + 1);
        if (lo < 0 || hi - lo <= 0 || hi - lo > kColSegMax || hi > a.max_segs) s_bad = 1;
    }
    __syncthreads();
    if (s_bad) {  // a plan that would index outside its arrays: leave the output alone
        if (threadIdx.x == 0 && blockIdx.x == 0) atomicCAS(a.status, FS_OK, FS_ERR_INVALID);
        return;
    }
    for (int64_t col = blockIdx.x; col < a.tw; col += gridDim.x) {
        for (int32_t base = threadIdx.x; base <= K; base += kColThreads * kColBatch) {
            int32_t g[kColBatch];
#pragma unroll
            for (int u = 0; u < kColBatch; ++u) {
                const int32_t v = base + u * kColThreads;
                g[u] = v <= K ? __ldg(a.src + v) : -2;
            }
#pragma unroll
            for (int u = 0; u < kColBatch; ++u)
                if (g[u] != -2)
                    cp16_zfill(slot + base + u * kColThreads,
                               g[u] >= 0 ? a.coded + (int64_t)g[u] * a.tw + col : a.coded,
                               g[u] >= 0 ? 16u : 0u);
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
        uint4 pf[kColAhead];
#pragma unroll
        for (int d = 0; d < kColAhead; ++d) pf[d] = record(a, s_step, d, n_steps);
        asm volatile("cp.async.wait_all;\n" ::: "memory");
        __syncthreads();
        for (int32_t i = 0; i < n_steps; ++i) {
            const uint4 rec = pf[0];
#pragma unroll
            for (int d = 0; d + 1 < kColAhead; ++d) pf[d] = pf[d + 1];
            pf[kColAhead - 1] = record(a, s_step, i + kColAhead, n_steps);
            if ((int32_t)threadIdx.x < step_at(a, s_step, i + 1) - step_at(a, s_step, i)) {
                uint4 acc = slot[rec.x & 0xffffu];
                xor16(acc, slot[rec.x >> 16]);
                xor16(acc, slot[rec.y & 0xffffu]);
                xor16(acc, slot[rec.y >> 16]);
                xor16(acc, slot[rec.z & 0xffffu]);
                xor16(acc, slot[rec.z >> 16]);
                xor16(acc, slot[rec.w & 0xffffu]);
                red_xor16(slot + (rec.w >> 16), acc);
            }
            __syncthreads();
        }
        for (int32_t v = threadIdx.x; v < K; v += blockDim.x) {
            const uint4 x = slot[v];
            if (v < a.b)
                a.data[(int64_t)v * a.tw + col] = x;
            else
                a.parity[(int64_t)(v - a.b) * a.tw + col] = x;
        }
        __syncthreads();  // the next column's copies overwrite the slots
    }
}

}  // namespace

bool col_fits(const fs_code *c) {
    return c->k_int >= 1 && c->k_int + 1 <= 65535 && c->tw >= 1 &&
           col_smem_bytes(c->k_int) <= c->smem_optin && plan_smem_bytes(c->k_int) <= c->smem_optin;
}

cudaError_t launch_col_plan(const fs_code *c, uint8_t *ws, cudaStream_t s) {
    const DecodeLayout L = decode_layout(c);
    ColPlanArgs a;
    a.con_ptr = c->con_ptr;
    a.con_idx = c->con_idx;
    a.pair_f = reinterpret_cast<const int32_t *>(ws + L.pair_f);
    a.pair_g = reinterpret_cast<const int32_t *>(ws + L.pair_g);
    a.level_off = reinterpret_cast<const int32_t *>(ws + L.level_off);
    a.hdr = reinterpret_cast<int32_t *>(ws);
    a.status = reinterpret_cast<int32_t *>(ws) + WS_STATUS;
    a.src = reinterpret_cast<int32_t *>(ws + L.col_src);
    a.step = reinterpret_cast<int32_t *>(ws + L.col_step);
    a.seg = reinterpret_cast<uint4 *>(ws + L.col_seg);
    a.k_int = c->k_int;
    a.n = c->n;
    a.n_con = c->n_con;
    a.max_segs = L.col_max_segs;
    a.max_steps = L.col_max_steps;
    const size_t smem = plan_smem_bytes(c->k_int);
    if (smem > 48 * 1024) {
        cudaError_t e =
            cudaFuncSetAttribute(k_col_plan, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_col_plan<<<1, kPlanThreads, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_peel_col(const fs_code *c, const uint4 *coded, uint4 *data_out, uint8_t *ws,
                            cudaStream_t s) {
    const DecodeLayout L = decode_layout(c);
    ColArgs a;
    a.coded = coded;
    a.data = data_out;
    a.parity = reinterpret_cast<uint4 *>(ws + L.parity);
    a.src = reinterpret_cast<const int32_t *>(ws + L.col_src);
    a.step = reinterpret_cast<const int32_t *>(ws + L.col_step);
    a.seg = reinterpret_cast<const uint4 *>(ws + L.col_seg);
    a.hdr = reinterpret_cast<const int32_t *>(ws);
    a.status = reinterpret_cast<int32_t *>(ws) + WS_STATUS;
    a.k_int = c->k_int;
    a.b = c->b;
    a.tw = c->tw;
    a.max_segs = L.col_max_segs;
    a.max_steps = L.col_max_steps;
    const size_t smem = col_smem_bytes(c->k_int);
    cudaError_t e =
        cudaFuncSetAttribute(k_peel_col, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_peel_col, kColThreads, smem);
    if (e != cudaSuccess) return e;
    if (occ < 1) occ = 1;
    int64_t grid = (int64_t)c->num_sms * occ;
    if (grid > c->tw) grid = c->tw;
    k_peel_col<<<(unsigned)grid, kColThreads, smem, s>>>(a);
    return cudaGetLastError();
}
