// fs_gather.cu - region-XOR gather kernels: encode (Section 2.2 steps (1)
// and (2)), conventional repair (Section 4) and the delta-XOR update.
//
// Work unit: a tile = (CSR row r, byte chunk of 16 KiB) of one output block.
// A tile first lists its sources (the row's neighbours; for the update only
// the neighbours that changed) as block pointers in shared memory, then every
// thread streams 4 words from each source, two sources at a time, so each
// thread keeps 8 independent 16-byte loads in flight. Tiles are numbered
// chunk-major, so the CTAs resident at one time work on about the same byte
// range of every block.
#include "fs_internal.cuh"

namespace {

constexpr int kGatherThreads = 256;
constexpr int kWpt = 4;                             // 16-byte words per thread per tile
constexpr int kChunkW = kGatherThreads * kWpt;      // words per tile (16 KiB)
constexpr int kSrcBatch = kGatherThreads;           // sources listed at a time
constexpr int kCtasPerSm = 8;

__device__ __forceinline__ void xor4(uint4 &a, const uint4 &b) {
    a.x ^= b.x;
    a.y ^= b.y;
    a.z ^= b.z;
    a.w ^= b.w;
}

__device__ __forceinline__ const uint4 *in_block(const GatherArgs &a, int32_t v) {
    return (v < a.split) ? a.inA + (int64_t)v * a.tw : a.inB + (int64_t)(v - a.split) * a.tw;
}

// acc[i] ^= src[k][w0 + threadIdx.x + i * blockDim.x] over the n listed sources
__device__ __forceinline__ void xor_sources(uint4 *acc, const uint4 *const *src, int n, int64_t w0,
                                            int64_t w1) {
    int64_t w[kWpt];
    bool ok[kWpt];
#pragma unroll
    for (int i = 0; i < kWpt; ++i) {
        w[i] = w0 + threadIdx.x + (int64_t)i * kGatherThreads;
        ok[i] = w[i] < w1;
    }
    int k = 0;
    for (; k + 2 <= n; k += 2) {
        const uint4 *s0 = src[k], *s1 = src[k + 1];
        uint4 x0[kWpt], x1[kWpt];
#pragma unroll
        for (int i = 0; i < kWpt; ++i) {
            x0[i] = ok[i] ? __ldg(s0 + w[i]) : make_uint4(0, 0, 0, 0);
            x1[i] = ok[i] ? __ldg(s1 + w[i]) : make_uint4(0, 0, 0, 0);
        }
#pragma unroll
        for (int i = 0; i < kWpt; ++i) {
            xor4(acc[i], x0[i]);
            xor4(acc[i], x1[i]);
        }
    }
    if (k < n) {
#pragma unroll
        for (int i = 0; i < kWpt; ++i)
            if (ok[i]) xor4(acc[i], __ldg(src[k] + w[i]));
    }
}

__global__ void __launch_bounds__(kGatherThreads, 4)
k_gather_xor(GatherArgs a, int32_t n_chunks) {
    __shared__ const uint4 *s_src[kSrcBatch];
    // without a row list nothing here can fail: report a clean call
    if (!a.rows && blockIdx.x == 0 && threadIdx.x == 0) *a.status = FS_OK;
    const int64_t n_tiles = (int64_t)n_chunks * a.n_rows;
    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const int32_t chunk = (int32_t)(tile / a.n_rows);
        const int32_t r = (int32_t)(tile - (int64_t)chunk * a.n_rows);
        int32_t row = a.row_base + r;
        if (a.rows) {
            row = __ldg(a.rows + r);
            if (row < 0 || row >= a.n_valid) {  // the same decision in every thread
                if (threadIdx.x == 0 && chunk == 0) atomicExch(a.status, FS_ERR_INVALID);
                continue;
            }
        }
        const int32_t e0 = __ldg(a.ptr + row), e1 = __ldg(a.ptr + row + 1);
        const int64_t w0 = (int64_t)chunk * kChunkW;
        const int64_t w1 = min(w0 + kChunkW, a.tw);
        uint4 acc[kWpt];
#pragma unroll
        for (int i = 0; i < kWpt; ++i) acc[i] = make_uint4(0, 0, 0, 0);
        for (int32_t base = e0; base < e1; base += kSrcBatch) {
            const int nb = min(kSrcBatch, e1 - base);
            __syncthreads();  // the previous batch is consumed
            if ((int)threadIdx.x < nb) s_src[threadIdx.x] = in_block(a, __ldg(a.idx + base + threadIdx.x));
            __syncthreads();
            xor_sources(acc, s_src, nb, w0, w1);
        }
        uint4 *dst = a.out + (int64_t)row * a.tw;
#pragma unroll
        for (int i = 0; i < kWpt; ++i) {
            const int64_t w = w0 + threadIdx.x + (int64_t)i * kGatherThreads;
            if (w < w1) __stcs(dst + w, acc[i]);
        }
    }
}

struct UpdArgs {
    const int32_t *idx;
    int32_t n_idx;
    const uint4 *d_new;
    uint4 *data, *parity, *coded;
    uint4 *delta, *pdelta;
    int32_t *mark, *pmark, *cmark, *plist, *clist;
    int32_t *n_plist, *n_clist;
    const int32_t *con_ptr, *con_idx, *pre_ptr, *pre_idx, *var_ptr, *var_idx;
    int32_t b, m, n;
    int64_t tw;
    int32_t *status;
};

__device__ __forceinline__ bool upd_ok(const UpdArgs &a) {
    return *(volatile int32_t *)a.status == FS_OK;
}

// One CTA: mark[i] = -1, pmark[j] = cmark[g] = 0, list counts 0, status
// FS_OK; then mark[idx[q]] = q (a repeated or out-of-range index flags the
// call invalid).
__global__ void __launch_bounds__(1024) k_update_init(UpdArgs a) {
    if (threadIdx.x == 0) {
        *a.status = FS_OK;
        *a.n_plist = 0;
        *a.n_clist = 0;
    }
    for (int64_t i = threadIdx.x; i < a.b; i += blockDim.x) a.mark[i] = -1;
    for (int64_t j = threadIdx.x; j < a.m; j += blockDim.x) a.pmark[j] = 0;
    for (int64_t g = threadIdx.x; g < a.n; g += blockDim.x) a.cmark[g] = 0;
    __syncthreads();
    for (int32_t q = threadIdx.x; q < a.n_idx; q += blockDim.x) {
        const int32_t i = a.idx[q];
        if (i < 0 || i >= a.b) {
            atomicExch(a.status, FS_ERR_INVALID);
            continue;
        }
        if (atomicCAS(a.mark + i, -1, q) != -1) atomicExch(a.status, FS_ERR_INVALID);
    }
}

// Appends constraint c (containing a changed variable) to its list once.
__device__ __forceinline__ void touch(const UpdArgs &a, int32_t c, bool coded_only) {
    if (c < a.n) {
        if (atomicExch(a.cmark + c, 1) == 0) a.clist[atomicAdd(a.n_clist, 1)] = c;
    } else if (!coded_only) {
        const int32_t j = c - a.n;
        if (atomicExch(a.pmark + j, 1) == 0) a.plist[atomicAdd(a.n_plist, 1)] = j;
    }
}

// Tiles (q, chunk): delta_q = old ^ new and data block idx[q] <- new over
// the chunk; the chunk-0 tile of q also lists every constraint containing
// that block (coded rows and checks).
__global__ void __launch_bounds__(kGatherThreads, 4)
k_update_delta(UpdArgs a, int32_t n_chunks) {
    if (!upd_ok(a)) return;
    const int64_t n_tiles = (int64_t)a.n_idx * n_chunks;
    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const int32_t q = (int32_t)(tile / n_chunks);
        const int32_t chunk = (int32_t)(tile - (int64_t)q * n_chunks);
        const int32_t i = a.idx[q];
        const int64_t w0 = (int64_t)chunk * kChunkW, w1 = min(w0 + kChunkW, a.tw);
        uint4 nw[kWpt], d[kWpt];
#pragma unroll
        for (int k = 0; k < kWpt; ++k) {
            const int64_t w = w0 + threadIdx.x + (int64_t)k * kGatherThreads;
            if (w < w1) {
                nw[k] = __ldg(a.d_new + (int64_t)q * a.tw + w);
                d[k] = a.data[(int64_t)i * a.tw + w];
            }
        }
#pragma unroll
        for (int k = 0; k < kWpt; ++k) {
            const int64_t w = w0 + threadIdx.x + (int64_t)k * kGatherThreads;
            if (w < w1) {
                xor4(d[k], nw[k]);
                a.delta[(int64_t)q * a.tw + w] = d[k];
                a.data[(int64_t)i * a.tw + w] = nw[k];
            }
        }
        if (chunk == 0)
            for (int32_t e = a.var_ptr[i] + threadIdx.x; e < a.var_ptr[i + 1]; e += blockDim.x)
                touch(a, a.var_idx[e], false);
    }
}

// Lists, in s_src, the deltas of the changed members among con_idx-style
// entries [base, base + nb) (data block v: its delta if it was rewritten;
// v >= b: parity v - b's delta if that check changed). Returns the count.
__device__ __forceinline__ int list_changed(const UpdArgs &a, const int32_t *members, int32_t base,
                                            int nb, const uint4 **s_src, int *s_n) {
    __syncthreads();  // the previous list is consumed
    if (threadIdx.x == 0) *s_n = 0;
    __syncthreads();
    if ((int)threadIdx.x < nb) {
        const int32_t v = members[base + threadIdx.x];
        const uint4 *p = nullptr;
        if (v < a.b) {
            const int32_t q = a.mark[v];
            if (q >= 0) p = a.delta + (int64_t)q * a.tw;
        } else if (a.pmark[v - a.b]) {
            p = a.pdelta + (int64_t)(v - a.b) * a.tw;
        }
        if (p) s_src[atomicAdd(s_n, 1)] = p;
    }
    __syncthreads();
    return *s_n;
}

// changed parity j ^= XOR of the deltas of its changed members; pdelta_j
// keeps that XOR; the chunk-0 tile of check j also lists the constraints
// that contain parity b + j (coded rows, and in a chained precode the later
// checks that read it). Only listed checks j in [j0, j1) (one precode level)
// are taken: a chained precode runs one launch per level, so every parity a
// check reads has its delta before the check does. Tiles (listed check,
// chunk), chunk-major.
__global__ void __launch_bounds__(kGatherThreads, 3)
k_update_parity(UpdArgs a, int32_t n_chunks, int32_t j0, int32_t j1) {
    __shared__ const uint4 *s_src[kSrcBatch];
    __shared__ int s_n, s_ok;
    if (threadIdx.x == 0) s_ok = upd_ok(a);  // one decision for the whole CTA
    __syncthreads();
    if (!s_ok) return;
    const int32_t np = *(volatile int32_t *)a.n_plist;
    const int64_t n_tiles = (int64_t)n_chunks * np;
    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const int32_t chunk = (int32_t)(tile / np);
        const int32_t j = a.plist[tile - (int64_t)chunk * np];
        if (j < j0 || j >= j1) continue;  // another level's check (uniform over the CTA)
        const int32_t e0 = a.pre_ptr[j], e1 = a.pre_ptr[j + 1];
        const int64_t w0 = (int64_t)chunk * kChunkW, w1 = min(w0 + kChunkW, a.tw);
        if (chunk == 0) {
            const int32_t v = a.b + j;
            for (int32_t e = a.var_ptr[v] + threadIdx.x; e < a.var_ptr[v + 1]; e += blockDim.x)
                touch(a, a.var_idx[e], false);
        }
        uint4 acc[kWpt];
#pragma unroll
        for (int i = 0; i < kWpt; ++i) acc[i] = make_uint4(0, 0, 0, 0);
        for (int32_t base = e0; base < e1; base += kSrcBatch) {
            const int n = list_changed(a, a.pre_idx, base, min(kSrcBatch, e1 - base), s_src, &s_n);
            xor_sources(acc, s_src, n, w0, w1);
        }
#pragma unroll
        for (int i = 0; i < kWpt; ++i) {
            const int64_t w = w0 + threadIdx.x + (int64_t)i * kGatherThreads;
            if (w >= w1) continue;
            a.pdelta[(int64_t)j * a.tw + w] = acc[i];
            uint4 p = a.parity[(int64_t)j * a.tw + w];
            xor4(p, acc[i]);
            a.parity[(int64_t)j * a.tw + w] = p;
        }
    }
}

// listed coded row g ^= XOR of the deltas of its changed neighbours (data
// blocks and parities). Tiles (listed row, chunk), chunk-major.
__global__ void __launch_bounds__(kGatherThreads, 3)
k_update_coded(UpdArgs a, int32_t n_chunks) {
    __shared__ const uint4 *s_src[kSrcBatch];
    __shared__ int s_n, s_ok;
    if (threadIdx.x == 0) s_ok = upd_ok(a);
    __syncthreads();
    if (!s_ok) return;
    const int32_t nc = *(volatile int32_t *)a.n_clist;
    const int64_t n_tiles = (int64_t)n_chunks * nc;
    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const int32_t chunk = (int32_t)(tile / nc);
        const int32_t g = a.clist[tile - (int64_t)chunk * nc];
        const int32_t e0 = a.con_ptr[g], e1 = a.con_ptr[g + 1];
        const int64_t w0 = (int64_t)chunk * kChunkW, w1 = min(w0 + kChunkW, a.tw);
        uint4 acc[kWpt];
#pragma unroll
        for (int i = 0; i < kWpt; ++i) {
            const int64_t w = w0 + threadIdx.x + (int64_t)i * kGatherThreads;
            acc[i] = w < w1 ? a.coded[(int64_t)g * a.tw + w] : make_uint4(0, 0, 0, 0);
        }
        for (int32_t base = e0; base < e1; base += kSrcBatch) {
            const int n = list_changed(a, a.con_idx, base, min(kSrcBatch, e1 - base), s_src, &s_n);
            xor_sources(acc, s_src, n, w0, w1);
        }
#pragma unroll
        for (int i = 0; i < kWpt; ++i) {
            const int64_t w = w0 + threadIdx.x + (int64_t)i * kGatherThreads;
            if (w < w1) a.coded[(int64_t)g * a.tw + w] = acc[i];
        }
    }
}

inline int32_t chunks_of(int64_t tw) { return (int32_t)((tw + kChunkW - 1) / kChunkW); }

inline int grid_for(int64_t n_tiles, int num_sms, int ctas_per_sm = kCtasPerSm) {
    const int64_t cap = (int64_t)num_sms * ctas_per_sm;
    const int64_t g = n_tiles < cap ? n_tiles : cap;
    return (int)(g < 1 ? 1 : g);
}

}  // namespace

cudaError_t launch_gather(const GatherArgs &a, int num_sms, int ctas_per_sm, cudaStream_t s) {
    if (a.n_rows <= 0 || a.tw <= 0) return cudaSuccess;
    const int32_t n_chunks = chunks_of(a.tw);
    k_gather_xor<<<grid_for((int64_t)n_chunks * a.n_rows, num_sms, ctas_per_sm), kGatherThreads, 0, s>>>(
        a, n_chunks);
    return cudaGetLastError();
}

cudaError_t launch_update(const fs_code *c, const int32_t *idx, int32_t n_idx, const uint4 *d_new,
                          uint4 *data, uint4 *parity, uint4 *coded, uint8_t *ws, cudaStream_t s) {
    const UpdateLayout L = update_layout(c, n_idx);
    UpdArgs a;
    a.idx = idx;
    a.n_idx = n_idx;
    a.d_new = d_new;
    a.data = data;
    a.parity = parity;
    a.coded = coded;
    a.delta = reinterpret_cast<uint4 *>(ws + L.delta);
    a.pdelta = reinterpret_cast<uint4 *>(ws + L.pdelta);
    a.mark = reinterpret_cast<int32_t *>(ws + L.mark);
    a.pmark = reinterpret_cast<int32_t *>(ws + L.pmark);
    a.cmark = reinterpret_cast<int32_t *>(ws + L.cmark);
    a.plist = reinterpret_cast<int32_t *>(ws + L.plist);
    a.clist = reinterpret_cast<int32_t *>(ws + L.clist);
    a.n_plist = reinterpret_cast<int32_t *>(ws) + WS_COUNT_A;
    a.n_clist = reinterpret_cast<int32_t *>(ws) + WS_COUNT_B;
    a.con_ptr = c->con_ptr;
    a.con_idx = c->con_idx;
    a.pre_ptr = c->pre_ptr;
    a.pre_idx = c->pre_idx;
    a.var_ptr = c->var_ptr;
    a.var_idx = c->var_idx;
    a.b = c->b;
    a.m = c->m;
    a.n = c->n;
    a.tw = c->tw;
    a.status = reinterpret_cast<int32_t *>(ws) + WS_STATUS;

    k_update_init<<<1, 1024, 0, s>>>(a);
    if (n_idx > 0) {
        const int32_t n_chunks = chunks_of(c->tw);
        k_update_delta<<<grid_for((int64_t)n_idx * n_chunks, c->num_sms), kGatherThreads, 0, s>>>(
            a, n_chunks);
        for (int32_t l = 0; l < c->n_pre_levels; ++l) {  // one level of checks per launch
            const int32_t j0 = c->chained ? c->pre_level_off[l] : 0;
            const int32_t j1 = c->chained ? c->pre_level_off[l + 1] : c->m;
            k_update_parity<<<grid_for((int64_t)n_chunks * c->m, c->num_sms), kGatherThreads, 0, s>>>(
                a, n_chunks, j0, j1);
        }
        if (c->n > 0)
            k_update_coded<<<grid_for((int64_t)n_chunks * c->n, c->num_sms), kGatherThreads, 0, s>>>(
                a, n_chunks);
    }
    return cudaGetLastError();
}
