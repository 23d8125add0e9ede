// fs_encode.cu - encoding (Section 2.2, steps (1) precode and (2) LDGM) as
// one persistent launch.
//
// Tiles are (row, chunk of kEncV * kEncThreads 16-byte words). A CTA takes
// tiles in ticket order from an atomic counter. Within the order, the m
// parity tiles of chunk c+1 come before the LT tiles of chunk c:
//     P0 P1 L0 P2 L1 ... P(C-1) L(C-2) L(C-1)
// so the resident CTAs all work on about one byte range of every block at a
// time (its k_int blocks stay in L2 while the rows that share them are
// computed) and parities are ready one chunk ahead of the rows that read
// them. An LT row that has a parity neighbour (its largest index is >= b)
// waits until every parity tile of its chunk is done (a per-chunk counter).
// The wait cannot deadlock: tickets are taken in order by CTAs that are
// running, so every parity tile of the chunk was taken earlier by a running
// CTA, and parity tiles never wait. The wait is still bounded; past the
// bound the call reports FS_ERR_TIMEOUT in the workspace status word.
#include "fs_internal.cuh"

namespace {

constexpr int kEncThreads = 256;
constexpr int kEncV = 2;  // words per thread per tile
constexpr long long kSpinLimit = 1ll << 22;

struct EncArgs {
    const int32_t *lt_ptr, *lt_idx, *pre_ptr, *pre_idx;
    const uint4 *data;
    uint4 *parity, *coded;
    int32_t b, m, n;
    int64_t tw;
    int32_t chunk_w, n_chunks;
    int32_t *tile_ctr, *done, *status;
};

__device__ __forceinline__ void xor4(uint4 &a, const uint4 &b) {
    a.x ^= b.x;
    a.y ^= b.y;
    a.z ^= b.z;
    a.w ^= b.w;
}

// Input block v: data for v < b (read-only for the whole launch), parity
// otherwise (written by this launch: read through L2 only).
__device__ __forceinline__ uint4 load_in(const EncArgs &a, int32_t v, int64_t w) {
    if (v < a.b) return __ldg(a.data + (int64_t)v * a.tw + w);
    return __ldcg(a.parity + (int64_t)(v - a.b) * a.tw + w);
}

// out[w] = XOR of in(idx[e])[w] for e in [e0, e1), for the kEncV words of
// this thread in [w0, w1).
// kStream: the output is not read again in this launch (coded rows): store
// with evict-first so L2 keeps the inputs of the current chunk.
template <bool kDataOnly, bool kStream>
__device__ __forceinline__ void gather_row(const EncArgs &a, const int32_t *idx, int32_t e0,
                                           int32_t e1, int64_t w0, int64_t w1, uint4 *out) {
    int64_t w[kEncV];
    bool ok[kEncV];
    uint4 acc[kEncV];
#pragma unroll
    for (int k = 0; k < kEncV; ++k) {
        w[k] = w0 + threadIdx.x + (int64_t)k * kEncThreads;
        ok[k] = w[k] < w1;
        acc[k] = make_uint4(0, 0, 0, 0);
    }
    int32_t e = e0;
    for (; e + 4 <= e1; e += 4) {
        int32_t v[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) v[j] = __ldg(idx + e + j);
        uint4 x[4][kEncV];
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int k = 0; k < kEncV; ++k)
                x[j][k] = ok[k] ? (kDataOnly ? __ldg(a.data + (int64_t)v[j] * a.tw + w[k])
                                             : load_in(a, v[j], w[k]))
                                : make_uint4(0, 0, 0, 0);
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int k = 0; k < kEncV; ++k) xor4(acc[k], x[j][k]);
    }
    for (; e < e1; ++e) {
        const int32_t v = __ldg(idx + e);
#pragma unroll
        for (int k = 0; k < kEncV; ++k)
            if (ok[k])
                xor4(acc[k], kDataOnly ? __ldg(a.data + (int64_t)v * a.tw + w[k])
                                       : load_in(a, v, w[k]));
    }
#pragma unroll
    for (int k = 0; k < kEncV; ++k) {
        if (!ok[k]) continue;
        if (kStream) __stcs(out + w[k], acc[k]);
        else __stcg(out + w[k], acc[k]);
    }
}

// Ticket t -> (is_parity, row, chunk) in the order P0 P1 L0 P2 L1 ...
__device__ __forceinline__ void decode_ticket(const EncArgs &a, int64_t t, bool *par, int32_t *row,
                                              int32_t *chunk) {
    const int64_t m = a.m, n = a.n, C = a.n_chunks;
    const int64_t head = m < 1 ? 0 : (C > 1 ? 2 * m : m);  // P0 (and P1)
    if (t < head) {
        *par = true;
        *chunk = (int32_t)(t / m);
        *row = (int32_t)(t - (int64_t)(*chunk) * m);
        return;
    }
    t -= head;
    // groups of (L c, then P c+2), for c = 0 .. C-1 (no P beyond C-1)
    const int64_t group = n + m;
    const int64_t full = C > 2 ? C - 2 : 0;  // groups that carry a parity part
    if (m > 0 && t < full * group) {
        const int64_t c = t / group, r = t - c * group;
        if (r < n) {
            *par = false;
            *chunk = (int32_t)c;
            *row = (int32_t)r;
        } else {
            *par = true;
            *chunk = (int32_t)(c + 2);
            *row = (int32_t)(r - n);
        }
        return;
    }
    if (m > 0) t -= full * group;
    const int64_t c0 = (m > 0) ? full : 0;
    if (n == 0) {  // unreachable: with no LT rows every ticket is a parity tile
        *par = true;
        *chunk = 0;
        *row = 0;
        return;
    }
    const int64_t c = c0 + t / n;
    *par = false;
    *chunk = (int32_t)c;
    *row = (int32_t)(t - (c - c0) * n);
}

__global__ void __launch_bounds__(kEncThreads, 4) k_encode(EncArgs a) {
    __shared__ int64_t s_tile;
    const int64_t n_tiles = (int64_t)a.n_chunks * (a.m + a.n);
    if (threadIdx.x == 0) s_tile = atomicAdd(a.tile_ctr, 1);
    __syncthreads();
    int64_t t = s_tile;
    while (t < n_tiles) {
        __syncthreads();  // every thread has read s_tile
        int32_t nxt = 0;
        if (threadIdx.x == 0) nxt = atomicAdd(a.tile_ctr, 1);  // in flight during the tile
        bool par;
        int32_t row, chunk;
        decode_ticket(a, t, &par, &row, &chunk);
        const int64_t w0 = (int64_t)chunk * a.chunk_w;
        const int64_t w1 = min(w0 + a.chunk_w, a.tw);
        if (par) {
            const int32_t e0 = __ldg(a.pre_ptr + row), e1 = __ldg(a.pre_ptr + row + 1);
            gather_row<true, false>(a, a.pre_idx, e0, e1, w0, w1, a.parity + (int64_t)row * a.tw);
            __threadfence();  // this thread's parity words are visible device-wide
            __syncthreads();  // ... for every thread of the tile
            if (threadIdx.x == 0) atomicAdd(a.done + chunk, 1);
        } else {
            const int32_t e0 = __ldg(a.lt_ptr + row), e1 = __ldg(a.lt_ptr + row + 1);
            const bool needs_parity = e1 > e0 && __ldg(a.lt_idx + e1 - 1) >= a.b;
            if (needs_parity) {
                if (threadIdx.x == 0) {
                    long long spins = 0;
                    while (atomicAdd(a.done + chunk, 0) < a.m) {
                        if (++spins > kSpinLimit) {
                            atomicExch(a.status, FS_ERR_TIMEOUT);
                            break;
                        }
                        __nanosleep(128);
                    }
                    __threadfence();
                }
                __syncthreads();
                gather_row<false, true>(a, a.lt_idx, e0, e1, w0, w1, a.coded + (int64_t)row * a.tw);
            } else {
                gather_row<true, true>(a, a.lt_idx, e0, e1, w0, w1, a.coded + (int64_t)row * a.tw);
            }
        }
        if (threadIdx.x == 0) s_tile = nxt;
        __syncthreads();
        t = s_tile;
    }
}

}  // namespace

int32_t encode_chunks(const fs_code *c) {
    const int64_t cw = (int64_t)kEncV * kEncThreads;
    return (int32_t)((c->tw + cw - 1) / cw);
}

size_t encode_ws_bytes(const fs_code *c) {
    return fs_align256(WS_HDR_BYTES + 4 * ((size_t)encode_chunks(c) + 1));
}

cudaError_t launch_encode(const fs_code *c, const void *data, void *parity, void *coded, uint8_t *ws,
                          cudaStream_t s) {
    EncArgs a;
    a.lt_ptr = c->con_ptr;
    a.lt_idx = c->con_idx;
    a.pre_ptr = c->pre_ptr;
    a.pre_idx = c->pre_idx;
    a.data = static_cast<const uint4 *>(data);
    a.parity = static_cast<uint4 *>(parity);
    a.coded = static_cast<uint4 *>(coded);
    a.b = c->b;
    a.m = c->m;
    a.n = c->n;
    a.tw = c->tw;
    a.n_chunks = encode_chunks(c);
    a.chunk_w = (int32_t)((int64_t)kEncV * kEncThreads);
    a.status = reinterpret_cast<int32_t *>(ws) + WS_STATUS;
    a.tile_ctr = reinterpret_cast<int32_t *>(ws) + WS_TILE_CTR;
    a.done = reinterpret_cast<int32_t *>(ws + WS_HDR_BYTES);
    // status, ticket counter and per-chunk parity counters start at zero
    cudaError_t e = cudaMemsetAsync(ws, 0, WS_HDR_BYTES + 4 * ((size_t)a.n_chunks + 1), s);
    if (e != cudaSuccess) return e;
    const int64_t n_tiles = (int64_t)a.n_chunks * (a.m + a.n);
    if (n_tiles == 0) return cudaSuccess;
    int64_t grid = (int64_t)c->num_sms * c->gather_ctas;
    if (grid > n_tiles) grid = n_tiles;
    k_encode<<<(unsigned)grid, kEncThreads, 0, s>>>(a);
    return cudaGetLastError();
}
