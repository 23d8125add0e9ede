// fs_gather.cu - region-XOR gather kernels: encode (Section 2.2 steps (1)
// and (2)), conventional repair (Section 4) and the delta-XOR update.
//
// Work unit: a tile = (CSR row r, byte chunk) of one output block. Tiles are
// numbered chunk-major, so the CTAs resident at one time all work on the same
// byte range of every block: the gathered inputs of that range (k_int blocks
// x one chunk) stay in L2 while the rows that share them are computed, and
// each input byte is fetched from HBM about once per launch.
#include "fs_internal.cuh"

namespace {

constexpr int kGatherThreads = 256;  // one 16-byte word per thread per chunk
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

__global__ void __launch_bounds__(kGatherThreads)
k_gather_xor(GatherArgs a, int32_t chunk_w, int32_t n_chunks) {
    // without a row list nothing here can fail: report a clean call
    if (!a.rows && blockIdx.x == 0 && threadIdx.x == 0) *a.status = FS_OK;
    const int64_t n_tiles = (int64_t)n_chunks * a.n_rows;
    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const int32_t chunk = (int32_t)(tile / a.n_rows);
        const int32_t r = (int32_t)(tile - (int64_t)chunk * a.n_rows);
        int32_t row = a.row_base + r;
        if (a.rows) {
            row = __ldg(a.rows + r);
            if (row < 0 || row >= a.n_valid) {
                if (threadIdx.x == 0 && chunk == 0) atomicExch(a.status, FS_ERR_INVALID);
                continue;
            }
        }
        const int32_t e0 = __ldg(a.ptr + row), e1 = __ldg(a.ptr + row + 1);
        const int64_t w0 = (int64_t)chunk * chunk_w;
        const int64_t w1 = min(w0 + chunk_w, a.tw);
        uint4 *dst = a.out + (int64_t)row * a.tw;
        for (int64_t w = w0 + threadIdx.x; w < w1; w += blockDim.x) {
            uint4 acc = make_uint4(0, 0, 0, 0);
            int32_t e = e0;
            for (; e + 4 <= e1; e += 4) {
                const int32_t v0 = __ldg(a.idx + e), v1 = __ldg(a.idx + e + 1);
                const int32_t v2 = __ldg(a.idx + e + 2), v3 = __ldg(a.idx + e + 3);
                const uint4 x0 = __ldg(in_block(a, v0) + w);
                const uint4 x1 = __ldg(in_block(a, v1) + w);
                const uint4 x2 = __ldg(in_block(a, v2) + w);
                const uint4 x3 = __ldg(in_block(a, v3) + w);
                xor4(acc, x0);
                xor4(acc, x1);
                xor4(acc, x2);
                xor4(acc, x3);
            }
            for (; e < e1; ++e) xor4(acc, __ldg(in_block(a, __ldg(a.idx + e)) + w));
            __stcs(dst + w, acc);
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

// mark[i] = -1, pmark[j] = cmark[g] = 0, list counts 0, status FS_OK
__global__ void k_update_init(UpdArgs a) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i0 == 0) {
        *a.status = FS_OK;
        *a.n_plist = 0;
        *a.n_clist = 0;
    }
    for (int64_t i = i0; i < a.b; i += stride) a.mark[i] = -1;
    for (int64_t j = i0; j < a.m; j += stride) a.pmark[j] = 0;
    for (int64_t g = i0; g < a.n; g += stride) a.cmark[g] = 0;
}

// mark[idx[q]] = q; a repeated or out-of-range index flags the call invalid
__global__ void k_update_mark(UpdArgs a) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < a.n_idx; q += stride) {
        const int32_t i = a.idx[q];
        if (i < 0 || i >= a.b) {
            atomicExch(a.status, FS_ERR_INVALID);
            continue;
        }
        if (atomicCAS(a.mark + i, -1, (int32_t)q) != -1) atomicExch(a.status, FS_ERR_INVALID);
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
__global__ void __launch_bounds__(kGatherThreads)
k_update_delta(UpdArgs a, int32_t chunk_w, int32_t n_chunks) {
    if (!upd_ok(a)) return;
    const int64_t n_tiles = (int64_t)a.n_idx * n_chunks;
    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const int32_t q = (int32_t)(tile / n_chunks);
        const int32_t chunk = (int32_t)(tile - (int64_t)q * n_chunks);
        const int32_t i = a.idx[q];
        const int64_t w0 = (int64_t)chunk * chunk_w, w1 = min(w0 + chunk_w, a.tw);
        for (int64_t w = w0 + threadIdx.x; w < w1; w += blockDim.x) {
            const uint4 nw = __ldg(a.d_new + (int64_t)q * a.tw + w);
            uint4 d = a.data[(int64_t)i * a.tw + w];
            xor4(d, nw);
            a.delta[(int64_t)q * a.tw + w] = d;
            a.data[(int64_t)i * a.tw + w] = nw;
        }
        if (chunk == 0)
            for (int32_t e = a.var_ptr[i] + threadIdx.x; e < a.var_ptr[i + 1]; e += blockDim.x)
                touch(a, a.var_idx[e], false);
    }
}

// CTA per changed check j: the coded rows containing parity b + j are listed.
__global__ void k_update_plist(UpdArgs a) {
    if (!upd_ok(a)) return;
    const int32_t np = *(volatile int32_t *)a.n_plist;
    for (int32_t k = blockIdx.x; k < np; k += gridDim.x) {
        const int32_t v = a.b + a.plist[k];
        for (int32_t e = a.var_ptr[v] + threadIdx.x; e < a.var_ptr[v + 1]; e += blockDim.x)
            touch(a, a.var_idx[e], true);
    }
}

// changed parity j ^= XOR of the deltas of its changed members; pdelta_j
// keeps that XOR. Tiles (listed check, chunk), chunk-major. Warp 0 first
// lists the changed members of the check (32 members per step, ballot).
__global__ void __launch_bounds__(kGatherThreads)
k_update_parity(UpdArgs a, int32_t chunk_w, int32_t n_chunks) {
    __shared__ int32_t s_q[kGatherThreads];
    __shared__ int s_nq, s_ok;
    if (threadIdx.x == 0) s_ok = upd_ok(a);  // one decision for the whole CTA
    __syncthreads();
    if (!s_ok) return;
    const int32_t np = *(volatile int32_t *)a.n_plist;
    const int64_t n_tiles = (int64_t)n_chunks * np;
    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const int32_t chunk = (int32_t)(tile / np);
        const int32_t j = a.plist[tile - (int64_t)chunk * np];
        const int32_t e0 = a.pre_ptr[j], e1 = a.pre_ptr[j + 1];
        const int64_t w0 = (int64_t)chunk * chunk_w, w1 = min(w0 + chunk_w, a.tw);
        if (threadIdx.x < 32) {
            int nq = 0;
            for (int32_t base = e0; base < e1; base += 32) {
                const int32_t e = base + (int32_t)threadIdx.x;
                const int32_t q = e < e1 ? a.mark[a.pre_idx[e]] : -1;
                const unsigned hit = __ballot_sync(0xffffffffu, q >= 0);
                const int pos = nq + __popc(hit & ((1u << threadIdx.x) - 1u));
                if (q >= 0 && pos < kGatherThreads) s_q[pos] = q;
                nq += __popc(hit);
            }
            if (threadIdx.x == 0) s_nq = nq;
        }
        __syncthreads();
        const int nq = s_nq;
        for (int64_t w = w0 + threadIdx.x; w < w1; w += blockDim.x) {
            uint4 acc = make_uint4(0, 0, 0, 0);
            if (nq <= kGatherThreads) {
                for (int k = 0; k < nq; ++k) xor4(acc, a.delta[(int64_t)s_q[k] * a.tw + w]);
            } else {  // more changed members than the list holds: scan the check
                for (int32_t e = e0; e < e1; ++e) {
                    const int32_t q = a.mark[a.pre_idx[e]];
                    if (q >= 0) xor4(acc, a.delta[(int64_t)q * a.tw + w]);
                }
            }
            a.pdelta[(int64_t)j * a.tw + w] = acc;
            uint4 p = a.parity[(int64_t)j * a.tw + w];
            xor4(p, acc);
            a.parity[(int64_t)j * a.tw + w] = p;
        }
        __syncthreads();
    }
}

// listed coded row g ^= XOR of the deltas of its changed neighbours (data
// blocks and parities). Tiles (listed row, chunk), chunk-major.
__global__ void __launch_bounds__(kGatherThreads)
k_update_coded(UpdArgs a, int32_t chunk_w, int32_t n_chunks) {
    if (!upd_ok(a)) return;
    const int32_t nc = *(volatile int32_t *)a.n_clist;
    const int64_t n_tiles = (int64_t)n_chunks * nc;
    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const int32_t chunk = (int32_t)(tile / nc);
        const int32_t g = a.clist[tile - (int64_t)chunk * nc];
        const int32_t e0 = a.con_ptr[g], e1 = a.con_ptr[g + 1];
        const int64_t w0 = (int64_t)chunk * chunk_w, w1 = min(w0 + chunk_w, a.tw);
        for (int64_t w = w0 + threadIdx.x; w < w1; w += blockDim.x) {
            uint4 acc = make_uint4(0, 0, 0, 0);
            for (int32_t e = e0; e < e1; ++e) {
                const int32_t v = a.con_idx[e];
                if (v < a.b) {
                    const int32_t q = a.mark[v];
                    if (q >= 0) xor4(acc, a.delta[(int64_t)q * a.tw + w]);
                } else if (a.pmark[v - a.b]) {
                    xor4(acc, a.pdelta[(int64_t)(v - a.b) * a.tw + w]);
                }
            }
            uint4 c = a.coded[(int64_t)g * a.tw + w];
            xor4(c, acc);
            a.coded[(int64_t)g * a.tw + w] = c;
        }
    }
}

inline void chunking(int64_t tw, int32_t *chunk_w, int32_t *n_chunks, int *threads) {
    const int64_t cw = tw < kGatherThreads ? tw : kGatherThreads;
    *chunk_w = (int32_t)cw;
    *n_chunks = (int32_t)((tw + cw - 1) / cw);
    int th = (int)((cw + 31) / 32 * 32);
    *threads = th < 32 ? 32 : th;
}

inline int grid_for(int64_t n_tiles, int num_sms, int ctas_per_sm = kCtasPerSm) {
    const int64_t cap = (int64_t)num_sms * ctas_per_sm;
    const int64_t g = n_tiles < cap ? n_tiles : cap;
    return (int)(g < 1 ? 1 : g);
}

}  // namespace

cudaError_t launch_gather(const GatherArgs &a, int num_sms, int ctas_per_sm, cudaStream_t s) {
    if (a.n_rows <= 0 || a.tw <= 0) return cudaSuccess;
    int32_t chunk_w, n_chunks;
    int threads;
    chunking(a.tw, &chunk_w, &n_chunks, &threads);
    k_gather_xor<<<grid_for((int64_t)n_chunks * a.n_rows, num_sms, ctas_per_sm), threads, 0, s>>>(a, chunk_w,
                                                                                   n_chunks);
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

    int64_t nb = c->b > c->m ? c->b : c->m;
    nb = nb > c->n ? nb : c->n;
    k_update_init<<<grid_for((nb + 255) / 256, c->num_sms), 256, 0, s>>>(a);
    if (n_idx > 0) {
        k_update_mark<<<grid_for((n_idx + 255) / 256, c->num_sms), 256, 0, s>>>(a);
        int32_t chunk_w, n_chunks;
        int threads;
        chunking(c->tw, &chunk_w, &n_chunks, &threads);
        k_update_delta<<<grid_for((int64_t)n_idx * n_chunks, c->num_sms), kGatherThreads, 0, s>>>(
            a, chunk_w, n_chunks);
        if (c->m > 0) {
            k_update_plist<<<grid_for(c->m, c->num_sms), 128, 0, s>>>(a);
            k_update_parity<<<grid_for((int64_t)n_chunks * c->m, c->num_sms), threads, 0, s>>>(
                a, chunk_w, n_chunks);
        }
        if (c->n > 0)
            k_update_coded<<<grid_for((int64_t)n_chunks * c->n, c->num_sms), threads, 0, s>>>(
                a, chunk_w, n_chunks);
    }
    return cudaGetLastError();
}
