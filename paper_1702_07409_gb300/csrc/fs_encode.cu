// fs_encode.cu - encoding (Section 2.2, steps (1) precode and (2) LDGM) in
// two launches of one kernel, k_rows: first the m precode rows (parities,
// over the data blocks), then the n LT rows (coded blocks, over the data
// blocks and parities). Stream order makes every parity final before an LT
// row reads it.
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
#include "fs_internal.cuh"

namespace {

constexpr int kEncThreads = 256;
constexpr int kEncV = 2;                      // words per thread per chunk
constexpr int kChunkW = kEncV * kEncThreads;  // 16-byte words per chunk (8 KiB)
constexpr int kRows = 16;                     // rows per ticket
constexpr int kStage = 2048;                  // neighbour entries of one ticket staged
constexpr int kCtasPerSm = 3;

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
    int32_t *ticket_ctr;  // workspace counter, zero at launch
};

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

__device__ __forceinline__ void store_row(const RowArgs &a, int32_t row, int64_t w0, int64_t w1,
                                          const uint4 *acc) {
    uint4 *out = a.out + (int64_t)row * a.tw;
#pragma unroll
    for (int v = 0; v < kEncV; ++v) {
        const int64_t w = w0 + threadIdx.x + (int64_t)v * kEncThreads;
        if (w >= w1) continue;
        if (a.stream_out) __stcs(out + w, acc[v]);
        else __stcg(out + w, acc[v]);
    }
}

__global__ void __launch_bounds__(kEncThreads, kCtasPerSm) k_rows(RowArgs a) {
    // ring of 3 pointer stages (two tickets ahead), 2 neighbour stages, 4 tickets
    __shared__ int32_t s_ptr[3][kRows + 1];
    __shared__ int32_t s_idx[2][kStage];
    __shared__ int32_t s_tk[4];
    const int32_t batches = (a.n_rows + a.rows - 1) / a.rows;
    const int32_t n_tickets = a.n_chunks * batches;

    auto stage_ptr = [&](int32_t t, int slot) {
        if (t >= n_tickets) return;
        const Ticket k = ticket_of(a, t, batches);
        for (int i = threadIdx.x; i <= k.nr; i += blockDim.x)
            cp_async4(&s_ptr[slot][i], a.ptr + k.r0 + i);
    };
    auto stage_idx = [&](int32_t t, int pslot, int islot) {
        if (t >= n_tickets) return;
        const int32_t e0 = s_ptr[pslot][0];
        const int32_t ne = s_ptr[pslot][ticket_of(a, t, batches).nr] - e0;
        if (ne > kStage) return;  // read straight from global memory instead
        for (int i = threadIdx.x; i < ne; i += blockDim.x)
            cp_async4(&s_idx[islot][i], a.idx + e0 + i);
    };

    // prologue: tickets 0..2 of this CTA, pointers of 0 and 1, list of 0
    if (threadIdx.x < 3) s_tk[threadIdx.x] = atomicAdd(a.ticket_ctr, 1);
    __syncthreads();
    stage_ptr(s_tk[0], 0);
    cp_async_commit();
    stage_ptr(s_tk[1], 1);
    cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();
    stage_idx(s_tk[0], 0, 0);
    cp_async_commit();
    for (int it = 0;; ++it) {
        // ticket it's list and ticket it+1's pointers are in
        cp_async_wait<0>();
        __syncthreads();
        const int32_t t = s_tk[it & 3];
        if (t >= n_tickets) break;  // tickets are taken in order: no later one is ours
        const int ps = it % 3, is = it & 1;
        if (threadIdx.x == 0) s_tk[(it + 3) & 3] = atomicAdd(a.ticket_ctr, 1);
        stage_ptr(s_tk[(it + 2) & 3], (it + 2) % 3);
        stage_idx(s_tk[(it + 1) & 3], (it + 1) % 3, (it + 1) & 1);
        cp_async_commit();

        const Ticket k = ticket_of(a, t, batches);
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
                    x[j][q] = (on && ok[q]) ? __ldg(src + w[q]) : make_uint4(0, 0, 0, 0);
            }
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                if (e + j >= e_end) break;
                while (e + j >= rp[r + 1]) {  // row r is complete (rows may be empty)
                    store_row(a, k.r0 + r, w0, w1, acc);
#pragma unroll
                    for (int v = 0; v < kEncV; ++v) acc[v] = make_uint4(0, 0, 0, 0);
                    ++r;
                }
#pragma unroll
                for (int q = 0; q < kEncV; ++q) xor4(acc[q], x[j][q]);
            }
        }
        for (; r < k.nr; ++r) {  // the last row with entries, then empty rows
            store_row(a, k.r0 + r, w0, w1, acc);
#pragma unroll
            for (int v = 0; v < kEncV; ++v) acc[v] = make_uint4(0, 0, 0, 0);
        }
    }
    cp_async_wait<0>();
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

cudaError_t launch_encode(const fs_code *c, const void *data, void *parity, void *coded, uint8_t *ws,
                          cudaStream_t s) {
    int32_t *hdr = reinterpret_cast<int32_t *>(ws);
    // status (nothing here can fail on the device) and both ticket counters
    cudaError_t e = cudaMemsetAsync(ws, 0, WS_HDR_BYTES, s);
    if (e != cudaSuccess) return e;
    const int32_t n_chunks = encode_chunks(c);
    const int ctas = c->gather_ctas < kCtasPerSm ? c->gather_ctas : kCtasPerSm;
    RowArgs a;
    a.tw = c->tw;
    a.n_chunks = n_chunks;
    if (c->m > 0) {  // step (1): parities over the data blocks
        a.ptr = c->pre_ptr;
        a.idx = c->pre_idx;
        a.inA = static_cast<const uint4 *>(data);
        a.inB = nullptr;
        a.split = c->b;
        a.out = static_cast<uint4 *>(parity);
        a.n_rows = c->m;
        a.stream_out = 0;
        a.rows = 1;  // check rows are long: one per ticket keeps every SM busy
        a.ticket_ctr = hdr + WS_COUNT_A;
        const int64_t tickets = (int64_t)n_chunks * c->m;
        k_rows<<<grid_for(tickets, c->num_sms, ctas), kEncThreads, 0, s>>>(a);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
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
        a.rows = kRows;
        a.ticket_ctr = hdr + WS_COUNT_B;
        const int64_t tickets = (int64_t)n_chunks * ((c->n + kRows - 1) / kRows);
        k_rows<<<grid_for(tickets, c->num_sms, ctas), kEncThreads, 0, s>>>(a);
        e = cudaGetLastError();
    }
    return e;
}
