// fs_peel.cu - peeling decode split into a symbolic pass and a payload pass.
//
// k_dpg: Decoding Path Generation (Algorithm 5, Section 3.2) on one CTA.
//   The state of the peel (residual unknown count per constraint, known flag
//   per intermediate, best decoder per intermediate, frontier lists) lives in
//   shared memory when it fits, else in the workspace. A level is:
//     A. every frontier constraint g (residual count 1 at the level start)
//        finds its one unknown f and bids key = (degree(g) << 32 | g) with an
//        atomicMin on best[f]: the lowest original degree wins, ties go to
//        the lowest constraint index (Section 3.1, second rule);
//     B. each f with a bid becomes a pair (f, g) of the path and is marked
//        known; its recipe (the neighbours of g other than f) is written
//        behind a block-wide prefix sum;
//     C. every constraint containing a newly known f is decremented; one
//        whose count goes 2 -> 1 joins the next frontier.
//   Known flags only change in B, after A has read them, so a level uses
//   only symbols decoded in earlier levels (Section 3.1, first rule).
//
// k_peel: the payload. Each CTA owns one byte slice of every block and walks
//   all levels; pairs of a level are independent (no intermediate is written
//   twice and none is read in the level that writes it), so one
//   __syncthreads between levels is the only ordering needed and no grid-wide
//   synchronisation or per-level launch is required.
#include "fs_internal.cuh"

namespace {

constexpr int kDpgThreads = 1024;
constexpr int kPeelThreads = 256;
constexpr unsigned long long kEmpty = ~0ull;

struct DpgArgs {
    const int32_t *con_ptr, *con_idx, *var_ptr, *var_idx;
    const uint8_t *erased;
    int32_t b, n, k_int, n_con;
    int two_pass;
    int use_smem;
    // workspace arrays (used directly when the state does not fit in smem)
    int32_t *res;
    unsigned long long *best;
    uint8_t *known;
    int32_t *front_a, *front_b, *touched;
    // outputs
    int32_t *pair_f, *pair_g, *level_off, *recipe_off, *recipe_h, *unrec_list, *hdr;
    uint8_t *unrecovered;
    int32_t *n_unrecovered;
};

// stage: -1 joint (every surviving coded row and every check), 0 coded rows
// only, 1 checks only (two-pass mode, Section 2.2)
__device__ __forceinline__ bool usable(const DpgArgs &a, int32_t g, int stage) {
    if (g < a.n) return stage <= 0 && a.erased[g] == 0;
    return stage != 0;
}

// Block-wide exclusive prefix sum of x; *total receives the sum. All threads
// of the block must call it.
__device__ int block_excl_scan(int x, int *total, int *s_warp) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    int v = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    if (lane == 31) s_warp[wid] = v;
    __syncthreads();
    if (wid == 0) {
        int s = lane < nw ? s_warp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        s_warp[lane] = s;  // inclusive warp totals
    }
    __syncthreads();
    const int before = wid > 0 ? s_warp[wid - 1] : 0;
    *total = s_warp[nw - 1];
    __syncthreads();
    return before + v - x;
}

__global__ void __launch_bounds__(kDpgThreads, 1) k_dpg(DpgArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_warp[32];
    __shared__ int s_nf, s_nt, s_nnext, s_cnt, s_cnt_data;

    const int tid = threadIdx.x, T = blockDim.x;
    const int32_t K = a.k_int, G = a.n_con;

    int32_t *res = a.res;
    unsigned long long *best = a.best;
    uint8_t *known = a.known;
    int32_t *front = a.front_a, *next = a.front_b, *touched = a.touched;
    if (a.use_smem) {
        unsigned char *p = smem;
        best = reinterpret_cast<unsigned long long *>(p);
        p += 8 * (size_t)(K + 1);
        res = reinterpret_cast<int32_t *>(p);
        p += 4 * (size_t)(G + 1);
        front = reinterpret_cast<int32_t *>(p);
        p += 4 * (size_t)(G + 1);
        next = reinterpret_cast<int32_t *>(p);
        p += 4 * (size_t)(G + 1);
        touched = reinterpret_cast<int32_t *>(p);
        p += 4 * (size_t)(K + 1);
        known = p;
    }

    if (tid == 0) a.hdr[WS_STATUS] = FS_OK;
    for (int32_t v = tid; v < K; v += T) {
        known[v] = 0;
        best[v] = kEmpty;
    }
    for (int32_t g = tid; g < G; g += T) res[g] = __ldg(a.con_ptr + g + 1) - __ldg(a.con_ptr + g);
    int stage = a.two_pass ? 0 : -1;
    if (tid == 0) s_nf = 0;
    __syncthreads();
    for (int32_t g = tid; g < G; g += T)
        if (usable(a, g, stage) && res[g] == 1) front[atomicAdd(&s_nf, 1)] = g;
    __syncthreads();

    int32_t np = 0, level = 0, rb = 0;
    for (;;) {
        int nf = s_nf;
        if (nf == 0) {
            if (stage != 0) break;
            // two-pass: coded rows are exhausted; peel the precode checks
            stage = 1;
            __syncthreads();
            for (int32_t g = a.n + tid; g < G; g += T)
                if (res[g] == 1) front[atomicAdd(&s_nf, 1)] = g;
            __syncthreads();
            nf = s_nf;
            if (nf == 0) break;
        }
        if (tid == 0) {
            s_nt = 0;
            s_nnext = 0;
        }
        __syncthreads();
        // A: frontier constraints bid for their single unknown
        for (int i = tid; i < nf; i += T) {
            const int32_t g = front[i];
            if (res[g] != 1) continue;
            const int32_t e0 = __ldg(a.con_ptr + g), e1 = __ldg(a.con_ptr + g + 1);
            int32_t f = -1;
            for (int32_t e = e0; e < e1; ++e) {
                const int32_t v = __ldg(a.con_idx + e);
                if (!known[v]) {
                    f = v;
                    break;
                }
            }
            if (f < 0) continue;  // unreachable while res[g] == 1
            const unsigned long long key = ((unsigned long long)(e1 - e0) << 32) | (uint32_t)g;
            if (atomicMin(best + f, key) == kEmpty) touched[atomicAdd(&s_nt, 1)] = f;
        }
        __syncthreads();
        const int nt = s_nt;
        if (tid == 0) a.level_off[level] = np;
        // B: pairs, recipes, known flags
        for (int base = 0; base < nt; base += T) {
            const int i = base + tid;
            int32_t f = -1, g = -1, sz = 0;
            if (i < nt) {
                f = touched[i];
                const unsigned long long key = best[f];
                g = (int32_t)(key & 0xffffffffull);
                sz = (int32_t)(key >> 32) - 1;
                best[f] = kEmpty;
                known[f] = 1;
                a.pair_f[np + i] = f;
                a.pair_g[np + i] = g;
            }
            int total;
            const int off = block_excl_scan(sz, &total, s_warp);
            if (i < nt) {
                int32_t o = rb + off;
                a.recipe_off[np + i] = o;
                const int32_t e0 = __ldg(a.con_ptr + g), e1 = __ldg(a.con_ptr + g + 1);
                for (int32_t e = e0; e < e1; ++e) {
                    const int32_t h = __ldg(a.con_idx + e);
                    if (h != f) a.recipe_h[o++] = h;
                }
            }
            rb += total;
        }
        __syncthreads();
        // C: decrement every constraint that contains a newly known symbol
        for (int i = tid; i < nt; i += T) {
            const int32_t f = touched[i];
            const int32_t e0 = __ldg(a.var_ptr + f), e1 = __ldg(a.var_ptr + f + 1);
            for (int32_t e = e0; e < e1; ++e) {
                const int32_t c = __ldg(a.var_idx + e);
                if (atomicSub(res + c, 1) == 2 && usable(a, c, stage))
                    next[atomicAdd(&s_nnext, 1)] = c;
            }
        }
        __syncthreads();
        int32_t *tmp = front;
        front = next;
        next = tmp;
        if (tid == 0) s_nf = s_nnext;
        np += nt;
        ++level;
        __syncthreads();
    }
    if (tid == 0) {
        a.level_off[level] = np;
        a.recipe_off[np] = rb;
        a.hdr[WS_N_LEVELS] = level;
        a.hdr[WS_N_PAIRS] = np;
        s_cnt = 0;
        s_cnt_data = 0;
    }
    __syncthreads();
    for (int32_t v = tid; v < K; v += T) {
        const uint8_t u = known[v] ? 0 : 1;
        a.unrecovered[v] = u;
        if (u) {
            atomicAdd(&s_cnt, 1);
            if (v < a.b) a.unrec_list[atomicAdd(&s_cnt_data, 1)] = v;
        }
    }
    __syncthreads();
    if (tid == 0) {
        *a.n_unrecovered = s_cnt;
        a.hdr[WS_N_UNREC_DATA] = s_cnt_data;
    }
}

struct PeelArgs {
    const uint4 *coded;
    uint4 *data;    // intermediates v < b
    uint4 *parity;  // intermediates v >= b (workspace)
    const int32_t *pair_f, *pair_g, *level_off, *recipe_off, *recipe_h, *unrec_list, *hdr;
    int32_t b, n;
    int64_t tw;
    int32_t slice_w;
};

__device__ __forceinline__ void xor4(uint4 &a, const uint4 &b) {
    a.x ^= b.x;
    a.y ^= b.y;
    a.z ^= b.z;
    a.w ^= b.w;
}

__global__ void __launch_bounds__(kPeelThreads) k_peel(PeelArgs a) {
    const int64_t w0 = (int64_t)blockIdx.x * a.slice_w;
    const int32_t lanes = (int32_t)min((int64_t)a.slice_w, a.tw - w0);
    const int32_t n_levels = a.hdr[WS_N_LEVELS];
    for (int32_t l = 0; l < n_levels; ++l) {
        const int32_t p0 = a.level_off[l], p1 = a.level_off[l + 1];
        const int32_t items = (p1 - p0) * lanes;
        for (int32_t it = threadIdx.x; it < items; it += blockDim.x) {
            const int32_t q = it / lanes;
            const int64_t w = w0 + (it - q * lanes);
            const int32_t p = p0 + q;
            const int32_t f = a.pair_f[p], g = a.pair_g[p];
            uint4 acc = make_uint4(0, 0, 0, 0);
            if (g < a.n) acc = __ldg(a.coded + (int64_t)g * a.tw + w);
            const int32_t r1 = a.recipe_off[p + 1];
            for (int32_t r = a.recipe_off[p]; r < r1; ++r) {
                const int32_t h = a.recipe_h[r];
                const uint4 *x = (h < a.b) ? a.data + (int64_t)h * a.tw
                                           : a.parity + (int64_t)(h - a.b) * a.tw;
                xor4(acc, x[w]);  // coherent load: written by this CTA in an earlier level
            }
            uint4 *y = (f < a.b) ? a.data + (int64_t)f * a.tw : a.parity + (int64_t)(f - a.b) * a.tw;
            y[w] = acc;
        }
        __syncthreads();
    }
    // unrecovered data blocks read as zero
    const int32_t nu = a.hdr[WS_N_UNREC_DATA];
    for (int32_t it = threadIdx.x; it < nu * lanes; it += blockDim.x) {
        const int32_t q = it / lanes;
        a.data[(int64_t)a.unrec_list[q] * a.tw + w0 + (it - q * lanes)] = make_uint4(0, 0, 0, 0);
    }
}

}  // namespace

size_t dpg_smem_bytes(const fs_code *c) {
    return 8 * (size_t)(c->k_int + 1) + 4 * 3 * (size_t)(c->n_con + 1) +
           4 * (size_t)(c->k_int + 1) + (size_t)(c->k_int + 1) + 64;
}

cudaError_t launch_dpg(const fs_code *c, const uint8_t *erased, uint8_t *ws, uint8_t *unrecovered,
                       int32_t *n_unrecovered, cudaStream_t s) {
    const DecodeLayout L = decode_layout(c);
    DpgArgs a;
    a.con_ptr = c->con_ptr;
    a.con_idx = c->con_idx;
    a.var_ptr = c->var_ptr;
    a.var_idx = c->var_idx;
    a.erased = erased;
    a.b = c->b;
    a.n = c->n;
    a.k_int = c->k_int;
    a.n_con = c->n_con;
    a.two_pass = (c->flags & FS_DECODE_TWO_PASS) ? 1 : 0;
    a.res = reinterpret_cast<int32_t *>(ws + L.res);
    a.best = reinterpret_cast<unsigned long long *>(ws + L.best);
    a.known = ws + L.known;
    a.front_a = reinterpret_cast<int32_t *>(ws + L.front_a);
    a.front_b = reinterpret_cast<int32_t *>(ws + L.front_b);
    a.touched = reinterpret_cast<int32_t *>(ws + L.touched);
    a.pair_f = reinterpret_cast<int32_t *>(ws + L.pair_f);
    a.pair_g = reinterpret_cast<int32_t *>(ws + L.pair_g);
    a.level_off = reinterpret_cast<int32_t *>(ws + L.level_off);
    a.recipe_off = reinterpret_cast<int32_t *>(ws + L.recipe_off);
    a.recipe_h = reinterpret_cast<int32_t *>(ws + L.recipe_h);
    a.unrec_list = reinterpret_cast<int32_t *>(ws + L.unrec_list);
    a.hdr = reinterpret_cast<int32_t *>(ws);
    a.unrecovered = unrecovered;
    a.n_unrecovered = n_unrecovered;
    const size_t smem = dpg_smem_bytes(c);
    a.use_smem = smem <= c->smem_optin ? 1 : 0;
    const size_t dyn = a.use_smem ? smem : 0;
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
    a.recipe_off = reinterpret_cast<const int32_t *>(ws + L.recipe_off);
    a.recipe_h = reinterpret_cast<const int32_t *>(ws + L.recipe_h);
    a.unrec_list = reinterpret_cast<const int32_t *>(ws + L.unrec_list);
    a.hdr = reinterpret_cast<const int32_t *>(ws);
    a.b = c->b;
    a.n = c->n;
    a.tw = c->tw;
    // about two slices per SM, each at least 16 words (256 bytes) wide
    int64_t sw = c->tw / (2 * (int64_t)c->num_sms);
    sw = sw < 16 ? 16 : sw;
    if (sw > c->tw) sw = c->tw;
    a.slice_w = (int32_t)sw;
    const int64_t n_slices = (c->tw + sw - 1) / sw;
    k_peel<<<(unsigned)n_slices, kPeelThreads, 0, s>>>(a);
    return cudaGetLastError();
}
