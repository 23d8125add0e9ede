// fs_api.cu - the C ABI of libfounsure_gpu.so: code creation (host-side graph
// validation, joint constraint graph and its transpose), workspace sizing
// and the enqueue of each operation's kernels on the caller's stream.
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "fs_internal.cuh"


bool csr_ok(const fs_csr *g, int32_t n_rows_expect, int32_t n_cols_expect) {
    if (!g) return false;
    if (g->n_rows < 0 || g->n_cols < 0) return false;
    if (n_rows_expect >= 0 && g->n_rows != n_rows_expect) return false;
    if (n_cols_expect >= 0 && g->n_cols != n_cols_expect) return false;
    if (!g->row_ptr) return false;
    if (g->row_ptr[0] != 0) return false;
    for (int32_t r = 0; r < g->n_rows; ++r) {
        const int32_t e0 = g->row_ptr[r], e1 = g->row_ptr[r + 1];
        if (e1 < e0) return false;
        if (e1 > e0 && !g->col_idx) return false;
        for (int32_t e = e0; e < e1; ++e) {
            const int32_t v = g->col_idx[e];
            if (v < 0 || v >= g->n_cols) return false;
            if (e > e0 && v <= g->col_idx[e - 1]) return false;
        }
    }
    return true;
}

namespace {

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

template <typename T>
cudaError_t upload(T **dst, const std::vector<T> &src) {
    const size_t bytes = sizeof(T) * (src.empty() ? 1 : src.size());
    cudaError_t e = cudaMalloc((void **)dst, bytes);
    if (e != cudaSuccess) return e;
    if (src.empty()) return cudaMemset(*dst, 0, bytes);
    return cudaMemcpy(*dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice);
}

void free_code(fs_code *c) {
    if (!c) return;
    cudaFree(c->con_ptr);
    cudaFree(c->con_idx);
    cudaFree(c->con_xs);
    cudaFree(c->con_sum);
    cudaFree(c->pre_ptr);
    cudaFree(c->pre_idx);
    cudaFree(c->var_ptr);
    cudaFree(c->var_idx);
    cudaFree(c->con_ptr4);
    cudaFree(c->con_idx4);
    free_slice_tables(c);
    free(c->pre_level_off);
    free(c);
}

fs_status cuda_status(cudaError_t e) { return e == cudaSuccess ? FS_OK : FS_ERR_CUDA; }

inline cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

}  // namespace

FS_API const char *fs_status_string(fs_status s) {
    switch (s) {
        case FS_OK: return "FS_OK";
        case FS_STALL: return "FS_STALL: decode finished with unrecovered intermediates";
        case FS_ERR_INVALID: return "FS_ERR_INVALID: bad argument, graph, alignment or index";
        case FS_ERR_CUDA: return "FS_ERR_CUDA: a CUDA runtime call failed";
        case FS_ERR_NOMEM: return "FS_ERR_NOMEM: device allocation failed";
        case FS_ERR_TIMEOUT: return "FS_ERR_TIMEOUT: a bounded device wait gave up";
        case FS_ERR_SCRATCH:
            return "FS_ERR_SCRATCH: the code needs more scratch than fs_encode_static holds";
    }
    return "unknown fs_status";
}

FS_API fs_status fs_code_create(const fs_csr *precode, const fs_csr *lt, size_t block_bytes,
                                int flags, fs_code **out) {
    if (!out || !lt) return FS_ERR_INVALID;
    *out = nullptr;
    if (block_bytes == 0 || (block_bytes & 15) != 0) return FS_ERR_INVALID;
    if (flags != FS_DECODE_JOINT && flags != FS_DECODE_TWO_PASS) return FS_ERR_INVALID;
    const int32_t m = precode ? precode->n_rows : 0;
    // a precode over the intermediates (as many columns as the LT graph) is
    // chained: check j may hold earlier parities b + i, i < j
    const bool chained = precode && m > 0 && precode->n_cols == lt->n_cols;
    const int32_t b = precode ? (chained ? precode->n_cols - m : precode->n_cols) : lt->n_cols;
    if (precode && !csr_ok(precode, -1, -1)) return FS_ERR_INVALID;
    if (b < 1 || m < 0 || (int64_t)b + m > INT32_MAX / 2) return FS_ERR_INVALID;
    if (!csr_ok(lt, -1, b + m)) return FS_ERR_INVALID;
    // chained: each check's level is 1 + the deepest parity among its members;
    // the checks must come in level order (each level is then one row range)
    std::vector<int32_t> level_off;
    if (chained) {
        std::vector<int32_t> lvl(m, 0);
        for (int32_t j = 0; j < m; ++j) {
            for (int32_t e = precode->row_ptr[j]; e < precode->row_ptr[j + 1]; ++e) {
                const int32_t v = precode->col_idx[e];
                if (v >= b + j) return FS_ERR_INVALID;  // not an earlier intermediate
                if (v >= b) lvl[j] = std::max(lvl[j], lvl[v - b] + 1);
            }
            if (j > 0 && lvl[j] < lvl[j - 1]) return FS_ERR_INVALID;
            while ((int32_t)level_off.size() <= lvl[j]) level_off.push_back(j);
        }
        level_off.push_back(m);
    }
    const int32_t n = lt->n_rows;
    const int64_t e_lt = lt->row_ptr[n];
    const int64_t e_pre = precode ? precode->row_ptr[m] : 0;
    const int64_t e_con = e_lt + e_pre + m;
    if (e_con + 3 * ((int64_t)n + m) >= INT32_MAX || (int64_t)n + m >= INT32_MAX)
        return FS_ERR_INVALID;

    const int32_t k_int = b + m, n_con = n + m;
    // joint constraint graph: coded rows, then checks (members + own parity)
    std::vector<int32_t> con_ptr((size_t)n_con + 1), con_idx((size_t)e_con);
    int32_t max_con_deg = 0;
    for (int32_t g = 0; g <= n; ++g) con_ptr[g] = lt->row_ptr[g];
    if (e_lt) memcpy(con_idx.data(), lt->col_idx, sizeof(int32_t) * (size_t)e_lt);
    int64_t o = e_lt;
    for (int32_t j = 0; j < m; ++j) {
        for (int32_t e = precode->row_ptr[j]; e < precode->row_ptr[j + 1]; ++e)
            con_idx[o++] = precode->col_idx[e];
        con_idx[o++] = b + j;  // larger than every member: rows stay ascending
        con_ptr[n + j + 1] = (int32_t)o;
    }
    // per constraint: degree bound, and the XOR and the sum of its variable
    // indices (the symbolic peel keeps one of them over the still-unknown
    // variables, so a constraint with one unknown names it without a scan;
    // rows are strictly ascending, so no index is counted twice)
    std::vector<int32_t> con_xs((size_t)n_con, 0), con_sum((size_t)n_con, 0);
    for (int32_t g = 0; g < n_con; ++g) {
        max_con_deg = std::max(max_con_deg, con_ptr[g + 1] - con_ptr[g]);
        uint32_t sum = 0;
        for (int32_t e = con_ptr[g]; e < con_ptr[g + 1]; ++e) {
            con_xs[g] ^= con_idx[e];
            sum += (uint32_t)con_idx[e];
        }
        con_sum[g] = (int32_t)sum;
    }
    // transpose: constraints containing each intermediate, ascending
    std::vector<int32_t> var_ptr((size_t)k_int + 1, 0), var_idx((size_t)e_con);
    for (int64_t e = 0; e < e_con; ++e) var_ptr[con_idx[e] + 1]++;
    int32_t max_var_deg = 0;
    for (int32_t v = 0; v < k_int; ++v) {
        max_var_deg = std::max(max_var_deg, var_ptr[v + 1]);
        var_ptr[v + 1] += var_ptr[v];
    }
    {
        std::vector<int32_t> fill(var_ptr.begin(), var_ptr.end() - 1);
        for (int32_t g = 0; g < n_con; ++g)
            for (int32_t e = con_ptr[g]; e < con_ptr[g + 1]; ++e) var_idx[fill[con_idx[e]]++] = g;
    }
    // rows padded to a multiple of 4 entries with -1, each starting on a
    // 16-byte boundary, so the payload kernel stages a row with one bulk copy
    std::vector<int32_t> con_ptr4((size_t)n_con + 1, 0);
    for (int32_t g = 0; g < n_con; ++g)
        con_ptr4[g + 1] = con_ptr4[g] + ((con_ptr[g + 1] - con_ptr[g] + 3) & ~3);
    std::vector<int32_t> con_idx4((size_t)con_ptr4[n_con], -1);
    for (int32_t g = 0; g < n_con; ++g)
        for (int32_t e = con_ptr[g]; e < con_ptr[g + 1]; ++e)
            con_idx4[(size_t)con_ptr4[g] + (e - con_ptr[g])] = con_idx[e];
    std::vector<int32_t> pre_ptr((size_t)m + 1, 0), pre_idx((size_t)e_pre);
    for (int32_t j = 0; j <= m && precode; ++j) pre_ptr[j] = precode->row_ptr[j];
    if (e_pre) memcpy(pre_idx.data(), precode->col_idx, sizeof(int32_t) * (size_t)e_pre);

    fs_code *c = (fs_code *)calloc(1, sizeof(fs_code));
    if (!c) return FS_ERR_NOMEM;
    c->b = b;
    c->m = m;
    c->n = n;
    c->k_int = k_int;
    c->n_con = n_con;
    c->t = (int64_t)block_bytes;
    c->tw = (int64_t)(block_bytes / 16);
    c->flags = flags;
    c->e_lt = e_lt;
    c->e_pre = e_pre;
    c->e_con = e_con;
    c->max_con_deg = max_con_deg;
    c->chained = chained ? 1 : 0;
    c->n_pre_levels = chained ? (int32_t)level_off.size() - 1 : (m > 0 ? 1 : 0);
    c->pre_level_off = nullptr;
    if (chained) {
        c->pre_level_off = (int32_t *)malloc(sizeof(int32_t) * level_off.size());
        if (!c->pre_level_off) {
            free(c);
            return FS_ERR_NOMEM;
        }
        memcpy(c->pre_level_off, level_off.data(), sizeof(int32_t) * level_off.size());
    }
    c->max_var_deg = max_var_deg;
    c->e_con4 = (int64_t)con_ptr4[n_con];
    c->peel_ctas = 1;
    c->gather_ctas = 8;
    c->dpg_compact = 1;
    c->l2_hints = 0;
    c->encode_slices = 1;
    c->rows_per_ticket = 16;
    c->peel_columns = 0;
    c->peel_flow = 2;
    cudaError_t e = cudaGetDevice(&c->device);
    int v = 0;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, c->device);
    c->num_sms = v > 0 ? v : 1;
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device);
    c->smem_optin = (size_t)(v > 1024 ? v - 1024 : 0);
    if (e == cudaSuccess) e = upload(&c->con_ptr, con_ptr);
    if (e == cudaSuccess) e = upload(&c->con_idx, con_idx);
    if (e == cudaSuccess) e = upload(&c->con_xs, con_xs);
    if (e == cudaSuccess) e = upload(&c->con_sum, con_sum);
    if (e == cudaSuccess) e = upload(&c->pre_ptr, pre_ptr);
    if (e == cudaSuccess) e = upload(&c->pre_idx, pre_idx);
    if (e == cudaSuccess) e = upload(&c->var_ptr, var_ptr);
    if (e == cudaSuccess) e = upload(&c->var_idx, var_idx);
    if (e == cudaSuccess) e = upload(&c->con_ptr4, con_ptr4);
    if (e == cudaSuccess) e = upload(&c->con_idx4, con_idx4);
    if (e == cudaSuccess) e = build_slice_tables(c, con_ptr.data(), con_idx.data());
    if (e != cudaSuccess) {
        free_code(c);
        return e == cudaErrorMemoryAllocation ? FS_ERR_NOMEM : FS_ERR_CUDA;
    }
    *out = c;
    return FS_OK;
}

FS_API void fs_code_destroy(fs_code *code) {
    if (!code) return;
    cudaDeviceSynchronize();
    free_code(code);
}

FS_API fs_status fs_code_info(const fs_code *c, int32_t *b, int32_t *m, int32_t *n,
                              size_t *block_bytes) {
    if (!c) return FS_ERR_INVALID;
    if (b) *b = c->b;
    if (m) *m = c->m;
    if (n) *n = c->n;
    if (block_bytes) *block_bytes = (size_t)c->t;
    return FS_OK;
}

FS_API fs_status fs_code_set_tuning(fs_code *c, int knob, int value) {
    if (!c) return FS_ERR_INVALID;
    switch (knob) {
        case FS_TUNE_PEEL_CTAS:
            if (value < 1 || value > 8) return FS_ERR_INVALID;
            c->peel_ctas = value;
            return FS_OK;
        case FS_TUNE_DPG_COMPACT:
            if (value != 0 && value != 1) return FS_ERR_INVALID;
            c->dpg_compact = value;
            return FS_OK;
        case FS_TUNE_ROWS_PER_TICKET:
            if (value < 1 || value > 16) return FS_ERR_INVALID;
            c->rows_per_ticket = value;
            return FS_OK;
        case FS_TUNE_ENCODE_SLICES:
            if (value < 0 || value > 3) return FS_ERR_INVALID;
            c->encode_slices = value;
            return FS_OK;
        case FS_TUNE_L2_HINTS:
            if (value != 0 && value != 1) return FS_ERR_INVALID;
            c->l2_hints = value;
            return FS_OK;
        case FS_TUNE_GATHER_CTAS:
            if (value < 1 || value > 16) return FS_ERR_INVALID;
            c->gather_ctas = value;
            return FS_OK;
        case FS_TUNE_PEEL_COLUMNS:
            if (value != 0 && value != 1) return FS_ERR_INVALID;
            c->peel_columns = value;
            return FS_OK;
        case FS_TUNE_PEEL_FLOW:
            if (value < 0 || value > 3) return FS_ERR_INVALID;
            c->peel_flow = value;
            return FS_OK;
    }
    return FS_ERR_INVALID;
}

FS_API size_t fs_workspace_bytes(const fs_code *c, int op, int32_t n_items) {
    if (!c) return 0;
    switch (op) {
        case FS_OP_ENCODE: return encode_ws_bytes(c);
        case FS_OP_REPAIR: return WS_HDR_BYTES;
        case FS_OP_DECODE: return decode_layout(c).total;
        case FS_OP_UPDATE: return update_layout(c, n_items < 0 ? 0 : n_items).total;
    }
    return 0;
}

namespace {

GatherArgs lt_args(const fs_code *c, const void *d_data, const void *d_parity, void *d_coded,
                   void *d_ws) {
    GatherArgs a;
    a.ptr = c->con_ptr;
    a.idx = c->con_idx;
    a.rows = nullptr;
    a.n_rows = c->n;
    a.row_base = 0;
    a.n_valid = c->n;
    a.inA = static_cast<const uint4 *>(d_data);
    a.inB = static_cast<const uint4 *>(d_parity);
    a.split = c->b;
    a.out = static_cast<uint4 *>(d_coded);
    a.tw = c->tw;
    a.status = static_cast<int32_t *>(d_ws) + WS_STATUS;
    return a;
}

}  // namespace

FS_API fs_status fs_encode(const fs_code *c, const void *d_data, void *d_parity, void *d_coded,
                           void *d_ws, void *stream) {
    if (!c || !d_data || !d_coded || !d_ws) return FS_ERR_INVALID;
    if ((c->m > 0) != (d_parity != nullptr)) return FS_ERR_INVALID;
    if (!aligned16(d_data) || !aligned16(d_parity) || !aligned16(d_coded) || !aligned16(d_ws))
        return FS_ERR_INVALID;
    return cuda_status(launch_encode(c, d_data, d_parity, d_coded, static_cast<uint8_t *>(d_ws),
                                     as_stream(stream)));
}

FS_API fs_status fs_encode_rows(const fs_code *c, int32_t row_begin, int32_t row_end,
                                const void *d_data, const void *d_parity, void *d_coded,
                                void *d_ws, void *stream) {
    if (!c || !d_data || !d_coded || !d_ws) return FS_ERR_INVALID;
    if (row_begin < 0 || row_end < row_begin || row_end > c->n) return FS_ERR_INVALID;
    if ((c->m > 0) != (d_parity != nullptr)) return FS_ERR_INVALID;
    if (!aligned16(d_data) || !aligned16(d_parity) || !aligned16(d_coded) || !aligned16(d_ws))
        return FS_ERR_INVALID;
    cudaStream_t s = as_stream(stream);
    cudaError_t e = cudaMemsetAsync(d_ws, 0, sizeof(int32_t), s);  // the status word
    GatherArgs a = lt_args(c, d_data, d_parity, d_coded, d_ws);
    a.row_base = row_begin;
    a.n_rows = row_end - row_begin;
    if (e == cudaSuccess) e = launch_gather(a, c->num_sms, c->gather_ctas, s);
    return cuda_status(e);
}

FS_API fs_status fs_decode_schedule(const fs_code *c, const uint8_t *d_erased,
                                    uint8_t *d_unrecovered, int32_t *d_n_unrecovered, void *d_ws,
                                    void *stream) {
    if (!c || !d_unrecovered || !d_n_unrecovered || !d_ws) return FS_ERR_INVALID;
    if (c->n > 0 && !d_erased) return FS_ERR_INVALID;
    if (!aligned16(d_ws)) return FS_ERR_INVALID;
    return cuda_status(launch_dpg(c, d_erased, static_cast<uint8_t *>(d_ws), d_unrecovered,
                                  d_n_unrecovered, as_stream(stream)));
}

FS_API fs_status fs_decode_payload(const fs_code *c, const void *d_coded, void *d_data_out,
                                   void *d_ws, void *stream) {
    if (!c || !d_data_out || !d_ws) return FS_ERR_INVALID;
    if (c->n > 0 && !d_coded) return FS_ERR_INVALID;
    if (!aligned16(d_coded) || !aligned16(d_data_out) || !aligned16(d_ws)) return FS_ERR_INVALID;
    return cuda_status(launch_peel(c, static_cast<const uint4 *>(d_coded),
                                   static_cast<uint4 *>(d_data_out), static_cast<uint8_t *>(d_ws),
                                   as_stream(stream)));
}

FS_API fs_status fs_decode(const fs_code *c, const void *d_coded, const uint8_t *d_erased,
                           void *d_data_out, uint8_t *d_unrecovered, int32_t *d_n_unrecovered,
                           void *d_ws, void *stream) {
    if (!c || !d_data_out) return FS_ERR_INVALID;
    if (c->n > 0 && !d_coded) return FS_ERR_INVALID;
    if (!aligned16(d_coded) || !aligned16(d_data_out)) return FS_ERR_INVALID;
    fs_status st = fs_decode_schedule(c, d_erased, d_unrecovered, d_n_unrecovered, d_ws, stream);
    if (st == FS_OK) st = fs_decode_payload(c, d_coded, d_data_out, d_ws, stream);
    return st;
}

FS_API fs_status fs_decode_path(const fs_code *c, const void *d_ws, fs_path_view *out) {
    if (!c || !d_ws || !out) return FS_ERR_INVALID;
    const DecodeLayout L = decode_layout(c);
    const uint8_t *w = static_cast<const uint8_t *>(d_ws);
    out->n_levels = reinterpret_cast<const int32_t *>(w) + WS_N_LEVELS;
    out->n_pairs = reinterpret_cast<const int32_t *>(w) + WS_N_PAIRS;
    out->level_off = reinterpret_cast<const int32_t *>(w + L.level_off);
    out->pair_f = reinterpret_cast<const int32_t *>(w + L.pair_f);
    out->pair_g = reinterpret_cast<const int32_t *>(w + L.pair_g);
    out->parity = w + L.parity;
    out->plan = reinterpret_cast<const int32_t *>(w + L.flow_hdr);
    return FS_OK;
}

FS_API fs_status fs_update(const fs_code *c, const int32_t *d_idx, int32_t n_idx,
                           const void *d_new, void *d_data, void *d_parity, void *d_coded,
                           void *d_ws, void *stream) {
    if (!c || n_idx < 0 || !d_data || !d_coded || !d_ws) return FS_ERR_INVALID;
    if (n_idx > 0 && (!d_idx || !d_new)) return FS_ERR_INVALID;
    if ((c->m > 0) != (d_parity != nullptr)) return FS_ERR_INVALID;
    if (!aligned16(d_new) || !aligned16(d_data) || !aligned16(d_parity) || !aligned16(d_coded) ||
        !aligned16(d_ws))
        return FS_ERR_INVALID;
    cudaError_t e = launch_update(c, d_idx, n_idx, static_cast<const uint4 *>(d_new),
                                  static_cast<uint4 *>(d_data), static_cast<uint4 *>(d_parity),
                                  static_cast<uint4 *>(d_coded), static_cast<uint8_t *>(d_ws),
                                  as_stream(stream));
    return cuda_status(e);
}

FS_API fs_status fs_repair(const fs_code *c, const int32_t *d_lost, int32_t n_lost,
                           const void *d_data, const void *d_parity, void *d_coded, void *d_ws,
                           void *stream) {
    if (!c || n_lost < 0 || !d_data || !d_coded || !d_ws) return FS_ERR_INVALID;
    if (n_lost > 0 && !d_lost) return FS_ERR_INVALID;
    if ((c->m > 0) != (d_parity != nullptr)) return FS_ERR_INVALID;
    if (!aligned16(d_data) || !aligned16(d_parity) || !aligned16(d_coded) || !aligned16(d_ws))
        return FS_ERR_INVALID;
    cudaStream_t s = as_stream(stream);
    cudaError_t e = cudaMemsetAsync(d_ws, 0, sizeof(int32_t), s);
    GatherArgs a = lt_args(c, d_data, d_parity, d_coded, d_ws);
    a.rows = d_lost;
    a.n_rows = n_lost;
    if (e == cudaSuccess) e = launch_gather(a, c->num_sms, c->gather_ctas, s);
    return cuda_status(e);
}
