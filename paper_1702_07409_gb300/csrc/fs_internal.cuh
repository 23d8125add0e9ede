// fs_internal.cuh - internal definitions shared by the translation units of
// libfounsure_gpu.so (code object, workspace layout, kernel launchers).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "founsure_gpu.h"

#define FS_API extern "C" __attribute__((visibility("default")))

// Joint constraint graph of a code (Algorithm 5 over coded rows and precode
// checks): constraint g < n is coded row g with payload c_g; constraint
// n + j is precode check j with payload zero and vars = members + {b + j}.
// The LT graph is the prefix con_ptr[0..n], con_idx[0..e_lt).
// Tables of one part of a code's slice encode (see fs_code::sl_part): one
// device array the kernel copies to shared memory, each piece 16-byte aligned:
//   grp   int2 [n_grp]       {first entry, columns of the group}
//   row   uint16 [32 n_grp]  output row of each lane (parity index or coded
//                            row), 0xFFFF pad
//   idx   uint16 [...]       group entries, column-major (32 lanes)
// The first n_grp_p groups are precode (parity) rows, groups up to n_grp_a
// coded rows that read no parity, the rest coded rows that read one.
constexpr int kSliceParts = 4;
constexpr int kSliceXPhases = 7;  // further precode levels a slice encode takes (chained)
struct SlicePart {
    unsigned char *tab = nullptr;
    int32_t tab_bytes = 0;  // multiple of 16
    int32_t n_grp = 0, n_grp_p = 0, n_grp_a = 0;
    int32_t off_row = 0, off_idx = 0;  // byte offsets
    // chained precode: the parity pieces of levels 1, 2, ... are the groups
    // [n_grp_a, xphase_end[0]), [xphase_end[0], xphase_end[1]), ...
    int32_t n_xphase = 0;
    int32_t xphase_end[kSliceXPhases] = {};
};

struct fs_code {
    int32_t b, m, n, k_int, n_con;
    int64_t t;            // block bytes
    int64_t tw;           // block size in 16-byte words
    int flags;
    int64_t e_lt, e_pre, e_con;
    int chained;          // 1: precode members are intermediates (check j's below b + j)
    int32_t n_pre_levels; // chained: levels of parities (level = 1 + deepest parity member)
    int32_t *pre_level_off;  // chained, host: first check of each level (rows in level order)
    int32_t max_con_deg;  // largest constraint degree
    int32_t max_var_deg;  // largest number of constraints containing one var
    // device arrays
    int32_t *con_ptr;     // [n_con + 1]
    int32_t *con_idx;     // [e_con]
    int32_t *con_xs;      // [n_con] XOR of the variable indices of each constraint
    int32_t *con_sum;     // [n_con] sum of the variable indices of each constraint (mod 2^32)
    int32_t *con_ptr4;    // [n_con + 1] row starts of con_idx4 (multiples of 4)
    int32_t *con_idx4;    // rows of the joint graph padded to 16 bytes with -1
    int64_t e_con4;       // entries of con_idx4
    int32_t *pre_ptr;     // [m + 1]   precode rows (members only)
    int32_t *pre_idx;     // [e_pre]
    int32_t *var_ptr;     // [k_int + 1] transpose of the joint graph
    int32_t *var_idx;     // [e_con]
    int device;
    int num_sms;
    size_t smem_optin;    // max dynamic shared memory per block
    // tuning knobs (fs_code_set_tuning); they never change results
    int peel_ctas;        // payload-peel CTAs per SM (slice width follows)
    int gather_ctas;      // resident CTAs per SM for the gather kernels
    int dpg_compact;      // 1: symbolic peel in the compact shared-memory form when it fits
    int l2_hints;         // 1: L2 evict-last / evict-first hints on the gathers
    int encode_slices;    // 1: shared-memory slice encode when the code fits
    int rows_per_ticket;  // coded rows per work ticket of the row-gather encode (1..16)
    int peel_columns;     // 1: column payload (every intermediate of a byte column in
                          // shared memory) when the code fits it; 0 (default): slice payload
    int peel_flow;        // 2 (default): the key walk for stripes of >= 64 MiB of
                          // intermediates; 3: the key walk at any size; 1: the
                          // dataflow walk without level barriers; 0: the level walk
                          // where its plan fits; 0 (default): level by level
    // slice encode tables (present when sl_slots > 0): every input block has
    // a 16-byte shared-memory slot per byte slice; data block v is slot v,
    // parity j is slot sl_bpad + j. The coded rows are split into sl_parts
    // parts (each with the parity rows too) so that every part's tables fit
    // shared memory beside the slot buffers; each part reads the data again.
    int32_t sl_box_rows;  // rows of one TMA box (data blocks per copy)
    int32_t sl_bpad;      // data slots, b rounded up to sl_box_rows
    int32_t sl_zbase;     // first of 8 zero slots (one per bank group), after the parities
    int32_t sl_slots;     // slots of one buffer (sl_zbase + 8)
    int32_t sl_parts;     // parts (1..kSliceParts)
    SlicePart sl_part[kSliceParts];
};

// A CSR with rows of strictly ascending in-range column indices (and the
// expected shape where an expectation is >= 0).
bool csr_ok(const fs_csr *g, int32_t n_rows_expect, int32_t n_cols_expect);

// Builds the slice encode tables of c (host arrays of the joint graph);
// leaves sl_slots = 0 when the code does not fit.
cudaError_t build_slice_tables(fs_code *c, const int32_t *con_ptr, const int32_t *con_idx);

// ---- batches of stripes (device plans built once, run many times) ---------
// Device copy of a host array for a batch plan: stream-ordered allocation and
// copy on a private non-blocking stream, so planning does not wait for work
// other streams have in flight. Free with plan_free.
template <typename T>
cudaError_t plan_upload(T **dst, const T *src, size_t count) {
    *dst = nullptr;
    if (count == 0) return cudaSuccess;
    cudaStream_t s;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
    e = cudaMallocAsync(reinterpret_cast<void **>(dst), sizeof(T) * count, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(*dst, src, sizeof(T) * count, cudaMemcpyHostToDevice, s);
    const cudaError_t e2 = cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
    return e != cudaSuccess ? e : e2;
}
template <typename T>
void plan_free(T *p) {
    if (p) cudaFree(p);
}
struct EncodeBatch;
cudaError_t encode_batch_plan(const fs_code *const *codes, const void *const *data,
                              void *const *parity, void *const *coded, int32_t n,
                              EncodeBatch **out);
cudaError_t encode_batch_run(const EncodeBatch *b, cudaStream_t s);
int32_t encode_batch_status_word(const EncodeBatch *b, int32_t *out);  // 0, or -1 on a CUDA error
void encode_batch_free(EncodeBatch *b);
struct DecodeBatch;
cudaError_t decode_batch_plan(const fs_code *const *codes, const void *const *coded,
                              const uint8_t *const *erased, void *const *data_out,
                              uint8_t *const *unrecovered, int32_t *const *n_unrecovered,
                              void *const *ws, int32_t n, bool schedule_only, DecodeBatch **out);
cudaError_t decode_batch_run(const DecodeBatch *b, cudaStream_t s);
void decode_batch_free(DecodeBatch *b);
void free_slice_tables(fs_code *c);

constexpr int kRecipeSeg = 8;  // recipe entries one payload thread gathers at once
constexpr int kColSegEntries = 7;  // row positions of one column-payload segment record
constexpr int kColSegMax = 256;    // segments of one column-payload step (one per thread)

// ---- workspace layouts (byte offsets from d_ws, 256-aligned) --------------
static inline size_t fs_align256(size_t x) { return (x + 255) & ~(size_t)255; }

// header words (int32) at the start of every workspace
enum {
    WS_STATUS = 0,      // fs_status of the last call (device side)
    WS_N_LEVELS = 1,
    WS_N_PAIRS = 2,
    WS_N_UNREC_DATA = 3,
    WS_COUNT_A = 4,     // scratch counters
    WS_COUNT_B = 5,
    WS_TILE_CTR = 6,
    WS_STAGED = 7,      // 1: every level fits the payload kernel's shared-memory stages
    WS_COL_STEPS = 8,   // steps of the column payload plan (-1: no plan)
    WS_ENC_TICKETS = 16,  // encode: ticket counters of the slice launches (one per part)
    WS_HDR_BYTES = 256
};

// Decode workspace. The DPG state arrays (res .. known) are a spill area used
// only when they do not fit in shared memory. The decoding path is written
// for the C API as level_off[l] (first pair of level l) and pair_f / pair_g,
// and for the payload kernel as
//   level_tab[2l]   = {first pair, pairs, first segment, segments}
//   level_tab[2l+1] = {first recipe chunk, recipe chunks, 0, 0}: a chunk is
//                  4 recipe entries (16 bytes); segment and chunk lists start
//                  on multiples of 4 entries
//   pair_rec[p]  = {f, g, ro, slot, e4, deg4, so, nseg}: ro = offset of its
//                  recipe in the level's recipe area, slot = its
//                  accumulator among the level's multi-segment pairs or -1,
//                  e4 / deg4 = its row in con_idx4, so / nseg = its first
//                  segment (level-relative) and segment count
//   seg_pair[s]  = pair of segment s (level-relative)
//   chunk_pair[c] = pair whose recipe holds chunk c (level-relative)
// The recipe of a pair is its padded row (f included and -1 padding, both
// skipped by the payload), gathered in segments of kRecipeSeg entries. All
// per-level ranges are 16-byte aligned so one bulk copy stages each.
// The column payload plan (built after the path when the code fits that
// kernel) is
//   col_src[v]  = coded row whose payload starts intermediate v, or -1 (a
//                 check, an unrecovered v, and v = k_int, the zero slot)
//   col_seg[s]  = segment record: 8 uint16 {e0..e6, f}; e_i are the
//                 intermediates at 7 consecutive positions of the row of g
//                 (k_int where the entry is f or past the row's end)
//   col_step[i] = first segment of step i; col_step[n_steps] = all segments.
//                 A step is at most kColSegMax segments of one level.
// The dataflow payload's plan (fs_peel.cu): the symbolic pass records the
// level of every recovered intermediate (flow_lvl) and clears the counters;
// k_flow_units turns every pair into units of gather work, kept per pair at
// its padded row's place (flow_raw: its loads from e4 on, flow_uarea /
// flow_ukey: its units and their keys from e4 / 4 on; a pair of padded degree
// deg4 has at most deg4 / 4 units and at most deg4 loads), counting units per
// key in flow_hist; k_flow_place puts the units in key order (flow_units),
// packs them into batches of at most 8 loads (flow_batch, 16 bytes each; at
// most one per unit) and lays their loads out in that order (flow_mem):
//   flow_hdr[0..7] = {units, loads, ok, check slots used, batches, slot
//                     counter, overflow, key walk fits}
//   flow_slot[s]   = segments of the check that sums into accumulator s
// The key walk's plan (FS_TUNE_PEEL_FLOW = 2, one CTA: k_key_plan) has the
// same units and loads, every heavy pair chained, without batches. The
// compact schedule records, for every constraint of degree >= kListDeg, its
// members in the order it recovered them (ascending level) at the
// constraint's padded row offset (flow_list, 16 bits each) and, for every
// pair p, its level | the degree of its constraint << 16 (flow_pinfo); units of key k
// (whole pairs, then chain links) and their loads fill one range each:
//   flow_ktab[2k..2k+1] = key k: {first unit, units, first unit rounded down
//                     to even, units from there rounded up to even}, {first
//                     load rounded down to a multiple of 8, loads from there
//                     rounded up to one, 0, 0}
constexpr int kFlowSlots = 128;  // check accumulator slots of the dataflow payload
struct DecodeLayout {
    size_t res, xs, best, known, front_a, front_b, touched, pair_f, pair_g, pair_rec, level_off,
        level_tab, seg_pair, chunk_pair, unrec_list, parity, col_src, col_step, col_seg, flow_hdr,
        flow_lvl, flow_hist, flow_ucnt, flow_uarea, flow_ukey, flow_raw, flow_units, flow_batch,
        flow_mem, flow_slot, flow_ktab, flow_list, flow_pinfo, total;
    int64_t col_max_segs, col_max_steps, flow_max_units, flow_max_loads;
};

static inline DecodeLayout decode_layout(const fs_code *c) {
    DecodeLayout L;
    size_t o = WS_HDR_BYTES;
    size_t K = (size_t)c->k_int, G = (size_t)c->n_con;
    L.res = o;        o = fs_align256(o + 4 * (G + 1));
    L.xs = o;         o = fs_align256(o + 4 * (G + 1));
    L.best = o;       o = fs_align256(o + 8 * (K + 1));
    L.known = o;      o = fs_align256(o + (K + 1));
    L.front_a = o;    o = fs_align256(o + 4 * (G + 1));
    L.front_b = o;    o = fs_align256(o + 4 * (G + 1));
    L.touched = o;    o = fs_align256(o + 4 * (K + 1));
    L.pair_f = o;     o = fs_align256(o + 4 * (K + 1));
    L.pair_g = o;     o = fs_align256(o + 4 * (K + 1));
    L.pair_rec = o;   o = fs_align256(o + 32 * (K + 1));
    L.level_off = o;  o = fs_align256(o + 4 * (K + 2));
    L.level_tab = o;  o = fs_align256(o + 32 * (K + 2));
    L.seg_pair = o;   o = fs_align256(o + 4 * (5 * K + (size_t)c->e_con4 / kRecipeSeg + 8));
    L.chunk_pair = o; o = fs_align256(o + 4 * (4 * K + (size_t)c->e_con4 / 4 + 8));
    L.unrec_list = o; o = fs_align256(o + 4 * (K + 1));
    L.parity = o;     o = fs_align256(o + (size_t)c->m * (size_t)c->t);
    // a constraint releases at most one intermediate, so the segments are at
    // most sum over constraints of ceil(degree / 7) <= e_con / 7 + K
    L.col_max_segs = (int64_t)c->e_con / kColSegEntries + (int64_t)K + 1;
    L.col_max_steps = (int64_t)K + L.col_max_segs / kColSegMax + 2;
    L.col_src = o;    o = fs_align256(o + 4 * (K + 1));
    L.col_step = o;   o = fs_align256(o + 4 * ((size_t)L.col_max_steps + 1));
    L.col_seg = o;    o = fs_align256(o + 16 * (size_t)L.col_max_segs);
    // units: at most e_con4 / 4 (deg4 / 4 per pair); loads: at most e_con4
    // plus one chain partial per unit
    L.flow_max_units = (int64_t)c->e_con4 / 4 + 1;
    L.flow_max_loads = (int64_t)c->e_con4 + L.flow_max_units;
    L.flow_hdr = o;   o = fs_align256(o + 64);
    L.flow_lvl = o;   o = fs_align256(o + 2 * (K + 1));
    L.flow_hist = o;  o = fs_align256(o + 4 * (K + 2));
    L.flow_ucnt = o;  o = fs_align256(o + 4 * (K + 1));
    L.flow_uarea = o; o = fs_align256(o + 8 * (size_t)L.flow_max_units);
    L.flow_ukey = o;  o = fs_align256(o + 2 * (size_t)L.flow_max_units);
    L.flow_raw = o;   o = fs_align256(o + 2 * (size_t)c->e_con4 + 16);
    L.flow_units = o; o = fs_align256(o + 8 * (size_t)L.flow_max_units + 16);
    L.flow_batch = o; o = fs_align256(o + 16 * (size_t)L.flow_max_units + 16);  // uint4 records
    L.flow_mem = o;   o = fs_align256(o + 2 * (size_t)L.flow_max_loads + 16);
    L.flow_slot = o;  o = fs_align256(o + 4 * (size_t)kFlowSlots);
    L.flow_ktab = o;  o = fs_align256(o + 32 * (K + 2));  // keys: at most levels + 1
    L.flow_list = o;  o = fs_align256(o + 2 * (size_t)c->e_con4 + 16);
    L.flow_pinfo = o; o = fs_align256(o + 4 * (K + 1));
    L.total = o;
    return L;
}

struct UpdateLayout {
    size_t mark, pmark, cmark, plist, clist, delta, pdelta, total;
};

static inline UpdateLayout update_layout(const fs_code *c, int32_t n_items) {
    UpdateLayout L;
    size_t o = WS_HDR_BYTES;
    L.mark = o;   o = fs_align256(o + 4 * ((size_t)c->b + 1));
    L.pmark = o;  o = fs_align256(o + 4 * ((size_t)c->m + 1));
    L.cmark = o;  o = fs_align256(o + 4 * ((size_t)c->n + 1));
    L.plist = o;  o = fs_align256(o + 4 * ((size_t)c->m + 1));
    L.clist = o;  o = fs_align256(o + 4 * ((size_t)c->n + 1));
    L.delta = o;  o = fs_align256(o + (size_t)(n_items > 0 ? n_items : 0) * (size_t)c->t);
    L.pdelta = o; o = fs_align256(o + (size_t)c->m * (size_t)c->t);
    L.total = o;
    return L;
}

// ---- L2 eviction-priority hints -------------------------------------------
// A cache policy (createpolicy) marks the lines an access brings into L2 as
// evict-last (data read again later in the same launch) or evict-first
// (data streamed through once). Used only where the tuning knob enables it.
#ifdef __CUDACC__
__device__ __forceinline__ uint64_t l2_policy_last() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;\n" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t l2_policy_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;\n" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint4 ld_nc_hint(const uint4 *ptr, uint64_t pol) {
    uint4 v;
    asm volatile("ld.global.nc.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;\n"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(ptr), "l"(pol));
    return v;
}
__device__ __forceinline__ uint4 ld_hint(const uint4 *ptr, uint64_t pol) {
    uint4 v;
    asm volatile("ld.global.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;\n"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(ptr), "l"(pol)
                 : "memory");
    return v;
}
__device__ __forceinline__ void st_hint(uint4 *ptr, const uint4 &v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.v4.u32 [%0], {%1, %2, %3, %4}, %5;\n" ::"l"(ptr),
                 "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w), "l"(pol)
                 : "memory");
}
#endif

// ---- kernel launchers (return cudaError_t of the launch) ----------------
// Gather-XOR over CSR rows: out row r = XOR of input blocks idx[ptr[r]..ptr[r+1]).
// Input block v lives at inA + v*tw (v < split) or inB + (v - split)*tw.
// rows == nullptr: row r writes out + r*tw; else it processes CSR row rows[r]
// (checked against n_valid) and writes out + rows[r]*tw.
struct GatherArgs {
    const int32_t *ptr;
    const int32_t *idx;
    const int32_t *rows;
    int32_t n_rows;
    int32_t row_base;    // added to r when rows == nullptr
    int32_t n_valid;     // bound for rows[r]
    const uint4 *inA;
    const uint4 *inB;
    int32_t split;
    uint4 *out;
    int64_t tw;
    int32_t *status;
};
cudaError_t launch_gather(const GatherArgs &a, int num_sms, int ctas_per_sm, cudaStream_t s);

// Encode (precode + LT) in one persistent launch; its workspace holds the
// status word, a tile counter and one counter per byte chunk.
size_t encode_ws_bytes(const fs_code *c);
cudaError_t launch_encode(const fs_code *c, const void *data, void *parity, void *coded, uint8_t *ws,
                          cudaStream_t s);

// Decoding path generation (Algorithm 5), one CTA.
cudaError_t launch_dpg(const fs_code *c, const uint8_t *erased, uint8_t *ws,
                       uint8_t *unrecovered, int32_t *n_unrecovered, cudaStream_t s);
// Payload of the decoding path.
cudaError_t launch_peel(const fs_code *c, const uint4 *coded, uint4 *data_out, uint8_t *ws,
                        cudaStream_t s);
// Column payload (fs_peel_col.cu). col_fits: the code's intermediates fit one
// CTA's shared memory as 16-byte slots (and 16-bit ids). The plan kernel runs
// after the symbolic pass when the column payload is selected and col_fits
// holds; the payload kernel then reads it (the symbolic pass marks the plan
// absent, and the payload reports FS_ERR_INVALID without one).
bool col_fits(const fs_code *c);
cudaError_t launch_col_plan(const fs_code *c, uint8_t *ws, cudaStream_t s);
cudaError_t launch_peel_col(const fs_code *c, const uint4 *coded, uint4 *data_out, uint8_t *ws,
                            cudaStream_t s);

// Update kernels.
cudaError_t launch_update(const fs_code *c, const int32_t *idx, int32_t n_idx, const uint4 *d_new,
                          uint4 *data, uint4 *parity, uint4 *coded, uint8_t *ws, cudaStream_t s);
