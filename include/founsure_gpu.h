/*
 * founsure_gpu.h - C ABI of the GB300 (sm_103a) Founsure gather-XOR library.
 *
 * Operations follow Arslan, "Founsure 1.0: An Erasure Code Library with
 * Efficient Repair and Update Features" (arXiv 1702.07409):
 *   encode  - Section 2.2: (1) precode parities (check #1), then (2) each of
 *             n coded blocks is the XOR (region XOR, Section 2.2) of its
 *             LDGM neighbours among the k_int = b + m intermediates.
 *   decode  - Algorithm 5 (Decoding Path Generation, Section 3.2) with the
 *             two rules of Section 3.1, then the payload of that path.
 *   repair  - Section 4 "conventional repair": a lost coded block is
 *             recomputed from the intermediates by the encoding rule.
 *   update  - data rewrite propagated by linearity: old XOR new of each
 *             rewritten block is XORed into every parity and coded block that
 *             has it as a neighbour (the paper's own "update", Section 2.9,
 *             generates extra coded rows, which is fs_encode_rows).
 *
 * Notation: b data blocks, m precode parities, k_int = b + m, n coded blocks,
 * t = block_bytes. Intermediate v is data block v for v < b and parity v - b
 * otherwise. Every payload buffer is block-major: block i occupies bytes
 * [i*t, (i+1)*t) of one contiguous buffer. t must be a positive multiple of
 * 16 and every device pointer 16-byte aligned.
 *
 * Ownership: the caller owns every device buffer (payloads, flags, index
 * lists, workspaces) and the stream. The library owns the fs_code object and
 * the device copies of its graphs, allocated once by fs_code_create.
 * Hot calls (fs_encode ... fs_update) allocate nothing: scratch comes from the
 * caller's workspace, sized by fs_workspace_bytes.
 *
 * Asynchrony and errors: every hot call only enqueues work on `stream` and
 * returns. Its return value covers host-side argument checks and launch
 * errors (FS_ERR_INVALID, FS_ERR_CUDA). Conditions found on the device (an
 * index out of range, a repeated update index, a bounded wait that gave up)
 * are written to the workspace status word (int32 at byte offset
 * FS_WS_STATUS_OFFSET of d_ws) as an fs_status value; it reads FS_OK after a
 * clean call. Decode stalls are results, not errors: the count of
 * unrecovered intermediates is written to *d_n_unrecovered. No call aborts
 * or traps.
 */
#ifndef FOUNSURE_GPU_H
#define FOUNSURE_GPU_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FS_OK = 0,
    FS_STALL = 1,       /* decode finished with unrecovered intermediates */
    FS_ERR_INVALID = 2, /* bad argument, graph, alignment or index */
    FS_ERR_CUDA = 3,    /* a CUDA runtime call failed */
    FS_ERR_NOMEM = 4,   /* fs_code_create could not allocate */
    FS_ERR_TIMEOUT = 5, /* a bounded device wait gave up */
    FS_ERR_SCRATCH = 6  /* fs_encode_static: the code needs more scratch than
                           its static area holds */
} fs_status;

/* A bipartite graph in CSR form, in HOST memory. Row r lists column indices
 * col_idx[row_ptr[r] .. row_ptr[r+1]) in strictly ascending order, each in
 * [0, n_cols). row_ptr has n_rows + 1 entries, row_ptr[0] == 0. */
typedef struct {
    int32_t n_rows;
    int32_t n_cols;
    const int32_t *row_ptr;
    const int32_t *col_idx;
} fs_csr;

typedef struct fs_code fs_code; /* opaque; owned by the library */

/* flags for fs_code_create (decoding mode, Section 2.2 / Algorithm 5) */
#define FS_DECODE_JOINT    0 /* peel coded rows and precode checks together */
#define FS_DECODE_TWO_PASS 1 /* peel coded rows to a fixpoint, then checks */

/* op codes for fs_workspace_bytes */
#define FS_OP_ENCODE 0
#define FS_OP_DECODE 1
#define FS_OP_UPDATE 2
#define FS_OP_REPAIR 3
#define FS_OP_SCHEDULE 4 /* fs_batch only: the decoding schedule alone (Algorithm 5) */

#define FS_WS_STATUS_OFFSET 0 /* int32 device status word inside every workspace */

/*
 * Creates a code from its two graphs (Section 2.2, Figure 2):
 *   precode: m rows (checks) over n_cols = b data blocks, or NULL for m = 0;
 *            or a chained precode over n_cols = k_int intermediates (the
 *            array LDPC checks of Algorithm 2): check j's members lie below
 *            b + j (data blocks and earlier parities; its own parity b + j is
 *            implied), and the checks come in level order (level = 1 + the
 *            deepest parity member). Chained codes encode level by level with
 *            the row-gather kernels (single calls and batches), and fs_update
 *            pushes deltas through the levels in order.
 *   lt:      n rows (coded blocks) over n_cols = k_int = b + m intermediates.
 * With precode == NULL, b is taken as lt->n_cols. block_bytes = t.
 * Validates both graphs on the host (bounds, ascending rows, sizes; empty
 * rows are allowed), builds the joint constraint graph and its transpose and
 * copies them to the current device. Returns FS_ERR_INVALID on a bad graph,
 * FS_ERR_NOMEM / FS_ERR_CUDA on allocation or copy failure. *out is set only
 * on FS_OK. Synchronous; not a hot call.
 */
fs_status fs_code_create(const fs_csr *precode, const fs_csr *lt, size_t block_bytes,
                         int flags, fs_code **out);
/* Frees the device graphs of the code (synchronises the device). NULL is a no-op. */
void fs_code_destroy(fs_code *code);
/* Sizes of the code: any out pointer may be NULL. */
fs_status fs_code_info(const fs_code *code, int32_t *b, int32_t *m, int32_t *n,
                       size_t *block_bytes);

/* Tuning knobs of a code. They change speed only, never a result.
 *   FS_TUNE_PEEL_CTAS    payload-peel CTAs per SM; each owns a slice of
 *                        every block sized so all slices run at once
 *                        (1..8; default 1)
 *   FS_TUNE_GATHER_CTAS  resident CTAs per SM of the gather kernels
 *                        (1..16; default 8)
 *   FS_TUNE_DPG_COMPACT  1 (default): the decoding schedule runs with 16-bit
 *                        indices and the whole graph in shared memory when
 *                        the code has at most 65536 intermediates and
 *                        constraints, no constraint of 65536 or more
 *                        members, and its graph and peeling state fit one
 *                        CTA's shared memory (219 KB at 4224 intermediates,
 *                        5528 constraints and 34799 edges); 0: the general
 *                        form
 *   FS_TUNE_L2_HINTS     1: encode and payload peel mark the blocks they
 *                        gather again as evict-last in L2 and streamed data
 *                        as evict-first; 0 (default): plain loads and stores
 *   FS_TUNE_ENCODE_SLICES 1 (default): encode holds one byte slice of every
 *                        data block and parity in shared memory and computes
 *                        all rows of that slice from it, when the code fits
 *                        (about 7000 data blocks + parities): 32-byte
 *                        slices when two buffers of them fit in shared
 *                        memory, or when d_coded is 32-byte aligned, t is a
 *                        multiple of 32 and the stripe has at least 8
 *                        slices per SM (each coded row's piece then goes out
 *                        as one 256-bit store), else 16-byte slices; 2:
 *                        always 16-byte slices; 3: always 32-byte slices
 *                        (when they fit); 0: row-gather encode through L2
 *   FS_TUNE_ROWS_PER_TICKET 1..16 (default 16): coded rows per work ticket of
 *                        the row-gather encode (single calls and batches);
 *                        fewer rows per ticket keep the tickets in flight on a
 *                        narrower byte range of every block (better L2 reuse
 *                        of the gathered inputs) at more scheduling cost
 *   FS_TUNE_PEEL_COLUMNS 1: the payload of a decode holds one 16-byte
 *                        column of every intermediate in shared memory and
 *                        walks all levels there, when the code fits (k_int + 1
 *                        16-byte slots: about 13500 intermediates); it moves
 *                        only the algorithmic bytes, in 16-byte pieces.
 *                        0 (default): the slice payload, which gathers
 *                        recovered blocks through L2 and HBM. Its plan is made
 *                        by the decoding schedule: set the knob before
 *                        fs_decode / fs_decode_schedule (a payload without
 *                        the plan reports FS_ERR_INVALID in the workspace)
 *   FS_TUNE_PEEL_FLOW    how the slice payload walks the decoding path.
 *                        The key walk: a heavy decoder (more than 8 loads:
 *                        precode checks, high-degree rows) is gathered in
 *                        pieces of 8 of its members, in the order the
 *                        schedule recovered them; each piece runs right
 *                        after the level that produced its last member
 *                        (while L2 still holds its members) and adds to a
 *                        partial sum kept in the output block; every other
 *                        pair is one gather at its own level; one barrier
 *                        per level. The schedule records the member order
 *                        and a one-CTA plan kernel lays the gathers out
 *                        (about 25 us at 4096 x 64 KiB, n = 5400, 20%
 *                        erased, where the payload reads 0.65 GB from HBM
 *                        against 1.04 GB level by level and runs 12%
 *                        faster).
 *                        2 (default): the key walk for codes whose
 *                        intermediates reach 64 MiB (k_int x t), the level
 *                        walk below that, where the recovered blocks stay in
 *                        L2 anyway and the plan's fixed cost (about 10-40
 *                        us) would not pay; 3: the key walk at any size;
 *                        1: the same pieces without level barriers, each
 *                        gather waiting only for the blocks it reads (fewer
 *                        HBM bytes still, more instructions: slower);
 *                        0: level by level, every pair whole.
 *                        Walks 1 to 3 apply to codes of at most 65535
 *                        intermediates and constraints, rows of at most
 *                        4000 entries and FS_TUNE_PEEL_CTAS = 1 (walks 2 and
 *                        3 also to the compact schedule), and to paths whose
 *                        plan fits the plan kernel's tables and the
 *                        payload's stages (at most 1024 levels); elsewhere
 *                        the payload walks level by level. Set it before
 *                        fs_decode / fs_decode_schedule (the schedule makes
 *                        the plan)
 * Returns FS_ERR_INVALID for an unknown knob or an out-of-range value. Not
 * thread-safe against concurrent hot calls on the same code. */
#define FS_TUNE_PEEL_CTAS   1
#define FS_TUNE_GATHER_CTAS 2
#define FS_TUNE_DPG_COMPACT 3
#define FS_TUNE_L2_HINTS    4
#define FS_TUNE_ENCODE_SLICES 5
#define FS_TUNE_ROWS_PER_TICKET 6
#define FS_TUNE_PEEL_COLUMNS 7
#define FS_TUNE_PEEL_FLOW    8
fs_status fs_code_set_tuning(fs_code *code, int knob, int value);

/* Bytes of caller-provided device workspace that op needs. n_items is the
 * largest n_idx an FS_OP_UPDATE call will pass (ignored for other ops).
 * Workspaces are 256-byte aligned by the caller; one workspace must not be
 * used by two calls that may overlap on the device. */
size_t fs_workspace_bytes(const fs_code *code, int op, int32_t n_items);

/*
 * Encode (Section 2.2, steps (1) and (2)).
 *   d_data   [b*t]  input, read only
 *   d_parity [m*t]  output parities (NULL iff m == 0)
 *   d_coded  [n*t]  output coded blocks
 *   d_ws     FS_OP_ENCODE workspace
 */
fs_status fs_encode(const fs_code *code, const void *d_data, void *d_parity, void *d_coded,
                    void *d_ws, void *stream);

/*
 * Encode only coded rows [row_begin, row_end) (the paper's update by code
 * extension, Section 2.9, when the LT graph was drawn with extra rows), from
 * resident intermediates d_data / d_parity. Writes rows row_begin..row_end-1
 * of d_coded (block-major over all n rows).
 */
fs_status fs_encode_rows(const fs_code *code, int32_t row_begin, int32_t row_end,
                         const void *d_data, const void *d_parity, void *d_coded, void *d_ws,
                         void *stream);

/*
 * Decode (Algorithm 5 + payload, Section 3.1 / 3.2).
 *   d_coded         [n*t]   received coded blocks; erased rows are ignored
 *   d_erased        [n]     uint8 flags, nonzero = coded block j erased
 *   d_data_out      [b*t]   recovered data; unrecovered blocks are zero
 *   d_unrecovered   [k_int] uint8 flags, 1 = intermediate not recovered
 *   d_n_unrecovered [1]     int32 count of unrecovered intermediates
 *   d_ws            FS_OP_DECODE workspace; also holds the parity
 *                   intermediates and the decoding path afterwards
 * Mode (joint / two-pass) comes from the code's flags.
 */
fs_status fs_decode(const fs_code *code, const void *d_coded, const uint8_t *d_erased,
                    void *d_data_out, uint8_t *d_unrecovered, int32_t *d_n_unrecovered,
                    void *d_ws, void *stream);

/*
 * The two halves of fs_decode, for callers that reuse one decoding path over
 * many stripes that share a graph and an erasure pattern (Section 2.2:
 * partitions of a file are coded with the same graph; a failed disk erases
 * the same rows of each):
 *   fs_decode_schedule - Algorithm 5 only: writes the path into d_ws and the
 *                        unrecovered flags / count (arguments as fs_decode);
 *   fs_decode_payload  - the payload of the path held in d_ws: reads d_coded,
 *                        writes d_data_out (unrecovered blocks zero) and the
 *                        parity intermediates inside d_ws.
 * fs_decode(...) is fs_decode_schedule followed by fs_decode_payload.
 */
fs_status fs_decode_schedule(const fs_code *code, const uint8_t *d_erased, uint8_t *d_unrecovered,
                             int32_t *d_n_unrecovered, void *d_ws, void *stream);
fs_status fs_decode_payload(const fs_code *code, const void *d_coded, void *d_data_out,
                            void *d_ws, void *stream);

/* Device pointers into a decode workspace, valid after fs_decode completes:
 * the decoding path DP of Algorithm 5 as pairs (pair_f[p], pair_g[p]) for
 * p < *n_pairs, level l owning pairs [level_off[l], level_off[l+1]) for
 * l < *n_levels. Inside a level the pair order is unspecified. Constraint g
 * is coded row g for g < n and precode check g - n otherwise. plan is the
 * header of the payload plan that FS_TUNE_PEEL_FLOW makes: {units, loads,
 * 1 when the plan was made, check slots, batches, checks seen, 1 when a pair
 * had too many segments, 1 when the plan suits the key walk} (all zero
 * when the knob is 0 or the code does not fit the plan). */
typedef struct {
    const int32_t *n_levels;  /* device int32 */
    const int32_t *n_pairs;   /* device int32 */
    const int32_t *level_off; /* device int32[k_int + 2] */
    const int32_t *pair_f;    /* device int32[k_int] */
    const int32_t *pair_g;    /* device int32[k_int] */
    const uint8_t *parity;    /* device [m*t]: recovered parity intermediates */
    const int32_t *plan;      /* device int32[8]: the payload plan's header */
} fs_path_view;
fs_status fs_decode_path(const fs_code *code, const void *d_ws, fs_path_view *out);

/*
 * Local recovery groups and repair from them (Section "Generating
 * Information for Efficient Repair", Algorithm 4 "Check Generation
 * Algorithm", and the repair process that peels over the groups).
 *
 * fs_local_create builds, on the host, from the same graph arguments as
 * fs_code_create:
 *   1. Algorithm 4 on the LT generator matrix B (k_int rows, column j = the
 *      intermediates of coded block j): sweeps over ordered column pairs
 *      (j, i) replace b_j by b_j XOR b_i (and l_j by l_j XOR l_i, L starting
 *      as the identity) when 2 w(b_j) > w(b_i) and w(b_j XOR b_i) < w(b_j),
 *      until n - k_int columns of B are zero, a sweep changes nothing, or
 *      max_sweeps sweeps ran (max_sweeps > 0). A zero column j gives the
 *      check #3 group l_j (coded blocks that XOR to zero); a column reduced
 *      to one intermediate i gives the check #2 equation x_i = XOR of l_j
 *      (the first such column per i);
 *   2. the set-XOR derivations: a coded block s of degree one over
 *      intermediate i adds (check #2 set of i) XOR {s}; a precode check whose
 *      members and parity all have check #2 sets adds the XOR of those sets;
 *   3. empty and repeated groups dropped (the first kept), the groups ordered
 *      by cardinality, ties in the order of steps 1-2.
 * The host work is sweeps x n^2 sorted-set comparisons (seconds at n ~ 5000).
 * Unless flags has FS_LOCAL_HOST_ONLY, the check #3 groups and their
 * transpose are copied to the current device. *out is set only on FS_OK.
 */
typedef struct fs_local fs_local; /* opaque; owned by the library */
#define FS_LOCAL_HOST_ONLY 1
fs_status fs_local_create(const fs_csr *precode, const fs_csr *lt, int32_t max_sweeps, int flags,
                          fs_local **out);
void fs_local_destroy(fs_local *local);
/* Sizes (any out pointer may be NULL): coded blocks, intermediates, check #3
 * groups and their total entries, check #2 equations and their total entries,
 * Algorithm 4 sweeps run. */
fs_status fs_local_info(const fs_local *local, int32_t *n, int32_t *k_int, int32_t *n_groups,
                        int64_t *group_entries, int32_t *n_check2, int64_t *check2_entries,
                        int32_t *sweeps);
/* Host copies. Check #3 groups in repair order as CSR: ptr[n_groups + 1],
 * idx[group_entries] (ascending coded indices per group). Check #2
 * equations in intermediate order: inter[n_check2], ptr[n_check2 + 1],
 * idx[check2_entries]. */
fs_status fs_local_groups(const fs_local *local, int32_t *ptr, int32_t *idx);
fs_status fs_local_check2(const fs_local *local, int32_t *inter, int32_t *ptr, int32_t *idx);
/* Device workspace of fs_repair_local (caller-owned, 16-byte aligned). */
size_t fs_local_workspace_bytes(const fs_local *local);
/*
 * Repairs lost coded blocks in place from the check #3 groups: d_lost[n]
 * flags (nonzero = lost), d_coded the n stored blocks of block_bytes each
 * (a multiple of 16; the lost ones are overwritten). Level by level, every
 * group with exactly one lost, not yet repaired member offers it; each
 * offered block takes the smallest offering group (ties: lowest group
 * index) and becomes the XOR of that group's other members; then the level's
 * blocks count as repaired. Lost blocks left unrepaired are zeroed and
 * flagged in d_unrepaired[n]; *d_n_unrepaired counts them. Asynchronous on
 * stream; FS_ERR_INVALID for a host-only fs_local or bad arguments.
 */
fs_status fs_repair_local(const fs_local *local, const uint8_t *d_lost, void *d_coded,
                          size_t block_bytes, uint8_t *d_unrepaired, int32_t *d_n_unrepaired,
                          void *d_ws, void *stream);
/* The repair path of the last fs_repair_local on d_ws, as device views: pair
 * (f, g) = coded block f from group g, levels as in fs_decode_path; parity and
 * plan are NULL. */
fs_status fs_local_path(const fs_local *local, const void *d_ws, fs_path_view *out);

/*
 * Update: data blocks d_idx[q] (q < n_idx, distinct, each < b) are replaced
 * by d_new[q*t .. (q+1)*t). For each one, delta = old XOR new is XORed into
 * every parity whose check contains it and every coded block whose
 * neighbours contain it or a changed parity, so that afterwards d_parity and
 * d_coded equal a full re-encode of the new data. d_data is updated in place.
 * A repeated or out-of-range index sets FS_ERR_INVALID in the workspace
 * status word. n_idx == 0 is a no-op.
 */
fs_status fs_update(const fs_code *code, const int32_t *d_idx, int32_t n_idx, const void *d_new,
                    void *d_data, void *d_parity, void *d_coded, void *d_ws, void *stream);

/*
 * Repair (conventional repair, Section 4): each lost coded block d_lost[q]
 * (q < n_lost, each < n) is recomputed from the resident intermediates
 * d_data / d_parity into its place in d_coded. An out-of-range index sets
 * FS_ERR_INVALID in the workspace status word and is skipped.
 */
fs_status fs_repair(const fs_code *code, const int32_t *d_lost, int32_t n_lost, const void *d_data,
                    const void *d_parity, void *d_coded, void *d_ws, void *stream);

/*
 * Encode without any caller workspace, for callers that cannot allocate
 * device memory (the paper has no counterpart: this is a deployment aid).
 * fs_encode needs a small workspace; a storage service that reserves all of
 * its device memory at start-up and forbids later allocation (cudaMalloc may
 * synchronise the device and can fail under memory pressure in the middle
 * of a request), or a binding with no device allocator, cannot supply one.
 * This call computes exactly what fs_encode computes (same arguments without
 * d_ws) using a static device area of FS_ENCODE_STATIC_SCRATCH_BYTES bytes
 * that every GPU loading the library holds until the process exits.
 *   d_status  optional device int32: receives the call's status word (FS_OK,
 *             or FS_ERR_TIMEOUT if a bounded wait gave up); NULL to skip
 * Returns FS_ERR_SCRATCH when fs_workspace_bytes(code, FS_OP_ENCODE, 0)
 * exceeds FS_ENCODE_STATIC_SCRATCH_BYTES (the encode of this library needs
 * only its status word and the work-ticket counters of its launches, 256
 * bytes whatever the block size, so every code fits today), FS_ERR_INVALID for bad
 * arguments or when the current device is not the
 * code's device. It calls no allocator. The first call on each device looks
 * up the area's device address (make it before any stream capture). All
 * calls share the area: calls that overlap on the GPU (other streams,
 * other threads) race and must be serialised by the caller.
 */
#define FS_ENCODE_STATIC_SCRATCH_BYTES 65536
fs_status fs_encode_static(const fs_code *code, const void *d_data, void *d_parity, void *d_coded,
                           int32_t *d_status, void *stream);

/* ---- batches of stripes --------------------------------------------------
 * Section 2.2 cuts the data into stripes (b blocks each) that are coded and
 * decoded independently; a batch runs many stripes, of any sizes and codes,
 * in a fixed number of launches (encode: one launch for every stripe's
 * precode rows, one for every stripe's LT rows; decode: one launch of the
 * symbolic pass, one CTA per stripe, per form, then one launch of the
 * payload over every (stripe, byte slice)). Each stripe's result is exactly
 * that of fs_encode / fs_decode on the same arguments.
 *
 * A stripe of a batch (host struct; the pointers are device pointers with
 * the same meaning, layout and alignment rules as the single calls):
 *   code             the stripe's code (every stripe of a batch on the
 *                    current device)
 *   encode: d_data (b·t in), d_parity (m·t out, NULL when m == 0),
 *           d_coded (n·t out)
 *   decode: d_coded (n·t in), d_erased (n flags), d_data_out (b·t out),
 *           d_unrecovered (k_int flags out), d_n_unrecovered (int32 out),
 *           d_ws (this stripe's fs_workspace_bytes(code, FS_OP_DECODE, 0)
 *           bytes, 16-byte aligned; after the run it holds the stripe's
 *           decoding path and status word like after fs_decode)
 * Unused fields are ignored. */
typedef struct {
    const fs_code *code;
    const void *d_data;
    void *d_parity;
    void *d_coded;
    const uint8_t *d_erased;
    void *d_data_out;
    uint8_t *d_unrecovered;
    int32_t *d_n_unrecovered;
    void *d_ws;
} fs_stripe;

typedef struct fs_batch fs_batch; /* opaque; owned by the library */

/* Plans a batch of n stripes for op (FS_OP_ENCODE, FS_OP_DECODE, or
 * FS_OP_SCHEDULE: the decoding schedule of every stripe without its payload,
 * for symbolic sweeps over erasure patterns such as the paper's simDisk
 * utility; it fills d_unrecovered, d_n_unrecovered and the path in d_ws, and
 * d_coded / d_data_out may be NULL): checks
 * every stripe (FS_ERR_INVALID on the first bad one, nothing created),
 * copies the per-stripe launch arguments to device memory (this call
 * allocates; the run does not). The stripes' buffers and codes must outlive
 * the batch. Blocks the host; not for stream capture. */
fs_status fs_batch_create(const fs_stripe *stripes, int32_t n, int op, fs_batch **out);

/* Enqueues the batch on stream (asynchronous, allocates nothing, no host
 * synchronisation: a run can be captured in a CUDA graph and the graph
 * replayed). FS_ERR_INVALID when the current device is not the batch's. */
fs_status fs_batch_run(const fs_batch *batch, void *stream);

/* The device status of the batch's last run (blocking: waits for the
 * copy): FS_OK, or FS_ERR_TIMEOUT when a bounded wait of the encode gave up.
 * A decode batch reports its stripes' statuses in their workspaces (as
 * fs_decode does) and always gives FS_OK here. */
fs_status fs_batch_status(const fs_batch *batch, int32_t *status);

/* Waits for the device, then frees the batch's device arrays. */
void fs_batch_destroy(fs_batch *batch);

/* Shows the library's wait-timeout path (no paper counterpart; for
 * failure-detection tests): enqueues one kernel whose bounded wait on an
 * mbarrier can never be satisfied (it expects bytes no copy delivers); when
 * the wait's iteration limit runs out the kernel writes FS_ERR_TIMEOUT to
 * *d_status (device int32, 4-byte aligned) and returns, leaving the context
 * usable. The payload and encode kernels bound their waits the same way and
 * report FS_ERR_TIMEOUT in their status words. */
fs_status fs_selftest_timeout(int32_t *d_status, void *stream);

/* Static string naming a status. */
const char *fs_status_string(fs_status s);

#ifdef __cplusplus
}
#endif
#endif
