// fs_local.cu - local recovery groups (check #2 and check #3 equations) and
// repair of lost coded blocks from them.
//
// Host, once per graph (fs_local_create): Algorithm 4 (Check Generation
// Algorithm) on the LT generator matrix B (k_int rows; column j = the
// intermediates of coded block j, a sorted set), with L starting as the
// identity; a column XOR is the symmetric difference of two sorted sets. A
// zero column j leaves the check #3 group l_j (coded blocks XORing to zero),
// a column reduced to {i} the check #2 equation x_i = XOR of l_j. The two
// set-XOR derivations of Section "Generating Information for Efficient
// Repair" add check #3 groups from degree-one coded blocks and from precode
// checks; the groups are then ordered by cardinality, so that the repair
// uses the smallest ones first.
//
// Device, per repair (fs_repair_local):
//   k_local_dpg (one CTA): the repair schedule, level by level like
//     Algorithm 5 with the lost coded blocks as the unknowns and the groups
//     as zero-payload constraints. Per group, res = lost members not yet
//     repaired and xs = the XOR of their indices, so a group with res == 1
//     names its unknown without a scan; each offered block takes the offering
//     group with the lowest (cardinality, index) key by a 64-bit atomicMin.
//     It then cuts every pair's group into chunks of kLocalChunk members (a
//     block scan gives each pair its first chunk) so that long groups spread
//     over many threads.
//   k_local_peel: each CTA owns a slice of 16-byte words of every block and
//     walks all levels (pairs of a level are independent: a level only reads
//     blocks repaired in earlier levels). One thread per (chunk, word) XORs
//     the chunk's members (eight loads in flight) and folds the result into a
//     shared-memory accumulator of its (pair, word) with 32-bit shared XOR
//     reductions; after a barrier the accumulators are written in place.
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <set>
#include <vector>

#include "fs_internal.cuh"

struct fs_local {
    int32_t n = 0, k_int = 0, sweeps = 0;
    std::vector<int32_t> g_ptr, g_idx;              // check #3 groups, repair order
    std::vector<int32_t> c2_inter, c2_ptr, c2_idx;  // check #2 equations
    bool on_device = false;
    int device = 0, num_sms = 1;
    int32_t *d_gptr = nullptr, *d_gidx = nullptr;  // groups
    int32_t *d_tptr = nullptr, *d_tidx = nullptr;  // transpose: coded block -> groups
};

namespace {

using Set = std::vector<int32_t>;

// w(a XOR b)
int32_t xor_size(const Set &a, const Set &b) {
    size_t i = 0, j = 0;
    int32_t w = 0;
    while (i < a.size() && j < b.size()) {
        if (a[i] == b[j]) {
            ++i;
            ++j;
        } else if (a[i] < b[j]) {
            ++i;
            ++w;
        } else {
            ++j;
            ++w;
        }
    }
    return w + (int32_t)(a.size() - i) + (int32_t)(b.size() - j);
}

// a = a XOR b
void xor_into(Set &a, const Set &b, Set &tmp) {
    tmp.clear();
    size_t i = 0, j = 0;
    while (i < a.size() && j < b.size()) {
        if (a[i] == b[j]) {
            ++i;
            ++j;
        } else if (a[i] < b[j]) {
            tmp.push_back(a[i++]);
        } else {
            tmp.push_back(b[j++]);
        }
    }
    tmp.insert(tmp.end(), a.begin() + i, a.end());
    tmp.insert(tmp.end(), b.begin() + j, b.end());
    a.swap(tmp);
}

// Algorithm 4. B[j] starts as row j of the LT graph (sorted, distinct), L[j]
// as {j}; returns the sweeps run.
int32_t run_cga(int32_t k, const fs_csr *lt, int32_t max_sweeps, std::vector<Set> &B,
                std::vector<Set> &L) {
    const int32_t n = lt->n_rows;
    B.assign(n, Set());
    L.assign(n, Set());
    for (int32_t j = 0; j < n; ++j) {
        B[j].assign(lt->col_idx + lt->row_ptr[j], lt->col_idx + lt->row_ptr[j + 1]);
        L[j].push_back(j);
    }
    int32_t sweeps = 0;
    Set tmp;
    for (;;) {
        int32_t zero = 0;
        for (int32_t j = 0; j < n; ++j) zero += B[j].empty() ? 1 : 0;
        if (zero >= n - k) break;
        if (max_sweeps > 0 && sweeps >= max_sweeps) break;
        bool changed = false;
        for (int32_t j = 0; j < n; ++j) {
            for (int32_t i = 0; i < n; ++i) {
                if (i == j || !(2 * (int64_t)B[j].size() > (int64_t)B[i].size())) continue;
                if (xor_size(B[j], B[i]) < (int32_t)B[j].size()) {
                    xor_into(B[j], B[i], tmp);
                    xor_into(L[j], L[i], tmp);
                    changed = true;
                }
            }
        }
        ++sweeps;
        if (!changed) break;
    }
    return sweeps;
}

void build_groups(fs_local *o, const fs_csr *precode, const fs_csr *lt, int32_t max_sweeps) {
    const int32_t n = lt->n_rows, k = o->k_int;
    const int32_t b = k - (precode ? precode->n_rows : 0);  // data blocks (plain or chained precode)
    std::vector<Set> B, L;
    o->sweeps = run_cga(k, lt, max_sweeps, B, L);
    std::vector<int32_t> c2_col(k, -1);  // first column reduced to {i}
    std::vector<Set> cand;
    for (int32_t j = 0; j < n; ++j) {
        if (B[j].empty())
            cand.push_back(L[j]);
        else if (B[j].size() == 1 && c2_col[B[j][0]] < 0)
            c2_col[B[j][0]] = j;
    }
    Set tmp;
    for (int32_t s = 0; s < n; ++s) {  // degree-one coded blocks
        if (lt->row_ptr[s + 1] - lt->row_ptr[s] != 1) continue;
        const int32_t i = lt->col_idx[lt->row_ptr[s]];
        if (c2_col[i] < 0) continue;
        Set g = L[c2_col[i]];
        xor_into(g, Set{s}, tmp);
        cand.push_back(g);
    }
    const int32_t m = precode ? precode->n_rows : 0;
    for (int32_t j = 0; j < m; ++j) {  // precode checks: members and parity b + j
        Set members(precode->col_idx + precode->row_ptr[j],
                    precode->col_idx + precode->row_ptr[j + 1]);
        members.push_back(b + j);
        bool all = true;
        for (int32_t v : members) all = all && c2_col[v] >= 0;
        if (!all) continue;
        Set g;
        for (int32_t v : members) xor_into(g, L[c2_col[v]], tmp);
        cand.push_back(g);
    }
    std::set<Set> seen;
    std::vector<Set> uniq;
    for (Set &g : cand)
        if (!g.empty() && seen.insert(g).second) uniq.push_back(g);
    std::stable_sort(uniq.begin(), uniq.end(),
                     [](const Set &x, const Set &y) { return x.size() < y.size(); });
    o->g_ptr.assign(1, 0);
    o->g_idx.clear();
    for (const Set &g : uniq) {
        o->g_idx.insert(o->g_idx.end(), g.begin(), g.end());
        o->g_ptr.push_back((int32_t)o->g_idx.size());
    }
    o->c2_inter.clear();
    o->c2_ptr.assign(1, 0);
    o->c2_idx.clear();
    for (int32_t i = 0; i < k; ++i) {
        if (c2_col[i] < 0) continue;
        o->c2_inter.push_back(i);
        o->c2_idx.insert(o->c2_idx.end(), L[c2_col[i]].begin(), L[c2_col[i]].end());
        o->c2_ptr.push_back((int32_t)o->c2_idx.size());
    }
}

template <typename T>
cudaError_t upload_vec(T **dst, const std::vector<T> &v) {
    const size_t bytes = sizeof(T) * (v.empty() ? 1 : v.size());
    cudaError_t e = cudaMalloc((void **)dst, bytes);
    if (e != cudaSuccess || v.empty()) return e;
    return cudaMemcpy(*dst, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice);
}

void free_local(fs_local *o) {
    for (int32_t *p : {o->d_gptr, o->d_gidx, o->d_tptr, o->d_tidx})
        if (p) cudaFree(p);
    delete o;
}

// ---- workspace ---------------------------------------------------------------
enum { LW_STATUS = 0, LW_N_LEVELS = 1, LW_N_PAIRS = 2, LW_N_UNREP = 3, LW_N_CHUNKS = 4 };

constexpr int kLocalDpgThreads = 1024;
constexpr int kLocalPeelThreads = 256;
constexpr int kLocalPeelCtasPerSm = 4;
constexpr int kLocalChunk = 64;     // group members one payload thread XORs
constexpr int kLocalAcc = 2048;     // (pair, word) accumulators of one payload CTA

struct LocalLayout {
    size_t res, xs, best, unknown, pair_f, pair_g, level_off, unrep, choff, chunk_pair,
        chunk_e0, level_chunk, total;
};

LocalLayout local_layout(const fs_local *o) {
    LocalLayout L;
    const size_t G = o->g_ptr.size() - 1, n = (size_t)o->n;
    // a group repairs at most one block, so the chunks are at most
    // sum over groups of ceil(|g| / kLocalChunk) <= entries / kLocalChunk + groups
    const size_t chunks = o->g_idx.size() / kLocalChunk + G + 1;
    size_t p = WS_HDR_BYTES;
    L.res = p;         p = fs_align256(p + 4 * (G + 1));
    L.xs = p;          p = fs_align256(p + 4 * (G + 1));
    L.best = p;        p = fs_align256(p + 8 * (n + 1));
    L.unknown = p;     p = fs_align256(p + (n + 1));
    L.pair_f = p;      p = fs_align256(p + 4 * (n + 1));
    L.pair_g = p;      p = fs_align256(p + 4 * (n + 1));
    L.level_off = p;   p = fs_align256(p + 4 * (n + 2));
    L.unrep = p;       p = fs_align256(p + 4 * (n + 1));
    L.choff = p;       p = fs_align256(p + 4 * (n + 1));
    L.chunk_pair = p;  p = fs_align256(p + 4 * chunks);
    L.chunk_e0 = p;    p = fs_align256(p + 4 * chunks);
    L.level_chunk = p; p = fs_align256(p + 4 * (n + 2));
    L.total = p;
    return L;
}

// ---- kernels -----------------------------------------------------------------

// In-place exclusive prefix sum of v[0, n) (global memory, read and written by
// the calling block only); returns the total to every thread. s_warp holds 33
// ints.
__device__ int32_t block_scan_global(int32_t *v, int32_t n, int32_t *s_warp) {
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
        __syncthreads();
    }
    return carry;
}

struct LocalDpgArgs {
    const int32_t *gptr, *gidx, *tptr, *tidx;
    const uint8_t *lost;
    int32_t n, G;
    int32_t *hdr;
    int32_t *res, *xs, *pair_f, *pair_g, *level_off, *unrep;
    int32_t *choff, *chunk_pair, *chunk_e0, *level_chunk;
    unsigned long long *best;
    uint8_t *unknown, *unrepaired;
    int32_t *n_unrepaired;
};

__global__ void __launch_bounds__(kLocalDpgThreads) k_local_dpg(LocalDpgArgs a) {
    __shared__ int32_t s_np, s_cnt, s_level, s_nu;
    __shared__ int32_t s_warp[33];
    for (int32_t g = threadIdx.x; g < a.G; g += blockDim.x) {
        a.res[g] = 0;
        a.xs[g] = 0;
    }
    for (int32_t s = threadIdx.x; s < a.n; s += blockDim.x) {
        a.unknown[s] = a.lost[s] ? 1 : 0;
        a.best[s] = ~0ull;
    }
    if (threadIdx.x == 0) {
        s_np = 0;
        s_level = 0;
        s_nu = 0;
    }
    __syncthreads();
    for (int32_t s = threadIdx.x; s < a.n; s += blockDim.x) {
        if (!a.lost[s]) continue;
        for (int32_t e = a.tptr[s]; e < a.tptr[s + 1]; ++e) {
            const int32_t h = a.tidx[e];
            atomicAdd(a.res + h, 1);
            atomicXor(a.xs + h, s);
        }
    }
    __syncthreads();
    for (;;) {
        // every group with one unknown bids for it; the lowest key wins
        for (int32_t g = threadIdx.x; g < a.G; g += blockDim.x) {
            if (a.res[g] != 1) continue;
            const unsigned long long key =
                (unsigned long long)(a.gptr[g + 1] - a.gptr[g]) << 32 | (unsigned)g;
            atomicMin(a.best + a.xs[g], key);
        }
        if (threadIdx.x == 0) s_cnt = 0;
        __syncthreads();
        const int32_t np0 = s_np;
        for (int32_t g = threadIdx.x; g < a.G; g += blockDim.x) {
            if (a.res[g] != 1) continue;
            const int32_t f = a.xs[g];
            const unsigned long long key =
                (unsigned long long)(a.gptr[g + 1] - a.gptr[g]) << 32 | (unsigned)g;
            if (a.best[f] != key) continue;
            const int32_t p = np0 + atomicAdd(&s_cnt, 1);
            a.pair_f[p] = f;
            a.pair_g[p] = g;
        }
        __syncthreads();
        const int32_t cnt = s_cnt;
        if (cnt == 0) break;
        // the level's blocks are repaired: update the groups that hold them
        for (int32_t p = np0 + threadIdx.x; p < np0 + cnt; p += blockDim.x) {
            const int32_t f = a.pair_f[p];
            a.unknown[f] = 0;
            a.best[f] = ~0ull;
            for (int32_t e = a.tptr[f]; e < a.tptr[f + 1]; ++e) {
                const int32_t h = a.tidx[e];
                atomicSub(a.res + h, 1);
                atomicXor(a.xs + h, f);
            }
        }
        if (threadIdx.x == 0) {
            a.level_off[s_level] = np0;
            s_np = np0 + cnt;
            ++s_level;
        }
        __syncthreads();
    }
    for (int32_t s = threadIdx.x; s < a.n; s += blockDim.x) {
        const uint8_t u = a.unknown[s];
        a.unrepaired[s] = u;
        if (u) a.unrep[atomicAdd(&s_nu, 1)] = s;
    }
    // chunks of every pair's group, in pair order; level l owns chunks
    // [level_chunk[l], level_chunk[l + 1])
    const int32_t np = s_np, nl = s_level;
    for (int32_t p = threadIdx.x; p < np; p += blockDim.x) {
        const int32_t g = a.pair_g[p];
        a.choff[p] = (a.gptr[g + 1] - a.gptr[g] + kLocalChunk - 1) / kLocalChunk;
    }
    __syncthreads();
    const int32_t n_chunks = block_scan_global(a.choff, np, s_warp);
    if (threadIdx.x == 0) a.choff[np] = n_chunks;
    __syncthreads();
    for (int32_t p = threadIdx.x; p < np; p += blockDim.x) {
        const int32_t g = a.pair_g[p], c0 = a.choff[p], nch = a.choff[p + 1] - c0;
        for (int32_t c = 0; c < nch; ++c) {
            a.chunk_pair[c0 + c] = p;
            a.chunk_e0[c0 + c] = a.gptr[g] + c * kLocalChunk;
        }
    }
    if (threadIdx.x == 0) a.level_off[nl] = np;
    __syncthreads();
    for (int32_t l = threadIdx.x; l <= nl; l += blockDim.x) a.level_chunk[l] = a.choff[a.level_off[l]];
    if (threadIdx.x == 0) {
        a.hdr[LW_N_LEVELS] = nl;
        a.hdr[LW_N_PAIRS] = np;
        a.hdr[LW_N_UNREP] = s_nu;
        a.hdr[LW_N_CHUNKS] = n_chunks;
        *a.n_unrepaired = s_nu;
    }
}

struct LocalPeelArgs {
    uint4 *coded;
    const int32_t *gptr, *gidx, *pair_f, *pair_g, *level_off, *unrep, *hdr;
    const int32_t *choff, *chunk_pair, *chunk_e0, *level_chunk;
    int64_t tw;
    int32_t L;  // words of every block per CTA
};

__device__ __forceinline__ void red_xor16(uint4 *d, const uint4 &v) {
    const uint32_t p = (uint32_t)__cvta_generic_to_shared(d);
    asm volatile("red.shared.xor.b32 [%0], %1;\n" ::"r"(p), "r"(v.x) : "memory");
    asm volatile("red.shared.xor.b32 [%0], %1;\n" ::"r"(p + 4), "r"(v.y) : "memory");
    asm volatile("red.shared.xor.b32 [%0], %1;\n" ::"r"(p + 8), "r"(v.z) : "memory");
    asm volatile("red.shared.xor.b32 [%0], %1;\n" ::"r"(p + 12), "r"(v.w) : "memory");
}

__global__ void __launch_bounds__(kLocalPeelThreads, kLocalPeelCtasPerSm)
    k_local_peel(LocalPeelArgs a) {
    __shared__ uint4 s_acc[kLocalAcc];
    const int64_t w0 = (int64_t)blockIdx.x * a.L;
    const int32_t lanes = (int32_t)min((int64_t)a.L, a.tw - w0);
    if (lanes <= 0) return;
    for (int32_t i = threadIdx.x; i < kLocalAcc; i += blockDim.x) s_acc[i] = make_uint4(0, 0, 0, 0);
    __syncthreads();
    const int32_t nl = a.hdr[LW_N_LEVELS];
    const int32_t per = kLocalAcc / lanes;  // pairs whose accumulators fit at once
    for (int32_t l = 0; l < nl; ++l) {
        const int32_t p1 = a.level_off[l + 1];
        for (int32_t pb = a.level_off[l]; pb < p1; pb += per) {
            const int32_t pe = min(p1, pb + per);
            const int32_t cb = a.choff[pb], items = (a.choff[pe] - cb) * lanes;
            for (int32_t it = threadIdx.x; it < items; it += blockDim.x) {
                const int32_t ci = cb + it / lanes, lane = it % lanes;
                const int32_t p = a.chunk_pair[ci], f = a.pair_f[p], g = a.pair_g[p];
                const int32_t e0 = a.chunk_e0[ci], e1 = min(e0 + kLocalChunk, a.gptr[g + 1]);
                const int64_t w = w0 + lane;
                uint4 acc = make_uint4(0, 0, 0, 0);
                int32_t e = e0;
                for (; e + 8 <= e1; e += 8) {  // eight loads in flight
                    uint4 v[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const int32_t h = __ldg(a.gidx + e + u);
                        v[u] = h != f ? a.coded[(int64_t)h * a.tw + w] : make_uint4(0, 0, 0, 0);
                    }
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        acc.x ^= v[u].x;
                        acc.y ^= v[u].y;
                        acc.z ^= v[u].z;
                        acc.w ^= v[u].w;
                    }
                }
                for (; e < e1; ++e) {
                    const int32_t h = __ldg(a.gidx + e);
                    if (h == f) continue;
                    const uint4 v = a.coded[(int64_t)h * a.tw + w];
                    acc.x ^= v.x;
                    acc.y ^= v.y;
                    acc.z ^= v.z;
                    acc.w ^= v.w;
                }
                red_xor16(s_acc + (p - pb) * lanes + lane, acc);
            }
            __syncthreads();
            for (int32_t it = threadIdx.x; it < (pe - pb) * lanes; it += blockDim.x) {
                const int32_t q = it / lanes, lane = it - q * lanes;
                a.coded[(int64_t)a.pair_f[pb + q] * a.tw + w0 + lane] = s_acc[it];
                s_acc[it] = make_uint4(0, 0, 0, 0);
            }
            __syncthreads();
        }
    }
    const int32_t nu = a.hdr[LW_N_UNREP];
    for (int32_t it = threadIdx.x; it < nu * lanes; it += blockDim.x) {
        const int32_t q = it / lanes, lane = it - q * lanes;
        a.coded[(int64_t)a.unrep[q] * a.tw + w0 + lane] = make_uint4(0, 0, 0, 0);
    }
}

bool al16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

}  // namespace

FS_API fs_status fs_local_create(const fs_csr *precode, const fs_csr *lt, int32_t max_sweeps,
                                 int flags, fs_local **out) {
    if (!out || !lt) return FS_ERR_INVALID;
    *out = nullptr;
    if (flags != 0 && flags != FS_LOCAL_HOST_ONLY) return FS_ERR_INVALID;
    const int32_t m = precode ? precode->n_rows : 0;
    const bool chained = precode && m > 0 && precode->n_cols == lt->n_cols;  // as fs_code_create
    const int32_t b = precode ? (chained ? precode->n_cols - m : precode->n_cols) : lt->n_cols;
    if (precode && !csr_ok(precode, -1, -1)) return FS_ERR_INVALID;
    if (b < 1 || m < 0 || (int64_t)b + m > INT32_MAX / 2) return FS_ERR_INVALID;
    if (!csr_ok(lt, -1, b + m)) return FS_ERR_INVALID;
    fs_local *o = new fs_local();
    o->n = lt->n_rows;
    o->k_int = b + m;
    build_groups(o, precode, lt, max_sweeps);
    if (o->g_idx.size() >= (size_t)INT32_MAX) {
        delete o;
        return FS_ERR_INVALID;
    }
    if (!(flags & FS_LOCAL_HOST_ONLY)) {
        // transpose: coded block -> the groups holding it
        std::vector<int32_t> tptr(o->n + 1, 0), tidx(o->g_idx.size());
        for (int32_t v : o->g_idx) ++tptr[v + 1];
        for (int32_t s = 0; s < o->n; ++s) tptr[s + 1] += tptr[s];
        std::vector<int32_t> fill(tptr.begin(), tptr.end() - 1);
        for (size_t g = 0; g + 1 < o->g_ptr.size(); ++g)
            for (int32_t e = o->g_ptr[g]; e < o->g_ptr[g + 1]; ++e)
                tidx[fill[o->g_idx[e]]++] = (int32_t)g;
        cudaError_t e = cudaGetDevice(&o->device);
        int v = 0;
        if (e == cudaSuccess)
            e = cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, o->device);
        o->num_sms = v > 0 ? v : 1;
        if (e == cudaSuccess) e = upload_vec(&o->d_gptr, o->g_ptr);
        if (e == cudaSuccess) e = upload_vec(&o->d_gidx, o->g_idx);
        if (e == cudaSuccess) e = upload_vec(&o->d_tptr, tptr);
        if (e == cudaSuccess) e = upload_vec(&o->d_tidx, tidx);
        if (e != cudaSuccess) {
            free_local(o);
            return e == cudaErrorMemoryAllocation ? FS_ERR_NOMEM : FS_ERR_CUDA;
        }
        o->on_device = true;
    }
    *out = o;
    return FS_OK;
}

FS_API void fs_local_destroy(fs_local *local) {
    if (!local) return;
    if (local->on_device) cudaDeviceSynchronize();
    free_local(local);
}

FS_API fs_status fs_local_info(const fs_local *o, int32_t *n, int32_t *k_int, int32_t *n_groups,
                               int64_t *group_entries, int32_t *n_check2, int64_t *check2_entries,
                               int32_t *sweeps) {
    if (!o) return FS_ERR_INVALID;
    if (n) *n = o->n;
    if (k_int) *k_int = o->k_int;
    if (n_groups) *n_groups = (int32_t)o->g_ptr.size() - 1;
    if (group_entries) *group_entries = (int64_t)o->g_idx.size();
    if (n_check2) *n_check2 = (int32_t)o->c2_inter.size();
    if (check2_entries) *check2_entries = (int64_t)o->c2_idx.size();
    if (sweeps) *sweeps = o->sweeps;
    return FS_OK;
}

FS_API fs_status fs_local_groups(const fs_local *o, int32_t *ptr, int32_t *idx) {
    if (!o || !ptr || (!idx && !o->g_idx.empty())) return FS_ERR_INVALID;
    memcpy(ptr, o->g_ptr.data(), sizeof(int32_t) * o->g_ptr.size());
    if (!o->g_idx.empty()) memcpy(idx, o->g_idx.data(), sizeof(int32_t) * o->g_idx.size());
    return FS_OK;
}

FS_API fs_status fs_local_check2(const fs_local *o, int32_t *inter, int32_t *ptr, int32_t *idx) {
    if (!o || !ptr || (!inter && !o->c2_inter.empty()) || (!idx && !o->c2_idx.empty()))
        return FS_ERR_INVALID;
    if (!o->c2_inter.empty())
        memcpy(inter, o->c2_inter.data(), sizeof(int32_t) * o->c2_inter.size());
    memcpy(ptr, o->c2_ptr.data(), sizeof(int32_t) * o->c2_ptr.size());
    if (!o->c2_idx.empty()) memcpy(idx, o->c2_idx.data(), sizeof(int32_t) * o->c2_idx.size());
    return FS_OK;
}

FS_API size_t fs_local_workspace_bytes(const fs_local *o) {
    return o ? local_layout(o).total : 0;
}

FS_API fs_status fs_repair_local(const fs_local *o, const uint8_t *d_lost, void *d_coded,
                                 size_t block_bytes, uint8_t *d_unrepaired,
                                 int32_t *d_n_unrepaired, void *d_ws, void *stream) {
    if (!o || !o->on_device || !d_lost || !d_coded || !d_unrepaired || !d_n_unrepaired || !d_ws)
        return FS_ERR_INVALID;
    if (block_bytes == 0 || (block_bytes & 15) != 0) return FS_ERR_INVALID;
    if (!al16(d_coded) || !al16(d_ws)) return FS_ERR_INVALID;
    if (o->n == 0) return FS_OK;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    uint8_t *w = static_cast<uint8_t *>(d_ws);
    const LocalLayout L = local_layout(o);
    cudaError_t e = cudaMemsetAsync(w, 0, WS_HDR_BYTES, s);
    if (e != cudaSuccess) return FS_ERR_CUDA;
    LocalDpgArgs a;
    a.gptr = o->d_gptr;
    a.gidx = o->d_gidx;
    a.tptr = o->d_tptr;
    a.tidx = o->d_tidx;
    a.lost = d_lost;
    a.n = o->n;
    a.G = (int32_t)o->g_ptr.size() - 1;
    a.hdr = reinterpret_cast<int32_t *>(w);
    a.res = reinterpret_cast<int32_t *>(w + L.res);
    a.xs = reinterpret_cast<int32_t *>(w + L.xs);
    a.best = reinterpret_cast<unsigned long long *>(w + L.best);
    a.unknown = w + L.unknown;
    a.pair_f = reinterpret_cast<int32_t *>(w + L.pair_f);
    a.pair_g = reinterpret_cast<int32_t *>(w + L.pair_g);
    a.level_off = reinterpret_cast<int32_t *>(w + L.level_off);
    a.unrep = reinterpret_cast<int32_t *>(w + L.unrep);
    a.choff = reinterpret_cast<int32_t *>(w + L.choff);
    a.chunk_pair = reinterpret_cast<int32_t *>(w + L.chunk_pair);
    a.chunk_e0 = reinterpret_cast<int32_t *>(w + L.chunk_e0);
    a.level_chunk = reinterpret_cast<int32_t *>(w + L.level_chunk);
    a.unrepaired = d_unrepaired;
    a.n_unrepaired = d_n_unrepaired;
    k_local_dpg<<<1, kLocalDpgThreads, 0, s>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return FS_ERR_CUDA;
    LocalPeelArgs p;
    p.coded = static_cast<uint4 *>(d_coded);
    p.gptr = o->d_gptr;
    p.gidx = o->d_gidx;
    p.pair_f = a.pair_f;
    p.pair_g = a.pair_g;
    p.level_off = a.level_off;
    p.unrep = a.unrep;
    p.hdr = a.hdr;
    p.choff = a.choff;
    p.chunk_pair = a.chunk_pair;
    p.chunk_e0 = a.chunk_e0;
    p.level_chunk = a.level_chunk;
    p.tw = (int64_t)(block_bytes / 16);
    int64_t ctas = (int64_t)o->num_sms * kLocalPeelCtasPerSm;
    if (ctas > p.tw) ctas = p.tw;
    int64_t Lw = (p.tw + ctas - 1) / ctas;
    if (Lw > kLocalAcc) Lw = kLocalAcc;  // a pair's accumulators fit beside the others
    p.L = (int32_t)Lw;
    ctas = (p.tw + Lw - 1) / Lw;
    k_local_peel<<<(unsigned)ctas, kLocalPeelThreads, 0, s>>>(p);
    return cudaGetLastError() == cudaSuccess ? FS_OK : FS_ERR_CUDA;
}

FS_API fs_status fs_local_path(const fs_local *o, const void *d_ws, fs_path_view *out) {
    if (!o || !d_ws || !out) return FS_ERR_INVALID;
    const uint8_t *w = static_cast<const uint8_t *>(d_ws);
    const LocalLayout L = local_layout(o);
    const int32_t *hdr = reinterpret_cast<const int32_t *>(w);
    out->n_levels = hdr + LW_N_LEVELS;
    out->n_pairs = hdr + LW_N_PAIRS;
    out->level_off = reinterpret_cast<const int32_t *>(w + L.level_off);
    out->pair_f = reinterpret_cast<const int32_t *>(w + L.pair_f);
    out->pair_g = reinterpret_cast<const int32_t *>(w + L.pair_g);
    out->parity = nullptr;
    out->plan = nullptr;
    return FS_OK;
}
