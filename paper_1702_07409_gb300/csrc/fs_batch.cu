// fs_batch.cu - batches of stripes: many independent stripes (Section 2.2:
// the data is cut into stripes that are coded and decoded independently) in
// a fixed number of launches, so small and uneven stripes keep the GPU busy
// and a batch can be captured in one CUDA graph and replayed.
#include <vector>

#include "fs_internal.cuh"

struct fs_batch {
    int op;
    int device;
    int32_t n;
    EncodeBatch *enc;
    DecodeBatch *dec;
};

namespace {

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

// argument checks of one stripe for op (the same rules as the single calls)
bool stripe_ok(const fs_stripe &s, int op, int device) {
    const fs_code *c = s.code;
    if (!c || c->device != device) return false;
    if (op == FS_OP_ENCODE) {
        if (!s.d_data || !s.d_coded) return false;
        if ((c->m > 0) != (s.d_parity != nullptr)) return false;
        return aligned16(s.d_data) && aligned16(s.d_parity) && aligned16(s.d_coded);
    }
    if (!s.d_unrecovered || !s.d_n_unrecovered || !s.d_ws) return false;
    if (c->n > 0 && !s.d_erased) return false;
    if (op == FS_OP_SCHEDULE) return aligned16(s.d_ws);
    if (!s.d_data_out || (c->n > 0 && !s.d_coded)) return false;
    return aligned16(s.d_coded) && aligned16(s.d_data_out) && aligned16(s.d_ws);
}

}  // namespace

FS_API fs_status fs_batch_create(const fs_stripe *stripes, int32_t n, int op, fs_batch **out) {
    if (!out) return FS_ERR_INVALID;
    *out = nullptr;
    if (n < 0 || (n > 0 && !stripes) ||
        (op != FS_OP_ENCODE && op != FS_OP_DECODE && op != FS_OP_SCHEDULE))
        return FS_ERR_INVALID;
    int device = -1;
    if (cudaGetDevice(&device) != cudaSuccess) return FS_ERR_CUDA;
    for (int32_t i = 0; i < n; ++i)
        if (!stripe_ok(stripes[i], op, device)) return FS_ERR_INVALID;
    std::vector<const fs_code *> codes(n);
    std::vector<const void *> cin(n);
    std::vector<void *> a(n), b(n), c(n), w(n);
    std::vector<const uint8_t *> er(n);
    std::vector<uint8_t *> un(n);
    std::vector<int32_t *> nu(n);
    for (int32_t i = 0; i < n; ++i) {
        codes[i] = stripes[i].code;
        cin[i] = op == FS_OP_ENCODE ? stripes[i].d_data : stripes[i].d_coded;
        a[i] = stripes[i].d_parity;
        b[i] = stripes[i].d_coded;
        c[i] = stripes[i].d_data_out;
        w[i] = stripes[i].d_ws;
        er[i] = stripes[i].d_erased;
        un[i] = stripes[i].d_unrecovered;
        nu[i] = stripes[i].d_n_unrecovered;
    }
    fs_batch *bt = new fs_batch();
    bt->op = op;
    bt->device = device;
    bt->n = n;
    bt->enc = nullptr;
    bt->dec = nullptr;
    cudaError_t e = op == FS_OP_ENCODE
                        ? encode_batch_plan(codes.data(), cin.data(), a.data(), b.data(), n, &bt->enc)
                        : decode_batch_plan(codes.data(), cin.data(), er.data(), c.data(), un.data(),
                                            nu.data(), w.data(), n, op == FS_OP_SCHEDULE, &bt->dec);
    if (e != cudaSuccess) {
        delete bt;
        return e == cudaErrorMemoryAllocation ? FS_ERR_NOMEM
               : e == cudaErrorInvalidValue   ? FS_ERR_INVALID
                                              : FS_ERR_CUDA;
    }
    *out = bt;
    return FS_OK;
}

FS_API fs_status fs_batch_run(const fs_batch *bt, void *stream) {
    if (!bt) return FS_ERR_INVALID;
    int device = -1;
    if (cudaGetDevice(&device) != cudaSuccess) return FS_ERR_CUDA;
    if (device != bt->device) return FS_ERR_INVALID;
    if (bt->n == 0) return FS_OK;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const cudaError_t e = bt->op == FS_OP_ENCODE ? encode_batch_run(bt->enc, s) : decode_batch_run(bt->dec, s);
    return e == cudaSuccess ? FS_OK : FS_ERR_CUDA;
}

FS_API fs_status fs_batch_status(const fs_batch *bt, int32_t *status) {
    if (!bt || !status) return FS_ERR_INVALID;
    *status = FS_OK;
    if (bt->op == FS_OP_ENCODE && bt->enc && encode_batch_status_word(bt->enc, status) != 0)
        return FS_ERR_CUDA;
    return FS_OK;
}

FS_API void fs_batch_destroy(fs_batch *bt) {
    if (!bt) return;
    cudaDeviceSynchronize();
    encode_batch_free(bt->enc);
    decode_batch_free(bt->dec);
    delete bt;
}
