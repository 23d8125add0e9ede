// fs_static.cu - fs_encode_static: the encode entry point for callers that
// cannot allocate device memory.
//
// fs_encode needs a small caller-provided workspace (a status word and the
// work-ticket counters of its kernels). Some callers have no way to
// provide one: a storage service that reserves all of its device memory at
// start-up and forbids any later allocation (cudaMalloc may synchronise the
// device and can fail under memory pressure in the middle of a request), or
// a foreign-language binding with no device allocator of its own. For them
// this entry point takes its scratch from g_encode_scratch, a file-scope
// device array of kStaticScratchBytes bytes that every GPU loading this
// library holds until the process exits.
//
// In host code the name g_encode_scratch is only a host-side stand-in, not a
// device address; the address is looked up once per device with
// cudaGetSymbolAddress (with that device current) on the first call made on
// that device, and cached. Every call shares the array: the counters are
// cleared (cudaMemsetAsync, no allocation) at the start of each call, and
// calls that overlap on the GPU race on it.
#include <mutex>

#include "fs_internal.cuh"

namespace {

constexpr size_t kStaticScratchBytes = FS_ENCODE_STATIC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_encode_scratch[kStaticScratchBytes];

std::mutex g_scratch_mu;
void *g_scratch_ptr[kMaxDevices];

// Device address of the scratch array on the current device (looked up on
// the first call on each device).
cudaError_t scratch_address(int device, void **out) {
    if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ptr[device]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_encode_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[device] = p;
    }
    *out = g_scratch_ptr[device];
    return cudaSuccess;
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

}  // namespace

FS_API fs_status fs_encode_static(const fs_code *c, const void *d_data, void *d_parity,
                                  void *d_coded, int32_t *d_status, void *stream) {
    if (!c || !d_data || !d_coded) return FS_ERR_INVALID;
    if ((c->m > 0) != (d_parity != nullptr)) return FS_ERR_INVALID;
    if (!aligned16(d_data) || !aligned16(d_parity) || !aligned16(d_coded) ||
        ((uintptr_t)d_status & 3u) != 0)
        return FS_ERR_INVALID;
    if (encode_ws_bytes(c) > kStaticScratchBytes) return FS_ERR_SCRATCH;
    int device = -1;
    if (cudaGetDevice(&device) != cudaSuccess) return FS_ERR_CUDA;
    if (device != c->device) return FS_ERR_INVALID;
    void *scratch = nullptr;
    if (scratch_address(device, &scratch) != cudaSuccess) return FS_ERR_CUDA;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = launch_encode(c, d_data, d_parity, d_coded,
                                  static_cast<uint8_t *>(scratch), s);
    if (e == cudaSuccess && d_status)
        e = cudaMemcpyAsync(d_status, static_cast<uint8_t *>(scratch) + FS_WS_STATUS_OFFSET,
                            sizeof(int32_t), cudaMemcpyDeviceToDevice, s);
    return e == cudaSuccess ? FS_OK : FS_ERR_CUDA;
}

namespace {

// Waits on an mbarrier that expects bytes no copy will deliver, with the same
// kind of bounded wait the payload and encode kernels use; when the bound
// runs out it records FS_ERR_TIMEOUT and returns (nothing is in flight).
__global__ void k_selftest_timeout(int32_t *status, long long limit) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(&bar);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(a) : "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], 16;\n" ::"r"(a) : "memory");
    uint32_t done = 0;
    for (long long i = 0; i < limit && !done; ++i)
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(a)
            : "memory");
    *status = done ? (int32_t)FS_OK : (int32_t)FS_ERR_TIMEOUT;
}

}  // namespace

FS_API fs_status fs_selftest_timeout(int32_t *d_status, void *stream) {
    if (!d_status || ((uintptr_t)d_status & 3u) != 0) return FS_ERR_INVALID;
    k_selftest_timeout<<<1, 32, 0, reinterpret_cast<cudaStream_t>(stream)>>>(d_status, 1ll << 16);
    return cudaGetLastError() == cudaSuccess ? FS_OK : FS_ERR_CUDA;
}
