// ctg_cgs2_noalloc: the CGS2 Arnoldi step of ctg_cgs2 for callers that may
// not allocate device memory themselves.  Such callers include applications
// whose own memory manager has reserved the whole device up front and
// forbids any further cudaMalloc, and plugins that run inside a host
// framework that owns every device allocation.  Instead of a caller-provided
// scratch buffer, this entry point uses a fixed array in device memory that
// is part of the library image: every GPU that loads the library holds it
// until the process exits.  Nothing here calls cudaMalloc, cudaFree or any
// allocating library routine.
#include <mutex>

#include "ctg_internal.cuh"

namespace {

// Largest problem the fixed scratch serves: k <= 256 basis vectors of
// length L <= 4,980,736 (608 blocks x 256 threads x 8 float4 groups, which
// covers a 2048 x 2048 image).  The reduction scratch for that size is
// 635,136 bytes; the array is 640 KiB, and every call checks the exact
// requirement against it.
constexpr int kNoAllocMaxK = 256;
constexpr int64_t kNoAllocMaxL = 4980736;
constexpr size_t kNoAllocScratchBytes = 640 * 1024;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void *g_scratch_addr[kMaxDevices] = {};   // device address of the array, per device

// Host code may not use g_noalloc_scratch's name as a device pointer (it is a
// host-side stand-in); ask the runtime for its address on the current device.
// The lookup is repeated on every call whose stream is not being captured,
// so an address from a context that has since been torn down (after
// cudaDeviceReset, say) is never used; during a capture the address found by
// an earlier call on this device is used.
int scratch_address(cudaStream_t st, void **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CTG_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return CTG_ERR_INVALID_ARG;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) return CTG_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (cs == cudaStreamCaptureStatusNone) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr) return CTG_ERR_CUDA;
        g_scratch_addr[dev] = p;
    } else if (g_scratch_addr[dev] == nullptr) {
        return CTG_ERR_CUDA;                 // first call made under capture
    }
    *out = g_scratch_addr[dev];
    return CTG_OK;
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

}  // namespace

extern "C" int ctg_cgs2_noalloc(const float *W_dev, int64_t ld_w, int64_t L, int32_t k,
                                float *q_dev, float *w_out_dev, double *h_out_dev,
                                void *stream) {
    if (L < 1 || k < 0 || ld_w < L || (ld_w & 3) != 0) return CTG_ERR_INVALID_ARG;
    if (k > kNoAllocMaxK || L > kNoAllocMaxL) return CTG_ERR_INVALID_ARG;
    if ((k > 0 && !W_dev) || !q_dev || !w_out_dev || !h_out_dev) return CTG_ERR_INVALID_ARG;
    if ((k > 0 && !aligned16(W_dev)) || !aligned16(q_dev) || !aligned16(w_out_dev))
        return CTG_ERR_INVALID_ARG;
    if (ctg_red_scratch_bytes(L, k + 1) > kNoAllocScratchBytes) return CTG_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    void *scratch = nullptr;
    const int rc = scratch_address(st, &scratch);
    if (rc != CTG_OK) return rc;
    RedScratch rs;
    ctg_red_scratch_carve(scratch, L, k + 1, &rs);
    // the array keeps the previous call's contents: the completion counters
    // must start at zero
    if (cudaMemsetAsync(rs.counter, 0, 4 * sizeof(unsigned), st) != cudaSuccess) return CTG_ERR_CUDA;
    if (ctg_cgs2_step(W_dev, CTG_BASIS_FP32, ld_w, L, k, q_dev, w_out_dev, h_out_dev, rs, st) != cudaSuccess)
        return CTG_ERR_CUDA;
    return CTG_OK;
}
