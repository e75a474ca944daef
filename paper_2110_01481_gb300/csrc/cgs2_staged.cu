// The middle pass of a CGS2 Arnoldi step (paper Sec. 2, algorithm box, with
// MGS replaced by classical Gram-Schmidt applied twice) with one read of the
// basis instead of two:
//   q1 = q - W h1;  h2 = W^T q1;  ||q1||^2.
// The update needs every basis vector before the dot products can start, so
// a streaming kernel reads W twice here.  This one stages W in shared memory
// instead: persistent blocks take slices of 128 consecutive elements, and
// the k x 128 sub-matrix of a slice is brought in by bulk asynchronous
// copies (cp.async.bulk, one per basis vector, completing on an mbarrier),
// double-buffered so that the next slice streams in while this one is
// used; the update and the dot products then both read shared memory.  With
// the first pass (h1 = W^T q) and the last (q -= W h2 and the scaling) the
// step streams W three times.  Every wait on an mbarrier is bounded: after
// spin_limit polls the block sets *err, gives its copies in flight a
// bounded time to land, and stops.
#include <algorithm>

#include "vecops.cuh"

namespace {

constexpr int kSlice = 128;              // elements per slice = threads per block
constexpr int kSWarps = kSlice / 32;

__device__ __forceinline__ unsigned smem_addr(const void *p) {
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ bool mbar_try_wait(unsigned bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for phase `parity` of the mbarrier; false if it gave up.
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity, long long limit) {
    for (long long i = 0; i <= limit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// One bulk copy of `bytes` (a multiple of 16, both ends 16-byte aligned)
// from global src to shared dst, completing on the mbarrier bar.
__device__ __forceinline__ void bulk_copy(float *dst, const float *src, unsigned bytes, unsigned bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        :
        : "r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

// Warp 0: the copies of slice s (elements [s S, s S + S)) into buffer buf,
// one per basis vector, spread over the lanes after lane 0 has announced
// their total size on the mbarrier.
__device__ __forceinline__ void issue_slice(const float *__restrict__ W, int64_t ldw, int64_t L, int k,
                                            int64_t s, float *buf, unsigned bar) {
    const int lane = threadIdx.x & 31;
    const int64_t i0 = s * kSlice;
    // never past element L - 1 of a vector (L is a multiple of 4, so the
    // size is a multiple of 16 bytes); the rest of the last slice's buffer
    // is masked on use
    const int64_t n = min((int64_t)kSlice, L - i0);
    const unsigned bytes = (unsigned)(4 * n);
    if (lane == 0)
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                     :
                     : "r"(bar), "r"(bytes * (unsigned)k)
                     : "memory");
    __syncwarp();
    for (int j = lane; j < k; j += 32) bulk_copy(buf + (size_t)j * kSlice, W + (size_t)j * ldw + i0, bytes, bar);
}

// k from *kdev when set (a step of a captured solver loop).  Grid: at most
// the blocks that fit at once (the host checks), each looping over the
// slices blockIdx.x, blockIdx.x + gridDim.x, ...; partial sums per block in
// partials[j * Gp + blk] (j <= k: h2 rows, then ||q1||^2), the last block to
// finish sums them in a fixed order in FP64 into red_out[0..k].
__global__ void __launch_bounds__(kSlice)
cgs_pass2_staged_kernel(const float *__restrict__ W, int64_t ldw, int k, const int *__restrict__ kdev,
                        float *__restrict__ q, int64_t L, const double *__restrict__ h1,
                        float *__restrict__ partials, int Gp, unsigned *__restrict__ counter,
                        double *__restrict__ red_out, int *__restrict__ err, long long spin_limit) {
    extern __shared__ __align__(128) float s_w[];     // 2 buffers of k x kSlice, then kSlice q values
                                                       // (16-byte aligned), k coefficients, k + 1 sums
    __shared__ __align__(8) unsigned long long s_bar[2];
    __shared__ bool s_last, s_fail;
    if (kdev) k = *kdev;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float *buf0 = s_w, *buf1 = s_w + (size_t)k * kSlice;
    float *s_q = buf1 + (size_t)k * kSlice;           // the slice's updated q
    float *s_c = s_q + kSlice;                        // h1 as FP32
    float *s_acc = s_c + k;                           // per-block sums: h2[0..k-1], ||q1||^2
    const unsigned bar0 = smem_addr(&s_bar[0]), bar1 = smem_addr(&s_bar[1]);
    const int64_t nslices = (L + kSlice - 1) / kSlice;
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" : : "r"(bar0) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" : : "r"(bar1) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" : : : "memory");
        s_fail = false;
    }
    for (int j = tid; j < k; j += kSlice) s_c[j] = (float)h1[j];
    for (int j = tid; j <= k; j += kSlice) s_acc[j] = 0.0f;
    __syncthreads();
    if (warp == 0) {
        if ((int64_t)blockIdx.x < nslices) issue_slice(W, ldw, L, k, blockIdx.x, buf0, bar0);
        if ((int64_t)blockIdx.x + gridDim.x < nslices)
            issue_slice(W, ldw, L, k, blockIdx.x + gridDim.x, buf1, bar1);
    }
    int t = 0;
    for (int64_t s = blockIdx.x; s < nslices; s += gridDim.x, ++t) {
        const int b = t & 1;
        float *buf = b ? buf1 : buf0;
        const unsigned bar = b ? bar1 : bar0;
        if (!mbar_wait(bar, (unsigned)((t >> 1) & 1), spin_limit)) {
            atomicOr(err, 1);
            s_fail = true;
        }
        __syncthreads();
        if (s_fail) break;
        const int64_t i = s * kSlice + tid;
        const int64_t rem = L - s * kSlice;               // valid elements of this slice
        const bool valid = i < L;
        // q1 = q - W h1 for this thread's element (column tid of the slice's
        // k x 128 buffer: consecutive threads, consecutive banks)
        float qi = valid ? q[i] : 0.0f;
        if (valid) {
            float a[4] = {0.0f, 0.0f, 0.0f, 0.0f};
            int j = 0;
            for (; j + 3 < k; j += 4) {
#pragma unroll
                for (int e = 0; e < 4; ++e) a[e] = fmaf(s_c[j + e], buf[(size_t)(j + e) * kSlice + tid], a[e]);
            }
            for (; j < k; ++j) a[0] = fmaf(s_c[j], buf[(size_t)j * kSlice + tid], a[0]);
            qi -= (a[0] + a[1]) + (a[2] + a[3]);
            q[i] = qi;
        }
        s_q[tid] = qi;                                    // 0 past L
        __syncthreads();
        // h2_j += W_j^T q1 over the slice: thread j (< k) takes row j of the
        // buffer, in float4 groups starting at group (lane) and wrapping, so
        // that a warp's reads fall in distinct banks; groups past L are zero
        // in q1 and skipped
        for (int j = tid; j < k; j += kSlice) {
            const float4 *row = reinterpret_cast<const float4 *>(buf + (size_t)j * kSlice);
            const float4 *qq = reinterpret_cast<const float4 *>(s_q);
            float d[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll 8
            for (int g = 0; g < kSlice / 4; ++g) {
                const int c4 = (g + lane) & (kSlice / 4 - 1);
                if (4 * c4 >= rem) continue;
                const float4 w = row[c4], v = qq[c4];
                d[0] = fmaf(w.x, v.x, d[0]);
                d[1] = fmaf(w.y, v.y, d[1]);
                d[2] = fmaf(w.z, v.z, d[2]);
                d[3] = fmaf(w.w, v.w, d[3]);
            }
            s_acc[j] += (d[0] + d[1]) + (d[2] + d[3]);
        }
        // ||q1||^2: the warps' sums added in warp order by thread 0
        const float nn = warp_sum(qi * qi);
        __shared__ float s_nn[kSWarps];
        if (lane == 0) s_nn[warp] = nn;
        __syncthreads();
        if (tid == 0) {
            float a = 0.0f;
            for (int w = 0; w < kSWarps; ++w) a += s_nn[w];
            s_acc[k] += a;
        }
        if (warp == 0) {
            // every thread is done with this buffer: refill it with the slice
            // two ahead (generic-proxy reads ordered before the async writes)
            const int64_t s2 = s + 2 * (int64_t)gridDim.x;
            if (s2 < nslices) {
                asm volatile("fence.proxy.async.shared::cta;" : : : "memory");
                issue_slice(W, ldw, L, k, s2, buf, bar);
            }
        }
        __syncthreads();
    }
    if (s_fail) {
        // copies may still be landing in this block's shared memory: give
        // both buffers a bounded time to complete before leaving
        if (tid == 0) {
            mbar_wait(bar0, (unsigned)((t >> 1) & 1), spin_limit);
            mbar_wait(bar1, (unsigned)(((t + 1) >> 1) & 1), spin_limit);
        }
        return;
    }
    // per-block partials, then the last block's fixed-order FP64 sums
    for (int j = tid; j <= k; j += kSlice) partials[(size_t)j * Gp + blockIdx.x] = s_acc[j];
    __threadfence();
    __syncthreads();
    if (tid == 0) s_last = atomicAdd(counter, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const int G = gridDim.x;
    for (int j = warp; j <= k; j += kSWarps) {
        double a = 0.0;
        for (int g = lane; g < G; g += 32) a += (double)__ldcg(partials + (size_t)j * Gp + g);
        a = warp_sum_d(a);
        if (lane == 0) red_out[j] = a;
    }
    if (tid == 0) *counter = 0u;
}

}  // namespace

// Largest k the staged pass serves (two k x 128 FP32 buffers in shared memory).
int ctg_cgs_staged_max_k() { return 200; }

bool ctg_cgs_staged_ok(int64_t L, int k) { return k >= 1 && k <= ctg_cgs_staged_max_k() && (L & 3) == 0; }

static size_t staged_smem(int kmax) {
    return sizeof(float) * (2 * (size_t)kmax * kSlice + (size_t)kmax + kSlice + (size_t)kmax + 1);
}

cudaError_t ctg_cgs_pass2_staged(const float *W, int64_t ldw, int kmax, const int *kdev, float *q, int64_t L,
                                 const RedScratch &rs, long long spin_limit, cudaStream_t st) {
    if (kmax < 1 || kmax > ctg_cgs_staged_max_k() || (ldw & 3) != 0 || (L & 3) != 0 ||
        ((uintptr_t)W & 15) != 0)
        return cudaErrorInvalidValue;
    const size_t smem = staged_smem(kmax);
    cudaError_t e = cudaFuncSetAttribute(cgs_pass2_staged_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0, dev = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cgs_pass2_staged_kernel, kSlice, smem)) !=
        cudaSuccess)
        return e;
    const int64_t nslices = (L + kSlice - 1) / kSlice;
    int64_t G = (int64_t)std::max(1, per_sm) * sms;
    G = std::min<int64_t>(G, std::min<int64_t>(nslices, rs.grid));   // partial rows hold rs.grid blocks
    const int Gp = padded_grid(rs.grid);
    cgs_pass2_staged_kernel<<<(unsigned)G, kSlice, smem, st>>>(W, ldw, kmax, kdev, q, L, rs.h1, rs.partials, Gp,
                                                                 rs.counter, rs.h2,
                                                                 reinterpret_cast<int *>(rs.counter + 2),
                                                                 spin_limit);
    return cudaGetLastError();
}
