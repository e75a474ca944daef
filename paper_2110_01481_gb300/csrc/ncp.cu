// The NCP stopping criterion of Sec. 6.4: how far the residual b - A x_k is
// from white noise, judged by its normalised cumulative periodogram.  The
// paper defines it only by citation; the reading implemented here: each
// projection (one angle, N_d bins) of the residual sinogram is a signal;
// with q = floor(N_d / 2) and rhat its DFT, p_i = |rhat_i|^2 (i = 1..q, the
// zero frequency left out), c_i = (p_1 + ... + p_i) / (p_1 + ... + p_q);
// the projection's distance is ||c - (1..q)/q||_2 (0 when p = 0), and the
// residual's distance is the mean over the projections.
//
// One block per projection.  The q periodogram ordinates are a direct DFT
// (q * N_d complex multiply-adds per projection, with the projection staged
// in shared memory, the twiddles advanced by a re-anchored rotating phasor);
// the cumulative sums are a chunked
// scan in FP64 in a fixed order, and the mean over projections is a
// fixed-order reduction, so the result is deterministic.
#include "ctg_internal.cuh"

namespace {

constexpr int kNcpThreads = 256;

__global__ void __launch_bounds__(kNcpThreads)
ncp_projection_kernel(const float *__restrict__ r, int n_det, const float2 *__restrict__ tw,
                      double *__restrict__ dist) {
    extern __shared__ float sm[];
    float *rs = sm;                 // n_det
    float *ps = sm + n_det;         // q
    __shared__ double s_part[kNcpThreads];
    __shared__ double s_red[kNcpThreads / 32];
    const int a = blockIdx.x, tid = threadIdx.x;
    const int q = n_det / 2;
    const float *ra = r + (size_t)a * n_det;
    for (int d = tid; d < n_det; d += kNcpThreads) rs[d] = ra[d];
    __syncthreads();
    // rhat_i = sum_d r_d z^d with z = exp(-2 pi i i / n_det): the phasor z^d
    // is advanced by complex multiplication and re-anchored from the exact
    // table every kAnchor bins, so its rounding drift stays ~kAnchor eps;
    // all lanes read the same r_d (a shared-memory broadcast)
    constexpr int kAnchor = 32;
    for (int i = tid + 1; i <= q; i += kNcpThreads) {
        const float2 w = tw[i];
        float re = 0.f, im = 0.f;
        int anchor = 0;                       // (i * d0) mod n_det
        for (int d0 = 0; d0 < n_det; d0 += kAnchor) {
            float2 z = tw[anchor];
            const int d1 = min(n_det, d0 + kAnchor);
            for (int d = d0; d < d1; ++d) {
                const float v = rs[d];
                re = fmaf(v, z.x, re);
                im = fmaf(v, z.y, im);
                const float zx = fmaf(z.x, w.x, -z.y * w.y);
                z.y = fmaf(z.x, w.y, z.y * w.x);
                z.x = zx;
            }
            anchor = (int)(((long long)i * d1) % n_det);
        }
        ps[i - 1] = fmaf(re, re, im * im);
    }
    __syncthreads();
    // chunked scan: thread t owns ordinates [t C, (t + 1) C)
    const int C = (q + kNcpThreads - 1) / kNcpThreads;
    const int i0 = min(q, tid * C), i1 = min(q, i0 + C);
    double part = 0.0;
    for (int i = i0; i < i1; ++i) part += (double)ps[i];
    s_part[tid] = part;
    __syncthreads();
    if (tid == 0) {
        double run = 0.0;
        for (int t = 0; t < kNcpThreads; ++t) {
            const double v = s_part[t];
            s_part[t] = run;        // exclusive prefix
            run += v;
        }
        s_red[0] = run;             // total, read below before s_red is reused
    }
    __syncthreads();
    const double total = s_red[0];
    double acc = 0.0;
    if (total > 0.0) {
        double cum = s_part[tid];
        for (int i = i0; i < i1; ++i) {
            cum += (double)ps[i];
            const double diff = cum / total - (double)(i + 1) / q;
            acc += diff * diff;
        }
    }
    __syncthreads();                // every thread has read s_red[0]
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((tid & 31) == 0) s_red[tid >> 5] = acc;
    __syncthreads();
    if (tid == 0) {
        double s = 0.0;
        for (int w = 0; w < kNcpThreads / 32; ++w) s += s_red[w];
        dist[a] = sqrt(s);
    }
}

__global__ void __launch_bounds__(kNcpThreads)
ncp_mean_kernel(const double *__restrict__ dist, int n_angles, double *__restrict__ out) {
    __shared__ double s[kNcpThreads];
    double acc = 0.0;
    for (int a = threadIdx.x; a < n_angles; a += kNcpThreads) acc += dist[a];
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int w = kNcpThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = s[0] / n_angles;
}

size_t ncp_smem_bytes(int n_det) { return sizeof(float) * ((size_t)n_det + n_det / 2); }

}  // namespace

cudaError_t ctg_ncp(const float *r, int n_angles, int n_det, const float2 *tw, double *dist_scratch,
                    double *out, cudaStream_t st) {
    if (n_det < 2 || n_det > kCtgNcpMaxDet) return cudaErrorInvalidValue;
    const size_t smem = ncp_smem_bytes(n_det);
    if (smem > 32 * 1024) {        // with the static arrays, past the default 48 KB
        const cudaError_t e = cudaFuncSetAttribute(ncp_projection_kernel,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    ncp_projection_kernel<<<n_angles, kNcpThreads, smem, st>>>(r, n_det, tw, dist_scratch);
    ncp_mean_kernel<<<1, kNcpThreads, 0, st>>>(dist_scratch, n_angles, out);
    return cudaGetLastError();
}
