// The matched back projector A^T of the Joseph forward projector, and the
// thresholded back projectors B_tau of Sec. 6.5, eq. (Btau): (B_tau)_ij =
// A_ji where A_ji >= tau max(A), else 0 (tau = 0 gives A^T).
//
// A^T is applied as a gather, one thread per pixel.  For a row-driven angle
// (c, s) = (cos, sin), ray d samples row i of the image at column
// u_d = (s_d - y_i s) / c + h, and the Joseph weight of pixel (i, j) in that
// ray is hat(u_d - j) / |c| with hat(z) = max(0, 1 - |z|).  With the pixel's
// detector coordinate t = (x_j c + y_i s) / ds + hd (the same t the
// pixel-driven B interpolates at), u_d - j = (d - t) ds / c, so
//   (A^T b)_ij = sum_a (1/|c_a|) sum_d hat((d - t) ds / |c_a|) b[a, d],
// and for a column-driven angle the same with |sin| in place of |cos|.
// Only the bins with |d - t| < |c| / ds contribute: two when ds >= |c|
// (always when ds >= 1), more for finer detector pitches.  B_tau keeps a
// term when its weight is >= the threshold tau max(A).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "ctg_internal.cuh"

namespace {

constexpr int kBX = 32, kBY = 8, kAChunk = 32;

__device__ __forceinline__ float val(float v) { return v; }
__device__ __forceinline__ float val(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float val(__half v) { return __half2float(v); }

__device__ __forceinline__ float frac24(long long U) {
    const unsigned f = (unsigned)((unsigned long long)U >> (CTG_FX_BITS - 24)) & 0xFFFFFFu;
    return (float)f * (1.0f / 16777216.0f);
}

struct ChunkAngle {
    float cf, sf, phi;    // tile-local slope and the fractional part at the tile origin
    int dbase;            // integer part at the tile origin
    float scale, inv_w;   // 1/|c|, ds/|c|
};

// Stage the parameters of angles a0 .. a0 + na - 1 for the tile at (i0, j0).
__device__ __forceinline__ void stage_chunk(ChunkAngle *sp, const BackAngle *tab,
                                            const MatchedAngle *mt, int a0, int na, int i0, int j0,
                                            int tid) {
    if (tid < na) {
        const BackAngle t = tab[a0 + tid];
        const long long U0 = t.C + (long long)j0 * t.COS + (long long)i0 * t.SIN;
        const MatchedAngle m = mt[a0 + tid];
        sp[tid] = ChunkAngle{t.cf, t.sf, frac24(U0), (int)(U0 >> CTG_FX_BITS), m.scale, m.inv_w};
    }
}

// MAX = false: x = B_thr b (+ add); MAX = true: the largest weight of A over
// the tile, folded into *max_bits (weights are >= 0, so their bit patterns
// order like the values).  rm: extra bins on each side beyond the two
// nearest (0 when every angle has ds >= |c|).
template <typename T, bool MAX>
__global__ void __launch_bounds__(kBX *kBY)
matched_back_kernel(const T *__restrict__ b, ColRef bc, int N, int n_angles, int n_det,
                    const BackAngle *__restrict__ tab, const MatchedAngle *__restrict__ mt, int rm,
                    float thr, const float *__restrict__ add, float *__restrict__ x,
                    unsigned *__restrict__ max_bits) {
    if (!MAX) b += col_offset(bc);
    __shared__ ChunkAngle sp[kAChunk];
    __shared__ float s_max[kBX * kBY / 32];
    const int j0 = blockIdx.x * kBX, i0 = blockIdx.y * kBY;
    const int dj = threadIdx.x, di = threadIdx.y, tid = di * kBX + dj;
    const int i = i0 + di, j = j0 + dj;
    const bool inside = i < N && j < N;
    const float fdj = (float)dj, fdi = (float)di;
    float acc = 0.0f;
    for (int a0 = 0; a0 < n_angles; a0 += kAChunk) {
        const int na = min(kAChunk, n_angles - a0);
        __syncthreads();
        stage_chunk(sp, tab, mt, a0, na, i0, j0, tid);
        __syncthreads();
        const T *brow = b + (size_t)a0 * n_det;
        for (int k = 0; k < na; ++k, brow += n_det) {
            const ChunkAngle p = sp[k];
            const float u = fmaf(fdi, p.sf, fmaf(fdj, p.cf, p.phi));
            const float fl = floorf(u);
            const float f = u - fl;                       // t = d0 + f
            const int d0 = p.dbase + (int)fl;
            for (int e = -rm; e <= rm + 1; ++e) {
                const float w = p.scale * fmaxf(0.0f, 1.0f - fabsf((float)e - f) * p.inv_w);
                const int d = d0 + e;
                if constexpr (MAX) {
                    if ((unsigned)d < (unsigned)n_det) acc = fmaxf(acc, w);
                } else {
                    if (w >= thr && w > 0.0f && (unsigned)d < (unsigned)n_det)
                        acc = fmaf(w, val(brow[d]), acc);
                }
            }
        }
    }
    if constexpr (MAX) {
        float m = inside ? acc : 0.0f;
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if ((tid & 31) == 0) s_max[tid >> 5] = m;
        __syncthreads();
        if (tid == 0) {
            for (int w = 1; w < kBX * kBY / 32; ++w) m = fmaxf(m, s_max[w]);
            atomicMax(max_bits, __float_as_uint(m));
        }
        return;
    }
    if (inside) {
        const size_t q = (size_t)i * N + j;
        x[q] = add ? acc + add[q] : acc;
    }
}

template <typename T>
cudaError_t launch_t(const T *b, ColRef bc, int N, int n_angles, int n_det, const BackAngle *tab,
                     const MatchedAngle *mt, int rm, float thr, const float *add, float *x,
                     cudaStream_t st) {
    const dim3 grid((N + kBX - 1) / kBX, (N + kBY - 1) / kBY);
    matched_back_kernel<T, false><<<grid, dim3(kBX, kBY), 0, st>>>(b, bc, N, n_angles, n_det, tab, mt, rm,
                                                                   thr, add, x, nullptr);
    return cudaGetLastError();
}

}  // namespace

cudaError_t ctg_launch_back_matched(const void *b, int dtype, int N, int n_angles, int n_det,
                                    const BackAngle *tab, const MatchedAngle *mt, int rm, float thr,
                                    const float *add, float *x, cudaStream_t st, ColRef bc) {
    switch (dtype) {
        case CTG_BASIS_FP32:
            return launch_t(static_cast<const float *>(b), bc, N, n_angles, n_det, tab, mt, rm, thr, add, x,
                            st);
        case CTG_BASIS_BF16:
            return launch_t(static_cast<const __nv_bfloat16 *>(b), bc, N, n_angles, n_det, tab, mt, rm, thr,
                            add, x, st);
        case CTG_BASIS_FP16:
            return launch_t(static_cast<const __half *>(b), bc, N, n_angles, n_det, tab, mt, rm, thr, add, x,
                            st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t ctg_matched_max(int N, int n_angles, int n_det, const BackAngle *tab,
                            const MatchedAngle *mt, int rm, unsigned *max_bits, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(max_bits, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    const dim3 grid((N + kBX - 1) / kBX, (N + kBY - 1) / kBY);
    matched_back_kernel<float, true><<<grid, dim3(kBX, kBY), 0, st>>>(
        nullptr, col_none(), N, n_angles, n_det, tab, mt, rm, 0.0f, nullptr, nullptr, max_bits);
    return cudaGetLastError();
}
