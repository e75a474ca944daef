// Matrix-free projectors of the unmatched pair (A, B) (paper Sec. 1,
// eq. (1.1)-(1.2)): the Joseph ray-driven forward projector A, one thread
// per ray, and the pixel-driven back projector B, one thread per pixel,
// gather-only (no atomics).
#include "ctg_internal.cuh"

namespace {

constexpr int kPadTile = 32;

// pad = [x with 2 zero columns on each side | x^T likewise]; the zero
// border columns are written once when the buffer is allocated.
__global__ void pad_transpose_kernel(const float *__restrict__ x, float *__restrict__ pad,
                                     int N) {
    __shared__ float tile[kPadTile][kPadTile + 1];
    const size_t P = ctg_pad_stride(N);
    float *xp = pad, *xtp = pad + (size_t)N * P;
    const int j0 = blockIdx.x * kPadTile, i0 = blockIdx.y * kPadTile;
    for (int r = threadIdx.y; r < kPadTile; r += blockDim.y) {
        const int i = i0 + r, j = j0 + threadIdx.x;
        if (i < N && j < N) {
            const float v = x[(size_t)i * N + j];
            tile[r][threadIdx.x] = v;
            xp[(size_t)i * P + 2 + j] = v;
        }
    }
    __syncthreads();
    for (int r = threadIdx.y; r < kPadTile; r += blockDim.y) {
        const int j = j0 + r, i = i0 + threadIdx.x;   // xT[j][i] = x[i][j]
        if (i < N && j < N) xtp[(size_t)j * P + 2 + i] = tile[threadIdx.x][r];
    }
}

__device__ __forceinline__ float fx_frac(long long U) {
    // top 24 bits of the 40-bit fraction, exact in float
    const unsigned f24 = (unsigned)((unsigned long long)U >> (CTG_FX_BITS - 24)) & 0xFFFFFFu;
    return (float)f24 * (1.0f / 16777216.0f);
}

// b[a * n_det + d] = scale_a * sum_t lerp(img_a[t, .], u(d, t)).
__global__ void __launch_bounds__(256)
joseph_forward_kernel(const float *__restrict__ pad, int N, int n_angles, int n_det,
                      const FwdAngle *__restrict__ tab, float *__restrict__ b) {
    const long long ray = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (ray >= (long long)n_angles * n_det) return;
    const int a = (int)(ray / n_det);
    const int d = (int)(ray - (long long)a * n_det);
    const FwdAngle t = tab[a];
    const size_t P = ctg_pad_stride(N);
    const float *img = pad + (t.row_driven ? 0 : (size_t)N * P) + 2;

    // walk range: steps whose taps can touch the image, -1 < u < N, with a
    // one-step margin; the tap index is clamped below, so the estimate only
    // skips work and never changes the result
    const float u0 = fmaf((float)d, t.pf, t.qf);
    int lo = 0, hi = N - 1;
    if (fabsf(t.df) > 1e-20f) {
        float r1 = (-1.0f - u0) / t.df, r2 = ((float)N - u0) / t.df;
        float tlo = fmaxf(fminf(r1, r2), -2.0f), thi = fminf(fmaxf(r1, r2), (float)N + 1);
        lo = max(0, (int)floorf(tlo) - 1);
        hi = min(N - 1, (int)ceilf(thi) + 1);
    } else if (!(u0 > -2.0f && u0 < (float)N + 1.0f)) {
        lo = 1;
        hi = 0;
    }
    long long U = t.Q + (long long)d * t.P + (long long)lo * t.D;
    float acc = 0.0f;
    for (int s = lo; s <= hi; ++s) {
        int j0 = (int)(U >> CTG_FX_BITS);
        j0 = min(max(j0, -2), N);          // clamped taps read the zero border
        const float f = fx_frac(U);
        const float *row = img + (size_t)s * P + j0;
        const float v0 = __ldg(row), v1 = __ldg(row + 1);
        acc += fmaf(f, v1 - v0, v0);
        U += t.D;
    }
    b[ray] = acc * t.scale;
}

constexpr int kBX = 32, kBY = 8, kAChunk = 256;

// x[i, j] = sum_a lerp(b[a, .], u_a(i, j)) (+ add[i, j]).  A block owns a
// 32 x 8 pixel tile; the tile origin's detector position is formed exactly
// in fixed point once per angle, and each pixel adds its small float offset.
__global__ void __launch_bounds__(kBX *kBY)
pixel_back_kernel(const float *__restrict__ b, int N, int n_angles, int n_det,
                  const BackAngle *__restrict__ tab, const float *__restrict__ add,
                  float *__restrict__ x) {
    __shared__ float4 sp[kAChunk];
    const int j0 = blockIdx.x * kBX, i0 = blockIdx.y * kBY;
    const int dj = threadIdx.x, di = threadIdx.y;
    const int tid = di * kBX + dj;
    const float fdj = (float)dj, fdi = (float)di;
    float acc = 0.0f;
    for (int a0 = 0; a0 < n_angles; a0 += kAChunk) {
        const int na = min(kAChunk, n_angles - a0);
        __syncthreads();
        if (tid < na) {
            const BackAngle t = tab[a0 + tid];
            const long long U0 = t.C + (long long)j0 * t.COS + (long long)i0 * t.SIN;
            sp[tid] = make_float4(t.cf, t.sf, fx_frac(U0),
                                  __int_as_float((int)(U0 >> CTG_FX_BITS)));
        }
        __syncthreads();
        const float *brow = b + (size_t)a0 * n_det;
#pragma unroll 4
        for (int k = 0; k < na; ++k, brow += n_det) {
            const float4 p = sp[k];
            const float u = fmaf(fdi, p.y, fmaf(fdj, p.x, p.z));
            const float fl = floorf(u);
            const int dd = __float_as_int(p.w) + (int)fl;
            const float f = u - fl;
            const float v0 = ((unsigned)dd < (unsigned)n_det) ? __ldg(brow + dd) : 0.0f;
            const float v1 = ((unsigned)(dd + 1) < (unsigned)n_det) ? __ldg(brow + dd + 1) : 0.0f;
            acc += fmaf(f, v1 - v0, v0);
        }
    }
    const int i = i0 + di, j = j0 + dj;
    if (i < N && j < N) {
        const size_t p = (size_t)i * N + j;
        x[p] = add ? acc + add[p] : acc;
    }
}

}  // namespace

cudaError_t ctg_launch_pad(const float *x, float *pad, int N, cudaStream_t st) {
    dim3 grid((N + kPadTile - 1) / kPadTile, (N + kPadTile - 1) / kPadTile);
    pad_transpose_kernel<<<grid, dim3(kPadTile, 8), 0, st>>>(x, pad, N);
    return cudaGetLastError();
}

cudaError_t ctg_launch_forward(const float *pad, int N, int n_angles, int n_det,
                               const FwdAngle *tab, float *b, cudaStream_t st) {
    const long long m = (long long)n_angles * n_det;
    const int threads = 256;
    const long long blocks = (m + threads - 1) / threads;
    joseph_forward_kernel<<<(unsigned)blocks, threads, 0, st>>>(pad, N, n_angles, n_det, tab, b);
    return cudaGetLastError();
}

cudaError_t ctg_launch_back(const float *b, int N, int n_angles, int n_det,
                            const BackAngle *tab, const float *add, float *x,
                            cudaStream_t st) {
    dim3 grid((N + kBX - 1) / kBX, (N + kBY - 1) / kBY);
    pixel_back_kernel<<<grid, dim3(kBX, kBY), 0, st>>>(b, N, n_angles, n_det, tab, add, x);
    return cudaGetLastError();
}
