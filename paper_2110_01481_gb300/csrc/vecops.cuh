// Vector helpers shared by the Krylov kernels (arnoldi.cu, lsq.cu): float4
// loads and stores with a ragged tail, 16-bit basis loads and conversions,
// warp sums, and the deterministic last-block reduction (every block writes
// its partial sums, the last block to arrive sums them in a fixed order in
// FP64; no block waits for another).
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <type_traits>

#include "ctg_internal.cuh"

namespace {

constexpr int kThreads = 256, kWarps = kThreads / 32;
constexpr int kMaxE = 8;               // float4 groups per thread, at most

__device__ __forceinline__ float4 ld4(const float *p, int64_t g, int64_t L) {
    const int64_t i = 4 * g;
    if (i + 3 < L) return __ldg(reinterpret_cast<const float4 *>(p + i));
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (i < L) v.x = p[i];
    if (i + 1 < L) v.y = p[i + 1];
    if (i + 2 < L) v.z = p[i + 2];
    return v;
}

__device__ __forceinline__ float4 ld4_rw(const float *p, int64_t g, int64_t L) {
    const int64_t i = 4 * g;
    if (i + 3 < L) return *reinterpret_cast<const float4 *>(p + i);
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (i < L) v.x = p[i];
    if (i + 1 < L) v.y = p[i + 1];
    if (i + 2 < L) v.z = p[i + 2];
    return v;
}

__device__ __forceinline__ void st4(float *p, int64_t g, int64_t L, float4 v) {
    const int64_t i = 4 * g;
    if (i + 3 < L) {
        *reinterpret_cast<float4 *>(p + i) = v;
        return;
    }
    if (i < L) p[i] = v.x;
    if (i + 1 < L) p[i + 1] = v.y;
    if (i + 2 < L) p[i + 2] = v.z;
}

// Basis vectors may be stored in FP32, BF16 or FP16; every kernel converts
// them to FP32 on use and accumulates in FP32 (cross-block sums compensated).  A
// float4 group of the FP32 work vector pairs with one 8-byte load of a
// 16-bit basis vector.
// Raw (unconverted) loads, so that a batch of loads is issued before any
// conversion consumes one: FP32 groups stay float4, 16-bit groups are
// loaded as uint2 and converted only when used.
template <typename T> struct RawOf { using type = uint2; };
template <> struct RawOf<float> { using type = float4; };

__device__ __forceinline__ float4 ldraw(const float *p, int64_t g, int64_t L) { return ld4(p, g, L); }

template <typename H>
__device__ __forceinline__ uint2 ldraw16(const H *p, int64_t g, int64_t L) {
    const int64_t i = 4 * g;
    if (i + 3 < L) return __ldg(reinterpret_cast<const uint2 *>(p + i));
    unsigned short h[4] = {0, 0, 0, 0};
    const unsigned short *ps = reinterpret_cast<const unsigned short *>(p);
    if (i < L) h[0] = ps[i];
    if (i + 1 < L) h[1] = ps[i + 1];
    if (i + 2 < L) h[2] = ps[i + 2];
    return make_uint2((unsigned)h[0] | ((unsigned)h[1] << 16), (unsigned)h[2] | ((unsigned)h[3] << 16));
}
__device__ __forceinline__ uint2 ldraw(const __nv_bfloat16 *p, int64_t g, int64_t L) { return ldraw16(p, g, L); }
__device__ __forceinline__ uint2 ldraw(const __half *p, int64_t g, int64_t L) { return ldraw16(p, g, L); }

template <typename T> __device__ __forceinline__ float4 cvt4(float4 r) { return r; }
template <typename T> __device__ __forceinline__ float4 cvt4(uint2 u);
template <> __device__ __forceinline__ float4 cvt4<__nv_bfloat16>(uint2 u) {
    // a bf16 is the top half of an FP32
    return make_float4(__uint_as_float(u.x << 16), __uint_as_float(u.x & 0xFFFF0000u),
                       __uint_as_float(u.y << 16), __uint_as_float(u.y & 0xFFFF0000u));
}
template <> __device__ __forceinline__ float4 cvt4<__half>(uint2 u) {
    __half2 a, b;
    memcpy(&a, &u.x, 4);
    memcpy(&b, &u.y, 4);
    const float2 fa = __half22float2(a), fb = __half22float2(b);
    return make_float4(fa.x, fa.y, fb.x, fb.y);
}

__device__ __forceinline__ void stw4(float *p, int64_t g, int64_t L, float4 v) { st4(p, g, L, v); }

template <typename H>
__device__ __forceinline__ H to16(float x) {
    if constexpr (std::is_same<H, __nv_bfloat16>::value) return __float2bfloat16_rn(x);
    else return __float2half_rn(x);
}

template <typename H>
__device__ __forceinline__ void stw4_16(H *p, int64_t g, int64_t L, float4 v) {
    const int64_t i = 4 * g;
    if (i + 3 < L) {
        H h[4] = {to16<H>(v.x), to16<H>(v.y), to16<H>(v.z), to16<H>(v.w)};
        uint2 u;
        memcpy(&u, h, 8);
        *reinterpret_cast<uint2 *>(p + i) = u;
        return;
    }
    if (i < L) p[i] = to16<H>(v.x);
    if (i + 1 < L) p[i + 1] = to16<H>(v.y);
    if (i + 2 < L) p[i + 2] = to16<H>(v.z);
}
__device__ __forceinline__ void stw4(__nv_bfloat16 *p, int64_t g, int64_t L, float4 v) { stw4_16(p, g, L, v); }
__device__ __forceinline__ void stw4(__half *p, int64_t g, int64_t L, float4 v) { stw4_16(p, g, L, v); }

__device__ __forceinline__ float dot4(float4 a, float4 b) {
    return fmaf(a.x, b.x, fmaf(a.y, b.y, fmaf(a.z, b.z, a.w * b.w)));
}

__device__ __forceinline__ float warp_sum(float s) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

__device__ __forceinline__ double warp_sum_d(double s) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

// Compensated FP32 sums (Neumaier's variant of Kahan summation): s holds
// the running FP32 sum and c the sum of the exact rounding errors of its
// additions, so s + c (formed in FP64) carries a sum of n FP32 terms to
// about n 2^-48 sum |x_i|, against n 2^-53 sum |x_i| for FP64 accumulation
// and n 2^-24 sum |x_i| for plain FP32.  GB300 issues FP64 adds at about
// 1/64 of the FP32 rate (measured: 1.6 against 100 per clock and SM), so the
// cross-block sums of the reductions use these pairs and FP64 only for the
// final s + c.
struct F2 {
    float s, c;
};

__device__ __forceinline__ F2 f2_add(F2 a, float x) {
    const float t = a.s + x;
    const float e = fabsf(a.s) >= fabsf(x) ? (a.s - t) + x : (x - t) + a.s;   // exact: a.s + x - t
    return F2{t, a.c + e};
}

__device__ __forceinline__ F2 f2_merge(F2 a, F2 b) {
    F2 r = f2_add(a, b.s);
    r.c += b.c;
    return r;
}

// Warp sum of F2 pairs; at each step the lane with the offset bit clear is
// the left operand, so both partners form bit-identical results and every
// lane ends with the same pair.
__device__ __forceinline__ F2 warp_sum_f2(F2 v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const F2 w{__shfl_xor_sync(0xffffffffu, v.s, o), __shfl_xor_sync(0xffffffffu, v.c, o)};
        v = (lane & o) ? f2_merge(w, v) : f2_merge(v, w);
    }
    return v;
}

__device__ __forceinline__ double f2_value(F2 v) { return (double)v.s + (double)v.c; }

// The plane rotation that zeroes b below a (Sec. 2's Givens update): c =
// a / r, s = b / r, r = (a^2 + b^2)^(1/2), or c = 1, s = 0 when b = 0; and
// R's new diagonal entry as its reciprocal, rinv = 1 / r (1 / a when b = 0,
// 0 for a zero entry), the form solve_y_warp takes.  On GB300 a dependent
// FP64 division takes ~640 cycles and a square root ~675, against ~65 for an
// FMA (measured), so the rotation takes one reciprocal square root and y_k no
// division at all.  The entries are Hessenberg coefficients of vectors of
// norm at most ||r0||, far from the range where a^2 + b^2 overflows.
__device__ __forceinline__ void givens_rotation(double a, double b, double &c, double &s, double &rinv) {
    if (b != 0.0) {
        const double ir = rsqrt(fma(a, a, b * b));
        c = a * ir;
        s = b * ir;
        rinv = ir;
    } else {
        c = 1.0;
        s = 0.0;
        rinv = a != 0.0 ? 1.0 / a : 0.0;
    }
}

// y = R_k^{-1} g_{1:k} by back substitution in one warp, R (upper
// triangle, column-major with leading dimension ldr; its diagonal stored as
// reciprocals, givens_rotation) staged in shared memory in packed form when
// it fits (packed: column j holds j + 1 entries from offset j (j + 1) / 2),
// else read from global memory.
__device__ void solve_y_warp(const double *__restrict__ R, int ldr, const double *__restrict__ g, int k,
                             double *__restrict__ y, double *s_pack, int pack_cap) {
    const int lane = threadIdx.x & 31;
    const bool packed = k <= pack_cap;
    if (packed)
        // independent loads over the k x k square (the upper triangle kept)
        for (int e = lane; e < k * k; e += 32) {
            const int j = e / k, i = e - j * k;
            if (i <= j) s_pack[j * (j + 1) / 2 + i] = R[(size_t)j * ldr + i];
        }
    // t = g; for i = k-1 .. 0: y_i = t_i (1 / R_ii), t_j -= R_ji y_i (j < i);
    // lane l owns t_j for j = l, l + 32, ... (k <= 256)
    if (k > 256) {
        // beyond the registers: a plain loop over y (rows of R from global)
        if (lane == 0)
            for (int i = k - 1; i >= 0; --i) {
                double acc = g[i];
                for (int j = i + 1; j < k; ++j) acc -= R[(size_t)j * ldr + i] * y[j];
                y[i] = acc * R[(size_t)i * ldr + i];
            }
        __syncwarp();
        return;
    }
    double t[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int j = lane + 32 * q;
        t[q] = j < k ? g[j] : 0.0;
    }
    __syncwarp();
    for (int i = k - 1; i >= 0; --i) {
        const int qi = i >> 5, li = i & 31;
        double ti = 0.0;
#pragma unroll
        for (int q = 0; q < 8; ++q)
            if (q == qi) ti = __shfl_sync(0xffffffffu, t[q], li);
        const double yi = ti * (packed ? s_pack[i * (i + 1) / 2 + i] : R[(size_t)i * ldr + i]);
        if (lane == 0) y[i] = yi;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int j = lane + 32 * q;
            if (j < i) t[q] -= (packed ? s_pack[i * (i + 1) / 2 + j] : R[(size_t)i * ldr + j]) * yi;
        }
    }
    __syncwarp();
}

// Partial sums are laid out [j][Gp] with Gp = G rounded up to 4, so the
// last block can read them as float4.
__host__ __device__ inline int padded_grid(int G) { return (G + 3) & ~3; }

__device__ __forceinline__ F2 shfl_xor_f2(F2 v, int o) {
    return F2{__shfl_xor_sync(0xffffffffu, v.s, o), __shfl_xor_sync(0xffffffffu, v.c, o)};
}

// Rows [row0, row0 + nrows) of the per-block partials (G blocks, row
// stride Gp) summed over the blocks in one fixed order, as compensated
// FP32 pairs; out[j] (j < nrows, FP64).  Each warp takes R rows at a time:
// every lane reads them as float4 (four blocks per load), two lane strides'
// loads issued together, and adds them into one pair per row; the warp sum
// is then a transposed butterfly: at each of the first log2(R) levels a lane
// keeps half of its rows and merges its partner's copy of them, so a warp
// spends log2(R) + log2(32 / R) dependent shuffle levels on R rows instead of
// R times 5 (the serial chain of the summation tail was ~3,500 cycles for
// four rows with one butterfly per row, measured).  Every merge takes the
// lower lane's value first, so the order is fixed and every block that sums
// the same partials gets the same bits.  The padding entries (block index
// >= G) are never read into a sum.
template <int R = 4>
__device__ __forceinline__ void sum_partial_rows(const float *__restrict__ partials, int row0, int nrows, int G,
                                                 int Gp, double *out) {
    static_assert(R == 2 || R == 4 || R == 8, "rows per warp");
    constexpr int LR = R == 8 ? 3 : (R == 4 ? 2 : 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int G4 = Gp / 4;
    for (int j0 = warp * R; j0 < nrows; j0 += kWarps * R) {
        F2 acc[R];
#pragma unroll
        for (int r = 0; r < R; ++r) acc[r] = F2{0.f, 0.f};
        for (int g4 = lane; g4 < G4; g4 += 64) {
            const bool two = g4 + 32 < G4;
            float4 v[2][R];
#pragma unroll
            for (int u = 0; u < 2; ++u)
#pragma unroll
                for (int r = 0; r < R; ++r)
                    v[u][r] = (j0 + r < nrows && (u == 0 || two))
                                  ? __ldcg(reinterpret_cast<const float4 *>(partials + (size_t)(row0 + j0 + r) * Gp) +
                                           g4 + 32 * u)
                                  : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                if (u == 1 && !two) break;
                const int b0 = 4 * (g4 + 32 * u);      // < G: g4 + 32 u < G4 and Gp - G < 4
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    acc[r] = f2_add(acc[r], v[u][r].x);
                    if (b0 + 1 < G) acc[r] = f2_add(acc[r], v[u][r].y);
                    if (b0 + 2 < G) acc[r] = f2_add(acc[r], v[u][r].z);
                    if (b0 + 3 < G) acc[r] = f2_add(acc[r], v[u][r].w);
                }
            }
        }
        int row = 0;
#pragma unroll
        for (int l = 0; l < LR; ++l) {
            const int o = 16 >> l, n = R >> l;
            const bool hi = lane & o;
#pragma unroll
            for (int i = 0; i < n / 2; ++i) {
                const F2 keep = hi ? acc[i + n / 2] : acc[i];
                const F2 recv = shfl_xor_f2(hi ? acc[i] : acc[i + n / 2], o);
                acc[i] = f2_merge(hi ? recv : keep, hi ? keep : recv);
            }
            if (hi) row += n / 2;
        }
        F2 t = acc[0];
#pragma unroll
        for (int o = 16 >> LR; o > 0; o >>= 1) {
            const F2 recv = shfl_xor_f2(t, o);
            const bool hi = lane & o;
            t = f2_merge(hi ? recv : t, hi ? t : recv);
        }
        if ((lane & ((32 >> LR) - 1)) == 0 && j0 + row < nrows) out[j0 + row] = f2_value(t);
    }
}

// Writes this block's nred partial sums, then lets the last block sum all
// blocks' partials (fixed order, compensated FP32 pairs, sum_partial_rows,
// eight rows per warp)
// into red_out[0..nred-1] in FP64, so the serial tail is a few L2 round
// trips.  Returns true in the last block (after red_out is written and the
// block has synchronised), false in the others.
__device__ bool block_reduce_finish(float *s_w, int nred, float *__restrict__ partials,
                                    unsigned *__restrict__ counter,
                                    double *__restrict__ red_out, int blk, int G) {
    __shared__ bool s_last;
    const int tid = threadIdx.x;
    const int Gp = padded_grid(G);
    __syncthreads();
    for (int j = tid; j < nred; j += kThreads) {
        float s = 0.f;
        for (int w = 0; w < kWarps; ++w) s += s_w[w * nred + j];
        partials[(size_t)j * Gp + blk] = s;
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) s_last = (atomicAdd(counter, 1u) == (unsigned)(G - 1));
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
    sum_partial_rows<8>(partials, 0, nred, G, Gp, red_out);
    if (tid == 0) *counter = 0u;
    __syncthreads();
    return true;
}

}  // namespace
