// Matrix-free projectors of the unmatched pair (A, B) (paper Sec. 1,
// eq. (1.1)-(1.2)): the Joseph ray-driven forward projector A, one thread
// per ray, and the pixel-driven back projector B, one thread per pixel
// (four pixels per thread), gather-only (no atomics).
//
// Both kernels read their input as (value, forward difference) pairs, so one
// 8-byte load and one FMA give a linear interpolation:
//   lerp(v, j + f) = v[j] + f (v[j+1] - v[j]).
#include <cooperative_groups.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <type_traits>

#include "ctg_internal.cuh"

namespace cg = cooperative_groups;

namespace {

constexpr int kPadTile = 32;
constexpr int kPadRows = 8;    // staging blocks are kPadTile x kPadRows threads

// Inputs that are Krylov basis vectors may be stored in BF16 or FP16.
__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float to_f(__half v) { return __half2float(v); }

__device__ __forceinline__ float2 lerp_pair(float v0, float v1) {
    // (v0 - dv, dv): with m = 1 + f, (v0 - dv) + m dv = v0 + f dv
    const float dv = v1 - v0;
    return make_float2(v0 - dv, dv);
}

// Stage the image for the forward projector (layout in ctg_internal.cuh):
// entries j = -1 .. N-1 of every row of x and of x^T; the other border
// entries are zero pairs written once when the buffer is allocated.  With
// kImgs = 2 two images x (type T) and x2 (FP32) are staged interleaved, each
// entry a float4 (pair of x, pair of x2), so that the forward projector
// reads both with one load.
template <int kImgs, typename T>
__device__ __forceinline__ void pad_pairs_block(const T *__restrict__ x, const float *__restrict__ x2,
                                                void *__restrict__ pad_out, int N, int stride, int border,
                                                int bx, int by) {
    using E = typename std::conditional<kImgs == 2, float4, float2>::type;
    // odd pitch: the column reads of the transposed copy hit 32 distinct banks
    __shared__ float tile[kImgs][kPadTile + 1][kPadTile + 1];
    E *pad = static_cast<E *>(pad_out);
    E *xp = pad + border, *xtp = pad + (size_t)N * stride + border;
    const int j0 = bx * kPadTile, i0 = by * kPadTile;
    // tile[q][r][c] = image q at (i0 + r, j0 + c) for r, c in [0, 33) (0
    // outside); every load is issued before the first shared store
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * kPadTile + tx;
    constexpr int kPasses = (kPadTile + kPadRows) / kPadRows;   // rows 0 .. kPadTile
    float v[kImgs][kPasses];
#pragma unroll
    for (int t = 0; t < kPasses; ++t) {
        const int r = ty + t * kPadRows, i = i0 + r, j = j0 + tx;
        const bool in = r <= kPadTile && i < N && j < N;
        v[0][t] = in ? to_f(x[(size_t)i * N + j]) : 0.0f;
        if (kImgs == 2) v[kImgs - 1][t] = in ? x2[(size_t)i * N + j] : 0.0f;
    }
    float edge[kImgs];                    // column kPadTile, rows 0 .. kPadTile
#pragma unroll
    for (int q = 0; q < kImgs; ++q) edge[q] = 0.0f;
    if (tid <= kPadTile) {
        const int i = i0 + tid, j = j0 + kPadTile;
        const bool in = i < N && j < N;
        edge[0] = in ? to_f(x[(size_t)i * N + j]) : 0.0f;
        if (kImgs == 2) edge[kImgs - 1] = in ? x2[(size_t)i * N + j] : 0.0f;
    }
#pragma unroll
    for (int q = 0; q < kImgs; ++q) {
#pragma unroll
        for (int t = 0; t < kPasses; ++t)
            if (ty + t * kPadRows <= kPadTile) tile[q][ty + t * kPadRows][tx] = v[q][t];
        if (tid <= kPadTile) tile[q][tid][kPadTile] = edge[q];
    }
    __syncthreads();
    auto entry = [&](int r0, int c0, int r1, int c1) -> E {
        if constexpr (kImgs == 2) {
            const float2 a = lerp_pair(tile[0][r0][c0], tile[0][r1][c1]);
            const float2 b = lerp_pair(tile[1][r0][c0], tile[1][r1][c1]);
            return make_float4(a.x, a.y, b.x, b.y);
        } else {
            return lerp_pair(tile[0][r0][c0], tile[0][r1][c1]);
        }
    };
    // both copies written along their own rows, so each warp store is one
    // contiguous run of 32 entries
    for (int r = threadIdx.y; r < kPadTile; r += kPadRows) {
        const int i = i0 + r, j = j0 + threadIdx.x;
        if (i < N && j < N) xp[(size_t)i * stride + j] = entry(r, threadIdx.x, r, threadIdx.x + 1);
    }
    for (int c = threadIdx.y; c < kPadTile; c += kPadRows) {
        const int j = j0 + c, i = i0 + threadIdx.x;
        if (i < N && j < N) xtp[(size_t)j * stride + i] = entry(threadIdx.x, c, threadIdx.x + 1, c);
    }
    // entry j = -1 of each row: (0 - x[0], x[0])
    auto first = [&](size_t p) -> E {
        if constexpr (kImgs == 2) {
            const float2 a = lerp_pair(0.0f, to_f(x[p])), b = lerp_pair(0.0f, x2[p]);
            return make_float4(a.x, a.y, b.x, b.y);
        } else {
            return lerp_pair(0.0f, to_f(x[p]));
        }
    };
    if (bx == 0)
        for (int r = threadIdx.y * blockDim.x + threadIdx.x; r < kPadTile; r += blockDim.x * blockDim.y) {
            const int i = i0 + r;
            if (i < N) xp[(size_t)i * stride - 1] = first((size_t)i * N);
        }
    if (by == 0)
        for (int c = threadIdx.y * blockDim.x + threadIdx.x; c < kPadTile; c += blockDim.x * blockDim.y) {
            const int j = j0 + c;
            if (j < N) xtp[(size_t)j * stride - 1] = first((size_t)j);
        }
}

// xc: the image is column xc of a basis (x + col_offset(xc)), or x itself.
template <int kImgs, typename T>
__global__ void pad_pairs_kernel(const T *__restrict__ x, ColRef xc, const float *__restrict__ x2,
                                 void *__restrict__ pad, int N, int stride, int border) {
    pad_pairs_block<kImgs, T>(x + col_offset(xc), x2, pad, N, stride, border, blockIdx.x, blockIdx.y);
}

__device__ __forceinline__ float fx_frac(long long U) {
    // top 24 bits of the 40-bit fraction of a 24.40 value, in [0, 1)
    const unsigned f24 = (unsigned)((unsigned long long)U >> (CTG_FX_BITS - 24)) & 0xFFFFFFu;
    return (float)f24 * (1.0f / 16777216.0f);
}

// floor(u) by the round-down magic-number add, for two positions at once in
// packed FP32 pairs: t = u + M rounded down (M = 1.5 * 2^23, so the low
// mantissa bits of t hold floor(u) for 0 <= u < 2^22) and f = u - (t - M),
// exactly the scalar sequence per position, with half the instructions.
__device__ __forceinline__ void floor_frac2(float u0, float u1, float &t0, float &t1, float &f0,
                                            float &f1) {
    asm("{\n\t.reg .b64 u, m, t, f;\n\t"
        "mov.b64 u, {%4, %5};\n\t"
        "mov.b64 m, {%6, %6};\n\t"
        "add.rm.f32x2 t, u, m;\n\t"
        "sub.rn.f32x2 f, t, m;\n\t"
        "sub.rn.f32x2 f, u, f;\n\t"
        "mov.b64 {%0, %1}, t;\n\t"
        "mov.b64 {%2, %3}, f;\n\t}"
        : "=f"(t0), "=f"(t1), "=f"(f0), "=f"(f1)
        : "f"(u0), "f"(u1), "f"(12582912.0f));
}

__device__ __forceinline__ float one_plus_frac(unsigned lo) {
    // 1 + (top 23 bits of a 32-bit fraction), exactly, in [1, 2): the low
    // word of (0x7F : lo) >> 9 is 0x3F800000 | (lo >> 9), one funnel shift
    return __uint_as_float(__funnelshift_r(lo, 0x7Fu, 9));
}

constexpr int kFwdAngles = kBatchFwdAngles;   // angles per batched block, one per warp
constexpr int kFwdDepth = 12;   // image loads in flight per lane (a multiple of 4): with warps of
                                // 4 angles, 12 measured 7% faster than 8 and 3% faster than 16 at
                                // 512^2 (with one angle per warp, 8 was 10% faster than 4)
constexpr int kBatchFwdDepth = 8;   // the batched kernel holds both clamp variants: 8 needs no spills
constexpr int kFwdDepth2 = 8;       // two images: 8 interleaved loads (16 B each) in flight per lane

// b[a * n_det + d] = scale_a * sum_t lerp(img_a[t, .], u(d, t)).
// A block holds kAngles consecutive angles; each warp holds kSplit of them
// and 32 / kSplit adjacent rays of each, and walks the union of its rays'
// chords' row ranges in lockstep, so each load instruction reads one image
// row per angle.  The walk position is 32.32 fixed point with the row stride
// folded into the step, so its high word is the staged-pair index and its
// low word the interpolation weight.  A lane outside its own chord reads
// zero pairs in the border (or, with kClamp, a clamped index into the
// 2-pair border).  The walk starts at a multiple of 4 and step s adds into
// accumulator s % 4, so a ray's sum depends on its own chord only: every
// block shape, warp layout and load depth gives the same result bit for
// bit.  kSplit > 1 needs the host's check (ctg_forward_split_safe) that
// every lane stays inside the border.
// kImgs = 2 projects two images staged interleaved (pad_pairs_block<2>) in
// the same walk, b from the first and b2 from the second: each ray's two
// sums are the ones the one-image kernel gives for each image alone.
template <bool kClamp, int kAngles = kFwdAngles, int kSplit = 1, int kDepth = kFwdDepth, int kImgs = 1>
__device__ __forceinline__ void joseph_forward_block(const void *__restrict__ pad_in, int N,
                                                     int stride, int border, int n_angles,
                                                     int n_det, const FwdAngle *__restrict__ tab,
                                                     float *__restrict__ b, float *__restrict__ b2,
                                                     int bx, int by) {
    using E = typename std::conditional<kImgs == 2, float4, float2>::type;
    constexpr int kRays = 32 / kSplit;
    const int lane = threadIdx.x & 31;
    const int a = by * kAngles + (threadIdx.x >> 5) * kSplit + lane / kRays;
    const bool live = a < n_angles;
    if (!__any_sync(0xffffffffu, live)) return;      // whole warp past the last angle
    const int d = bx * kRays + lane % kRays;
    const FwdAngle t = tab[live ? a : n_angles - 1];
    const E *img = static_cast<const E *>(pad_in) + (t.row_driven ? 0 : (size_t)N * stride) + border;

    // this ray's steps whose taps can touch the image (-1 < u < N), with a
    // one-step margin; rays past the last detector or angle take an empty
    // range
    int lo = N, hi = -1;
    if (live && d < n_det) {
        const float u0 = fmaf((float)d, t.pf, t.qf);
        if (fabsf(t.df) > 1e-20f) {
            const float r1 = (-1.0f - u0) / t.df, r2 = ((float)N - u0) / t.df;
            const float tlo = fmaxf(fminf(r1, r2), -2.0f), thi = fminf(fmaxf(r1, r2), (float)N + 1);
            lo = max(0, (int)floorf(tlo) - 1);
            hi = min(N - 1, (int)ceilf(thi) + 1);
        } else if (u0 > -2.0f && u0 < (float)N + 1.0f) {
            lo = 0;
            hi = N - 1;
        }
    }
    const int wlo = __reduce_min_sync(0xffffffffu, lo) & ~3;
    const int whi = __reduce_max_sync(0xffffffffu, hi);
    // acc[i] for image 1, acc[4 + i] for image 2, i = step mod 4
    float acc[4 * kImgs];
#pragma unroll
    for (int i = 0; i < 4 * kImgs; ++i) acc[i] = 0.0f;
    auto add = [&](float *ac, float mw, const E &p) {
        if constexpr (kImgs == 2) {
            ac[0] = fmaf(mw, p.y, ac[0] + p.x);
            ac[4] = fmaf(mw, p.w, ac[4] + p.z);
        } else {
            ac[0] = fmaf(mw, p.y, ac[0] + p.x);
        }
    };
    if (!kClamp) {
        const long long Ds = t.D + ((long long)stride << CTG_FXF_BITS);
        long long U = t.Q + (long long)d * t.P + (long long)wlo * Ds;
        int s = wlo;
        for (; s + kDepth - 1 <= whi; s += kDepth) {
            E p[kDepth];
            float mw[kDepth];
#pragma unroll
            for (int i = 0; i < kDepth; ++i) {
                p[i] = __ldg(img + (int)(U >> CTG_FXF_BITS));
                mw[i] = one_plus_frac((unsigned)U);
                U += Ds;
            }
#pragma unroll
            for (int i = 0; i < kDepth; ++i) add(acc + (i & 3), mw[i], p[i]);
        }
        for (; s + 3 <= whi; s += 4) {
            E p[4];
            float mw[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                p[i] = __ldg(img + (int)(U >> CTG_FXF_BITS));
                mw[i] = one_plus_frac((unsigned)U);
                U += Ds;
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) add(acc + i, mw[i], p[i]);
        }
        // at most three steps left, s a multiple of 4
#pragma unroll
        for (int i = 0; i < 3; ++i)
            if (s + i <= whi) {
                const E pa = __ldg(img + (int)(U >> CTG_FXF_BITS));
                add(acc + i, one_plus_frac((unsigned)U), pa);
                U += Ds;
            }
    } else {
        long long U = t.Q + (long long)d * t.P + (long long)wlo * t.D;
        for (int s = wlo; s <= whi; ++s) {
            const int j = min(max((int)(U >> CTG_FXF_BITS), -2), N);
            const E pa = __ldg(img + (size_t)s * stride + j);
            add(acc, one_plus_frac((unsigned)U), pa);
            U += t.D;
        }
    }
    if (live && d < n_det) {
        b[(size_t)a * n_det + d] = ((acc[0] + acc[2]) + (acc[1] + acc[3])) * t.scale;
        if constexpr (kImgs == 2) b2[(size_t)a * n_det + d] = ((acc[4] + acc[6]) + (acc[5] + acc[7])) * t.scale;
    }
}

// One block per (ray group bx, angle group by), on a 1-D grid of gx * gy
// blocks; block i takes tile order[i] = by * gx + bx (order NULL: tile i),
// so that the dispatch order can put the longest walks first.
template <bool kClamp, int kAngles, int kSplit, int kImgs>
__global__ void __launch_bounds__(32 * kAngles / kSplit)
joseph_forward_kernel(const void *__restrict__ pad, int N, int stride, int border,
                      int n_angles, int n_det, const FwdAngle *__restrict__ tab,
                      float *__restrict__ b, float *__restrict__ b2, const int *__restrict__ order,
                      int gx) {
    const int tile = order ? order[blockIdx.x] : (int)blockIdx.x;
    joseph_forward_block<kClamp, kAngles, kSplit, kImgs == 2 ? kFwdDepth2 : kFwdDepth, kImgs>(
        pad, N, stride, border, n_angles, n_det, tab, b, b2, tile % gx, tile / gx);
}

// ---------------------------------------------------------------------------
// Pixel-driven back projection.  A thread-block cluster of kBSplit CTAs owns
// a 32 x 32 pixel tile; each CTA (256 threads, four rows each) sums a
// contiguous quarter of the angles.  For a chunk of angles a CTA stages, per
// angle, the detector window that the tile projects onto as
// (b[d], b[d+1] - b[d]) pairs in shared memory (zeros outside the
// detector), so the inner loop has no bounds test and one 8-byte shared
// load per interpolation.  The tile origin's detector position is formed
// exactly in fixed point; each pixel adds a small float offset.  The CTAs'
// partial sums are then added through distributed shared memory in rank
// order (deterministic, no atomics), each CTA finishing a quarter of the
// tile's rows.
constexpr int kBT = 32;          // tile side
constexpr int kBRows = 4;        // rows per thread (threads: 32 x 8), batched launches
constexpr int kBThreads = 256;
constexpr int kBRowsTiled = 4;   // rows per thread of the single launch (8 rows and 32 x 4
                                 // threads measured 6 % slower: fewer warps to hide latency)
template <int kRows>
__host__ __device__ constexpr int back_threads() { return kBT * (kBT / kRows); }
constexpr int kBChunk = 32;      // angles staged per pass
constexpr int kBSplit = 4;       // CTAs per cluster = angle groups per tile

// Body of one CTA of the back-projection cluster for tile (bx, by).  Every
// CTA of a cluster must call it (it synchronises the cluster twice).
// kModel: 0 the pixel-driven B (linear interpolation on the detector);
// 1 the matched A^T and 2 the thresholded B_tau, whose weights for the two
// nearest bins d0, d0 + 1 of a pixel at detector position d0 + f are
// scale * max(0, 1 - f inv_w) and scale * max(0, 1 - (1 - f) inv_w) (terms
// below thr dropped for 2).  The staged pairs are (b[d], b[d+1] - b[d]) for
// the pixel-driven B and (b[d], b[d+1]) for the others.
// kRows: pixel rows per thread, kBT / kRows row threads per column (rows
// di, di + kBT / kRows, ...): more rows per thread spread the per-angle
// setup over more interpolations.
template <typename T, int kModel = 0, int kChunk = kBChunk, int kRows = kBRows>
__device__ __forceinline__ void pixel_back_tile(const T *__restrict__ b, int N, int n_angles,
                                                int n_det, const BackAngle *__restrict__ tab,
                                                int W, const float *__restrict__ add,
                                                float *__restrict__ x, int bx, int by,
                                                const MatchedAngle *__restrict__ mt = nullptr,
                                                float thr = 0.0f) {
    constexpr int kThr = back_threads<kRows>(), kRT = kBT / kRows;
    static_assert(kChunk <= kThr && kRows % 2 == 0 && kRows <= 16, "back tile shape");
    extern __shared__ float2 s_pairs[];               // kChunk * W pairs
    __shared__ float4 s_par[kChunk];                  // cf, sf, u0' (window-relative), origin
    __shared__ float4 s_wt[kModel ? kChunk : 1];      // scale, scale inv_w, scale - scale inv_w
    __shared__ float s_part[kRows][kThr];             // this CTA's partial sums
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();       // == blockIdx.z
    const int j0 = bx * kBT, i0 = by * kBT;
    const int dj = threadIdx.x & 31, di = threadIdx.x >> 5;   // di in [0, kRT)
    const float fdj = (float)dj, fdi = (float)di;
    const int per = (n_angles + kBSplit - 1) / kBSplit;
    const int a_begin = min(n_angles, rank * per), a_end = min(n_angles, a_begin + per);
    float acc[kRows];
#pragma unroll
    for (int r = 0; r < kRows; ++r) acc[r] = 0.f;
    for (int a0 = a_begin; a0 < a_end; a0 += kChunk) {
        const int na = min(kChunk, a_end - a0);
        __syncthreads();
        if (threadIdx.x < na) {
            const BackAngle t = tab[a0 + threadIdx.x];
            const long long U0 = t.C + (long long)j0 * t.COS + (long long)i0 * t.SIN;
            const int dbase = (int)(U0 >> CTG_FX_BITS);
            const float phi = fx_frac(U0);
            // lowest detector position over the tile (a corner), minus one
            const float umin = phi + fminf(0.f, (kBT - 1) * t.cf) + fminf(0.f, (kBT - 1) * t.sf);
            const int org = dbase + (int)floorf(umin) - 1;
            s_par[threadIdx.x] = make_float4(t.cf, t.sf, (float)(dbase - org) + phi,
                                             __int_as_float(org));
            if constexpr (kModel != 0) {
                const MatchedAngle m = mt[a0 + threadIdx.x];
                const float sw = m.scale * m.inv_w;
                s_wt[threadIdx.x] = make_float4(m.scale, sw, m.scale - sw, 0.0f);
            }
        }
        __syncthreads();
        // one warp per staged angle, lanes along its window (no division)
        for (int k = threadIdx.x >> 5; k < na; k += kThr / 32) {
            const int org = __float_as_int(s_par[k].w);
            const T *brow = b + (size_t)(a0 + k) * n_det;
            float2 *dst = s_pairs + k * W;
            for (int w = threadIdx.x & 31; w < W; w += 32) {
                const int dd = org + w;
                const float v0 = ((unsigned)dd < (unsigned)n_det) ? to_f(__ldg(brow + dd)) : 0.0f;
                const float v1 = ((unsigned)(dd + 1) < (unsigned)n_det) ? to_f(__ldg(brow + dd + 1)) : 0.0f;
                dst[w] = kModel == 0 ? make_float2(v0, v1 - v0) : make_float2(v0, v1);
            }
        }
        __syncthreads();
        // shared address of an angle's window less the magic number's bits
        // times 8, so that row r's pair is at sb + 8 t_r (32-bit wrap-around)
        // with t_r the bits of u_r + M: one shift-add per pair address
        unsigned sb = (unsigned)__cvta_generic_to_shared(s_pairs) - (0x4B400000u << 3);
#pragma unroll 2
        for (int k = 0; k < na; ++k, sb += 8u * (unsigned)W) {
            const float4 p = s_par[k];
            const float du = (float)kRT * p.y;
            float u[kRows];
            u[0] = fmaf(fdi, p.y, fmaf(fdj, p.x, p.z));
#pragma unroll
            for (int r = 1; r < kRows; ++r) u[r] = u[r - 1] + du;
            float tt[kRows], ff[kRows];
#pragma unroll
            for (int r = 0; r < kRows; r += 2) floor_frac2(u[r], u[r + 1], tt[r], tt[r + 1], ff[r], ff[r + 1]);
            float4 wt = make_float4(0.f, 0.f, 0.f, 0.f);
            if constexpr (kModel != 0) wt = s_wt[k];
#pragma unroll
            for (int r = 0; r < kRows; ++r) {
                const float f = ff[r];
                const float2 pr =
                    *static_cast<const float2 *>(__cvta_shared_to_generic(sb + (__float_as_uint(tt[r]) << 3)));
                if constexpr (kModel == 0) {
                    acc[r] += fmaf(f, pr.y, pr.x);
                } else {
                    float w0 = fmaxf(0.0f, fmaf(-f, wt.y, wt.x));
                    float w1 = fmaxf(0.0f, fmaf(f, wt.y, wt.z));
                    if constexpr (kModel == 2) {
                        w0 = w0 >= thr ? w0 : 0.0f;
                        w1 = w1 >= thr ? w1 : 0.0f;
                    }
                    acc[r] = fmaf(w0, pr.x, fmaf(w1, pr.y, acc[r]));
                }
            }
        }
    }
#pragma unroll
    for (int r = 0; r < kRows; ++r) s_part[r][threadIdx.x] = acc[r];
    cluster.sync();
    // this CTA finishes row groups rank, rank + kBSplit, ... of every
    // thread: pixel rows di + kRT r
#pragma unroll
    for (int r = rank; r < kRows; r += kBSplit) {
        float sum = 0.0f;
#pragma unroll
        for (int q = 0; q < kBSplit; ++q)
            sum += cluster.map_shared_rank(&s_part[r][0], q)[threadIdx.x];
        const int i = i0 + di + kRT * r, j = j0 + dj;
        if (i < N && j < N) {
            const size_t p = (size_t)i * N + j;
            x[p] = add ? sum + add[p] : sum;
        }
    }
    cluster.sync();   // peers' shared memory must outlive the reads above
}

// bc: the input is column bc of a basis (b + col_offset(bc)), or b itself.
template <typename T, int kChunk>
__global__ void __cluster_dims__(1, 1, kBSplit) __launch_bounds__(back_threads<kBRowsTiled>())
pixel_back_tiled_kernel(const T *__restrict__ b, ColRef bc, int N, int n_angles, int n_det,
                        const BackAngle *__restrict__ tab, int W, const float *__restrict__ add,
                        float *__restrict__ x) {
    pixel_back_tile<T, 0, kChunk, kBRowsTiled>(b + col_offset(bc), N, n_angles, n_det, tab, W, add, x,
                                               blockIdx.x, blockIdx.y);
}

// A^T (kModel 1) or B_tau (kModel 2) with the tiled design above.
template <typename T, int kModel>
__global__ void __cluster_dims__(1, 1, kBSplit) __launch_bounds__(kBThreads)
matched_back_tiled_kernel(const T *__restrict__ b, ColRef bc, int N, int n_angles, int n_det,
                          const BackAngle *__restrict__ tab, int W, const MatchedAngle *__restrict__ mt,
                          float thr, const float *__restrict__ add, float *__restrict__ x) {
    pixel_back_tile<T, kModel>(b + col_offset(bc), N, n_angles, n_det, tab, W, add, x, blockIdx.x, blockIdx.y,
                               mt, thr);
}

// Generic pixel-driven back projection (any detector pitch): 32 x 8 tiles,
// taps read through L1 with bounds tests.
constexpr int kBX = 32, kBY = 8, kAChunk = 256;

template <typename T>
__global__ void __launch_bounds__(kBX *kBY)
pixel_back_kernel(const T *__restrict__ b, ColRef bc, int N, int n_angles, int n_det,
                  const BackAngle *__restrict__ tab, const float *__restrict__ add,
                  float *__restrict__ x) {
    __shared__ float4 sp[kAChunk];
    b += col_offset(bc);
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
        const T *brow = b + (size_t)a0 * n_det;
#pragma unroll 4
        for (int k = 0; k < na; ++k, brow += n_det) {
            const float4 p = sp[k];
            const float u = fmaf(fdi, p.y, fmaf(fdj, p.x, p.z));
            const float fl = floorf(u);
            const int dd = __float_as_int(p.w) + (int)fl;
            const float f = u - fl;
            const float v0 = ((unsigned)dd < (unsigned)n_det) ? to_f(__ldg(brow + dd)) : 0.0f;
            const float v1 = ((unsigned)(dd + 1) < (unsigned)n_det) ? to_f(__ldg(brow + dd + 1)) : 0.0f;
            acc += fmaf(f, v1 - v0, v0);
        }
    }
    const int i = i0 + di, j = j0 + dj;
    if (i < N && j < N) {
        const size_t p = (size_t)i * N + j;
        x[p] = add ? acc + add[p] : acc;
    }
}

// ---- batched kernels: one launch for the same phase of every instance ----
// map[blockIdx.x] = (instance, local block of that instance's own grid).

// One instance's tile with its back projector.
template <typename T, int kChunk>
__device__ __forceinline__ void batch_back_tile(const BatchInst &I, const T *in, int bx, int by) {
    if (I.back_model == CTG_BACK_MATCHED)
        pixel_back_tile<T, 1, kChunk>(in, I.N, I.n_angles, I.n_det, I.back, I.back_window, nullptr, I.vn, bx,
                                      by, I.mt, 0.0f);
    else if (I.back_model == CTG_BACK_THRESHOLD)
        pixel_back_tile<T, 2, kChunk>(in, I.N, I.n_angles, I.n_det, I.back, I.back_window, nullptr, I.vn, bx,
                                      by, I.mt, I.back_thr);
    else
        pixel_back_tile<T, 0, kChunk>(in, I.N, I.n_angles, I.n_det, I.back, I.back_window, nullptr, I.vn, bx,
                                      by);
}

// T = float: AB instances with an FP32 basis (back-projecting w_k) and all
// BA instances (back-projecting the FP32 t_k = A w_k); T = BF16 / FP16: AB
// instances whose basis is stored in that type (their own launch, so that
// each kernel holds the tile code of one input type only).
// kChunk: angles staged per pass (the result does not depend on it).
template <typename T, int kChunk>
__global__ void __cluster_dims__(1, 1, kBSplit) __launch_bounds__(kBThreads)
batch_back_kernel(const BatchInst *__restrict__ insts, const int2 *__restrict__ map) {
    const int2 mp = map[blockIdx.x];
    const BatchInst &I = insts[mp.x];
    // the same decision in all CTAs of the cluster (they share blockIdx.x)
    if (!I.active) return;
    constexpr int kType = std::is_same<T, __nv_bfloat16>::value ? CTG_BASIS_BF16
                          : std::is_same<T, __half>::value      ? CTG_BASIS_FP16
                                                                : CTG_BASIS_FP32;
    if (I.variant == CTG_AB && I.wtype != kType) return;
    if (I.variant == CTG_BA && kType != CTG_BASIS_FP32) return;
    const int tx = (I.N + kBT - 1) / kBT;
    const T *in;
    if constexpr (kType == CTG_BASIS_FP32)
        in = I.variant == CTG_AB ? static_cast<const float *>(I.W) + (size_t)(I.k - 1) * I.ldw : I.vm;
    else
        in = static_cast<const T *>(I.W) + (size_t)(I.k - 1) * I.ldw;
    batch_back_tile<T, kChunk>(I, in, mp.y % tx, mp.y / tx);
}

// AB: stage t = B w_k (in vn); BA: stage w_{k+1} (stored type), with x_k
// interleaved for the DP stop.
template <int kVariant>
__global__ void batch_pad_kernel(const BatchInst *__restrict__ insts, const int2 *__restrict__ map) {
    const int2 mp = map[blockIdx.x];
    const BatchInst &I = insts[mp.x];
    if (!I.active) return;
    const int tx = (I.N + kPadTile - 1) / kPadTile, bx = mp.y % tx, by = mp.y / tx;
    if (kVariant == CTG_AB) {
        pad_pairs_block<1, float>(I.vn, nullptr, I.pad, I.N, I.pad_stride, I.pad_border, bx, by);
        return;
    }
    const size_t off = (size_t)I.k * I.ldw;
    const bool two = I.target > 0.0;
    auto stage = [&](auto *w) {
        if (two) pad_pairs_block<2>(w + off, I.x, I.pad2, I.N, I.pad_stride, I.pad_border, bx, by);
        else pad_pairs_block<1>(w + off, nullptr, I.pad, I.N, I.pad_stride, I.pad_border, bx, by);
    };
    if (I.wtype == CTG_BASIS_BF16) stage(static_cast<const __nv_bfloat16 *>(I.W));
    else if (I.wtype == CTG_BASIS_FP16) stage(static_cast<const __half *>(I.W));
    else stage(static_cast<const float *>(I.W));
}

// kAngles, kSplit: the forward shape of the launch (one for all instances).
// AB: q = A t (into vm); BA: t_{k+1} = A w_{k+1} (into vm) and, with the DP
// stop, A x_k (into vr) from the two-image staging.
template <int kVariant, int kAngles, int kSplit>
__global__ void __launch_bounds__(32 * kAngles / kSplit)
batch_forward_kernel(const BatchInst *__restrict__ insts, const int2 *__restrict__ map) {
    const int2 mp = map[blockIdx.x];
    const BatchInst &I = insts[mp.x];
    if (!I.active) return;
    const int bxn = (I.n_det + 32 / kSplit - 1) / (32 / kSplit);
    const int bx = mp.y % bxn, by = mp.y / bxn;
    if (kVariant == CTG_BA && I.target > 0.0) {
        if (I.pad_clamp)
            joseph_forward_block<true, kAngles, kSplit, kBatchFwdDepth, 2>(
                I.pad2, I.N, I.pad_stride, I.pad_border, I.n_angles, I.n_det, I.fwd, I.vm, I.vr, bx, by);
        else
            joseph_forward_block<false, kAngles, kSplit, kBatchFwdDepth, 2>(
                I.pad2, I.N, I.pad_stride, I.pad_border, I.n_angles, I.n_det, I.fwd, I.vm, I.vr, bx, by);
        return;
    }
    if (I.pad_clamp)
        joseph_forward_block<true, kAngles, kSplit, kBatchFwdDepth>(I.pad, I.N, I.pad_stride, I.pad_border,
                                                                    I.n_angles, I.n_det, I.fwd, I.vm, nullptr,
                                                                    bx, by);
    else
        joseph_forward_block<false, kAngles, kSplit, kBatchFwdDepth>(I.pad, I.N, I.pad_stride, I.pad_border,
                                                                     I.n_angles, I.n_det, I.fwd, I.vm, nullptr,
                                                                     bx, by);
}

}  // namespace

int ctg_back_tiles(int N) {
    const int t = (N + kBT - 1) / kBT;
    return t * t;
}
int ctg_pad_tiles(int N) {
    const int t = (N + kPadTile - 1) / kPadTile;
    return t * t;
}
int ctg_fwd_blocks(int n_angles, int n_det) {
    static_assert(kFwdShapeAngles[0] == kFwdAngles && kFwdShapeSplit[0] == 1, "batched forward shape");
    static_assert(kFwdShapeSplit[kBatchFwdSplitShape] > 1, "batched split shape");
    return ctg_fwd_shape_blocks(0, n_angles, n_det);
}
// largest window the tiled back projector can stage in shared memory
int ctg_back_window_max() { return (40 * 1024) / (int)(sizeof(float2) * kBChunk); }

namespace {
template <int kChunk>
void batch_back_t(BatchInst *insts, const int2 *map, int nblocks, int max_window, cudaStream_t st, int wtype) {
    const size_t smem = sizeof(float2) * (size_t)kChunk * max_window;
    const dim3 grid(nblocks, 1, kBSplit);
    if (wtype == CTG_BASIS_BF16)
        batch_back_kernel<__nv_bfloat16, kChunk><<<grid, kBThreads, smem, st>>>(insts, map);
    else if (wtype == CTG_BASIS_FP16)
        batch_back_kernel<__half, kChunk><<<grid, kBThreads, smem, st>>>(insts, map);
    else
        batch_back_kernel<float, kChunk><<<grid, kBThreads, smem, st>>>(insts, map);
}
}  // namespace

bool ctg_batch_back_chunk_ok(int chunk, int max_window) {
    return (chunk == 16 || chunk == 32 || chunk == 64) && (size_t)chunk * max_window * sizeof(float2) <= 40 * 1024;
}

cudaError_t ctg_batch_back(BatchInst *insts, const int2 *map, int nblocks, int max_window,
                           cudaStream_t st, int wtype, int chunk) {
    if (nblocks <= 0) return cudaSuccess;
    if (!ctg_batch_back_chunk_ok(chunk, max_window)) chunk = kBChunk;
    if (chunk == 16) batch_back_t<16>(insts, map, nblocks, max_window, st, wtype);
    else if (chunk == 64) batch_back_t<64>(insts, map, nblocks, max_window, st, wtype);
    else batch_back_t<kBChunk>(insts, map, nblocks, max_window, st, wtype);
    return cudaGetLastError();
}

cudaError_t ctg_batch_pad(BatchInst *insts, const int2 *map, int nblocks, int variant, cudaStream_t st) {
    if (nblocks <= 0) return cudaSuccess;
    if (variant == CTG_AB) batch_pad_kernel<CTG_AB><<<nblocks, dim3(kPadTile, kPadRows), 0, st>>>(insts, map);
    else batch_pad_kernel<CTG_BA><<<nblocks, dim3(kPadTile, kPadRows), 0, st>>>(insts, map);
    return cudaGetLastError();
}

namespace {
template <int kVariant>
void batch_forward_t(BatchInst *insts, const int2 *map, int nblocks, cudaStream_t st, int shape) {
    constexpr int SA = kFwdShapeAngles[kBatchFwdSplitShape], SS = kFwdShapeSplit[kBatchFwdSplitShape];
    if (shape == kBatchFwdSplitShape)
        batch_forward_kernel<kVariant, SA, SS><<<nblocks, 32 * SA / SS, 0, st>>>(insts, map);
    else
        batch_forward_kernel<kVariant, kFwdAngles, 1><<<nblocks, 32 * kFwdAngles, 0, st>>>(insts, map);
}
}  // namespace

cudaError_t ctg_batch_forward(BatchInst *insts, const int2 *map, int nblocks, int variant, cudaStream_t st,
                              int shape) {
    if (nblocks <= 0) return cudaSuccess;
    if (variant == CTG_AB) batch_forward_t<CTG_AB>(insts, map, nblocks, st, shape);
    else batch_forward_t<CTG_BA>(insts, map, nblocks, st, shape);
    return cudaGetLastError();
}

int ctg_back_window(const BackAngle *host_tab, int n_angles) {
    // detector span of a 32 x 32 tile at any angle, plus the floor/ceil and
    // second-tap margins
    double span = 0.0;
    for (int a = 0; a < n_angles; ++a) {
        const double s = (kBT - 1) * ((double)fabsf(host_tab[a].cf) + (double)fabsf(host_tab[a].sf));
        if (s > span) span = s;
    }
    return (int)ceil(span) + 4;
}

cudaError_t ctg_launch_pad(const void *x, int dtype, float2 *pad, int N, const PadLayout &pl,
                           cudaStream_t st, ColRef xc) {
    dim3 grid((N + kPadTile - 1) / kPadTile, (N + kPadTile - 1) / kPadTile), block(kPadTile, kPadRows);
    switch (dtype) {
        case CTG_BASIS_FP32:
            pad_pairs_kernel<1><<<grid, block, 0, st>>>(static_cast<const float *>(x), xc, nullptr, pad, N,
                                                        pl.stride, pl.border);
            break;
        case CTG_BASIS_BF16:
            pad_pairs_kernel<1><<<grid, block, 0, st>>>(static_cast<const __nv_bfloat16 *>(x), xc, nullptr,
                                                        pad, N, pl.stride, pl.border);
            break;
        case CTG_BASIS_FP16:
            pad_pairs_kernel<1><<<grid, block, 0, st>>>(static_cast<const __half *>(x), xc, nullptr, pad, N,
                                                        pl.stride, pl.border);
            break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t ctg_launch_pad2(const void *x, int dtype, ColRef xc, const float *x2, float4 *pad2, int N,
                            const PadLayout &pl, cudaStream_t st) {
    dim3 grid((N + kPadTile - 1) / kPadTile, (N + kPadTile - 1) / kPadTile), block(kPadTile, kPadRows);
    switch (dtype) {
        case CTG_BASIS_FP32:
            pad_pairs_kernel<2><<<grid, block, 0, st>>>(static_cast<const float *>(x), xc, x2, pad2, N,
                                                        pl.stride, pl.border);
            break;
        case CTG_BASIS_BF16:
            pad_pairs_kernel<2><<<grid, block, 0, st>>>(static_cast<const __nv_bfloat16 *>(x), xc, x2, pad2,
                                                        N, pl.stride, pl.border);
            break;
        case CTG_BASIS_FP16:
            pad_pairs_kernel<2><<<grid, block, 0, st>>>(static_cast<const __half *>(x), xc, x2, pad2, N,
                                                        pl.stride, pl.border);
            break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

namespace {

template <int kAngles, int kSplit, int kImgs>
void launch_forward_t(const void *pad, int N, const PadLayout &pl, int n_angles, int n_det,
                      const FwdAngle *tab, float *b, float *b2, cudaStream_t st, const int *order) {
    constexpr int kRays = 32 / kSplit;
    const int gx = (n_det + kRays - 1) / kRays, gy = (n_angles + kAngles - 1) / kAngles;
    const unsigned grid = (unsigned)gx * (unsigned)gy;
    if (pl.clamp)
        joseph_forward_kernel<true, kAngles, kSplit, kImgs><<<grid, 32 * kAngles / kSplit, 0, st>>>(
            pad, N, pl.stride, pl.border, n_angles, n_det, tab, b, b2, order, gx);
    else
        joseph_forward_kernel<false, kAngles, kSplit, kImgs><<<grid, 32 * kAngles / kSplit, 0, st>>>(
            pad, N, pl.stride, pl.border, n_angles, n_det, tab, b, b2, order, gx);
}

template <int kImgs>
void launch_forward_shape(int shape, const void *pad, int N, const PadLayout &pl, int n_angles, int n_det,
                          const FwdAngle *tab, float *b, float *b2, cudaStream_t st, const int *order) {
    switch (shape) {
        case 1: launch_forward_t<4, 1, kImgs>(pad, N, pl, n_angles, n_det, tab, b, b2, st, order); break;
        case 2: launch_forward_t<8, 4, kImgs>(pad, N, pl, n_angles, n_det, tab, b, b2, st, order); break;
        case 3: launch_forward_t<16, 4, kImgs>(pad, N, pl, n_angles, n_det, tab, b, b2, st, order); break;
        default: launch_forward_t<8, 1, kImgs>(pad, N, pl, n_angles, n_det, tab, b, b2, st, order); break;
    }
}

// walk range [lo, hi] of ray d of angle t, as joseph_forward_block
// estimates it (host arithmetic; may differ from the device's by a step)
void ray_range(const FwdAngle &t, int N, int d, int &lo, int &hi) {
    const float u0 = (float)d * t.pf + t.qf;
    lo = N;
    hi = -1;
    if (std::fabs(t.df) > 1e-20f) {
        const float r1 = (-1.0f - u0) / t.df, r2 = ((float)N - u0) / t.df;
        const float tlo = std::max(std::min(r1, r2), -2.0f);
        const float thi = std::min(std::max(r1, r2), (float)N + 1);
        lo = std::max(0, (int)std::floor(tlo) - 1);
        hi = std::min(N - 1, (int)std::ceil(thi) + 1);
    } else if (u0 > -2.0f && u0 < (float)N + 1.0f) {
        lo = 0;
        hi = N - 1;
    }
}

// union walk range of rays d0 .. d1 - 1 of angle t: a ray's range ends are
// clamped linear functions of d, so the first and last ray give it (all
// rays when the walk is parallel to the detector, D = 0)
void group_range(const FwdAngle &t, int N, int d0, int d1, int &wlo, int &whi) {
    const bool all = !(std::fabs(t.df) > 1e-20f);
    wlo = N;
    whi = -1;
    for (int d = d0; d < d1; d += (all || d + 1 == d1) ? 1 : d1 - 1 - d) {
        int lo, hi;
        ray_range(t, N, d, lo, hi);
        wlo = std::min(wlo, lo);
        whi = std::max(whi, hi);
    }
}

}  // namespace

cudaError_t ctg_launch_forward(const float2 *pad, int N, const PadLayout &pl, int n_angles,
                               int n_det, const FwdAngle *tab, float *b, cudaStream_t st,
                               int shape, const int *order) {
    // every ray's sum depends on its own chord only, so the result depends
    // on neither the shape nor the dispatch order
    launch_forward_shape<1>(shape, pad, N, pl, n_angles, n_det, tab, b, nullptr, st, order);
    return cudaGetLastError();
}

cudaError_t ctg_launch_forward2(const float4 *pad2, int N, const PadLayout &pl, int n_angles, int n_det,
                                const FwdAngle *tab, float *b, float *b2, cudaStream_t st, int shape,
                                const int *order) {
    launch_forward_shape<2>(shape, pad2, N, pl, n_angles, n_det, tab, b, b2, st, order);
    return cudaGetLastError();
}

int ctg_fwd_shape_blocks(int shape, int n_angles, int n_det) {
    const int rays = 32 / kFwdShapeSplit[shape], angles = kFwdShapeAngles[shape];
    return ((n_det + rays - 1) / rays) * ((n_angles + angles - 1) / angles);
}

void ctg_forward_order(const FwdAngle *tab, int N, int n_angles, int n_det, int shape,
                       std::vector<int> &order) {
    const int A = kFwdShapeAngles[shape], S = kFwdShapeSplit[shape], R = 32 / S;
    const int gx = (n_det + R - 1) / R, gy = (n_angles + A - 1) / A;
    // work of a tile: the steps of its warps' lockstep walks plus a fixed
    // cost per warp
    std::vector<long long> cost((size_t)gx * gy, 0);
    for (int a0 = 0; a0 < n_angles; a0 += S)
        for (int bx = 0; bx < gx; ++bx) {
            int wlo = N, whi = -1;
            for (int a = a0; a < std::min(n_angles, a0 + S); ++a) {
                int lo, hi;
                group_range(tab[a], N, bx * R, std::min(n_det, bx * R + R), lo, hi);
                wlo = std::min(wlo, lo);
                whi = std::max(whi, hi);
            }
            cost[(size_t)(a0 / A) * gx + bx] += (whi >= wlo ? whi - (wlo & ~3) + 1 : 0) + 16;
        }
    order.resize(cost.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost[x] > cost[y]; });
}

bool ctg_forward_split_safe(const FwdAngle *tab, int N, int n_angles, int n_det, const PadLayout &pl,
                            int split) {
    if (pl.clamp) return true;                      // indices are clamped
    const int R = 32 / split;
    for (int a0 = 0; a0 < n_angles; a0 += split)
        for (int d0 = 0; d0 < n_det; d0 += R) {
            int wlo = N, whi = -1;
            for (int a = a0; a < std::min(n_angles, a0 + split); ++a) {
                int lo, hi;
                group_range(tab[a], N, d0, std::min(n_det, d0 + R), lo, hi);
                wlo = std::min(wlo, lo);
                whi = std::max(whi, hi);
            }
            if (whi < wlo) continue;
            // the device's range may differ from this estimate by a step:
            // check a wider one
            const int s_lo = std::max(0, (wlo & ~3) - 4), s_hi = std::min(N - 1, whi + 4);
            // a lane's column is affine in its ray d, so the warp's first and
            // last ray of each angle are its extremes (lanes past the last
            // angle walk with the last angle's table)
            for (int a = a0; a < a0 + split; ++a) {
                const FwdAngle &t = tab[std::min(n_angles - 1, a)];
                for (const long long d : {(long long)d0, (long long)(d0 + R - 1)})
                    for (const long long s : {(long long)s_lo, (long long)s_hi}) {
                        const long long j = (t.Q + d * t.P + s * t.D) >> CTG_FXF_BITS;
                        if (j < -pl.border || j > N - 1 + pl.border) return false;
                    }
            }
        }
    return true;
}

namespace {

template <typename T, int kChunk>
void launch_back_tiled(const T *b, ColRef bc, int N, int n_angles, int n_det, const BackAngle *tab,
                       int window, const float *add, float *x, cudaStream_t st) {
    const size_t smem = sizeof(float2) * (size_t)kChunk * window;
    const dim3 grid((N + kBT - 1) / kBT, (N + kBT - 1) / kBT, kBSplit);
    pixel_back_tiled_kernel<T, kChunk><<<grid, back_threads<kBRowsTiled>(), smem, st>>>(b, bc, N, n_angles, n_det, tab,
                                                                      window, add, x);
}

// back_chunk: angles staged per pass (16, 32 or 64).  Each pixel sums its
// angles in the same order whatever the chunk, so the result does not
// depend on it.
template <typename T>
cudaError_t launch_back_t(const T *b, ColRef bc, int N, int n_angles, int n_det, const BackAngle *tab,
                          int window, const float *add, float *x, cudaStream_t st, int back_chunk) {
    const size_t bytes_per_angle = sizeof(float2) * (size_t)window;
    if (window > 0 && back_chunk == 64 && 64 * bytes_per_angle <= 40 * 1024) {
        launch_back_tiled<T, 64>(b, bc, N, n_angles, n_det, tab, window, add, x, st);
    } else if (window > 0 && back_chunk == 16 && 16 * bytes_per_angle <= 40 * 1024) {
        launch_back_tiled<T, 16>(b, bc, N, n_angles, n_det, tab, window, add, x, st);
    } else if (window > 0 && kBChunk * bytes_per_angle <= 40 * 1024) {
        launch_back_tiled<T, kBChunk>(b, bc, N, n_angles, n_det, tab, window, add, x, st);
    } else {
        dim3 grid((N + kBX - 1) / kBX, (N + kBY - 1) / kBY);
        pixel_back_kernel<T><<<grid, dim3(kBX, kBY), 0, st>>>(b, bc, N, n_angles, n_det, tab, add, x);
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_matched_tiled_t(const T *b, ColRef bc, int N, int n_angles, int n_det,
                                   const BackAngle *tab, int window, const MatchedAngle *mt, float thr,
                                   const float *add, float *x, cudaStream_t st) {
    const size_t smem = sizeof(float2) * (size_t)kBChunk * window;
    const dim3 grid((N + kBT - 1) / kBT, (N + kBT - 1) / kBT, kBSplit);
    if (thr > 0.0f)
        matched_back_tiled_kernel<T, 2><<<grid, kBThreads, smem, st>>>(b, bc, N, n_angles, n_det, tab,
                                                                       window, mt, thr, add, x);
    else
        matched_back_tiled_kernel<T, 1><<<grid, kBThreads, smem, st>>>(b, bc, N, n_angles, n_det, tab,
                                                                       window, mt, thr, add, x);
    return cudaGetLastError();
}

}  // namespace

cudaError_t ctg_launch_back_matched_tiled(const void *b, int dtype, int N, int n_angles, int n_det,
                                          const BackAngle *tab, int window, const MatchedAngle *mt,
                                          float thr, const float *add, float *x, cudaStream_t st,
                                          ColRef bc) {
    if (window <= 0 || window > ctg_back_window_max()) return cudaErrorInvalidValue;
    switch (dtype) {
        case CTG_BASIS_FP32:
            return launch_matched_tiled_t(static_cast<const float *>(b), bc, N, n_angles, n_det, tab, window,
                                          mt, thr, add, x, st);
        case CTG_BASIS_BF16:
            return launch_matched_tiled_t(static_cast<const __nv_bfloat16 *>(b), bc, N, n_angles, n_det, tab,
                                          window, mt, thr, add, x, st);
        case CTG_BASIS_FP16:
            return launch_matched_tiled_t(static_cast<const __half *>(b), bc, N, n_angles, n_det, tab, window,
                                          mt, thr, add, x, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t ctg_launch_back(const void *b, int dtype, int N, int n_angles, int n_det,
                            const BackAngle *tab, int window, const float *add, float *x,
                            cudaStream_t st, int back_chunk, ColRef bc) {
    switch (dtype) {
        case CTG_BASIS_FP32:
            return launch_back_t(static_cast<const float *>(b), bc, N, n_angles, n_det, tab, window, add, x, st,
                                 back_chunk);
        case CTG_BASIS_BF16:
            return launch_back_t(static_cast<const __nv_bfloat16 *>(b), bc, N, n_angles, n_det, tab, window,
                                 add, x, st, back_chunk);
        case CTG_BASIS_FP16:
            return launch_back_t(static_cast<const __half *>(b), bc, N, n_angles, n_det, tab, window, add, x,
                                 st, back_chunk);
        default: return cudaErrorInvalidValue;
    }
}
