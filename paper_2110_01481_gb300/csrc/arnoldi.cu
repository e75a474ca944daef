// Arnoldi orthogonalisation of the Krylov basis (paper Sec. 2, algorithm
// box: h_{i,k} = q_k^T w_i, q_k -= h_{i,k} w_i, h_{k+1,k} = ||q_k||,
// w_{k+1} = q_k / h_{k+1,k}), done as classical Gram-Schmidt applied twice
// (CGS2), which equals the paper's MGS loop in exact arithmetic but needs
// three sweeps over W instead of k dependent ones:
//   pass 1  h1 = W^T q,                ||q||^2      (one read of W)
//   pass 2  q -= W h1,  h2 = W^T q,    ||q1||^2     (two reads of W)
//   pass 3  q -= W h2,  w_{k+1} = q / ||q||         (one read of W)
// with ||q||^2 = ||q1||^2 - ||h2||^2 after pass 3 (exact for orthonormal W;
// h2 is at the rounding level of ||q1|| after the first pass, so nothing
// cancels), h_{1:k,k} = h1 + h2, h_{k+1,k} = ||q||.
// Each pass is one launch: every block reduces its slice with warp shuffles
// into per-block partials, and the last block to finish (atomic ticket, no
// waiting) sums the partials in a fixed order (compensated FP32 pairs,
// FP64 results), so results are deterministic run to run.
#include <atomic>

#include "loop_device.cuh"

namespace {

// Vectors per load batch: BYTES of basis data in flight per thread (128
// where registers are short, as in the one-launch step; 256 in the separate
// passes, measured 6-8 % faster at k = 100).
template <typename T, int E, int BYTES = 128>
__host__ __device__ constexpr int batch_vectors() {
    return (int)(BYTES / (4 * sizeof(T) * E)) > 0 ? (int)(BYTES / (4 * sizeof(T) * E)) : 1;
}

// acc += sum_j c_j V_j over this thread's E float4 groups, loads issued in
// batches of JB vectors so that 128 bytes per thread are in flight.
template <typename T, int E>
__device__ __forceinline__ void accumulate_batched(const T *__restrict__ V, int64_t ldv, int k,
                                                   const float *c, int64_t g0, int64_t L,
                                                   float4 (&acc)[E]) {
    constexpr int JB = batch_vectors<T, E>();
    for (int j0 = 0; j0 < k; j0 += JB) {
        typename RawOf<T>::type w[JB][E];
#pragma unroll
        for (int jj = 0; jj < JB; ++jj) {
            const T *Vj = V + (size_t)min(j0 + jj, k - 1) * ldv;   // see cgs_pass_kernel
#pragma unroll
            for (int e = 0; e < E; ++e) w[jj][e] = ldraw(Vj, g0 + (int64_t)e * kThreads, L);
        }
#pragma unroll
        for (int jj = 0; jj < JB; ++jj) {
            const float cj = (j0 + jj < k) ? c[j0 + jj] : 0.f;
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const float4 wf = cvt4<T>(w[jj][e]);
                acc[e].x = fmaf(cj, wf.x, acc[e].x);
                acc[e].y = fmaf(cj, wf.y, acc[e].y);
                acc[e].z = fmaf(cj, wf.z, acc[e].z);
                acc[e].w = fmaf(cj, wf.w, acc[e].w);
            }
        }
    }
}

// qv -= sum_j c_j W_j over this thread's slice.  Loads are issued in batches
// of JB vectors before any of them is used, so each thread keeps 128 bytes of
// HBM reads outstanding (8 float4 of an FP32 basis, 16 half-width groups of a
// 16-bit one).  Past the last vector the load repeats vector k-1 (a cache
// hit) and its coefficient / dot is dropped, so every load of the batch is
// unconditional and issued before any use.
template <typename T, int E, int BYTES = 128>
__device__ __forceinline__ void update_slice(const T *__restrict__ W, int64_t ldw, int k,
                                             const float *s_coef, int64_t g0, int64_t L,
                                             float4 (&qv)[E]) {
    constexpr int JB = batch_vectors<T, E, BYTES>();
    for (int j0 = 0; j0 < k; j0 += JB) {
        typename RawOf<T>::type w[JB][E];
#pragma unroll
        for (int jj = 0; jj < JB; ++jj) {
            const T *Wj = W + (size_t)min(j0 + jj, k - 1) * ldw;
#pragma unroll
            for (int e = 0; e < E; ++e) w[jj][e] = ldraw(Wj, g0 + (int64_t)e * kThreads, L);
        }
#pragma unroll
        for (int jj = 0; jj < JB; ++jj) {
            const float c = (j0 + jj < k) ? s_coef[j0 + jj] : 0.f;
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const float4 wf = cvt4<T>(w[jj][e]);
                qv[e].x = fmaf(-c, wf.x, qv[e].x);
                qv[e].y = fmaf(-c, wf.y, qv[e].y);
                qv[e].z = fmaf(-c, wf.z, qv[e].z);
                qv[e].w = fmaf(-c, wf.w, qv[e].w);
            }
        }
    }
}

// Warp sums of W_j^T qv (j < k) into s_w[warp * nred + j] and, with NORM,
// of qv^T qv into s_w[warp * nred + k]; same load batching as update_slice.
// REV visits the vectors from the last to the first.  The separate passes
// alternate the direction of their sweeps over W (pass 1's dots last to
// first, pass 2's update first to last and its dots last to first, the
// last update first to last), so each sweep starts on the vectors that the
// one before read last, which a basis larger than L2 still finds there.
// The order of the vectors does not change any sum.
template <typename T, int E, bool NORM, bool REV = false, int BYTES = 128>
__device__ __forceinline__ void dots_slice(const T *__restrict__ W, int64_t ldw, int k, int64_t g0,
                                           int64_t L, const float4 (&qv)[E], float *s_w, int nred) {
    constexpr int JB = batch_vectors<T, E, BYTES>();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int t0 = 0; t0 < k; t0 += JB) {
        typename RawOf<T>::type w[JB][E];
#pragma unroll
        for (int jj = 0; jj < JB; ++jj) {
            const int t = min(t0 + jj, k - 1);
            const T *Wj = W + (size_t)(REV ? k - 1 - t : t) * ldw;
#pragma unroll
            for (int e = 0; e < E; ++e) w[jj][e] = ldraw(Wj, g0 + (int64_t)e * kThreads, L);
        }
#pragma unroll
        for (int jj = 0; jj < JB; ++jj) {
            float sj = 0.f;
#pragma unroll
            for (int e = 0; e < E; ++e) sj += dot4(cvt4<T>(w[jj][e]), qv[e]);
            sj = warp_sum(sj);
            const int t = t0 + jj;
            if (lane == 0 && t < k) s_w[warp * nred + (REV ? k - 1 - t : t)] = sj;
        }
    }
    if (NORM) {
        float s = 0.f;
#pragma unroll
        for (int e = 0; e < E; ++e) s += dot4(qv[e], qv[e]);
        s = warp_sum(s);
        if (lane == 0) s_w[warp * nred + k] = s;
    }
}

// One CGS2 pass over a slice of E float4 groups per thread.
//   UPDATE: q -= sum_j coef_j W_j (coef: k doubles)
//   DOTS:   red_out[j] = W_j^T q (after the update)      j < k
//   NORM:   red_out[DOTS ? k : 0] = q^T q (after the update)
template <typename T, int E, bool UPDATE, bool DOTS, bool NORM>
__device__ __forceinline__ void cgs_pass_body(const T *__restrict__ W, int64_t ldw, int k,
                                              float *__restrict__ q, int64_t L,
                                              const double *__restrict__ coef,
                                              float *__restrict__ partials,
                                              unsigned *__restrict__ counter,
                                              double *__restrict__ red_out, int blk, int G) {
    extern __shared__ float smem[];
    const int tid = threadIdx.x;
    const int nred = (DOTS ? k : 0) + (NORM ? 1 : 0);
    float *s_coef = smem;                       // k floats (UPDATE)
    float *s_w = smem + (UPDATE ? k : 0);       // kWarps * nred floats
    if (UPDATE)
        for (int j = tid; j < k; j += kThreads) s_coef[j] = (float)coef[j];
    const int64_t g0 = (int64_t)blk * kThreads * E + tid;
    float4 qv[E];
#pragma unroll
    for (int e = 0; e < E; ++e) qv[e] = ld4_rw(q, g0 + (int64_t)e * kThreads, L);
    if (UPDATE) {
        __syncthreads();
        update_slice<T, E, 256>(W, ldw, k, s_coef, g0, L, qv);
#pragma unroll
        for (int e = 0; e < E; ++e) st4(q, g0 + (int64_t)e * kThreads, L, qv[e]);
    }
    if (DOTS) {
        dots_slice<T, E, NORM, true, 256>(W, ldw, k, g0, L, qv, s_w, nred);
    } else if (NORM) {
        float s = 0.f;
#pragma unroll
        for (int e = 0; e < E; ++e) s += dot4(qv[e], qv[e]);
        s = warp_sum(s);
        if ((tid & 31) == 0) s_w[(tid >> 5) * nred] = s;
    }
    block_reduce_finish(s_w, nred, partials, counter, red_out, blk, G);
}

// kdev: k read on the device (a step of a captured solver loop), or NULL.
template <typename T, int E, bool UPDATE, bool DOTS, bool NORM>
__global__ void __launch_bounds__(kThreads, 2)
cgs_pass_kernel(const T *__restrict__ W, int64_t ldw, int k, const int *__restrict__ kdev,
                float *__restrict__ q, int64_t L, const double *__restrict__ coef,
                float *__restrict__ partials, unsigned *__restrict__ counter,
                double *__restrict__ red_out) {
    if (kdev) k = *kdev;
    cgs_pass_body<T, E, UPDATE, DOTS, NORM>(W, ldw, k, q, L, coef, partials, counter, red_out,
                                            blockIdx.x, gridDim.x);
}

// Every block sums the partial rows [row0, row0 + nrows) of all blocks in
// one fixed order (compensated FP32 pairs, FP64 results), so all blocks
// hold identical coefficients.
__device__ __forceinline__ void reduce_rows(const float *__restrict__ partials, int row0, int nrows,
                                            int G, int Gp, double *out) {
    sum_partial_rows(partials, row0, nrows, G, Gp, out);
}

__device__ __forceinline__ void write_rows(const float *s_w, int nred, int row0, float *partials,
                                           int Gp, int blk) {
    for (int j = threadIdx.x; j < nred; j += kThreads) {
        float t = 0.f;
        for (int w = 0; w < kWarps; ++w) t += s_w[w * nred + j];
        partials[(size_t)(row0 + j) * Gp + blk] = t;
    }
}

// Grid-wide barrier for a launch whose blocks are all resident at once,
// with a bounded wait: thread 0 of each block adds one arrival to *count
// and waits until `target` arrivals are in (target = barrier index x grid
// size, so one counter serves successive barriers).  After spin_limit polls
// (about 100 ns apart) it gives up: it sets *err and returns false, as does
// every block that finds *err set while it waits, so no block waits for
// ever.  Returns true when the barrier completed.
__device__ __forceinline__ bool grid_barrier(unsigned *count, unsigned target, long long spin_limit,
                                             int *err) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(count, 1u);
        int ok = 1;
        long long spins = 0;
        for (;;) {
            unsigned v;
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(count) : "memory");
            if (v >= target) break;
            int e;
            asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(e) : "l"(err) : "memory");
            if (e != 0 || ++spins > spin_limit) {
                atomicOr(err, 1);
                ok = 0;
                break;
            }
            __nanosleep(100);
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// The three CGS2 passes and the scaling as one launch, for small k, where
// four separate launches are bound by their latency rather than by the
// basis reads.  The launch must keep every block resident (the host checks
// the occupancy and launches it cooperatively); the passes are separated by
// bounded grid barriers (grid_barrier), so a block that is not scheduled
// makes the others give up with *err set instead of waiting for ever.  The
// slice of q stays in registers across the passes; each pass writes its
// per-block partial sums to its own rows of the partials ([0, k] pass 1,
// [k+1, 2k] pass 2, so no block overwrites rows another block may still be
// reading), and after the barrier every block sums the partials of all
// blocks in the same fixed order (compensated FP32 pairs), so all blocks
// hold identical coefficients and the result is deterministic.
// Step: k, w_out and h_out as given, or (kdev set, a step of a captured
// solver loop) k = *kdev, w_out = column k of W and h_out = column k of H
// (leading dimension ldh).  bar[0] counts barrier arrivals (zero at launch;
// the last block to leave sets it back to zero); on a timeout h_out[0..k]
// is set to NaN.
// With giv_mode >= 0 (a step of the device-driven solver loop), block 0
// then runs the step's FP64 Givens update (loop_givens_warp) on the column it
// has just written, and, by the mode, the end of the step, so the step needs
// no launch of its own for them; its shared memory holds kcap_giv staging
// entries and the packed triangle for y_k beyond the step's own.
template <typename T, int E>
__global__ void __launch_bounds__(kThreads, 2)
cgs2_fused_kernel(const T *__restrict__ W, int64_t ldw, int k, const int *__restrict__ kdev,
                  float *__restrict__ q, int64_t L, T *__restrict__ w_out, double *__restrict__ h_out,
                  double *__restrict__ H, int64_t ldh, float *__restrict__ partials,
                  double *__restrict__ h1g, double *__restrict__ h2g, double *__restrict__ scal,
                  unsigned *__restrict__ bar, int *__restrict__ err, long long spin_limit,
                  LoopBufs lb, int giv_mode, int kcap_giv, int pack_cap) {
    if (kdev) {
        k = *kdev;
        w_out = const_cast<T *>(W) + (size_t)k * ldw;
        h_out = H + (size_t)(k - 1) * ldh;
    }
    extern __shared__ double smem_d[];
    double *s_stage = smem_d;                       // 3 kcap_giv + 1: the Givens staging
    double *s_pack = s_stage + (giv_mode >= 0 ? 3 * kcap_giv + 1 : 0);   // packed R for y_k
    double *s_h1 = s_pack + (giv_mode >= 0 && (giv_mode & kGivY) ? pack_cap * (pack_cap + 1) / 2 : 0);
    double *s_h2 = s_h1 + (k + 1);                  // k + 2: h2, ||q1||^2, then ||q2||^2
    float *s_c = reinterpret_cast<float *>(s_h2 + (k + 2));   // k coefficients
    float *s_w = s_c + k;                           // kWarps * (k + 1)
    const int tid = threadIdx.x, blk = blockIdx.x, G = gridDim.x, Gp = padded_grid(G);
    const unsigned nbar = k > 0 ? 2u : 1u;
    const int64_t g0 = (int64_t)blk * kThreads * E + tid;
    float4 qv[E];
#pragma unroll
    for (int e = 0; e < E; ++e) qv[e] = ld4_rw(q, g0 + (int64_t)e * kThreads, L);
    // pass 1: h1 = W^T q, ||q||^2
    dots_slice<T, E, true, true>(W, ldw, k, g0, L, qv, s_w, k + 1);
    __syncthreads();
    write_rows(s_w, k + 1, 0, partials, Gp, blk);
    bool ok = grid_barrier(bar, (unsigned)G, spin_limit, err);
    double nrm2 = 0.0;
    if (ok) {
        reduce_rows(partials, 0, k + 1, G, Gp, s_h1);
        __syncthreads();
        nrm2 = s_h1[k];
    }
    if (ok && k > 0) {
        // pass 2: q1 = q - W h1; h2 = W^T q1, ||q1||^2
        for (int j = tid; j < k; j += kThreads) s_c[j] = (float)s_h1[j];
        __syncthreads();
        update_slice<T, E>(W, ldw, k, s_c, g0, L, qv);
        dots_slice<T, E, true, true>(W, ldw, k, g0, L, qv, s_w, k + 1);
        __syncthreads();
        write_rows(s_w, k + 1, k + 1, partials, Gp, blk);
        ok = grid_barrier(bar, 2u * (unsigned)G, spin_limit, err);
        if (ok) {
            reduce_rows(partials, k + 1, k + 1, G, Gp, s_h2);
            __syncthreads();
            // pass 3: q2 = q1 - W h2.  With W orthonormal, ||q2||^2 = ||q1||^2 -
            // ||h2||^2 exactly; h2 is at the rounding level of ||q1|| after the
            // first pass, so the difference loses nothing, and the step needs no
            // third grid-wide reduction.  Every block forms it in the same order.
            for (int j = tid; j < k; j += kThreads) s_c[j] = (float)s_h2[j];
            if (tid < 32) {
                // ||h2||^2 once per block (FP64 issues slowly): lane-strided
                // sums, then a fixed xor tree, the same bits in every block
                double t = 0.0;
                for (int j = tid; j < k; j += 32) t = fma(s_h2[j], s_h2[j], t);
                t = warp_sum_d(t);
                if (tid == 0) s_h2[k + 1] = fmax(0.0, s_h2[k] - t);
            }
            __syncthreads();
            update_slice<T, E>(W, ldw, k, s_c, g0, L, qv);
            nrm2 = s_h2[k + 1];
        }
    }
    if (!ok) {
        // gave up at a barrier: leave q and W alone and mark the column; the
        // Givens update takes the NaN column for a breakdown, and the step's
        // end reports the timeout
        for (int j = tid; j <= k; j += kThreads) h_out[j] = __longlong_as_double(0x7ff8000000000000LL);
        if (giv_mode >= 0 && blk == 0) {
            __syncthreads();
            if (tid < 32) loop_givens_warp(lb, k, h_out, 0.0, giv_mode, s_pack, pack_cap,
                                           k <= kcap_giv ? s_stage : nullptr);
        }
        return;
    }
    // w_{k+1} = q / ||q||; q keeps the orthogonalised vector.  One FP64
    // reciprocal square root (a dependent division and a square root each
    // take ~650 cycles on GB300), and ||q|| = nrm2 rnorm
    const double rnorm = nrm2 > 0.0 ? rsqrt(nrm2) : 0.0;
    const float inv = (float)rnorm;
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int64_t g = g0 + (int64_t)e * kThreads;
        st4(q, g, L, qv[e]);
        stw4(w_out, g, L, make_float4(qv[e].x * inv, qv[e].y * inv, qv[e].z * inv, qv[e].w * inv));
    }
    if (blk == 0) {
        for (int j = tid; j < k; j += kThreads) {
            h_out[j] = s_h1[j] + s_h2[j];
            h1g[j] = s_h1[j];
            h2g[j] = s_h2[j];
        }
        if (tid == 0) {
            h_out[k] = nrm2 * rnorm;
            h1g[k] = s_h1[k];
            scal[0] = s_h1[k];
            scal[1] = nrm2;
        }
    }
    // the last block out resets the barrier counter for the next launch
    // (every block has read k by now: it passed both barriers)
    if (tid == 0 && atomicAdd(bar, 1u) == (nbar + 1u) * (unsigned)G - 1u) atomicExch(bar, 0u);
    if (giv_mode >= 0 && blk == 0) {
        __syncthreads();                            // the column is written
        if (tid < 32) loop_givens_warp(lb, k, h_out, s_h1[k], giv_mode, s_pack, pack_cap,
                                       k <= kcap_giv ? s_stage : nullptr);
    }
}

// w_out = q / sqrt(nrm2) (0 if nrm2 == 0); block 0 also assembles the
// Hessenberg column h_out[0..k-1] = h1 + h2, h_out[k] = sqrt(nrm2).
// q and w_out may be the same vector (FP32 storage only).
template <typename T>
__device__ __forceinline__ void scale_body(const float *q, const double *__restrict__ nrm2,
                                           T *w_out, int64_t L, int k,
                                           const double *__restrict__ h1,
                                           const double *__restrict__ h2,
                                           double *__restrict__ h_out, int blk, int nblk) {
    const double nn = *nrm2;
    const double rnorm = nn > 0.0 ? rsqrt(nn) : 0.0;
    const float inv = (float)rnorm;
    const int64_t L4 = (L + 3) / 4;
    for (int64_t g = (int64_t)blk * blockDim.x + threadIdx.x; g < L4;
         g += (int64_t)nblk * blockDim.x) {
        float4 v = ld4_rw(q, g, L);
        v.x *= inv; v.y *= inv; v.z *= inv; v.w *= inv;
        stw4(w_out, g, L, v);
    }
    if (h_out != nullptr && blk == 0) {
        for (int j = threadIdx.x; j < k; j += blockDim.x) h_out[j] = h1[j] + h2[j];
        if (threadIdx.x == 0) h_out[k] = nn * rnorm;
    }
}

// The last CGS2 pass and the scaling in one sweep: q -= sum_j h2_j W_j, then
// w_out = q / ||q||, with ||q||^2 = h2[k] - ||h2[0..k-1]||^2 (h2[k] =
// ||q1||^2 from the second pass; exact for orthonormal W, and h2 is at the
// rounding level of ||q1||, so nothing cancels).  Block 0 writes the
// Hessenberg column h_out[0..k] and *nrm2_out.
template <typename T, int E>
__device__ __forceinline__ void update_scale_body(const T *__restrict__ W, int64_t ldw, int k,
                                                  float *__restrict__ q, int64_t L,
                                                  const double *__restrict__ h1,
                                                  const double *__restrict__ h2, T *w_out,
                                                  double *__restrict__ h_out,
                                                  double *__restrict__ nrm2_out, int blk) {
    extern __shared__ float smem[];
    float *s_coef = smem;                                   // k floats
    __shared__ double s_nn;
    const int tid = threadIdx.x;
    for (int j = tid; j < k; j += kThreads) s_coef[j] = (float)h2[j];
    if (tid < 32) {
        // ||h2||^2 in a fixed order: lane-strided sums, then a fixed tree
        double t = 0.0;
        for (int j = tid; j < k; j += 32) t = fma(h2[j], h2[j], t);
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (tid == 0) s_nn = fmax(0.0, h2[k] - t);
    }
    __syncthreads();
    const double nn = s_nn;
    const double rnorm = nn > 0.0 ? rsqrt(nn) : 0.0;
    const float inv = (float)rnorm;
    const int64_t g0 = (int64_t)blk * kThreads * E + tid;
    float4 qv[E];
#pragma unroll
    for (int e = 0; e < E; ++e) qv[e] = ld4_rw(q, g0 + (int64_t)e * kThreads, L);
    update_slice<T, E, 256>(W, ldw, k, s_coef, g0, L, qv);
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int64_t g = g0 + (int64_t)e * kThreads;
        st4(q, g, L, qv[e]);
        stw4(w_out, g, L, make_float4(qv[e].x * inv, qv[e].y * inv, qv[e].z * inv, qv[e].w * inv));
    }
    if (blk == 0) {
        if (h_out != nullptr) {
            for (int j = tid; j < k; j += kThreads) h_out[j] = h1[j] + h2[j];
            if (tid == 0) h_out[k] = nn * rnorm;
        }
        if (tid == 0) *nrm2_out = nn;
    }
}

// kdev set: k = *kdev, w_out = column k of W, h_out = column k of H.
template <typename T, int E>
__global__ void __launch_bounds__(kThreads, 2)
update_scale_kernel(const T *__restrict__ W, int64_t ldw, int k, const int *__restrict__ kdev,
                    float *__restrict__ q, int64_t L, const double *__restrict__ h1,
                    const double *__restrict__ h2, T *w_out, double *__restrict__ h_out,
                    double *__restrict__ H, int64_t ldh, double *__restrict__ nrm2_out) {
    if (kdev) {
        k = *kdev;
        w_out = const_cast<T *>(W) + (size_t)k * ldw;
        h_out = H + (size_t)(k - 1) * ldh;
    }
    update_scale_body<T, E>(W, ldw, k, q, L, h1, h2, w_out, h_out, nrm2_out, blockIdx.x);
}

template <typename T>
__global__ void scale_kernel(const float *q, const double *__restrict__ nrm2, T *w_out, int64_t L,
                             int k, const double *__restrict__ h1, const double *__restrict__ h2,
                             double *__restrict__ h_out) {
    scale_body<T>(q, nrm2, w_out, L, k, h1, h2, h_out, blockIdx.x, gridDim.x);
}

// out = base + sum_j y_j W_j (j < k; k = *kdev + koff when kdev is set).
template <typename T, int E>
__global__ void __launch_bounds__(kThreads, 2)
gemv_kernel(const T *__restrict__ W, int64_t ldw, int k, const int *__restrict__ kdev, int koff,
            const double *__restrict__ y, const float *__restrict__ base, float *__restrict__ out,
            int64_t L) {
    extern __shared__ float s_y[];
    if (kdev) k = *kdev + koff;
    for (int j = threadIdx.x; j < k; j += kThreads) s_y[j] = (float)y[j];
    __syncthreads();
    const int64_t g0 = (int64_t)blockIdx.x * kThreads * E + threadIdx.x;
    float4 acc[E];
#pragma unroll
    for (int e = 0; e < E; ++e)
        acc[e] = base ? ld4(base, g0 + (int64_t)e * kThreads, L) : make_float4(0.f, 0.f, 0.f, 0.f);
    accumulate_batched<T, E>(W, ldw, k, s_y, g0, L, acc);
#pragma unroll
    for (int e = 0; e < E; ++e) st4(out, g0 + (int64_t)e * kThreads, L, acc[e]);
}

// out = a - c (or a), res = ||out||^2; out may be the same vector as a or c.
template <int E>
__global__ void __launch_bounds__(kThreads, 2)
sub_norm2_kernel(const float *a, const float *c, float *out, int64_t L,
                 float *__restrict__ partials,
                 unsigned *__restrict__ counter, double *__restrict__ res) {
    __shared__ float s_w[kWarps];
    const int tid = threadIdx.x;
    const int64_t g0 = (int64_t)blockIdx.x * kThreads * E + tid;
    float s = 0.f;
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int64_t g = g0 + (int64_t)e * kThreads;
        float4 v = ld4_rw(a, g, L);
        if (c) {
            const float4 w = ld4_rw(c, g, L);
            v.x -= w.x; v.y -= w.y; v.z -= w.z; v.w -= w.w;
        }
        if (out) st4(out, g, L, v);
        s += dot4(v, v);
    }
    s = warp_sum(s);
    if ((tid & 31) == 0) s_w[tid >> 5] = s;
    block_reduce_finish(s_w, 1, partials, counter, res, blockIdx.x, gridDim.x);
}

// ---- batched kernels (one launch for every instance of a batch) ----------
// E = 1 passes; map[blockIdx.x] = (instance, block of that instance).

__device__ __forceinline__ int vec_blocks_dev(long long L) {
    return (int)(((L + 3) / 4 + kThreads - 1) / kThreads);
}

// T: the basis element type of the instances in this launch's map (one
// launch per type, so that each kernel keeps the registers of its own type).
template <typename T, bool UPDATE, bool DOTS, bool NORM>
__global__ void __launch_bounds__(kThreads, 2)
batch_cgs_pass_kernel(BatchInst *__restrict__ insts, const int2 *__restrict__ map) {
    const int2 mp = map[blockIdx.x];
    BatchInst &I = insts[mp.x];
    if (!I.active) return;
    float *q = I.variant == CTG_AB ? I.vm : I.vn;
    const double *coef = UPDATE ? (DOTS ? I.h1 : I.h2) : nullptr;
    double *red_out = DOTS ? (UPDATE ? I.h2 : I.h1) : I.scal + 1;
    cgs_pass_body<T, 1, UPDATE, DOTS, NORM>(static_cast<const T *>(I.W), I.ldw, I.k, q, I.L, coef,
                                            I.partials, I.counter, red_out, mp.y, I.G);
}

// Last CGS2 pass and scaling of every instance (update_scale_body): the new
// basis vector w_{k+1}, rounded to the basis type, and Hessenberg column k.
template <typename T>
__global__ void __launch_bounds__(kThreads, 2)
batch_update_scale_kernel(BatchInst *__restrict__ insts, const int2 *__restrict__ map) {
    const int2 mp = map[blockIdx.x];
    BatchInst &I = insts[mp.x];
    if (!I.active) return;
    float *q = I.variant == CTG_AB ? I.vm : I.vn;
    update_scale_body<T, 1>(static_cast<const T *>(I.W), I.ldw, I.k, q, I.L, I.h1, I.h2,
                            static_cast<T *>(I.W) + (size_t)I.k * I.ldw,
                            I.H + (size_t)(I.k - 1) * (I.maxit + 1), I.scal + 1, mp.y);
}

// One warp per instance: FP64 Givens update of the Hessenberg least-squares
// problem with the new column (rotations kept in gc/gs, rotated column in
// R, rotated right-hand side gg), the breakdown test, and for BA with the
// discrepancy stop, y_k = R^{-1} gg.  The column and the rotations are
// staged in shared memory (all lanes load, lane 0 runs the recurrence), and
// for y_k the packed triangle when it fits (dynamic shared memory of
// pack_cap (pack_cap + 1) / 2 doubles).
constexpr int kBatchGivStage = 1024;   // = the batches' largest maxit

// The update of instance I by one warp, its column, rotations and rotated
// column staged in s_h (k + 1), s_gc, s_gs (k - 1 each).
__device__ void batch_givens_warp(BatchInst &I, double *s_h, double *s_gc, double *s_gs, double *s_pack,
                                  int pack_cap) {
    const int k = I.k, lane = threadIdx.x & 31, ldr = I.maxit;
    const double *h = I.H + (size_t)(k - 1) * (I.maxit + 1);
    double *Rk = I.R + (size_t)(k - 1) * ldr;         // column k of R
    for (int i = lane; i <= k; i += 32) s_h[i] = h[i];
    for (int i = lane; i < k - 1; i += 32) {
        s_gc[i] = I.gc[i];
        s_gs[i] = I.gs[i];
    }
    __syncwarp();
    if (lane == 0) {
        double r_prev = s_h[0];
        for (int i = 0; i < k - 1; ++i) {
            const double a = r_prev, b = s_h[i + 1];
            s_h[i] = s_gc[i] * a + s_gs[i] * b;
            r_prev = -s_gs[i] * a + s_gc[i] * b;
        }
        const double a = r_prev, b = s_h[k];
        double c, sn, rinv;
        givens_rotation(a, b, c, sn, rinv);
        I.gc[k - 1] = c;
        I.gs[k - 1] = sn;
        s_h[k - 1] = rinv;                              // R's diagonal as its reciprocal
        I.gg[k] = -sn * I.gg[k - 1];
        I.gg[k - 1] = c * I.gg[k - 1];
        I.rho = fabs(I.gg[k]);
        I.breakdown = b * b <= 1e-12 * I.h1[k];      // b <= 1e-6 ||q before CGS2|| (h1[k] its square)
    }
    __syncwarp();
    for (int i = lane; i < k; i += 32) Rk[i] = s_h[i];
    __syncwarp();
    if (I.variant == CTG_BA && I.target > 0.0) solve_y_warp(I.R, ldr, I.gg, k, I.y, s_pack, pack_cap);
}

__global__ void batch_givens_kernel(BatchInst *__restrict__ insts, int pack_cap) {
    extern __shared__ double s_pack[];
    __shared__ double s_h[kBatchGivStage + 1], s_gc[kBatchGivStage], s_gs[kBatchGivStage];
    BatchInst &I = insts[blockIdx.x];
    if (!I.active) return;
    batch_givens_warp(I, s_h, s_gc, s_gs, s_pack, pack_cap);
}

// The batched one-launch CGS2 step (as cgs2_fused_kernel) for every active
// instance of the map's launch, with each instance's Givens update in its
// block 0: E = kBatchFusedE float4 groups per thread, batch_fused_blocks(L)
// blocks per instance; the grid barriers span the whole launch (bar[0]:
// arrivals, zero at launch, reset by the last block out; *err: set by a
// wait that gave up; *spin: the polls a wait may take), and the blocks of
// inactive instances only take part in them.  Each instance's partial rows ([0, k] pass 1, [k+1, 2k+1] pass 2)
// are its own, and every block of an instance sums them in the same fixed
// order.  Shared memory for k <= kcap: Givens staging (3 kcap + 1
// doubles), the packed R for y_k (pack_cap), h1, h2, coefficients and the
// warps' partial sums.  After a timed-out barrier the block leaves with
// *err set; the round's stopping rules then end the batch.
template <typename T>
__global__ void __launch_bounds__(kThreads, 2)
batch_cgs2_fused_kernel(BatchInst *__restrict__ insts, const int2 *__restrict__ map, unsigned *__restrict__ bar,
                        int *__restrict__ err, const long long *__restrict__ spin, int kcap, int pack_cap) {
    constexpr int E = kBatchFusedE;
    const long long spin_limit = *spin;
    const int2 mp = map[blockIdx.x];
    BatchInst &I = insts[mp.x];
    const bool on = I.active != 0;
    const int k = on ? I.k : 0;
    extern __shared__ double smem_d[];
    double *s_stage = smem_d;                                        // 3 kcap + 1
    double *s_pack = s_stage + 3 * kcap + 1;                         // pack_cap (pack_cap + 1) / 2
    double *s_h1 = s_pack + pack_cap * (pack_cap + 1) / 2;           // kcap + 1
    double *s_h2 = s_h1 + kcap + 1;                                  // kcap + 2
    float *s_c = reinterpret_cast<float *>(s_h2 + kcap + 2);         // kcap
    float *s_w = s_c + kcap;                                         // kWarps (kcap + 1)
    const int tid = threadIdx.x, G = gridDim.x;
    const int Gi = batch_fused_blocks(I.L), Gpi = padded_grid(Gi);
    const T *W = static_cast<const T *>(I.W);
    float *q = I.variant == CTG_AB ? I.vm : I.vn;
    const int64_t L = I.L, ldw = I.ldw;
    const int64_t g0 = (int64_t)mp.y * kThreads * E + tid;
    float4 qv[E];
    if (on) {
#pragma unroll
        for (int e = 0; e < E; ++e) qv[e] = ld4_rw(q, g0 + (int64_t)e * kThreads, L);
        dots_slice<T, E, true, true>(W, ldw, k, g0, L, qv, s_w, k + 1);
        __syncthreads();
        write_rows(s_w, k + 1, 0, I.partials, Gpi, mp.y);
    }
    bool ok = grid_barrier(bar, (unsigned)G, spin_limit, err);
    if (on && ok) {
        reduce_rows(I.partials, 0, k + 1, Gi, Gpi, s_h1);
        __syncthreads();
        for (int j = tid; j < k; j += kThreads) s_c[j] = (float)s_h1[j];
        __syncthreads();
        update_slice<T, E>(W, ldw, k, s_c, g0, L, qv);
        dots_slice<T, E, true, true>(W, ldw, k, g0, L, qv, s_w, k + 1);
        __syncthreads();
        write_rows(s_w, k + 1, k + 1, I.partials, Gpi, mp.y);
    }
    if (ok) ok = grid_barrier(bar, 2u * (unsigned)G, spin_limit, err);
    if (!ok) return;
    if (on) {
        reduce_rows(I.partials, k + 1, k + 1, Gi, Gpi, s_h2);
        __syncthreads();
        for (int j = tid; j < k; j += kThreads) s_c[j] = (float)s_h2[j];
        if (tid < 32) {
            double t = 0.0;
            for (int j = tid; j < k; j += 32) t = fma(s_h2[j], s_h2[j], t);
            t = warp_sum_d(t);
            if (tid == 0) s_h2[k + 1] = fmax(0.0, s_h2[k] - t);
        }
        __syncthreads();
        update_slice<T, E>(W, ldw, k, s_c, g0, L, qv);
        const double nrm2 = s_h2[k + 1];
        // as in cgs2_fused_kernel: one reciprocal square root, ||q|| = nrm2 rnorm
        const double rnorm = nrm2 > 0.0 ? rsqrt(nrm2) : 0.0;
        const float inv = (float)rnorm;
        T *w_out = const_cast<T *>(W) + (size_t)k * ldw;
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int64_t g = g0 + (int64_t)e * kThreads;
            st4(q, g, L, qv[e]);
            stw4(w_out, g, L, make_float4(qv[e].x * inv, qv[e].y * inv, qv[e].z * inv, qv[e].w * inv));
        }
        if (mp.y == 0) {
            double *h_out = I.H + (size_t)(k - 1) * (I.maxit + 1);
            for (int j = tid; j < k; j += kThreads) {
                h_out[j] = s_h1[j] + s_h2[j];
                I.h1[j] = s_h1[j];
                I.h2[j] = s_h2[j];
            }
            if (tid == 0) {
                h_out[k] = nrm2 * rnorm;
                I.h1[k] = s_h1[k];
                I.scal[1] = nrm2;
            }
        }
    }
    // the last block out resets the barrier counter for the next launch
    if (tid == 0 && atomicAdd(bar, 1u) == 3u * (unsigned)G - 1u) atomicExch(bar, 0u);
    if (on && mp.y == 0) {
        __syncthreads();                            // the column is written
        if (tid < 32) batch_givens_warp(I, s_stage, s_stage + kcap + 1, s_stage + 2 * kcap + 1, s_pack, pack_cap);
    }
}

// BA with the discrepancy stop: x_k = x0 + W_k y_k into the solve's x
// (E = 1 slices; the map's local blocks cover n).
template <typename T>
__device__ __forceinline__ void batch_iterate_body(BatchInst &I, int blk, float *s_y) {
    for (int j = threadIdx.x; j < I.k; j += kThreads) s_y[j] = (float)I.y[j];
    __syncthreads();
    const int64_t g0 = (int64_t)blk * kThreads + threadIdx.x;
    float4 acc[1];
    acc[0] = I.x0 ? ld4(I.x0, g0, I.n) : make_float4(0.f, 0.f, 0.f, 0.f);
    accumulate_batched<T, 1>(static_cast<const T *>(I.W), I.ldw, I.k, s_y, g0, I.n, acc);
    st4(I.x, g0, I.n, acc[0]);
}

__global__ void __launch_bounds__(kThreads, 2)
batch_iterate_kernel(BatchInst *__restrict__ insts, const int2 *__restrict__ map) {
    extern __shared__ float s_y[];
    const int2 mp = map[blockIdx.x];
    BatchInst &I = insts[mp.x];
    if (!I.active || I.variant != CTG_BA || !(I.target > 0.0)) return;
    if (I.wtype == CTG_BASIS_BF16) batch_iterate_body<__nv_bfloat16>(I, mp.y, s_y);
    else if (I.wtype == CTG_BASIS_FP16) batch_iterate_body<__half>(I, mp.y, s_y);
    else batch_iterate_body<float>(I, mp.y, s_y);
}

// BA with the discrepancy stop: ||b - A x_k||^2 into scal[4] (A x_k in vr).
__global__ void __launch_bounds__(kThreads, 2)
batch_residual_kernel(BatchInst *__restrict__ insts, const int2 *__restrict__ map) {
    __shared__ float s_w[kWarps];
    const int2 mp = map[blockIdx.x];
    BatchInst &I = insts[mp.x];
    if (!I.active || I.variant != CTG_BA || !(I.target > 0.0)) return;
    const int64_t g = (int64_t)mp.y * kThreads + threadIdx.x;
    float4 v = ld4(I.b, g, I.m);
    const float4 w = ld4(I.vr, g, I.m);
    v.x -= w.x; v.y -= w.y; v.z -= w.z; v.w -= w.w;
    float s = warp_sum(dot4(v, v));
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = s;
    block_reduce_finish(s_w, 1, I.partials, I.counter, I.scal + 4, mp.y, vec_blocks_dev(I.m));
}

// One thread per instance: the stopping rules (Sec. 6.4), then k -> k + 1.
__global__ void batch_finish_kernel(BatchInst *__restrict__ insts, int n, int *active_count) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    BatchInst &I = insts[i];
    if (!I.active) return;
    const int k = I.k;
    const bool dp = I.target > 0.0;
    if (I.variant == CTG_BA && dp) I.resnorm = sqrt(I.scal[4]);
    I.hist[k] = (I.variant == CTG_BA && dp) ? I.resnorm : I.rho;
    int stop = -1;
    if (I.breakdown) stop = CTG_STOP_BREAKDOWN;
    else if (dp && (I.variant == CTG_AB ? I.rho : I.resnorm) <= I.target) stop = CTG_STOP_DP;
    else if (k == I.maxit) stop = CTG_STOP_MAXIT;
    if (stop >= 0) {
        I.active = 0;
        I.iters = k;
        I.stop_reason = stop;
        atomicSub(active_count, 1);
    } else {
        I.k = k + 1;
    }
}

// The stopping rules of a round inside the batch's while-loop graph, in one
// block (n <= 1024): as batch_finish_kernel, then thread 0 counts the round
// (ctl[1]) and ends the loop once no instance is active (ctl[0]) or
// max_rounds rounds have run (every instance stops by its maxit, so the
// second condition only guards the first).
__global__ void batch_finish_loop_kernel(BatchInst *__restrict__ insts, int n, int *ctl, int max_rounds,
                                         cudaGraphConditionalHandle h, cudaGraphConditionalHandle h_next,
                                         int fused_max) {
    __shared__ int s_beyond;
    if (threadIdx.x == 0) s_beyond = 0;
    __syncthreads();
    const bool timed_out = atomicAdd(&ctl[3], 0) != 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        BatchInst &I = insts[i];
        if (!I.active) continue;
        if (timed_out) {
            // a fused step gave up at a barrier: every solve stops here (the
            // host reports the timeout)
            I.active = 0;
            I.iters = I.k - 1;
            I.stop_reason = CTG_STOP_MAXIT;
            atomicSub(&ctl[0], 1);
            continue;
        }
        const int k = I.k;
        const bool dp = I.target > 0.0;
        if (I.variant == CTG_BA && dp) I.resnorm = sqrt(I.scal[4]);
        I.hist[k] = (I.variant == CTG_BA && dp) ? I.resnorm : I.rho;
        int stop = -1;
        if (I.breakdown) stop = CTG_STOP_BREAKDOWN;
        else if (dp && (I.variant == CTG_AB ? I.rho : I.resnorm) <= I.target) stop = CTG_STOP_DP;
        else if (k == I.maxit) stop = CTG_STOP_MAXIT;
        if (stop >= 0) {
            I.active = 0;
            I.iters = k;
            I.stop_reason = stop;
            atomicSub(&ctl[0], 1);
        } else {
            I.k = k + 1;
            if (fused_max > 0 && k + 1 > fused_max) s_beyond = 1;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int r = ++ctl[1];
        if (atomicAdd(&ctl[0], 0) <= 0 || r >= max_rounds || timed_out) {
            cudaGraphSetConditional(h, 0u);
            if (h_next) cudaGraphSetConditional(h_next, 0u);
        } else if (s_beyond) {
            cudaGraphSetConditional(h, 0u);
        }
    }
}

// Exit: y = R^{-1} gg for each finished instance's k (one warp each; the
// packed triangle staged in shared memory when it fits).
__global__ void batch_solve_y_kernel(BatchInst *__restrict__ insts, int pack_cap) {
    extern __shared__ double s_pack[];
    BatchInst &I = insts[blockIdx.x];
    if (I.iters > 0) solve_y_warp(I.R, I.maxit, I.gg, I.iters, I.y, s_pack, pack_cap);
}

template <typename K>
cudaError_t ensure_smem(K kernel, size_t bytes) {
    return ctg_allow_dyn_smem((const void *)kernel, bytes);
}

// k: the step's k, or (kdev set) the largest k the launch may see, which
// sizes its shared memory.
template <typename T, bool UPDATE, bool DOTS, bool NORM>
cudaError_t launch_pass(const T *W, int64_t ldw, int k, const int *kdev, float *q, int64_t L,
                        const double *coef, const RedScratch &rs, double *red_out,
                        cudaStream_t st) {
    int E;
    const int G = ctg_red_grid(L, &E);
    const int nred = (DOTS ? k : 0) + (NORM ? 1 : 0);
    const size_t smem = sizeof(float) * ((UPDATE ? k : 0) + (size_t)kWarps * nred);
    cudaError_t err = cudaSuccess;
#define CTG_PASS_CASE(EE)                                                            \
    case EE: {                                                                       \
        auto kern = cgs_pass_kernel<T, EE, UPDATE, DOTS, NORM>;                      \
        if ((err = ensure_smem(kern, smem)) != cudaSuccess) return err;              \
        kern<<<G, kThreads, smem, st>>>(W, ldw, k, kdev, q, L, coef, rs.partials,     \
                                        rs.counter, red_out);                        \
        break;                                                                       \
    }
    switch (E) {
        CTG_PASS_CASE(1)
        CTG_PASS_CASE(2)
        CTG_PASS_CASE(4)
        CTG_PASS_CASE(8)
        default: return cudaErrorInvalidValue;
    }
#undef CTG_PASS_CASE
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_update_scale(const T *W, int64_t ldw, int k, const int *kdev, double *H, int64_t ldh,
                                float *q, int64_t L, const RedScratch &rs, T *w_out, double *h_out,
                                cudaStream_t st) {
    int E;
    const int G = ctg_red_grid(L, &E);
    const size_t smem = sizeof(float) * (size_t)k;
    cudaError_t err = cudaSuccess;
#define CTG_US_CASE(EE)                                                                          \
    case EE: {                                                                                   \
        auto kern = update_scale_kernel<T, EE>;                                                  \
        if ((err = ensure_smem(kern, smem)) != cudaSuccess) return err;                          \
        kern<<<G, kThreads, smem, st>>>(W, ldw, k, kdev, q, L, rs.h1, rs.h2, w_out, h_out, H, ldh, \
                                        rs.scal + 1);                                            \
        break;                                                                                   \
    }
    switch (E) {
        CTG_US_CASE(1)
        CTG_US_CASE(2)
        CTG_US_CASE(4)
        CTG_US_CASE(8)
        default: return cudaErrorInvalidValue;
    }
#undef CTG_US_CASE
    return cudaGetLastError();
}

}  // namespace

namespace {

constexpr int kMaxDevices = 64;

// Per-device cache of an int computed once (0 = not yet known, so the
// static zero-initialisation needs no constructor); thread-safe: a race
// computes the value twice and stores the same result.
template <typename F>
int per_device_cached(std::atomic<int> (&cache)[kMaxDevices], F compute) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return compute(-1);
    }
    const int v = cache[dev].load(std::memory_order_acquire);
    if (v != 0) return v - 1;
    const int c = compute(dev);
    cache[dev].store(c + 1, std::memory_order_release);
    return c;
}

std::atomic<int> g_target_grid[kMaxDevices];

}  // namespace

int ctg_target_grid() {
    return per_device_cached(g_target_grid, [](int dev) {
        int sms = 0;
        if (dev < 0 || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            sms < 1) {
            cudaGetLastError();
            sms = 152;                      // no device: size for a GB300 (152 SMs)
        }
        return 2 * sms;
    });
}

int ctg_red_grid(int64_t L, int *E_out) {
    const int64_t L4 = (L + 3) / 4;
    const int target = ctg_target_grid();
    int E = 1;
    while (E < kMaxE && (L4 + (int64_t)kThreads * E - 1) / ((int64_t)kThreads * E) > target) E *= 2;
    int64_t G = (L4 + (int64_t)kThreads * E - 1) / ((int64_t)kThreads * E);
    if (G < 1) G = 1;
    *E_out = E;
    return (int)G;
}

static int red_grid_max(int64_t L) {
    int E;
    const int G = ctg_red_grid(L, &E);
    return G > ctg_target_grid() ? G : ctg_target_grid();
}

static size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// The fused step is used for k <= kFusedMaxK: measured at L = 522,000 it
// takes 21 / 27 / 44 / 81 / 130 / 166 us at k = 4 / 12 / 32 / 64 / 100 / 128
// against 137 us for the separate passes at k = 100 and 176 us at k = 129
// (the one launch keeps q on chip and saves two launches and a summation
// tail; at 4.19M the two are level).  A solver step that also forms y_k
// (kGivY) stages R's packed triangle in shared memory, which beyond k = 64
// would take the L1 capacity the step's own re-reads of its basis slice
// use; such steps take the one launch up to kFusedMaxKY, as do batches.
constexpr int kFusedMaxK = 128;
constexpr int kFusedMaxKY = 64;

// Partial rows: kmax + 2 for the separate passes; the fused step needs 2k + 2.
static size_t partial_rows(int kmax) {
    const size_t fused = 2 * (size_t)(kmax < kFusedMaxK ? kmax : kFusedMaxK) + 2;
    return (size_t)kmax + 2 > fused ? (size_t)kmax + 2 : fused;
}

size_t ctg_red_scratch_bytes(int64_t L, int kmax) {
    const size_t G = (size_t)padded_grid(red_grid_max(L));
    return align256(sizeof(float) * partial_rows(kmax) * G) +
           2 * align256(sizeof(double) * (size_t)(kmax + 2)) + align256(sizeof(double) * 8) +
           align256(sizeof(unsigned) * 4);
}

void ctg_red_scratch_carve(void *base, int64_t L, int kmax, RedScratch *rs) {
    char *p = static_cast<char *>(base);
    const size_t G = (size_t)padded_grid(red_grid_max(L));
    rs->partials = reinterpret_cast<float *>(p);
    rs->rows = (int)partial_rows(kmax);
    p += align256(sizeof(float) * partial_rows(kmax) * G);
    rs->h1 = reinterpret_cast<double *>(p);
    p += align256(sizeof(double) * (size_t)(kmax + 2));
    rs->h2 = reinterpret_cast<double *>(p);
    p += align256(sizeof(double) * (size_t)(kmax + 2));
    rs->scal = reinterpret_cast<double *>(p);
    p += align256(sizeof(double) * 8);
    rs->counter = reinterpret_cast<unsigned *>(p);
    rs->grid = (int)G;
    ctg_red_grid(L, &rs->E);
}

namespace {

// giv_mode >= 0: with the Givens staging (3 k + 1 doubles) and, for y_k,
// the packed triangle (loop_pack_cap(k) columns) in front
size_t fused_smem_bytes(int k, int giv_mode = -1) {
    size_t giv = 0;
    if (giv_mode >= 0) {
        giv = 3 * (size_t)k + 1;
        if (giv_mode & kGivY) giv += (size_t)loop_pack_cap(k) * (loop_pack_cap(k) + 1) / 2;
    }
    return sizeof(double) * (giv + 2 * (size_t)k + 3) + sizeof(float) * ((size_t)k + (size_t)kWarps * (k + 1));
}

int scale_blocks(int64_t L) {
    const int64_t L4 = (L + 3) / 4;
    int blocks = (int)((L4 + 255) / 256);
    if (blocks > 4 * ctg_target_grid()) blocks = 4 * ctg_target_grid();
    return blocks < 1 ? 1 : blocks;
}

// The fused step needs the 2k + 2 partial rows in the reduction scratch and
// every block of its grid resident at once (checked once per kernel
// instantiation).

template <typename T, int E>
int fused_resident_blocks() {
    static std::atomic<int> cache[kMaxDevices];
    return per_device_cached(cache, [](int dev) {
        int per_sm = 0, sms = 0;
        const size_t smem = std::max(fused_smem_bytes(kFusedMaxKY, kGivY), fused_smem_bytes(kFusedMaxK, kGivZ));
        if (dev < 0 || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            ctg_allow_dyn_smem((const void *)cgs2_fused_kernel<T, E>, smem) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cgs2_fused_kernel<T, E>, kThreads,
                                                          smem) != cudaSuccess) {
            cudaGetLastError();
            per_sm = 0;
        }
        return per_sm * sms;
    });
}

// Launches the fused step (k, w_out, h_out fixed; or from the loop step
// `ls` when ls is non-null).  *done = false when the grid cannot be
// resident at once (the caller then takes the separate passes).  With
// `cooperative` the launch asks the runtime to guarantee residency (it
// fails rather than runs otherwise); without it the occupancy check alone
// stands behind the bounded barriers.
template <typename T, int E>
cudaError_t launch_fused(const T *W, int64_t ldw, int64_t L, int k, float *q, T *w_out,
                         double *h_out, const LoopStep *ls, const RedScratch &rs, int G,
                         long long spin_limit, bool cooperative, cudaStream_t st, bool *done) {
    *done = false;
    if (G > fused_resident_blocks<T, E>()) return cudaSuccess;
    const int kcap = ls ? ls->kmax : k;
    const int giv_mode = ls && ls->lb ? ls->giv_mode : -1;
    if (giv_mode >= 0 && (giv_mode & kGivY) && kcap > kFusedMaxKY) return cudaSuccess;
    const size_t smem = fused_smem_bytes(kcap, giv_mode);
    const cudaError_t ea = ctg_allow_dyn_smem((const void *)cgs2_fused_kernel<T, E>, smem);
    if (ea != cudaSuccess) return ea;
    const LoopBufs lb = ls && ls->lb ? *ls->lb : LoopBufs{};
    const int pack_cap = loop_pack_cap(kcap);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(G);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = cooperative ? 1 : 0;
    const int *kdev = ls ? ls->k : nullptr;
    double *H = ls ? ls->H : nullptr;
    const int64_t ldh = ls ? ls->ldh : 0;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, cgs2_fused_kernel<T, E>, W, ldw, k, kdev, q, L, w_out,
                                             h_out, H, ldh, rs.partials, rs.h1, rs.h2, rs.scal,
                                             rs.counter + 1, reinterpret_cast<int *>(rs.counter + 2),
                                             spin_limit, lb, giv_mode, kcap, pack_cap);
    *done = e == cudaSuccess;
    return e;
}

// The fused step's grid: that of the separate passes (two blocks per SM),
// or with small_grid about one block per SM.  At the solvers' small k the
// basis is L2-resident and the step is bound by its grid barriers and
// summation tails, which fewer blocks shorten (512^2 AB + BA pair, 720
// angles: CGS2 phase 0.72 -> 0.69 ms per pair); at large k streaming the basis needs
// the two blocks per SM (k = 100, L = 522,000: 130 against 175 us).
constexpr int kSmallGridMaxK = 24;

static int fused_grid(int64_t L, int *E_out, bool small_grid) {
    if (!small_grid) return ctg_red_grid(L, E_out);
    const int64_t L4 = (L + 3) / 4;
    const int target = ctg_target_grid() / 2;
    int E = 1;
    while (E < kMaxE && (L4 + (int64_t)kThreads * E - 1) / ((int64_t)kThreads * E) > target) E *= 2;
    int64_t G = (L4 + (int64_t)kThreads * E - 1) / ((int64_t)kThreads * E);
    if (G < 1) G = 1;
    *E_out = E;
    return (int)G;
}

template <typename T>
cudaError_t fused_dispatch(const T *W, int64_t ldw, int64_t L, int k, float *q, T *w_out, double *h_out,
                           const LoopStep *ls, const RedScratch &rs, long long spin_limit,
                           bool cooperative, cudaStream_t st, bool *done) {
    int E;
    const int G = fused_grid(L, &E, ls && ls->small_grid);
    switch (E) {
        case 1: return launch_fused<T, 1>(W, ldw, L, k, q, w_out, h_out, ls, rs, G, spin_limit, cooperative, st, done);
        case 2: return launch_fused<T, 2>(W, ldw, L, k, q, w_out, h_out, ls, rs, G, spin_limit, cooperative, st, done);
        case 4: return launch_fused<T, 4>(W, ldw, L, k, q, w_out, h_out, ls, rs, G, spin_limit, cooperative, st, done);
        case 8: return launch_fused<T, 8>(W, ldw, L, k, q, w_out, h_out, ls, rs, G, spin_limit, cooperative, st, done);
        default: *done = false; return cudaSuccess;
    }
}

template <typename T>
cudaError_t cgs2_step_t(const T *W, int64_t ldw, int64_t L, int k, float *q, T *w_out,
                        double *h_out, const RedScratch &rs, long long spin_limit, cudaStream_t st,
                        int *nkern) {
    cudaError_t err;
    if (nkern) *nkern = k > 0 ? 3 : 2;
    if (k <= kFusedMaxK && rs.rows >= 2 * k + 2) {
        bool done = false;
        err = fused_dispatch<T>(W, ldw, L, k, q, w_out, h_out, nullptr, rs, spin_limit, true, st, &done);
        if (err != cudaSuccess) return err;
        if (done) {
            if (nkern) *nkern = 1;
            return cudaSuccess;
        }
    }
    // pass 1: h1 = W^T q and ||q_pre||^2 (h1[k]); keep the latter in scal[0]
    if ((err = launch_pass<T, false, true, true>(W, ldw, k, nullptr, q, L, nullptr, rs, rs.h1, st)) != cudaSuccess)
        return err;
    if ((err = cudaMemcpyAsync(rs.scal, rs.h1 + k, sizeof(double), cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
        return err;
    if (k > 0) {
        // pass 2: q -= W h1; h2 = W^T q, ||q||^2 (h2[k])
        if ((err = launch_pass<T, true, true, true>(W, ldw, k, nullptr, q, L, rs.h1, rs, rs.h2, st)) != cudaSuccess)
            return err;
        // q -= W h2 and w_out = q / ||q|| in one sweep; ||q||^2 -> scal[1]
        return launch_update_scale<T>(W, ldw, k, nullptr, nullptr, 0, q, L, rs, w_out, h_out, st);
    }
    if ((err = cudaMemcpyAsync(rs.scal + 1, rs.scal, sizeof(double), cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
        return err;
    scale_kernel<T><<<scale_blocks(L), 256, 0, st>>>(q, rs.scal + 1, w_out, L, k, rs.h1, rs.h2, h_out);
    return cudaGetLastError();
}

// A step of a captured solver loop (k >= 1 read on the device): the fused
// launch or the three separate passes, as ls.fused says.  ||q_pre||^2 is
// left in rs.h1[k] (not copied to scal[0], whose source would depend on k).
template <typename T>
cudaError_t cgs2_loop_t(const T *W, int64_t ldw, int64_t L, float *q, const LoopStep &ls,
                        const RedScratch &rs, long long spin_limit, bool cooperative, cudaStream_t st,
                        int *nkern) {
    cudaError_t err;
    if (ls.fused) {
        bool done = false;
        err = fused_dispatch<T>(W, ldw, L, 0, q, nullptr, nullptr, &ls, rs, spin_limit, cooperative, st, &done);
        if (nkern) *nkern = 1;
        if (err != cudaSuccess) return err;
        return done ? cudaSuccess : cudaErrorInvalidConfiguration;
    }
    if (nkern) *nkern = 3;
    if ((err = launch_pass<T, false, true, true>(W, ldw, ls.kmax, ls.k, q, L, nullptr, rs, rs.h1, st)) != cudaSuccess)
        return err;
    if ((err = launch_pass<T, true, true, true>(W, ldw, ls.kmax, ls.k, q, L, rs.h1, rs, rs.h2, st)) != cudaSuccess)
        return err;
    return launch_update_scale<T>(W, ldw, ls.kmax, ls.k, ls.H, ls.ldh, q, L, rs, nullptr, nullptr, st);
}

template <typename T>
cudaError_t gemv_t(const T *W, int64_t ldw, int64_t L, int k, const int *kdev, int koff, const double *y,
                   const float *base, float *out, cudaStream_t st) {
    int E;
    const int G = ctg_red_grid(L, &E);
    const size_t smem = sizeof(float) * (size_t)(k > 0 ? k : 1);
    cudaError_t err = cudaSuccess;
    switch (E) {
#define CTG_GEMV_CASE(EE)                                                             \
    case EE:                                                                          \
        if ((err = ensure_smem(gemv_kernel<T, EE>, smem)) != cudaSuccess) return err; \
        gemv_kernel<T, EE><<<G, kThreads, smem, st>>>(W, ldw, k, kdev, koff, y, base, out, L); \
        break;
        CTG_GEMV_CASE(1)
        CTG_GEMV_CASE(2)
        CTG_GEMV_CASE(4)
        CTG_GEMV_CASE(8)
#undef CTG_GEMV_CASE
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t ctg_cgs2_step(const void *W, int dtype, int64_t ldw, int64_t L, int k, float *q,
                          void *w_out, double *h_out, const RedScratch &rs, cudaStream_t st,
                          int *nkern, long long spin_limit) {
    switch (dtype) {
        case CTG_BASIS_FP32:
            return cgs2_step_t(static_cast<const float *>(W), ldw, L, k, q,
                               static_cast<float *>(w_out), h_out, rs, spin_limit, st, nkern);
        case CTG_BASIS_BF16:
            return cgs2_step_t(static_cast<const __nv_bfloat16 *>(W), ldw, L, k, q,
                               static_cast<__nv_bfloat16 *>(w_out), h_out, rs, spin_limit, st, nkern);
        case CTG_BASIS_FP16:
            return cgs2_step_t(static_cast<const __half *>(W), ldw, L, k, q,
                               static_cast<__half *>(w_out), h_out, rs, spin_limit, st, nkern);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t ctg_cgs2_step_loop(const void *W, int dtype, int64_t ldw, int64_t L, float *q, const LoopStep &ls,
                               const RedScratch &rs, long long spin_limit, bool cooperative, cudaStream_t st,
                               int *nkern) {
    switch (dtype) {
        case CTG_BASIS_FP32:
            return cgs2_loop_t(static_cast<const float *>(W), ldw, L, q, ls, rs, spin_limit, cooperative, st, nkern);
        case CTG_BASIS_BF16:
            return cgs2_loop_t(static_cast<const __nv_bfloat16 *>(W), ldw, L, q, ls, rs, spin_limit, cooperative,
                               st, nkern);
        case CTG_BASIS_FP16:
            return cgs2_loop_t(static_cast<const __half *>(W), ldw, L, q, ls, rs, spin_limit, cooperative, st,
                               nkern);
        default: return cudaErrorInvalidValue;
    }
}

int ctg_cgs2_small_grid_max() { return kSmallGridMaxK; }

bool ctg_cgs2_fused_ok(int dtype, int64_t L, int kmax, const RedScratch &rs, bool small_grid) {
    if (kmax > kFusedMaxK || rs.rows < 2 * kmax + 2) return false;
    int E;
    const int G = fused_grid(L, &E, small_grid);
    int cap = 0;
    switch (dtype * 16 + E) {
#define CTG_FOK(DT, T)                                                  \
    case DT * 16 + 1: cap = fused_resident_blocks<T, 1>(); break;       \
    case DT * 16 + 2: cap = fused_resident_blocks<T, 2>(); break;       \
    case DT * 16 + 4: cap = fused_resident_blocks<T, 4>(); break;       \
    case DT * 16 + 8: cap = fused_resident_blocks<T, 8>(); break;
        CTG_FOK(CTG_BASIS_FP32, float)
        CTG_FOK(CTG_BASIS_BF16, __nv_bfloat16)
        CTG_FOK(CTG_BASIS_FP16, __half)
#undef CTG_FOK
        default: return false;
    }
    return G <= cap;
}

int ctg_cgs2_fused_max(bool need_y) { return need_y ? kFusedMaxKY : kFusedMaxK; }

cudaError_t ctg_gemv(const void *W, int dtype, int64_t ldw, int64_t L, int k, const double *y,
                     const float *base, float *out, cudaStream_t st, const int *kdev, int koff) {
    switch (dtype) {
        case CTG_BASIS_FP32: return gemv_t(static_cast<const float *>(W), ldw, L, k, kdev, koff, y, base, out, st);
        case CTG_BASIS_BF16:
            return gemv_t(static_cast<const __nv_bfloat16 *>(W), ldw, L, k, kdev, koff, y, base, out, st);
        case CTG_BASIS_FP16:
            return gemv_t(static_cast<const __half *>(W), ldw, L, k, kdev, koff, y, base, out, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t ctg_sub_norm2(const float *a, const float *c, float *out, int64_t L,
                          double *res, const RedScratch &rs, cudaStream_t st) {
    int E;
    const int G = ctg_red_grid(L, &E);
    switch (E) {
#define CTG_SN_CASE(EE)                                                                        \
    case EE:                                                                                   \
        sub_norm2_kernel<EE><<<G, kThreads, 0, st>>>(a, c, out, L, rs.partials, rs.counter, res); \
        break;
        CTG_SN_CASE(1)
        CTG_SN_CASE(2)
        CTG_SN_CASE(4)
        CTG_SN_CASE(8)
#undef CTG_SN_CASE
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t ctg_scale(const float *v, const double *nrm2, void *out, int dtype, int64_t L,
                      cudaStream_t st) {
    switch (dtype) {
        case CTG_BASIS_FP32:
            scale_kernel<float><<<scale_blocks(L), 256, 0, st>>>(v, nrm2, static_cast<float *>(out), L,
                                                                 0, nullptr, nullptr, nullptr);
            break;
        case CTG_BASIS_BF16:
            scale_kernel<__nv_bfloat16><<<scale_blocks(L), 256, 0, st>>>(
                v, nrm2, static_cast<__nv_bfloat16 *>(out), L, 0, nullptr, nullptr, nullptr);
            break;
        case CTG_BASIS_FP16:
            scale_kernel<__half><<<scale_blocks(L), 256, 0, st>>>(v, nrm2, static_cast<__half *>(out),
                                                                  L, 0, nullptr, nullptr, nullptr);
            break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

int ctg_vec_blocks(long long L) { return (int)(((L + 3) / 4 + kThreads - 1) / kThreads); }

namespace {

template <typename T>
void launch_batch_cgs2(BatchInst *insts, const int2 *map, int nblocks, size_t smem, cudaStream_t st) {
    // pass 1: h1, ||q||^2; pass 2: q -= W h1, h2, ||q1||^2; then the last
    // update and the scaling in one sweep
    batch_cgs_pass_kernel<T, false, true, true><<<nblocks, kThreads, smem, st>>>(insts, map);
    batch_cgs_pass_kernel<T, true, true, true><<<nblocks, kThreads, smem, st>>>(insts, map);
    batch_update_scale_kernel<T><<<nblocks, kThreads, smem, st>>>(insts, map);
}

template <typename T>
cudaError_t prepare_batch_cgs2(size_t smem) {
    cudaError_t err;
    if ((err = ensure_smem(batch_cgs_pass_kernel<T, false, true, true>, smem)) != cudaSuccess) return err;
    if ((err = ensure_smem(batch_cgs_pass_kernel<T, true, true, true>, smem)) != cudaSuccess) return err;
    return ensure_smem(batch_update_scale_kernel<T>, smem);
}

}  // namespace

cudaError_t ctg_batch_cgs2(BatchInst *insts, const int2 *map, int nblocks, int max_k,
                           cudaStream_t st, int wtype) {
    if (nblocks <= 0) return cudaSuccess;
    const size_t smem = sizeof(float) * ((size_t)max_k + (size_t)kWarps * (max_k + 1));
    if (wtype == CTG_BASIS_BF16) launch_batch_cgs2<__nv_bfloat16>(insts, map, nblocks, smem, st);
    else if (wtype == CTG_BASIS_FP16) launch_batch_cgs2<__half>(insts, map, nblocks, smem, st);
    else launch_batch_cgs2<float>(insts, map, nblocks, smem, st);
    return cudaGetLastError();
}

cudaError_t ctg_batch_prepare(int max_k) {
    const size_t smem = sizeof(float) * ((size_t)max_k + (size_t)kWarps * (max_k + 1));
    cudaError_t err;
    if ((err = prepare_batch_cgs2<float>(smem)) != cudaSuccess) return err;
    if ((err = prepare_batch_cgs2<__nv_bfloat16>(smem)) != cudaSuccess) return err;
    if ((err = prepare_batch_cgs2<__half>(smem)) != cudaSuccess) return err;
    const int cap = max_k < 160 ? max_k : 160;
    if ((err = ensure_smem(batch_givens_kernel, sizeof(double) * (size_t)cap * (cap + 1) / 2)) != cudaSuccess)
        return err;
    return ensure_smem(batch_iterate_kernel, sizeof(float) * (size_t)(max_k > 0 ? max_k : 1));
}

cudaError_t ctg_batch_givens(BatchInst *insts, int n_inst, int max_k, cudaStream_t st) {
    if (n_inst <= 0) return cudaSuccess;
    const int cap = max_k < 160 ? max_k : 160;
    const size_t smem = sizeof(double) * (size_t)cap * (cap + 1) / 2;
    cudaError_t e = ensure_smem(batch_givens_kernel, smem);
    if (e != cudaSuccess) return e;
    batch_givens_kernel<<<n_inst, 32, smem, st>>>(insts, cap);
    return cudaGetLastError();
}

cudaError_t ctg_batch_iterate(BatchInst *insts, const int2 *map_n, int nblocks, int max_k, cudaStream_t st) {
    if (nblocks <= 0) return cudaSuccess;
    const size_t smem = sizeof(float) * (size_t)(max_k > 0 ? max_k : 1);
    batch_iterate_kernel<<<nblocks, kThreads, smem, st>>>(insts, map_n);
    return cudaGetLastError();
}

cudaError_t ctg_batch_residual(BatchInst *insts, const int2 *map_m, int nblocks, cudaStream_t st) {
    if (nblocks <= 0) return cudaSuccess;
    batch_residual_kernel<<<nblocks, kThreads, 0, st>>>(insts, map_m);
    return cudaGetLastError();
}

cudaError_t ctg_batch_finish(BatchInst *insts, int n_inst, int *active_count, cudaStream_t st) {
    if (n_inst <= 0) return cudaSuccess;
    batch_finish_kernel<<<(n_inst + 127) / 128, 128, 0, st>>>(insts, n_inst, active_count);
    return cudaGetLastError();
}

cudaError_t ctg_batch_finish_loop(BatchInst *insts, int n_inst, int *ctl, int max_rounds,
                                  cudaGraphConditionalHandle h, cudaStream_t st,
                                  cudaGraphConditionalHandle h_next, int fused_max) {
    if (n_inst <= 0 || n_inst > 1024) return cudaErrorInvalidValue;
    batch_finish_loop_kernel<<<1, n_inst < 128 ? 128 : 1024, 0, st>>>(insts, n_inst, ctl, max_rounds, h,
                                                                        h_next, fused_max);
    return cudaGetLastError();
}

namespace {

size_t batch_fused_smem(int kcap) {
    const int pc = kcap;
    return sizeof(double) * ((size_t)3 * kcap + 1 + (size_t)pc * (pc + 1) / 2 + (size_t)2 * kcap + 3) +
           sizeof(float) * ((size_t)kcap + (size_t)kWarps * (kcap + 1));
}

template <typename T>
int batch_fused_resident_t(int kcap) {
    int dev = -1, per_sm = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        ensure_smem(batch_cgs2_fused_kernel<T>, batch_fused_smem(kcap)) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_cgs2_fused_kernel<T>, kThreads,
                                                      batch_fused_smem(kcap)) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return per_sm * sms;
}

template <typename T>
cudaError_t launch_batch_fused(BatchInst *insts, const int2 *map, int nblocks, int kcap, unsigned *bar, int *err,
                               const long long *spin_limit, cudaStream_t st) {
    const size_t smem = batch_fused_smem(kcap);
    cudaError_t e = ensure_smem(batch_cgs2_fused_kernel<T>, smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nblocks);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, batch_cgs2_fused_kernel<T>, insts, map, bar, err, spin_limit, kcap, kcap);
}

}  // namespace

int ctg_batch_fused_max_k() { return kFusedMaxKY; }

int ctg_batch_fused_resident(int kcap, int wtype) {
    if (kcap < 1 || kcap > kFusedMaxKY) return 0;
    if (wtype == CTG_BASIS_BF16) return batch_fused_resident_t<__nv_bfloat16>(kcap);
    if (wtype == CTG_BASIS_FP16) return batch_fused_resident_t<__half>(kcap);
    return batch_fused_resident_t<float>(kcap);
}

cudaError_t ctg_batch_cgs2_fused(BatchInst *insts, const int2 *map, int nblocks, int kcap, unsigned *bar,
                                 int *err, const long long *spin_limit, cudaStream_t st, int wtype) {
    if (nblocks <= 0) return cudaSuccess;
    if (kcap < 1 || kcap > kFusedMaxKY) return cudaErrorInvalidValue;
    if (wtype == CTG_BASIS_BF16)
        return launch_batch_fused<__nv_bfloat16>(insts, map, nblocks, kcap, bar, err, spin_limit, st);
    if (wtype == CTG_BASIS_FP16) return launch_batch_fused<__half>(insts, map, nblocks, kcap, bar, err, spin_limit, st);
    return launch_batch_fused<float>(insts, map, nblocks, kcap, bar, err, spin_limit, st);
}

cudaError_t ctg_batch_solve_y(BatchInst *insts, int n_inst, int max_k, cudaStream_t st) {
    if (n_inst <= 0) return cudaSuccess;
    const int cap = max_k < 160 ? max_k : 160;
    const size_t smem = sizeof(double) * (size_t)cap * (cap + 1) / 2;
    cudaError_t e = ensure_smem(batch_solve_y_kernel, smem);
    if (e != cudaSuccess) return e;
    batch_solve_y_kernel<<<n_inst, 32, smem, st>>>(insts, cap);
    return cudaGetLastError();
}
