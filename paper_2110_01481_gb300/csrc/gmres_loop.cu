// Device side of the AB-GMRES / BA-GMRES iteration (paper Sec. 2, algorithm
// box) for a solver loop that runs without the host: the FP64 Givens update
// of the Hessenberg least-squares problem min || beta e1 - H_k y ||, the
// iterate's coefficients y_k, and the stopping rules of Sec. 6.4 (the
// discrepancy principle on ||b - A x_k||, the NCP criterion, maxit,
// breakdown).  Every kernel reads the step k from the solve's device state,
// so one captured sequence of launches serves every step; the kernel that
// ends a step either advances k or stops the solve, and, inside a CUDA
// graph, also sets the condition of the graph's while-loop nodes.
#include "loop_device.cuh"

namespace {

// Step k's Givens update and stopping rule as a kernel of its own (where
// the CGS2 step cannot run it: the separate passes).
__global__ void loop_givens_kernel(LoopBufs B, int mode, int pack_cap) {
    extern __shared__ double s_pack[];
    __shared__ double s_stage[3 * kGivStage + 1];
    const int k = B.S->k;
    const double *h = B.H + (size_t)(k - 1) * B.ldh;
    loop_givens_warp(B, k, h, B.h1[k], mode, s_pack, pack_cap, k <= kGivStage ? s_stage : nullptr);
}

// BA with the discrepancy principle or NCP: r = b - A x_k (Ax = A x_k from
// the step's two-image forward projection), ||r||^2 reduced across blocks by the
// last block, which records ||b - A x_k|| and, with `decide` (DP), ends
// the step: stop at a pending breakdown, at ||r|| <= target (DP), at a
// pending maxit, else k + 1.  r_out: NULL, or where r is written (NCP).
template <int E>
__global__ void __launch_bounds__(kThreads, 2)
loop_resid_kernel(const float *__restrict__ b, const float *__restrict__ Ax, float *__restrict__ r_out,
                  int64_t L, float *__restrict__ partials, unsigned *__restrict__ counter, LoopBufs B,
                  int decide) {
    __shared__ float s_w[kWarps];
    const int tid = threadIdx.x;
    const int64_t g0 = (int64_t)blockIdx.x * kThreads * E + tid;
    float s = 0.f;
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int64_t g = g0 + (int64_t)e * kThreads;
        float4 v = ld4(b, g, L);
        const float4 w = ld4(Ax, g, L);
        v.x -= w.x; v.y -= w.y; v.z -= w.z; v.w -= w.w;
        if (r_out) st4(r_out, g, L, v);
        s += dot4(v, v);
    }
    s = warp_sum(s);
    if ((tid & 31) == 0) s_w[tid >> 5] = s;
    if (!block_reduce_finish(s_w, 1, partials, counter, B.scal + 4, blockIdx.x, gridDim.x)) return;
    if (tid != 0) return;
    GmresState &S = *B.S;
    const int k = S.k;
    const double res = sqrt(B.scal[4]);
    S.resnorm = res;
    if (S.rule == kRuleDP) B.hist[k] = res;
    if (!decide) return;
    int stop = 0;
    if (S.pending == CTG_STOP_BREAKDOWN + 1) stop = S.pending;
    else if (res <= S.target) stop = CTG_STOP_DP + 1;
    else stop = S.pending;
    S.pending = 0;
    end_step(B, stop, k);
}

// NCP (Sec. 6.4): d_k = scal[6], the NCP distance of b - A x_k; the solve
// returns x_{k-1} at the first k with d_k > d_{k-1}; else a pending stop;
// else k + 1.
__global__ void loop_ncp_decide_kernel(LoopBufs B) {
    GmresState &S = *B.S;
    const int k = S.k;
    const double d = B.scal[6];
    B.ncph[k] = d;
    int stop = S.pending, iters = k;
    if (d > S.dprev) {
        stop = CTG_STOP_NCP + 1;
        iters = k - 1;
    }
    S.dprev = d;
    S.pending = 0;
    end_step(B, stop, iters);
}

// End of a step whose last kernel is a projection (BA, maxit rule).
__global__ void loop_advance_kernel(LoopBufs B) {
    GmresState &S = *B.S;
    const int stop = S.pending;
    S.pending = 0;
    end_step(B, stop, S.k);
}

// Start of the solve, after r0 and its norms are in scal: scal[2] =
// ||r0||^2 (AB: r0 = b - A x0; BA: r0 = B (b - A x0)), scal[4] =
// ||b - A x0||^2 (BA), scal[6] = d_0 (NCP).  g = beta e1; a k = 0 stop when
// beta = 0 (breakdown) or x0 already meets the discrepancy principle.
__global__ void loop_init_kernel(LoopBufs B, int variant, int rule, int maxit, double target) {
    GmresState &S = *B.S;
    const double beta = sqrt(B.scal[2]);
    const double res0 = variant == CTG_BA ? sqrt(B.scal[4]) : beta;
    S.variant = variant;
    S.rule = rule;
    S.maxit = maxit;
    S.target = target;
    S.beta = beta;
    S.res0 = res0;
    S.rho = beta;
    S.resnorm = res0;
    S.k = 1;
    S.iters = 0;
    S.pending = 0;
    S.steps = 0;
    S.timed_out = 0;
    S.stop_reason = CTG_STOP_MAXIT;
    B.gg[0] = beta;
    B.rhoh[0] = beta;
    B.hist[0] = (variant == CTG_BA && rule == kRuleDP) ? res0 : beta;
    if (rule == kRuleNCP) {
        S.dprev = B.scal[6];
        B.ncph[0] = B.scal[6];
    }
    const bool dp0 = rule == kRuleDP && res0 <= target;
    if (dp0 || beta == 0.0) {
        S.active = 0;
        S.stop_reason = dp0 ? CTG_STOP_DP : CTG_STOP_BREAKDOWN;
        set_cond(B.c_small, B.in_graph, 0u);
        set_cond(B.c_fused, B.in_graph, 0u);
        set_cond(B.c_pass, B.in_graph, 0u);
    } else {
        S.active = 1;
    }
}

// Exit: y = y_iters into B.y for the iterate's formation.  After an NCP
// stop (iters = k - 1, while step k has already rotated g) it is the
// y_{k-1} kept in yring; otherwise it is R^{-1} g_{1:iters}.  Also rho of
// the returned iterate.
__global__ void loop_exit_y_kernel(LoopBufs B, int pack_cap) {
    extern __shared__ double s_pack[];
    GmresState &S = *B.S;
    const int it = S.iters, lane = threadIdx.x;
    if (it > 0) {
        if (S.stop_reason == CTG_STOP_NCP) {
            const double *yr = B.yring + (size_t)(it % 3) * B.ldr;
            for (int i = lane; i < it; i += 32) B.y[i] = yr[i];
        } else {
            solve_y_warp(B.R, B.ldr, B.gg, it, B.y, s_pack, pack_cap);
        }
    }
    if (lane == 0) S.rho = B.rhoh[it];
}

// After the returned iterate's true residual is in scal[5].
__global__ void loop_final_kernel(LoopBufs B) {
    B.S->resnorm = sqrt(B.scal[5]);
}

int ensure_dyn_smem(const void *kern, size_t bytes) {
    return ctg_allow_dyn_smem(kern, bytes) == cudaSuccess ? 0 : -1;
}

}  // namespace

// Packed R of up to this many columns is staged in shared memory.
int ctg_loop_pack_cap(int maxit) { return maxit < 160 ? maxit : 160; }
static size_t pack_bytes(int cap) { return sizeof(double) * (size_t)cap * (cap + 1) / 2; }

cudaError_t ctg_loop_init(const LoopBufs &B, int variant, int rule, int maxit, double target, cudaStream_t st) {
    loop_init_kernel<<<1, 1, 0, st>>>(B, variant, rule, maxit, target);
    return cudaGetLastError();
}

cudaError_t ctg_loop_givens(const LoopBufs &B, bool need_y, bool need_z, bool end, int maxit, cudaStream_t st) {
    const int cap = need_y ? ctg_loop_pack_cap(maxit) : 0;
    const size_t smem = need_y ? pack_bytes(cap) : 0;
    if (ensure_dyn_smem((const void *)loop_givens_kernel, smem)) return cudaErrorInvalidValue;
    const int mode = (need_y ? kGivY : 0) | (need_z ? kGivZ : 0) | (end ? kGivEnd : 0);
    loop_givens_kernel<<<1, 32, smem, st>>>(B, mode, cap);
    return cudaGetLastError();
}

cudaError_t ctg_loop_resid(const LoopBufs &B, const float *b, const float *Ax, float *r_out, int64_t L,
                           const RedScratch &rs, bool decide, cudaStream_t st) {
    int E;
    const int G = ctg_red_grid(L, &E);
    switch (E) {
#define CTG_LR_CASE(EE)                                                                                   \
    case EE:                                                                                              \
        loop_resid_kernel<EE><<<G, kThreads, 0, st>>>(b, Ax, r_out, L, rs.partials, rs.counter, B, decide); \
        break;
        CTG_LR_CASE(1)
        CTG_LR_CASE(2)
        CTG_LR_CASE(4)
        CTG_LR_CASE(8)
#undef CTG_LR_CASE
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t ctg_loop_ncp_decide(const LoopBufs &B, cudaStream_t st) {
    loop_ncp_decide_kernel<<<1, 1, 0, st>>>(B);
    return cudaGetLastError();
}

cudaError_t ctg_loop_advance(const LoopBufs &B, cudaStream_t st) {
    loop_advance_kernel<<<1, 1, 0, st>>>(B);
    return cudaGetLastError();
}

cudaError_t ctg_loop_exit_y(const LoopBufs &B, int maxit, cudaStream_t st) {
    const int cap = ctg_loop_pack_cap(maxit);
    const size_t smem = pack_bytes(cap);
    if (ensure_dyn_smem((const void *)loop_exit_y_kernel, smem)) return cudaErrorInvalidValue;
    loop_exit_y_kernel<<<1, 32, smem, st>>>(B, cap);
    return cudaGetLastError();
}

cudaError_t ctg_loop_final(const LoopBufs &B, cudaStream_t st) {
    loop_final_kernel<<<1, 1, 0, st>>>(B);
    return cudaGetLastError();
}
