// LSQR (Paige & Saunders 1982) and LSMR (Fong & Saunders 2011), damping 0:
// the matched-case comparators of Sec. 5 (AB-GMRES with B = A^T equals LSQR,
// BA-GMRES with B = A^T equals LSMR, in exact arithmetic).  With an
// unmatched B in place of A^T they are run as the paper discusses them: on
// the unmatched normal equations.
//
// One iteration is a Golub-Kahan bidiagonalisation step
//   beta_{k+1} u_{k+1} = A v_k - alpha_k u_k,
//   alpha_{k+1} v_{k+1} = B u_{k+1} - beta_{k+1} v_k,
// then the plane rotations of the method (one thread, FP64) and one fused
// vector update.  All scalars live in a device LsqState, so a step needs no
// host round trip; the host only reads the `live` flag, one step behind.
// u is kept unnormalised (u~ = beta u), which saves a scaling pass:
// u~_{k+1} = A v_k - (alpha_k / beta_k) u~_k and B u_{k+1} = (B u~_{k+1}) / beta_{k+1}.
// For LSMR the residual r_k = b - A x_k is tracked in sinogram space (it has
// no cheap norm estimate of its own): A h_k and A hbar_k follow the same
// recurrences as h_k and hbar_k, with A v_k = p taken from the step.
#include "vecops.cuh"

namespace {

template <int E>
__global__ void __launch_bounds__(kThreads, 2)
bidiag_u_kernel(const float *__restrict__ p, float *__restrict__ u, int64_t L, LsqState *S,
                float *__restrict__ partials, unsigned *__restrict__ counter) {
    __shared__ float s_w[kWarps];
    const float c = (float)(S->beta > 0.0 ? S->alpha / S->beta : 0.0);
    const int64_t g0 = (int64_t)blockIdx.x * kThreads * E + threadIdx.x;
    float s = 0.f;
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int64_t g = g0 + (int64_t)e * kThreads;
        const float4 a = ld4(p, g, L), b = ld4_rw(u, g, L);
        const float4 v = make_float4(fmaf(-c, b.x, a.x), fmaf(-c, b.y, a.y), fmaf(-c, b.z, a.z),
                                     fmaf(-c, b.w, a.w));
        st4(u, g, L, v);
        s += dot4(v, v);
    }
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = s;
    block_reduce_finish(s_w, 1, partials, counter, &S->beta2, blockIdx.x, gridDim.x);
}

template <int E>
__global__ void __launch_bounds__(kThreads, 2)
bidiag_v_kernel(const float *__restrict__ q, float *__restrict__ v, int64_t L, LsqState *S,
                float *__restrict__ partials, unsigned *__restrict__ counter) {
    __shared__ float s_w[kWarps];
    const double bd = sqrt(S->beta2);
    const float bp = (float)bd, ib = (float)(bd > 0.0 ? 1.0 / bd : 0.0);
    const int64_t g0 = (int64_t)blockIdx.x * kThreads * E + threadIdx.x;
    float s = 0.f;
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int64_t g = g0 + (int64_t)e * kThreads;
        const float4 a = ld4(q, g, L), b = ld4_rw(v, g, L);
        const float4 w = make_float4(fmaf(a.x, ib, -bp * b.x), fmaf(a.y, ib, -bp * b.y),
                                     fmaf(a.z, ib, -bp * b.z), fmaf(a.w, ib, -bp * b.w));
        st4(v, g, L, w);
        s += dot4(w, w);
    }
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = s;
    block_reduce_finish(s_w, 1, partials, counter, &S->alpha2, blockIdx.x, gridDim.x);
}

__device__ void stop_with(LsqState *S, int reason) {
    S->live = 0;
    S->iters = S->k;
    S->stop_reason = reason;
}

// One thread: the rotations of iteration k from alpha_{k+1}, beta_{k+1}.
__global__ void scalars_kernel(LsqState *S) {
    if (!S->live) {
        S->live_update = 0;
        return;
    }
    S->live_update = 1;
    const double beta = sqrt(S->beta2), alpha = sqrt(S->alpha2);   // beta_{k+1}, alpha_{k+1}
    const bool exhausted = !(alpha > 0.0) || !(beta > 0.0);
    S->inv_alpha = alpha > 0.0 ? 1.0 / alpha : 0.0;
    S->alpha = alpha;       // u~_{k+2} = A v_{k+1} - (alpha_{k+1} / beta_{k+1}) u~_{k+1}
    S->beta = beta;
    if (S->method == CTG_LSQR) {
        const double rho = hypot(S->rhobar, beta);
        const double c = rho > 0.0 ? S->rhobar / rho : 1.0, s = rho > 0.0 ? beta / rho : 0.0;
        const double theta = s * alpha, phi = c * S->phibar;
        S->rhobar = -c * alpha;
        S->phibar = s * S->phibar;
        S->cx = rho > 0.0 ? phi / rho : 0.0;
        S->cw = rho > 0.0 ? theta / rho : 0.0;
        const double est = fabs(S->phibar);            // ||b - A x_k|| in exact arithmetic
        S->hist[S->k] = est;
        S->status[1] = est;
        if (exhausted) stop_with(S, CTG_STOP_BREAKDOWN);
        else if (S->target > 0.0 && est <= S->target) stop_with(S, CTG_STOP_DP);
        else if (S->k == S->maxit) stop_with(S, CTG_STOP_MAXIT);
        else S->k += 1;
        S->status[0] = S->live;
    } else {
        const double rho = hypot(S->alphabar, beta);
        const double c = rho > 0.0 ? S->alphabar / rho : 1.0, s = rho > 0.0 ? beta / rho : 0.0;
        const double theta_new = s * alpha;
        S->alphabar = c * alpha;
        const double thetabar = S->sbar * rho;
        const double rhobar = hypot(S->cbar * rho, theta_new);
        const double cbar = rhobar > 0.0 ? S->cbar * rho / rhobar : 1.0;
        const double sbar = rhobar > 0.0 ? theta_new / rhobar : 0.0;
        const double zeta = cbar * S->zetabar;
        S->zetabar = -sbar * S->zetabar;
        S->cbar = cbar;
        S->sbar = sbar;
        const double den = S->rho_old * S->rhobar_old;
        S->chbar = den != 0.0 ? thetabar * rho / den : 0.0;
        S->cx = rho * rhobar != 0.0 ? zeta / (rho * rhobar) : 0.0;
        S->ch_prev = S->ch;
        S->ch = rho > 0.0 ? theta_new / rho : 0.0;
        S->rho_old = rho;
        S->rhobar_old = rhobar;
        // the stopping rules wait for the tracked residual (check_kernel);
        // an exhausted Krylov space is flagged here
        S->stop_reason = exhausted ? CTG_STOP_BREAKDOWN : -1;
    }
}

__global__ void check_kernel(LsqState *S) {
    if (!S->live_update) return;
    const double est = sqrt(S->r2);
    S->hist[S->k] = est;
    S->status[1] = est;
    if (S->stop_reason == CTG_STOP_BREAKDOWN) stop_with(S, CTG_STOP_BREAKDOWN);
    else if (S->target > 0.0 && est <= S->target) stop_with(S, CTG_STOP_DP);
    else if (S->k == S->maxit) stop_with(S, CTG_STOP_MAXIT);
    else S->k += 1;
    S->status[0] = S->live;
}

__device__ __forceinline__ float4 axpy4(float a, float4 x, float4 y) {   // a x + y
    return make_float4(fmaf(a, x.x, y.x), fmaf(a, x.y, y.y), fmaf(a, x.z, y.z), fmaf(a, x.w, y.w));
}
__device__ __forceinline__ float4 scal4(float a, float4 x) {
    return make_float4(a * x.x, a * x.y, a * x.z, a * x.w);
}

__global__ void __launch_bounds__(kThreads)
update_kernel(const LsqState *__restrict__ S, float *v, float *a, float *c, float *x, int64_t n) {
    if (!S->live_update) return;
    const int64_t g = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (4 * g >= n) return;
    const float ia = (float)S->inv_alpha, cx = (float)S->cx;
    const float4 vv = scal4(ia, ld4_rw(v, g, n));
    st4(v, g, n, vv);
    if (S->method == CTG_LSQR) {
        const float cw = (float)S->cw;
        const float4 w = ld4_rw(a, g, n);
        st4(x, g, n, axpy4(cx, w, ld4_rw(x, g, n)));
        st4(a, g, n, axpy4(-cw, w, vv));
    } else {
        const float chbar = (float)S->chbar, ch = (float)S->ch;
        const float4 h = ld4_rw(a, g, n);
        const float4 hb = axpy4(-chbar, ld4_rw(c, g, n), h);
        st4(c, g, n, hb);
        st4(x, g, n, axpy4(cx, hb, ld4_rw(x, g, n)));
        st4(a, g, n, axpy4(-ch, h, vv));
    }
}

template <int E>
__global__ void __launch_bounds__(kThreads, 2)
residual_kernel(const LsqState *S, const float *__restrict__ p, float *Ah, float *Ahbar, float *r,
                int64_t L, double *r2, float *__restrict__ partials, unsigned *__restrict__ counter) {
    __shared__ float s_w[kWarps];
    if (!S->live_update) return;     // uniform over the grid: no block takes part
    const float chp = (float)S->ch_prev, chbar = (float)S->chbar, cx = (float)S->cx;
    const int64_t g0 = (int64_t)blockIdx.x * kThreads * E + threadIdx.x;
    float s = 0.f;
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int64_t g = g0 + (int64_t)e * kThreads;
        const float4 ah = axpy4(-chp, ld4_rw(Ah, g, L), ld4(p, g, L));
        const float4 ahb = axpy4(-chbar, ld4_rw(Ahbar, g, L), ah);
        const float4 rr = axpy4(-cx, ahb, ld4_rw(r, g, L));
        st4(Ah, g, L, ah);
        st4(Ahbar, g, L, ahb);
        st4(r, g, L, rr);
        s += dot4(rr, rr);
    }
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = s;
    block_reduce_finish(s_w, 1, partials, counter, r2, blockIdx.x, gridDim.x);
}

__global__ void __launch_bounds__(kThreads)
start_kernel(const LsqState *__restrict__ S, float *v, float *a, float *c, int64_t n) {
    const int64_t g = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (4 * g >= n) return;
    const float4 vv = scal4((float)S->inv_alpha, ld4_rw(v, g, n));
    st4(v, g, n, vv);
    st4(a, g, n, vv);
    if (c) st4(c, g, n, make_float4(0.f, 0.f, 0.f, 0.f));
}

int elem_blocks(int64_t n) { return (int)(((n + 3) / 4 + kThreads - 1) / kThreads); }

}  // namespace

#define CTG_E_DISPATCH(KERNEL, ...)                                                   \
    do {                                                                             \
        switch (E) {                                                                 \
            case 1: KERNEL<1><<<G, kThreads, 0, st>>>(__VA_ARGS__); break;           \
            case 2: KERNEL<2><<<G, kThreads, 0, st>>>(__VA_ARGS__); break;           \
            case 4: KERNEL<4><<<G, kThreads, 0, st>>>(__VA_ARGS__); break;           \
            case 8: KERNEL<8><<<G, kThreads, 0, st>>>(__VA_ARGS__); break;           \
            default: return cudaErrorInvalidValue;                                   \
        }                                                                            \
    } while (0)

cudaError_t ctg_lsq_bidiag_u(const float *p, float *u, int64_t m, LsqState *state,
                             const RedScratch &rs, cudaStream_t st) {
    int E;
    const int G = ctg_red_grid(m, &E);
    CTG_E_DISPATCH(bidiag_u_kernel, p, u, m, state, rs.partials, rs.counter);
    return cudaGetLastError();
}

cudaError_t ctg_lsq_bidiag_v(const float *q, float *v, int64_t n, LsqState *state,
                             const RedScratch &rs, cudaStream_t st) {
    int E;
    const int G = ctg_red_grid(n, &E);
    CTG_E_DISPATCH(bidiag_v_kernel, q, v, n, state, rs.partials, rs.counter);
    return cudaGetLastError();
}

cudaError_t ctg_lsq_scalars(LsqState *state, cudaStream_t st) {
    scalars_kernel<<<1, 1, 0, st>>>(state);
    return cudaGetLastError();
}

cudaError_t ctg_lsq_update(const LsqState *state, float *v, float *a, float *c, float *x,
                           int64_t n, cudaStream_t st) {
    update_kernel<<<elem_blocks(n), kThreads, 0, st>>>(state, v, a, c, x, n);
    return cudaGetLastError();
}

cudaError_t ctg_lsq_residual(LsqState *state, const float *p, float *Ah, float *Ahbar, float *r,
                             int64_t m, const RedScratch &rs, cudaStream_t st) {
    int E;
    const int G = ctg_red_grid(m, &E);
    CTG_E_DISPATCH(residual_kernel, state, p, Ah, Ahbar, r, m, &state->r2, rs.partials, rs.counter);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    check_kernel<<<1, 1, 0, st>>>(state);
    return cudaGetLastError();
}

cudaError_t ctg_lsq_start(const LsqState *state, float *v, float *a, float *c, int64_t n,
                          cudaStream_t st) {
    start_kernel<<<elem_blocks(n), kThreads, 0, st>>>(state, v, a, c, n);
    return cudaGetLastError();
}
