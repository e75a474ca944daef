// Device side of one step of the AB-/BA-GMRES loop (paper Sec. 2,
// algorithm box): the FP64 Givens update of the Hessenberg least-squares
// problem, y_k, and the end of a step (advance k, or stop the solve and end
// the CUDA graph's while loops).  Shared by the loop's own Givens kernel
// (gmres_loop.cu) and the one-launch CGS2 step, whose block 0 runs it once
// the new Hessenberg column is known (arnoldi.cu).
#pragma once
#include "vecops.cuh"

namespace {

__device__ __forceinline__ void set_cond(cudaGraphConditionalHandle h, bool in_graph, unsigned v) {
    if (in_graph) cudaGraphSetConditional(h, v);
}

// End of step k (one thread): stop the solve with `stop` (a CTG_STOP_*
// value + 1, 0 to go on) returning x_iters, or move to step k + 1.  A
// timed-out grid barrier (counter[2] set) stops the solve too; the host
// reports it.
__device__ void end_step(const LoopBufs &B, int stop, int iters) {
    GmresState &S = *B.S;
    S.steps += 1;
    if (B.counter[2] != 0u) {
        stop = CTG_STOP_MAXIT + 1;
        S.timed_out = 1;
    }
    if (stop) {
        S.active = 0;
        S.stop_reason = stop - 1;
        S.iters = iters;
        set_cond(B.c_small, B.in_graph, 0u);
        set_cond(B.c_fused, B.in_graph, 0u);
        set_cond(B.c_pass, B.in_graph, 0u);
    } else {
        const int k1 = S.k + 1;
        S.k = k1;
        if (k1 > B.small_max) set_cond(B.c_small, B.in_graph, 0u);
        if (k1 > B.fused_max) set_cond(B.c_fused, B.in_graph, 0u);
    }
}

// Modes of the Givens update (kGivY, kGivZ, kGivEnd in ctg_internal.cuh):
//   kGivY  y_k into y and yring[k % 3] (BA with a residual rule, AB NCP),
//   kGivZ  z = beta e1 - H_k y_k, the residual's coefficients in W_{k+1}
//          (AB NCP), by the rotations applied backwards,
//   kGivEnd  end the step here (AB with DP / maxit): stop at breakdown, at
//          rho_k <= target (DP) or at k = maxit, else k + 1.
// Otherwise a breakdown or k = maxit is left in S.pending for the step's
// last kernel.  hist[k] = rho_k unless BA with the discrepancy rule (its
// history is the true residual).
constexpr int kGivStage = 512;     // steps staged in shared memory; beyond, lane 0 reads global memory

// Step k after its CGS2 step: Hessenberg column h[0..k] (global or shared
// memory) and ||q before CGS2||^2 = qpre2.  Run by one whole warp (lane =
// threadIdx.x & 31).  The column, the rotations and the rotated column are
// staged in s_stage (3 k + 1 doubles; NULL: global memory) so that lane 0's
// recurrence does no global round trips; the packed triangle of R for y_k
// in s_pack when k <= pack_cap.  A NaN column (a CGS2 step that gave up at
// a grid barrier) counts as a breakdown; end_step then reports the timeout.
__device__ void loop_givens_warp(const LoopBufs &B, int k, const double *h, double qpre2, int mode,
                                 double *s_pack, int pack_cap, double *s_stage) {
    GmresState &S = *B.S;
    const int lane = threadIdx.x & 31;
    double *Rk = B.R + (size_t)(k - 1) * B.ldr;
    double *s_h = s_stage, *s_gc = s_stage ? s_stage + (k + 1) : nullptr, *s_gs = s_gc ? s_gc + k : nullptr;
    if (s_stage) {
        for (int i = lane; i <= k; i += 32) s_h[i] = h[i];
        for (int i = lane; i < k - 1; i += 32) {
            s_gc[i] = B.gc[i];
            s_gs[i] = B.gs[i];
        }
    }
    __syncwarp();
    const double *hh = s_stage ? s_h : h;
    const double *gcc = s_stage ? s_gc : B.gc;
    const double *gss = s_stage ? s_gs : B.gs;
    double rho = 0.0;
    int brk = 0;
    if (lane == 0) {
        double r_prev = hh[0];
        for (int i = 0; i < k - 1; ++i) {
            const double a = r_prev, b = hh[i + 1];
            const double t = gcc[i] * a + gss[i] * b;
            if (s_stage) s_h[i] = t;           // rotated column, stored below
            else Rk[i] = t;
            r_prev = -gss[i] * a + gcc[i] * b;
        }
        const double a = r_prev, b = hh[k];
        double c, sn, rinv;
        givens_rotation(a, b, c, sn, rinv);
        B.gc[k - 1] = c;
        B.gs[k - 1] = sn;
        if (s_stage) s_h[k - 1] = rinv;        // R's diagonal as its reciprocal
        else Rk[k - 1] = rinv;
        B.gg[k] = -sn * B.gg[k - 1];
        B.gg[k - 1] = c * B.gg[k - 1];
        rho = fabs(B.gg[k]);
        S.rho = rho;
        B.rhoh[k] = rho;
        // b <= 1e-6 ||q before CGS2||, squared (b >= 0): no square root
        brk = (!(b == b) || b * b <= 1e-12 * qpre2) ? 1 : 0;
    }
    rho = __shfl_sync(0xffffffffu, rho, 0);
    brk = __shfl_sync(0xffffffffu, brk, 0);
    if (s_stage)
        for (int i = lane; i < k; i += 32) Rk[i] = s_h[i];
    __syncwarp();
    if (mode & kGivY) {
        solve_y_warp(B.R, B.ldr, B.gg, k, B.y, s_pack, pack_cap);
        double *yr = B.yring + (size_t)(k % 3) * B.ldr;
        for (int i = lane; i < k; i += 32) yr[i] = B.y[i];
    }
    if ((mode & kGivZ) && lane == 0) {
        // z = G_1^T ... G_k^T (g_{k+1} e_{k+1}), G_i acting on entries i-1, i
        for (int i = 0; i <= k; ++i) B.z[i] = 0.0;
        B.z[k] = B.gg[k];
        for (int i = k - 1; i >= 0; --i) {
            const double a = B.z[i], b = B.z[i + 1];
            B.z[i] = B.gc[i] * a - B.gs[i] * b;
            B.z[i + 1] = B.gs[i] * a + B.gc[i] * b;
        }
    }
    if (lane != 0) return;
    if (!(S.variant == CTG_BA && S.rule == kRuleDP)) B.hist[k] = rho;
    const int pending = brk ? CTG_STOP_BREAKDOWN + 1 : (k == S.maxit ? CTG_STOP_MAXIT + 1 : 0);
    if (mode & kGivEnd) {
        int stop = pending;
        if (!brk && S.rule == kRuleDP && rho <= S.target) stop = CTG_STOP_DP + 1;
        end_step(B, stop, k);
    } else {
        S.pending = pending;
    }
}

// Shared memory loop_givens_warp needs beside the caller's own: the packed
// triangle for y_k (pack_cap (pack_cap + 1) / 2 doubles) and the staging
// (3 k + 1 doubles).
__host__ __device__ inline int loop_pack_cap(int maxit) { return maxit < 160 ? maxit : 160; }

}  // namespace
