// Internal declarations shared by the CUDA translation units of libctgmres.
//
// Positions along a ray or across the detector are carried in fixed point
// (int64): integer steps are exact, so the interpolation index and weight
// stay accurate to ~1e-7 pixel at every image size without FP64 arithmetic
// on the device (FP32 alone loses ~1e-4 pixel at N = 2048).  The forward
// projector uses 32.32 (the high word is then directly an index), the back
// projector 24.40.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/ctgmres.h"

#define CTG_FX_BITS 40       // back projector
#define CTG_FXF_BITS 32      // forward projector

// Forward (Joseph) parameters of one angle.  With (c, s) = (cos, sin) for a
// row-driven ray and (sin, cos) for a column-driven one, the interpolation
// position of ray d at walk step t (row or column index) is
//   u(d, t) = Q + d * P + t * D,  P = ds / c,  Q = (h s - hd ds) / c + h,
//   D = -s / c,  h = (N-1)/2,  hd = (n_det-1)/2,
// and the ray sum is scaled by 1/|c|.  P, Q, D are 32.32 fixed point.
struct FwdAngle {
    long long P, Q, D;     // fixed point
    float pf, qf, df;      // the same in float, for the walk-range estimate
    float scale;           // 1 / |c|
    int row_driven;        // 1: walk rows of x; 0: walk rows of x^T
    int pad_;
};

// Back-projection parameters of one angle: the detector position of pixel
// (i, j) is u(i, j) = C + j * COS + i * SIN with COS = cos/ds, SIN = sin/ds,
// C = hd - h (cos + sin) / ds.
struct BackAngle {
    long long C, COS, SIN; // fixed point
    float cf, sf;          // COS, SIN in float (tile-local offsets)
};

// Matched back projector A^T (and B_tau) of one angle: with c = cos for a
// row-driven angle and sin for a column-driven one, pixel (i, j) takes bin
// d with weight scale * max(0, 1 - |d - u(i, j)| * inv_w), u as in
// BackAngle, scale = 1/|c|, inv_w = ds/|c|.
struct MatchedAngle {
    float scale, inv_w;
};

// Staged image read by the forward projector: two copies, x and x^T, each N
// rows of `stride` pairs (v[j] - dv[j], dv[j]) with dv[j] = v[j+1] - v[j]
// for columns j = -border .. N + border - 1 (zeros outside the image), so
// that with m = 1 + f in [1, 2): v0 + dv * m = lerp(v, j + f).
// The border is wide enough that every lane of a warp walking the union of
// its 32 rays' chords stays inside the buffer: such a lane is at most
// 31 |P| + 6 from the image (31 rays apart from a lane whose range starts or
// ends there, a step of margin on each side of that range, up to 3 steps
// more where the walk starts at a multiple of 4, |D| <= 1), and the border
// is 31 sqrt(2) ds + 10 or more; for very coarse detector pitches the border
// is 2 and the kernel clamps the tap index instead.
struct PadLayout {
    int border;            // zero pairs on each side of a row
    int stride;            // pairs per row = N + 2 * border
    bool clamp;            // tap index clamped to [-2, N]
    size_t floats;         // total floats of the staged image (both copies)
};
static inline PadLayout ctg_pad_layout(int N, double det_spacing) {
    PadLayout p;
    // |P| = ds / max(|cos|, |sin|) <= sqrt(2) ds
    const double need = 31.0 * 1.41421356237309515 * det_spacing + 10.0;
    p.clamp = need > 256.0;
    p.border = p.clamp ? 2 : (int)need + 1;
    p.stride = N + 2 * p.border;
    p.floats = 4 * (size_t)N * (size_t)p.stride;
    return p;
}

// A vector that is column (*k + off) of a basis with a stride of ld
// elements, the step index k being read on the device when the kernel runs
// (so that one captured launch serves every step of a solver loop); with
// k == nullptr, the vector is the given pointer itself.
struct ColRef {
    const int *k;
    int off;
    long long ld;
};
static inline ColRef col_none() { return ColRef{nullptr, 0, 0}; }
static inline ColRef col_at(const int *k, int off, long long ld) { return ColRef{k, off, ld}; }
#ifdef __CUDACC__
__device__ __forceinline__ size_t col_offset(const ColRef &c) {
    return c.k ? (size_t)(*c.k + c.off) * (size_t)c.ld : 0;
}
#endif

// ---- projector launchers (projectors.cu) --------------------------------
// Stage x (n elements of type `dtype`, a CTG_BASIS_* value; column xc of a
// basis at x when xc.k is set) for the forward projector.
cudaError_t ctg_launch_pad(const void *x, int dtype, float2 *pad, int N, const PadLayout &pl,
                           cudaStream_t st, ColRef xc = col_none());
// Stage two images for ctg_launch_forward2, interleaved: x (type `dtype`,
// column xc of a basis when xc.k is set) and x2 (FP32).  pad2 holds twice
// the floats of pl (PadLayout::floats * 2).
cudaError_t ctg_launch_pad2(const void *x, int dtype, ColRef xc, const float *x2, float4 *pad2, int N,
                            const PadLayout &pl, cudaStream_t st);
// Forward projector block shapes, the tile autotuner's candidates: angles
// per block x angles per warp (a warp holds 32 / angles-per-warp adjacent
// rays of each of its angles).  Every shape gives the same result bit for
// bit.  Shapes with several angles per warp are used only where
// ctg_forward_split_safe holds for the geometry.
constexpr int kFwdShapes = 4;
constexpr int kFwdShapeAngles[kFwdShapes] = {8, 4, 8, 16};
constexpr int kFwdShapeSplit[kFwdShapes] = {1, 1, 4, 4};
// Forward shapes of batched launches: shape 0 (kBatchFwdAngles angles per
// block, one per warp), or kBatchFwdSplitShape when every instance of the
// round allows several angles per warp.
constexpr int kBatchFwdAngles = 8;
constexpr int kBatchFwdSplitShape = 3;
// shape: an index into the tables above.  order: NULL, or the device copy
// of ctg_forward_order's permutation for the same shape.
cudaError_t ctg_launch_forward(const float2 *pad, int N, const PadLayout &pl, int n_angles,
                               int n_det, const FwdAngle *tab, float *b, cudaStream_t st,
                               int shape = 0, const int *order = nullptr);
// b = A x and b2 = A x2 in one walk, from the interleaved staging of
// ctg_launch_pad2; each ray's sums equal ctg_launch_forward's bit for bit.
cudaError_t ctg_launch_forward2(const float4 *pad2, int N, const PadLayout &pl, int n_angles, int n_det,
                                const FwdAngle *tab, float *b, float *b2, cudaStream_t st, int shape = 0,
                                const int *order = nullptr);
// Blocks of one forward launch of `shape`.
int ctg_fwd_shape_blocks(int shape, int n_angles, int n_det);
// Dispatch order of the forward projector's blocks of `shape` (tile index
// by * gx + bx, bx the ray group and by the angle group): longest estimated
// walk first, which shortens the tail of the launch where the chord
// lengths, and so the blocks' run times, differ.  From the host copy of the
// angle table.
void ctg_forward_order(const FwdAngle *host_tab, int N, int n_angles, int n_det, int shape,
                       std::vector<int> &order);
// Whether every lane of a warp holding `split` angles stays inside the
// staged image's border over its warp's whole walk (checked at both ends of
// a walk a few steps wider than the kernel's, in the kernel's fixed point).
// Adjacent angles of a fine angular sampling pass; widely spaced ones, whose
// chords differ, may not.
bool ctg_forward_split_safe(const FwdAngle *host_tab, int N, int n_angles, int n_det,
                            const PadLayout &pl, int split);
// Detector-window width (in bins) that the tiled back projector stages per
// angle, from the host copy of the angle table.
int ctg_back_window(const BackAngle *host_tab, int n_angles);
// x = B b (+ add, if add != NULL); b has element type `dtype`; window from
// ctg_back_window
// back_chunk: angles staged per pass, 16, 32 or 64 (tuned like the forward shape;
// the result does not depend on it).
// bc: the input is column bc of a basis at b (bc.k set), or b itself.
cudaError_t ctg_launch_back(const void *b, int dtype, int N, int n_angles, int n_det,
                            const BackAngle *tab, int window, const float *add, float *x,
                            cudaStream_t st, int back_chunk = 32, ColRef bc = col_none());

// ---- matched back projector (matched.cu) ----------------------------------
// x = B_thr b (+ add): the transpose of the forward projector, keeping the
// terms whose weight is >= thr (thr = 0: A^T exactly); rm = extra detector
// bins on each side beyond the two nearest (0 when ds >= max |c|).
cudaError_t ctg_launch_back_matched(const void *b, int dtype, int N, int n_angles, int n_det,
                                    const BackAngle *tab, const MatchedAngle *mt, int rm, float thr,
                                    const float *add, float *x, cudaStream_t st, ColRef bc = col_none());
// The same with the tiled design of the pixel-driven B (projectors.cu), for
// rm = 0 and window <= ctg_back_window_max().
cudaError_t ctg_launch_back_matched_tiled(const void *b, int dtype, int N, int n_angles, int n_det,
                                          const BackAngle *tab, int window, const MatchedAngle *mt,
                                          float thr, const float *add, float *x, cudaStream_t st,
                                          ColRef bc = col_none());
// *max_bits = bit pattern of max_ij A_ij (a float >= 0), on the device.
cudaError_t ctg_matched_max(int N, int n_angles, int n_det, const BackAngle *tab,
                            const MatchedAngle *mt, int rm, unsigned *max_bits, cudaStream_t st);

// ---- NCP stopping criterion (ncp.cu) --------------------------------------
constexpr int kCtgNcpMaxDet = 8192;
// *out (device double) = mean over the n_angles projections of the NCP
// distance of the residual sinogram r (n_angles x n_det); tw[j] =
// (cos, -sin)(2 pi j / n_det); dist_scratch: n_angles doubles.
cudaError_t ctg_ncp(const float *r, int n_angles, int n_det, const float2 *tw, double *dist_scratch,
                    double *out, cudaStream_t st);

// ---- Krylov kernels (arnoldi.cu) -----------------------------------------
// Reduction scratch for one vector length L and up to kmax coefficients.
struct RedScratch {
    float *partials;       // (kmax + 2) * grid floats
    double *h1, *h2;       // kmax + 2 doubles each
    double *scal;          // 8 doubles: [0] = ||q_pre||^2, [1] = ||q||^2, ...
    unsigned int *counter; // 4 words, zero between solves: [0] the last-block
                           // ticket of a reduction, [1] the fused step's
                           // grid-barrier arrivals, [2] its timeout flag
    int grid;              // blocks of every reduction pass for this L
    int E;                 // float4 groups per thread
    int rows = 0;          // partial-sum rows available (kmax + 2, or 2k + 2 for a fused step)
};
// Blocks a reduction pass aims for: 2 on every SM of the current device
// (queried once per device; 2 x 152 when no device can be queried).
int ctg_target_grid();
int ctg_red_grid(int64_t L, int *E_out);
size_t ctg_red_scratch_bytes(int64_t L, int kmax);
void ctg_red_scratch_carve(void *base, int64_t L, int kmax, RedScratch *rs);

// Basis element size in bytes for a CTG_BASIS_* type (0 if unknown).
static inline size_t ctg_basis_bytes(int dtype) {
    return dtype == CTG_BASIS_FP32 ? 4 : (dtype == CTG_BASIS_BF16 || dtype == CTG_BASIS_FP16) ? 2 : 0;
}

// Polls of a bounded device-side wait (about 100 ns apart) before it gives
// up: about half a second.
constexpr long long kCtgDefaultSpinLimit = 1LL << 22;

// One CGS2 Arnoldi step: orthogonalise the FP32 vector q (length L) against
// k vectors of W (element type `dtype`, stride ldw elements),
// h_out[0..k-1] = h1 + h2, h_out[k] = ||q||, and write w_out = q / ||q||
// (rounded to `dtype`) when ||q|| > 0.  Also leaves ||q_pre||^2 in
// rs.scal[0].
// *nkern (if given) = the kernels launched: 1 for the fused step (small k,
// scratch and residency permitting), else 3 (2 when k = 0).  The fused
// step's grid barriers give up after spin_limit polls, setting
// rs.counter[2] and h_out[0..k] to NaN.
cudaError_t ctg_cgs2_step(const void *W, int dtype, int64_t ldw, int64_t L, int k, float *q,
                          void *w_out, double *h_out, const RedScratch &rs, cudaStream_t st,
                          int *nkern = nullptr, long long spin_limit = kCtgDefaultSpinLimit);
// A CGS2 step inside a captured solver loop: k >= 1 is read on the device
// (*k), the new vector goes to column k of W and the Hessenberg column to
// H + (k - 1) ldh; kmax bounds k (it sizes shared memory); fused selects
// the one-launch step (needs ctg_cgs2_fused_ok) or the three passes.
// ||q_pre||^2 is left in rs.h1[k].
struct LoopBufs;
struct LoopStep {
    const int *k;
    double *H;
    long long ldh;
    int kmax;
    bool fused;
    // with the fused step: the loop whose Givens update (and, by giv_mode's
    // end flag, the end of the step) block 0 runs once the column is known;
    // giv_mode < 0: none
    const LoopBufs *lb;
    int giv_mode;
    // the fused step on one block per SM (small k, L2-resident basis: fewer
    // blocks make the grid barriers and the summation tails shorter)
    bool small_grid;
};
cudaError_t ctg_cgs2_step_loop(const void *W, int dtype, int64_t ldw, int64_t L, float *q, const LoopStep &ls,
                               const RedScratch &rs, long long spin_limit, bool cooperative, cudaStream_t st,
                               int *nkern = nullptr);
// Whether the fused step serves k <= kmax at length L with this scratch
// (every block of its grid resident at once).
bool ctg_cgs2_fused_ok(int dtype, int64_t L, int kmax, const RedScratch &rs, bool small_grid = false);
// The largest k a solver runs the fused step on one block per SM.
int ctg_cgs2_small_grid_max();
// The largest k the fused step serves: smaller for solver steps that also
// form y_k in the step (need_y), whose packed triangle takes shared memory.
int ctg_cgs2_fused_max(bool need_y);
// out = base + sum_j y_j W_j (base may be NULL); y: k doubles (device); with
// kdev set, k = *kdev + koff read on the device (k is then only the bound
// that sizes the launch's shared memory).
cudaError_t ctg_gemv(const void *W, int dtype, int64_t ldw, int64_t L, int k, const double *y,
                     const float *base, float *out, cudaStream_t st, const int *kdev = nullptr,
                     int koff = 0);
// out = a - c (c may be NULL -> out = a) and *res = ||a - c||^2 (double, device).
cudaError_t ctg_sub_norm2(const float *a, const float *c, float *out, int64_t L,
                          double *res, const RedScratch &rs, cudaStream_t st);
// out = v / sqrt(*nrm2) rounded to `dtype` (nrm2 on device; out = 0 when
// nrm2 == 0).
cudaError_t ctg_scale(const float *v, const double *nrm2, void *out, int dtype, int64_t L,
                      cudaStream_t st);

// ---- the device-driven GMRES loop (gmres_loop.cu) ---------------------------
// Stopping rules of a solve: maxit only, the discrepancy principle, NCP.
enum { kRuleMaxit = 0, kRuleDP = 1, kRuleNCP = 2 };
// Device state of one AB-/BA-GMRES solve.  The kernels of a step read k
// here; the step's last kernel advances it or stops the solve.
struct GmresState {
    int k;                // the step being performed (1-based)
    int active;           // 1 while iterating
    int iters;            // k of the iterate to return
    int stop_reason;      // CTG_STOP_*
    int pending;          // breakdown / maxit seen by the Givens kernel (CTG_STOP_* + 1), for the step's end
    int steps;            // steps executed
    int timed_out;        // a CGS2 grid barrier gave up
    int variant, rule, maxit;
    double target;        // tau ||e||
    double beta;          // ||r0||
    double rho;           // |g_{k+1}| of the latest step (at exit: of the returned iterate)
    double resnorm;       // latest ||b - A x_k|| (BA with DP / NCP; at exit: of the returned iterate)
    double res0;          // ||b - A x0||
    double dprev;         // NCP: the previous step's distance
};
// Where the loop kernels find a solve's state (device pointers).
struct LoopBufs {
    GmresState *S;
    double *H;            // Hessenberg matrix, column-major, leading dimension ldh
    long long ldh;
    double *gc, *gs, *gg; // Givens cosines, sines (maxit) and rotated right-hand side (maxit + 1)
    double *R;            // rotated columns (upper triangle), column-major, leading dimension ldr
    int ldr;              // = maxit
    double *y;            // y of the latest step / of the returned iterate (maxit)
    double *yring;        // y_j at yring + (j % 3) ldr (NCP returns x_{k-1})
    double *z;            // AB NCP: coefficients of r_k in W_{k+1} (maxit + 1)
    double *hist;         // ctg_info history (maxit + 1)
    double *rhoh;         // rho_k (maxit + 1)
    double *ncph;         // NCP distances (maxit + 2)
    double *scal;         // the reduction scratch's scalars
    double *h1;           // the reduction scratch's h1 (h1[k] = ||q_pre||^2)
    unsigned *counter;    // the reduction scratch's counters ([2]: barrier timeout)
    cudaGraphConditionalHandle c_small, c_fused, c_pass;   // while-loop conditions (in_graph)
    int in_graph;
    int small_max;        // last k of the loop of fused steps on one block per SM (0: none)
    int fused_max;        // last k of the fused-CGS2 loop
};
// Modes of a step's Givens update: y_k every step (kGivY), AB NCP's
// residual coefficients (kGivZ), the update ends the step (kGivEnd).
enum { kGivY = 1, kGivZ = 2, kGivEnd = 4 };
cudaError_t ctg_loop_init(const LoopBufs &B, int variant, int rule, int maxit, double target, cudaStream_t st);
// need_y: y_k every step; need_z: AB NCP residual coefficients; end: the
// Givens kernel ends the step (AB with DP or maxit)
cudaError_t ctg_loop_givens(const LoopBufs &B, bool need_y, bool need_z, bool end, int maxit, cudaStream_t st);
// ||b - Ax||^2 (r_out: NULL or where b - Ax goes); decide: end the step (BA, DP)
cudaError_t ctg_loop_resid(const LoopBufs &B, const float *b, const float *Ax, float *r_out, int64_t L,
                           const RedScratch &rs, bool decide, cudaStream_t st);
cudaError_t ctg_loop_ncp_decide(const LoopBufs &B, cudaStream_t st);
cudaError_t ctg_loop_advance(const LoopBufs &B, cudaStream_t st);
cudaError_t ctg_loop_exit_y(const LoopBufs &B, int maxit, cudaStream_t st);
cudaError_t ctg_loop_final(const LoopBufs &B, cudaStream_t st);

// ---- LSQR / LSMR (lsq.cu) --------------------------------------------------
// Device state of one LSQR or LSMR solve (Golub-Kahan bidiagonalisation with
// the scalar recurrences on the device, so the host only watches `live`).
// The vectors u are kept unnormalised (u~ = beta u).  Written by the host
// at the start, then only by the kernels.
struct LsqState {
    double alpha2, beta2;         // ||v~||^2, ||u~||^2 of the latest bidiagonalisation step
    double alpha, beta;           // alpha_k, beta_k (normalisers of v_k, u_k)
    double rhobar, phibar;        // LSQR
    double alphabar, zetabar, rho_old, rhobar_old, cbar, sbar;   // LSMR
    double inv_alpha;             // 1 / alpha_{k+1} for the update
    double cx, cw;                // LSQR: x += cx w, w = v - cw w
    double chbar, ch, ch_prev;    // LSMR: hbar = h - chbar hbar, x += cx hbar, h = v - ch h
    double r2;                    // LSMR: ||r_k||^2 of the tracked residual
    double target;                // tau ||e|| (0: no discrepancy stop)
    double *hist;                 // residual history (maxit + 1 doubles, device)
    int method;                   // CTG_LSQR / CTG_LSMR
    int k, maxit;                 // iteration being performed
    int live;                     // 1 while iterating
    int live_update;              // the current iteration's update is applied
    int iters, stop_reason;
    double status[2];             // {live, latest residual estimate} for the host
};
// u = p - (alpha/beta) u, state->beta2 = ||u||^2
cudaError_t ctg_lsq_bidiag_u(const float *p, float *u, int64_t m, LsqState *state,
                             const RedScratch &rs, cudaStream_t st);
// v = q / beta' - beta' v with beta' = sqrt(state->beta2), state->alpha2 = ||v||^2
cudaError_t ctg_lsq_bidiag_v(const float *q, float *v, int64_t n, LsqState *state,
                             const RedScratch &rs, cudaStream_t st);
// rotations and update coefficients of iteration k, the stopping rules
cudaError_t ctg_lsq_scalars(LsqState *state, cudaStream_t st);
// LSQR: v /= alpha, x += cx w, w = v - cw w; LSMR: v /= alpha,
// hbar = h - chbar hbar, x += cx hbar, h = v - ch h (a = w or h, c = hbar)
cudaError_t ctg_lsq_update(const LsqState *state, float *v, float *a, float *c, float *x,
                           int64_t n, cudaStream_t st);
// LSMR residual r_k = b - A x_k tracked in sinogram space from p = A v_k:
// Ah = p - ch_prev Ah, Ahbar = Ah - chbar Ahbar, r -= cx Ahbar, r2 = ||r||^2;
// then the discrepancy test on it
cudaError_t ctg_lsq_residual(LsqState *state, const float *p, float *Ah, float *Ahbar, float *r,
                             int64_t m, const RedScratch &rs, cudaStream_t st);
// start: v = v~ / alpha_1 and w = v (LSQR) or h = v, hbar = 0 (LSMR)
cudaError_t ctg_lsq_start(const LsqState *state, float *v, float *a, float *c, int64_t n,
                          cudaStream_t st);

// ---- batched engine (batch.cu; kernels in projectors.cu and arnoldi.cu) ----
// Device-resident state of one instance (one solve) of a batch.  A round of
// the batch advances every active instance by one Arnoldi step (k -> k+1)
// with one launch per kernel for all instances; kernels read k and the
// activity flag from here, so one captured CUDA graph serves every round.
struct BatchInst {
    // geometry
    int N, n_angles, n_det, variant;      // variant: CTG_AB / CTG_BA
    const FwdAngle *fwd;
    const BackAngle *back;
    int back_window;
    int pad_stride, pad_border, pad_clamp;
    long long n, m, L;
    // iteration state
    int k;                // the step to perform: orthogonalise against w_1..w_k
    int active;           // 1 while iterating
    int maxit;
    int stop_reason;
    int iters;
    int breakdown;        // set by the Givens kernel for the finish kernel
    double target;        // tau ||e|| (<= 0: no discrepancy stop)
    double rho;           // last GMRES residual |g_{k+1}|
    double resnorm;       // last ||b - A x_k|| (BA with the DP stop)
    // buffers (the basis in FP32, BF16 or FP16; everything else FP32 / FP64)
    void *W;              // (maxit + 1) x ldw elements of type wtype
    long long ldw;
    double *H;            // (maxit + 1) x maxit, column-major, unrotated
    double *R;            // maxit x maxit, column-major: rotated H (upper triangle)
    double *gc, *gs, *gg; // Givens cosines, sines (maxit), rotated rhs (maxit + 1)
    double *y;            // maxit: the least-squares solution y_k (BA with the DP stop, and at exit)
    double *hist;         // maxit + 1: history as in ctg_info
    float *vn, *vm;       // work vectors of length n and m (BA: vm holds t_k = A w_k)
    float *vr;            // BA with the DP stop: A x_k
    float2 *pad;          // staged image for the forward projector
    float4 *pad2;         // BA with the DP stop: staging of w_{k+1} and x_k, interleaved
    const float *b;       // the solve's data b (m floats), start x0 (or NULL) and
    const float *x0;      // iterate x (n floats; BA with the DP stop forms x_k
    float *x;             // there every round)
    // reduction scratch of this instance (E = 1 passes, grid G)
    float *partials;
    double *h1, *h2, *scal;
    unsigned *counter;
    int G;                // blocks of this instance's CGS2 / vector passes
    int back_model;       // CTG_BACK_*: the tiled pixel-driven B, A^T or B_tau
    const MatchedAngle *mt;   // A^T / B_tau weights (back_model != CTG_BACK_PIXEL)
    float back_thr;       // B_tau threshold tau max(A) (0: A^T)
    int wtype;            // CTG_BASIS_*: element type of the stored basis W
};

// Block maps: entry b of a batched launch's map is (instance, local block).
// The back projection of a round: q = B w_k (AB) or q = B t_k (BA, t_k = A
// w_k from the round before).  wtype: CTG_BASIS_FP32 launches the kernel
// for AB instances with an FP32 basis and all BA instances; BF16 / FP16
// launch it for the AB instances whose basis has that type.
// chunk: angles staged per pass, 16, 32 or 64 (ctg_batch_back_chunk_ok;
// otherwise 32); the result does not depend on it.
cudaError_t ctg_batch_back(BatchInst *insts, const int2 *map, int nblocks, int max_window,
                           cudaStream_t st, int wtype = CTG_BASIS_FP32, int chunk = 32);
bool ctg_batch_back_chunk_ok(int chunk, int max_window);
// Staging for the forward projector: AB stages t = B w_k (variant CTG_AB);
// BA stages w_{k+1}, with x_k interleaved when it has the DP stop
// (variant CTG_BA).
cudaError_t ctg_batch_pad(BatchInst *insts, const int2 *map, int nblocks, int variant, cudaStream_t st);
// The forward projection: AB q = A t; BA t_{k+1} = A w_{k+1} and, with the
// DP stop, A x_k in the same walk.  shape: 0, or kBatchFwdSplitShape when
// every instance of the launch allows it (ctg_forward_split_safe); the
// map's local blocks are that shape's.
cudaError_t ctg_batch_forward(BatchInst *insts, const int2 *map, int nblocks, int variant, cudaStream_t st,
                              int shape = 0);
// Local block counts of one instance for the maps above.
int ctg_back_tiles(int N);
int ctg_pad_tiles(int N);
int ctg_fwd_blocks(int n_angles, int n_det);
int ctg_back_window_max();
// the three CGS2 passes and the scaling for the instances in `map`, whose
// basis has element type wtype
cudaError_t ctg_batch_cgs2(BatchInst *insts, const int2 *map, int nblocks, int max_k,
                           cudaStream_t st, int wtype = CTG_BASIS_FP32);
// Set the batched kernels' shared-memory attributes (before graph capture).
cudaError_t ctg_batch_prepare(int max_k);
cudaError_t ctg_batch_givens(BatchInst *insts, int n_inst, int max_k, cudaStream_t st);
// BA with the DP stop: x_k = x0 + W_k y_k (map over n-blocks of those
// instances), and ||b - A x_k||^2 (map over their m-blocks) into scal[4].
cudaError_t ctg_batch_iterate(BatchInst *insts, const int2 *map_n, int nblocks, int max_k, cudaStream_t st);
cudaError_t ctg_batch_residual(BatchInst *insts, const int2 *map_m, int nblocks, cudaStream_t st);
cudaError_t ctg_batch_finish(BatchInst *insts, int n_inst, int *active_count, cudaStream_t st);
// The stopping rules of a round of a batch's while-loop graph (n_inst <=
// 1024): ctl[0] active solves, ctl[1] rounds run, ctl[3] set when a fused
// step's wait gave up (every solve then stops).  Ends both loops (handles
// h and h_next) when no solve is active, after max_rounds rounds or after a
// timeout; with fused_max > 0 (the loop of fused steps) it also ends loop h
// alone once an active solve's next step is beyond fused_max.
cudaError_t ctg_batch_finish_loop(BatchInst *insts, int n_inst, int *ctl, int max_rounds,
                                  cudaGraphConditionalHandle h, cudaStream_t st,
                                  cudaGraphConditionalHandle h_next = 0, int fused_max = 0);
// Exit: y = R^{-1} g for the instance's final k.
cudaError_t ctg_batch_solve_y(BatchInst *insts, int n_inst, int max_k, cudaStream_t st);
int ctg_vec_blocks(long long L);          // blocks of an E = 1 vector pass over L

// The batched one-launch CGS2 step with each instance's Givens update
// (steps k <= ctg_batch_fused_max_k()): kBatchFusedE float4 groups per
// thread, batch_fused_blocks(L) blocks per instance, one cooperative launch
// per basis type whose blocks must all be resident at once.
constexpr int kBatchFusedE = 4;
__host__ __device__ inline int batch_fused_blocks(long long L) {
    return (int)(((L + 3) / 4 + 256LL * kBatchFusedE - 1) / (256LL * kBatchFusedE));
}
int ctg_batch_fused_max_k();
// Blocks of one fused launch that fit at once for steps up to kcap (0 if
// the occupancy query fails).
int ctg_batch_fused_resident(int kcap, int wtype);
// bar: barrier arrivals (zero at launch), err: set when a bounded wait gave
// up, spin_limit: the polls a wait may take (device memory, read at
// launch); kcap: the largest k of the launch (<= ctg_batch_fused_max_k()).
cudaError_t ctg_batch_cgs2_fused(BatchInst *insts, const int2 *map, int nblocks, int kcap, unsigned *bar,
                                 int *err, const long long *spin_limit, cudaStream_t st,
                                 int wtype = CTG_BASIS_FP32);
// Allow `bytes` of dynamic shared memory for a kernel: set only when its
// static and dynamic shared memory together pass the default 48 KB.
inline cudaError_t ctg_allow_dyn_smem(const void *kernel, size_t bytes) {
    cudaFuncAttributes a;
    const cudaError_t e = cudaFuncGetAttributes(&a, kernel);
    if (e != cudaSuccess) return e;
    if (a.sharedSizeBytes + bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}
// The context's bounded-wait limit (ctg_set_wait_limit).
long long ctg_ctx_wait_limit(const ctg_ctx *ctx);
// Tile shapes forced on the context (ctg_set_tiles / ctg_set_fwd_tiles):
// *fwd_split 0 when the forward shape is not forced, else its angles per
// warp; *back_chunk 0 when not forced.
void ctg_ctx_forced_tiles(const ctg_ctx *ctx, int *fwd_split, int *back_chunk);

// ---- host helpers shared by api.cu and batch.cu --------------------------
bool ctg_geom_valid(const ctg_geom *g);
// Matched-projector weights of a geometry (api.cu); *rm = extra bins beyond
// the two nearest that the widest angle needs (0: the tiled kernels apply).
void ctg_build_matched(const ctg_geom *g, std::vector<MatchedAngle> &mt, int *rm);
bool ctg_opts_valid(const ctg_opts *o);
void ctg_build_tables(const ctg_geom *g, std::vector<FwdAngle> &fw, std::vector<BackAngle> &bk);
