/*
 * ctgmres: AB-GMRES and BA-GMRES for 2D parallel-beam CT with an unmatched
 * back projector B != A^T, on one NVIDIA GB300 (sm_103a).
 *
 * Problem (paper Sec. 1, eq. (1.1)): A x ~ b with b = A x_bar + e,
 * A in R^{m x n} the forward projector, B in R^{n x m} the back projector,
 * n = N^2 pixels, m = n_angles * n_det rays.  The solvers (Sec. 2, algorithm
 * box) build the Krylov space K_k(BA, B r0) and minimise ||b - A x|| (AB) or
 * ||B b - B A x|| (BA); the discrepancy principle (Sec. 6.4) stops at the
 * first k with ||b - A x_k|| <= tau ||e||.
 *
 * Discretisation (the paper names ASTRA's interpolation/Joseph model for A
 * but gives no formulas; this is the library's fixed reading):
 *   pixel (i, j) (row i, column j) has centre (j - (N-1)/2, i - (N-1)/2),
 *   pixel size 1; angle a is theta_a = start + a * range / n_angles degrees
 *   (start and range integers, endpoint excluded); detector d has centre
 *   s_d = (d - (n_det-1)/2) * det_spacing; ray (a, d) is the line
 *   x cos(theta_a) + y sin(theta_a) = s_d.
 *   A (Joseph): rays with theta mod 180 in [0, 45] or [135, 180) step over
 *   image rows, the others over columns; per step one linear interpolation
 *   between the two nearest pixels (pixels outside the image are 0), the
 *   sum scaled by 1/|cos| (rows) or 1/|sin| (columns).
 *   B (pixel-driven): (B b)[i, j] = sum_a lerp of b[a, .] at detector
 *   position u = (x_j cos + y_i sin)/det_spacing + (n_det-1)/2; bins outside
 *   the detector are 0.  B gathers only; it is not the transpose of A.
 *
 * Layouts: image x[i * N + j] (row-major float32); sinogram b[a * n_det + d]
 * (angle-major float32).  All vectors are caller-owned DEVICE memory unless
 * stated otherwise.
 *
 * Errors: every int-returning call returns CTG_OK (0) or a negative status;
 * ctg_status_string() names it.  Invalid arguments are rejected on the host
 * before any launch.  Calls enqueue work on `stream` (a cudaStream_t; NULL is
 * the legacy default stream) and return without waiting, except the two
 * solvers, which synchronise `stream` before returning to fill ctg_info.
 */
#ifndef CTGMRES_H
#define CTGMRES_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    CTG_OK = 0,
    CTG_ERR_INVALID_ARG = -1,  /* bad geometry, null pointer, size or option */
    CTG_ERR_OOM = -2,          /* device allocation failed                   */
    CTG_ERR_CUDA = -3,         /* a CUDA runtime call failed                 */
    CTG_ERR_TIMEOUT = -4,      /* a bounded device-side wait gave up         */
    CTG_ERR_WORKSPACE = -5,    /* caller workspace smaller than required     */
    CTG_ERR_BUSY = -6          /* serving engine: no free slot, or the
                                  request does not fit the memory budget now;
                                  retry after a completion                   */
};

enum { CTG_AB = 0, CTG_BA = 1, CTG_LSQR = 2, CTG_LSMR = 3 };                       /* solver variant    */
enum { CTG_STOP_MAXIT = 0, CTG_STOP_DP = 1, CTG_STOP_BREAKDOWN = 2, CTG_STOP_NCP = 3 };
/* Stopping rule (Sec. 6.4).  CTG_RULE_DP: the discrepancy principle when
 * noise_norm > 0, else maxit.  CTG_RULE_NCP: the NCP criterion (see
 * ctg_ncp_distance): the solve returns x_k at the first k with
 * d_{k+1} > d_k, d_k the NCP distance of b - A x_k (noise_norm is not
 * used); needs 2 <= n_det <= 8192. */
enum { CTG_RULE_DP = 0, CTG_RULE_NCP = 1 };
enum { CTG_BASIS_FP32 = 0, CTG_BASIS_BF16 = 1, CTG_BASIS_FP16 = 2 };  /* basis storage */
/* Back projector B of a geometry.
 * CTG_BACK_PIXEL: the unmatched pixel-driven back projector (linear
 *   interpolation on the detector at each pixel centre), the paper's B.
 * CTG_BACK_MATCHED: B = A^T, the exact transpose of the Joseph forward
 *   projector (the matched case of Sec. 5).
 * CTG_BACK_THRESHOLD: B_tau of Sec. 6.5, eq. (Btau): (B_tau)_ij = A_ji where
 *   A_ji >= back_tau * max(A), else 0; max(A) is taken over all entries of A
 *   (computed once per geometry on the device, in FP32). */
enum { CTG_BACK_PIXEL = 0, CTG_BACK_MATCHED = 1, CTG_BACK_THRESHOLD = 2 };

/* 2D parallel-beam geometry (paper Sec. 6.1, Table 1).  Limits: 1 <= N <=
 * 16384, 1 <= n_angles, 1 <= n_det <= 65536, start and range integral
 * degrees with 0 < range <= 360, det_spacing > 0, n_det * det_spacing <=
 * 2^20, 1.5 N / det_spacing + n_det < 2^22; back_tau in [0, 1] for
 * CTG_BACK_THRESHOLD and 0 otherwise. */
typedef struct {
    int32_t N;                /* image side; n = N * N pixels               */
    int32_t n_angles;         /* N_ang                                      */
    int32_t n_det;            /* N_det                                      */
    int32_t back_model;       /* CTG_BACK_PIXEL, _MATCHED or _THRESHOLD     */
    double angle_start_deg;   /* theta_0, integer degrees                   */
    double angle_range_deg;   /* angles span [start, start + range)        */
    double det_spacing;       /* detector pitch in pixel units (1 = pixel)  */
    double back_tau;          /* threshold tau of B_tau                      */
} ctg_geom;

/* Solver options. */
typedef struct {
    int32_t maxit;            /* iteration cap, >= 1                        */
    int32_t basis_dtype;      /* CTG_BASIS_FP32, _BF16 or _FP16: element type
                                 of the stored Krylov basis W; arithmetic is
                                 FP32 (cross-block sums as compensated FP32
                                 pairs with FP64 results; FP64 for the
                                 Hessenberg problem) in every case         */
    double tau;               /* DP safety factor tau >= 1 (Sec. 6.4)       */
    double noise_norm;        /* ||e||; <= 0 disables the DP stop           */
    int32_t stop_rule;        /* CTG_RULE_DP or CTG_RULE_NCP                */
} ctg_opts;

/* Solver report, filled on return (host memory). */
typedef struct {
    int32_t iters;            /* k of the returned iterate x_k (0 = x0)     */
    int32_t stop_reason;      /* CTG_STOP_*                                 */
    double resnorm;           /* ||b - A x_k|| of the returned iterate,
                                 recomputed from x_k in FP32/FP64           */
    double rho;               /* GMRES residual: | ||r0|| e1 - H_k y_k |    */
    double *history;          /* optional caller host array, >= maxit + 1
                                 entries, or NULL: entry k = ||b - A x_k||
                                 as used by the DP test (AB: the Hessenberg
                                 residual, equal in exact arithmetic)      */
    double *ncp_history;      /* optional caller host array, >= maxit + 2
                                 entries, or NULL: with CTG_RULE_NCP, entry
                                 k = the NCP distance d_k, for k = 0 .. the
                                 last step evaluated (iters + 1 at an NCP
                                 stop)                                      */
} ctg_info;

/* Where the solver keeps its state inside a caller workspace (byte offsets
 * from the workspace base).  The basis W holds vectors w_1..w_{k+1}, each of
 * length L (L = m for AB, n for BA) at stride ld_w floats (ld_w >= L, a
 * multiple of 64); H is the FP64 (maxit+1) x maxit Hessenberg matrix stored
 * column by column with leading dimension maxit+1 (h_{i,k} at
 * H[(k-1) * (maxit+1) + (i-1)]). After a solve these hold the final basis
 * and Hessenberg matrix, so callers can inspect them. */
typedef struct {
    size_t off_w;
    size_t ld_w;              /* in elements                               */
    size_t off_h;
    size_t total_bytes;       /* == ctg_workspace_bytes()                  */
} ctg_layout;

typedef struct ctg_ctx ctg_ctx;

/* Create / destroy a context on the current CUDA device.  The context caches
 * per-geometry angle tables and a pinned host staging area; it is not
 * thread-safe (use one context per host thread). */
int ctg_create(ctg_ctx **out);
void ctg_destroy(ctg_ctx *ctx);

/* b = A x: Joseph forward projection (eq. (1.1)).
 * x: n floats (device, read-only); b: m floats (device, overwritten).
 * Needs no workspace beyond a context-owned padded image copy (allocated on
 * first use per geometry; CTG_ERR_OOM if that fails). */
int ctg_project(ctg_ctx *ctx, const ctg_geom *g, const float *x_dev,
                float *b_dev, void *stream);

/* x = B b with the geometry's back projector: by default the pixel-driven
 * unmatched back projection (B in eq. (1.2)); A^T or B_tau (Sec. 6.5) when
 * g->back_model selects them.  b: m floats (device, read-only); x: n floats
 * (device, overwritten). */
int ctg_backproject(ctg_ctx *ctx, const ctg_geom *g, const float *b_dev,
                    float *x_dev, void *stream);

/* Projector tile shapes.  By default the context times, at the first use of
 * a geometry, the forward projector with 8 and 4 angles per block (one angle
 * per warp, 32 adjacent rays) and with 8 and 16 angles per block (4 angles
 * per warp, 8 adjacent rays of each), and the pixel-driven back projector
 * with 16, 32 and 64 angles staged per pass (CUDA events, 3 launches each on
 * zero inputs, with temporary buffers of about 5n + m floats), and keeps the
 * fastest.  The shapes with 4 angles per warp are candidates only where the
 * host has checked that every warp's walk stays inside the staged image
 * (adjacent angles of a fine angular sampling; not widely spaced ones).  The
 * candidates sum every ray and every pixel in the same order, so results do
 * not depend on the choice.  ctg_set_tiles forces shapes instead, the
 * forward one with one angle per warp (0, 0 restores autotuning);
 * ctg_set_fwd_tiles forces the forward shape as angles per block and per
 * warp, (4, 1), (8, 1), (8, 4) or (16, 4) ((0, 0): autotuned; a shape with
 * 4 angles per warp falls back to (8, 1) where the geometry does not allow
 * it).  Both take effect at each geometry's next use and return
 * CTG_ERR_INVALID_ARG for other values.  ctg_get_tuning reports the shapes
 * in use for a geometry (tuning it first if needed) and the measured times
 * (0 for a shape not timed). */
typedef struct {
    int32_t fwd_angles;       /* angles per forward block: 4, 8 or 16       */
    int32_t back_chunk;       /* 16, 32 or 64                               */
    int32_t tuned;            /* 1 if chosen by timing                      */
    float fwd_us[2];          /* measured: 8, 4 angles per block, 1 per warp */
    float back_us[3];         /* measured: 16, 32, 64 angles per pass       */
    int32_t fwd_warp_angles;  /* angles per warp of the forward shape: 1, 4 */
    float fwd_split_us[2];    /* measured: 8, 16 angles per block, 4 per warp */
} ctg_tuning;
int ctg_set_tiles(ctg_ctx *ctx, int32_t fwd_angles, int32_t back_chunk);
int ctg_set_fwd_tiles(ctg_ctx *ctx, int32_t angles_per_block, int32_t angles_per_warp);
int ctg_get_tuning(ctg_ctx *ctx, const ctg_geom *g, ctg_tuning *out);

/* The NCP distance of Sec. 6.4's NCP criterion for a residual sinogram r
 * (m floats, device): the paper defines the criterion by citation; reading
 * taken here: each projection (N_d bins of one angle) is a signal; with
 * q = floor(N_d / 2) and rhat its DFT, p_i = |rhat_i|^2 (i = 1..q, the zero
 * frequency left out), c_i = (p_1 + ... + p_i) / (p_1 + ... + p_q); the
 * distance of a projection is ||c - (1..q)/q||_2 (0 when p = 0), and *out
 * (host) is the mean over the projections.  Needs 2 <= n_det <= 8192;
 * synchronises `stream`. */
int ctg_ncp_distance(ctg_ctx *ctx, const ctg_geom *g, const float *r_dev, double *out, void *stream);

/* Bytes of device workspace a solve of `variant` (CTG_AB, CTG_BA, CTG_LSQR or
 * CTG_LSMR) with these options needs; 0 if the arguments are invalid.  For
 * the GMRES variants it is the basis, (maxit + 1) vectors of length L of
 * the basis type (L = m for AB, n for BA: the paper's storage law k * L,
 * Table 3), plus O(n + m) floats (one n-vector, two m-vectors, the staged
 * image) and O(maxit^2) doubles (the Hessenberg matrix and its rotated
 * form); LSQR and LSMR need O(n + m) whatever maxit. */
size_t ctg_workspace_bytes(const ctg_geom *g, int variant, const ctg_opts *o);

/* Fill *out with the workspace layout for these arguments (for CTG_LSQR and
 * CTG_LSMR only total_bytes is meaningful: they keep no basis). */
int ctg_workspace_layout(const ctg_geom *g, int variant, const ctg_opts *o,
                         ctg_layout *out);

/* AB-GMRES (Sec. 2, left column): x = x0 + B W_k y_k.
 * b: m floats; x0: n floats or NULL (x0 = 0); x: n floats (output).
 * workspace: device memory of >= workspace_bytes bytes, 256-byte aligned, or
 * NULL, in which case the library allocates and frees it per call.  The
 * caller owns b, x0, x and the workspace; none may alias another.  Runs on
 * `stream`, synchronises it before returning and fills *info (info may not
 * be NULL).  A breakdown (h_{k+1,k} <= 1e-6 ||A B w_k||) is reported in
 * info->stop_reason, not as an error.
 * The iteration runs on the device: the FP64 Givens update of the
 * Hessenberg least-squares problem, y_k and the stopping rule are device
 * kernels, and the whole solve is one CUDA graph (the start, while-loop
 * nodes over the steps, the exit) that the context captures on first use
 * and replays for later calls with the same pointers and options; the host
 * waits once, at the end.  With phase tracing on (ctg_set_timing) the same
 * kernels are enqueued step by step instead.  Returns CTG_ERR_TIMEOUT if a
 * bounded device-side wait gave up (ctg_set_wait_limit). */
int ctg_ab_gmres(ctg_ctx *ctx, const ctg_geom *g, const float *b_dev,
                 const float *x0_dev, float *x_dev, const ctg_opts *o,
                 void *workspace_dev, size_t workspace_bytes, ctg_info *info,
                 void *stream);

/* BA-GMRES (Sec. 2, right column): x = x0 + W_k y_k; same conventions.
 * The DP test (and the NCP rule) uses the true residual ||b - A x_k||: each
 * step forms x_k = x0 + W_k y_k and projects it in the same walk as the
 * next step's A w_{k+1} (one two-image forward projection), so the
 * workspace keeps no A W_k and its size follows the storage law k n.
 * With a BF16 basis at 1% noise the true residual was measured to level
 * off above tau ||e|| (the iterate is a combination of the rounded basis
 * vectors themselves), so the DP stop may never trigger and the solve then
 * runs to maxit; FP32 and FP16 bases reach it. */
int ctg_ba_gmres(ctg_ctx *ctx, const ctg_geom *g, const float *b_dev,
                 const float *x0_dev, float *x_dev, const ctg_opts *o,
                 void *workspace_dev, size_t workspace_bytes, ctg_info *info,
                 void *stream);

/* LSQR (Paige & Saunders) and LSMR (Fong & Saunders), no damping: the
 * matched-case comparators of Sec. 5, where AB-GMRES with B = A^T equals
 * LSQR and BA-GMRES with B = A^T equals LSMR in exact arithmetic.  The
 * geometry's back projector plays the role of A^T (CTG_BACK_MATCHED for the
 * methods proper; with an unmatched B they solve the unmatched normal
 * equations, which Sec. 5 notes is not well founded).  Same arguments and
 * ownership as ctg_ab_gmres; opts->basis_dtype must be CTG_BASIS_FP32 (there
 * is no basis: the workspace, ctg_workspace_bytes(g, CTG_LSQR or CTG_LSMR,
 * opts), is O(n + m) whatever maxit).  Short recurrences, no
 * reorthogonalisation.  Stopping: the discrepancy principle of Sec. 6.4 on
 * LSQR's residual estimate |phibar_{k+1}| = ||b - A x_k|| (exact in exact
 * arithmetic), and for LSMR on ||r_k|| tracked in sinogram space through the
 * recurrences of x_k; else maxit, or CTG_STOP_BREAKDOWN when alpha or beta
 * vanishes.  info->rho = the last residual estimate, info->resnorm =
 * ||b - A x|| recomputed, history[k] = the estimates. */
int ctg_lsqr(ctg_ctx *ctx, const ctg_geom *g, const float *b_dev, const float *x0_dev, float *x_dev,
             const ctg_opts *opts, void *workspace, size_t workspace_bytes, ctg_info *info,
             void *stream);
int ctg_lsmr(ctg_ctx *ctx, const ctg_geom *g, const float *b_dev, const float *x0_dev, float *x_dev,
             const ctg_opts *opts, void *workspace, size_t workspace_bytes, ctg_info *info,
             void *stream);

/* Batched AB-/BA-GMRES: n independent solves of possibly different
 * geometries, variants (CTG_AB / CTG_BA) and options advance together, one
 * Arnoldi step of every active solve per round (Sec. 2 algorithm box for
 * each), with the Hessenberg least-squares update (FP64 Givens) and the
 * discrepancy-principle stop (Sec. 6.4) done on the device.  A round is one
 * launch per phase for all solves and is replayed as a captured CUDA graph.
 * ctg_batch_create: geoms, variants, opts are arrays of n (any basis type,
 * mixed freely across solves; the CTG_RULE_DP stopping rule, maxit <= 1024, det_spacing >= ~0.25; any
 * back projector, A^T and B_tau only where two detector bins per pixel
 * suffice, i.e. det_spacing >= max |cos|, |sin|, which holds for
 * det_spacing >= 1); the batch owns its device workspace
 * (ctg_batch_workspace_bytes) and a stream of its own.  Invalid or
 * unsupported arguments return CTG_ERR_INVALID_ARG.
 *   At creation the batch times its forward and back projection launches in
 *   the tile shapes the result does not depend on and keeps the faster ones
 *   (shapes forced with ctg_set_tiles / ctg_set_fwd_tiles are used as given).
 * ctg_batch_solve: b_dev, x_dev: host arrays of n device pointers (m and n
 * floats of each solve); x0_dev: NULL or an array whose entries may be NULL;
 * infos: n reports, filled as by ctg_ab_gmres.  Work is ordered after prior
 * work on `stream`, and `stream` waits for it; the call returns when done.
 * Steps k <= 64 run every solve's CGS2 step and Givens update in one
 * cooperative launch per basis type when its blocks fit on the device at
 * once, later steps (or batches too large for that) the separate passes;
 * each solve's result does not depend on the others in the batch as long as
 * the batch takes the same form.  A wait of that launch that runs out (see
 * ctg_set_wait_limit) stops every solve at its last completed step, whose
 * iterate is formed and reported, and the call returns CTG_ERR_TIMEOUT. */
typedef struct ctg_batch ctg_batch;
int ctg_batch_create(ctg_ctx *ctx, int32_t n, const ctg_geom *geoms, const int32_t *variants,
                     const ctg_opts *opts, ctg_batch **out);
size_t ctg_batch_workspace_bytes(const ctg_batch *batch);
int ctg_batch_solve(ctg_batch *batch, const float *const *b_dev, const float *const *x0_dev,
                    float *const *x_dev, ctg_info *infos, void *stream);
void ctg_batch_destroy(ctg_batch *batch);

/* Serving engine: continuous batching of independent solves (the batched
 * rounds above, with solves joining and leaving between steps).
 * ctg_engine_create: at most max_slots solves in flight (1..4096), whose
 *   workspaces (allocated per solve, stream-ordered, from a memory pool of
 *   the engine that keeps up to hbm_budget_bytes mapped) together stay
 *   within hbm_budget_bytes.  Uses the current device.
 * ctg_engine_request_bytes: device bytes one solve occupies while in flight
 *   (its Krylov basis dominates: the storage law k L of Table 3), or 0 if the
 *   arguments are invalid or unsupported (the same conditions as for
 *   ctg_batch_create).
 * ctg_engine_submit: admits one solve, or returns CTG_ERR_BUSY if no slot is
 *   free or its bytes do not fit the remaining budget, CTG_ERR_OOM if they
 *   exceed the whole budget.  b_dev must be ready
 *   on `stream`; b_dev, x0_dev (or NULL), x_dev and history (NULL or maxit + 1
 *   doubles of host memory) must stay valid until the solve is reported.
 *   Computes r0 and starts the solve before returning.
 * ctg_engine_step: runs `rounds` Arnoldi rounds of every running solve, then
 *   forms the iterate x of up to max_done finished solves and reports their
 *   tags and ctg_info (x_dev is complete when reported) and releases their
 *   memory; *n_done is the number reported.  Returns when done.
 * ctg_engine_in_flight: solves admitted and not yet reported.
 * A solve's result does not depend on which others share the engine. */
typedef struct ctg_engine ctg_engine;
int ctg_engine_create(ctg_ctx *ctx, int32_t max_slots, size_t hbm_budget_bytes, ctg_engine **out);
size_t ctg_engine_request_bytes(const ctg_geom *g, int32_t variant, const ctg_opts *o);
int ctg_engine_submit(ctg_engine *engine, const ctg_geom *g, int32_t variant, const ctg_opts *o,
                      const float *b_dev, const float *x0_dev, float *x_dev, double *history,
                      int64_t tag, void *stream);
int ctg_engine_step(ctg_engine *engine, int32_t rounds, int32_t max_done, int64_t *done_tags,
                    ctg_info *done_infos, int32_t *n_done);
int32_t ctg_engine_in_flight(const ctg_engine *engine);
void ctg_engine_destroy(ctg_engine *engine);

/* One classical Gram-Schmidt step with reorthogonalisation (CGS2) of q
 * against the k orthonormal columns of W, the Arnoldi step of Sec. 2 with
 * MGS replaced by CGS2 (equal in exact arithmetic):
 *   h = W^T q; q -= W h; h' = W^T q; q -= W h';  h_out[0..k-1] = h + h',
 *   h_out[k] = ||q||, and, if h_out[k] > 0, w_out = q / ||q||.
 * ||q|| is formed as sqrt(||q1||^2 - ||h'||^2), q1 the vector after the
 * first pass, which is ||q1 - W h'|| exactly for orthonormal W and agrees
 * with the direct norm to rounding (h' is at the rounding level of ||q1||).
 * For k <= 128 the step is one cooperative launch when its grid fits on the
 * device at once, else three launches.
 * W: k vectors of length L at stride ld_w floats (ld_w >= L, multiple of
 * 4), device, read-only; q: L floats, device, overwritten by the
 * orthogonalised vector; w_out: L floats, device (may equal q);
 * h_out: k + 1 doubles, device; 0 <= k <= 4096.
 * scratch: device memory of >= ctg_cgs2_scratch_bytes(L, k) bytes (256-byte
 * aligned), owned by the caller; its contents need no initialisation. */
size_t ctg_cgs2_scratch_bytes(int64_t L, int32_t k);
int ctg_cgs2(const float *W_dev, int64_t ld_w, int64_t L, int32_t k,
             float *q_dev, float *w_out_dev, double *h_out_dev,
             void *scratch_dev, size_t scratch_bytes, void *stream);

/* ctg_cgs2 without caller scratch and without any allocation.  The paper
 * has no counterpart: this exists for callers that cannot call cudaMalloc,
 * for example an application whose memory manager has reserved all device
 * memory up front and forbids further allocations, or a plugin running
 * inside a host framework that owns every device allocation.
 * Same arguments and results as ctg_cgs2, minus the scratch.  The scratch is
 * a fixed 640 KiB array in device memory that is part of the library (every
 * GPU that loads the library holds it until the process exits); it serves
 * k <= 256 and L <= 4,980,736, and larger sizes return CTG_ERR_INVALID_ARG.
 * Each call looks up the array's device address on the current device
 * (so an address from a torn-down context is never reused); a call whose
 * stream is being captured uses the address that an earlier call on the
 * device found, so make the first call before any stream capture (a first
 * call under capture returns CTG_ERR_CUDA).  Every call on a device shares
 * the one array, which keeps the previous call's contents; each call first
 * clears the part that must start at zero.  Calls whose work overlaps on the GPU (for example on two streams)
 * race on the array and give wrong results: serialise them.
 * Calls no cudaMalloc, cudaFree or allocating library routine. */
int ctg_cgs2_noalloc(const float *W_dev, int64_t ld_w, int64_t L, int32_t k,
                     float *q_dev, float *w_out_dev, double *h_out_dev,
                     void *stream);

/* Bounded device-side waits (the paper has no counterpart).  The one-launch
 * CGS2 step of the solvers separates its passes with grid-wide barriers,
 * which rely on every block of the launch being resident.  Each wait polls
 * at most `polls` times (about 100 ns apart; 0 restores the default of
 * 2^22, about half a second) and then gives up: the solve stops and
 * ctg_ab_gmres / ctg_ba_gmres return CTG_ERR_TIMEOUT (the context stays
 * usable; x then holds no meaningful iterate).  The batched one-launch step
 * of ctg_batch_solve, for batches created on this context, takes the same
 * limit.  A limit of 1 makes a wait give up unless every block has already
 * arrived, which tests use to exercise this path.  Takes effect at the next
 * solve. */
int ctg_set_wait_limit(ctg_ctx *ctx, int64_t polls);

/* Phase tracing (the paper has no counterpart; it reports no timings).
 * When enabled, the solvers bracket each phase with CUDA events on the
 * solver's stream and accumulate its device time; kernel launches are
 * counted whether or not timing is enabled.  Phases: 0 forward projection
 * (the Joseph A kernel; a launch that projects two images at once counts
 * as two executions), 1 back projection (B), 2 Arnoldi CGS2 step,
 * 3 everything else (the forward projector's image staging, residual
 * norms, iterate formation). */
typedef struct {
    double ms[4];             /* accumulated device milliseconds per phase */
    int64_t calls[4];         /* phase executions per phase                */
    int64_t kernels;          /* kernels launched by the library           */
} ctg_timing;
int ctg_set_timing(ctg_ctx *ctx, int enable);
/* Copy the counters into *out; reset them if `reset` is nonzero. */
int ctg_get_timing(ctg_ctx *ctx, ctg_timing *out, int reset);

const char *ctg_status_string(int status);

#ifdef __cplusplus
}
#endif
#endif /* CTGMRES_H */
