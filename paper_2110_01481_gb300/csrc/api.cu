// C-ABI of libctgmres (declared in include/ctgmres.h): geometry tables,
// workspace layout and the host loops of AB-GMRES and BA-GMRES (paper
// Sec. 2, algorithm box), with the Hessenberg least-squares problem solved
// by FP64 Givens rotations on the host and the discrepancy-principle stop
// of Sec. 6.4.
#include <cmath>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "ctg_internal.cuh"

namespace {

constexpr int kMaxIt = 4096;

// Pinned ring of the LSQR / LSMR loop: the slot of step k holds its status
// words (live flag, residual estimate).
constexpr int kRing = 4;
size_t ring_slot_doubles(int maxit) { return 2 * (size_t)maxit + 8; }

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }
size_t round_up(size_t v, size_t m) { return (v + m - 1) / m * m; }

bool geom_valid(const ctg_geom *g) {
    if (!g || g->back_model < CTG_BACK_PIXEL || g->back_model > CTG_BACK_THRESHOLD) return false;
    if (!std::isfinite(g->back_tau) || g->back_tau < 0.0 || g->back_tau > 1.0) return false;
    if (g->back_model != CTG_BACK_THRESHOLD && g->back_tau != 0.0) return false;
    if (g->N < 1 || g->N > 16384 || g->n_angles < 1 || g->n_angles > (1 << 20)) return false;
    if (g->n_det < 1 || g->n_det > 65536) return false;
    if (!(g->det_spacing > 0.0) || !std::isfinite(g->det_spacing)) return false;
    if ((double)g->n_det * g->det_spacing > (double)(1 << 20)) return false;
    // detector coordinates of every pixel fit the 24-bit integer part of the
    // back projectors' 24.40 fixed point
    if (1.5 * g->N / g->det_spacing + g->n_det >= (double)(1 << 22)) return false;
    const double S = g->angle_start_deg, R = g->angle_range_deg;
    if (!std::isfinite(S) || !std::isfinite(R) || S != std::floor(S) || R != std::floor(R)) return false;
    if (R <= 0.0 || R > 360.0 || std::fabs(S) > 3600.0) return false;
    return true;
}

bool opts_valid(const ctg_opts *o) {
    if (!o || o->maxit < 1 || o->maxit > kMaxIt) return false;
    if (ctg_basis_bytes(o->basis_dtype) == 0) return false;
    if (!std::isfinite(o->tau) || !std::isfinite(o->noise_norm)) return false;
    if (o->noise_norm > 0.0 && !(o->tau > 0.0)) return false;
    if (o->stop_rule != CTG_RULE_DP && o->stop_rule != CTG_RULE_NCP) return false;
    return true;
}

long long to_fx(double v) { return std::llround(std::ldexp(v, CTG_FX_BITS)); }
long long to_fxf(double v) { return std::llround(std::ldexp(v, CTG_FXF_BITS)); }

// theta_a = S + a R / N_a degrees, i.e. theta_a * N_a = num (an integer).
void angle_of(const ctg_geom *g, int a, double *c, double *s, int *row_driven) {
    const long long Na = g->n_angles;
    const long long num = (long long)g->angle_start_deg * Na + (long long)a * (long long)g->angle_range_deg;
    const long long half_turn = 180 * Na;
    long long T = num % half_turn;
    if (T < 0) T += half_turn;
    // row-driven iff theta mod 180 in [0, 45] or [135, 180)
    *row_driven = (4 * T <= half_turn) || (4 * T >= 3 * half_turn);
    const long long quarter = 90 * Na;
    if (num % quarter == 0) {
        long long q = (num / quarter) % 4;
        if (q < 0) q += 4;
        static const double cq[4] = {1.0, 0.0, -1.0, 0.0}, sq[4] = {0.0, 1.0, 0.0, -1.0};
        *c = cq[q];
        *s = sq[q];
    } else {
        const double th = (double)num / (double)half_turn * M_PI;
        *c = std::cos(th);
        *s = std::sin(th);
    }
}

void build_tables(const ctg_geom *g, std::vector<FwdAngle> &fw, std::vector<BackAngle> &bk) {
    const double h = 0.5 * (g->N - 1), hd = 0.5 * (g->n_det - 1), ds = g->det_spacing;
    fw.resize(g->n_angles);
    bk.resize(g->n_angles);
    for (int a = 0; a < g->n_angles; ++a) {
        double cs, sn;
        int rd;
        angle_of(g, a, &cs, &sn, &rd);
        const double c = rd ? cs : sn, s = rd ? sn : cs;
        const double P = ds / c, Q = (h * s - hd * ds) / c + h, D = -s / c;
        FwdAngle &f = fw[a];
        f.P = to_fxf(P);
        f.Q = to_fxf(Q);
        f.D = to_fxf(D);
        f.pf = (float)P;
        f.qf = (float)Q;
        f.df = (float)D;
        f.scale = (float)(1.0 / std::fabs(c));
        f.row_driven = rd;
        f.pad_ = 0;
        BackAngle &b = bk[a];
        b.COS = to_fx(cs / ds);
        b.SIN = to_fx(sn / ds);
        b.C = to_fx(hd - h * (cs + sn) / ds);
        b.cf = (float)(cs / ds);
        b.sf = (float)(sn / ds);
    }
}

// Per-angle weights of the matched back projector; *rm = the extra detector
// bins on each side that the widest angle needs beyond the two nearest.
void build_matched(const ctg_geom *g, std::vector<MatchedAngle> &mt, int *rm) {
    mt.resize(g->n_angles);
    double wmax = 0.0;
    for (int a = 0; a < g->n_angles; ++a) {
        double cs, sn;
        int rd;
        angle_of(g, a, &cs, &sn, &rd);
        const double c = std::fabs(rd ? cs : sn);      // >= 1/sqrt(2)
        mt[a].scale = (float)(1.0 / c);
        mt[a].inv_w = (float)(g->det_spacing / c);
        wmax = std::max(wmax, c / g->det_spacing);
    }
    *rm = std::max(0, (int)std::ceil(wmax) - 1);
}

}  // namespace

bool ctg_geom_valid(const ctg_geom *g) { return geom_valid(g); }
bool ctg_opts_valid(const ctg_opts *o) { return opts_valid(o); }
void ctg_build_matched(const ctg_geom *g, std::vector<MatchedAngle> &mt, int *rm) {
    build_matched(g, mt, rm);
}
void ctg_build_tables(const ctg_geom *g, std::vector<FwdAngle> &fw, std::vector<BackAngle> &bk) {
    build_tables(g, fw, bk);
}

namespace {

bool same_geom(const ctg_geom &a, const ctg_geom &b) {
    return a.N == b.N && a.n_angles == b.n_angles && a.n_det == b.n_det &&
           a.angle_start_deg == b.angle_start_deg && a.angle_range_deg == b.angle_range_deg &&
           a.det_spacing == b.det_spacing && a.back_model == b.back_model &&
           a.back_tau == b.back_tau;
}

struct GeomEntry {
    ctg_geom g;
    FwdAngle *fwd = nullptr;
    BackAngle *back = nullptr;
    int back_window = 0;        // detector window of the tiled back projector
    PadLayout pl{};             // staged-image layout of the forward projector
    float2 *pad = nullptr;      // context-owned staged image for ctg_project
    float2 *tw = nullptr;       // NCP: DFT twiddles of length n_det (on first use)
    MatchedAngle *mt = nullptr; // matched / thresholded back projector
    int rm = 0;
    float thr = 0.0f;           // B_tau threshold tau * max(A) (0: A^T)
    int *fwd_order = nullptr;   // forward dispatch orders of the shapes, one after another
    size_t fwd_order_off[kFwdShapes] = {};
    bool fwd_split_ok = false;  // shapes with several angles per warp are safe here
    int fwd_shape = 0;          // tile shapes in use (autotuned unless forced)
    int back_chunk = 32;
    bool tuned = false;
    int tuned_fwd_shape = 0, tuned_back_chunk = 32;   // the autotuner's choice, kept while forced
    float fwd_us[kFwdShapes] = {}, back_us[3] = {0, 0, 0};   // measured (0: not timed)
    unsigned long long last_use = 0;
    unsigned long long serial = 0;   // identifies the entry's device tables (graphs captured with them)
    const int *order_for(int shape) const { return fwd_order ? fwd_order + fwd_order_off[shape] : nullptr; }
};

// x = B b (+ add) with the geometry's back projector; b of type `btype`
// (column bc of a basis at b when bc.k is set).
cudaError_t back_apply(const GeomEntry *ge, const void *b, int btype, const float *add, float *x,
                       cudaStream_t st, ColRef bc = col_none()) {
    const ctg_geom *g = &ge->g;
    if (g->back_model == CTG_BACK_PIXEL)
        return ctg_launch_back(b, btype, g->N, g->n_angles, g->n_det, ge->back, ge->back_window, add,
                               x, st, ge->back_chunk, bc);
    if (ge->rm == 0 && ge->back_window <= ctg_back_window_max())
        return ctg_launch_back_matched_tiled(b, btype, g->N, g->n_angles, g->n_det, ge->back,
                                             ge->back_window, ge->mt, ge->thr, add, x, st, bc);
    return ctg_launch_back_matched(b, btype, g->N, g->n_angles, g->n_det, ge->back, ge->mt, ge->rm,
                                   ge->thr, add, x, st, bc);
}

struct WsLayout {
    size_t off_w, ld_w, off_h, off_pad, off_vn0, off_vm0, off_vm1, off_y, off_red, total;
    size_t off_n[4], off_m[5], off_state, off_hist;   // LSQR / LSMR; off_state, off_hist also GMRES
    size_t off_ncp;                // NCP distances of the projections (n_angles doubles)
    // GMRES loop state: Givens rotations, rotated right-hand side, rotated
    // columns R, y of the last three steps, NCP residual coefficients,
    // rho and NCP histories
    size_t off_gc, off_gs, off_gg, off_R, off_yring, off_z, off_rhoh, off_ncph;
    size_t off_pad2;               // BA: the staging of two interleaved images
    int64_t L, n, m;
    int kmax;
    int dtype;      // basis element type
    size_t es;      // basis element bytes
};

// LSQR / LSMR: no basis; n-vectors v, w or h, hbar, B u; m-vectors u, p = A v
// and (LSMR) A h, A hbar, r; the staged image, the device state and history.
bool layout_lsq(const ctg_geom *g, int variant, const ctg_opts *o, WsLayout *ly) {
    if (o->basis_dtype != CTG_BASIS_FP32 || o->stop_rule != CTG_RULE_DP) return false;
    *ly = WsLayout{};
    const int64_t n = (int64_t)g->N * g->N, m = (int64_t)g->n_angles * g->n_det;
    ly->n = n;
    ly->m = m;
    ly->L = n;
    ly->kmax = o->maxit;
    ly->dtype = CTG_BASIS_FP32;
    ly->es = 4;
    size_t off = 0;
    ly->off_pad = off;
    off = align256(off + sizeof(float) * ctg_pad_layout(g->N, g->det_spacing).floats);
    for (int i = 0; i < 4; ++i) {
        ly->off_n[i] = off;
        off = align256(off + sizeof(float) * round_up((size_t)n, 64));
    }
    const int nm = variant == CTG_LSMR ? 5 : 2;
    for (int i = 0; i < 5; ++i) {
        ly->off_m[i] = off;
        if (i < nm) off = align256(off + sizeof(float) * round_up((size_t)m, 64));
    }
    ly->off_vm0 = ly->off_m[0];
    ly->off_vm1 = ly->off_m[1];
    ly->off_vn0 = ly->off_n[3];
    ly->off_state = off;
    off = align256(off + sizeof(LsqState));
    ly->off_hist = off;
    off = align256(off + sizeof(double) * (size_t)(o->maxit + 1));
    ly->off_red = off;
    off = align256(off + ctg_red_scratch_bytes(n > m ? n : m, 2));
    ly->total = off;
    return true;
}

int rule_of(const ctg_opts *o) {
    return o->stop_rule == CTG_RULE_NCP ? kRuleNCP : (o->noise_norm > 0.0 ? kRuleDP : kRuleMaxit);
}

// AB / BA: the basis W ((maxit + 1) vectors of length L, the storage law k L
// of Table 3), the Hessenberg matrix, the staged image (BA also a staging of
// two interleaved images), one n-vector, two m-vectors, the iterate
// coefficients, the loop state (O(maxit^2) doubles for the rotated
// Hessenberg columns) and the reduction scratch.
bool layout_of(const ctg_geom *g, int variant, const ctg_opts *o, WsLayout *ly) {
    if (!geom_valid(g) || !opts_valid(o)) return false;
    if (variant == CTG_LSQR || variant == CTG_LSMR) return layout_lsq(g, variant, o, ly);
    if (variant != CTG_AB && variant != CTG_BA) return false;
    if (o->stop_rule == CTG_RULE_NCP && (g->n_det < 2 || g->n_det > kCtgNcpMaxDet)) return false;
    *ly = WsLayout{};
    const int64_t n = (int64_t)g->N * g->N, m = (int64_t)g->n_angles * g->n_det;
    const int64_t L = variant == CTG_AB ? m : n;
    const size_t K = (size_t)o->maxit;
    ly->n = n;
    ly->m = m;
    ly->L = L;
    ly->kmax = o->maxit;
    ly->dtype = o->basis_dtype;
    ly->es = ctg_basis_bytes(o->basis_dtype);
    ly->ld_w = round_up((size_t)L, 64);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t at = off;
        off = align256(off + bytes);
        return at;
    };
    ly->off_w = take(ly->es * ly->ld_w * (K + 1));
    ly->off_h = take(sizeof(double) * (K + 1) * K);
    const size_t pad_floats = ctg_pad_layout(g->N, g->det_spacing).floats;
    ly->off_pad = take(sizeof(float) * pad_floats);
    ly->off_pad2 = variant == CTG_BA ? take(sizeof(float) * 2 * pad_floats) : 0;
    ly->off_vn0 = take(sizeof(float) * round_up((size_t)n, 64));
    ly->off_vm0 = take(sizeof(float) * round_up((size_t)m, 64));
    ly->off_vm1 = take(sizeof(float) * round_up((size_t)m, 64));
    ly->off_y = take(sizeof(double) * (K + 2));
    ly->off_state = take(sizeof(GmresState));
    ly->off_gc = take(sizeof(double) * K);
    ly->off_gs = take(sizeof(double) * K);
    ly->off_gg = take(sizeof(double) * (K + 1));
    ly->off_R = take(sizeof(double) * K * K);
    ly->off_yring = take(sizeof(double) * 3 * K);
    ly->off_z = take(sizeof(double) * (K + 1));
    ly->off_hist = take(sizeof(double) * (K + 1));
    ly->off_rhoh = take(sizeof(double) * (K + 1));
    ly->off_ncph = take(sizeof(double) * (K + 2));
    ly->off_ncp = take(sizeof(double) * (size_t)g->n_angles);
    const int64_t Lmax = n > m ? n : m;
    ly->off_red = take(ctg_red_scratch_bytes(Lmax, o->maxit + 1));
    ly->total = off;
    return true;
}

}  // namespace

struct ctg_ctx {
    int device = 0;
    std::vector<GeomEntry> cache;
    unsigned long long tick = 0;
    double *pinned = nullptr;     // host staging for Hessenberg columns and scalars
    size_t pinned_count = 0;
    // phase tracing: events bracket each phase on the launching stream and
    // are resolved into per-phase milliseconds once they have completed
    struct Mark {
        int phase;
        cudaEvent_t a, b;
    };
    bool timing = false;
    std::vector<cudaEvent_t> events;
    size_t events_used = 0;
    std::vector<Mark> marks;
    double ms[4] = {0, 0, 0, 0};
    long long calls[4] = {0, 0, 0, 0};
    long long kernels = 0;
    // completion events of the pipelined solver loops (no timing)
    cudaEvent_t ev_h[4] = {nullptr, nullptr, nullptr, nullptr};
    cudaEvent_t ev_r[4] = {nullptr, nullptr, nullptr, nullptr};
    cudaEvent_t ev_init = nullptr;   // a solve's start values are in the pinned scratch
    // projector tile shapes: 0 = autotuned per geometry, else forced
    int force_fwd_angles = 0, force_fwd_split = 1, force_back_chunk = 0;
    // bounded device-side waits: polls before a wait gives up
    long long spin_limit = kCtgDefaultSpinLimit;
    // captured solver loops (CUDA graphs with while-loop nodes), each for
    // one set of solve arguments, most recently used last
    struct LoopGraph {
        std::vector<long long> key;
        unsigned long long geom_serial;
        cudaGraphExec_t exec;
        int n_init, n_small, n_fused, n_pass, n_exit;   // kernels per launch of each part
        int small_max, fused_max;
    };
    std::vector<LoopGraph> graphs;
    cudaStream_t cap_st[2] = {nullptr, nullptr};   // capture streams
    bool capturing = false;     // launches are being captured (not counted as run)
    long long captured_kernels = 0;
    int graph_mode = 0;        // 0 untried, 1 cooperative fused step, 2 plain fused step, -1 no graphs
};

namespace {

int fail_cuda(cudaError_t e) {
    if (e == cudaErrorMemoryAllocation) return CTG_ERR_OOM;
    return CTG_ERR_CUDA;
}

#define CTG_CK(call)                                  \
    do {                                              \
        cudaError_t e_ = (call);                      \
        if (e_ != cudaSuccess) return fail_cuda(e_);  \
    } while (0)

// geometries a context keeps (tables, dispatch orders, tuned tile shapes);
// enough for a served mix of request shapes to be tuned once each
constexpr size_t kMaxCachedGeoms = 64;

// Projector tile autotuner.  Candidate shapes leave every sum in the same
// order (forward: angles per block and per warp, each ray still summed by
// one lane over its own chord in a fixed accumulator order; pixel-driven
// back projection: angles staged per pass, each pixel's angles still in
// order), so the choice changes the speed only.  Shapes with several angles
// per warp are timed only where the geometry allows them (fwd_split_ok).  Each candidate is timed
// with CUDA events over 3 launches (after one untimed) on zero inputs of the
// geometry's sizes on a private stream; the fastest is kept.
int tune_geometry(GeomEntry *ge) {
    const ctg_geom *g = &ge->g;
    const size_t n = (size_t)g->N * g->N, m = (size_t)g->n_angles * g->n_det;
    float2 *pad = nullptr;
    float *bv = nullptr, *xv = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t err = cudaMalloc(&pad, sizeof(float) * ge->pl.floats);
    if (err == cudaSuccess) err = cudaMalloc(&bv, sizeof(float) * m);
    if (err == cudaSuccess) err = cudaMalloc(&xv, sizeof(float) * n);
    if (err == cudaSuccess) err = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    // zero inputs, ordered before the timed launches on the same stream
    if (err == cudaSuccess) err = cudaMemsetAsync(pad, 0, sizeof(float) * ge->pl.floats, st);
    if (err == cudaSuccess) err = cudaMemsetAsync(bv, 0, sizeof(float) * m, st);
    if (err == cudaSuccess) err = cudaEventCreate(&e0);
    if (err == cudaSuccess) err = cudaEventCreate(&e1);
    auto timed = [&](auto launch, float *us) {
        if (err != cudaSuccess) return;
        launch();
        err = cudaEventRecord(e0, st);
        for (int r = 0; r < 3 && err == cudaSuccess; ++r) launch();
        if (err == cudaSuccess) err = cudaEventRecord(e1, st);
        if (err == cudaSuccess) err = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
        *us = ms * 1e3f / 3.0f;
    };
    for (int c = 0; c < kFwdShapes; ++c) {
        ge->fwd_us[c] = 0.0f;
        if (kFwdShapeSplit[c] > 1 && !ge->fwd_split_ok) continue;
        timed([&] {
            if (err == cudaSuccess)
                err = ctg_launch_forward(pad, g->N, ge->pl, g->n_angles, g->n_det, ge->fwd, bv, st, c,
                                         ge->order_for(c));
        }, &ge->fwd_us[c]);
    }
    const int back_cand[3] = {16, 32, 64};
    if (g->back_model == CTG_BACK_PIXEL)
        for (int c = 0; c < 3; ++c)
            timed([&] {
                if (err == cudaSuccess)
                    err = ctg_launch_back(bv, CTG_BASIS_FP32, g->N, g->n_angles, g->n_det, ge->back,
                                          ge->back_window, nullptr, xv, st, back_cand[c]);
            }, &ge->back_us[c]);
    if (err == cudaSuccess) {
        int fs = 0;
        for (int c = 1; c < kFwdShapes; ++c)
            if (ge->fwd_us[c] > 0.0f && ge->fwd_us[c] < ge->fwd_us[fs]) fs = c;
        ge->fwd_shape = ge->tuned_fwd_shape = fs;
        int best = 1;
        if (g->back_model == CTG_BACK_PIXEL)
            for (int c = 0; c < 3; ++c)
                if (ge->back_us[c] < ge->back_us[best]) best = c;
        ge->back_chunk = ge->tuned_back_chunk = back_cand[best];
        ge->tuned = true;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    cudaFree(pad);
    cudaFree(bv);
    cudaFree(xv);
    return err == cudaSuccess ? CTG_OK : fail_cuda(err);
}

// Destroys the captured loops that use a geometry's tables (serial), or all
// of them (serial 0).
void drop_graphs(ctg_ctx *ctx, unsigned long long serial) {
    for (size_t i = 0; i < ctx->graphs.size();) {
        if (serial == 0 || ctx->graphs[i].geom_serial == serial) {
            cudaGraphExecDestroy(ctx->graphs[i].exec);
            ctx->graphs.erase(ctx->graphs.begin() + i);
        } else {
            ++i;
        }
    }
}

int apply_tiles(ctg_ctx *ctx, GeomEntry *ge) {
    if (ctx->force_fwd_angles || ctx->force_back_chunk) {
        // a forced shape with several angles per warp falls back to one
        // angle per warp where the geometry does not allow it
        int split = ctx->force_fwd_angles ? ctx->force_fwd_split : 1;
        if (split > 1 && !ge->fwd_split_ok) split = 1;
        int angles = ctx->force_fwd_angles ? ctx->force_fwd_angles : 8;
        if (split == 1) angles = std::min(angles, 8);
        ge->fwd_shape = 0;
        for (int c = 0; c < kFwdShapes; ++c)
            if (kFwdShapeAngles[c] == angles && kFwdShapeSplit[c] == split) ge->fwd_shape = c;
        ge->back_chunk = ctx->force_back_chunk ? ctx->force_back_chunk : 32;
        return CTG_OK;
    }
    if (!ge->tuned) return tune_geometry(ge);
    ge->fwd_shape = ge->tuned_fwd_shape;     // back from forced shapes
    ge->back_chunk = ge->tuned_back_chunk;
    return CTG_OK;
}

int get_geom(ctg_ctx *ctx, const ctg_geom *g, GeomEntry **out) {
    for (auto &e : ctx->cache)
        if (same_geom(e.g, *g)) {
            e.last_use = ++ctx->tick;
            *out = &e;
            return apply_tiles(ctx, &e);
        }
    if (ctx->cache.size() >= kMaxCachedGeoms) {
        // evict the least recently used geometry; its tables may still be
        // read by queued work, so wait for the device first
        size_t victim = 0;
        for (size_t i = 1; i < ctx->cache.size(); ++i)
            if (ctx->cache[i].last_use < ctx->cache[victim].last_use) victim = i;
        CTG_CK(cudaDeviceSynchronize());
        drop_graphs(ctx, ctx->cache[victim].serial);
        cudaFree(ctx->cache[victim].fwd);
        cudaFree(ctx->cache[victim].back);
        cudaFree(ctx->cache[victim].pad);
        cudaFree(ctx->cache[victim].mt);
        cudaFree(ctx->cache[victim].tw);
        cudaFree(ctx->cache[victim].fwd_order);
        ctx->cache.erase(ctx->cache.begin() + victim);
    }
    std::vector<FwdAngle> fw;
    std::vector<BackAngle> bk;
    build_tables(g, fw, bk);
    GeomEntry e;
    e.g = *g;
    e.last_use = ++ctx->tick;
    e.serial = e.last_use;
    e.back_window = ctg_back_window(bk.data(), g->n_angles);
    e.pl = ctg_pad_layout(g->N, g->det_spacing);
    cudaError_t err = cudaMalloc(&e.fwd, sizeof(FwdAngle) * fw.size());
    if (err == cudaSuccess) err = cudaMalloc(&e.back, sizeof(BackAngle) * bk.size());
    if (err == cudaSuccess)
        err = cudaMemcpy(e.fwd, fw.data(), sizeof(FwdAngle) * fw.size(), cudaMemcpyHostToDevice);
    if (err == cudaSuccess)
        err = cudaMemcpy(e.back, bk.data(), sizeof(BackAngle) * bk.size(), cudaMemcpyHostToDevice);
    if (err == cudaSuccess) {
        e.fwd_split_ok = ctg_forward_split_safe(fw.data(), g->N, g->n_angles, g->n_det, e.pl, 4);
        std::vector<int> all, o;
        for (int c = 0; c < kFwdShapes; ++c) {
            e.fwd_order_off[c] = all.size();
            ctg_forward_order(fw.data(), g->N, g->n_angles, g->n_det, c, o);
            all.insert(all.end(), o.begin(), o.end());
        }
        err = cudaMalloc(&e.fwd_order, sizeof(int) * all.size());
        if (err == cudaSuccess)
            err = cudaMemcpy(e.fwd_order, all.data(), sizeof(int) * all.size(), cudaMemcpyHostToDevice);
    }
    if (err == cudaSuccess && g->back_model != CTG_BACK_PIXEL) {
        std::vector<MatchedAngle> mt;
        build_matched(g, mt, &e.rm);
        err = cudaMalloc(&e.mt, sizeof(MatchedAngle) * mt.size());
        if (err == cudaSuccess)
            err = cudaMemcpy(e.mt, mt.data(), sizeof(MatchedAngle) * mt.size(), cudaMemcpyHostToDevice);
        if (err == cudaSuccess && g->back_model == CTG_BACK_THRESHOLD) {
            // tau * max(A), max over every entry of A (one pass, once per geometry)
            unsigned *bits = nullptr;
            unsigned host_bits = 0;
            err = cudaMalloc(&bits, sizeof(unsigned));
            if (err == cudaSuccess)
                err = ctg_matched_max(g->N, g->n_angles, g->n_det, e.back, e.mt, e.rm, bits, nullptr);
            if (err == cudaSuccess) err = cudaMemcpy(&host_bits, bits, sizeof(unsigned), cudaMemcpyDeviceToHost);
            cudaFree(bits);
            float amax;
            std::memcpy(&amax, &host_bits, sizeof(float));
            e.thr = (float)(g->back_tau * (double)amax);
        }
    }
    if (err != cudaSuccess) {
        cudaFree(e.fwd);
        cudaFree(e.back);
        cudaFree(e.mt);
        cudaFree(e.fwd_order);
        return fail_cuda(err);
    }
    ctx->cache.push_back(e);
    *out = &ctx->cache.back();
    return apply_tiles(ctx, *out);
}

// (cos, -sin)(2 pi j / n_det), j < n_det, for the NCP periodograms
int ensure_twiddles(GeomEntry *ge) {
    if (ge->tw) return CTG_OK;
    const int nd = ge->g.n_det;
    std::vector<float2> t(nd);
    for (int j = 0; j < nd; ++j) {
        const double ph = 2.0 * M_PI * (double)j / (double)nd;
        t[j] = make_float2((float)std::cos(ph), (float)-std::sin(ph));
    }
    CTG_CK(cudaMalloc(&ge->tw, sizeof(float2) * nd));
    CTG_CK(cudaMemcpy(ge->tw, t.data(), sizeof(float2) * nd, cudaMemcpyHostToDevice));
    return CTG_OK;
}

cudaEvent_t next_event(ctg_ctx *ctx) {
    if (ctx->events_used == ctx->events.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        ctx->events.push_back(e);
    }
    return ctx->events[ctx->events_used++];
}

// Runs f() (which enqueues `nkern` kernels on st) as `ncalls` executions of
// `phase` (a projection of two images counts as two), bracketed by events
// when tracing is on.
template <typename F>
cudaError_t traced(ctg_ctx *ctx, int phase, int nkern, cudaStream_t st, F f, int ncalls = 1) {
    if (ctx->capturing) {            // counted per launch of the captured graph
        ctx->captured_kernels += nkern;
        return f();
    }
    ctx->kernels += nkern;
    ctx->calls[phase] += ncalls;
    if (!ctx->timing) return f();
    cudaEvent_t a = next_event(ctx), b = next_event(ctx);
    if (a) cudaEventRecord(a, st);
    cudaError_t e = f();
    if (b) cudaEventRecord(b, st);
    if (a && b) ctx->marks.push_back({phase, a, b});
    return e;
}

// Waits for the recorded events and folds them into the phase totals.
int resolve_marks(ctg_ctx *ctx) {
    for (const auto &mk : ctx->marks) {
        float t = 0.f;
        CTG_CK(cudaEventSynchronize(mk.b));
        CTG_CK(cudaEventElapsedTime(&t, mk.a, mk.b));
        ctx->ms[mk.phase] += t;
    }
    ctx->marks.clear();
    ctx->events_used = 0;
    return CTG_OK;
}

int ensure_pinned(ctg_ctx *ctx, size_t count) {
    if (ctx->pinned_count >= count) return CTG_OK;
    if (ctx->pinned) cudaFreeHost(ctx->pinned);
    ctx->pinned = nullptr;
    ctx->pinned_count = 0;
    CTG_CK(cudaMallocHost(&ctx->pinned, sizeof(double) * count));
    ctx->pinned_count = count;
    return CTG_OK;
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

struct SolveCtx {
    ctg_ctx *ctx;
    const ctg_geom *g;
    GeomEntry *ge;
    WsLayout ly;
    char *ws;
    RedScratch rs;
    cudaStream_t st;
    void *W() const { return ws + ly.off_w; }
    void *Wcol(int j) const { return ws + ly.off_w + (size_t)j * ly.ld_w * ly.es; }
    double *Hcol(int k) const {   // column k (1-based)
        return reinterpret_cast<double *>(ws + ly.off_h) + (size_t)(k - 1) * (ly.kmax + 1);
    }
    float2 *pad() const { return reinterpret_cast<float2 *>(ws + ly.off_pad); }
    float *vn0() const { return reinterpret_cast<float *>(ws + ly.off_vn0); }
    float *vm0() const { return reinterpret_cast<float *>(ws + ly.off_vm0); }
    float *vm1() const { return reinterpret_cast<float *>(ws + ly.off_vm1); }
    double *ydev() const { return reinterpret_cast<double *>(ws + ly.off_y); }
    double *ncpd() const { return reinterpret_cast<double *>(ws + ly.off_ncp); }
    template <typename TT> TT *at(size_t off) const { return reinterpret_cast<TT *>(ws + off); }
    GmresState *state() const { return at<GmresState>(ly.off_state); }
    // device pointers of the loop state for the loop kernels
    LoopBufs loop_bufs() const {
        LoopBufs B{};
        B.S = state();
        B.H = at<double>(ly.off_h);
        B.ldh = ly.kmax + 1;
        B.gc = at<double>(ly.off_gc);
        B.gs = at<double>(ly.off_gs);
        B.gg = at<double>(ly.off_gg);
        B.R = at<double>(ly.off_R);
        B.ldr = ly.kmax;
        B.y = ydev();
        B.yring = at<double>(ly.off_yring);
        B.z = at<double>(ly.off_z);
        B.hist = at<double>(ly.off_hist);
        B.rhoh = at<double>(ly.off_rhoh);
        B.ncph = at<double>(ly.off_ncph);
        B.scal = rs.scal;
        B.h1 = rs.h1;
        B.counter = rs.counter;
        return B;
    }
    // *out (device) = the NCP distance of the residual sinogram r
    cudaError_t ncp(const float *r, double *out) const {
        return traced(ctx, 3, 2, st, [&] {
            return ctg_ncp(r, g->n_angles, g->n_det, ge->tw, ncpd(), out, st);
        });
    }

    // b = A x; x of type xtype, column xc of a basis when xc.k is set
    cudaError_t forward(const void *x, float *b, int xtype = CTG_BASIS_FP32, ColRef xc = col_none()) const {
        // the image staging is traced as phase 3, so that phase 0 times the
        // Joseph kernel alone
        const cudaError_t e = traced(ctx, 3, 1, st, [&] {
            return ctg_launch_pad(x, xtype, pad(), g->N, ge->pl, st, xc);
        });
        if (e != cudaSuccess) return e;
        return traced(ctx, 0, 1, st, [&] {
            return ctg_launch_forward(pad(), g->N, ge->pl, g->n_angles, g->n_det, ge->fwd, b, st,
                                      ge->fwd_shape, ge->order_for(ge->fwd_shape));
        });
    }
    // b = A x and b2 = A x2 in one walk (x: column xc of the basis)
    cudaError_t forward2(ColRef xc, const float *x2, float *b, float *b2) const {
        float4 *p4 = at<float4>(ly.off_pad2);
        const cudaError_t e = traced(ctx, 3, 1, st, [&] {
            return ctg_launch_pad2(W(), ly.dtype, xc, x2, p4, g->N, ge->pl, st);
        });
        if (e != cudaSuccess) return e;
        return traced(ctx, 0, 1, st, [&] {
            return ctg_launch_forward2(p4, g->N, ge->pl, g->n_angles, g->n_det, ge->fwd, b, b2, st,
                                       ge->fwd_shape, ge->order_for(ge->fwd_shape));
        }, 2);
    }
    cudaError_t back(const void *b, const float *add, float *x, int btype = CTG_BASIS_FP32,
                     ColRef bc = col_none()) const {
        return traced(ctx, 1, 1, st, [&] { return back_apply(ge, b, btype, add, x, st, bc); });
    }
    // one CGS2 step of the loop (k on the device); with the fused step, its
    // block 0 also runs the step's Givens update in mode giv_mode (lb)
    cudaError_t cgs2_loop(int64_t L, float *q, int kmax, bool fused, bool cooperative,
                          const LoopBufs *lb = nullptr, int giv_mode = -1, bool small_grid = false) const {
        int nk = 0;
        const LoopStep ls{&state()->k, at<double>(ly.off_h), ly.kmax + 1, kmax, fused, lb, giv_mode, small_grid};
        const cudaError_t e = traced(ctx, 2, 0, st, [&] {
            return ctg_cgs2_step_loop(W(), ly.dtype, ly.ld_w, L, q, ls, rs, ctx->spin_limit, cooperative, st, &nk);
        });
        if (ctx->capturing) ctx->captured_kernels += nk;
        else ctx->kernels += nk;
        return e;
    }
    // out = base + W y with k = *kdev + koff columns (kmax bounds it)
    cudaError_t gemv_dev(int64_t L, const int *kdev, int koff, int kmax, const double *y, const float *base,
                         float *out) const {
        return traced(ctx, 3, 1, st, [&] {
            return ctg_gemv(W(), ly.dtype, ly.ld_w, L, kmax, y, base, out, st, kdev, koff);
        });
    }
    cudaError_t sub_norm2(const float *a, const float *c, float *out, int64_t L, double *res) const {
        return traced(ctx, 3, 1, st, [&] { return ctg_sub_norm2(a, c, out, L, res, rs, st); });
    }
    // out (a basis vector) = v / sqrt(*nrm2), rounded to the basis type
    cudaError_t scale(const float *v, const double *nrm2, void *out, int64_t L) const {
        return traced(ctx, 3, 1, st, [&] { return ctg_scale(v, nrm2, out, ly.dtype, L, st); });
    }
    // copy `count` doubles from the device to the pinned area and wait
    // pinned staging outside the pipeline ring (which queued copies of
    // speculative Arnoldi steps may still be writing)
    double *pinned_scratch() const { return ctx->pinned + kRing * ring_slot_doubles(ly.kmax); }
    int fetch(const double *src, size_t count, double **host) const {
        double *hs = pinned_scratch();
        CTG_CK(cudaMemcpyAsync(hs, src, sizeof(double) * count, cudaMemcpyDeviceToHost, st));
        CTG_CK(cudaStreamSynchronize(st));
        *host = hs;
        return CTG_OK;
    }
    // ||b - A x||, using vm1 as scratch
    int true_resnorm(const float *b, const float *x, double *out) const {
        CTG_CK(forward(x, vm1()));
        CTG_CK(sub_norm2(b, vm1(), nullptr, ly.m, rs.scal + 4));
        double *h;
        int rc = fetch(rs.scal + 4, 1, &h);
        if (rc) return rc;
        *out = std::sqrt(h[0]);
        return CTG_OK;
    }
};

int solve_setup(ctg_ctx *ctx, const ctg_geom *g, int variant, const ctg_opts *o,
                const float *b, float *x, void *ws, size_t ws_bytes, ctg_info *info,
                void *stream, SolveCtx *sc, void **owned) {
    *owned = nullptr;
    if (!ctx || !b || !x || !info || !layout_of(g, variant, o, &sc->ly)) return CTG_ERR_INVALID_ARG;
    if (!aligned16(b) || !aligned16(x)) return CTG_ERR_INVALID_ARG;
    sc->ctx = ctx;
    sc->g = g;
    sc->st = static_cast<cudaStream_t>(stream);
    int rc = get_geom(ctx, g, &sc->ge);
    if (rc) return rc;
    // after the ring: a GMRES solve's state and histories, or a staged LsqState
    rc = ensure_pinned(ctx, kRing * ring_slot_doubles(o->maxit) + 3 * (size_t)o->maxit + 64);
    if (rc) return rc;
    if (ws == nullptr) {
        cudaError_t e = cudaMallocAsync(&ws, sc->ly.total, sc->st);
        if (e != cudaSuccess) return fail_cuda(e);
        *owned = ws;
    } else {
        if (ws_bytes < sc->ly.total) return CTG_ERR_WORKSPACE;
        if (((uintptr_t)ws & 255u) != 0) return CTG_ERR_INVALID_ARG;
    }
    sc->ws = static_cast<char *>(ws);
    const bool lsq = variant == CTG_LSQR || variant == CTG_LSMR;
    ctg_red_scratch_carve(sc->ws + sc->ly.off_red, sc->ly.n > sc->ly.m ? sc->ly.n : sc->ly.m,
                          lsq ? 2 : o->maxit + 1, &sc->rs);
    CTG_CK(cudaMemsetAsync(sc->rs.counter, 0, 4 * sizeof(unsigned), sc->st));
    CTG_CK(cudaMemsetAsync(sc->pad(), 0, sizeof(float) * sc->ge->pl.floats, sc->st));
    if (sc->ly.off_pad2)
        CTG_CK(cudaMemsetAsync(sc->ws + sc->ly.off_pad2, 0, sizeof(float) * 2 * sc->ge->pl.floats, sc->st));
    if (!lsq)
        CTG_CK(cudaMemsetAsync(sc->ws + sc->ly.off_h, 0,
                               sizeof(double) * (size_t)(o->maxit + 1) * o->maxit, sc->st));
    info->iters = 0;
    info->stop_reason = CTG_STOP_MAXIT;
    info->resnorm = 0.0;
    info->rho = 0.0;
    return CTG_OK;
}

int finish(const SolveCtx &sc, void *owned, int rc) {
    if (owned) {
        cudaError_t e = cudaFreeAsync(owned, sc.st);
        if (rc == CTG_OK && e != cudaSuccess) rc = fail_cuda(e);
        cudaError_t e2 = cudaStreamSynchronize(sc.st);
        if (rc == CTG_OK && e2 != cudaSuccess) rc = fail_cuda(e2);
    }
    return rc;
}

int ensure_events(ctg_ctx *ctx) {
    if (!ctx->ev_init) CTG_CK(cudaEventCreateWithFlags(&ctx->ev_init, cudaEventDisableTiming));
    for (int i = 0; i < kRing; ++i) {
        if (!ctx->ev_h[i]) CTG_CK(cudaEventCreateWithFlags(&ctx->ev_h[i], cudaEventDisableTiming));
        if (!ctx->ev_r[i]) CTG_CK(cudaEventCreateWithFlags(&ctx->ev_r[i], cudaEventDisableTiming));
    }
    return CTG_OK;
}

int copy_x0(const SolveCtx &sc, const float *x0, float *x) {
    if (x0) CTG_CK(cudaMemcpyAsync(x, x0, sizeof(float) * sc.ly.n, cudaMemcpyDeviceToDevice, sc.st));
    else CTG_CK(cudaMemsetAsync(x, 0, sizeof(float) * sc.ly.n, sc.st));
    return CTG_OK;
}

struct Pipeline {
    SolveCtx &sc;
    int maxit;
    cudaEvent_t *ev_h, *ev_r;
    double *slot(int k) const { return sc.ctx->pinned + (size_t)(k % kRing) * ring_slot_doubles(maxit); }
    int wait_step(int k, const double **h) const {
        CTG_CK(cudaEventSynchronize(ev_h[k % kRing]));
        *h = slot(k);
        return CTG_OK;
    }
};

int ensure_events(ctg_ctx *ctx);

// ---------------------------------------------------------------------------
// AB-GMRES and BA-GMRES (Sec. 2 algorithm box) as a loop that runs on the
// device.  The kernels of a step read k from the solve's device state
// (GmresState); the FP64 Givens update, y_k and the stopping rule of Sec.
// 6.4 are device kernels too (gmres_loop.cu), and the kernel that ends a
// step advances k or stops the solve.  So the whole solve is one CUDA graph:
// the start (r0, beta, w_1), two while-loop nodes over the steps (the first
// with the one-launch CGS2 step for k <= 128, or 64 where the step forms
// y_k, the second with its separate
// passes) and the exit (y_k, x_k and its true residual), launched once and
// read back once.  With phase tracing on (or where such a graph cannot be
// built) the host enqueues the same kernels step by step instead and reads
// the activity flag after each step.
//
// A step, AB (basis length m):  t = B w_k;  q = A t;  CGS2;  Givens and
//   the stop (DP on rho_k = ||b - A x_k||, equal in exact arithmetic).
//   With NCP: y_k, r_k = W_{k+1} z_k, its NCP distance, the stop.
// A step, BA (basis length n), with t_k = A w_k from the step before:
//   q = B t_k;  CGS2;  Givens;  with DP / NCP x_k = x0 + W_k y_k, then
//   t_{k+1} = A w_{k+1} and A x_k in one two-image walk, ||b - A x_k||
//   (and its NCP distance) and the stop.  No A W_k is stored: the basis is
//   the only O(k L) storage, the storage law of Table 3.

struct LoopPlan {
    int variant, rule, maxit;
    double target;
    bool fused;        // the one-launch CGS2 step serves k <= fused_max
    int fused_max;
    int small_max;     // ... on one block per SM for k <= small_max (0: none)
    bool cooperative;  // launch it cooperatively
};

int enqueue_init(SolveCtx &sc, const LoopPlan &lp, const float *b, const float *x0, const LoopBufs &B) {
    const int64_t n = sc.ly.n, m = sc.ly.m;
    double *scal = sc.rs.scal;
    if (lp.variant == CTG_AB) {
        // r0 = b - A x0 in vm0, ||r0||^2 -> scal[2]
        if (x0) {
            CTG_CK(sc.forward(x0, sc.vm0()));
            CTG_CK(sc.sub_norm2(b, sc.vm0(), sc.vm0(), m, scal + 2));
        } else {
            CTG_CK(sc.sub_norm2(b, nullptr, sc.vm0(), m, scal + 2));
        }
        if (lp.rule == kRuleNCP) CTG_CK(sc.ncp(sc.vm0(), scal + 6));
        CTG_CK(sc.scale(sc.vm0(), scal + 2, sc.Wcol(0), m));              // w_1 = r0 / beta
    } else {
        // r = b - A x0 in vm1 (||r||^2 -> scal[4]); r0 = B r, ||r0||^2 -> scal[2]
        if (x0) {
            CTG_CK(sc.forward(x0, sc.vm0()));
            CTG_CK(sc.sub_norm2(b, sc.vm0(), sc.vm1(), m, scal + 4));
        } else {
            CTG_CK(sc.sub_norm2(b, nullptr, sc.vm1(), m, scal + 4));
        }
        if (lp.rule == kRuleNCP) CTG_CK(sc.ncp(sc.vm1(), scal + 6));
        CTG_CK(sc.back(sc.vm1(), nullptr, sc.vn0()));
        CTG_CK(sc.sub_norm2(sc.vn0(), nullptr, nullptr, n, scal + 2));
        CTG_CK(sc.scale(sc.vn0(), scal + 2, sc.Wcol(0), n));              // w_1 = r0 / beta
        CTG_CK(sc.forward(sc.Wcol(0), sc.vm0(), sc.ly.dtype));            // t_1 = A w_1
    }
    CTG_CK(traced(sc.ctx, 3, 1, sc.st, [&] {
        return ctg_loop_init(B, lp.variant, lp.rule, lp.maxit, lp.target, sc.st);
    }));
    return CTG_OK;
}

int enqueue_step(SolveCtx &sc, const LoopPlan &lp, const float *b, const float *x0, float *x,
                 const LoopBufs &B, bool fused, bool small_grid = false) {
    const int64_t n = sc.ly.n, m = sc.ly.m;
    const int *kdev = &sc.state()->k;
    const int kmax = fused ? lp.fused_max : lp.maxit;
    auto givens = [&](bool need_y, bool need_z, bool end) {
        return traced(sc.ctx, 3, 1, sc.st, [&] {
            return ctg_loop_givens(B, need_y, need_z, end, lp.maxit, sc.st);
        });
    };
    // the Givens update runs in the fused CGS2 step's block 0, else on its own
    auto cgs2_givens = [&](int64_t L, float *q, bool need_y, bool need_z, bool end) -> int {
        if (fused) {
            const int mode = (need_y ? kGivY : 0) | (need_z ? kGivZ : 0) | (end ? kGivEnd : 0);
            CTG_CK(sc.cgs2_loop(L, q, kmax, true, lp.cooperative, &B, mode, small_grid));
            return CTG_OK;
        }
        CTG_CK(sc.cgs2_loop(L, q, kmax, false, lp.cooperative));
        CTG_CK(givens(need_y, need_z, end));
        return CTG_OK;
    };
    if (lp.variant == CTG_AB) {
        CTG_CK(sc.back(sc.W(), nullptr, sc.vn0(), sc.ly.dtype, col_at(kdev, -1, (long long)sc.ly.ld_w)));
        CTG_CK(sc.forward(sc.vn0(), sc.vm0()));                           // q = A B w_k
        const bool ncp = lp.rule == kRuleNCP;
        if (const int rc = cgs2_givens(m, sc.vm0(), ncp, ncp, !ncp)) return rc;
        if (ncp) {
            // r_k = W_{k+1} z_k, its NCP distance, the stop
            CTG_CK(sc.gemv_dev(m, kdev, 1, kmax + 1, B.z, nullptr, sc.vm1()));
            CTG_CK(sc.ncp(sc.vm1(), sc.rs.scal + 6));
            CTG_CK(traced(sc.ctx, 3, 1, sc.st, [&] { return ctg_loop_ncp_decide(B, sc.st); }));
        }
        return CTG_OK;
    }
    CTG_CK(sc.back(sc.vm0(), nullptr, sc.vn0()));                         // q = B t_k
    const bool resid = lp.rule != kRuleMaxit;
    if (const int rc = cgs2_givens(n, sc.vn0(), resid, false, false)) return rc;
    const ColRef wnext = col_at(kdev, 0, (long long)sc.ly.ld_w);         // w_{k+1}
    if (!resid) {
        CTG_CK(sc.forward(sc.W(), sc.vm0(), sc.ly.dtype, wnext));         // t_{k+1}
        CTG_CK(traced(sc.ctx, 3, 1, sc.st, [&] { return ctg_loop_advance(B, sc.st); }));
        return CTG_OK;
    }
    CTG_CK(sc.gemv_dev(n, kdev, 0, kmax, B.y, x0, x));                   // x_k = x0 + W_k y_k
    CTG_CK(sc.forward2(wnext, x, sc.vm0(), sc.vm1()));                    // t_{k+1}, A x_k
    if (lp.rule == kRuleDP) {
        CTG_CK(traced(sc.ctx, 3, 1, sc.st, [&] {
            return ctg_loop_resid(B, b, sc.vm1(), nullptr, m, sc.rs, true, sc.st);
        }));
    } else {
        CTG_CK(traced(sc.ctx, 3, 1, sc.st, [&] {
            return ctg_loop_resid(B, b, sc.vm1(), sc.vm1(), m, sc.rs, false, sc.st);
        }));
        CTG_CK(sc.ncp(sc.vm1(), sc.rs.scal + 6));
        CTG_CK(traced(sc.ctx, 3, 1, sc.st, [&] { return ctg_loop_ncp_decide(B, sc.st); }));
    }
    return CTG_OK;
}

// y of the returned iterate, x = x0 + B W y (AB) or x0 + W y (BA), and
// ||b - A x||.
int enqueue_exit(SolveCtx &sc, const LoopPlan &lp, const float *b, const float *x0, float *x,
                 const LoopBufs &B) {
    const int *idev = &sc.state()->iters;
    CTG_CK(traced(sc.ctx, 3, 1, sc.st, [&] { return ctg_loop_exit_y(B, lp.maxit, sc.st); }));
    if (lp.variant == CTG_AB) {
        CTG_CK(sc.gemv_dev(sc.ly.m, idev, 0, lp.maxit, B.y, nullptr, sc.vm0()));
        CTG_CK(sc.back(sc.vm0(), x0, x));
    } else {
        CTG_CK(sc.gemv_dev(sc.ly.n, idev, 0, lp.maxit, B.y, x0, x));
        // BA with the DP stop already has ||b - A x|| of this very iterate
        // (the same y, the same sweep, projected and reduced by the same
        // arithmetic in the step that stopped; at k = 0 the start's residual)
        if (lp.rule == kRuleDP) return CTG_OK;
    }
    CTG_CK(sc.forward(x, sc.vm1()));
    CTG_CK(sc.sub_norm2(b, sc.vm1(), nullptr, sc.ly.m, sc.rs.scal + 5));
    CTG_CK(traced(sc.ctx, 3, 1, sc.st, [&] { return ctg_loop_final(B, sc.st); }));
    return CTG_OK;
}

int ensure_capture_streams(ctg_ctx *ctx) {
    for (int i = 0; i < 2; ++i)
        if (!ctx->cap_st[i]) CTG_CK(cudaStreamCreateWithFlags(&ctx->cap_st[i], cudaStreamNonBlocking));
    return CTG_OK;
}

// Captures the whole solve into an executable graph (see above).
int build_loop_graph(SolveCtx &sc, const LoopPlan &lp, const float *b, const float *x0, float *x,
                     ctg_ctx::LoopGraph *out) {
    ctg_ctx *ctx = sc.ctx;
    int rc = ensure_capture_streams(ctx);
    if (rc) return rc;
    cudaStream_t user = sc.st;
    cudaStream_t cs = ctx->cap_st[0], bs = ctx->cap_st[1];
    const bool use_small = lp.fused && lp.small_max > 0;
    const bool use_fused = lp.fused && lp.fused_max > lp.small_max;
    const bool use_pass = !lp.fused || lp.maxit > lp.fused_max;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    ctx->capturing = true;
    auto fail = [&](cudaError_t e) {
        ctx->capturing = false;
        sc.st = user;
        cudaStreamCaptureStatus st_ = cudaStreamCaptureStatusNone;
        for (cudaStream_t q : {cs, bs})
            if (cudaStreamIsCapturing(q, &st_) == cudaSuccess && st_ != cudaStreamCaptureStatusNone) {
                cudaGraph_t g2 = nullptr;
                cudaStreamEndCapture(q, &g2);
                if (g2) cudaGraphDestroy(g2);
            }
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return fail_cuda(e == cudaSuccess ? cudaErrorUnknown : e);
    };
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) return fail(e);
    LoopBufs B = sc.loop_bufs();
    B.in_graph = 1;
    B.fused_max = lp.fused ? lp.fused_max : 0;
    B.small_max = use_small ? lp.small_max : 0;
    // the handles belong to the graph being captured
    cudaStreamCaptureStatus cstat;
    cudaGraph_t cg = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    size_t ndeps = 0;
    if ((e = cudaStreamGetCaptureInfo(cs, &cstat, nullptr, &cg, &deps, nullptr, &ndeps)) != cudaSuccess)
        return fail(e);
    if ((e = cudaGraphConditionalHandleCreate(&B.c_small, cg, use_small ? 1u : 0u, cudaGraphCondAssignDefault)) !=
        cudaSuccess)
        return fail(e);
    if ((e = cudaGraphConditionalHandleCreate(&B.c_fused, cg, use_fused ? 1u : 0u, cudaGraphCondAssignDefault)) !=
        cudaSuccess)
        return fail(e);
    if ((e = cudaGraphConditionalHandleCreate(&B.c_pass, cg, 1u, cudaGraphCondAssignDefault)) != cudaSuccess)
        return fail(e);
    const long long k0 = ctx->captured_kernels;
    sc.st = cs;
    if ((rc = enqueue_init(sc, lp, b, x0, B))) return fail(cudaErrorUnknown);
    out->n_init = (int)(ctx->captured_kernels - k0);
    // while-loop nodes: their bodies are captured on the second stream
    auto add_loop = [&](cudaGraphConditionalHandle h, bool fused, bool small_grid, int *nkern) -> cudaError_t {
        cudaError_t e2 = cudaStreamGetCaptureInfo(cs, &cstat, nullptr, &cg, &deps, nullptr, &ndeps);
        if (e2 != cudaSuccess) return e2;
        cudaGraphNodeParams cp = {};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t node;
        if ((e2 = cudaGraphAddNode(&node, cg, deps, nullptr, ndeps, &cp)) != cudaSuccess) return e2;
        if ((e2 = cudaStreamUpdateCaptureDependencies(cs, &node, nullptr, 1, cudaStreamSetCaptureDependencies)) !=
            cudaSuccess)
            return e2;
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        if ((e2 = cudaStreamBeginCaptureToGraph(bs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed)) !=
            cudaSuccess)
            return e2;
        sc.st = bs;
        const long long kb = ctx->captured_kernels;
        const int rc2 = enqueue_step(sc, lp, b, x0, x, B, fused, small_grid);
        *nkern = (int)(ctx->captured_kernels - kb);
        sc.st = cs;
        cudaGraph_t body_out = nullptr;
        const cudaError_t e3 = cudaStreamEndCapture(bs, &body_out);
        if (rc2) return cudaErrorUnknown;
        return e3;
    };
    out->n_small = out->n_fused = out->n_pass = 0;
    if (use_small && (e = add_loop(B.c_small, true, true, &out->n_small)) != cudaSuccess) return fail(e);
    if (use_fused && (e = add_loop(B.c_fused, true, false, &out->n_fused)) != cudaSuccess) return fail(e);
    if (use_pass && (e = add_loop(B.c_pass, false, false, &out->n_pass)) != cudaSuccess) return fail(e);
    const long long ke = ctx->captured_kernels;
    if ((rc = enqueue_exit(sc, lp, b, x0, x, B))) return fail(cudaErrorUnknown);
    out->n_exit = (int)(ctx->captured_kernels - ke);
    if ((e = cudaStreamEndCapture(cs, &graph)) != cudaSuccess) return fail(e);
    ctx->capturing = false;
    sc.st = user;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    graph = nullptr;
    if (e != cudaSuccess) return fail(e);
    out->exec = exec;
    out->small_max = B.small_max;
    out->fused_max = B.fused_max;
    return CTG_OK;
}

// Reads the solve's outcome back and fills *info.
int read_outcome(SolveCtx &sc, const LoopPlan &lp, ctg_info *info, GmresState *hs) {
    double *pin = sc.pinned_scratch();
    const size_t sd = (sizeof(GmresState) + sizeof(double) - 1) / sizeof(double);
    CTG_CK(cudaMemcpyAsync(pin, sc.state(), sizeof(GmresState), cudaMemcpyDeviceToHost, sc.st));
    CTG_CK(cudaMemcpyAsync(pin + sd, sc.at<double>(sc.ly.off_hist), sizeof(double) * (lp.maxit + 1),
                           cudaMemcpyDeviceToHost, sc.st));
    if (lp.rule == kRuleNCP)
        CTG_CK(cudaMemcpyAsync(pin + sd + lp.maxit + 1, sc.at<double>(sc.ly.off_ncph),
                               sizeof(double) * (lp.maxit + 2), cudaMemcpyDeviceToHost, sc.st));
    CTG_CK(cudaStreamSynchronize(sc.st));
    std::memcpy(hs, pin, sizeof(GmresState));
    info->iters = hs->iters;
    info->stop_reason = hs->stop_reason;
    info->rho = hs->rho;
    info->resnorm = hs->resnorm;
    if (info->history)
        for (int k = 0; k <= hs->iters; ++k) info->history[k] = pin[sd + k];
    if (info->ncp_history && lp.rule == kRuleNCP) {
        // d_0 .. d_{iters+1} at an NCP stop, else the distances evaluated
        const int last = hs->stop_reason == CTG_STOP_NCP ? hs->iters + 1 : hs->iters;
        for (int k = 0; k <= last; ++k) info->ncp_history[k] = pin[sd + lp.maxit + 1 + k];
    }
    return hs->timed_out ? CTG_ERR_TIMEOUT : CTG_OK;
}

int run_gmres(SolveCtx &sc, int variant, const float *b, const float *x0, float *x, const ctg_opts *o,
              ctg_info *info) {
    ctg_ctx *ctx = sc.ctx;
    LoopPlan lp{};
    lp.variant = variant;
    lp.rule = rule_of(o);
    lp.maxit = o->maxit;
    lp.target = lp.rule == kRuleDP ? o->tau * o->noise_norm : 0.0;
    // steps that form y_k (BA with a residual rule, AB with NCP) take the
    // one-launch step up to a smaller k than those that do not
    const bool need_y = variant == CTG_AB ? lp.rule == kRuleNCP : lp.rule != kRuleMaxit;
    lp.fused_max = std::min(o->maxit, ctg_cgs2_fused_max(need_y));
    lp.fused = ctg_cgs2_fused_ok(sc.ly.dtype, sc.ly.L, lp.fused_max, sc.rs);
    if (!lp.fused) lp.fused_max = 0;
    lp.small_max = lp.fused && ctg_cgs2_fused_ok(sc.ly.dtype, sc.ly.L, lp.fused_max, sc.rs, true)
                       ? std::min(lp.fused_max, ctg_cgs2_small_grid_max())
                       : 0;
    int rc = CTG_OK;
    if (lp.rule == kRuleNCP && (rc = ensure_twiddles(sc.ge))) return rc;
    GmresState hs{};
    if (!ctx->timing && ctx->graph_mode >= 0) {
        lp.cooperative = ctx->graph_mode != 2;
        // the captured graph bakes in every pointer and option of the solve
        long long target_bits = 0;
        std::memcpy(&target_bits, &lp.target, sizeof(double));
        const std::vector<long long> key = {
            (long long)sc.ge->serial, sc.ge->fwd_shape, sc.ge->back_chunk, variant, o->maxit,
            o->basis_dtype, lp.rule, target_bits, (long long)(uintptr_t)sc.ws,
            (long long)(uintptr_t)b, (long long)(uintptr_t)x0, (long long)(uintptr_t)x, ctx->spin_limit,
            lp.cooperative ? 1 : 0, lp.fused ? 1 : 0};
        size_t gi = ctx->graphs.size();
        for (size_t i = 0; i < ctx->graphs.size(); ++i)
            if (ctx->graphs[i].key == key) gi = i;
        if (gi == ctx->graphs.size()) {
            ctg_ctx::LoopGraph lg{};
            lg.key = key;
            lg.geom_serial = sc.ge->serial;
            rc = build_loop_graph(sc, lp, b, x0, x, &lg);
            if (rc != CTG_OK && lp.cooperative) {
                // a cooperative launch may not be capturable inside a loop
                // body: fall back to the occupancy-checked plain launch
                lp.cooperative = false;
                lg.key[13] = 0;
                rc = build_loop_graph(sc, lp, b, x0, x, &lg);
                if (rc == CTG_OK) ctx->graph_mode = 2;
            }
            if (rc != CTG_OK) {
                ctx->graph_mode = -1;                  // no graphs here: the host drives the loop
            } else {
                if (ctx->graph_mode == 0) ctx->graph_mode = 1;
                if (ctx->graphs.size() >= 16) {
                    cudaGraphExecDestroy(ctx->graphs.front().exec);
                    ctx->graphs.erase(ctx->graphs.begin());
                }
                ctx->graphs.push_back(lg);
                gi = ctx->graphs.size() - 1;
            }
        } else {
            // most recently used last
            std::rotate(ctx->graphs.begin() + gi, ctx->graphs.begin() + gi + 1, ctx->graphs.end());
            gi = ctx->graphs.size() - 1;
        }
        if (ctx->graph_mode > 0) {
            const ctg_ctx::LoopGraph &lg = ctx->graphs[gi];
            CTG_CK(cudaGraphLaunch(lg.exec, sc.st));
            rc = read_outcome(sc, lp, info, &hs);
            const long long steps = hs.steps;
            const long long ss = lg.n_small ? std::min<long long>(steps, lg.small_max) : 0;
            const long long sf = lg.n_fused ? std::min<long long>(steps, lg.fused_max) - ss : 0;
            ctx->kernels += lg.n_init + lg.n_exit + ss * lg.n_small + sf * lg.n_fused + (steps - ss - sf) * lg.n_pass;
            return rc;
        }
    }
    // host-driven: the same kernels, one step at a time
    lp.cooperative = true;
    LoopBufs B = sc.loop_bufs();
    B.in_graph = 0;
    B.fused_max = lp.fused ? lp.fused_max : 0;
    B.small_max = lp.fused ? lp.small_max : 0;
    if ((rc = enqueue_init(sc, lp, b, x0, B))) return rc;
    int *flag = reinterpret_cast<int *>(sc.pinned_scratch());
    if ((rc = ensure_events(ctx))) return rc;
    for (int k = 1; k <= lp.maxit; ++k) {
        // the step is skipped when the start already stopped the solve
        if (k == 1) {
            CTG_CK(cudaMemcpyAsync(flag, &sc.state()->active, sizeof(int), cudaMemcpyDeviceToHost, sc.st));
            CTG_CK(cudaEventRecord(ctx->ev_init, sc.st));
            CTG_CK(cudaEventSynchronize(ctx->ev_init));
            if (!*flag) break;
        }
        if ((rc = enqueue_step(sc, lp, b, x0, x, B, lp.fused && k <= lp.fused_max,
                               lp.fused && k <= lp.small_max)))
            return rc;
        CTG_CK(cudaMemcpyAsync(flag, &sc.state()->active, sizeof(int), cudaMemcpyDeviceToHost, sc.st));
        CTG_CK(cudaEventRecord(ctx->ev_init, sc.st));
        CTG_CK(cudaEventSynchronize(ctx->ev_init));
        if (!*flag) break;
    }
    if ((rc = enqueue_exit(sc, lp, b, x0, x, B))) return rc;
    return read_outcome(sc, lp, info, &hs);
}

// LSQR / LSMR (Sec. 5's comparators) with the geometry's back projector in
// the role of A^T.  Each iteration is enqueued before the host reads the
// previous one's `live` flag; the device decides the stop, so an iteration
// enqueued after it changes nothing.
int run_lsq(SolveCtx &sc, int method, const float *b, const float *x0, float *x,
            const ctg_opts *o, ctg_info *info) {
    const int64_t n = sc.ly.n, m = sc.ly.m;
    char *ws = sc.ws;
    auto nv = [&](int i) { return reinterpret_cast<float *>(ws + sc.ly.off_n[i]); };
    auto mv = [&](int i) { return reinterpret_cast<float *>(ws + sc.ly.off_m[i]); };
    float *v = nv(0), *a = nv(1), *c = method == CTG_LSMR ? nv(2) : nullptr, *q = nv(3);
    float *u = mv(0), *p = mv(1);
    LsqState *S = reinterpret_cast<LsqState *>(ws + sc.ly.off_state);
    double *hist = reinterpret_cast<double *>(ws + sc.ly.off_hist);
    const bool dp = o->noise_norm > 0.0;
    const double target = dp ? o->tau * o->noise_norm : 0.0;
    // u~_1 = b - A x0, beta_1^2 = ||u~_1||^2 (into S->beta2)
    if (x0) {
        CTG_CK(sc.forward(x0, p));
        CTG_CK(sc.sub_norm2(b, p, u, m, &S->beta2));
    } else {
        CTG_CK(sc.sub_norm2(b, nullptr, u, m, &S->beta2));
    }
    // v~_1 = B u~_1 / beta_1, alpha_1^2 = ||v~_1||^2
    CTG_CK(cudaMemsetAsync(v, 0, sizeof(float) * n, sc.st));
    CTG_CK(sc.back(u, nullptr, q));
    CTG_CK(traced(sc.ctx, 3, 1, sc.st, [&] { return ctg_lsq_bidiag_v(q, v, n, S, sc.rs, sc.st); }));
    double *hp;
    int rc = sc.fetch(&S->alpha2, 2, &hp);   // alpha2, beta2
    if (rc) return rc;
    const double alpha = std::sqrt(hp[0]), beta = std::sqrt(hp[1]);
    info->rho = beta;
    info->resnorm = beta;
    if (info->history) info->history[0] = beta;
    if ((dp && beta <= target) || beta == 0.0 || alpha == 0.0) {
        info->stop_reason = dp && beta <= target ? CTG_STOP_DP : CTG_STOP_BREAKDOWN;
        return copy_x0(sc, x0, x);
    }
    LsqState h0{};
    h0.alpha2 = hp[0];
    h0.beta2 = hp[1];
    h0.alpha = alpha;
    h0.beta = beta;
    h0.rhobar = alpha;
    h0.phibar = beta;
    h0.alphabar = alpha;
    h0.zetabar = alpha * beta;
    h0.rho_old = 1.0;
    h0.rhobar_old = 1.0;
    h0.cbar = 1.0;
    h0.sbar = 0.0;
    h0.inv_alpha = 1.0 / alpha;
    h0.target = target;
    h0.hist = hist;
    h0.method = method;
    h0.k = 1;
    h0.maxit = o->maxit;
    h0.live = 1;
    h0.live_update = 1;
    h0.stop_reason = CTG_STOP_MAXIT;
    h0.status[0] = 1.0;
    h0.status[1] = beta;
    double *stage = sc.pinned_scratch();
    static_assert(sizeof(LsqState) % sizeof(double) == 0, "LsqState is staged as doubles");
    static_assert(sizeof(LsqState) / sizeof(double) + 1 <= 64, "pinned staging area");
    std::memcpy(stage, &h0, sizeof(LsqState));
    stage[sizeof(LsqState) / sizeof(double)] = beta;          // history[0] = ||r_0||
    CTG_CK(cudaMemcpyAsync(S, stage, sizeof(LsqState), cudaMemcpyHostToDevice, sc.st));
    CTG_CK(cudaMemcpyAsync(hist, stage + sizeof(LsqState) / sizeof(double), sizeof(double),
                           cudaMemcpyHostToDevice, sc.st));
    if ((rc = copy_x0(sc, x0, x))) return rc;
    CTG_CK(ctg_lsq_start(S, v, a, c, n, sc.st));
    if (method == CTG_LSMR) {
        CTG_CK(cudaMemcpyAsync(mv(4), u, sizeof(float) * m, cudaMemcpyDeviceToDevice, sc.st));  // r_0
        CTG_CK(cudaMemsetAsync(mv(2), 0, sizeof(float) * m, sc.st));
        CTG_CK(cudaMemsetAsync(mv(3), 0, sizeof(float) * m, sc.st));
    }
    if ((rc = ensure_events(sc.ctx))) return rc;
    Pipeline pl{sc, o->maxit, sc.ctx->ev_h, sc.ctx->ev_r};
    auto enqueue = [&](int kk) -> int {
        CTG_CK(sc.forward(v, p));                                              // p = A v_k
        CTG_CK(traced(sc.ctx, 3, 1, sc.st, [&] { return ctg_lsq_bidiag_u(p, u, m, S, sc.rs, sc.st); }));
        CTG_CK(sc.back(u, nullptr, q));                                        // q = B u~_{k+1}
        CTG_CK(traced(sc.ctx, 3, 4, sc.st, [&] {
            cudaError_t e = ctg_lsq_bidiag_v(q, v, n, S, sc.rs, sc.st);
            if (e == cudaSuccess) e = ctg_lsq_scalars(S, sc.st);
            if (e == cudaSuccess) e = ctg_lsq_update(S, v, a, c, x, n, sc.st);
            if (e == cudaSuccess && method == CTG_LSMR)
                e = ctg_lsq_residual(S, p, mv(2), mv(3), mv(4), m, sc.rs, sc.st);
            return e;
        }));
        double *sl = pl.slot(kk);
        CTG_CK(cudaMemcpyAsync(sl, S->status, sizeof(double) * 2, cudaMemcpyDeviceToHost, sc.st));
        CTG_CK(cudaEventRecord(pl.ev_h[kk % kRing], sc.st));
        return CTG_OK;
    };
    int next = 1;
    for (int k = 1; k <= o->maxit; ++k) {
        if (next == k && (rc = enqueue(next++))) return rc;
        if (next == k + 1 && k + 1 <= o->maxit && (rc = enqueue(next++))) return rc;
        const double *st;
        if ((rc = pl.wait_step(k, &st))) return rc;
        if (st[0] == 0.0) break;
    }
    // final state, history and the true residual of x
    double *fin;
    if ((rc = sc.fetch(reinterpret_cast<const double *>(S), sizeof(LsqState) / sizeof(double), &fin)))
        return rc;
    LsqState hs;
    std::memcpy(&hs, fin, sizeof(LsqState));
    info->iters = hs.iters;
    info->stop_reason = hs.stop_reason;
    info->rho = hs.status[1];
    if (info->history && hs.iters > 0)
        CTG_CK(cudaMemcpyAsync(info->history + 1, hist + 1, sizeof(double) * hs.iters,
                               cudaMemcpyDeviceToHost, sc.st));
    return sc.true_resnorm(b, x, &info->resnorm);
}

int solve(int variant, ctg_ctx *ctx, const ctg_geom *g, const float *b, const float *x0,
          float *x, const ctg_opts *o, void *ws, size_t ws_bytes, ctg_info *info,
          void *stream) {
    if (x0 && !aligned16(x0)) return CTG_ERR_INVALID_ARG;
    SolveCtx sc;
    void *owned = nullptr;
    int rc = solve_setup(ctx, g, variant, o, b, x, ws, ws_bytes, info, stream, &sc, &owned);
    if (rc) {
        if (owned) cudaFreeAsync(owned, sc.st);
        return rc;
    }
    rc = (variant == CTG_AB || variant == CTG_BA) ? run_gmres(sc, variant, b, x0, x, o, info)
                                                  : run_lsq(sc, variant, b, x0, x, o, info);
    if (rc == CTG_OK) {
        cudaError_t e = cudaStreamSynchronize(sc.st);
        if (e != cudaSuccess) rc = fail_cuda(e);
    }
    if (rc == CTG_OK) rc = resolve_marks(ctx);
    return finish(sc, owned, rc);
}

}  // namespace

extern "C" {

int ctg_create(ctg_ctx **out) {
    if (!out) return CTG_ERR_INVALID_ARG;
    ctg_ctx *c = new (std::nothrow) ctg_ctx();
    if (!c) return CTG_ERR_OOM;
    if (cudaGetDevice(&c->device) != cudaSuccess) {
        delete c;
        return CTG_ERR_CUDA;
    }
    *out = c;
    return CTG_OK;
}

void ctg_destroy(ctg_ctx *ctx) {
    if (!ctx) return;
    cudaDeviceSynchronize();
    for (auto ev : ctx->events) cudaEventDestroy(ev);
    for (int i = 0; i < 4; ++i) {
        if (ctx->ev_h[i]) cudaEventDestroy(ctx->ev_h[i]);
        if (ctx->ev_r[i]) cudaEventDestroy(ctx->ev_r[i]);
    }
    for (auto &e : ctx->cache) {
        cudaFree(e.fwd);
        cudaFree(e.back);
        cudaFree(e.fwd_order);
        cudaFree(e.pad);
        cudaFree(e.mt);
        cudaFree(e.tw);
    }
    drop_graphs(ctx, 0);
    for (cudaStream_t q : ctx->cap_st)
        if (q) cudaStreamDestroy(q);
    if (ctx->ev_init) cudaEventDestroy(ctx->ev_init);
    if (ctx->pinned) cudaFreeHost(ctx->pinned);
    delete ctx;
}

int ctg_set_wait_limit(ctg_ctx *ctx, int64_t polls) {
    if (!ctx || polls < 0) return CTG_ERR_INVALID_ARG;
    ctx->spin_limit = polls == 0 ? kCtgDefaultSpinLimit : (long long)polls;
    return CTG_OK;
}

int ctg_project(ctg_ctx *ctx, const ctg_geom *g, const float *x_dev, float *b_dev, void *stream) {
    if (!ctx || !geom_valid(g) || !x_dev || !b_dev) return CTG_ERR_INVALID_ARG;
    GeomEntry *ge;
    int rc = get_geom(ctx, g, &ge);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (!ge->pad) {
        const size_t bytes = sizeof(float) * ge->pl.floats;
        CTG_CK(cudaMalloc(&ge->pad, bytes));
        CTG_CK(cudaMemsetAsync(ge->pad, 0, bytes, st));   // ordered before the staging on st
    }
    CTG_CK(traced(ctx, 3, 1, st, [&] {
        return ctg_launch_pad(x_dev, CTG_BASIS_FP32, ge->pad, g->N, ge->pl, st);
    }));
    CTG_CK(traced(ctx, 0, 1, st, [&] {
        return ctg_launch_forward(ge->pad, g->N, ge->pl, g->n_angles, g->n_det, ge->fwd, b_dev, st,
                                  ge->fwd_shape, ge->order_for(ge->fwd_shape));
    }));
    return CTG_OK;
}

int ctg_backproject(ctg_ctx *ctx, const ctg_geom *g, const float *b_dev, float *x_dev, void *stream) {
    if (!ctx || !geom_valid(g) || !b_dev || !x_dev) return CTG_ERR_INVALID_ARG;
    GeomEntry *ge;
    int rc = get_geom(ctx, g, &ge);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    CTG_CK(traced(ctx, 1, 1, st, [&] { return back_apply(ge, b_dev, CTG_BASIS_FP32, nullptr, x_dev, st); }));
    return CTG_OK;
}

int ctg_set_tiles(ctg_ctx *ctx, int32_t fwd_angles, int32_t back_chunk) {
    if (!ctx || (fwd_angles != 0 && fwd_angles != 4 && fwd_angles != 8) ||
        (back_chunk != 0 && back_chunk != 16 && back_chunk != 32 && back_chunk != 64))
        return CTG_ERR_INVALID_ARG;
    ctx->force_fwd_angles = fwd_angles;
    ctx->force_fwd_split = 1;
    ctx->force_back_chunk = back_chunk;
    return CTG_OK;    // applied to every geometry at its next use
}

int ctg_set_fwd_tiles(ctg_ctx *ctx, int32_t angles_per_block, int32_t angles_per_warp) {
    if (!ctx) return CTG_ERR_INVALID_ARG;
    if (angles_per_block == 0 && angles_per_warp == 0) {
        ctx->force_fwd_angles = 0;
        ctx->force_fwd_split = 1;
        return CTG_OK;
    }
    for (int c = 0; c < kFwdShapes; ++c)
        if (kFwdShapeAngles[c] == angles_per_block && kFwdShapeSplit[c] == angles_per_warp) {
            ctx->force_fwd_angles = angles_per_block;
            ctx->force_fwd_split = angles_per_warp;
            return CTG_OK;
        }
    return CTG_ERR_INVALID_ARG;
}

int ctg_get_tuning(ctg_ctx *ctx, const ctg_geom *g, ctg_tuning *out) {
    if (!ctx || !geom_valid(g) || !out) return CTG_ERR_INVALID_ARG;
    GeomEntry *ge;
    const int rc = get_geom(ctx, g, &ge);
    if (rc) return rc;
    out->fwd_angles = kFwdShapeAngles[ge->fwd_shape];
    out->back_chunk = ge->back_chunk;
    out->tuned = ge->tuned ? 1 : 0;
    for (int c = 0; c < 2; ++c) out->fwd_us[c] = ge->fwd_us[c];
    for (int c = 0; c < 3; ++c) out->back_us[c] = ge->back_us[c];
    out->fwd_warp_angles = kFwdShapeSplit[ge->fwd_shape];
    for (int c = 0; c < 2; ++c) out->fwd_split_us[c] = ge->fwd_us[2 + c];
    return CTG_OK;
}

int ctg_ncp_distance(ctg_ctx *ctx, const ctg_geom *g, const float *r_dev, double *out, void *stream) {
    if (!ctx || !geom_valid(g) || !r_dev || !out || g->n_det < 2 || g->n_det > kCtgNcpMaxDet)
        return CTG_ERR_INVALID_ARG;
    GeomEntry *ge;
    int rc = get_geom(ctx, g, &ge);
    if (rc) return rc;
    if ((rc = ensure_twiddles(ge))) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    double *scratch = nullptr;
    CTG_CK(cudaMallocAsync(&scratch, sizeof(double) * ((size_t)g->n_angles + 1), st));
    cudaError_t e = ctg_ncp(r_dev, g->n_angles, g->n_det, ge->tw, scratch + 1, scratch, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, scratch, sizeof(double), cudaMemcpyDeviceToHost, st);
    const cudaError_t e2 = cudaFreeAsync(scratch, st);
    const cudaError_t e3 = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = e2 != cudaSuccess ? e2 : e3;
    return e == cudaSuccess ? CTG_OK : fail_cuda(e);
}

size_t ctg_workspace_bytes(const ctg_geom *g, int variant, const ctg_opts *o) {
    WsLayout ly;
    return layout_of(g, variant, o, &ly) ? ly.total : 0;
}

int ctg_workspace_layout(const ctg_geom *g, int variant, const ctg_opts *o, ctg_layout *out) {
    WsLayout ly;
    if (!out || !layout_of(g, variant, o, &ly)) return CTG_ERR_INVALID_ARG;
    out->off_w = ly.off_w;
    out->ld_w = ly.ld_w;
    out->off_h = ly.off_h;
    out->total_bytes = ly.total;
    return CTG_OK;
}

int ctg_ab_gmres(ctg_ctx *ctx, const ctg_geom *g, const float *b_dev, const float *x0_dev,
                 float *x_dev, const ctg_opts *o, void *workspace_dev, size_t workspace_bytes,
                 ctg_info *info, void *stream) {
    return solve(CTG_AB, ctx, g, b_dev, x0_dev, x_dev, o, workspace_dev, workspace_bytes, info, stream);
}

int ctg_lsqr(ctg_ctx *ctx, const ctg_geom *g, const float *b_dev, const float *x0_dev, float *x_dev,
             const ctg_opts *opts, void *workspace, size_t workspace_bytes, ctg_info *info,
             void *stream) {
    return solve(CTG_LSQR, ctx, g, b_dev, x0_dev, x_dev, opts, workspace, workspace_bytes, info, stream);
}

int ctg_lsmr(ctg_ctx *ctx, const ctg_geom *g, const float *b_dev, const float *x0_dev, float *x_dev,
             const ctg_opts *opts, void *workspace, size_t workspace_bytes, ctg_info *info,
             void *stream) {
    return solve(CTG_LSMR, ctx, g, b_dev, x0_dev, x_dev, opts, workspace, workspace_bytes, info, stream);
}

int ctg_ba_gmres(ctg_ctx *ctx, const ctg_geom *g, const float *b_dev, const float *x0_dev,
                 float *x_dev, const ctg_opts *o, void *workspace_dev, size_t workspace_bytes,
                 ctg_info *info, void *stream) {
    return solve(CTG_BA, ctx, g, b_dev, x0_dev, x_dev, o, workspace_dev, workspace_bytes, info, stream);
}

size_t ctg_cgs2_scratch_bytes(int64_t L, int32_t k) {
    if (L < 1 || k < 0 || k > kMaxIt) return 0;
    return ctg_red_scratch_bytes(L, k + 1);
}

int ctg_cgs2(const float *W_dev, int64_t ld_w, int64_t L, int32_t k, float *q_dev,
             float *w_out_dev, double *h_out_dev, void *scratch_dev, size_t scratch_bytes,
             void *stream) {
    if (L < 1 || k < 0 || k > kMaxIt || ld_w < L || (ld_w & 3) != 0) return CTG_ERR_INVALID_ARG;
    if ((k > 0 && !W_dev) || !q_dev || !w_out_dev || !h_out_dev || !scratch_dev) return CTG_ERR_INVALID_ARG;
    if ((k > 0 && !aligned16(W_dev)) || !aligned16(q_dev) || !aligned16(w_out_dev)) return CTG_ERR_INVALID_ARG;
    if (((uintptr_t)scratch_dev & 255u) != 0) return CTG_ERR_INVALID_ARG;
    if (scratch_bytes < ctg_cgs2_scratch_bytes(L, k)) return CTG_ERR_WORKSPACE;
    RedScratch rs;
    ctg_red_scratch_carve(scratch_dev, L, k + 1, &rs);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    CTG_CK(cudaMemsetAsync(rs.counter, 0, 4 * sizeof(unsigned), st));
    CTG_CK(ctg_cgs2_step(W_dev, CTG_BASIS_FP32, ld_w, L, k, q_dev, w_out_dev, h_out_dev, rs, st));
    return CTG_OK;
}

int ctg_set_timing(ctg_ctx *ctx, int enable) {
    if (!ctx) return CTG_ERR_INVALID_ARG;
    int rc = resolve_marks(ctx);
    ctx->timing = enable != 0;
    return rc;
}

int ctg_get_timing(ctg_ctx *ctx, ctg_timing *out, int reset) {
    if (!ctx || !out) return CTG_ERR_INVALID_ARG;
    int rc = resolve_marks(ctx);
    for (int p = 0; p < 4; ++p) {
        out->ms[p] = ctx->ms[p];
        out->calls[p] = ctx->calls[p];
    }
    out->kernels = ctx->kernels;
    if (reset) {
        for (int p = 0; p < 4; ++p) {
            ctx->ms[p] = 0.0;
            ctx->calls[p] = 0;
        }
        ctx->kernels = 0;
    }
    return rc;
}

const char *ctg_status_string(int status) {
    switch (status) {
        case CTG_OK: return "ok";
        case CTG_ERR_INVALID_ARG: return "invalid argument";
        case CTG_ERR_OOM: return "out of device memory";
        case CTG_ERR_CUDA: return "CUDA runtime error";
        case CTG_ERR_TIMEOUT: return "device-side wait timed out";
        case CTG_ERR_WORKSPACE: return "workspace too small";
        case CTG_ERR_BUSY: return "no free slot or memory budget; retry after a completion";
        default: return "unknown status";
    }
}

}  // extern "C"

long long ctg_ctx_wait_limit(const ctg_ctx *ctx) { return ctx ? ctx->spin_limit : kCtgDefaultSpinLimit; }

void ctg_ctx_forced_tiles(const ctg_ctx *ctx, int *fwd_split, int *back_chunk) {
    *fwd_split = ctx && ctx->force_fwd_angles ? ctx->force_fwd_split : 0;
    *back_chunk = ctx ? ctx->force_back_chunk : 0;
}
