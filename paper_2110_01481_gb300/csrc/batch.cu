// Batched AB-/BA-GMRES: many independent solves of different geometries,
// variants and iteration budgets advance together, one Arnoldi step per
// round.  A round is one launch per phase for all instances (projectors,
// CGS2 passes, Givens update, discrepancy residual, stopping rules), with all
// per-instance state on the device, so the round is captured once as a CUDA
// graph and replayed; the host only checks every few rounds whether any
// instance is still active.  The Hessenberg least-squares update runs on the
// device in FP64 (one warp per instance).
#include <cmath>
#include <cstring>
#include <new>
#include <memory>
#include <vector>

#include "ctg_internal.cuh"

namespace {

constexpr int kRoundsPerCheck = 4;

size_t al256(size_t v) { return (v + 255) & ~(size_t)255; }
size_t rup(size_t v, size_t m) { return (v + m - 1) / m * m; }
int padded4(int G) { return (G + 3) & ~3; }

// Forward projector plan of a geometry: whether warps of several angles
// are safe for it, and the dispatch orders (longest walk first) of its
// blocks in the batched shapes 0 and kBatchFwdSplitShape.
struct FwdPlan {
    bool split_ok = false;
    std::vector<int> order[2];
};

struct InstPlan {
    ctg_geom g;
    ctg_opts o;
    int variant;
    size_t off, bytes;         // this instance's slice of the batch workspace
    BatchInst d;               // device pointers filled in at create
    std::shared_ptr<const FwdPlan> fwd;   // forward projector plan (shared per geometry)
};

// Geometries with the same forward projector (its tables do not depend on
// the back projector model).
bool same_fwd_geom(const ctg_geom &a, const ctg_geom &b) {
    return a.N == b.N && a.n_angles == b.n_angles && a.n_det == b.n_det &&
           a.angle_start_deg == b.angle_start_deg && a.angle_range_deg == b.angle_range_deg &&
           a.det_spacing == b.det_spacing;
}

// Forward projector plan of a geometry, from its host angle table.
std::shared_ptr<const FwdPlan> plan_forward(const ctg_geom &g, const std::vector<FwdAngle> &fw) {
    auto f = std::make_shared<FwdPlan>();
    const PadLayout pl = ctg_pad_layout(g.N, g.det_spacing);
    f->split_ok = ctg_forward_split_safe(fw.data(), g.N, g.n_angles, g.n_det, pl, 4);
    ctg_forward_order(fw.data(), g.N, g.n_angles, g.n_det, 0, f->order[0]);
    ctg_forward_order(fw.data(), g.N, g.n_angles, g.n_det, kBatchFwdSplitShape, f->order[1]);
    return f;
}

int ck(cudaError_t e) {
    return e == cudaSuccess ? CTG_OK : (e == cudaErrorMemoryAllocation ? CTG_ERR_OOM : CTG_ERR_CUDA);
}
#define B_CK(call)                           \
    do {                                     \
        int rc_ = ck(call);                  \
        if (rc_ != CTG_OK) return rc_;       \
    } while (0)

// Lay out one instance; when base is non-null, fill the device pointers.
size_t plan_instance(InstPlan &p, char *base) {
    const ctg_geom &g = p.g;
    const int maxit = p.o.maxit;
    const long long n = (long long)g.N * g.N, m = (long long)g.n_angles * g.n_det;
    const bool ba = p.variant == CTG_BA;
    const long long L = ba ? n : m;
    const PadLayout pl = ctg_pad_layout(g.N, g.det_spacing);
    const size_t ldw = rup((size_t)L, 64);
    const bool dp = p.o.noise_norm > 0.0;
    const int Gn = ctg_vec_blocks(n), Gm = ctg_vec_blocks(m);
    const int Gp = padded4(Gn > Gm ? Gn : Gm);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = al256(off + bytes);
        return base ? base + o : nullptr;
    };
    BatchInst &d = p.d;
    std::memset(&d, 0, sizeof(d));
    d.N = g.N;
    d.n_angles = g.n_angles;
    d.n_det = g.n_det;
    d.variant = p.variant;
    d.pad_stride = pl.stride;
    d.pad_border = pl.border;
    d.pad_clamp = pl.clamp;
    d.n = n;
    d.m = m;
    d.L = L;
    d.maxit = maxit;
    d.ldw = (long long)ldw;
    d.G = ctg_vec_blocks(L);
    d.target = p.o.noise_norm > 0.0 ? p.o.tau * p.o.noise_norm : 0.0;
    d.wtype = p.o.basis_dtype;
    // the basis is the only O(maxit L) buffer: the storage law k L of Table 3
    d.W = take(ctg_basis_bytes(p.o.basis_dtype) * ldw * (size_t)(maxit + 1));
    d.H = (double *)take(sizeof(double) * (size_t)(maxit + 1) * maxit);
    d.R = (double *)take(sizeof(double) * (size_t)maxit * maxit);
    d.gc = (double *)take(sizeof(double) * maxit);
    d.gs = (double *)take(sizeof(double) * maxit);
    d.gg = (double *)take(sizeof(double) * (maxit + 1));
    d.y = (double *)take(sizeof(double) * maxit);
    d.hist = (double *)take(sizeof(double) * (maxit + 1));
    d.vn = (float *)take(sizeof(float) * rup((size_t)n, 64));
    d.vm = (float *)take(sizeof(float) * rup((size_t)m, 64));
    d.vr = ba && dp ? (float *)take(sizeof(float) * rup((size_t)m, 64)) : nullptr;
    d.pad = (float2 *)take(sizeof(float) * pl.floats);
    d.pad2 = ba && dp ? (float4 *)take(sizeof(float) * 2 * pl.floats) : nullptr;
    d.fwd = (const FwdAngle *)take(sizeof(FwdAngle) * g.n_angles);
    d.back = (const BackAngle *)take(sizeof(BackAngle) * g.n_angles);
    d.back_model = g.back_model;
    d.mt = g.back_model != CTG_BACK_PIXEL ? (const MatchedAngle *)take(sizeof(MatchedAngle) * g.n_angles)
                                          : nullptr;
    d.back_thr = 0.0f;
    // partial rows: maxit + 3 rows of the E = 1 passes, or 2 k + 2 rows of
    // the fused step (k <= its largest k) over its blocks
    const int kf = maxit < ctg_batch_fused_max_k() ? maxit : ctg_batch_fused_max_k();
    const size_t rows_pass = (size_t)(maxit + 3) * Gp;
    const size_t rows_fused = (size_t)(2 * kf + 2) * padded4(batch_fused_blocks(L));
    d.partials = (float *)take(sizeof(float) * (rows_pass > rows_fused ? rows_pass : rows_fused));
    d.h1 = (double *)take(sizeof(double) * (maxit + 3));
    d.h2 = (double *)take(sizeof(double) * (maxit + 3));
    d.scal = (double *)take(sizeof(double) * 8);
    d.counter = (unsigned *)take(sizeof(unsigned) * 4);
    return off;
}

// Batched solves take every back projector the tiled kernels apply: the
// pixel-driven B, and A^T / B_tau when two bins per pixel suffice (rm = 0).
bool back_model_batchable(const ctg_geom *g) {
    if (g->back_model == CTG_BACK_PIXEL) return true;
    std::vector<MatchedAngle> mt;
    int rm = 0;
    ctg_build_matched(g, mt, &rm);
    return rm == 0;
}

// Upload the instance's angle tables (its slice must be planned with a base)
// and, for B_tau, form the threshold tau max(A) (one device pass).
int upload_tables(InstPlan &p, cudaStream_t st) {
    std::vector<FwdAngle> fw;
    std::vector<BackAngle> bk;
    ctg_build_tables(&p.g, fw, bk);
    if (!p.fwd) p.fwd = plan_forward(p.g, fw);
    BatchInst &d = p.d;
    d.back_window = ctg_back_window(bk.data(), p.g.n_angles);
    B_CK(cudaMemcpyAsync((void *)d.fwd, fw.data(), sizeof(FwdAngle) * fw.size(), cudaMemcpyHostToDevice, st));
    B_CK(cudaMemcpyAsync((void *)d.back, bk.data(), sizeof(BackAngle) * bk.size(), cudaMemcpyHostToDevice, st));
    if (d.mt) {
        std::vector<MatchedAngle> mt;
        int rm = 0;
        ctg_build_matched(&p.g, mt, &rm);
        B_CK(cudaMemcpyAsync((void *)d.mt, mt.data(), sizeof(MatchedAngle) * mt.size(), cudaMemcpyHostToDevice, st));
        if (p.g.back_model == CTG_BACK_THRESHOLD) {
            unsigned bits = 0;
            B_CK(ctg_matched_max(p.g.N, p.g.n_angles, p.g.n_det, d.back, d.mt, rm, d.counter + 3, st));
            B_CK(cudaMemcpyAsync(&bits, d.counter + 3, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
            B_CK(cudaStreamSynchronize(st));
            float amax;
            std::memcpy(&amax, &bits, sizeof(float));
            d.back_thr = (float)(p.g.back_tau * (double)amax);
        }
    }
    B_CK(cudaStreamSynchronize(st));       // the host vectors go out of scope
    return CTG_OK;
}

// x = B b (+ add) with the instance's back projector
cudaError_t back_inst(const InstPlan &p, const float *b, const float *add, float *x, cudaStream_t st) {
    const BatchInst &d = p.d;
    if (d.back_model == CTG_BACK_PIXEL)
        return ctg_launch_back(b, CTG_BASIS_FP32, p.g.N, p.g.n_angles, p.g.n_det, d.back, d.back_window,
                               add, x, st);
    return ctg_launch_back_matched_tiled(b, CTG_BASIS_FP32, p.g.N, p.g.n_angles, p.g.n_det, d.back,
                                         d.back_window, d.mt, d.back_thr, add, x, st);
}

RedScratch scratch_of(const BatchInst &d) {
    RedScratch rs;
    rs.partials = d.partials;
    rs.h1 = d.h1;
    rs.h2 = d.h2;
    rs.scal = d.scal;
    rs.counter = d.counter;
    rs.grid = d.G;
    rs.E = 1;
    return rs;
}

}  // namespace

struct ctg_batch {
    ctg_ctx *ctx = nullptr;
    int n = 0;
    std::vector<InstPlan> inst;
    char *ws = nullptr;
    size_t ws_bytes = 0;
    BatchInst *d_insts = nullptr;
    int2 *d_maps = nullptr;
    int max_window = 0, max_maxit = 0;
    int *d_active = nullptr;
    int *h_active = nullptr;     // pinned
    double *h_stage = nullptr;   // pinned: per instance scal[0..7]
    cudaStream_t st = nullptr, st_body = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    cudaGraphExec_t round = nullptr;
    cudaGraphExec_t loop = nullptr;   // the whole iteration (while-loop graph), if it could be built
};

namespace {

void release(ctg_batch *b) {
    if (!b) return;
    if (b->st) cudaStreamSynchronize(b->st);
    if (b->round) cudaGraphExecDestroy(b->round);
    if (b->loop) cudaGraphExecDestroy(b->loop);
    if (b->st_body) cudaStreamDestroy(b->st_body);
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    if (b->ev_out) cudaEventDestroy(b->ev_out);
    if (b->st) cudaStreamDestroy(b->st);
    cudaFree(b->ws);
    cudaFree(b->d_insts);
    cudaFree(b->d_maps);
    cudaFree(b->d_active);
    if (b->h_active) cudaFreeHost(b->h_active);
    if (b->h_stage) cudaFreeHost(b->h_stage);
    delete b;
}

// The launches of a round, in order, each with its block map (offsets /
// lengths into one map array):
//   back: q = B w_k (AB) or B t_k (BA), FP32 launch and the AB BF16 / FP16
//     ones; AB: stage t, q = A t; CGS2 per basis type; Givens; BA with the
//     DP stop: x_k = x0 + W_k y_k; BA: stage w_{k+1} (and x_k), t_{k+1} =
//     A w_{k+1} (and A x_k); BA with the DP stop: ||b - A x_k||; the
//     stopping rules.
// MB_CGSF*: the blocks of the one-launch CGS2 step with the Givens update
// (batch_fused_blocks per instance), used instead of MB_CGS* and the
// separate Givens launch while every step is at most fused_kcap.
enum { MB_BACK, MB_B16, MB_H16, MB_PAD_AB, MB_FWD_AB, MB_CGS, MB_CGS_B16, MB_CGS_H16,
       MB_ITER, MB_PAD_BA, MB_FWD_BA, MB_RES, MB_CGSF, MB_CGSF_B16, MB_CGSF_H16, MB_COUNT };
struct RoundSpec {
    BatchInst *insts;
    int n_inst;
    const int2 *maps;
    int off[MB_COUNT], len[MB_COUNT];
    int max_window, max_maxit;
    int *d_active;
    int fwd_shape_ab, fwd_shape_ba;   // forward shapes of the two forward launches
    int back_chunk;                   // angles staged per pass by the back projections (0: 32)
    // the fused step: its largest k (0: the batch takes the separate
    // passes only), and in device memory the barrier counter, the timeout
    // word and the wait limit
    int fused_kcap;
    unsigned *bar;
    int *err;
    const long long *spin;
};

// Build the block maps of instances `ids` (indices into the instance array).
// split_ab / split_ba: the AB / BA forward launch may take the shape with
// several angles per warp (it does when every one of its instances allows it).
template <typename Plans>
void build_maps(const Plans &plans, const std::vector<int> &ids, std::vector<int2> &maps, RoundSpec &rs,
                bool split_ab = true, bool split_ba = true) {
    maps.clear();
    auto add = [&](int which, auto count) {
        rs.off[which] = (int)maps.size();
        for (int i : ids) {
            const int c = count(plans[i]);
            for (int j = 0; j < c; ++j) maps.push_back(make_int2(i, j));
        }
        rs.len[which] = (int)maps.size() - rs.off[which];
    };
    auto is_ab = [](const InstPlan &p) { return p.variant == CTG_AB; };
    auto ba_dp = [](const InstPlan &p) { return p.variant == CTG_BA && p.o.noise_norm > 0.0; };
    add(MB_BACK, [&](const InstPlan &p) {
        return (!is_ab(p) || p.o.basis_dtype == CTG_BASIS_FP32) ? ctg_back_tiles(p.g.N) : 0;
    });
    add(MB_B16, [&](const InstPlan &p) {
        return is_ab(p) && p.o.basis_dtype == CTG_BASIS_BF16 ? ctg_back_tiles(p.g.N) : 0;
    });
    add(MB_H16, [&](const InstPlan &p) {
        return is_ab(p) && p.o.basis_dtype == CTG_BASIS_FP16 ? ctg_back_tiles(p.g.N) : 0;
    });
    add(MB_PAD_AB, [&](const InstPlan &p) { return is_ab(p) ? ctg_pad_tiles(p.g.N) : 0; });
    // one forward shape per forward launch: several angles per warp when
    // every instance of the launch allows it
    auto shape_for = [&](bool ab) {
        bool split = false, any = false;
        for (int i : ids)
            if (is_ab(plans[i]) == ab) {
                split = (any ? split : true) && plans[i].fwd && plans[i].fwd->split_ok;
                any = true;
            }
        return any && split && (ab ? split_ab : split_ba) ? kBatchFwdSplitShape : 0;
    };
    rs.fwd_shape_ab = shape_for(true);
    rs.fwd_shape_ba = shape_for(false);
    auto add_fwd = [&](int which, bool ab) {
        const int fs = ab ? rs.fwd_shape_ab : rs.fwd_shape_ba;
        add(which, [&](const InstPlan &p) {
            return is_ab(p) == ab ? ctg_fwd_shape_blocks(fs, p.g.n_angles, p.g.n_det) : 0;
        });
        // each instance's forward blocks longest first (the result is the
        // same in any order; the launch's tail is shorter)
        for (int t = rs.off[which]; t < rs.off[which] + rs.len[which]; ++t) {
            const InstPlan &p = plans[maps[t].x];
            if (!p.fwd) continue;
            const std::vector<int> &o = p.fwd->order[fs == kBatchFwdSplitShape ? 1 : 0];
            if ((int)o.size() == ctg_fwd_shape_blocks(fs, p.g.n_angles, p.g.n_det)) maps[t].y = o[maps[t].y];
        }
    };
    add_fwd(MB_FWD_AB, true);
    auto cgs_blocks = [](const InstPlan &p, int wtype) {
        if (p.o.basis_dtype != wtype) return 0;
        return ctg_vec_blocks(p.variant == CTG_BA ? (long long)p.g.N * p.g.N
                                                  : (long long)p.g.n_angles * p.g.n_det);
    };
    add(MB_CGS, [&](const InstPlan &p) { return cgs_blocks(p, CTG_BASIS_FP32); });
    add(MB_CGS_B16, [&](const InstPlan &p) { return cgs_blocks(p, CTG_BASIS_BF16); });
    add(MB_CGS_H16, [&](const InstPlan &p) { return cgs_blocks(p, CTG_BASIS_FP16); });
    add(MB_ITER, [&](const InstPlan &p) { return ba_dp(p) ? ctg_vec_blocks((long long)p.g.N * p.g.N) : 0; });
    add(MB_PAD_BA, [&](const InstPlan &p) { return is_ab(p) ? 0 : ctg_pad_tiles(p.g.N); });
    add_fwd(MB_FWD_BA, false);
    add(MB_RES, [&](const InstPlan &p) {
        return ba_dp(p) ? ctg_vec_blocks((long long)p.g.n_angles * p.g.n_det) : 0;
    });
    auto fused_blocks = [](const InstPlan &p, int wtype) {
        if (p.o.basis_dtype != wtype) return 0;
        return batch_fused_blocks(p.variant == CTG_BA ? (long long)p.g.N * p.g.N
                                                      : (long long)p.g.n_angles * p.g.n_det);
    };
    add(MB_CGSF, [&](const InstPlan &p) { return fused_blocks(p, CTG_BASIS_FP32); });
    add(MB_CGSF_B16, [&](const InstPlan &p) { return fused_blocks(p, CTG_BASIS_BF16); });
    add(MB_CGSF_H16, [&](const InstPlan &p) { return fused_blocks(p, CTG_BASIS_FP16); });
}

// The largest k of the fused step for a batch whose maps are in rs (0 when
// a fused launch's blocks would not all be resident at once: the batch
// then takes the separate passes throughout).
int fused_kcap_of(const RoundSpec &rs, int max_maxit) {
    const int kcap = max_maxit < ctg_batch_fused_max_k() ? max_maxit : ctg_batch_fused_max_k();
    const int which[3] = {MB_CGSF, MB_CGSF_B16, MB_CGSF_H16};
    const int types[3] = {CTG_BASIS_FP32, CTG_BASIS_BF16, CTG_BASIS_FP16};
    for (int t = 0; t < 3; ++t)
        if (rs.len[which[t]] > 0 && rs.len[which[t]] > ctg_batch_fused_resident(kcap, types[t])) return 0;
    return kcap;
}

// Which launches a round makes (a launcher skips a phase with no blocks):
// two rounds with the same signature capture the same kernels in the same
// order.
unsigned round_signature(const RoundSpec &r) {
    unsigned sig = 0;
    for (int i = 0; i < MB_COUNT; ++i) sig |= (r.len[i] > 0 ? 1u : 0u) << i;
    return sig | (unsigned)r.fwd_shape_ab << 16 | (unsigned)r.fwd_shape_ba << 20;
}

// Enqueue one round's launches on st (ending it with the stopping rules;
// inside a while-loop body, loop_ctl and the loop's handle end the loop
// when no solve is left).
// fused: the round's CGS2 step and Givens update by the one-launch kernel
// (steps <= r.fused_kcap); h_next: the while loop that follows this one.
cudaError_t enqueue_round(const RoundSpec &r, cudaStream_t st, int *loop_ctl = nullptr,
                          cudaGraphConditionalHandle h = 0, bool fused = false,
                          cudaGraphConditionalHandle h_next = 0) {
    cudaError_t e = cudaSuccess;
    const int2 *M = r.maps;
    auto map = [&](int w) { return M + r.off[w]; };
    if (e == cudaSuccess)
        e = ctg_batch_back(r.insts, map(MB_BACK), r.len[MB_BACK], r.max_window, st, CTG_BASIS_FP32, r.back_chunk);
    if (e == cudaSuccess)
        e = ctg_batch_back(r.insts, map(MB_B16), r.len[MB_B16], r.max_window, st, CTG_BASIS_BF16, r.back_chunk);
    if (e == cudaSuccess)
        e = ctg_batch_back(r.insts, map(MB_H16), r.len[MB_H16], r.max_window, st, CTG_BASIS_FP16, r.back_chunk);
    if (e == cudaSuccess) e = ctg_batch_pad(r.insts, map(MB_PAD_AB), r.len[MB_PAD_AB], CTG_AB, st);
    if (e == cudaSuccess)
        e = ctg_batch_forward(r.insts, map(MB_FWD_AB), r.len[MB_FWD_AB], CTG_AB, st, r.fwd_shape_ab);
    if (fused) {
        const int which[3] = {MB_CGSF, MB_CGSF_B16, MB_CGSF_H16};
        const int types[3] = {CTG_BASIS_FP32, CTG_BASIS_BF16, CTG_BASIS_FP16};
        for (int t = 0; t < 3 && e == cudaSuccess; ++t)
            e = ctg_batch_cgs2_fused(r.insts, map(which[t]), r.len[which[t]], r.fused_kcap, r.bar, r.err, r.spin,
                                     st, types[t]);
    } else {
        if (e == cudaSuccess) e = ctg_batch_cgs2(r.insts, map(MB_CGS), r.len[MB_CGS], r.max_maxit, st);
        if (e == cudaSuccess)
            e = ctg_batch_cgs2(r.insts, map(MB_CGS_B16), r.len[MB_CGS_B16], r.max_maxit, st, CTG_BASIS_BF16);
        if (e == cudaSuccess)
            e = ctg_batch_cgs2(r.insts, map(MB_CGS_H16), r.len[MB_CGS_H16], r.max_maxit, st, CTG_BASIS_FP16);
        if (e == cudaSuccess) e = ctg_batch_givens(r.insts, r.n_inst, r.max_maxit, st);
    }
    if (e == cudaSuccess) e = ctg_batch_iterate(r.insts, map(MB_ITER), r.len[MB_ITER], r.max_maxit, st);
    if (e == cudaSuccess) e = ctg_batch_pad(r.insts, map(MB_PAD_BA), r.len[MB_PAD_BA], CTG_BA, st);
    if (e == cudaSuccess)
        e = ctg_batch_forward(r.insts, map(MB_FWD_BA), r.len[MB_FWD_BA], CTG_BA, st, r.fwd_shape_ba);
    if (e == cudaSuccess) e = ctg_batch_residual(r.insts, map(MB_RES), r.len[MB_RES], st);
    if (e == cudaSuccess) {
        if (loop_ctl)
            e = ctg_batch_finish_loop(r.insts, r.n_inst, loop_ctl, r.max_maxit, h, st, h_next,
                                      fused ? r.fused_kcap : 0);
        else e = ctg_batch_finish(r.insts, r.n_inst, r.d_active, st);
    }
    return e;
}

// Capture one round into *out.  If *out already holds an executable graph
// captured with the same kernel sequence (sig_prev == this round's
// signature), it is updated in place, which is much cheaper than
// instantiating a new one; otherwise it is replaced.
int capture_round(const RoundSpec &r, cudaStream_t st, cudaGraphExec_t *out, unsigned sig_prev = ~0u) {
    cudaGraph_t graph = nullptr;
    B_CK(ctg_batch_prepare(r.max_maxit));   // kernel attributes, set outside the capture
    B_CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = enqueue_round(r, st);
    cudaError_t e2 = cudaStreamEndCapture(st, &graph);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess && *out != nullptr) {
        cudaGraphExecUpdateResultInfo info;
        if (sig_prev != round_signature(r) || cudaGraphExecUpdate(*out, graph, &info) != cudaSuccess) {
            cudaGetLastError();                      // another kernel sequence: instantiate anew
            cudaGraphExecDestroy(*out);
            *out = nullptr;
        }
    }
    if (e == cudaSuccess && *out == nullptr) e = cudaGraphInstantiate(out, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    return ck(e);
}

// Capture the whole iteration of a batch as one graph: a while-loop node
// whose body is a round, ended on the device by the round's stopping-rule
// kernel (loop_ctl: active solves, rounds run), so no host check runs
// between rounds.  With the fused step (r.fused_kcap > 0) two while loops
// follow each other: rounds with the one-launch CGS2 step until a solve's
// next step is beyond fused_kcap, then rounds with the separate passes (the
// first loop ends both once no solve is left).  st captures, bs the bodies.
int capture_loop(const RoundSpec &r, cudaStream_t st, cudaStream_t bs, int *loop_ctl, cudaGraphExec_t *out) {
    if (r.n_inst > 1024) return CTG_ERR_INVALID_ARG;
    B_CK(ctg_batch_prepare(r.max_maxit));
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed);
    cudaStreamCaptureStatus cs;
    cudaGraph_t cg = nullptr;
    const int nloops = r.fused_kcap > 0 ? 2 : 1;
    cudaGraphConditionalHandle h[2] = {0, 0};
    if (e == cudaSuccess) e = cudaStreamGetCaptureInfo(st, &cs, nullptr, &cg, nullptr, nullptr, nullptr);
    for (int l = 0; l < nloops && e == cudaSuccess; ++l)
        e = cudaGraphConditionalHandleCreate(&h[l], cg, 1u, cudaGraphCondAssignDefault);
    for (int l = 0; l < nloops && e == cudaSuccess; ++l) {
        const cudaGraphNode_t *deps = nullptr;
        size_t ndeps = 0;
        e = cudaStreamGetCaptureInfo(st, &cs, nullptr, nullptr, &deps, nullptr, &ndeps);
        cudaGraphNodeParams cp = {};
        cudaGraphNode_t node;
        if (e == cudaSuccess) {
            cp.type = cudaGraphNodeTypeConditional;
            cp.conditional.handle = h[l];
            cp.conditional.type = cudaGraphCondTypeWhile;
            cp.conditional.size = 1;
            e = cudaGraphAddNode(&node, cg, deps, nullptr, ndeps, &cp);
        }
        if (e == cudaSuccess)
            e = cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
        if (e == cudaSuccess) {
            e = cudaStreamBeginCaptureToGraph(bs, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                              cudaStreamCaptureModeRelaxed);
            if (e == cudaSuccess) {
                const bool fused = nloops == 2 && l == 0;
                e = enqueue_round(r, bs, loop_ctl, h[l], fused, fused ? h[1] : 0);
                cudaGraph_t body = nullptr;
                const cudaError_t e2 = cudaStreamEndCapture(bs, &body);
                if (e == cudaSuccess) e = e2;
            }
        }
    }
    const cudaError_t e3 = cudaStreamEndCapture(st, &graph);
    if (e == cudaSuccess) e = e3;
    if (e == cudaSuccess) e = cudaGraphInstantiate(out, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *out = nullptr;
    }
    return ck(e);
}

// The batched autotuner: times the launches whose shape the result does
// not depend on (each ray and each pixel is summed in the same order in
// every shape): the forward projections with four angles per warp against
// one, and the back projection with 16, 32 and 64 angles staged per pass.
// Each candidate runs once untimed and 3 times timed with CUDA events, on
// the instances' zero buffers at k = 1 (their state is set up again at every
// solve).  Writes the faster choices.
int tune_batch(ctg_batch *b, const std::vector<int> &ids, bool tune_fwd, bool tune_back, bool *split_ab,
               bool *split_ba, int *chunk) {
    const int n = b->n;
    std::vector<BatchInst> hi(n);
    for (int i = 0; i < n; ++i) {
        hi[i] = b->inst[i].d;
        hi[i].active = 1;
        hi[i].k = 1;
    }
    B_CK(cudaMemcpy(b->d_insts, hi.data(), sizeof(BatchInst) * n, cudaMemcpyHostToDevice));
    std::vector<int2> ms, mp;
    RoundSpec rs{}, rp{};
    build_maps(b->inst, ids, ms, rs, true, true);
    build_maps(b->inst, ids, mp, rp, false, false);
    int2 *d = nullptr;
    B_CK(cudaMalloc(&d, sizeof(int2) * (ms.size() + mp.size() + 1)));
    int rc = ck(cudaMemcpy(d, ms.data(), sizeof(int2) * ms.size(), cudaMemcpyHostToDevice));
    if (rc == CTG_OK)
        rc = ck(cudaMemcpy(d + ms.size(), mp.data(), sizeof(int2) * mp.size(), cudaMemcpyHostToDevice));
    const int2 *ds = d, *dp = d + ms.size();
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (rc == CTG_OK) rc = ck(cudaEventCreate(&e0));
    if (rc == CTG_OK) rc = ck(cudaEventCreate(&e1));
    auto timed = [&](auto launch) -> float {
        if (rc != CTG_OK) return 0.0f;
        rc = ck(launch());
        if (rc == CTG_OK) rc = ck(cudaEventRecord(e0, b->st));
        for (int t = 0; t < 3 && rc == CTG_OK; ++t) rc = ck(launch());
        if (rc == CTG_OK) rc = ck(cudaEventRecord(e1, b->st));
        if (rc == CTG_OK) rc = ck(cudaEventSynchronize(e1));
        float ms_ = 0.0f;
        if (rc == CTG_OK) rc = ck(cudaEventElapsedTime(&ms_, e0, e1));
        return ms_;
    };
    if (tune_fwd) {
        const int which[2] = {MB_FWD_AB, MB_FWD_BA}, variants[2] = {CTG_AB, CTG_BA};
        const int shapes[2] = {rs.fwd_shape_ab, rs.fwd_shape_ba};
        bool *out[2] = {split_ab, split_ba};
        for (int v = 0; v < 2; ++v) {
            if (shapes[v] != kBatchFwdSplitShape || rs.len[which[v]] <= 0) continue;
            const float t_split = timed([&] {
                return ctg_batch_forward(b->d_insts, ds + rs.off[which[v]], rs.len[which[v]], variants[v], b->st,
                                         kBatchFwdSplitShape);
            });
            const float t_one = timed([&] {
                return ctg_batch_forward(b->d_insts, dp + rp.off[which[v]], rp.len[which[v]], variants[v], b->st, 0);
            });
            *out[v] = t_split <= t_one;
        }
    }
    if (tune_back && rp.len[MB_BACK] > 0) {
        float best = 0.0f;
        for (const int c : {32, 16, 64}) {
            if (!ctg_batch_back_chunk_ok(c, b->max_window)) continue;
            const float t = timed([&] {
                return ctg_batch_back(b->d_insts, dp + rp.off[MB_BACK], rp.len[MB_BACK], b->max_window, b->st,
                                      CTG_BASIS_FP32, c);
            });
            if (rc == CTG_OK && (c == 32 || t < best)) {
                best = t;
                *chunk = c;
            }
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(d);
    return rc;
}

}  // namespace

extern "C" int ctg_batch_create(ctg_ctx *ctx, int32_t n, const ctg_geom *geoms,
                                const int32_t *variants, const ctg_opts *opts, ctg_batch **out) {
    if (!ctx || n < 1 || !geoms || !variants || !opts || !out) return CTG_ERR_INVALID_ARG;
    *out = nullptr;
    ctg_batch *b = new (std::nothrow) ctg_batch();
    if (!b) return CTG_ERR_OOM;
    b->ctx = ctx;
    b->n = n;
    b->inst.resize(n);
    size_t total = 0;
    std::vector<std::vector<FwdAngle>> fw(n);
    std::vector<std::vector<BackAngle>> bk(n);
    for (int i = 0; i < n; ++i) {
        InstPlan &p = b->inst[i];
        p.g = geoms[i];
        p.o = opts[i];
        p.variant = variants[i];
        if (!ctg_geom_valid(&p.g) || !back_model_batchable(&p.g) || !ctg_opts_valid(&p.o) ||
            p.o.stop_rule != CTG_RULE_DP ||
            p.o.maxit > 1024 || (p.variant != CTG_AB && p.variant != CTG_BA)) {
            release(b);
            return CTG_ERR_INVALID_ARG;
        }
        ctg_build_tables(&p.g, fw[i], bk[i]);
        p.fwd = plan_forward(p.g, fw[i]);
        const int win = ctg_back_window(bk[i].data(), p.g.n_angles);
        if (win > ctg_back_window_max()) {   // detector pitch too fine for the batched tiles
            release(b);
            return CTG_ERR_INVALID_ARG;
        }
        if (win > b->max_window) b->max_window = win;
        if (p.o.maxit > b->max_maxit) b->max_maxit = p.o.maxit;
        p.off = total;
        p.bytes = plan_instance(p, nullptr);
        total = al256(total + p.bytes);
    }
    b->ws_bytes = total;
    // everything below is ordered on the batch's own (non-blocking) stream:
    // a legacy-stream memset of the workspace would not be ordered before
    // the table uploads on it
    int rc = ck(cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking));
    if (rc == CTG_OK) rc = ck(cudaStreamCreateWithFlags(&b->st_body, cudaStreamNonBlocking));
    if (rc == CTG_OK) rc = ck(cudaMalloc(&b->ws, total));
    if (rc == CTG_OK) rc = ck(cudaMemsetAsync(b->ws, 0, total, b->st));
    std::vector<int> ids(n);
    for (int i = 0; i < n; ++i) ids[i] = i;
    if (rc == CTG_OK) rc = ck(cudaMalloc(&b->d_insts, sizeof(BatchInst) * n));
    // active solves, rounds run, the fused step's barrier counter and
    // timeout word, then (8-byte aligned) the wait limit
    if (rc == CTG_OK) rc = ck(cudaMalloc(&b->d_active, 8 * sizeof(int)));
    if (rc == CTG_OK) rc = ck(cudaMemsetAsync(b->d_active, 0, 8 * sizeof(int), b->st));
    if (rc == CTG_OK) rc = ck(cudaMallocHost(&b->h_active, sizeof(int)));
    if (rc == CTG_OK) rc = ck(cudaMallocHost(&b->h_stage, sizeof(double) * 8 * n));
    if (rc == CTG_OK) rc = ck(cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming));
    if (rc == CTG_OK) rc = ck(cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming));
    for (int i = 0; rc == CTG_OK && i < n; ++i) {
        InstPlan &p = b->inst[i];
        plan_instance(p, b->ws + p.off);
        rc = upload_tables(p, b->st);
    }
    if (rc == CTG_OK) rc = ck(cudaStreamSynchronize(b->st));
    // tile shapes: forced on the context, else the batched autotuner's
    int f_split = 0, f_chunk = 0;
    ctg_ctx_forced_tiles(ctx, &f_split, &f_chunk);
    bool split_ab = f_split != 1, split_ba = f_split != 1;
    int chunk = f_chunk && ctg_batch_back_chunk_ok(f_chunk, b->max_window) ? f_chunk : 32;
    if (rc == CTG_OK && (!f_split || !f_chunk))
        rc = tune_batch(b, ids, !f_split, !f_chunk, &split_ab, &split_ba, &chunk);
    // block maps
    std::vector<int2> maps;
    RoundSpec spec{};
    build_maps(b->inst, ids, maps, spec, split_ab, split_ba);
    spec.back_chunk = chunk;
    if (rc == CTG_OK) rc = ck(cudaMalloc(&b->d_maps, sizeof(int2) * (maps.empty() ? 1 : maps.size())));
    if (rc == CTG_OK && !maps.empty())
        rc = ck(cudaMemcpy(b->d_maps, maps.data(), sizeof(int2) * maps.size(), cudaMemcpyHostToDevice));
    if (rc == CTG_OK) {
        RoundSpec r = spec;
        r.insts = b->d_insts;
        r.n_inst = n;
        r.maps = b->d_maps;
        r.max_window = b->max_window;
        r.max_maxit = b->max_maxit;
        r.d_active = b->d_active;
        r.bar = reinterpret_cast<unsigned *>(b->d_active + 2);
        r.err = b->d_active + 3;
        r.spin = reinterpret_cast<const long long *>(b->d_active + 4);
        rc = capture_round(r, b->st, &b->round);   // the host-driven round: separate passes
        r.fused_kcap = rc == CTG_OK ? fused_kcap_of(r, b->max_maxit) : 0;
        // the whole iteration as one graph; without it the host replays the
        // round graph and checks the active count every few rounds
        if (rc == CTG_OK && capture_loop(r, b->st, b->st_body, b->d_active, &b->loop) != CTG_OK) b->loop = nullptr;
    }
    if (rc != CTG_OK) {
        release(b);
        return rc;
    }
    *out = b;
    return CTG_OK;
}

extern "C" void ctg_batch_destroy(ctg_batch *b) { release(b); }

extern "C" size_t ctg_batch_workspace_bytes(const ctg_batch *b) { return b ? b->ws_bytes : 0; }

namespace {

// Enqueue the start of one solve: r0 (AB: b - A x0 in vm; BA: B (b - A x0)
// in vn), ||r0||^2 in scal[2] and (BA) ||b - A x0||^2 in scal[4]; copies
// scal[0..7] to `stage` (pinned).
int enqueue_start(InstPlan &p, const float *b, const float *x0, double *stage, cudaStream_t st) {
    BatchInst &d = p.d;
    const RedScratch rs = scratch_of(d);
    const PadLayout pl = ctg_pad_layout(p.g.N, p.g.det_spacing);
    B_CK(cudaMemsetAsync(d.counter, 0, 4 * sizeof(unsigned), st));
    B_CK(cudaMemsetAsync(d.gg, 0, sizeof(double) * (p.o.maxit + 1), st));
    B_CK(cudaMemsetAsync(d.H, 0, sizeof(double) * (size_t)(p.o.maxit + 1) * p.o.maxit, st));
    B_CK(cudaMemsetAsync(d.hist, 0, sizeof(double) * (p.o.maxit + 1), st));
    B_CK(cudaMemsetAsync(d.pad, 0, sizeof(float) * pl.floats, st));
    if (d.pad2) B_CK(cudaMemsetAsync(d.pad2, 0, sizeof(float) * 2 * pl.floats, st));
    if (x0) {
        B_CK(ctg_launch_pad(x0, CTG_BASIS_FP32, d.pad, p.g.N, pl, st));
        B_CK(ctg_launch_forward(d.pad, p.g.N, pl, p.g.n_angles, p.g.n_det, d.fwd, d.vm, st));
    }
    if (p.variant == CTG_AB) {
        B_CK(ctg_sub_norm2(b, x0 ? d.vm : nullptr, d.vm, d.m, d.scal + 2, rs, st));
    } else {
        B_CK(ctg_sub_norm2(b, x0 ? d.vm : nullptr, d.vm, d.m, d.scal + 4, rs, st));
        B_CK(back_inst(p, d.vm, nullptr, d.vn, st));
        B_CK(ctg_sub_norm2(d.vn, nullptr, nullptr, d.n, d.scal + 2, rs, st));
    }
    B_CK(cudaMemcpyAsync(stage, d.scal, sizeof(double) * 8, cudaMemcpyDeviceToHost, st));
    return CTG_OK;
}

// After enqueue_start has completed (stage holds scal): either a k = 0 stop
// (returns 0, the solve is finished with x = x0) or w_1 = r0 / beta and the
// rotated right-hand side beta e1 are enqueued (returns 1, the solve is
// active).  stage[6] is used as the upload slot for beta.
int activate(InstPlan &p, double *stage, ctg_info *info, cudaStream_t st, int *active_out) {
    BatchInst &d = p.d;
    const double beta = std::sqrt(stage[2]);
    const double res0 = p.variant == CTG_AB ? beta : std::sqrt(stage[4]);
    d.k = 1;
    d.iters = 0;
    d.breakdown = 0;
    d.rho = beta;
    d.resnorm = res0;
    d.stop_reason = CTG_STOP_MAXIT;
    info->iters = 0;
    info->stop_reason = CTG_STOP_MAXIT;
    info->rho = beta;
    info->resnorm = res0;
    if (info->history) info->history[0] = d.target > 0.0 ? res0 : beta;
    const bool dp0 = d.target > 0.0 && res0 <= d.target;
    if (dp0 || beta == 0.0) {
        d.active = 0;
        d.stop_reason = dp0 ? CTG_STOP_DP : CTG_STOP_BREAKDOWN;
        info->stop_reason = d.stop_reason;
        *active_out = 0;
        return CTG_OK;
    }
    d.active = 1;
    B_CK(ctg_scale(p.variant == CTG_AB ? d.vm : d.vn, d.scal + 2, d.W, d.wtype, d.L, st));
    if (p.variant == CTG_BA) {
        // t_1 = A w_1, which the first round back-projects
        const PadLayout pl = ctg_pad_layout(p.g.N, p.g.det_spacing);
        B_CK(ctg_launch_pad(d.W, d.wtype, d.pad, p.g.N, pl, st));
        B_CK(ctg_launch_forward(d.pad, p.g.N, pl, p.g.n_angles, p.g.n_det, d.fwd, d.vm, st));
    }
    stage[6] = beta;
    B_CK(cudaMemcpyAsync(d.gg, &stage[6], sizeof(double), cudaMemcpyHostToDevice, st));
    *active_out = 1;
    return CTG_OK;
}

// Enqueue the end of a finished solve (d: its device state after the
// rounds, with y = R^{-1} g already solved): x = x0 + B W y (AB) or
// x0 + W y (BA), ||b - A x||^2 into stage[5], the history into the caller's
// array.  The caller reads stage[5] after synchronising.
int enqueue_finish(const InstPlan &p, const BatchInst &d, const float *b, const float *x0, float *x,
                   ctg_info *info, double *stage, cudaStream_t st) {
    const RedScratch rs = scratch_of(d);
    const PadLayout pl = ctg_pad_layout(p.g.N, p.g.det_spacing);
    const int k = d.iters;
    info->iters = k;
    info->stop_reason = d.stop_reason;
    if (k == 0) {
        if (x0) B_CK(cudaMemcpyAsync(x, x0, sizeof(float) * d.n, cudaMemcpyDeviceToDevice, st));
        else B_CK(cudaMemsetAsync(x, 0, sizeof(float) * d.n, st));
        return CTG_OK;
    }
    info->rho = d.rho;
    if (p.variant == CTG_AB) {
        B_CK(ctg_gemv(d.W, d.wtype, d.ldw, d.m, k, d.y, nullptr, d.vm, st));
        B_CK(back_inst(p, d.vm, x0, x, st));
    } else {
        B_CK(ctg_gemv(d.W, d.wtype, d.ldw, d.n, k, d.y, x0, x, st));
    }
    B_CK(ctg_launch_pad(x, CTG_BASIS_FP32, d.pad, p.g.N, pl, st));
    B_CK(ctg_launch_forward(d.pad, p.g.N, pl, p.g.n_angles, p.g.n_det, d.fwd, d.vm, st));
    B_CK(ctg_sub_norm2(b, d.vm, nullptr, d.m, d.scal + 5, rs, st));
    B_CK(cudaMemcpyAsync(stage + 5, d.scal + 5, sizeof(double), cudaMemcpyDeviceToHost, st));
    if (info->history)
        B_CK(cudaMemcpyAsync(info->history + 1, d.hist + 1, sizeof(double) * k, cudaMemcpyDeviceToHost, st));
    return CTG_OK;
}

}  // namespace

extern "C" int ctg_batch_solve(ctg_batch *b, const float *const *b_dev, const float *const *x0_dev,
                               float *const *x_dev, ctg_info *infos, void *stream) {
    if (!b || !b_dev || !x_dev || !infos) return CTG_ERR_INVALID_ARG;
    const int n = b->n;
    for (int i = 0; i < n; ++i)
        if (!b_dev[i] || !x_dev[i]) return CTG_ERR_INVALID_ARG;
    cudaStream_t user = static_cast<cudaStream_t>(stream);
    cudaStream_t st = b->st;
    B_CK(cudaEventRecord(b->ev_in, user));
    B_CK(cudaStreamWaitEvent(st, b->ev_in, 0));
    for (int i = 0; i < n; ++i) {
        const int rc = enqueue_start(b->inst[i], b_dev[i], x0_dev ? x0_dev[i] : nullptr,
                                     b->h_stage + 8 * i, st);
        if (rc) return rc;
    }
    B_CK(cudaStreamSynchronize(st));
    int active = 0;
    for (int i = 0; i < n; ++i) {
        int a = 0;
        const int rc = activate(b->inst[i], b->h_stage + 8 * i, &infos[i], st, &a);
        if (rc) return rc;
        active += a;
    }
    std::vector<BatchInst> hi(n);
    for (int i = 0; i < n; ++i) {
        BatchInst &d = b->inst[i].d;
        d.b = b_dev[i];
        d.x0 = x0_dev ? x0_dev[i] : nullptr;
        d.x = x_dev[i];
        hi[i] = d;
    }
    B_CK(cudaMemcpyAsync(b->d_insts, hi.data(), sizeof(BatchInst) * n, cudaMemcpyHostToDevice, st));
    *b->h_active = active;
    B_CK(cudaMemcpyAsync(b->d_active, b->h_active, sizeof(int), cudaMemcpyHostToDevice, st));
    B_CK(cudaMemsetAsync(b->d_active + 1, 0, 3 * sizeof(int), st));   // rounds, barrier, timeout
    const long long wait_limit = ctg_ctx_wait_limit(b->ctx);
    B_CK(cudaMemcpyAsync(b->d_active + 4, &wait_limit, sizeof(long long), cudaMemcpyHostToDevice, st));
    // ---- rounds -----------------------------------------------------------
    if (active > 0 && b->loop) {
        B_CK(cudaGraphLaunch(b->loop, st));
        active = 0;
    }
    int rounds = 0;
    while (active > 0 && rounds < b->max_maxit) {
        const int r = std::min(kRoundsPerCheck, b->max_maxit - rounds);
        for (int j = 0; j < r; ++j) B_CK(cudaGraphLaunch(b->round, st));
        rounds += r;
        B_CK(cudaMemcpyAsync(b->h_active, b->d_active, sizeof(int), cudaMemcpyDeviceToHost, st));
        B_CK(cudaStreamSynchronize(st));
        active = *b->h_active;
    }
    // ---- exit: y_k, x_k and its residual -----------------------------------
    B_CK(ctg_batch_solve_y(b->d_insts, n, b->max_maxit, st));
    B_CK(cudaMemcpyAsync(hi.data(), b->d_insts, sizeof(BatchInst) * n, cudaMemcpyDeviceToHost, st));
    B_CK(cudaMemcpyAsync(b->h_active, b->d_active + 3, sizeof(int), cudaMemcpyDeviceToHost, st));
    B_CK(cudaStreamSynchronize(st));
    // a fused step gave up at a grid barrier: every solve stopped at its last
    // completed step, whose iterate is still formed below
    const bool timed_out = *b->h_active != 0;
    for (int i = 0; i < n; ++i) {
        const int rc = enqueue_finish(b->inst[i], hi[i], b_dev[i], x0_dev ? x0_dev[i] : nullptr,
                                      x_dev[i], &infos[i], b->h_stage + 8 * i, st);
        if (rc) return rc;
    }
    B_CK(cudaStreamSynchronize(st));
    for (int i = 0; i < n; ++i)
        if (infos[i].iters > 0) infos[i].resnorm = std::sqrt(b->h_stage[8 * i + 5]);
    B_CK(cudaEventRecord(b->ev_out, st));
    B_CK(cudaStreamWaitEvent(user, b->ev_out, 0));
    return timed_out ? CTG_ERR_TIMEOUT : CTG_OK;
}

// ---------------------------------------------------------------------------
// Serving engine: continuous batching.  Solves are admitted one at a time
// into free slots while others are running (admission by the device memory
// their Krylov basis needs against a budget), each keeps its basis,
// Hessenberg matrix and iterate resident in its own workspace, and every
// step advances all running solves by a few rounds of the same batched
// kernels.  The round graph is re-captured only when new solves have joined
// since the last step; finished solves are formed, reported and their
// memory released at the end of the step that finished them.
struct ctg_engine {
    struct Slot {
        int state = 0;          // 0 free, 1 running, 2 finished, not yet reported
        InstPlan plan;
        char *ws = nullptr;
        size_t bytes = 0;
        const float *b = nullptr;
        const float *x0 = nullptr;
        float *x = nullptr;
        ctg_info info{};
        long long tag = 0;
    };
    ctg_ctx *ctx = nullptr;
    int max_slots = 0;
    size_t budget = 0, in_use = 0;
    std::vector<Slot> slots;
    BatchInst *d_insts = nullptr;
    std::vector<BatchInst> h_insts;
    BatchInst *h_pinned = nullptr;   // pinned mirror used for transfers
    int2 *d_maps = nullptr;
    size_t maps_cap = 0;
    bool dirty = true;
    unsigned round_sig = ~0u;        // kernel sequence of the captured round
    int running = 0;
    int *d_active = nullptr, *h_active = nullptr;
    double *h_stage = nullptr;       // 8 per slot
    cudaStream_t st = nullptr;
    cudaEvent_t ev_in = nullptr;
    cudaGraphExec_t round = nullptr;
    cudaMemPool_t pool = nullptr;    // per-solve workspaces, kept mapped up to the budget
    // forward plans of the geometries served so far (a few ms of host work
    // each, so made once per geometry)
    std::vector<std::pair<ctg_geom, std::shared_ptr<const FwdPlan>>> fwd_plans;
};

namespace {

void release_engine(ctg_engine *e) {
    if (!e) return;
    if (e->st) cudaStreamSynchronize(e->st);
    for (auto &s : e->slots)
        if (s.ws) cudaFreeAsync(s.ws, e->st);
    if (e->st) cudaStreamSynchronize(e->st);
    if (e->pool) cudaMemPoolDestroy(e->pool);
    if (e->round) cudaGraphExecDestroy(e->round);
    if (e->ev_in) cudaEventDestroy(e->ev_in);
    if (e->st) cudaStreamDestroy(e->st);
    cudaFree(e->d_insts);
    cudaFree(e->d_maps);
    cudaFree(e->d_active);
    if (e->h_active) cudaFreeHost(e->h_active);
    if (e->h_stage) cudaFreeHost(e->h_stage);
    if (e->h_pinned) cudaFreeHost(e->h_pinned);
    delete e;
}

bool plan_valid(const ctg_geom *g, int variant, const ctg_opts *o) {
    if (!ctg_geom_valid(g) || !back_model_batchable(g) || !ctg_opts_valid(o) ||
        o->stop_rule != CTG_RULE_DP ||
        o->maxit > 1024 || (variant != CTG_AB && variant != CTG_BA))
        return false;
    std::vector<FwdAngle> fw;
    std::vector<BackAngle> bk;
    ctg_build_tables(g, fw, bk);
    return ctg_back_window(bk.data(), g->n_angles) <= ctg_back_window_max();
}

// The slots' plans indexed by slot, as build_maps reads them (no copies).
struct SlotPlans {
    const ctg_engine *e;
    const InstPlan &operator[](size_t i) const { return e->slots[i].plan; }
};

int recapture(ctg_engine *e) {
    std::vector<int> ids;
    for (int i = 0; i < e->max_slots; ++i)
        if (e->slots[i].state == 1) ids.push_back(i);
    SlotPlans plans{e};
    std::vector<int2> maps;
    RoundSpec r{};
    build_maps(plans, ids, maps, r);
    if (maps.size() > e->maps_cap) {
        cudaFree(e->d_maps);
        e->d_maps = nullptr;
        e->maps_cap = 0;
        B_CK(cudaMalloc(&e->d_maps, sizeof(int2) * maps.size()));
        e->maps_cap = maps.size();
    }
    if (!maps.empty())
        B_CK(cudaMemcpyAsync(e->d_maps, maps.data(), sizeof(int2) * maps.size(), cudaMemcpyHostToDevice, e->st));
    r.insts = e->d_insts;
    r.n_inst = e->max_slots;
    r.maps = e->d_maps;
    r.max_window = 1;
    r.max_maxit = 1;
    for (int i : ids) {
        r.max_window = std::max(r.max_window, e->slots[i].plan.d.back_window);
        r.max_maxit = std::max(r.max_maxit, e->slots[i].plan.o.maxit);
    }
    r.d_active = e->d_active;
    B_CK(cudaStreamSynchronize(e->st));        // maps uploaded before they are captured
    const int rc = capture_round(r, e->st, &e->round, e->round_sig);
    e->round_sig = round_signature(r);
    if (rc) return rc;
    e->dirty = false;
    return CTG_OK;
}

}  // namespace

extern "C" int ctg_engine_create(ctg_ctx *ctx, int32_t max_slots, size_t hbm_budget_bytes,
                                 ctg_engine **out) {
    if (!ctx || max_slots < 1 || max_slots > 4096 || !out) return CTG_ERR_INVALID_ARG;
    *out = nullptr;
    ctg_engine *e = new (std::nothrow) ctg_engine();
    if (!e) return CTG_ERR_OOM;
    e->ctx = ctx;
    e->max_slots = max_slots;
    e->budget = hbm_budget_bytes;
    e->slots.resize(max_slots);
    e->h_insts.assign(max_slots, BatchInst{});
    int rc = ck(cudaMalloc(&e->d_insts, sizeof(BatchInst) * max_slots));
    if (rc == CTG_OK) rc = ck(cudaMemset(e->d_insts, 0, sizeof(BatchInst) * max_slots));   // all inactive
    // the memset ran on the legacy stream; the engine's own stream is not
    // ordered after it
    if (rc == CTG_OK) rc = ck(cudaDeviceSynchronize());
    if (rc == CTG_OK) rc = ck(cudaMalloc(&e->d_active, sizeof(int)));
    if (rc == CTG_OK) rc = ck(cudaMallocHost(&e->h_active, sizeof(int)));
    if (rc == CTG_OK) rc = ck(cudaMallocHost(&e->h_stage, sizeof(double) * 8 * max_slots));
    if (rc == CTG_OK) rc = ck(cudaMallocHost(&e->h_pinned, sizeof(BatchInst) * max_slots));
    if (rc == CTG_OK) rc = ck(cudaStreamCreateWithFlags(&e->st, cudaStreamNonBlocking));
    if (rc == CTG_OK) rc = ck(cudaEventCreateWithFlags(&e->ev_in, cudaEventDisableTiming));
    int dev = 0;
    if (rc == CTG_OK) rc = ck(cudaGetDevice(&dev));
    if (rc == CTG_OK) {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        rc = ck(cudaMemPoolCreate(&e->pool, &props));
    }
    if (rc == CTG_OK) {
        // freed workspaces stay mapped for the next admissions
        unsigned long long keep = hbm_budget_bytes;
        rc = ck(cudaMemPoolSetAttribute(e->pool, cudaMemPoolAttrReleaseThreshold, &keep));
    }
    if (rc != CTG_OK) {
        release_engine(e);
        return rc;
    }
    *out = e;
    return CTG_OK;
}

extern "C" void ctg_engine_destroy(ctg_engine *e) { release_engine(e); }

extern "C" size_t ctg_engine_request_bytes(const ctg_geom *g, int32_t variant, const ctg_opts *o) {
    if (!plan_valid(g, variant, o)) return 0;
    InstPlan p;
    p.g = *g;
    p.o = *o;
    p.variant = variant;
    return al256(plan_instance(p, nullptr));
}

extern "C" int32_t ctg_engine_in_flight(const ctg_engine *e) {
    if (!e) return 0;
    int c = 0;
    for (const auto &s : e->slots) c += s.state != 0;
    return c;
}

extern "C" int ctg_engine_submit(ctg_engine *e, const ctg_geom *g, int32_t variant,
                                 const ctg_opts *o, const float *b_dev, const float *x0_dev,
                                 float *x_dev, double *history, int64_t tag, void *stream) {
    if (!e || !b_dev || !x_dev || !plan_valid(g, variant, o)) return CTG_ERR_INVALID_ARG;
    int slot = -1;
    for (int i = 0; i < e->max_slots && slot < 0; ++i)
        if (e->slots[i].state == 0) slot = i;
    const size_t bytes = ctg_engine_request_bytes(g, variant, o);
    if (bytes > e->budget) return CTG_ERR_OOM;      // would never fit
    if (slot < 0 || e->in_use + bytes > e->budget) return CTG_ERR_BUSY;
    ctg_engine::Slot &s = e->slots[slot];
    s.plan = InstPlan{};
    s.plan.g = *g;
    s.plan.o = *o;
    s.plan.variant = variant;
    for (const auto &fp : e->fwd_plans)
        if (same_fwd_geom(fp.first, *g)) s.plan.fwd = fp.second;
    B_CK(cudaEventRecord(e->ev_in, static_cast<cudaStream_t>(stream)));
    B_CK(cudaStreamWaitEvent(e->st, e->ev_in, 0));
    void *ws = nullptr;
    B_CK(cudaMallocFromPoolAsync(&ws, bytes, e->pool, e->st));
    s.ws = static_cast<char *>(ws);
    s.bytes = bytes;
    plan_instance(s.plan, s.ws);
    const bool new_plan = !s.plan.fwd;
    if (const int urc = upload_tables(s.plan, e->st)) {
        cudaFreeAsync(s.ws, e->st);
        cudaStreamSynchronize(e->st);
        s = ctg_engine::Slot{};
        return urc;
    }
    if (new_plan) {
        if (e->fwd_plans.size() >= 256) e->fwd_plans.clear();
        e->fwd_plans.emplace_back(*g, s.plan.fwd);
    }
    s.b = b_dev;
    s.x0 = x0_dev;
    s.x = x_dev;
    s.tag = tag;
    s.info = ctg_info{};
    s.info.history = history;
    double *stage = e->h_stage + 8 * slot;
    int rc = enqueue_start(s.plan, b_dev, x0_dev, stage, e->st);
    if (rc == CTG_OK) rc = ck(cudaStreamSynchronize(e->st));   // tables copied, start read back
    int act = 0;
    if (rc == CTG_OK) rc = activate(s.plan, stage, &s.info, e->st, &act);
    if (rc != CTG_OK) {
        cudaFreeAsync(s.ws, e->st);
        cudaStreamSynchronize(e->st);
        s = ctg_engine::Slot{};
        return rc;
    }
    e->in_use += bytes;
    s.plan.d.b = b_dev;
    s.plan.d.x0 = x0_dev;
    s.plan.d.x = x_dev;
    e->h_pinned[slot] = s.plan.d;
    B_CK(cudaMemcpyAsync(e->d_insts + slot, e->h_pinned + slot, sizeof(BatchInst), cudaMemcpyHostToDevice, e->st));
    B_CK(cudaStreamSynchronize(e->st));
    if (act) {
        s.state = 1;
        ++e->running;
        e->dirty = true;
    } else {
        s.state = 2;    // finished at k = 0; x = x0 is formed by the next step
    }
    return CTG_OK;
}

extern "C" int ctg_engine_step(ctg_engine *e, int32_t rounds, int32_t max_done, int64_t *done_tags,
                               ctg_info *done_infos, int32_t *n_done) {
    if (!e || rounds < 0 || max_done < 0 || !n_done || (max_done > 0 && (!done_tags || !done_infos)))
        return CTG_ERR_INVALID_ARG;
    *n_done = 0;
    cudaStream_t st = e->st;
    if (e->running > 0 && rounds > 0) {
        if (e->dirty) {
            const int rc = recapture(e);
            if (rc) return rc;
        }
        *e->h_active = e->running;
        B_CK(cudaMemcpyAsync(e->d_active, e->h_active, sizeof(int), cudaMemcpyHostToDevice, st));
        for (int j = 0; j < rounds; ++j) B_CK(cudaGraphLaunch(e->round, st));
        B_CK(ctg_batch_solve_y(e->d_insts, e->max_slots, 1024, st));   // y of solves that just finished
        B_CK(cudaMemcpyAsync(e->h_pinned, e->d_insts, sizeof(BatchInst) * e->max_slots,
                             cudaMemcpyDeviceToHost, st));
        B_CK(cudaMemcpyAsync(e->h_active, e->d_active, sizeof(int), cudaMemcpyDeviceToHost, st));
        B_CK(cudaStreamSynchronize(st));
        e->running = *e->h_active;
        for (int i = 0; i < e->max_slots; ++i)
            if (e->slots[i].state == 1 && !e->h_pinned[i].active) e->slots[i].state = 2;
    }
    // form and report finished solves
    std::vector<int> fin;
    for (int i = 0; i < e->max_slots && (int)fin.size() < max_done; ++i)
        if (e->slots[i].state == 2) fin.push_back(i);
    for (int i : fin) {
        ctg_engine::Slot &s = e->slots[i];
        const BatchInst d = e->h_pinned[i];    // state after the last rounds (or at admission)
        const int rc = enqueue_finish(s.plan, d, s.b, s.x0, s.x, &s.info, e->h_stage + 8 * i, st);
        if (rc) return rc;
    }
    if (!fin.empty()) B_CK(cudaStreamSynchronize(st));
    for (int i : fin) {
        ctg_engine::Slot &s = e->slots[i];
        if (s.info.iters > 0) s.info.resnorm = std::sqrt(e->h_stage[8 * i + 5]);
        done_tags[*n_done] = s.tag;
        done_infos[*n_done] = s.info;
        ++*n_done;
        B_CK(cudaFreeAsync(s.ws, st));
        e->in_use -= s.bytes;
        s = ctg_engine::Slot{};
        e->h_pinned[i] = BatchInst{};             // inactive
        B_CK(cudaMemcpyAsync(e->d_insts + i, e->h_pinned + i, sizeof(BatchInst), cudaMemcpyHostToDevice, st));
    }
    if (!fin.empty()) B_CK(cudaStreamSynchronize(st));
    return CTG_OK;
}
