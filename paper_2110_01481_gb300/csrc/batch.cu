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
#include <vector>

#include "ctg_internal.cuh"

namespace {

constexpr int kRoundsPerCheck = 4;

size_t al256(size_t v) { return (v + 255) & ~(size_t)255; }
size_t rup(size_t v, size_t m) { return (v + m - 1) / m * m; }
int padded4(int G) { return (G + 3) & ~3; }

struct InstPlan {
    ctg_geom g;
    ctg_opts o;
    int variant;
    size_t off, bytes;         // this instance's slice of the batch workspace
    BatchInst d;               // device pointers filled in at create
};

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
    const size_t ldw = rup((size_t)L, 64), ldt = rup((size_t)m, 64);
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
    d.ldt = (long long)ldt;
    d.G = ctg_vec_blocks(L);
    d.target = p.o.noise_norm > 0.0 ? p.o.tau * p.o.noise_norm : 0.0;
    d.W = (float *)take(sizeof(float) * ldw * (size_t)(maxit + 1));
    d.T = ba ? (float *)take(sizeof(float) * ldt * (size_t)(maxit + 1)) : nullptr;
    d.H = (double *)take(sizeof(double) * (size_t)(maxit + 1) * maxit);
    d.R = (double *)take(sizeof(double) * (size_t)maxit * maxit);
    d.gc = (double *)take(sizeof(double) * maxit);
    d.gs = (double *)take(sizeof(double) * maxit);
    d.gg = (double *)take(sizeof(double) * (maxit + 1));
    d.y = (double *)take(sizeof(double) * maxit);
    d.hist = (double *)take(sizeof(double) * (maxit + 1));
    d.vn = (float *)take(sizeof(float) * rup((size_t)n, 64));
    d.vm = (float *)take(sizeof(float) * rup((size_t)m, 64));
    d.r0m = ba ? (float *)take(sizeof(float) * rup((size_t)m, 64)) : nullptr;
    d.pad = (float2 *)take(sizeof(float) * pl.floats);
    d.fwd = (const FwdAngle *)take(sizeof(FwdAngle) * g.n_angles);
    d.back = (const BackAngle *)take(sizeof(BackAngle) * g.n_angles);
    d.partials = (float *)take(sizeof(float) * (size_t)(maxit + 3) * Gp);
    d.h1 = (double *)take(sizeof(double) * (maxit + 3));
    d.h2 = (double *)take(sizeof(double) * (maxit + 3));
    d.scal = (double *)take(sizeof(double) * 8);
    d.counter = (unsigned *)take(sizeof(unsigned) * 4);
    return off;
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
    int map_back = 0, map_pad = 0, map_fwd = 0, map_cgs = 0, map_m = 0;   // offsets
    int n_back = 0, n_pad = 0, n_fwd = 0, n_cgs = 0, n_m = 0;             // lengths
    int max_window = 0, max_maxit = 0;
    int *d_active = nullptr;
    int *h_active = nullptr;     // pinned
    double *h_stage = nullptr;   // pinned: per instance scal[0..7]
    cudaStream_t st = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    cudaGraphExec_t round = nullptr;
};

namespace {

void release(ctg_batch *b) {
    if (!b) return;
    if (b->st) cudaStreamSynchronize(b->st);
    if (b->round) cudaGraphExecDestroy(b->round);
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

int capture_round(ctg_batch *b) {
    cudaGraph_t graph = nullptr;
    B_CK(ctg_batch_prepare(b->max_maxit));   // kernel attributes, set outside the capture
    B_CK(cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    const int2 *M = b->d_maps;
    if (e == cudaSuccess) e = ctg_batch_back(b->d_insts, M + b->map_back, b->n_back, CTG_PH_BACK_AB, b->max_window, b->st);
    if (e == cudaSuccess) e = ctg_batch_pad(b->d_insts, M + b->map_pad, b->n_pad, b->st);
    if (e == cudaSuccess) e = ctg_batch_forward(b->d_insts, M + b->map_fwd, b->n_fwd, b->st);
    if (e == cudaSuccess) e = ctg_batch_back(b->d_insts, M + b->map_back, b->n_back, CTG_PH_BACK_BA, b->max_window, b->st);
    if (e == cudaSuccess) e = ctg_batch_cgs2(b->d_insts, M + b->map_cgs, b->n_cgs, b->max_maxit, b->st);
    if (e == cudaSuccess) e = ctg_batch_givens(b->d_insts, b->n, b->st);
    if (e == cudaSuccess) e = ctg_batch_residual(b->d_insts, M + b->map_m, b->n_m, b->max_maxit, b->st);
    if (e == cudaSuccess) e = ctg_batch_finish(b->d_insts, b->n, b->d_active, b->st);
    cudaError_t e2 = cudaStreamEndCapture(b->st, &graph);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->round, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    return ck(e);
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
        if (!ctg_geom_valid(&p.g) || !ctg_opts_valid(&p.o) || p.o.basis_dtype != CTG_BASIS_FP32 ||
            p.o.maxit > 1024 || (p.variant != CTG_AB && p.variant != CTG_BA)) {
            release(b);
            return CTG_ERR_INVALID_ARG;
        }
        ctg_build_tables(&p.g, fw[i], bk[i]);
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
    int rc = ck(cudaMalloc(&b->ws, total));
    if (rc == CTG_OK) rc = ck(cudaMemset(b->ws, 0, total));
    // block maps
    std::vector<int2> maps;
    auto add_map = [&](int &off, int &len, auto count) {
        off = (int)maps.size();
        for (int i = 0; i < n; ++i) {
            const int c = count(b->inst[i]);
            for (int j = 0; j < c; ++j) maps.push_back(make_int2(i, j));
        }
        len = (int)maps.size() - off;
    };
    add_map(b->map_back, b->n_back, [](const InstPlan &p) { return ctg_back_tiles(p.g.N); });
    add_map(b->map_pad, b->n_pad, [](const InstPlan &p) { return ctg_pad_tiles(p.g.N); });
    add_map(b->map_fwd, b->n_fwd, [](const InstPlan &p) { return ctg_fwd_blocks(p.g.n_angles, p.g.n_det); });
    add_map(b->map_cgs, b->n_cgs, [](const InstPlan &p) {
        return ctg_vec_blocks(p.variant == CTG_BA ? (long long)p.g.N * p.g.N
                                                  : (long long)p.g.n_angles * p.g.n_det);
    });
    add_map(b->map_m, b->n_m, [](const InstPlan &p) {
        return (p.variant == CTG_BA && p.o.noise_norm > 0.0)
                   ? ctg_vec_blocks((long long)p.g.n_angles * p.g.n_det) : 0;
    });
    if (rc == CTG_OK) rc = ck(cudaMalloc(&b->d_maps, sizeof(int2) * (maps.empty() ? 1 : maps.size())));
    if (rc == CTG_OK && !maps.empty())
        rc = ck(cudaMemcpy(b->d_maps, maps.data(), sizeof(int2) * maps.size(), cudaMemcpyHostToDevice));
    if (rc == CTG_OK) rc = ck(cudaMalloc(&b->d_insts, sizeof(BatchInst) * n));
    if (rc == CTG_OK) rc = ck(cudaMalloc(&b->d_active, sizeof(int)));
    if (rc == CTG_OK) rc = ck(cudaMallocHost(&b->h_active, sizeof(int)));
    if (rc == CTG_OK) rc = ck(cudaMallocHost(&b->h_stage, sizeof(double) * 8 * n));
    if (rc == CTG_OK) rc = ck(cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking));
    if (rc == CTG_OK) rc = ck(cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming));
    if (rc == CTG_OK) rc = ck(cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming));
    for (int i = 0; rc == CTG_OK && i < n; ++i) {
        InstPlan &p = b->inst[i];
        plan_instance(p, b->ws + p.off);
        rc = ck(cudaMemcpy((void *)p.d.fwd, fw[i].data(), sizeof(FwdAngle) * fw[i].size(), cudaMemcpyHostToDevice));
        if (rc == CTG_OK)
            rc = ck(cudaMemcpy((void *)p.d.back, bk[i].data(), sizeof(BackAngle) * bk[i].size(), cudaMemcpyHostToDevice));
        p.d.back_window = ctg_back_window(bk[i].data(), p.g.n_angles);
    }
    if (rc == CTG_OK) rc = capture_round(b);
    if (rc != CTG_OK) {
        release(b);
        return rc;
    }
    *out = b;
    return CTG_OK;
}

extern "C" void ctg_batch_destroy(ctg_batch *b) { release(b); }

extern "C" size_t ctg_batch_workspace_bytes(const ctg_batch *b) { return b ? b->ws_bytes : 0; }

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
    // ---- per instance: r0, beta and (BA) ||b - A x0|| ------------------
    for (int i = 0; i < n; ++i) {
        InstPlan &p = b->inst[i];
        BatchInst &d = p.d;
        const float *x0 = x0_dev ? x0_dev[i] : nullptr;
        const RedScratch rs = scratch_of(d);
        const PadLayout pl = ctg_pad_layout(p.g.N, p.g.det_spacing);
        B_CK(cudaMemsetAsync(d.counter, 0, 4 * sizeof(unsigned), st));
        B_CK(cudaMemsetAsync(d.gg, 0, sizeof(double) * (p.o.maxit + 1), st));
        B_CK(cudaMemsetAsync(d.H, 0, sizeof(double) * (size_t)(p.o.maxit + 1) * p.o.maxit, st));
        B_CK(cudaMemsetAsync(d.hist, 0, sizeof(double) * (p.o.maxit + 1), st));
        B_CK(cudaMemsetAsync(d.pad, 0, sizeof(float) * pl.floats, st));
        if (x0) {
            B_CK(ctg_launch_pad(x0, CTG_BASIS_FP32, d.pad, p.g.N, pl, st));
            B_CK(ctg_launch_forward(d.pad, p.g.N, pl, p.g.n_angles, p.g.n_det, d.fwd, d.vm, st));
        }
        if (p.variant == CTG_AB) {
            B_CK(ctg_sub_norm2(b_dev[i], x0 ? d.vm : nullptr, d.vm, d.m, d.scal + 2, rs, st));
        } else {
            B_CK(ctg_sub_norm2(b_dev[i], x0 ? d.vm : nullptr, d.r0m, d.m, d.scal + 4, rs, st));
            B_CK(ctg_launch_back(d.r0m, CTG_BASIS_FP32, p.g.N, p.g.n_angles, p.g.n_det, d.back,
                                 d.back_window, nullptr, d.vn, st));
            B_CK(ctg_sub_norm2(d.vn, nullptr, nullptr, d.n, d.scal + 2, rs, st));
        }
        B_CK(cudaMemcpyAsync(b->h_stage + 8 * i, d.scal, sizeof(double) * 8, cudaMemcpyDeviceToHost, st));
    }
    B_CK(cudaStreamSynchronize(st));
    int active = 0;
    for (int i = 0; i < n; ++i) {
        InstPlan &p = b->inst[i];
        BatchInst &d = p.d;
        const double beta = std::sqrt(b->h_stage[8 * i + 2]);
        const double res0 = p.variant == CTG_AB ? beta : std::sqrt(b->h_stage[8 * i + 4]);
        d.k = 1;
        d.iters = 0;
        d.breakdown = 0;
        d.rho = beta;
        d.resnorm = res0;
        d.stop_reason = CTG_STOP_MAXIT;
        infos[i].iters = 0;
        infos[i].rho = beta;
        infos[i].resnorm = res0;
        if (infos[i].history) infos[i].history[0] = d.target > 0.0 ? res0 : beta;
        const bool dp0 = d.target > 0.0 && res0 <= d.target;
        if (dp0 || beta == 0.0) {                   // k = 0: x = x0
            d.active = 0;
            d.stop_reason = dp0 ? CTG_STOP_DP : CTG_STOP_BREAKDOWN;
            continue;
        }
        d.active = 1;
        ++active;
        // w_1 = r0 / beta and the rotated right-hand side beta e1
        B_CK(ctg_scale(p.variant == CTG_AB ? d.vm : d.vn, d.scal + 2, d.W, CTG_BASIS_FP32, d.L, st));
        b->h_stage[8 * i + 6] = beta;
        B_CK(cudaMemcpyAsync(d.gg, &b->h_stage[8 * i + 6], sizeof(double), cudaMemcpyHostToDevice, st));
    }
    std::vector<BatchInst> hi(n);
    for (int i = 0; i < n; ++i) hi[i] = b->inst[i].d;
    B_CK(cudaMemcpyAsync(b->d_insts, hi.data(), sizeof(BatchInst) * n, cudaMemcpyHostToDevice, st));
    *b->h_active = active;
    B_CK(cudaMemcpyAsync(b->d_active, b->h_active, sizeof(int), cudaMemcpyHostToDevice, st));
    // ---- rounds -----------------------------------------------------------
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
    B_CK(ctg_batch_solve_y(b->d_insts, n, st));
    B_CK(cudaMemcpyAsync(hi.data(), b->d_insts, sizeof(BatchInst) * n, cudaMemcpyDeviceToHost, st));
    B_CK(cudaStreamSynchronize(st));
    for (int i = 0; i < n; ++i) {
        InstPlan &p = b->inst[i];
        const BatchInst &d = hi[i];
        const float *x0 = x0_dev ? x0_dev[i] : nullptr;
        const RedScratch rs = scratch_of(d);
        const PadLayout pl = ctg_pad_layout(p.g.N, p.g.det_spacing);
        const int k = d.active ? d.k : d.iters;   // d.active cannot remain set after the rounds
        infos[i].iters = k;
        infos[i].stop_reason = d.stop_reason;
        infos[i].rho = k > 0 ? d.rho : infos[i].rho;
        if (k == 0) {
            if (x0) B_CK(cudaMemcpyAsync(x_dev[i], x0, sizeof(float) * d.n, cudaMemcpyDeviceToDevice, st));
            else B_CK(cudaMemsetAsync(x_dev[i], 0, sizeof(float) * d.n, st));
            continue;
        }
        if (p.variant == CTG_AB) {
            B_CK(ctg_gemv(d.W, CTG_BASIS_FP32, d.ldw, d.m, k, d.y, nullptr, d.vm, st));
            B_CK(ctg_launch_back(d.vm, CTG_BASIS_FP32, p.g.N, p.g.n_angles, p.g.n_det, d.back,
                                 d.back_window, x0, x_dev[i], st));
        } else {
            B_CK(ctg_gemv(d.W, CTG_BASIS_FP32, d.ldw, d.n, k, d.y, x0, x_dev[i], st));
        }
        B_CK(ctg_launch_pad(x_dev[i], CTG_BASIS_FP32, d.pad, p.g.N, pl, st));
        B_CK(ctg_launch_forward(d.pad, p.g.N, pl, p.g.n_angles, p.g.n_det, d.fwd, d.vm, st));
        B_CK(ctg_sub_norm2(b_dev[i], d.vm, nullptr, d.m, d.scal + 5, rs, st));
        B_CK(cudaMemcpyAsync(b->h_stage + 8 * i + 5, d.scal + 5, sizeof(double), cudaMemcpyDeviceToHost, st));
        if (infos[i].history)
            B_CK(cudaMemcpyAsync(infos[i].history + 1, d.hist + 1, sizeof(double) * k,
                                 cudaMemcpyDeviceToHost, st));
    }
    B_CK(cudaStreamSynchronize(st));
    for (int i = 0; i < n; ++i)
        if (infos[i].iters > 0) infos[i].resnorm = std::sqrt(b->h_stage[8 * i + 5]);
    B_CK(cudaEventRecord(b->ev_out, st));
    B_CK(cudaStreamWaitEvent(user, b->ev_out, 0));
    return CTG_OK;
}
