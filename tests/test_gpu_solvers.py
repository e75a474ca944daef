"""Parity of the CUDA AB-GMRES / BA-GMRES path with the FP64 oracle.

The GMRES iterate x_k of an ill-posed CT problem is an ill-conditioned
function of the arithmetic once k passes ~15: two FP64 orderings of the
same method (MGS vs CGS2) already differ by up to ~1e-4 there.  So parity
is checked in two ways:
  * iterate parity, ||x_k^gpu - x_k^orc|| <= 1e-4 ||x_k^orc||, at the
    well-conditioned early iterations and at the discrepancy-principle stop
    of the 1%-noise random-ellipse workloads (k_DP ~ 13);
  * step-wise parity at EVERY k: the oracle applies M = AB (or BA) in FP64
    to the GPU's own basis vectors (read back from the caller workspace) and
    must reproduce the GPU's Hessenberg columns, M W_k = W_{k+1} H_k, the
    orthonormality of W, and x_k = x0 + B W_k y_k (AB) / x0 + W_k y_k (BA)
    with y_k the FP64 least-squares solution for the GPU's H_k.
"""
import numpy as np
import pytest

from paper_2110_01481_gb300 import inputs as I

pytestmark = pytest.mark.gpu
X_TOL = 1e-4


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2110_01481_gb300 as P
    return P


def _problem(O, N, Na, phantom="ellipses", eta=0.01, seed=1001):
    Nd = I.detector_count(N)
    og = O.Geometry(N, Na, Nd)
    xt = I.shepp_logan(N) if phantom == "shepp" else I.random_ellipses(N, seed)
    b, enorm = I.add_noise(O.forward(og, xt), eta, seed)
    b = b.astype(np.float32).astype(np.float64)         # the GPU sees FP32 data
    return og, xt.ravel(), b, enorm


def _ops(O, og):
    return (lambda v: O.forward(og, v)), (lambda v: O.backproject(og, v))


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _solve(P, variant, og, b, maxit, **kw):
    import torch
    g = P.Geometry(og.N, og.n_angles, og.n_det)
    bt = torch.tensor(b, dtype=torch.float32, device="cuda")
    fn = P.ab_gmres if variant == "ab" else P.ba_gmres
    if "x0" in kw and kw["x0"] is not None:
        kw["x0"] = torch.tensor(kw["x0"], dtype=torch.float32, device="cuda")
    r = fn(g, bt, maxit, **kw)
    torch.cuda.synchronize()
    return g, r


@pytest.mark.parametrize("variant", ["ab", "ba"])
@pytest.mark.parametrize("phantom", ["shepp", "ellipses"])
def test_early_iterates_match_oracle(P, oracle_mod, variant, phantom):
    O = oracle_mod
    og, xt, b, _ = _problem(O, 64, 90, phantom)
    A, B = _ops(O, og)
    ref = (O.ab_gmres if variant == "ab" else O.ba_gmres)(A, B, b, 10, keep_iterates=True)
    for k in (1, 2, 3, 5, 8, 10):
        _, r = _solve(P, variant, og, b, k)
        assert r.iters == k and r.stop_reason == 0
        x = r.x.double().cpu().numpy()
        assert _rel(x, ref["iterates"][k]) <= X_TOL, k
        assert r.resnorm == pytest.approx(ref["resnorm"][k], rel=1e-5)


def _check_stepwise(P, O, variant, K):
    og, xt, b, _ = _problem(O, 64, 90, "shepp")
    A, B = _ops(O, og)
    g, r = _solve(P, variant, og, b, K, keep_workspace=True)
    assert r.iters == K
    W = r.basis(g, variant, K).double().cpu().numpy()           # (K+1, L)
    H = r.hessenberg(g, variant, K).cpu().numpy()               # (K+1, K)
    M = (lambda v: A(B(v))) if variant == "ab" else (lambda v: B(A(v)))
    # w_1 = r0 / ||r0|| with x0 = 0: r0 = b (AB) or B b (BA)
    r0 = b if variant == "ab" else B(b)
    assert _rel(W[0], r0 / np.linalg.norm(r0)) <= 1e-5
    assert np.abs(W @ W.T - np.eye(K + 1)).max() <= 2e-5
    for k in range(1, K + 1):
        Mw = M(W[k - 1])
        # Hessenberg column from the GPU's own basis, in FP64
        resid = Mw - W[: k + 1].T @ H[: k + 1, k - 1]
        assert np.linalg.norm(resid) <= 2e-5 * np.linalg.norm(Mw), k
        assert np.all(H[k + 1:, k - 1] == 0.0)
    # x_K from the GPU's (W, H) in FP64
    e1 = np.zeros(K + 1)
    e1[0] = np.linalg.norm(r0)
    y = np.linalg.lstsq(H, e1, rcond=None)[0]
    x_ref = B(W[:K].T @ y) if variant == "ab" else W[:K].T @ y
    return r, e1, H, y, x_ref


@pytest.mark.parametrize("variant", ["ab", "ba"])
def test_stepwise_arnoldi_parity_every_k(P, oracle_mod, variant):
    r, e1, H, y, x_ref = _check_stepwise(P, oracle_mod, variant, 50)
    assert _rel(r.x.double().cpu().numpy(), x_ref) <= 1e-5
    assert r.rho == pytest.approx(np.linalg.norm(e1 - H @ y), rel=1e-6)
    # GMRES residual is non-increasing
    if variant == "ab":
        hist = np.array(r.history)
        assert np.all(np.diff(hist) <= 1e-6 * hist[0])


@pytest.mark.parametrize("variant", ["ab", "ba"])
def test_stepwise_arnoldi_parity_across_the_one_launch_limit(P, oracle_mod, variant):
    """Without a stopping rule neither variant forms y_k in its steps, so
    steps up to k = 128 run the one-launch CGS2 step and later ones the
    separate passes: every Hessenberg column on both sides of the switch
    reproduces M w_k from the GPU's own basis in FP64, and the basis stays
    orthonormal, to k = 140."""
    r, e1, H, y, x_ref = _check_stepwise(P, oracle_mod, variant, 140)
    assert r.rho == pytest.approx(np.linalg.norm(e1 - H @ y), rel=1e-4)


@pytest.mark.parametrize("variant", ["ab", "ba"])
@pytest.mark.parametrize("N,Na", [(64, 90), (128, 180)])
def test_discrepancy_principle_stop(P, oracle_mod, variant, N, Na):
    """Sec. 6.4: stop at the first k with ||b - A x_k|| <= tau ||e||; the
    index may differ by one only when the residual sits within 1e-4 of the
    threshold."""
    O = oracle_mod
    og, xt, b, enorm = _problem(O, N, Na, "ellipses", seed=1000 + N)
    A, B = _ops(O, og)
    tau = 1.02
    solver = O.ab_gmres if variant == "ab" else O.ba_gmres
    ref = solver(A, B, b, 60, tau=tau, noise_norm=enorm, keep_iterates=True)
    _, r = _solve(P, variant, og, b, 60, tau=tau, noise_norm=enorm)
    target = tau * enorm
    assert r.stop_reason == 1 and ref["stop_reason"] == 1
    kg, ko = r.iters, ref["k"]
    if kg != ko:
        assert abs(kg - ko) == 1
        kk = min(kg, ko)
        assert abs(ref["resnorm"][kk] - target) < 1e-4 * target
    else:
        assert _rel(r.x.double().cpu().numpy(), ref["x"]) <= X_TOL
    assert r.resnorm <= target * (1 + 1e-5)


@pytest.mark.parametrize("variant", ["ab", "ba"])
def test_nonzero_initial_guess(P, oracle_mod, variant):
    O = oracle_mod
    og, xt, b, _ = _problem(O, 48, 60)
    A, B = _ops(O, og)
    x0 = (0.5 * I.random_ellipses(48, 5).ravel()).astype(np.float32).astype(np.float64)
    ref = (O.ab_gmres if variant == "ab" else O.ba_gmres)(A, B, b, 6, x0=x0)
    _, r = _solve(P, variant, og, b, 6, x0=x0)
    assert _rel(r.x.double().cpu().numpy(), ref["x"]) <= X_TOL


@pytest.mark.parametrize("variant", ["ab", "ba"])
def test_nonzero_initial_guess_with_discrepancy_stop(P, oracle_mod, variant):
    """x0 != 0 together with the DP stop: the residual of x_k is measured
    from b - A x0 (BA reuses the basis vectors' projections for it)."""
    O = oracle_mod
    og, xt, b, enorm = _problem(O, 64, 90, seed=1064)
    A, B = _ops(O, og)
    x0 = (0.3 * I.random_ellipses(64, 6).ravel()).astype(np.float32).astype(np.float64)
    solver = O.ab_gmres if variant == "ab" else O.ba_gmres
    ref = solver(A, B, b, 60, x0=x0, tau=1.02, noise_norm=enorm)
    _, r = _solve(P, variant, og, b, 60, x0=x0, tau=1.02, noise_norm=enorm)
    assert r.stop_reason == 1 and ref["stop_reason"] == 1
    target = 1.02 * enorm
    if r.iters == ref["k"]:
        assert _rel(r.x.double().cpu().numpy(), ref["x"]) <= X_TOL
    else:
        assert abs(r.iters - ref["k"]) == 1
        kk = min(r.iters, ref["k"])
        assert abs(ref["resnorm"][kk] - target) < 1e-4 * target
    assert r.resnorm == pytest.approx(np.linalg.norm(b - A(r.x.double().cpu().numpy())), rel=1e-5)


@pytest.mark.parametrize("variant", ["ab", "ba"])
def test_degenerate_starts(P, oracle_mod, variant):
    import torch
    O = oracle_mod
    og, xt, b, _ = _problem(O, 32, 24)
    # b = 0: r0 = 0, nothing to do; x = x0 = 0 with a breakdown report
    _, r = _solve(P, variant, og, np.zeros_like(b), 5)
    assert r.iters == 0 and r.stop_reason == 2 and torch.count_nonzero(r.x) == 0
    # x0 already satisfies the discrepancy principle: k = 0, x = x0
    x0 = xt.astype(np.float32)
    bb = O.forward(og, x0.astype(np.float64))
    _, r = _solve(P, variant, og, bb, 5, x0=x0, noise_norm=1e-2)
    assert r.iters == 0 and r.stop_reason == 1
    np.testing.assert_array_equal(r.x.cpu().numpy(), x0)


@pytest.mark.parametrize("variant", ["ab", "ba"])
def test_workspace_modes_and_determinism(P, oracle_mod, variant):
    import torch
    O = oracle_mod
    og, xt, b, _ = _problem(O, 64, 90)
    g = P.Geometry(64, 90, og.n_det)
    bt = torch.tensor(b, dtype=torch.float32, device="cuda")
    fn = P.ab_gmres if variant == "ab" else P.ba_gmres
    r1 = fn(g, bt, 20)
    ws = torch.empty(P.workspace_bytes(g, variant, 20), dtype=torch.uint8, device="cuda")
    r2 = fn(g, bt, 20, workspace=ws)
    r3 = fn(g, bt, 20, workspace=ws)
    torch.cuda.synchronize()
    assert torch.equal(r1.x, r2.x) and torch.equal(r2.x, r3.x)
    from paper_2110_01481_gb300 import _native as nat
    with pytest.raises(nat.CtgError) as ei:
        fn(g, bt, 20, workspace=ws[: ws.numel() // 2])
    assert ei.value.status == nat.CTG_ERR_WORKSPACE


@pytest.mark.parametrize("L,k", [(1, 0), (3, 1), (1000, 7), (4099, 33), (522000, 64),
                                 (262144 + 3, 150),
                                 # the middle pass staged through shared memory (FP32, L % 4 == 0,
                                 # 64 < k <= 200), with a partial last slice of 104 elements
                                 (1000, 80), (522000, 100), (262144, 150), (524288, 200)])
def test_cgs2_entry_point(P, oracle_mod, L, k):
    """One CGS2 step against the oracle's FP64 classical Gram-Schmidt applied
    twice: h within 1e-5 of ||q||, w_out = q / ||q|| within 1e-5."""
    import torch
    from oracle import krylov
    rng = np.random.default_rng(L + k)
    Wd = np.linalg.qr(rng.standard_normal((L, max(k, 1))))[0].T[:k] if k else np.zeros((0, L))
    q = rng.standard_normal(L) + (Wd.T @ rng.standard_normal(k) if k else 0)
    ld = (L + 63) // 64 * 64
    Wt = torch.zeros((max(k, 1), ld), dtype=torch.float32, device="cuda")
    if k:
        Wt[:k, :L] = torch.tensor(Wd, dtype=torch.float32)
    qt = torch.tensor(q, dtype=torch.float32, device="cuda")
    Wf = Wt[:k, :L].double().cpu().numpy()
    qf = qt.double().cpu().numpy()
    h, w = P.cgs2(Wt, k, qt)
    torch.cuda.synchronize()
    qo, ho = krylov._orthogonalise(qf.copy(), Wf, k, "cgs2")
    nq = np.linalg.norm(qo)
    h = h.cpu().numpy()
    if k:
        assert np.abs(h[:k] - ho).max() <= 1e-5 * np.linalg.norm(qf)
    assert h[k] == pytest.approx(nq, rel=1e-4, abs=1e-5 * np.linalg.norm(qf))
    assert _rel(w.double().cpu().numpy(), qo / nq) <= 1e-4


@pytest.mark.parametrize("variant", ["ab", "ba"])
def test_full_size_sampled_parity(P, oracle_mod, variant):
    """512^2, 720 angles, 725 bins: early iterates against the oracle, and
    the step-wise Hessenberg check on a sample of later columns."""
    O = oracle_mod
    og, xt, b, enorm = _problem(O, 512, 720, seed=2001)
    A, B = _ops(O, og)
    ref = (O.ab_gmres if variant == "ab" else O.ba_gmres)(A, B, b, 4, keep_iterates=True)
    K = 40
    g, r = _solve(P, variant, og, b, K, keep_workspace=True)
    W = r.basis(g, variant, K)
    H = r.hessenberg(g, variant, K).cpu().numpy()
    M = (lambda v: A(B(v))) if variant == "ab" else (lambda v: B(A(v)))
    for k in (1, 2, 10, 25, 40):
        Wk = W[: k + 1].double().cpu().numpy()
        Mw = M(Wk[k - 1])
        assert np.linalg.norm(Mw - Wk.T @ H[: k + 1, k - 1]) <= 2e-5 * np.linalg.norm(Mw), k
    for k in (1, 2, 4):
        _, rk = _solve(P, variant, og, b, k)
        assert _rel(rk.x.double().cpu().numpy(), ref["iterates"][k]) <= X_TOL, k



@pytest.mark.parametrize("N,Na", [(4, 8), (6, 10)])
@pytest.mark.parametrize("variant", ["ab", "ba"])
def test_breakdown_when_the_krylov_space_is_exhausted(P, oracle_mod, variant, N, Na):
    """On an N x N image with N^2 < m, the Krylov space of B A (square,
    nonsingular) or of A B (rank N^2) is exhausted after about N^2 steps:
    h_{k+1,k} falls to the rounding level and both sides stop with a
    breakdown.  The GPU tests h_{k+1,k} <= 1e-6 ||q|| on FP32 vectors where
    the oracle tests 1e-14 in FP64, so the GPU may stop up to two steps
    earlier.  BA: the iterate is the unique minimiser of ||B b - B A x||, so
    x matches the oracle's.  AB: A B is singular, the projected least-squares
    problem becomes ill-conditioned as the space fills, and its FP32 basis
    error (~1e-7 of ||A B||) is amplified in x (Sec. 2 minimises over the
    space; at exhaustion the minimiser is min_z ||b - A B z||); the GPU's
    residual stays within a factor 2 of that minimum, and the residual it
    reports is the true ||b - A x|| of the x it returns."""
    O = oracle_mod
    og, _, b, _ = _problem(O, N, Na, seed=11)
    A, B = _ops(O, og)
    ref = (O.ab_gmres if variant == "ab" else O.ba_gmres)(A, B, b, 80)
    _, r = _solve(P, variant, og, b, 80)
    assert r.stop_reason == ref["stop_reason"] == 2
    assert ref["k"] - 2 <= r.iters <= ref["k"]
    x = r.x.double().cpu().numpy()
    true_res = np.linalg.norm(b - A(x))
    assert r.resnorm == pytest.approx(true_res, rel=1e-4)
    if variant == "ba":
        assert _rel(x, ref["x"]) <= X_TOL
        # the residual is ~1% of ||b||, so x's 1e-4 carries into it ~100-fold
        assert r.resnorm == pytest.approx(ref["resnorm"][-1], rel=1e-3)
    else:
        assert (1 - 1e-9) * ref["resnorm"][-1] <= true_res <= 2.0 * ref["resnorm"][-1]
