"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: each test checks a closed
form, an exact invariant, a brute-force minimiser, an independently derived
library result or a value printed in the paper.  CPU only.
"""
import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg  # noqa: F401
import pytest
import scipy.sparse.linalg as sla

from paper_2110_01481_gb300 import inputs as I

CFG1 = dict(N=64, n_angles=90, n_det=91)


def geom(O, **kw):
    return O.Geometry(**kw)


# ---------------------------------------------------------------- geometry
def test_angle_table_tie_rule_and_snapping(oracle_mod):
    O = oracle_mod
    g = geom(O, N=8, n_angles=8, n_det=13)          # 0, 22.5, ..., 157.5
    c, s, rd = O.angles(g)
    assert list(rd) == [1, 1, 1, 0, 0, 0, 1, 1]     # 45 and 135 are row-driven
    assert (c[0], s[0]) == (1.0, 0.0) and (c[4], s[4]) == (0.0, 1.0)
    np.testing.assert_allclose(c, np.cos(np.arange(8) * np.pi / 8), atol=1e-15)
    np.testing.assert_allclose(s, np.sin(np.arange(8) * np.pi / 8), atol=1e-15)
    g2 = geom(O, N=8, n_angles=3, n_det=13, angle_start_deg=90, angle_range_deg=270)
    c, s, rd = O.angles(g2)                          # 90, 180, 270
    assert list(c) == [0.0, -1.0, 0.0] and list(s) == [1.0, 0.0, -1.0]
    assert list(rd) == [0, 1, 0]
    with pytest.raises(ValueError):
        O.forward(geom(O, N=8, n_angles=4, n_det=13, angle_start_deg=0.5),
                  np.zeros(64))


# ----------------------------------------------------------- Joseph A pins
def _rand_img(N, seed=1):
    return np.random.default_rng(seed).uniform(0, 1, (N, N))


def test_joseph_theta0_closed_form(oracle_mod):
    """At theta = 0 with N even and N_det odd the rays fall half-way between
    pixel columns: each detector sums half of two adjacent columns."""
    O = oracle_mod
    N, Nd = 8, 13
    x = _rand_img(N)
    b = O.forward(geom(O, N=N, n_angles=4, n_det=Nd), x).reshape(4, Nd)
    colsum = np.concatenate([[0.0], x.sum(axis=0), [0.0]])   # zero-padded
    for d in range(Nd):
        u = (d - (Nd - 1) / 2) + (N - 1) / 2                 # half-integer
        j0 = math.floor(u)
        expect = 0.5 * (colsum[j0 + 1] + colsum[j0 + 2]) if -1 <= j0 < N else 0.0
        assert b[0, d] == pytest.approx(expect, rel=1e-14, abs=1e-14)


def test_joseph_theta0_even_detector_reads_single_column(oracle_mod):
    O = oracle_mod
    N, Nd = 8, 12                                             # f = 0 everywhere
    x = _rand_img(N)
    b = O.forward(geom(O, N=N, n_angles=2, n_det=Nd), x).reshape(2, Nd)
    for d in range(Nd):
        j = d - (Nd - 1) / 2 + (N - 1) / 2
        expect = x[:, int(j)].sum() if 0 <= j < N else 0.0
        assert b[0, d] == pytest.approx(expect, rel=1e-14, abs=1e-14)


def test_joseph_theta90_closed_form(oracle_mod):
    O = oracle_mod
    N, Nd = 8, 13
    x = _rand_img(N, 2)
    b = O.forward(geom(O, N=N, n_angles=2, n_det=Nd), x).reshape(2, Nd)
    rowsum = np.concatenate([[0.0], x.sum(axis=1), [0.0]])
    for d in range(Nd):
        i0 = math.floor(d - (Nd - 1) / 2 + (N - 1) / 2)
        expect = 0.5 * (rowsum[i0 + 1] + rowsum[i0 + 2]) if -1 <= i0 < N else 0.0
        assert b[1, d] == pytest.approx(expect, rel=1e-14, abs=1e-14)


def test_joseph_theta45_weights_and_positions(oracle_mod):
    """At 45 degrees (row-driven by the tie rule) the per-row position is
    u = sqrt(2) s_d + (N-1) - i and the weight is 1/cos 45 = sqrt(2)."""
    O = oracle_mod
    N, Nd = 8, 13
    x = _rand_img(N, 3)
    b = O.forward(geom(O, N=N, n_angles=4, n_det=Nd), x).reshape(4, Nd)
    for d in range(Nd):
        sd = d - (Nd - 1) / 2
        acc = 0.0
        for i in range(N):
            u = math.sqrt(2) * sd + (N - 1) - i
            j0 = math.floor(u)
            f = u - j0
            for j, w in ((j0, 1 - f), (j0 + 1, f)):
                if 0 <= j < N:
                    acc += w * x[i, j]
        assert b[1, d] == pytest.approx(math.sqrt(2) * acc, rel=1e-12, abs=1e-12)


def _ellipse_radon(N, rho, a, b, x0, y0, phi, theta, s):
    """Exact line integral of one ellipse (normalised units scaled by N/2)
    along x cos(theta) + y sin(theta) = s, in pixel units."""
    A, B, cx, cy = a * N / 2, b * N / 2, x0 * N / 2, y0 * N / 2
    sp = s - (cx * np.cos(theta) + cy * np.sin(theta))
    al = theta - phi
    a2 = (A * np.cos(al)) ** 2 + (B * np.sin(al)) ** 2
    arg = np.maximum(a2 - sp ** 2, 0.0)
    return rho * 2 * A * B * np.sqrt(arg) / a2


def test_joseph_matches_analytic_radon_of_ellipse(oracle_mod):
    """Pins the sign and rotation convention s = x cos + y sin: the Joseph
    projection of a pixelised off-centre rotated ellipse converges to its
    exact Radon transform as N grows."""
    O = oracle_mod
    prm = (0.8, 0.35, 0.2, 0.25, -0.3, 0.6)
    errs = []
    for N in (64, 256):
        Na, Nd = 12, I.detector_count(N)
        x = I.single_ellipse(N, *prm)
        b = O.forward(geom(O, N=N, n_angles=Na, n_det=Nd), x).reshape(Na, Nd)
        th = np.arange(Na) * np.pi / Na
        s = np.arange(Nd) - (Nd - 1) / 2
        exact = _ellipse_radon(N, *prm, th[:, None], s[None, :])
        errs.append(np.linalg.norm(b - exact) / np.linalg.norm(exact))
        # a mirrored convention (s = x cos - y sin) would be far off
        wrong = _ellipse_radon(N, *prm, -th[:, None], s[None, :])
        assert np.linalg.norm(b - wrong) / np.linalg.norm(exact) > 0.3
    assert errs[0] < 0.05 and errs[1] < errs[0] / 2, errs


def test_joseph_adjoint_and_explicit_form(oracle_mod):
    O = oracle_mod
    g = geom(O, **CFG1)
    A = O.matrix_A(g)
    rng = np.random.default_rng(4)
    x, y = rng.standard_normal(g.n), rng.standard_normal(g.m)
    Ax = O.forward(g, x)
    assert np.abs(A @ x - Ax).max() <= 1e-13 * np.abs(Ax).max()
    assert (Ax @ y) == pytest.approx(x @ (A.T @ y), rel=1e-12)


# ----------------------------------------------------- pixel-driven B pins
@pytest.mark.parametrize("N,Na,Nd,S,R", [(64, 90, 91, 0, 180), (7, 5, 10, 0, 180),
                                         (16, 9, 23, 10, 120)])
def test_backprojector_of_ones_is_angle_count(oracle_mod, N, Na, Nd, S, R):
    """Every pixel centre projects inside the detector (N_det >= sqrt(2) N)
    and the two linear weights sum to 1, so B 1_m = N_a 1_n exactly."""
    O = oracle_mod
    g = geom(O, N=N, n_angles=Na, n_det=Nd, angle_start_deg=S, angle_range_deg=R)
    np.testing.assert_array_equal(O.backproject(g, np.ones(g.m)),
                                  np.full(g.n, float(Na)))


def test_backprojector_impulse_is_hat_function(oracle_mod):
    O = oracle_mod
    N, Na, Nd = 16, 6, 23
    g = geom(O, N=N, n_angles=Na, n_det=Nd)
    a, d = 2, 9
    e = np.zeros(g.m)
    e[a * Nd + d] = 1.0
    img = O.backproject(g, e).reshape(N, N)
    th = a * np.pi / Na
    h = (N - 1) / 2
    jj, ii = np.meshgrid(np.arange(N), np.arange(N))
    u = (jj - h) * np.cos(th) + (ii - h) * np.sin(th) + (Nd - 1) / 2
    np.testing.assert_allclose(img, np.maximum(0.0, 1 - np.abs(u - d)), atol=1e-12)


def test_backprojector_explicit_form_and_unmatchedness(oracle_mod):
    O = oracle_mod
    g = geom(O, **CFG1)
    A, B = O.matrix_A(g), O.matrix_B(g)
    y = np.random.default_rng(5).standard_normal(g.m)
    np.testing.assert_allclose(B @ y, O.backproject(g, y), rtol=0, atol=1e-12)
    rel = math.sqrt((B - A.T).power(2).sum() / A.power(2).sum())
    # B is a genuinely different discretisation of the same back projection:
    # clearly nonzero, of the size of the ASTRA pairs of Table 2 (0.14-0.37)
    assert 0.05 < rel < 0.4, rel


# ------------------------------------------------------------ solver pins
def _tiny_problem(O, seed=11):
    g = geom(O, N=6, n_angles=8, n_det=9)
    A, B = O.matrix_A(g).toarray(), O.matrix_B(g).toarray()
    x = I.random_ellipses(6, seed, 4)
    b, _ = I.add_noise(A @ x.ravel(), 0.02, seed)
    return g, A, B, b


def _krylov_basis(M, d, k):
    K = np.empty((d.size, k))
    v = d.copy()
    for j in range(k):
        K[:, j] = v
        v = M @ v
    return np.linalg.qr(K)[0]


def test_thresholded_back_projector_against_matrix_free_columns(oracle_mod):
    """Sec. 6.5, eq. (Btau): B_tau keeps the entries of A^T that are at least
    tau max(A).  The explicit form is checked against the columns of A taken
    one by one from the matrix-free forward projector (A e_j), thresholded
    by hand; tau = 0 is A^T itself."""
    O = oracle_mod
    for g in (O.Geometry(9, 7, 13, 0, 180), O.Geometry(8, 6, 12, 30, 120, 0.75)):
        cols = np.stack([O.forward(g, np.eye(g.n)[j]) for j in range(g.n)], axis=1)   # m x n
        amax = cols.max()
        for tau in (0.0, 0.1, 0.5, 0.9):
            ref = np.where(cols >= tau * amax, cols, 0.0).T
            got = O.matrix_B_tau(g, tau).toarray()
            assert np.allclose(got, ref, rtol=0, atol=1e-13), (g, tau)
        assert np.array_equal(O.matrix_B_tau(g, 0.0).toarray(), O.matrix_A(g).toarray().T)


def test_unmatchedness_grows_with_tau(oracle_mod):
    """Table 4's measure ||B_tau - A^T||_F / ||A||_F is 0 at tau = 0 and grows
    with tau; B_tau at tau = 1 keeps only the largest entries."""
    O = oracle_mod
    g = O.Geometry(32, 45, I.detector_count(32), 0, 180)
    A = O.matrix_A(g)
    AT = A.T.tocsr()
    fa = sp.linalg.norm(A)
    meas = [sp.linalg.norm(O.matrix_B_tau(g, t) - AT) / fa for t in (0.0, 0.01, 0.1, 0.3, 0.5)]
    assert meas[0] == 0.0
    assert all(b > a for a, b in zip(meas, meas[1:]))
    B1 = O.matrix_B_tau(g, 1.0)
    assert B1.nnz >= 1 and np.all(B1.data == A.data.max())


def test_ncp_closed_forms(oracle_mod):
    """The NCP reading of Sec. 6.4: an impulse has a flat periodogram, so its
    NCP is the white-noise line exactly; a sinusoid at frequency f puts all
    its power at f, so its NCP is the step 1[i >= f]; the periodogram equals
    the DFT written out as a sum."""
    O = oracle_mod
    for n_det in (10, 11, 64):
        q = n_det // 2
        line = np.arange(1, q + 1) / q
        e0 = np.zeros(n_det)
        e0[3] = 2.5
        assert np.allclose(O.ncp(e0), line, atol=1e-14)
        for f in (1, 2, q - 1):
            r = np.cos(2 * np.pi * f * np.arange(n_det) / n_det + 0.3)
            step = (np.arange(1, q + 1) >= f).astype(float)
            assert np.allclose(O.ncp(r), step, atol=1e-12)
            want = math.sqrt(np.sum((step - line) ** 2))
            assert O.ncp_distance(np.tile(r, 3), 3, n_det) == pytest.approx(want, rel=1e-12)
    rng = np.random.default_rng(4)
    r = rng.standard_normal(11)
    dft = np.array([abs(sum(r[d] * np.exp(-2j * np.pi * i * d / 11) for d in range(11))) ** 2
                    for i in range(1, 6)])
    assert np.allclose(O.ncp(r), np.cumsum(dft) / dft.sum(), atol=1e-13)


def test_ncp_of_white_noise_matches_its_distribution(oracle_mod):
    """For white Gaussian noise the periodogram ordinates are i.i.d.
    exponential, so c_i ~ Beta(i, q - i) and E ||c - i/q||^2 = (q - 1) / (6 q)."""
    O = oracle_mod
    rng = np.random.default_rng(5)
    n_a, n_det = 3000, 129                         # odd: no real Nyquist ordinate
    q = n_det // 2
    R = rng.standard_normal((n_a, n_det))
    line = np.arange(1, q + 1) / q
    d2 = np.mean([np.sum((O.ncp(row) - line) ** 2) for row in R])
    assert d2 == pytest.approx((q - 1) / (6 * q), rel=0.06)
    assert O.first_local_minimum([5, 4, 3, 3.5, 1]) == 2
    assert O.first_local_minimum([5, 4, 3]) == 2
    assert O.first_local_minimum([1, 2]) == 0


def test_ncp_stop_of_gmres(oracle_mod, cfg1_problem):
    """The NCP stop returns the iterate at the first local minimum of the
    NCP distance; on these problems it stops before the discrepancy
    principle, as Sec. 6.4 observes."""
    O = oracle_mod
    og, A, B, xt, b, enorm = cfg1_problem
    for fn in (O.ab_gmres, O.ba_gmres):
        r = fn(A, B, b, 40, ncp_shape=(og.n_angles, og.n_det), keep_iterates=True)
        k = r["k"]
        assert r["stop_reason"] == 3 and k == O.first_local_minimum(r["ncp"])
        assert np.array_equal(r["x"], r["iterates"][k])
        for j in (0, k, k + 1):
            assert r["ncp"][j] == pytest.approx(
                O.ncp_distance(b - A @ r["iterates"][j], og.n_angles, og.n_det), rel=1e-12)
        dp = fn(A, B, b, 40, noise_norm=enorm)
        assert k < dp["k"]


@pytest.mark.parametrize("ortho", ["mgs", "cgs2"])
def test_gmres_matches_brute_force_krylov_minimiser(oracle_mod, ortho):
    """Sec. 2: both methods search x0 + K_k(BA, B r0); AB minimises
    ||b - A x||, BA minimises ||B b - B A x||."""
    O = oracle_mod
    g, A, B, b = _tiny_problem(O)
    x0 = np.random.default_rng(3).uniform(0, 0.1, g.n)
    r0 = b - A @ x0
    M, d = B @ A, B @ r0
    ab = O.ab_gmres(A, B, b, 6, x0=x0, ortho=ortho, keep_iterates=True)
    ba = O.ba_gmres(A, B, b, 6, x0=x0, ortho=ortho, keep_iterates=True)
    for k in range(1, 7):
        Q = _krylov_basis(M, d, k)
        c_ab = np.linalg.lstsq(A @ Q, r0, rcond=None)[0]
        c_ba = np.linalg.lstsq(M @ Q, d, rcond=None)[0]
        x_ab, x_ba = x0 + Q @ c_ab, x0 + Q @ c_ba
        assert np.linalg.norm(ab["iterates"][k] - x_ab) <= 1e-10 * np.linalg.norm(x_ab)
        assert np.linalg.norm(ba["iterates"][k] - x_ba) <= 1e-10 * np.linalg.norm(x_ba)
        assert ab["resnorm"][k] == pytest.approx(np.linalg.norm(b - A @ x_ab), rel=1e-10)


@pytest.fixture(scope="module")
def cfg1_problem(oracle_mod):
    O = oracle_mod
    g = geom(O, **CFG1)
    A, B = O.matrix_A(g), O.matrix_B(g)
    xt = I.shepp_logan(64).ravel()
    b, enorm = I.add_noise(A @ xt, 0.01, 1000)
    return g, A, B, xt, b, enorm


def test_matched_case_ab_equals_lsqr_and_ba_equals_lsmr(oracle_mod, cfg1_problem):
    """Sec. 5: with B = A^T and x0 = 0, AB-GMRES iterates equal LSQR's and
    BA-GMRES iterates equal LSMR's.  LSQR/LSMR use full reorthogonalisation.

    Past k ~ 15 the iterates of the ill-posed CT problem are ill-conditioned
    functions of the rounding (two FP64 orderings of one method differ by up
    to ~1e-4 around k = 25), so the CT operator pins k <= 12 and a
    well-conditioned random operator pins every k up to the full dimension."""
    O = oracle_mod
    g, A, _, _, b, _ = cfg1_problem
    K = 12
    ab = O.ab_gmres(A, A.T, b, K, keep_iterates=True)
    ba = O.ba_gmres(A, A.T, b, K, keep_iterates=True)
    xq, xm = O.lsqr(A, b, K), O.lsmr(A, b, K)
    for k in range(1, K + 1):
        for got, ref in ((ab["iterates"][k], xq[k - 1]), (ba["iterates"][k], xm[k - 1])):
            assert np.linalg.norm(got - ref) <= 1e-10 * np.linalg.norm(ref), k
    rng = np.random.default_rng(21)
    # square and well conditioned, so that AA^T and A^TA are both nonsingular
    Ar = rng.standard_normal((40, 40)) + 8.0 * np.eye(40)
    br = rng.standard_normal(40)
    K = 40
    ab = O.ab_gmres(Ar, Ar.T, br, K, keep_iterates=True)
    ba = O.ba_gmres(Ar, Ar.T, br, K, keep_iterates=True)
    xq, xm = O.lsqr(Ar, br, K), O.lsmr(Ar, br, K)
    for k in range(1, K + 1):
        for got, ref in ((ab["iterates"][k], xq[k - 1]), (ba["iterates"][k], xm[k - 1])):
            assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref), k
    xls = np.linalg.solve(Ar, br)                # k = n: the exact solution
    assert np.linalg.norm(ab["x"] - xls) <= 1e-9 * np.linalg.norm(xls)
    assert np.linalg.norm(ba["x"] - xls) <= 1e-9 * np.linalg.norm(xls)


def test_lsqr_lsmr_against_scipy(oracle_mod, cfg1_problem):
    """Independent library cross-check (scipy: no reorthogonalisation)."""
    O = oracle_mod
    _, A, _, _, b, _ = cfg1_problem
    xq, xm = O.lsqr(A, b, 10), O.lsmr(A, b, 10)
    for k in (1, 2, 5, 10):
        sq = sla.lsqr(A, b, atol=0, btol=0, conlim=0, iter_lim=k)[0]
        sm = sla.lsmr(A, b, atol=0, btol=0, conlim=0, maxiter=k)[0]
        assert np.linalg.norm(xq[k - 1] - sq) <= 1e-6 * np.linalg.norm(sq)
        assert np.linalg.norm(xm[k - 1] - sm) <= 1e-6 * np.linalg.norm(sm)


@pytest.mark.parametrize("ortho,orth_tol", [("mgs", 1e-10), ("cgs2", 1e-13)])
@pytest.mark.parametrize("variant", ["ab", "ba"])
def test_arnoldi_invariants(oracle_mod, cfg1_problem, variant, ortho, orth_tol):
    """Algorithm box of Sec. 2: M W_k = W_{k+1} H_k with M = AB (or BA),
    W orthonormal, GMRES residual non-increasing; for AB the Hessenberg
    residual equals the true residual ||b - A x_k||.  MGS loses
    orthogonality in proportion to the Krylov condition number; CGS2 keeps
    it at the rounding level."""
    O = oracle_mod
    _, A, B, _, b, _ = cfg1_problem
    K = 30
    r = (O.ab_gmres if variant == "ab" else O.ba_gmres)(A, B, b, K, ortho=ortho)
    W, H = r["W"], r["H"]
    M = (lambda v: A @ (B @ v)) if variant == "ab" else (lambda v: B @ (A @ v))
    MW = np.stack([M(W[j]) for j in range(K)], axis=1)
    assert np.linalg.norm(MW - W.T @ H) <= 1e-12 * np.linalg.norm(H)
    assert np.abs(W @ W.T - np.eye(K + 1)).max() <= orth_tol
    rho = np.array(r["rho"])
    assert np.all(np.diff(rho) <= 1e-12 * rho[0])
    if variant == "ab":
        np.testing.assert_allclose(rho, r["resnorm"], rtol=1e-10)


def test_discrepancy_principle(oracle_mod, cfg1_problem):
    """Sec. 6.4: k_DP is the smallest k with ||b - A x_k|| <= tau ||e||."""
    O = oracle_mod
    _, A, B, xt, b, enorm = cfg1_problem
    full = O.ab_gmres(A, B, b, 50)
    stop = O.ab_gmres(A, B, b, 50, tau=1.02, noise_norm=enorm)
    res = np.array(full["resnorm"])
    k_dp = int(np.argmax(res <= 1.02 * enorm))
    assert res[k_dp] <= 1.02 * enorm and stop["k"] == k_dp
    assert stop["stop_reason"] == 1 and 0 < k_dp < 50
    # x0 already below the bound: k = 0 and x0 itself is returned
    x0 = xt.copy()
    r0 = O.ab_gmres(A, B, A @ xt, 10, x0=x0, noise_norm=1e-3)
    assert r0["k"] == 0 and np.array_equal(r0["x"], x0)
    # no k satisfies the bound: x_maxit is returned
    rm = O.ba_gmres(A, B, b, 5, noise_norm=1e-6)
    assert rm["k"] == 5 and rm["stop_reason"] == 0
    # semi-convergence (Sec. 4): at the paper's higher noise level 0.03 the
    # error history has an interior minimum, and DP stops before it
    b3, e3 = I.add_noise(A @ xt, 0.03, 1000)
    it = O.ab_gmres(A, B, b3, 60, keep_iterates=True)["iterates"]
    err = [np.linalg.norm(x - xt) for x in it]
    k_min = int(np.argmin(err))
    assert 0 < k_min < 60 and err[-1] > 1.2 * err[k_min]
    assert O.ab_gmres(A, B, b3, 60, noise_norm=e3)["k"] <= k_min


def test_breakdown_returns_exact_solution(oracle_mod):
    """With A = B = I, AB = I: the Krylov space is exhausted at k = 1 and
    the square Hessenberg system gives the exact solution."""
    O = oracle_mod
    b = np.random.default_rng(9).standard_normal(7)
    for solver in (O.ab_gmres, O.ba_gmres):
        r = solver(np.eye(7), np.eye(7), b, 5)
        assert r["k"] == 1 and r["stop_reason"] == 2
        np.testing.assert_allclose(r["x"], b, rtol=1e-14)



@pytest.mark.parametrize("N,Na", [(4, 8), (6, 10), (5, 7)])
def test_breakdown_of_a_singular_ab_reaches_the_least_squares_minimum(oracle_mod, N, Na):
    """On a tiny geometry (n = N^2 < m) A B is m x m of rank n, so the Krylov
    space K_k(A B, b) is exhausted after about n + 1 steps and the run ends in
    a breakdown with a singular square H_k.  The returned iterate must still
    attain min_z ||b - A B z|| (Sec. 2: AB-GMRES minimises ||b - A B u|| over
    the Krylov space, which at exhaustion holds the minimiser), computed
    here from the explicit matrices by a library least-squares solve; the
    residual history is non-increasing up to rounding (GMRES minimises over
    nested spaces).  BA-GMRES on the square nonsingular B A of the same
    geometry ends in a breakdown at the exact minimiser of ||B b - B A x||."""
    O = oracle_mod
    og = O.Geometry(N, Na, I.detector_count(N))
    n = N * N
    m = Na * og.n_det
    A = np.stack([O.forward(og, e) for e in np.eye(n)], 1)
    B = np.stack([O.backproject(og, e) for e in np.eye(m)], 1)
    assert np.linalg.matrix_rank(A @ B) == n < m
    b = A @ I.random_ellipses(N, 11).ravel() + 0.01 * np.random.default_rng(1).standard_normal(m)
    r = O.ab_gmres(A, B, b, 4 * n)
    assert r["stop_reason"] == 2 and n <= r["k"] <= n + 3
    z = np.linalg.lstsq(A @ B, b, rcond=None)[0]
    best = np.linalg.norm(b - A @ (B @ z))
    assert np.linalg.norm(b - A @ r["x"]) == pytest.approx(best, rel=1e-9)
    res = np.array(r["resnorm"])
    assert np.all(np.diff(res) <= 1e-9 * res[0])
    rb = O.ba_gmres(A, B, b, 4 * n)
    assert rb["stop_reason"] == 2 and rb["k"] <= n + 3
    xb = np.linalg.solve(B @ A, B @ b)
    np.testing.assert_allclose(rb["x"], xb, rtol=1e-8 * np.linalg.cond(B @ A), atol=0)

# ------------------------------------------------------------ input pins
def test_shepp_logan_and_noise_generators():
    x = I.shepp_logan(128)
    assert x.min() >= 0.0 and x.max() == pytest.approx(1.0)
    assert len(I._MODIFIED_SHEPP_LOGAN) == 10
    vals = np.unique(np.round(x, 12))
    assert set(vals) <= {0.0, 0.1, 0.2, 0.3, 0.4, 1.0}
    e = I.random_ellipses(64, 7)
    assert 0.0 <= e.min() and e.max() <= 1.0 and (e > 0).mean() > 0.1
    assert np.array_equal(e, I.random_ellipses(64, 7))
    bb = np.random.default_rng(0).uniform(size=500)
    b, en = I.add_noise(bb, 0.03, 5)
    assert en == pytest.approx(0.03 * np.linalg.norm(bb), rel=1e-14)
    assert np.linalg.norm(b - bb) == pytest.approx(en, rel=1e-14)
    assert I.detector_count(512) == 725 and I.detector_count(2048) == 2897
    assert I.detector_count(64) == 91
