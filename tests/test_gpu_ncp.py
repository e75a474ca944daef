"""The NCP stopping criterion of Sec. 6.4 on the GPU against the oracle.

Checked: the NCP distance of residual sinograms (even and odd detector
counts, the 2048^2 workload's 2897 bins, the 8192-bin limit) element for
element against the oracle, and its closed forms (an impulse is white, a
sinusoid is a step); AB-GMRES / BA-GMRES with the NCP stop return the
oracle's stopping index and iterate, with the NCP distance history matching
the oracle's.
"""
import math

import numpy as np
import pytest

from paper_2110_01481_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2110_01481_gb300 as P
    return P


def _t(a):
    import torch
    return torch.tensor(np.asarray(a), dtype=torch.float32, device="cuda")


@pytest.mark.parametrize("Na,Nd", [(90, 91), (60, 64), (7, 2897), (3, 8192), (5, 2), (200, 3)])
def test_ncp_distance_matches_oracle(P, oracle_mod, Na, Nd):
    g = P.Geometry(64, Na, Nd)
    rng = np.random.default_rng(Na * Nd)
    # white noise plus a smooth component: a residual between the extremes
    d = np.arange(Nd)
    R = rng.standard_normal((Na, Nd)) + 3.0 * np.exp(-((d - Nd / 3) / (0.1 * Nd + 1)) ** 2)
    r = R.astype(np.float32).ravel()
    want = oracle_mod.ncp_distance(r.astype(np.float64), Na, Nd)
    got = P.ncp_distance(g, _t(r))
    assert got == pytest.approx(want, rel=1e-4, abs=1e-6)


def test_ncp_distance_closed_forms(P, oracle_mod):
    Na, Nd = 4, 100
    g = P.Geometry(64, Na, Nd)
    q = Nd // 2
    line = np.arange(1, q + 1) / q
    imp = np.zeros((Na, Nd))
    imp[:, 17] = 1.5
    assert P.ncp_distance(g, _t(imp.ravel())) == pytest.approx(0.0, abs=1e-5)
    for f in (1, 9, q - 1):
        r = np.tile(np.cos(2 * np.pi * f * np.arange(Nd) / Nd + 0.4), Na)
        step = (np.arange(1, q + 1) >= f).astype(float)
        want = math.sqrt(np.sum((step - line) ** 2))
        assert P.ncp_distance(g, _t(r)) == pytest.approx(want, rel=1e-4, abs=1e-5)
    assert P.ncp_distance(g, _t(np.zeros(Na * Nd))) == 0.0


def _problem(O, N, Na, eta, seed):
    og = O.Geometry(N, Na, I.detector_count(N))
    xt = I.random_ellipses(N, seed)
    b, enorm = I.add_noise(O.forward(og, xt), eta, seed)
    return og, xt.ravel(), b.astype(np.float32).astype(np.float64), enorm


@pytest.mark.parametrize("variant", ["ab", "ba"])
@pytest.mark.parametrize("N,Na,eta,seed", [(64, 90, 0.01, 6100), (128, 180, 0.01, 6200),
                                           (96, 120, 0.003, 6300)])
def test_ncp_stop_matches_oracle(P, oracle_mod, variant, N, Na, eta, seed):
    O = oracle_mod
    og, xt, b, enorm = _problem(O, N, Na, eta, seed)
    A = lambda v: O.forward(og, v)
    B = lambda v: O.backproject(og, v)
    ref = (O.ab_gmres if variant == "ab" else O.ba_gmres)(
        A, B, b, 60, ncp_shape=(og.n_angles, og.n_det))
    assert ref["stop_reason"] == 3
    g = P.Geometry(N, Na, og.n_det)
    fn = P.ab_gmres if variant == "ab" else P.ba_gmres
    got = fn(g, _t(b), 60, stop="ncp")
    assert got.stop_reason == 3
    k = got.iters
    assert len(got.ncp_history) == k + 2
    assert np.allclose(got.ncp_history, ref["ncp"][: k + 2], rtol=1e-3)
    assert k == ref["k"]
    x = got.x.double().cpu().numpy()
    assert np.linalg.norm(x - ref["x"]) <= 1e-4 * np.linalg.norm(ref["x"])
    assert got.resnorm == pytest.approx(ref["resnorm"][k], rel=1e-4)
    # as Sec. 6.4 observes, NCP stops before the discrepancy principle
    dp = fn(g, _t(b), 60, tau=1.0, noise_norm=enorm)
    assert k < dp.iters


def test_ncp_stop_with_a_start_vector(P, oracle_mod):
    O = oracle_mod
    og, xt, b, enorm = _problem(O, 64, 90, 0.01, 6400)
    x0 = 0.3 * xt
    A = lambda v: O.forward(og, v)
    B = lambda v: O.backproject(og, v)
    g = P.Geometry(64, 90, og.n_det)
    for variant, fn, gfn in (("ab", O.ab_gmres, P.ab_gmres), ("ba", O.ba_gmres, P.ba_gmres)):
        ref = fn(A, B, b, 60, x0=x0, ncp_shape=(og.n_angles, og.n_det))
        got = gfn(g, _t(b), 60, x0=_t(x0), stop="ncp")
        assert got.iters == ref["k"], variant
        x = got.x.double().cpu().numpy()
        assert np.linalg.norm(x - ref["x"]) <= 1e-4 * np.linalg.norm(ref["x"])
