"""Oracle parity on the benchmark workload itself.

The benchmark solves a 512 x 512 random-ellipse phantom (20 ellipses, seed
2000) from 720 angles over [0, 180) and 725 detector bins, with 1% white
Gaussian noise (same seed), AB-GMRES and BA-GMRES up to 150 iterations,
stopped by the discrepancy principle of Sec. 6.4 with tau = 1.02.  Here the
same instance is built with the oracle's FP64 forward projector (b_bar =
A x_bar, the inverse crime of Sec. 1), and the CUDA path must give, for
both methods (Sec. 2 algorithm box):

  * x_k within 1e-4 of the oracle's x_k (relative 2-norm) at EVERY
    k = 1 .. k_stop;
  * the oracle's discrepancy-principle stop index, or one step off only when
    the residual there lies within 1e-4 of tau ||e||;
  * at the stop, the returned x within 1e-4 of the oracle's, and the
    returned resnorm equal to ||b - A x|| of the returned x, recomputed by
    the oracle in FP64, to 1e-5;
  * the same from one batched solve (ctg_batch_solve) of the instance's AB
    and BA problems together.
"""
import numpy as np
import pytest

from paper_2110_01481_gb300 import inputs as I

pytestmark = pytest.mark.gpu

N, N_ANG, SEED, ETA, TAU, MAXIT = 512, 720, 2000, 0.01, 1.02, 150
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


@pytest.fixture(scope="module")
def workload(oracle_mod):
    O = oracle_mod
    og = O.Geometry(N, N_ANG, I.detector_count(N))
    xt = I.random_ellipses(N, SEED)
    b, enorm = I.add_noise(O.forward(og, xt), ETA, SEED)
    b = b.astype(np.float32).astype(np.float64)          # the GPU sees FP32 data
    return og, b, enorm


@pytest.fixture(scope="module")
def oracle_runs(oracle_mod, workload):
    O = oracle_mod
    og, b, enorm = workload
    A = lambda v: O.forward(og, v)
    B = lambda v: O.backproject(og, v)
    return {v: (O.ab_gmres if v == "ab" else O.ba_gmres)(A, B, b, MAXIT, tau=TAU, noise_norm=enorm,
                                                          keep_iterates=True)
            for v in ("ab", "ba")}


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _check_stop(O, og, b, enorm, ref, iters, stop_reason, x, resnorm):
    target = TAU * enorm
    assert ref["stop_reason"] == 1 and stop_reason == 1
    if iters != ref["k"]:
        assert abs(iters - ref["k"]) == 1
        kk = min(iters, ref["k"])
        assert abs(ref["resnorm"][kk] - target) < 1e-4 * target
    else:
        assert _rel(x, ref["x"]) <= X_TOL
    assert resnorm <= target * (1 + 1e-5)
    assert resnorm == pytest.approx(np.linalg.norm(b - O.forward(og, x)), rel=1e-5)


@pytest.mark.parametrize("variant", ["ab", "ba"])
def test_every_iterate_up_to_the_stop(P, oracle_mod, workload, oracle_runs, variant):
    import torch
    og, b, enorm = workload
    ref = oracle_runs[variant]
    g = P.Geometry(N, N_ANG, og.n_det)
    bt = torch.tensor(b, dtype=torch.float32, device="cuda")
    fn = P.ab_gmres if variant == "ab" else P.ba_gmres
    assert ref["k"] >= 8                     # the solves run past the first few steps
    for k in range(1, ref["k"] + 1):
        r = fn(g, bt, k)
        torch.cuda.synchronize()
        assert r.iters == k and r.stop_reason == 0
        assert _rel(r.x.double().cpu().numpy(), ref["iterates"][k]) <= X_TOL, k


@pytest.mark.parametrize("variant", ["ab", "ba"])
def test_discrepancy_stop_and_returned_result(P, oracle_mod, workload, oracle_runs, variant):
    import torch
    og, b, enorm = workload
    g = P.Geometry(N, N_ANG, og.n_det)
    bt = torch.tensor(b, dtype=torch.float32, device="cuda")
    fn = P.ab_gmres if variant == "ab" else P.ba_gmres
    r = fn(g, bt, MAXIT, tau=TAU, noise_norm=enorm)
    torch.cuda.synchronize()
    _check_stop(oracle_mod, og, b, enorm, oracle_runs[variant], r.iters, r.stop_reason,
                r.x.double().cpu().numpy(), r.resnorm)


def test_batched_solve_of_the_workload(P, oracle_mod, workload, oracle_runs):
    import torch
    og, b, enorm = workload
    g = P.Geometry(N, N_ANG, og.n_det)
    bt = torch.tensor(b, dtype=torch.float32, device="cuda")
    probs = [{"geometry": g, "variant": v, "maxit": MAXIT, "tau": TAU, "noise_norm": enorm}
             for v in ("ab", "ba")]
    res = P.Batch(probs).solve([bt, bt])
    torch.cuda.synchronize()
    for v, r in zip(("ab", "ba"), res):
        _check_stop(oracle_mod, og, b, enorm, oracle_runs[v], r.iters, r.stop_reason,
                    r.x.double().cpu().numpy(), r.resnorm)
