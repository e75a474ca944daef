"""Batched AB-/BA-GMRES (ctg_batch_*): solves of different sizes, variants,
angle ranges and budgets advance together, one Arnoldi step per round, with
the Givens update and the stopping rule on the device.

Checked: every solve of a mixed batch agrees with the single-solve path
(same stop, iterate within 1e-4 at the discrepancy stop, which falls in the
well-conditioned range of these problems); a solve's result is the same,
bit for bit, alone and in the mix; oracle parity at the discrepancy stop;
the k = 0 stops and b = 0 inside a batch.
"""
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


def _case(O, N, Na, rng_deg, eta, seed):
    og = O.Geometry(N, Na, I.detector_count(N), 0, rng_deg)
    xt = I.random_ellipses(N, seed)
    b, enorm = I.add_noise(O.forward(og, xt), eta, seed)
    return og, xt.ravel(), b.astype(np.float32), enorm


MIX = [  # N, angles, range, noise, variant, maxit, use DP
    (64, 60, 180, 0.01, "ab", 40, True),
    (128, 180, 180, 0.02, "ba", 40, True),
    (96, 90, 120, 0.03, "ab", 30, True),
    (64, 45, 180, 0.01, "ba", 12, False),
    (160, 90, 180, 0.005, "ab", 25, False),
    (128, 120, 120, 0.015, "ba", 40, True),
]


def _problems(P, O):
    cases, probs = [], []
    for i, (N, Na, R, eta, v, maxit, dp) in enumerate(MIX):
        og, xt, b, enorm = _case(O, N, Na, R, eta, 3000 + i)
        cases.append((og, xt, b, enorm))
        probs.append({"geometry": P.Geometry(N, Na, og.n_det, 0, R), "variant": v,
                      "maxit": maxit, "tau": 1.02, "noise_norm": enorm if dp else None})
    return cases, probs


def test_batch_matches_single_solves(P, oracle_mod):
    import torch
    cases, probs = _problems(P, oracle_mod)
    bs = [torch.tensor(c[2], device="cuda") for c in cases]
    batch = P.Batch(probs)
    res = batch.solve(bs)
    torch.cuda.synchronize()
    for (og, xt, b, enorm), p, r, bt in zip(cases, probs, res, bs):
        fn = P.ab_gmres if p["variant"] == "ab" else P.ba_gmres
        ref = fn(p["geometry"], bt, p["maxit"], tau=1.02, noise_norm=p["noise_norm"])
        torch.cuda.synchronize()
        assert r.stop_reason == ref.stop_reason
        assert abs(r.iters - ref.iters) <= (1 if p["noise_norm"] else 0)
        if r.iters == ref.iters:
            d = (r.x - ref.x).double().norm() / ref.x.double().norm()
            # no-DP runs to a fixed k are compared where the iterate is well
            # conditioned (k <= 25 here); DP stops fall there too
            assert d.item() <= 1e-4, (p, d.item())
        assert r.resnorm == pytest.approx(ref.resnorm, rel=1e-3)
        if p["noise_norm"]:
            assert r.resnorm <= 1.02 * enorm * (1 + 1e-5)


def test_batch_result_is_independent_of_the_mix(P, oracle_mod):
    import torch
    cases, probs = _problems(P, oracle_mod)
    bs = [torch.tensor(c[2], device="cuda") for c in cases]
    mixed = P.Batch(probs).solve(bs)
    for i in (1, 4):
        alone = P.Batch([probs[i]]).solve([bs[i]])[0]
        torch.cuda.synchronize()
        assert alone.iters == mixed[i].iters
        assert torch.equal(alone.x, mixed[i].x)


def test_batch_discrepancy_stop_matches_oracle(P, oracle_mod):
    import torch
    O = oracle_mod
    cases, probs = _problems(P, O)
    sel = [0, 1]
    batch = P.Batch([probs[i] for i in sel])
    res = batch.solve([torch.tensor(cases[i][2], device="cuda") for i in sel])
    for i, r in zip(sel, res):
        og, xt, b, enorm = cases[i]
        A = lambda v: O.forward(og, v)
        B = lambda v: O.backproject(og, v)
        solver = O.ab_gmres if probs[i]["variant"] == "ab" else O.ba_gmres
        ref = solver(A, B, b.astype(np.float64), probs[i]["maxit"], tau=1.02, noise_norm=enorm)
        assert r.stop_reason == 1 and ref["stop_reason"] == 1
        if r.iters == ref["k"]:
            x = r.x.double().cpu().numpy()
            assert np.linalg.norm(x - ref["x"]) <= 1e-4 * np.linalg.norm(ref["x"])
        else:
            assert abs(r.iters - ref["k"]) == 1


def test_batch_zero_iteration_stops(P, oracle_mod):
    import torch
    O = oracle_mod
    og, xt, b, enorm = _case(O, 48, 40, 180, 0.01, 3100)
    g = P.Geometry(48, 40, og.n_det)
    x0 = torch.tensor(xt, dtype=torch.float32, device="cuda")
    bb = P.project(g, x0)
    probs = [{"geometry": g, "variant": "ab", "maxit": 5, "noise_norm": 1e-3},
             {"geometry": g, "variant": "ba", "maxit": 5},
             {"geometry": g, "variant": "ba", "maxit": 60, "tau": 1.02, "noise_norm": enorm}]
    res = P.Batch(probs).solve([bb, torch.zeros_like(bb), torch.tensor(b, device="cuda")],
                               x0s=[x0, None, None])
    torch.cuda.synchronize()
    assert res[0].iters == 0 and res[0].stop_reason == 1 and torch.equal(res[0].x, x0)
    assert res[1].iters == 0 and res[1].stop_reason == 2 and torch.count_nonzero(res[1].x) == 0
    assert res[2].iters > 0 and res[2].stop_reason == 1


def test_batch_with_matched_and_thresholded_back_projectors(P, oracle_mod):
    """Sec. 6.5's sweep as one batch: the same problem with B = A^T and B_tau
    for several tau, in AB and BA form, each solve equal to its single-solve
    run (stop and iterate) and, bit for bit, to itself run alone."""
    import torch
    O = oracle_mod
    og, xt, b, enorm = _case(O, 96, 120, 180, 0.01, 3200)
    bt = torch.tensor(b, device="cuda")
    probs = []
    for model, tb in (("pixel", 0.0), ("matched", 0.0), ("threshold", 0.1), ("threshold", 0.5)):
        g = P.Geometry(96, 120, og.n_det, 0, 180, 1.0, model, tb)
        for v in ("ab", "ba"):
            probs.append({"geometry": g, "variant": v, "maxit": 40, "tau": 1.02, "noise_norm": enorm})
    res = P.Batch(probs).solve([bt] * len(probs))
    torch.cuda.synchronize()
    for p, r in zip(probs, res):
        fn = P.ab_gmres if p["variant"] == "ab" else P.ba_gmres
        ref = fn(p["geometry"], bt, 40, tau=1.02, noise_norm=enorm)
        assert r.stop_reason == ref.stop_reason
        assert abs(r.iters - ref.iters) <= (1 if r.stop_reason == 1 else 0)
        if r.iters == ref.iters:
            d = (r.x - ref.x).double().norm() / ref.x.double().norm()
            assert d.item() <= 1e-4, (p["geometry"].back_model, p["variant"], d.item())
    for i in (3, 6):
        alone = P.Batch([probs[i]]).solve([bt])[0]
        assert alone.iters == res[i].iters and torch.equal(alone.x, res[i].x)
    # an engine serving the sweep gives the results of the batch: the same
    # stop, and the iterate to the rounding of the CGS2 sums (the engine,
    # whose solves are at different steps, takes the separate passes; the
    # batch takes the one-launch step up to k = 64)
    eng = P.Engine(4, 1 << 34)
    pending, got = list(range(len(probs))), {}
    while pending or eng.in_flight:
        while pending and eng.submit(probs[pending[0]]["geometry"], bt, probs[pending[0]]["variant"], 40,
                                     tau=1.02, noise_norm=enorm, tag=pending[0]) is not None:
            pending.pop(0)
        got.update(dict(eng.step(3)))
    for i, r in enumerate(res):
        assert got[i].iters == r.iters and got[i].stop_reason == r.stop_reason
        d = (got[i].x - r.x).double().norm() / r.x.double().norm()
        assert d.item() <= 1e-5, (i, d.item())


def test_batch_with_16bit_bases(P, oracle_mod):
    """Solves with FP32, BF16 and FP16 bases in one batch (AB and BA).  Each
    equals itself run alone bit for bit; against the single-solve path with
    the same basis type (another reduction order, so a 16-bit rounding may
    fall the other way) the iterate at a fixed early k is within a few
    storage unit roundoffs and the discrepancy stop within two steps at the
    same error; a 16-bit basis about halves the batch's memory."""
    import torch
    O = oracle_mod
    og, xt, b, enorm = _case(O, 96, 120, 180, 0.01, 3300)
    bt = torch.tensor(b, device="cuda")
    g = P.Geometry(96, 120, og.n_det)
    unit = {"fp32": 2.0 ** -24, "bf16": 2.0 ** -8, "fp16": 2.0 ** -11}
    probs = [{"geometry": g, "variant": v, "maxit": 6, "basis": t}
             for t in ("fp32", "bf16", "fp16") for v in ("ab", "ba")]
    res = P.Batch(probs).solve([bt] * len(probs))
    torch.cuda.synchronize()
    for p, r in zip(probs, res):
        fn = P.ab_gmres if p["variant"] == "ab" else P.ba_gmres
        ref = fn(g, bt, 6, basis=p["basis"])
        assert r.iters == ref.iters == 6
        d = ((r.x - ref.x).double().norm() / ref.x.double().norm()).item()
        assert d <= max(1e-4, 10 * unit[p["basis"]]), (p["variant"], p["basis"], d)
    for i in (2, 5):
        alone = P.Batch([probs[i]]).solve([bt])[0]
        assert torch.equal(alone.x, res[i].x)
    # discrepancy stops (AB with either 16-bit type, BA with FP16: the cases
    # whose stop the 16-bit basis keeps, see the precision tests)
    xt_t = torch.tensor(xt, device="cuda", dtype=torch.float64)
    dp = [{"geometry": g, "variant": v, "maxit": 60, "basis": t, "tau": 1.02, "noise_norm": enorm}
          for v, t in (("ab", "bf16"), ("ab", "fp16"), ("ba", "fp16"))]
    got = P.Batch(dp).solve([bt] * len(dp))
    for p, r in zip(dp, got):
        fn = P.ab_gmres if p["variant"] == "ab" else P.ba_gmres
        ref = fn(g, bt, 60, tau=1.02, noise_norm=enorm, basis=p["basis"])
        assert r.stop_reason == ref.stop_reason == 1 and abs(r.iters - ref.iters) <= 2
        e_b = ((r.x.double() - xt_t).norm() / xt_t.norm()).item()
        e_s = ((ref.x.double() - xt_t).norm() / xt_t.norm()).item()
        assert abs(e_b - e_s) <= 0.08 * e_s
    w32 = P.Batch([dict(probs[0], maxit=60)]).workspace_bytes
    w16 = P.Batch([dict(probs[2], maxit=60)]).workspace_bytes
    assert w16 < 0.6 * w32


def test_batch_crosses_from_fused_steps_to_separate_passes(P, oracle_mod):
    """Steps k <= 64 of a batch run the one-launch CGS2 step with each
    solve's Givens update in it (the first while loop of the batch graph),
    later steps the separate passes and Givens launch (the second loop).  Run
    to maxit = 80 without a discrepancy stop, each solve's residual history
    agrees with the single-solve path across the switch."""
    import torch
    specs = [(64, 60, "ab", 3101), (64, 60, "ba", 3102)]
    cases, probs = [], []
    for N, Na, v, seed in specs:
        og, xt, b, enorm = _case(oracle_mod, N, Na, 180, 0.01, seed)
        cases.append(b)
        probs.append({"geometry": P.Geometry(N, Na, og.n_det), "variant": v, "maxit": 80, "tau": 1.02,
                      "noise_norm": None})
    bs = [torch.tensor(b, device="cuda") for b in cases]
    res = P.Batch(probs).solve(bs)
    torch.cuda.synchronize()
    for p, r, bt in zip(probs, res, bs):
        fn = P.ab_gmres if p["variant"] == "ab" else P.ba_gmres
        ref = fn(p["geometry"], bt, 80)
        torch.cuda.synchronize()
        assert r.iters == ref.iters == 80 and r.stop_reason == ref.stop_reason == 0
        h, hr = np.array(r.history), np.array(ref.history)
        assert len(h) == len(hr) == 81
        assert np.all(np.abs(h - hr) <= 1e-3 * hr[0]), (p["variant"], np.abs(h - hr).max() / hr[0])
        assert r.rho == pytest.approx(ref.rho, rel=1e-2, abs=1e-3 * hr[0])


def test_batch_fused_step_timeout_is_reported_and_recoverable(P, oracle_mod):
    """With every bounded wait limited to one poll, the batch's one-launch
    CGS2 step (an AB and a BA solve at 512^2, 720 angles: 192 blocks) cannot
    see all blocks arrive at its first grid barrier: the solve raises
    CTG_ERR_TIMEOUT, nothing waits for ever, and with the default limit the
    same batch solves exactly as a fresh one."""
    import torch
    from paper_2110_01481_gb300 import _native as nat
    cases, probs = [], []
    for v, seed in (("ab", 3201), ("ba", 3202)):
        og, xt, b, enorm = _case(oracle_mod, 512, 720, 180, 0.01, seed)
        cases.append(b)
        probs.append({"geometry": P.Geometry(512, 720, og.n_det), "variant": v, "maxit": 30, "tau": 1.02,
                      "noise_norm": enorm})
    bs = [torch.tensor(b, device="cuda") for b in cases]
    batch = P.Batch(probs)
    try:
        batch.ctx.set_wait_limit(1)
        with pytest.raises(nat.CtgError) as ei:
            batch.solve(bs)
        assert ei.value.status == nat.CTG_ERR_TIMEOUT
    finally:
        batch.ctx.set_wait_limit(0)
    again = batch.solve(bs)
    fresh = P.Batch(probs).solve(bs)
    torch.cuda.synchronize()
    for a, f in zip(again, fresh):
        assert a.iters == f.iters and a.stop_reason == f.stop_reason == 1
        assert torch.equal(a.x, f.x)


def test_batch_autotuned_shapes_are_result_invariant(P, oracle_mod):
    """The batched autotuner picks, by timing, the forward launches' shape
    (four angles per warp or one) and the back projection's staging chunk
    (16, 32 or 64 angles per pass).  Forcing each choice on the context gives
    the same solves bit for bit: the tuner changes the speed only."""
    import torch
    cases, probs = [], []
    for N, Na, v, seed in ((256, 360, "ab", 3301), (256, 360, "ba", 3302), (128, 180, "ba", 3303)):
        og, xt, b, enorm = _case(oracle_mod, N, Na, 180, 0.01, seed)
        cases.append(b)
        probs.append({"geometry": P.Geometry(N, Na, og.n_det), "variant": v, "maxit": 40, "tau": 1.02,
                      "noise_norm": enorm})
    bs = [torch.tensor(b, device="cuda") for b in cases]
    ctx = P.Context.get(bs[0].device)
    ref = P.Batch(probs).solve(bs)
    torch.cuda.synchronize()
    try:
        for angles, per_warp in ((8, 1), (16, 4)):
            for chunk in (16, 32, 64):
                ctx.set_tiles(angles, chunk, per_warp)
                res = P.Batch(probs).solve(bs)
                torch.cuda.synchronize()
                for a, r in zip(res, ref):
                    assert a.iters == r.iters and a.stop_reason == r.stop_reason
                    assert torch.equal(a.x, r.x), (angles, per_warp, chunk)
    finally:
        ctx.set_tiles(0, 0)


def test_batch_created_after_other_work_sees_its_tables(P, oracle_mod):
    """A batch created while the device has just been busy (here a single
    solve) must upload its angle tables after, not before, the zeroing of
    its workspace (both ordered on the batch's own stream).  At 2048^2 the
    zeroing takes long enough that a legacy-stream memset raced the table
    uploads and left the forward table zero (t_1 = 0, a breakdown at k = 1)."""
    import torch
    og, xt, b, enorm = _case(oracle_mod, 2048, 180, 180, 0.01, 3401)
    p = {"geometry": P.Geometry(2048, 180, og.n_det), "variant": "ba", "maxit": 30, "tau": 1.02,
         "noise_norm": enorm}
    bt = torch.tensor(b, device="cuda")
    ref = P.ba_gmres(p["geometry"], bt, 30, tau=1.02, noise_norm=enorm)
    for _ in range(2):
        r = P.Batch([p]).solve([bt])[0]
        torch.cuda.synchronize()
        assert r.stop_reason == ref.stop_reason == 1 and abs(r.iters - ref.iters) <= 1
        if r.iters == ref.iters:
            d = (r.x - ref.x).double().norm() / ref.x.double().norm()
            assert d.item() <= 1e-4
        P.ba_gmres(p["geometry"], bt, 30, tau=1.02, noise_norm=enorm)     # busy the device again
