"""Serving engine (ctg_engine_*): continuous batching of independent solves.

Checked: a solve's result is the same, bit for bit, whether it runs alone or
joins a stream of other solves at any round (slots reused by solves of other
sizes, the round graph re-captured as membership changes); the discrepancy
stop agrees with the single-solve path; admission refuses a request when no
slot is free or its workspace does not fit the remaining memory budget, and
rejects one that can never fit; k = 0 stops are reported with x = x0.
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


STREAM = [  # N, angles, range, noise, variant, maxit, use DP
    (64, 60, 180, 0.01, "ab", 40, True),
    (128, 180, 180, 0.02, "ba", 40, True),
    (96, 90, 120, 0.03, "ab", 30, True),
    (64, 45, 180, 0.01, "ba", 12, False),
    (160, 90, 180, 0.005, "ab", 25, False),
    (128, 120, 120, 0.015, "ba", 40, True),
    (80, 72, 180, 0.02, "ba", 30, True),
    (112, 100, 150, 0.01, "ab", 35, True),
]


def _requests(P, O):
    reqs = []
    for i, (N, Na, R, eta, v, maxit, dp) in enumerate(STREAM):
        og = O.Geometry(N, Na, I.detector_count(N), 0, R)
        xt = I.random_ellipses(N, 4000 + i)
        b, enorm = I.add_noise(O.forward(og, xt), eta, 4000 + i)
        reqs.append({"geometry": P.Geometry(N, Na, og.n_det, 0, R), "variant": v, "maxit": maxit,
                     "tau": 1.02, "noise_norm": enorm if dp else None,
                     "b": b.astype(np.float32)})
    return reqs


def _submit(eng, r, bt, tag):
    return eng.submit(r["geometry"], bt, r["variant"], r["maxit"], tau=r["tau"],
                      noise_norm=r["noise_norm"], tag=tag)


def test_engine_result_independent_of_the_stream(P, oracle_mod):
    import torch
    reqs = _requests(P, oracle_mod)
    bs = [torch.tensor(r["b"], device="cuda") for r in reqs]
    # alone: one slot, one solve at a time
    alone = {}
    eng1 = P.Engine(1, 1 << 34)
    for i, r in enumerate(reqs):
        assert _submit(eng1, r, bs[i], i) == i
        for t, res in eng1.drain(rounds=3):
            alone[t] = res
    # stream: 3 slots, solves join at different rounds as slots free up
    eng = P.Engine(3, 1 << 34)
    mixed, pending, rounds = {}, list(range(len(reqs))), 0
    while pending or eng.in_flight:
        while pending and _submit(eng, reqs[pending[0]], bs[pending[0]], pending[0]) is not None:
            pending.pop(0)
        for t, res in eng.step(rounds=1 + rounds % 3):
            mixed[t] = res
        rounds += 1
    assert sorted(mixed) == list(range(len(reqs)))
    for i in range(len(reqs)):
        a, m = alone[i], mixed[i]
        assert (a.iters, a.stop_reason) == (m.iters, m.stop_reason), i
        assert torch.equal(a.x, m.x), i
        assert a.resnorm == m.resnorm and a.history == m.history


def test_engine_matches_batch_and_single(P, oracle_mod):
    import torch
    reqs = _requests(P, oracle_mod)[:6]
    bs = [torch.tensor(r["b"], device="cuda") for r in reqs]
    batch = P.Batch([{k: r[k] for k in ("geometry", "variant", "maxit", "tau", "noise_norm")}
                     for r in reqs]).solve(bs)
    eng = P.Engine(8, 1 << 34)
    for i, r in enumerate(reqs):
        assert _submit(eng, r, bs[i], i) == i
    got = dict(eng.drain(rounds=4))
    for i, r in enumerate(reqs):
        # the batch takes the one-launch CGS2 step up to k = 64, the engine
        # the separate passes: the same stop, the iterate to the rounding of
        # the CGS2 sums
        assert got[i].iters == batch[i].iters and got[i].stop_reason == batch[i].stop_reason
        d = (got[i].x - batch[i].x).double().norm() / batch[i].x.double().norm()
        assert d.item() <= 1e-5, (i, d.item())
        if r["noise_norm"]:
            fn = P.ab_gmres if r["variant"] == "ab" else P.ba_gmres
            ref = fn(r["geometry"], bs[i], r["maxit"], tau=1.02, noise_norm=r["noise_norm"])
            torch.cuda.synchronize()
            assert got[i].stop_reason == 1 == ref.stop_reason
            assert abs(got[i].iters - ref.iters) <= 1
            if got[i].iters == ref.iters:
                d = (got[i].x - ref.x).double().norm() / ref.x.double().norm()
                assert d.item() <= 1e-4
            assert got[i].resnorm <= 1.02 * r["noise_norm"] * (1 + 1e-5)


def test_engine_admission_by_slots_and_budget(P, oracle_mod):
    import torch
    r = _requests(P, oracle_mod)[1]
    g = r["geometry"]
    need = P.Engine.request_bytes(g, r["variant"], r["maxit"], r["tau"], r["noise_norm"])
    # the Krylov basis of the BA solve dominates: (maxit + 1) vectors of n floats
    assert need >= 4 * g.n * (r["maxit"] + 1)
    assert need < 4 * (g.n * (r["maxit"] + 1) + g.m * (r["maxit"] + 1)) + 4 * 10 * (g.n + g.m) + (1 << 20)
    bt = torch.tensor(r["b"], device="cuda")
    eng = P.Engine(3, 2 * need + need // 2)
    assert _submit(eng, r, bt, 0) == 0
    assert _submit(eng, r, bt, 1) == 1
    assert _submit(eng, r, bt, 2) is None              # budget: 2.5 requests
    assert eng.in_flight == 2
    done = eng.drain()
    assert sorted(t for t, _ in done) == [0, 1]
    assert torch.equal(done[0][1].x, done[1][1].x)
    assert _submit(eng, r, bt, 2) == 2                 # memory released
    eng.drain()
    eng_slots = P.Engine(1, 1 << 34)
    assert _submit(eng_slots, r, bt, 0) == 0
    assert _submit(eng_slots, r, bt, 1) is None         # slots
    eng_slots.drain()
    small = P.Engine(2, need // 2)
    from paper_2110_01481_gb300 import _native
    with pytest.raises(_native.CtgError):               # can never fit
        _submit(small, r, bt, 0)


def test_engine_zero_iteration_stops(P, oracle_mod):
    import torch
    O = oracle_mod
    og = O.Geometry(48, 40, I.detector_count(48), 0, 180)
    xt = I.random_ellipses(48, 4100)
    g = P.Geometry(48, 40, og.n_det)
    x0 = torch.tensor(xt.ravel(), dtype=torch.float32, device="cuda")
    bb = P.project(g, x0)
    z = torch.zeros_like(bb)
    eng = P.Engine(4, 1 << 32)
    assert eng.submit(g, bb, "ab", 5, noise_norm=1e-3, x0=x0, tag=7) == 7
    assert eng.submit(g, z, "ba", 5, tag=8) == 8
    got = dict(eng.drain())
    assert got[7].iters == 0 and got[7].stop_reason == 1 and torch.equal(got[7].x, x0)
    assert got[8].iters == 0 and got[8].stop_reason == 2 and torch.count_nonzero(got[8].x) == 0


def test_engine_stream_with_mixed_basis_types(P, oracle_mod):
    """Solves whose Krylov bases are FP32, BF16 or FP16 join the engine at
    different rounds (the round graph changes its kernel sequence as the
    basis types present change); each result equals the same solve run
    alone, bit for bit, and a 16-bit solve's admission costs about half."""
    import torch
    reqs = _requests(P, oracle_mod)
    types = ["fp32", "bf16", "fp16", "bf16", "fp32", "fp16", "fp32", "bf16"]
    for r, t in zip(reqs, types):
        r["basis"] = t if r["variant"] == "ab" else ("fp32" if t == "bf16" else t)
    bs = [torch.tensor(r["b"], device="cuda") for r in reqs]

    def submit(eng, i):
        r = reqs[i]
        return eng.submit(r["geometry"], bs[i], r["variant"], r["maxit"], tau=r["tau"],
                          noise_norm=r["noise_norm"], tag=i, basis=r["basis"])

    alone = {}
    eng1 = P.Engine(1, 1 << 34)
    for i in range(len(reqs)):
        assert submit(eng1, i) == i
        alone.update(dict(eng1.drain(rounds=2)))
    eng = P.Engine(3, 1 << 34)
    mixed, pending, rounds = {}, list(range(len(reqs))), 0
    while pending or eng.in_flight:
        while pending and submit(eng, pending[0]) is not None:
            pending.pop(0)
        mixed.update(dict(eng.step(rounds=1 + rounds % 2)))
        rounds += 1
    for i in range(len(reqs)):
        assert alone[i].iters == mixed[i].iters, i
        assert torch.isfinite(mixed[i].x).all(), i
        assert torch.equal(alone[i].x, mixed[i].x), i
    g, r = reqs[0]["geometry"], reqs[0]
    b32 = P.Engine.request_bytes(g, "ab", 40, basis="fp32")
    b16 = P.Engine.request_bytes(g, "ab", 40, basis="bf16")
    assert b16 < 0.65 * b32          # fixed-size buffers weigh more at 64^2
