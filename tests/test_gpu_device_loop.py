"""The device-driven solver loop.

An AB-/BA-GMRES solve runs as one CUDA graph (while-loop nodes over the
Arnoldi steps, with the FP64 Givens update and the stopping rule on the
device); with phase tracing on, the host enqueues the same kernels step by
step.  Both drivers must give the same result bit for bit, a replayed graph
the same as its first launch, and a bounded device-side wait that gives up
must come back as CTG_ERR_TIMEOUT with the context still usable.
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


def _case(O, N, Na, seed, eta=0.01):
    og = O.Geometry(N, Na, I.detector_count(N))
    xt = I.random_ellipses(N, seed)
    b, enorm = I.add_noise(O.forward(og, xt), eta, seed)
    return og, b.astype(np.float32), enorm


@pytest.mark.parametrize("variant", ["ab", "ba"])
@pytest.mark.parametrize("stop", ["dp", "maxit", "ncp"])
def test_graph_and_host_driven_loops_agree(P, oracle_mod, variant, stop):
    import torch
    og, b, enorm = _case(oracle_mod, 96, 120, 7100)
    g = P.Geometry(96, 120, og.n_det)
    bt = torch.tensor(b, device="cuda")
    fn = P.ab_gmres if variant == "ab" else P.ba_gmres
    kw = {"maxit": 40 if stop != "maxit" else 12}
    if stop == "dp":
        kw.update(tau=1.02, noise_norm=enorm)
    if stop == "ncp":
        kw.update(stop="ncp")
    ws = torch.empty(P.workspace_bytes(g, variant, kw["maxit"], stop=kw.get("stop", "dp")),
                     dtype=torch.uint8, device="cuda")
    ctx = P.Context.get(bt.device)
    outs = []
    for timing in (False, False, True):       # graph, graph replayed, host-driven
        ctx.set_timing(timing)
        x = torch.empty(g.n, device="cuda")
        r = fn(g, bt, out=x, workspace=ws, **kw)
        torch.cuda.synchronize()
        outs.append(r)
    ctx.set_timing(False)
    ctx.timing(reset=True)
    ref = outs[0]
    assert ref.iters >= 1
    for r in outs[1:]:
        assert r.iters == ref.iters and r.stop_reason == ref.stop_reason
        assert torch.equal(r.x, ref.x)
        assert r.resnorm == ref.resnorm and r.rho == ref.rho
        assert r.history == ref.history


def test_wait_timeout_is_reported_and_recoverable(P, oracle_mod):
    """With every bounded wait limited to one poll, the one-launch CGS2 step
    (304 blocks at this length) cannot see all blocks arrive at its first
    grid barrier: the solve stops with CTG_ERR_TIMEOUT, nothing waits for
    ever, and the next solve with the default limit is exact."""
    import torch
    from paper_2110_01481_gb300 import _native as nat
    og, b, enorm = _case(oracle_mod, 512, 720, 7200)
    g = P.Geometry(512, 720, og.n_det)
    bt = torch.tensor(b, device="cuda")
    ctx = P.Context.get(bt.device)
    ref = P.ab_gmres(g, bt, 8)
    torch.cuda.synchronize()
    try:
        ctx.set_wait_limit(1)
        with pytest.raises(nat.CtgError) as ei:
            P.ab_gmres(g, bt, 8)
        assert ei.value.status == nat.CTG_ERR_TIMEOUT
    finally:
        ctx.set_wait_limit(0)
    again = P.ab_gmres(g, bt, 8)
    torch.cuda.synchronize()
    assert again.iters == ref.iters == 8
    assert torch.equal(again.x, ref.x)
