"""Parity of the CUDA projectors with the FP64 oracle (relative 2-norm
<= 1e-5, the FP32 projection tolerance), on seeded phantoms and random
vectors, over small ragged geometries and the full workload sizes."""
import numpy as np
import pytest

from paper_2110_01481_gb300 import inputs as I

pytestmark = pytest.mark.gpu
TOL = 1e-5

GEOMS = [
    # N, n_angles, n_det, start, range, det_spacing
    (64, 90, 91, 0, 180, 1.0),        # 64^2 modified Shepp-Logan workload
    (33, 17, 50, 0, 180, 1.0),        # ragged tiles, odd N
    (48, 30, 68, 0, 120, 1.0),        # limited angle [0, 120)
    (40, 20, 80, 10, 180, 0.75),      # start offset, finer detector pitch
    (64, 16, 40, 0, 180, 1.0),        # detector narrower than the image
    (37, 45, 53, 0, 360, 1.3),        # full turn, coarse pitch
    (1, 1, 1, 0, 180, 1.0),           # degenerate one-pixel, one-ray case
]


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2110_01481_gb300 as P
    return P


def _pair(P, O, N, Na, Nd, S, R, ds):
    return (P.Geometry(N, Na, Nd, S, R, ds), O.Geometry(N, Na, Nd, S, R, ds))


def _rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


@pytest.mark.parametrize("geom", GEOMS)
def test_forward_parity(P, oracle_mod, geom):
    import torch
    g, og = _pair(P, oracle_mod, *geom)
    N = geom[0]
    for x in (I.random_ellipses(N, 3), np.random.default_rng(1).uniform(-1, 1, (N, N))):
        xt = torch.tensor(x.ravel(), dtype=torch.float32, device="cuda")
        got = P.project(g, xt).double().cpu().numpy()
        ref = oracle_mod.forward(og, x.astype(np.float32).astype(np.float64))
        assert _rel(got, ref) <= TOL
        assert np.abs(got - ref).max() <= TOL * max(np.abs(ref).max(), 1e-30) * 10


@pytest.mark.parametrize("geom", GEOMS)
def test_back_parity(P, oracle_mod, geom):
    import torch
    g, og = _pair(P, oracle_mod, *geom)
    rng = np.random.default_rng(2)
    for b in (rng.uniform(0, 1, g.m), rng.standard_normal(g.m)):
        bt = torch.tensor(b, dtype=torch.float32, device="cuda")
        got = P.backproject(g, bt).double().cpu().numpy()
        ref = oracle_mod.backproject(og, b.astype(np.float32).astype(np.float64))
        assert _rel(got, ref) <= TOL
        assert np.abs(got - ref).max() <= TOL * max(np.abs(ref).max(), 1e-30) * 10


def test_back_of_ones_is_angle_count(P):
    """B 1 = N_a exactly when every pixel centre lies inside the detector."""
    import torch
    g = P.Geometry(96, 45, I.detector_count(96))
    x = P.backproject(g, torch.ones(g.m, device="cuda")).cpu().numpy()
    np.testing.assert_allclose(x, 45.0, rtol=2e-7)


@pytest.mark.parametrize("N,Na", [(512, 720), (2048, 1800)])
def test_full_size_parity(P, oracle_mod, N, Na):
    """512^2 x 720 angles x 725 bins and 2048^2 x 1800 x 2897, in the launch
    configuration the solvers and the benchmark use."""
    import torch
    Nd = I.detector_count(N)
    g, og = P.Geometry(N, Na, Nd), oracle_mod.Geometry(N, Na, Nd)
    x = I.random_ellipses(N, 2000 + N).astype(np.float32)
    xt = torch.tensor(x.ravel(), device="cuda")
    got = P.project(g, xt).double().cpu().numpy()
    ref = oracle_mod.forward(og, x.astype(np.float64))
    assert _rel(got, ref) <= TOL
    bt = torch.tensor(ref, dtype=torch.float32, device="cuda")
    gotb = P.backproject(g, bt).double().cpu().numpy()
    refb = oracle_mod.backproject(og, ref.astype(np.float32).astype(np.float64))
    assert _rel(gotb, refb) <= TOL


def test_rejects_bad_arguments(P):
    import torch
    from paper_2110_01481_gb300 import _native as nat
    g = P.Geometry(16, 8, 23)
    with pytest.raises(ValueError):
        P.project(g, torch.zeros(10, device="cuda"))
    with pytest.raises(nat.CtgError):
        P.project(P.Geometry(16, 8, 23, angle_start_deg=0.5), torch.zeros(256, device="cuda"))
    with pytest.raises(nat.CtgError):
        P.backproject(P.Geometry(0, 8, 23), torch.zeros(184, device="cuda"),
                      out=torch.zeros(0, device="cuda"))


def test_tile_autotuner_is_result_invariant(P):
    """The autotuned tile shapes (angles per forward block and per warp,
    angles staged per back-projection pass) change the speed only: every
    shape gives the same projections bit for bit, and the tuner reports the
    timed candidates.  The shapes with 4 angles per warp are timed where the
    angular sampling is fine enough for them (90 angles over 180 degrees) and
    fall back to one angle per warp elsewhere (45 angles over 360)."""
    import torch
    ctx = P.Context.get(torch.device("cuda", 0))
    cases = [P.Geometry(200, 90, 283), P.Geometry(96, 37, 150, 0, 120), P.Geometry(64, 45, 91, 10, 360, 1.3)]
    gen = torch.Generator(device="cuda").manual_seed(21)
    try:
        for g in cases:
            x = torch.rand(g.n, device="cuda", generator=gen)
            y = torch.randn(g.m, device="cuda", generator=gen)
            ctx.set_tiles(0, 0)
            t = ctx.tuning(g)
            assert t["tuned"] and t["back_chunk"] in (16, 32, 64)
            assert (t["fwd_angles"], t["fwd_warp_angles"]) in ((4, 1), (8, 1), (8, 4), (16, 4))
            assert t["fwd_us"]["8x1"] > 0 and t["fwd_us"]["4x1"] > 0
            assert all(v > 0 for v in t["back_us"].values())
            if g.n_angles == 90:
                assert t["fwd_us"]["8x4"] > 0 and t["fwd_us"]["16x4"] > 0
            ref_a, ref_b = P.project(g, x), P.backproject(g, y)
            for fa, fw, bc in ((8, 1, 32), (4, 1, 16), (4, 1, 64), (8, 1, 64), (8, 1, 16), (8, 4, 32),
                               (16, 4, 64)):
                ctx.set_tiles(fa, bc, fw)
                tt = ctx.tuning(g)
                split_ok = tt["fwd_us"]["8x4"] > 0
                want = (fa, fw) if fw == 1 or split_ok else (8, 1)
                assert (tt["fwd_angles"], tt["fwd_warp_angles"]) == want and tt["back_chunk"] == bc
                assert torch.equal(P.project(g, x), ref_a), (g, fa, fw)
                assert torch.equal(P.backproject(g, y), ref_b), (g, bc)
            # clearing the forced shapes restores the autotuner's choice
            ctx.set_tiles(0, 0)
            tt = ctx.tuning(g)
            assert (tt["fwd_angles"], tt["fwd_warp_angles"], tt["back_chunk"]) == \
                (t["fwd_angles"], t["fwd_warp_angles"], t["back_chunk"])
    finally:
        ctx.set_tiles(0, 0)
