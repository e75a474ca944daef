"""Torch-facing wrappers of the C-ABI (include/ctgmres.h).

Arguments are torch tensors on a CUDA device (float32, contiguous, 16-byte
aligned); calls are enqueued on torch's current stream of that device.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass, field
from typing import Optional

import torch

from . import _native as nat


@dataclass(frozen=True)
class Geometry:
    """2D parallel-beam geometry (paper Sec. 6.1, Table 1) and its back
    projector: "pixel" (the unmatched pixel-driven B), "matched" (A^T) or
    "threshold" (B_tau of Sec. 6.5 with tau = back_tau)."""
    N: int
    n_angles: int
    n_det: int
    angle_start_deg: float = 0.0
    angle_range_deg: float = 180.0
    det_spacing: float = 1.0
    back_model: str = "pixel"
    back_tau: float = 0.0

    @property
    def n(self) -> int:
        return self.N * self.N

    @property
    def m(self) -> int:
        return self.n_angles * self.n_det

    def c(self) -> nat.CtgGeom:
        if self.back_model not in nat.BACK:
            raise ValueError(f"back_model must be one of {sorted(nat.BACK)}")
        return nat.CtgGeom(self.N, self.n_angles, self.n_det, nat.BACK[self.back_model],
                           float(self.angle_start_deg), float(self.angle_range_deg),
                           float(self.det_spacing), float(self.back_tau))


class Context:
    """One ctg_ctx per CUDA device (cached angle tables, pinned staging)."""
    _per_device: dict = {}

    def __init__(self, device: int):
        self.device = device
        self.handle = ctypes.c_void_p()
        with torch.cuda.device(device):
            nat.check(nat.lib().ctg_create(ctypes.byref(self.handle)), "ctg_create")

    @classmethod
    def get(cls, device) -> "Context":
        idx = torch.device(device).index
        if idx is None:
            idx = torch.cuda.current_device()
        ctx = cls._per_device.get(idx)
        if ctx is None:
            ctx = cls._per_device[idx] = Context(idx)
        return ctx

    def set_timing(self, enable: bool) -> None:
        with torch.cuda.device(self.device):
            nat.check(nat.lib().ctg_set_timing(self.handle, int(enable)), "ctg_set_timing")

    def timing(self, reset: bool = False) -> dict:
        """Per-phase device milliseconds and call counts, and the number of
        kernels the library launched, since the last reset."""
        t = nat.CtgTiming()
        with torch.cuda.device(self.device):
            nat.check(nat.lib().ctg_get_timing(self.handle, ctypes.byref(t), int(reset)),
                      "ctg_get_timing")
        out = {p: {"ms": t.ms[i], "calls": int(t.calls[i])} for i, p in enumerate(nat.PHASES)}
        out["kernels"] = int(t.kernels)
        return out

    def set_wait_limit(self, polls: int = 0) -> None:
        """Polls of a bounded device-side wait before it gives up (the solve
        then raises CtgError with CTG_ERR_TIMEOUT); 0 restores the default."""
        nat.check(nat.lib().ctg_set_wait_limit(self.handle, int(polls)), "ctg_set_wait_limit")

    def set_tiles(self, fwd_angles: int = 0, back_chunk: int = 0, fwd_warp_angles: int = 1) -> None:
        """Force the projectors' tile shapes (0, 0: autotuned per geometry).
        The forward shape is fwd_angles angles per block with fwd_warp_angles
        per warp: (4, 1), (8, 1), (8, 4) or (16, 4)."""
        lib = nat.lib()
        if fwd_warp_angles == 1:
            nat.check(lib.ctg_set_tiles(self.handle, int(fwd_angles), int(back_chunk)), "ctg_set_tiles")
        else:
            nat.check(lib.ctg_set_tiles(self.handle, 0, int(back_chunk)), "ctg_set_tiles")
            nat.check(lib.ctg_set_fwd_tiles(self.handle, int(fwd_angles), int(fwd_warp_angles)),
                      "ctg_set_fwd_tiles")

    def tuning(self, g: "Geometry") -> dict:
        """Tile shapes in use for geometry g and the autotuner's timings (us)."""
        t = nat.CtgTuning()
        with torch.cuda.device(self.device):
            nat.check(nat.lib().ctg_get_tuning(self.handle, ctypes.byref(g.c()), ctypes.byref(t)),
                      "ctg_get_tuning")
        return {"fwd_angles": t.fwd_angles, "fwd_warp_angles": t.fwd_warp_angles,
                "back_chunk": t.back_chunk, "tuned": bool(t.tuned),
                "fwd_us": {"8x1": t.fwd_us[0], "4x1": t.fwd_us[1], "8x4": t.fwd_split_us[0],
                           "16x4": t.fwd_split_us[1]},
                "back_us": {16: t.back_us[0], 32: t.back_us[1], 64: t.back_us[2]}}

    def __del__(self):
        h = getattr(self, "handle", None)
        if h and nat._lib is not None:
            try:
                with torch.cuda.device(self.device):
                    nat.lib().ctg_destroy(h)
            except Exception:
                pass


def _dev_ptr(t: torch.Tensor, numel: int, name: str, dtype=torch.float32) -> int:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype or not t.is_contiguous() or t.numel() != numel:
        raise ValueError(f"{name}: expected a contiguous {dtype} tensor of {numel} elements, "
                         f"got {t.dtype} {tuple(t.shape)}")
    return t.data_ptr()


def _stream(device) -> int:
    return torch.cuda.current_stream(device).cuda_stream


def project(g: Geometry, x: torch.Tensor, out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """b = A x (Joseph forward projection); x: n floats (any shape)."""
    if out is None:
        out = torch.empty(g.m, device=x.device, dtype=torch.float32)
    px, pb = _dev_ptr(x, g.n, "x"), _dev_ptr(out, g.m, "out")
    ctx = Context.get(x.device)
    with torch.cuda.device(x.device):
        nat.check(nat.lib().ctg_project(ctx.handle, ctypes.byref(g.c()), px, pb,
                                        _stream(x.device)), "ctg_project")
    return out


def backproject(g: Geometry, b: torch.Tensor, out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """x = B b with the geometry's back projector (by default the unmatched
    pixel-driven B; A^T or B_tau by back_model); b: m floats."""
    if out is None:
        out = torch.empty(g.n, device=b.device, dtype=torch.float32)
    pb, px = _dev_ptr(b, g.m, "b"), _dev_ptr(out, g.n, "out")
    ctx = Context.get(b.device)
    with torch.cuda.device(b.device):
        nat.check(nat.lib().ctg_backproject(ctx.handle, ctypes.byref(g.c()), pb, px,
                                            _stream(b.device)), "ctg_backproject")
    return out


_TORCH_BASIS = {"fp32": torch.float32, "bf16": torch.bfloat16, "fp16": torch.float16}


def _opts(maxit: int, tau: float, noise_norm: Optional[float], basis: str = "fp32",
          stop: str = "dp") -> nat.CtgOpts:
    if basis not in nat.BASIS:
        raise ValueError(f"basis must be one of {sorted(nat.BASIS)}")
    if stop not in nat.RULES:
        raise ValueError(f"stop must be one of {sorted(nat.RULES)}")
    return nat.CtgOpts(int(maxit), nat.BASIS[basis], float(tau),
                       float(noise_norm) if noise_norm else 0.0, nat.RULES[stop])


def workspace_bytes(g: Geometry, variant: str, maxit: int, basis: str = "fp32",
                    stop: str = "dp") -> int:
    """Device bytes one solve needs (0 if the arguments are invalid);
    variant: "ab", "ba", "lsqr" or "lsmr"."""
    v = nat.VARIANTS[variant]
    return int(nat.lib().ctg_workspace_bytes(ctypes.byref(g.c()), v,
                                             ctypes.byref(_opts(maxit, 1.0, None, basis, stop))))


def workspace_layout(g: Geometry, variant: str, maxit: int, basis: str = "fp32") -> nat.CtgLayout:
    v = nat.CTG_AB if variant == "ab" else nat.CTG_BA
    out = nat.CtgLayout()
    nat.check(nat.lib().ctg_workspace_layout(ctypes.byref(g.c()), v,
                                             ctypes.byref(_opts(maxit, 1.0, None, basis)),
                                             ctypes.byref(out)), "ctg_workspace_layout")
    return out


@dataclass
class SolveResult:
    x: torch.Tensor
    iters: int
    stop_reason: int          # 0 maxit, 1 discrepancy principle, 2 breakdown
    resnorm: float            # ||b - A x_k|| of the returned iterate
    rho: float                # GMRES residual of the last step
    history: list = field(default_factory=list)
    workspace: Optional[torch.Tensor] = None
    basis_type: str = "fp32"
    ncp_history: list = field(default_factory=list)   # NCP distances d_0.. (stop="ncp")

    def basis(self, g: Geometry, variant: str, maxit: int) -> torch.Tensor:
        """View of the final Krylov basis W (iters+1 vectors, stored element
        type) in the workspace."""
        ly = workspace_layout(g, variant, maxit, self.basis_type)
        L = g.m if variant == "ab" else g.n
        dt = _TORCH_BASIS[self.basis_type]
        es = torch.empty(0, dtype=dt).element_size()
        nbytes = es * ly.ld_w * (maxit + 1)
        W = self.workspace[ly.off_w: ly.off_w + nbytes].view(dt).view(maxit + 1, ly.ld_w)
        return W[: self.iters + 1, :L]

    def hessenberg(self, g: Geometry, variant: str, maxit: int) -> torch.Tensor:
        """The (iters+1) x iters Hessenberg matrix H_k (FP64) from the workspace."""
        ly = workspace_layout(g, variant, maxit, self.basis_type)
        d = self.workspace[ly.off_h: ly.off_h + 8 * (maxit + 1) * maxit].view(torch.float64)
        H = d.view(maxit, maxit + 1).t()          # column-major storage
        return H[: self.iters + 1, : self.iters]


def _solve(fn, variant: str, g: Geometry, b: torch.Tensor, maxit: int,
           x0: Optional[torch.Tensor], tau: float, noise_norm: Optional[float],
           out: Optional[torch.Tensor], workspace: Optional[torch.Tensor],
           keep_workspace: bool, basis: str = "fp32", stop: str = "dp") -> SolveResult:
    dev = b.device
    pb = _dev_ptr(b, g.m, "b")
    px0 = _dev_ptr(x0, g.n, "x0") if x0 is not None else None
    if out is None:
        out = torch.empty(g.n, device=dev, dtype=torch.float32)
    px = _dev_ptr(out, g.n, "out")
    o = _opts(maxit, tau, noise_norm, basis, stop)
    need = workspace_bytes(g, variant, maxit, basis, stop)
    name = f"ctg_{variant}" if variant in ("lsqr", "lsmr") else f"ctg_{variant}_gmres"
    if need == 0:
        raise nat.CtgError(nat.CTG_ERR_INVALID_ARG, name)
    if workspace is None and keep_workspace:
        workspace = torch.empty(need, device=dev, dtype=torch.uint8)
    pws, nws = (None, 0)
    if workspace is not None:
        pws, nws = _dev_ptr(workspace, workspace.numel(), "workspace", torch.uint8), workspace.numel()
    # the library fills entries 0..iters (the arrays start zeroed)
    hist = (ctypes.c_double * (maxit + 1))()
    dncp = (ctypes.c_double * (maxit + 2))() if stop == "ncp" else None
    info = nat.CtgInfo(0, 0, 0.0, 0.0, hist, dncp)
    ctx = Context.get(dev)
    with torch.cuda.device(dev):
        nat.check(fn(ctx.handle, ctypes.byref(g.c()), pb, px0, px, ctypes.byref(o), pws, nws,
                     ctypes.byref(info), _stream(dev)), name)
    nd = info.iters + (2 if info.stop_reason == nat.CTG_STOP_NCP else 1) if stop == "ncp" else 0
    return SolveResult(out, info.iters, info.stop_reason, info.resnorm, info.rho,
                       list(hist[: info.iters + 1]), workspace, basis,
                       list(dncp[:nd]) if dncp is not None else [])


def ab_gmres(g: Geometry, b: torch.Tensor, maxit: int, x0=None, tau: float = 1.0,
             noise_norm: Optional[float] = None, out=None, workspace=None,
             keep_workspace: bool = False, basis: str = "fp32", stop: str = "dp") -> SolveResult:
    """AB-GMRES (paper Sec. 2) with the discrepancy-principle stop when
    noise_norm is given (Sec. 6.4), or the NCP stop with stop="ncp".  basis:
    storage type of the Krylov basis ("fp32", "bf16" or "fp16"; arithmetic
    stays FP32/FP64)."""
    return _solve(nat.lib().ctg_ab_gmres, "ab", g, b, maxit, x0, tau, noise_norm, out,
                  workspace, keep_workspace, basis, stop)


def ba_gmres(g: Geometry, b: torch.Tensor, maxit: int, x0=None, tau: float = 1.0,
             noise_norm: Optional[float] = None, out=None, workspace=None,
             keep_workspace: bool = False, basis: str = "fp32", stop: str = "dp") -> SolveResult:
    """BA-GMRES (paper Sec. 2); same conventions as ``ab_gmres``."""
    return _solve(nat.lib().ctg_ba_gmres, "ba", g, b, maxit, x0, tau, noise_norm, out,
                  workspace, keep_workspace, basis, stop)


def ncp_distance(g: Geometry, r: torch.Tensor) -> float:
    """The NCP distance (Sec. 6.4's NCP criterion) of a residual sinogram r:
    the mean over the projections of the distance of the normalised
    cumulative periodogram from the white-noise line."""
    out = ctypes.c_double()
    ctx = Context.get(r.device)
    with torch.cuda.device(r.device):
        nat.check(nat.lib().ctg_ncp_distance(ctx.handle, ctypes.byref(g.c()), _dev_ptr(r, g.m, "r"),
                                             ctypes.byref(out), _stream(r.device)), "ctg_ncp_distance")
    return out.value


def lsqr(g: Geometry, b: torch.Tensor, maxit: int, x0=None, tau: float = 1.0,
         noise_norm: Optional[float] = None, out=None, workspace=None,
         keep_workspace: bool = False) -> SolveResult:
    """LSQR (Sec. 5's matched-case comparator) with the geometry's back
    projector as A^T (use back_model="matched" for LSQR proper); the
    discrepancy-principle stop on its residual estimate when noise_norm is
    given.  history[k] = the estimate of ||b - A x_k||."""
    return _solve(nat.lib().ctg_lsqr, "lsqr", g, b, maxit, x0, tau, noise_norm, out,
                  workspace, keep_workspace)


def lsmr(g: Geometry, b: torch.Tensor, maxit: int, x0=None, tau: float = 1.0,
         noise_norm: Optional[float] = None, out=None, workspace=None,
         keep_workspace: bool = False) -> SolveResult:
    """LSMR (Sec. 5's matched-case comparator); same conventions as ``lsqr``,
    history[k] = ||b - A x_k|| tracked through the recurrences."""
    return _solve(nat.lib().ctg_lsmr, "lsmr", g, b, maxit, x0, tau, noise_norm, out,
                  workspace, keep_workspace)


def cgs2(W: torch.Tensor, k: int, q: torch.Tensor, w_out: Optional[torch.Tensor] = None,
         scratch: Optional[torch.Tensor] = None):
    """One CGS2 Arnoldi step of q against the first k rows of W (2-D tensor,
    rows = basis vectors).  Returns (h, w_out), h = k+1 doubles."""
    L = q.numel()
    ldw = W.stride(0) if W.dim() == 2 else L
    if W.dtype != torch.float32 or not W.is_cuda or W.stride(-1) != 1:
        raise ValueError("W must be a CUDA float32 tensor with unit inner stride")
    if w_out is None:
        w_out = torch.empty_like(q)
    h = torch.empty(k + 1, device=q.device, dtype=torch.float64)
    need = int(nat.lib().ctg_cgs2_scratch_bytes(L, k))
    if scratch is None:
        scratch = torch.empty(need, device=q.device, dtype=torch.uint8)
    with torch.cuda.device(q.device):
        nat.check(nat.lib().ctg_cgs2(W.data_ptr(), ldw, L, k, _dev_ptr(q, L, "q"),
                                     _dev_ptr(w_out, L, "w_out"), h.data_ptr(),
                                     scratch.data_ptr(), scratch.numel(),
                                     _stream(q.device)), "ctg_cgs2")
    return h, w_out


class Batch:
    """Batched AB-/BA-GMRES (ctg_batch_*): solves of different geometries,
    variants and options advance together, one Arnoldi step per round, with
    the Hessenberg update and the stopping rule on the device and each round
    replayed as a captured CUDA graph.

    problems: list of dicts with keys geometry (Geometry), variant ("ab" or
    "ba"), maxit, and optionally tau, noise_norm, basis ("fp32", "bf16" or
    "fp16": storage type of that solve's Krylov basis)."""

    def __init__(self, problems, device=None):
        if not problems:
            raise ValueError("empty batch")
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.problems = list(problems)
        n = len(problems)
        geoms = (nat.CtgGeom * n)(*[p["geometry"].c() for p in problems])
        variants = (ctypes.c_int32 * n)(*[nat.CTG_AB if p["variant"] == "ab" else nat.CTG_BA
                                          for p in problems])
        opts = (nat.CtgOpts * n)(*[_opts(p["maxit"], p.get("tau", 1.0), p.get("noise_norm"),
                                         p.get("basis", "fp32"))
                                   for p in problems])
        self.ctx = Context.get(self.device)
        self.handle = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            nat.check(nat.lib().ctg_batch_create(self.ctx.handle, n, geoms, variants, opts,
                                                 ctypes.byref(self.handle)), "ctg_batch_create")

    @property
    def workspace_bytes(self) -> int:
        return int(nat.lib().ctg_batch_workspace_bytes(self.handle))

    def solve(self, bs, x0s=None, outs=None):
        """bs: list of CUDA tensors (m floats each); returns a list of
        SolveResult in the same order."""
        n = len(self.problems)
        if len(bs) != n:
            raise ValueError("one right-hand side per problem")
        if outs is None:
            outs = [torch.empty(p["geometry"].n, device=self.device, dtype=torch.float32)
                    for p in self.problems]
        pb = (ctypes.c_void_p * n)(*[_dev_ptr(b, p["geometry"].m, "b") for b, p in zip(bs, self.problems)])
        px = (ctypes.c_void_p * n)(*[_dev_ptr(x, p["geometry"].n, "x") for x, p in zip(outs, self.problems)])
        px0 = None
        if x0s is not None:
            px0 = (ctypes.c_void_p * n)(*[_dev_ptr(x0, p["geometry"].n, "x0") if x0 is not None else None
                                          for x0, p in zip(x0s, self.problems)])
        hists = [(ctypes.c_double * (p["maxit"] + 1))()
                 for p in self.problems]
        infos = (nat.CtgInfo * n)(*[nat.CtgInfo(0, 0, 0.0, 0.0, h) for h in hists])
        with torch.cuda.device(self.device):
            nat.check(nat.lib().ctg_batch_solve(self.handle, pb, px0, px, infos,
                                                _stream(self.device)), "ctg_batch_solve")
        return [SolveResult(outs[i], infos[i].iters, infos[i].stop_reason, infos[i].resnorm,
                            infos[i].rho, list(hists[i][: infos[i].iters + 1])) for i in range(n)]

    def __del__(self):
        h = getattr(self, "handle", None)
        if h and nat._lib is not None:
            try:
                with torch.cuda.device(self.device):
                    nat.lib().ctg_batch_destroy(h)
            except Exception:
                pass


class Engine:
    """Serving engine (ctg_engine_*): continuous batching of independent
    AB-/BA-GMRES solves.  ``submit`` admits a solve while others run, if a
    slot is free and its workspace fits the device-memory budget; ``step``
    advances every running solve by ``rounds`` Arnoldi steps and returns the
    solves that finished, as (tag, SolveResult) pairs.  The tensors of a
    solve are held here until it is reported."""

    def __init__(self, max_slots, hbm_budget_bytes, device=None):
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.max_slots = int(max_slots)
        self.ctx = Context.get(self.device)
        self.handle = ctypes.c_void_p()
        self._held = {}
        self._next_tag = 0
        with torch.cuda.device(self.device):
            nat.check(nat.lib().ctg_engine_create(self.ctx.handle, self.max_slots, int(hbm_budget_bytes),
                                                  ctypes.byref(self.handle)), "ctg_engine_create")

    @staticmethod
    def request_bytes(geometry, variant, maxit, tau=1.0, noise_norm=None, basis="fp32") -> int:
        """Device bytes one solve occupies while in flight (0: invalid)."""
        g = geometry.c()
        o = _opts(maxit, tau, noise_norm, basis)
        v = nat.CTG_AB if variant == "ab" else nat.CTG_BA
        return int(nat.lib().ctg_engine_request_bytes(ctypes.byref(g), v, ctypes.byref(o)))

    @property
    def in_flight(self) -> int:
        return int(nat.lib().ctg_engine_in_flight(self.handle))

    def submit(self, geometry, b, variant="ab", maxit=100, tau=1.0, noise_norm=None,
               x0=None, out=None, tag=None, basis="fp32"):
        """Admit one solve; returns its tag, or None if the engine is busy
        (no free slot, or not enough of the memory budget left).  basis:
        storage type of its Krylov basis ("fp32", "bf16" or "fp16")."""
        if tag is None:
            tag = self._next_tag
        self._next_tag = max(self._next_tag, int(tag) + 1)
        if out is None:
            out = torch.empty(geometry.n, device=self.device, dtype=torch.float32)
        g = geometry.c()
        o = _opts(maxit, tau, noise_norm, basis)
        hist = (ctypes.c_double * (maxit + 1))()
        pb = _dev_ptr(b, geometry.m, "b")
        px = _dev_ptr(out, geometry.n, "x")
        px0 = _dev_ptr(x0, geometry.n, "x0") if x0 is not None else None
        with torch.cuda.device(self.device):
            rc = nat.lib().ctg_engine_submit(self.handle, ctypes.byref(g),
                                             nat.CTG_AB if variant == "ab" else nat.CTG_BA,
                                             ctypes.byref(o), pb, px0, px, hist, int(tag),
                                             _stream(self.device))
        if rc == nat.CTG_ERR_BUSY:
            return None
        nat.check(rc, "ctg_engine_submit")
        self._held[int(tag)] = (b, x0, out, hist)
        return int(tag)

    def step(self, rounds=4):
        """Run ``rounds`` rounds; returns [(tag, SolveResult)] of the solves
        that finished (their x is complete)."""
        cap = max(self.max_slots, 1)
        tags = (ctypes.c_int64 * cap)()
        infos = (nat.CtgInfo * cap)()
        n = ctypes.c_int32(0)
        with torch.cuda.device(self.device):
            nat.check(nat.lib().ctg_engine_step(self.handle, int(rounds), cap, tags, infos,
                                                ctypes.byref(n)), "ctg_engine_step")
        done = []
        for i in range(n.value):
            t = int(tags[i])
            _, _, out, hist = self._held.pop(t)
            inf = infos[i]
            done.append((t, SolveResult(out, inf.iters, inf.stop_reason, inf.resnorm, inf.rho,
                                        list(hist[: inf.iters + 1]))))
        return done

    def drain(self, rounds=4):
        """Step until every admitted solve is reported."""
        done = []
        while self.in_flight:
            done += self.step(rounds)
        return done

    def __del__(self):
        h = getattr(self, "handle", None)
        if h and nat._lib is not None:
            try:
                with torch.cuda.device(self.device):
                    nat.lib().ctg_engine_destroy(h)
            except Exception:
                pass
