"""The C-ABI library loads and exports every declared symbol; host-side
argument checks and the workspace-size law.  CPU only: no compute calls."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ctgmres.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2110_01481_gb300 import build, _native
    build.build()
    return _native.lib()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ctg_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("ctg_project", "ctg_backproject", "ctg_ab_gmres", "ctg_ba_gmres",
                     "ctg_workspace_bytes", "ctg_create", "ctg_destroy",
                     "ctg_status_string", "ctg_cgs2"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2110_01481_gb300 import _native
    raw = ctypes.CDLL(_native.LIB_PATH)
    for name in declared_functions():
        assert hasattr(raw, name), name
    assert set(_native.EXPORTS) == set(declared_functions())


def test_status_strings(lib):
    assert lib.ctg_status_string(0) == b"ok"
    assert lib.ctg_status_string(-5) == b"workspace too small"
    assert lib.ctg_status_string(-99) == b"unknown status"


def _g(N, Na, Nd, S=0.0, R=180.0, ds=1.0, model=0, tau=0.0):
    from paper_2110_01481_gb300 import _native as nat
    return nat.CtgGeom(N, Na, Nd, model, S, R, ds, tau)


def _o(maxit, basis=0):
    from paper_2110_01481_gb300 import _native as nat
    return nat.CtgOpts(maxit, basis, 1.0, 0.0)


def test_invalid_arguments_are_rejected_on_the_host(lib):
    ws = lambda g, v, o: lib.ctg_workspace_bytes(ctypes.byref(g), v, ctypes.byref(o))
    assert ws(_g(64, 90, 91), 0, _o(10)) > 0
    assert ws(_g(0, 90, 91), 0, _o(10)) == 0            # empty image
    assert ws(_g(64, 0, 91), 0, _o(10)) == 0            # no angles
    assert ws(_g(64, 90, 0), 1, _o(10)) == 0            # no detectors
    assert ws(_g(64, 90, 91, S=0.5), 0, _o(10)) == 0    # non-integer start
    assert ws(_g(64, 90, 91, R=0.0), 0, _o(10)) == 0
    assert ws(_g(64, 90, 91, ds=0.0), 0, _o(10)) == 0
    assert ws(_g(64, 90, 91), 0, _o(0)) == 0            # maxit >= 1
    assert ws(_g(64, 90, 91), 4, _o(10)) == 0            # unknown variant
    assert ws(_g(64, 90, 91, model=3), 0, _o(10)) == 0   # unknown back projector
    assert ws(_g(64, 90, 91, model=2, tau=1.5), 0, _o(10)) == 0   # B_tau needs tau in [0, 1]
    assert ws(_g(64, 90, 91, model=2, tau=-0.1), 0, _o(10)) == 0
    assert ws(_g(64, 90, 91, model=1, tau=0.3), 0, _o(10)) == 0   # tau only with B_tau
    assert ws(_g(64, 90, 91, model=2, tau=0.3), 0, _o(10)) > 0
    assert ws(_g(64, 90, 91, model=1), 1, _o(10)) > 0
    o = _o(10)
    o.stop_rule = 2                                       # unknown stopping rule
    assert ws(_g(64, 90, 91), 0, o) == 0
    o.stop_rule = 1                                       # NCP: needs 2 <= n_det <= 8192
    assert ws(_g(64, 90, 91), 0, o) > 0 and ws(_g(64, 90, 91), 1, o) > 0
    assert ws(_g(64, 90, 9000, ds=0.5), 0, o) == 0
    assert ws(_g(64, 90, 91), 2, o) == 0                 # LSQR / LSMR: DP rule only
    # solvers and projectors refuse null pointers before touching the GPU
    assert lib.ctg_project(None, ctypes.byref(_g(64, 90, 91)), None, None, None) == -1
    assert lib.ctg_ab_gmres(None, ctypes.byref(_g(64, 90, 91)), None, None, None,
                            ctypes.byref(_o(10)), None, 0, None, None) == -1
    assert lib.ctg_cgs2(None, 8, 8, 1, None, None, None, None, 0, None) == -1
    assert lib.ctg_set_tiles(None, 8, 32) == -1
    assert lib.ctg_set_fwd_tiles(None, 8, 4) == -1
    assert lib.ctg_cgs2_scratch_bytes(0, 1) == 0


def test_workspace_follows_the_krylov_storage_law(lib):
    """Table 3 of the paper: storing k basis vectors costs k * L entries,
    L = m (AB) or n (BA).  The basis dominates the workspace; each vector is
    padded to a multiple of 64 floats."""
    from paper_2110_01481_gb300 import _native as nat
    sizes = {"small": (128, 180, 128), "large": (420, 600, 420)}
    path = os.path.join(ROOT, "tests", "golden", "table3_storage.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    assert len(rows) == 24
    for _, meth, size, k, storage in rows:
        N, Na, Nd = sizes[size]
        k, storage = int(k), int(storage)
        L = Na * Nd if meth == "AB" else N * N
        assert k * L == storage
        g = _g(N, Na, Nd)
        v = nat.CTG_AB if meth == "AB" else nat.CTG_BA
        ly = nat.CtgLayout()
        assert lib.ctg_workspace_layout(ctypes.byref(g), v, ctypes.byref(_o(k)),
                                        ctypes.byref(ly)) == 0
        assert L <= ly.ld_w < L + 64 and ly.ld_w % 64 == 0
        basis_bytes = 4 * (k + 1) * ly.ld_w
        assert abs(basis_bytes // 4 - storage) <= L + 64 * (k + 1)
        total = lib.ctg_workspace_bytes(ctypes.byref(g), v, ctypes.byref(_o(k)))
        assert total == ly.total_bytes
        n, m = N * N, Na * Nd
        other = total - basis_bytes
        # beyond the basis: the staged image (BA also a two-image staging),
        # one n-vector and two m-vectors, O(k^2) doubles of Hessenberg and
        # Givens state, and the reduction scratch; no A W_k
        staged = 4 * 4 * N * (N + 2 * 51) * (3 if meth == "BA" else 1)
        assert 0 < other <= staged + 4 * 2 * (n + 2 * m) + 8 * (2 * k + 8) * (k + 2) \
            + 4 * (k + 4) * 1300 + 16384


def test_lsqr_lsmr_workspace_is_independent_of_maxit(lib):
    """LSQR and LSMR keep no basis (short recurrences): O(n + m) bytes, plus
    the residual history (one double per iteration)."""
    from paper_2110_01481_gb300 import _native as nat
    g = _g(128, 180, 182, model=1)
    n, m = 128 * 128, 180 * 182
    ws = lambda v, k: lib.ctg_workspace_bytes(ctypes.byref(g), v, ctypes.byref(_o(k)))
    for v, nm in ((nat.CTG_LSQR, 2), (nat.CTG_LSMR, 5)):
        assert 0 < ws(v, 1000) - ws(v, 10) <= 8 * 990 + 256
        staged = 4 * 4 * 128 * (128 + 2 * 51)
        assert 4 * (4 * n + nm * m) < ws(v, 10) <= staged + 4 * (4 * n + nm * m) + 8 * 1001 + 65536
    o = _o(10)
    o.basis_dtype = nat.CTG_BASIS_BF16      # no basis to store in 16 bits
    assert lib.ctg_workspace_bytes(ctypes.byref(g), nat.CTG_LSQR, ctypes.byref(o)) == 0
    # a GMRES workspace grows with maxit (the basis)
    assert ws(nat.CTG_AB, 100) > ws(nat.CTG_AB, 10)


def test_engine_admission_bytes_on_the_host(lib):
    """The serving engine sizes a request without touching the GPU: about
    (maxit + 1) basis vectors; unsupported options are refused."""
    from paper_2110_01481_gb300 import _native as nat
    g, o = _g(128, 180, 182), _o(40)
    rb = lambda g, v, o: lib.ctg_engine_request_bytes(ctypes.byref(g), v, ctypes.byref(o))
    ab, ba = rb(g, nat.CTG_AB, o), rb(g, nat.CTG_BA, o)
    assert 4 * 41 * 180 * 182 <= ab < 4 * 41 * 180 * 182 + (4 << 20)
    # BA: the basis (n) and O(n + m) vectors, no A W: the storage law k n
    assert 4 * 41 * 128 * 128 <= ba < 4 * 41 * 128 * 128 + (4 << 20)
    o_dp = _o(40)
    o_dp.noise_norm = 1.0                                 # DP: A x_k and the two-image staging too
    assert ba <= rb(g, nat.CTG_BA, o_dp) < 4 * 41 * 128 * 128 + (4 << 20)
    # A^T and B_tau batch when two detector bins per pixel suffice (pitch >= 1)
    assert rb(_g(128, 180, 182, model=1), nat.CTG_AB, o) >= ab
    assert rb(_g(128, 180, 182, model=2, tau=0.3), nat.CTG_BA, o) >= ba
    assert rb(_g(128, 180, 364, ds=0.5, model=1), nat.CTG_AB, o) == 0
    assert rb(g, nat.CTG_LSQR, o) == 0
    o.stop_rule = 1                                       # NCP: single solves only
    assert rb(g, nat.CTG_AB, o) == 0
    o.stop_rule = 0
    o.basis_dtype = nat.CTG_BASIS_BF16                    # a 16-bit basis halves the request
    ab16 = rb(g, nat.CTG_AB, o)
    assert 2 * 41 * 180 * 182 <= ab16 < ab - 4 * 41 * 180 * 182 // 2 + (1 << 20)
    o.basis_dtype = nat.CTG_BASIS_FP32
    o.maxit = 1025
    assert rb(g, nat.CTG_AB, o) == 0


def test_gmres_workspace_is_the_basis_at_the_benchmark_size(lib):
    """512^2, 720 angles, 725 bins, maxit 150 (the benchmark workload): the
    Krylov basis, (maxit + 1) vectors of length L, is the storage of both
    methods (Table 3's k L), so BA (L = n) needs about half of AB (L = m)
    and a 16-bit basis about half of an FP32 one."""
    from paper_2110_01481_gb300 import _native as nat
    g = _g(512, 720, 725)
    n, m, k = 512 * 512, 720 * 725, 150
    ws = lambda v, basis: lib.ctg_workspace_bytes(ctypes.byref(g), v, ctypes.byref(_o(k, basis)))
    for v, L in ((nat.CTG_AB, m), (nat.CTG_BA, n)):
        basis = 4 * (k + 1) * ((L + 63) // 64 * 64)
        assert basis <= ws(v, 0) <= 1.15 * basis
    assert ws(nat.CTG_BA, 0) < 200e6
    assert ws(nat.CTG_BA, 0) < 0.6 * ws(nat.CTG_AB, 0)
    for v in (nat.CTG_AB, nat.CTG_BA):
        assert ws(v, nat.CTG_BASIS_BF16) < 0.6 * ws(v, 0)
        assert ws(v, nat.CTG_BASIS_FP16) == ws(v, nat.CTG_BASIS_BF16)
