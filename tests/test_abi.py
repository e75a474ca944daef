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


def _g(N, Na, Nd, S=0.0, R=180.0, ds=1.0):
    from paper_2110_01481_gb300 import _native as nat
    return nat.CtgGeom(N, Na, Nd, 0, S, R, ds)


def _o(maxit):
    from paper_2110_01481_gb300 import _native as nat
    return nat.CtgOpts(maxit, 0, 1.0, 0.0)


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
    assert ws(_g(64, 90, 91), 2, _o(10)) == 0            # unknown variant
    g = _g(64, 90, 91)
    g.reserved = 1
    assert ws(g, 0, _o(10)) == 0
    # solvers and projectors refuse null pointers before touching the GPU
    assert lib.ctg_project(None, ctypes.byref(_g(64, 90, 91)), None, None, None) == -1
    assert lib.ctg_ab_gmres(None, ctypes.byref(_g(64, 90, 91)), None, None, None,
                            ctypes.byref(_o(10)), None, 0, None, None) == -1
    assert lib.ctg_cgs2(None, 8, 8, 1, None, None, None, None, 0, None) == -1
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
        # BA also keeps T = A W_k (the forward projections of the basis
        # vectors, reused by the discrepancy-principle residual)
        t_bytes = 4 * (k + 2) * ((m + 63) // 64 * 64) if meth == "BA" else 0
        staged = 4 * 4 * N * (N + 2 * 51)
        assert 0 < other <= t_bytes + staged + 4 * 2 * (n + 2 * m) + 8 * (k + 1) * (k + 2) \
            + 4 * (k + 4) * 1300 + 16384
