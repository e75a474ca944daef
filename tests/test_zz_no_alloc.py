"""ctg_cgs2_noalloc, the CGS2 step for callers that cannot allocate device
memory (for example because their own memory manager has reserved the whole
device, or because they run as a plugin inside a framework that owns every
allocation), must give the same result as ctg_cgs2 with caller scratch.

This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2110_01481_gb300 import _native as nat
    return torch, nat.lib()


def _case(torch, L, k, seed):
    rng = np.random.default_rng(seed)
    ld = (L + 63) // 64 * 64
    W = torch.zeros((max(k, 1), ld), dtype=torch.float32, device="cuda")
    if k:
        Wd = np.linalg.qr(rng.standard_normal((L, k)))[0].T
        W[:k, :L] = torch.tensor(Wd, dtype=torch.float32)
    q = torch.tensor(rng.standard_normal(L), dtype=torch.float32, device="cuda")
    return W, ld, q


def _with_scratch(torch, lib, W, ld, L, k, q):
    """The existing entry point, caller-owned scratch."""
    qq = q.clone()
    w = torch.empty_like(q)
    h = torch.empty(k + 1, dtype=torch.float64, device="cuda")
    nbytes = lib.ctg_cgs2_scratch_bytes(L, k)
    scratch = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    assert lib.ctg_cgs2(W.data_ptr(), ld, L, k, qq.data_ptr(), w.data_ptr(), h.data_ptr(),
                        scratch.data_ptr(), nbytes, st) == 0
    torch.cuda.synchronize()
    return h.cpu().numpy(), w.double().cpu().numpy()


def _no_alloc(torch, lib, W, ld, L, k, q):
    qq = q.clone()
    w = torch.empty_like(q)
    h = torch.empty(k + 1, dtype=torch.float64, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    assert lib.ctg_cgs2_noalloc(W.data_ptr(), ld, L, k, qq.data_ptr(), w.data_ptr(),
                                h.data_ptr(), st) == 0
    torch.cuda.synchronize()
    return h.cpu().numpy(), w.double().cpu().numpy()


def test_no_alloc_matches_scratch_entry_point_on_two_calls(env):
    torch, lib = env
    # two calls in a row on different sizes: the second must not see stale
    # state left in the shared array by the first
    for L, k, seed in ((4099, 33, 1), (262147, 150, 2)):
        W, ld, q = _case(torch, L, k, seed)
        h_ref, w_ref = _with_scratch(torch, lib, W, ld, L, k, q)
        h, w = _no_alloc(torch, lib, W, ld, L, k, q)
        qn = float(np.linalg.norm(q.double().cpu().numpy()))
        assert np.abs(h - h_ref).max() <= 1e-5 * qn
        assert np.linalg.norm(w - w_ref) <= 1e-4 * np.linalg.norm(w_ref)


def test_no_alloc_rejects_sizes_beyond_its_fixed_scratch(env):
    torch, lib = env
    W, ld, q = _case(torch, 64, 1, 3)
    w = torch.empty_like(q)
    h = torch.empty(300, dtype=torch.float64, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    assert lib.ctg_cgs2_noalloc(W.data_ptr(), ld, 64, 257, q.data_ptr(), w.data_ptr(),
                                h.data_ptr(), st) == -1          # k > 256
    assert lib.ctg_cgs2_noalloc(W.data_ptr(), 4980740, 4980740, 1, q.data_ptr(),
                                w.data_ptr(), h.data_ptr(), st) == -1   # L too long
