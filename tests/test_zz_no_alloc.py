"""The allocation-free Morton ordering against start_build_trees.

Callers that own all device memory (their own pool, or a fixed budget) use
start_morton_order_noalloc, whose scratch is a fixed array inside the
library.  Its keys, order and frame must equal what the regular path
computes for the same particles, on consecutive calls that reuse the shared
scratch.  This file is collected last so that a failure here leaves every
other test already run.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _regular(S, pos):
    n = pos.shape[1]
    ctx = S.Context()
    ctx.build_trees(pos, np.full(n, 0.05, np.float32), np.zeros((3, 0), np.float32), np.zeros(0))
    lo, side = ctx.frame()
    return ctx.keys(0), ctx.perm(0), np.array([*lo, side])


def test_noalloc_matches_build_trees_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1005_5312_gb300 as S
    S.build()
    L = S.lib()
    rng = np.random.default_rng(21)
    # two calls in a row with different sizes (the second smaller and ragged)
    # so that stale scratch contents from the first would show
    for n, box in ((70001, 5.0), (4099, 0.7)):
        pos = rng.uniform(-box, box, size=(3, n)).astype(np.float32)
        pos[:, 5] = pos[:, 4]                       # equal keys keep input order
        d_pos = torch.from_numpy(pos).cuda()
        d_keys = torch.zeros(n, dtype=torch.uint64, device="cuda")
        d_perm = torch.zeros(n, dtype=torch.int32, device="cuda")
        d_frame = torch.zeros(4, dtype=torch.float64, device="cuda")
        rc = L.start_morton_order_noalloc(C.c_void_p(d_pos.data_ptr()), n,
                                          C.c_void_p(d_keys.data_ptr()),
                                          C.c_void_p(d_perm.data_ptr()),
                                          C.c_void_p(d_frame.data_ptr()), None)
        assert rc == S.START_OK
        torch.cuda.synchronize()
        keys, perm, frame = _regular(S, pos)
        assert np.array_equal(d_keys.cpu().numpy().astype(np.uint64), keys)
        assert np.array_equal(d_perm.cpu().numpy().astype(np.uint32), perm)
        assert np.array_equal(d_frame.cpu().numpy(), frame)


def test_noalloc_rejects_oversize_and_host_pointers():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1005_5312_gb300 as S
    L = S.lib()
    d = torch.zeros(12, dtype=torch.float32, device="cuda")
    k = torch.zeros(4, dtype=torch.uint64, device="cuda")
    p = torch.zeros(4, dtype=torch.int32, device="cuda")
    too_many = (1 << 20) + 1
    assert L.start_morton_order_noalloc(C.c_void_p(d.data_ptr()), too_many, C.c_void_p(k.data_ptr()),
                                        C.c_void_p(p.data_ptr()), None, None) == S.START_ERANGE
    host = np.zeros(12, np.float32)
    assert L.start_morton_order_noalloc(C.c_void_p(host.ctypes.data), 4, C.c_void_p(k.data_ptr()),
                                        C.c_void_p(p.data_ptr()), None, None) == S.START_EINVAL


def _noalloc(S, L, torch, pos, with_frame=True):
    n = pos.shape[1]
    d_pos = torch.from_numpy(pos).cuda()
    d_keys = torch.zeros(max(n, 1), dtype=torch.uint64, device="cuda")
    d_perm = torch.zeros(max(n, 1), dtype=torch.int32, device="cuda")
    d_frame = torch.zeros(4, dtype=torch.float64, device="cuda") if with_frame else None
    rc = L.start_morton_order_noalloc(C.c_void_p(d_pos.data_ptr()), n,
                                      C.c_void_p(d_keys.data_ptr()),
                                      C.c_void_p(d_perm.data_ptr()),
                                      C.c_void_p(d_frame.data_ptr()) if with_frame else None,
                                      None)
    torch.cuda.synchronize()
    return rc, d_keys[:n].cpu().numpy().astype(np.uint64), \
        d_perm[:n].cpu().numpy().astype(np.uint32), \
        None if d_frame is None else d_frame.cpu().numpy()


def test_noalloc_small_full_and_invalid_inputs():
    """A set that the regular path sorts in one block (1000 particles), one
    that fills the scratch exactly (2^20 particles), a call without a frame
    output, and a non-finite position (START_EINVAL; the next call is still
    correct)."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1005_5312_gb300 as S
    S.build()
    L = S.lib()
    rng = np.random.default_rng(22)
    for n, box, with_frame in ((1000, 2.0, True), (1 << 20, 5.0, True), (3001, 1.0, False)):
        pos = rng.uniform(-box, box, size=(3, n)).astype(np.float32)
        pos[:, 7] = pos[:, 3]
        rc, keys, perm, frame = _noalloc(S, L, torch, pos, with_frame)
        assert rc == S.START_OK
        k_ref, p_ref, f_ref = _regular(S, pos)
        assert np.array_equal(keys, k_ref)
        assert np.array_equal(perm, p_ref)
        if with_frame:
            assert np.array_equal(frame, f_ref)
    bad = rng.uniform(-1, 1, size=(3, 500)).astype(np.float32)
    bad[1, 123] = np.nan
    rc, _, _, _ = _noalloc(S, L, torch, bad)
    assert rc == S.START_EINVAL
    pos = rng.uniform(-1, 1, size=(3, 777)).astype(np.float32)
    rc, keys, perm, frame = _noalloc(S, L, torch, pos)
    k_ref, p_ref, f_ref = _regular(S, pos)
    assert rc == S.START_OK and np.array_equal(keys, k_ref) and np.array_equal(perm, p_ref)
    assert np.array_equal(frame, f_ref)
