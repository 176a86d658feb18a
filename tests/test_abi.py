"""The C-ABI library builds, loads and exports every function declared in
include/start.h; host-only entry points behave (no GPU needed)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "start.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(start_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libstart():
    from paper_1005_5312_gb300._build_lib import build
    path = build()
    return C.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("start_build_trees", "start_rt_solve", "start_ionize", "start_rt_solve_oneshot",
              "start_create", "start_destroy", "start_set_state", "start_get_lists"):
        assert n in names


def test_library_exports_every_declared_symbol(libstart):
    missing = [n for n in _declared() if not hasattr(libstart, n)]
    assert not missing, missing


def test_default_params_and_status_strings(libstart):
    import paper_1005_5312_gb300 as S
    p = S.default_params()
    assert p.src_leaf == 1 and p.sigma_cm2 == 6.3e-18 and p.len_unit_cm == 3.0857e21
    assert p.tau_cut == 110.0 and p.march_group == 2 and p.march_mode == 1
    L = S.lib()
    assert L.start_status_string(S.START_EINVAL) == b"START_EINVAL"
    assert L.start_status_string(S.START_ECHAIN) == b"START_ECHAIN"
    assert L.start_default_params(None) == S.START_EINVAL


def test_create_rejects_bad_params_before_touching_the_device(libstart):
    import paper_1005_5312_gb300 as S
    L = S.lib()
    h = C.c_void_p()
    for bad in (dict(src_leaf=0), dict(sigma_cm2=-1.0), dict(march_group=7), dict(tau_cut=0.0)):
        p = S.default_params(**bad)
        assert L.start_create(C.byref(h), C.byref(p)) == S.START_EINVAL
    assert L.start_create(None, None) == S.START_EINVAL
    # NULL contexts are rejected, never dereferenced
    assert L.start_destroy(None) == S.START_EINVAL
    assert L.start_rt_solve(None, None, C.c_float(0.5), None) == S.START_EINVAL
    assert L.start_last_error(None) == b"NULL context"


def test_params_struct_layout_matches_header():
    import paper_1005_5312_gb300 as S
    src = open(HEADER).read()
    body = src[src.index("typedef struct start_params"):src.index("} start_params;")]
    fields = re.findall(r"\b(?:int|double|long long|void \*)\s*\**\s*([a-zA-Z_0-9]+);", body)
    assert [f for f, _ in S.StartParams._fields_] == fields


def test_stats_struct_layout_and_phases_match_header():
    import paper_1005_5312_gb300 as S
    src = open(HEADER).read()
    body = src[src.index("typedef struct start_stats"):src.index("} start_stats;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"\blong long\s+([a-zA-Z_0-9]+);", body)
    assert [f for f, _ in S.StartStats._fields_] == fields
    n = int(re.search(r"#define START_NPHASES (\d+)", src).group(1))
    assert len(S.Context.PHASES) == n


def _bins_by_rule(d, N):
    """The binning rule of start_direction_bins, written from its description."""
    a = np.argmax(np.abs(d), axis=1)
    neg = d[np.arange(len(d)), a] < 0
    f = 2 * a + neg
    m = np.abs(d[np.arange(len(d)), a])
    others = {0: (1, 2), 1: (2, 0), 2: (0, 1)}
    s = np.empty(len(d))
    t = np.empty(len(d))
    for ax, (i, j) in others.items():
        k = a == ax
        s[k] = d[k, i]
        t[k] = d[k, j]
    iu = np.clip(np.floor((s / m + 1.0) * N / 2.0), 0, N - 1).astype(int)
    iv = np.clip(np.floor((t / m + 1.0) * N / 2.0), 0, N - 1).astype(int)
    return (f * N + iu) * N + iv


@pytest.mark.parametrize("N", [2, 3, 4, 5, 6])
def test_direction_bin_cones_contain_their_bins(libstart, N):
    """Every sampled direction lies within its bin's cone (the pruning of
    the upstream search is exact only if it does), and the cones are tight:
    the farthest sampled direction of every bin is within a few degrees of
    the cone's edge."""
    import paper_1005_5312_gb300 as S
    L = S.lib()
    nb = 6 * N * N
    cones = np.zeros(8 * nb, np.float32)
    assert L.start_direction_bins(N, cones.ctypes.data_as(C.POINTER(C.c_float))) == S.START_OK
    cones = cones.reshape(nb, 8).astype(np.float64)
    axis, cr, sr, rho = cones[:, :3], cones[:, 3], cones[:, 4], cones[:, 5]
    assert np.allclose(np.linalg.norm(axis, axis=1), 1.0, atol=1e-6)
    assert np.allclose(np.cos(rho), cr, atol=1e-6) and np.allclose(np.sin(rho), sr, atol=1e-6)
    rng = np.random.default_rng(N)
    d = rng.normal(size=(400000, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    # plus the bins' corners and edges, where the cone is tightest
    g = np.linspace(-1.0, 1.0, 2 * N + 1)
    u, v = np.meshgrid(g, g)
    face = np.stack([np.ones(u.size), u.ravel(), v.ravel()], axis=1)
    extra = np.concatenate([np.roll(sg * face, r, axis=1) for r in range(3) for sg in (1, -1)])
    d = np.concatenate([d, extra / np.linalg.norm(extra, axis=1)[:, None]])
    b = _bins_by_rule(d, N)
    ang = np.arccos(np.clip(np.sum(d * axis[b], axis=1), -1.0, 1.0))
    assert np.all(ang <= rho[b] + 1e-6)
    far = np.zeros(nb)
    np.maximum.at(far, b, ang)
    assert np.all(far >= rho - 2e-3 - 0.05)
    assert np.bincount(b, minlength=nb).min() > 0
    assert L.start_direction_bins(1, cones.ctypes.data_as(C.POINTER(C.c_float))) == S.START_EINVAL
    assert L.start_direction_bins(N, None) == S.START_EINVAL
