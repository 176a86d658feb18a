"""The C-ABI library builds, loads and exports every function declared in
include/start.h; host-only entry points behave (no GPU needed)."""
import ctypes as C
import os
import re

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
