"""Full-size structure and Gamma checks in the launch configuration bench.py
uses.

Bit-exact against the oracle, for every particle: the frame, Morton keys,
sort orders, the three octrees (structure, FP64 cubes and luminosities,
float32 centres), the neighbour sets, and every target's interaction list
(Eqs. con1, con2), compared through 64-bit FNV-1a checksums of whole rows
because the lists hold 1e8 to 3e9 entries.  Workloads: the 64^3
multiple-source set at theta = 0.5 and 1.0, and the 128^3 diffuse set (every
particle emitting) at theta = 0.7.  Gamma: 1024 sampled targets of the 64^3
set at theta = 0.5 and 1.0 within |dG| <= 1e-4 G + G_abs.
"""
import numpy as np
import pytest

import oracle
from start_inputs import MYR_S, SIGMA_CM2, config2, config3

pytestmark = pytest.mark.gpu

G_ABS = 1e-8 / (SIGMA_CM2 * MYR_S)
PTREE_LEAF = 16


@pytest.fixture(scope="module")
def S():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1005_5312_gb300 as S
    S.build()
    return S


def _mix(k):
    """splitmix64's finaliser on uint64 arrays (wrapping arithmetic)."""
    x = (np.asarray(k, np.uint64) + np.uint64(0x9E3779B97F4A7C15))
    x = (x ^ (x >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
    x = (x ^ (x >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return x ^ (x >> np.uint64(31))


def _row_sums(off, vals):
    """Per-row wrapping sums of vals over the CSR rows off."""
    cs = np.zeros(len(vals) + 1, np.uint64)
    np.cumsum(vals, dtype=np.uint64, out=cs[1:])
    off = np.asarray(off, np.int64)
    return cs[off[1:]] - cs[off[:-1]]


def _same_neighbour_sets(ctx, orc):
    og, ig = ctx.neighbors()
    oo, io = orc.neighbours()
    assert np.array_equal(og.astype(np.int64), oo)
    # rows are sets (the library's rows are in any order): compare two
    # order-independent sums of mixed indices per row
    for salt in (0, 0x5A5A5A5A5A5A5A5A):
        a = _row_sums(og, _mix(ig.astype(np.uint64) ^ np.uint64(salt)))
        b = _row_sums(oo, _mix(io.astype(np.uint64) ^ np.uint64(salt)))
        assert np.array_equal(a, b)


def _same_structure(ctx, orc, trees):
    lo_g, side_g = ctx.frame()
    lo_o, side_o = orc.frame()
    assert np.array_equal(lo_g, lo_o) and side_g == side_o
    for which in (0, 1):
        assert np.array_equal(ctx.keys(which), orc.keys(which))
        assert np.array_equal(ctx.perm(which).astype(np.int64), orc.perm(which))
    for which in trees:
        tg, to = ctx.tree(which), orc.tree(which)
        assert len(tg["level"]) == len(to["level"]), which
        for k in ("level", "first", "count", "skip", "leaf"):
            assert np.array_equal(tg[k].astype(np.int64), to[k].astype(np.int64)), (which, k)
        assert np.array_equal(tg["cube"], to["cube"]), which
        if which != 0:
            assert np.array_equal(tg["L"], to["L"]), which
            assert np.array_equal(tg["cen"], to["cen"]), which
    _same_neighbour_sets(ctx, orc)


def _same_lists(ctx, orc, theta):
    hg, cg = ctx.list_hashes(theta)
    ho, co = orc.list_hashes(theta)
    assert np.array_equal(cg.astype(np.int64), co)
    bad = np.nonzero(hg != ho)[0]
    assert len(bad) == 0, f"{len(bad)} rows differ, first {bad[:5]}"
    return int(co.sum())


@pytest.fixture(scope="module")
def cfg2():
    return config2()


def test_config2_structure_and_every_list_bitexact(S, cfg2):
    w = cfg2
    ctx = S.Context(ptree_leaf=PTREE_LEAF)
    ctx.build_trees(w.pos, w.h, w.src_pos, w.src_L)
    orc = oracle.Oracle.from_workload(w, ptree_leaf=PTREE_LEAF)
    _same_structure(ctx, orc, trees=(0, 1))
    for theta in (0.5, 1.0):
        n = _same_lists(ctx, orc, theta)
        assert n > 10 * w.n_p
    ctx.close()


@pytest.mark.parametrize("theta", [0.5, 1.0])
def test_config2_gamma_1024_sampled_targets(S, cfg2, theta):
    """The benchmark's launch configuration (memoised march, two lanes per
    later hop, default chunking) on the neutral start."""
    w = cfg2
    ctx = S.Context(march_group=2)
    ctx.build_trees(w.pos, w.h, w.src_pos, w.src_L)
    nHI = w.n_HI()
    g = np.zeros(w.n_p, np.float32)
    ctx.rt_solve(theta, n_HI=nHI, gamma_out=g)
    orc = oracle.Oracle.from_workload(w, ptree_leaf=PTREE_LEAF)
    idx = np.random.default_rng(11 + int(10 * theta)).choice(w.n_p, 1024, replace=False)
    ref = orc.gamma(nHI, theta, targets=idx)
    err = np.abs(g[idx].astype(np.float64) - ref)
    tol = 1e-4 * np.abs(ref) + G_ABS
    assert np.all(err <= tol), (int((err > tol).sum()), float((err / tol).max()))
    ctx.close()


def test_config3_diffuse_structure_and_every_list_bitexact(S):
    w = config3()
    ctx = S.Context(ptree_leaf=PTREE_LEAF)
    ctx.build_trees(w.pos, w.h, w.src_pos, w.src_L, w.V, diffuse=True)
    ctx.set_state(w.n_H, w.y0)
    orc = oracle.Oracle.from_workload(w, ptree_leaf=PTREE_LEAF)
    orc.set_emitters(w.y0, w.n_H)
    n = _same_lists(ctx, orc, 0.7)
    assert n > 100 * w.n_p
    _same_structure(ctx, orc, trees=(0, 1, 2))
    ctx.close()
