"""GPU path vs the FP64 oracle on the same seeded inputs.

Bit-exact: frame, Morton keys, sort permutations, octrees (structure, FP64
cubes, FP64 luminosities, float32 centres), neighbour sets, interaction
lists and the number of rays and hops (every upstream choice agrees).
Within tolerance: Gamma (|dG| <= 1e-4 G_ref + G_abs, G_abs = 1e-8 / (sigma
dt), i.e. a flux whose k dt is 1e-8 for dt = 1 Myr) and x_HII (abs 1e-3).
"""
import math

import numpy as np
import pytest

import oracle
from start_inputs import (ALPHA_A, ALPHA_B, KPC_CM, MYR_S, SIGMA_CM2, config1, config2,
                          jittered_lattice, lattice_workload, smoothing_lengths)

pytestmark = pytest.mark.gpu

DT = MYR_S
G_ABS = 1e-8 / (SIGMA_CM2 * DT)
G_REL = 1e-4
X_ABS = 1e-3
PTREE_LEAF = 16
PHYS = dict(sigma_cm2=SIGMA_CM2, len_unit_cm=KPC_CM, alpha_A=ALPHA_A, alpha_B=ALPHA_B)


@pytest.fixture(scope="module")
def S():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1005_5312_gb300 as S
    S.build()
    S.lib()
    return S


def make_pair(S, w, tau_cut=1e30, **over):
    """GPU context and oracle over one workload (same inputs)."""
    ctx = S.Context(tau_cut=tau_cut, ptree_leaf=PTREE_LEAF, **over)
    ctx.build_trees(w.pos, w.h, w.src_pos, w.src_L, w.V if w.diffuse else None, diffuse=w.diffuse)
    orc = oracle.Oracle.from_workload(w, ptree_leaf=PTREE_LEAF,
                                      src_leaf=over.get("src_leaf", 1))
    return ctx, orc


def gamma_close(g, ref):
    g = np.asarray(g, np.float64)
    err = np.abs(g - ref)
    tol = G_REL * np.abs(ref) + G_ABS
    bad = np.nonzero(err > tol)[0]
    assert len(bad) == 0, (f"{len(bad)} targets off; worst i={bad[np.argmax(err[bad] / tol[bad])]}",
                           g[bad[:5]], ref[bad[:5]])


def decode(ent):
    ent = np.asarray(ent, np.int64)
    src = (ent & 0x80000000) != 0
    emit = (ent & 0x40000000) != 0
    ident = ent & 0x3FFFFFFF
    return np.where(src, -(1 + ident), ident), emit


def random_workload(n_p, n_s, seed, box=3.0, dups=0, diffuse=False):
    rng = np.random.default_rng(seed)
    pos = rng.uniform(0, box, size=(3, n_p)).astype(np.float32)
    for d in range(dups):
        pos[:, 2 * d + 1] = pos[:, 2 * d]
    h = smoothing_lengths(pos)
    w = lattice_workload("tmp", 2, 1.0, 0, seed)   # container for the fields
    w.pos, w.h = pos, h
    w.src_pos = rng.uniform(0, box, size=(3, n_s)).astype(np.float32)
    w.src_L = rng.lognormal(np.log(1e48), 1.0, size=n_s)
    w.n_H = np.full(n_p, 1e-3, np.float32)
    w.y0 = rng.uniform(0.0, 1.0, n_p)
    w.V = np.full(n_p, box ** 3 / n_p)
    w.diffuse = diffuse
    w.params["diffuse"] = diffuse
    return w


@pytest.fixture(scope="module")
def cfg1():
    return config1()


@pytest.fixture(scope="module")
def ragged():
    # not a multiple of any tile; two pairs of identical positions
    return random_workload(5003, 77, 11, dups=2)


@pytest.fixture(scope="module")
def clustered():
    # sources in close pairs (1e-5 of the box apart: chains of single-child
    # cells down to the deepest levels), particles in tight clumps
    w = random_workload(3001, 64, 12, dups=3)
    rng = np.random.default_rng(13)
    w.src_pos[:, 1::2] = w.src_pos[:, 0::2] + np.float32(3e-5) * rng.uniform(
        0.1, 1.0, size=(3, 32)).astype(np.float32)
    w.pos[:, 1000:1200] = (w.pos[:, 1000:1001]
                           + np.float32(1e-4) * rng.uniform(0, 1, (3, 200)).astype(np.float32))
    w.h = smoothing_lengths(w.pos)
    return w


# ------------------------------------------------------------------ structure
@pytest.mark.parametrize("which_w", ["cfg1", "ragged", "clustered"])
def test_frame_keys_perm_trees_neighbours_bitexact(S, which_w, request):
    w = request.getfixturevalue(which_w)
    ctx, orc = make_pair(S, w)
    lo_g, side_g = ctx.frame()
    lo_o, side_o = orc.frame()
    assert np.array_equal(lo_g, lo_o) and side_g == side_o
    for which in (0, 1):
        assert np.array_equal(ctx.keys(which), orc.keys(which))
        assert np.array_equal(ctx.perm(which).astype(np.int64), orc.perm(which))
    for which in (0, 1):
        tg, to = ctx.tree(which), orc.tree(which)
        assert len(tg["level"]) == len(to["level"])
        for k in ("level", "first", "count", "skip", "leaf"):
            assert np.array_equal(tg[k].astype(np.int64), to[k].astype(np.int64)), k
        assert np.array_equal(tg["cube"], to["cube"])
        if which == 1:
            assert np.array_equal(tg["L"], to["L"])
            assert np.array_equal(tg["cen"], to["cen"])
    og, ig = ctx.neighbors()
    oo, io = orc.neighbours()
    assert np.array_equal(og.astype(np.int64), oo)
    for i in range(w.n_p):
        assert sorted(ig[og[i]:og[i + 1]].tolist()) == io[oo[i]:oo[i + 1]].tolist()


@pytest.mark.parametrize("theta", [0.0, 0.5, 1.0])
def test_lists_bitexact(S, cfg1, theta):
    ctx, orc = make_pair(S, cfg1)
    off, ent = ctx.lists(theta)
    dec, emit = decode(ent)
    assert not emit.any()
    for i in range(0, cfg1.n_p, 97):
        assert dec[off[i]:off[i + 1]].tolist() == orc.list(theta, i).tolist()


# ------------------------------------------------------------------ Gamma
def hops_checked(st, ref, mode, counts):
    """The memoised march counts chain links only in the counting form."""
    if mode == 1 and counts == 0:
        assert st["hops"] == -1 and st["max_hops"] == -1
    else:
        assert st["hops"] == ref


MODES = [(0, 0), (1, 0), (1, 1)]   # (march_mode, link_counts)


@pytest.mark.parametrize("mode,counts", MODES)
@pytest.mark.parametrize("theta", [0.0, 0.5, 1.0])
def test_gamma_parity_config1(S, cfg1, theta, mode, counts):
    ctx, orc = make_pair(S, cfg1, march_mode=mode, link_counts=counts)
    nHI = cfg1.n_HI()
    g = np.zeros(cfg1.n_p, np.float32)
    ctx.rt_solve(theta, n_HI=nHI, gamma_out=g)
    ref = orc.gamma(nHI, theta)
    gamma_close(g, ref)
    st = ctx.stats()
    assert st["rays"] == orc.last_stats["rays"]
    hops_checked(st, orc.last_stats["hops"], mode, counts)


@pytest.mark.parametrize("mode,counts", MODES)
@pytest.mark.parametrize("theta", [0.0, 0.7])
def test_gamma_parity_ragged_nonuniform(S, ragged, theta, mode, counts):
    ctx, orc = make_pair(S, ragged, march_mode=mode, link_counts=counts)
    nHI = (ragged.y0 * 1e-3).astype(np.float32)
    g = np.zeros(ragged.n_p, np.float32)
    ctx.rt_solve(theta, n_HI=nHI, gamma_out=g)
    ref = orc.gamma(nHI, theta)
    gamma_close(g, ref)
    st = ctx.stats()
    assert st["rays"] == orc.last_stats["rays"]
    hops_checked(st, orc.last_stats["hops"], mode, counts)


@pytest.mark.parametrize("mode,counts", MODES)
def test_gamma_parity_mixed_neighbour_counts(S, mode, counts):
    """Every other particle has a 1.8x smoothing length (about 190 neighbours
    instead of 32), so the first hop of the memoised march takes both its
    staged path and its global-memory path; two pairs of particles coincide."""
    w = random_workload(3001, 40, 12, dups=2)
    w.h = w.h.copy()
    w.h[::2] *= np.float32(1.8)
    ctx, orc = make_pair(S, w, march_mode=mode, link_counts=counts)
    og, _ = ctx.neighbors()
    cnt = np.diff(og.astype(np.int64))
    assert cnt.max() > 64 and cnt.min() <= 64
    nHI = (w.y0 * 1e-3).astype(np.float32)
    g = np.zeros(w.n_p, np.float32)
    ctx.rt_solve(0.6, n_HI=nHI, gamma_out=g)
    ref = orc.gamma(nHI, 0.6)
    gamma_close(g, ref)
    st = ctx.stats()
    assert st["rays"] == orc.last_stats["rays"]
    hops_checked(st, orc.last_stats["hops"], mode, counts)


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("group", [1, 4, 16, 32])
def test_march_group_is_result_neutral(S, cfg1, group, mode):
    ctx = S.Context(march_group=group, ptree_leaf=PTREE_LEAF, march_mode=mode)
    ctx.build_trees(cfg1.pos, cfg1.h, cfg1.src_pos, cfg1.src_L)
    ref_ctx = S.Context(march_group=8, ptree_leaf=PTREE_LEAF, march_mode=mode)
    ref_ctx.build_trees(cfg1.pos, cfg1.h, cfg1.src_pos, cfg1.src_L)
    nHI = cfg1.n_HI()
    a = np.zeros(cfg1.n_p, np.float32)
    b = np.zeros(cfg1.n_p, np.float32)
    ctx.rt_solve(0.5, n_HI=nHI, gamma_out=a)
    ref_ctx.rt_solve(0.5, n_HI=nHI, gamma_out=b)
    assert np.array_equal(a, b)


def test_memoised_and_per_ray_march_agree(S, cfg1):
    """Same chains, so the same rays and chain links (counted by the counting
    form of the pointer jumping); tau differs only in the order and precision
    of the additions, in either form."""
    nHI = cfg1.n_HI()
    out = {}
    for mode, counts in MODES:
        ctx = S.Context(march_mode=mode, tau_cut=1e30, link_counts=counts)
        ctx.build_trees(cfg1.pos, cfg1.h, cfg1.src_pos, cfg1.src_L)
        g = np.zeros(cfg1.n_p, np.float32)
        ctx.rt_solve(0.5, n_HI=nHI, gamma_out=g)
        out[mode, counts] = (g.astype(np.float64), ctx.stats())
    g0, s0 = out[0, 0]
    for (g1, s1) in (out[1, 0], out[1, 1]):
        assert s0["rays"] == s1["rays"]
        assert 0 < s1["evals"] < s0["evals"] / 5      # the links are shared
        assert s1["evals"] >= s1["rays"] and s1["links"] == s1["evals"]
        assert np.all(np.abs(g1 - g0) <= 2e-5 * np.abs(g0) + G_ABS)
    assert out[1, 1][1]["hops"] == s0["hops"] and out[1, 0][1]["hops"] == -1


@pytest.mark.parametrize("theta,max_pairs", [(0.0, 0), (0.0, 300000), (0.6, 0)])
def test_one_walk_lists_match_the_per_ray_path(S, theta, max_pairs):
    """The memoised march takes its lists from one walk into a scratch row of
    1024 ids per target; longer rows (every row at theta = 0 with 1100
    sources) are walked again into place.  Same rays and chain links as the
    per-ray march (which counts, then fills), Gamma within the summation-order
    tolerance, and the oracle on a few targets."""
    w = lattice_workload("rows-10^3-1100src", 10, 2.0, 1100, 97, L=2e47)
    nHI = w.n_HI()
    out = {}
    for mode in (0, 1):
        ctx = S.Context(march_mode=mode, tau_cut=1e30, ptree_leaf=PTREE_LEAF,
                        max_pairs=max_pairs, link_counts=1)
        ctx.build_trees(w.pos, w.h, w.src_pos, w.src_L)
        g = np.zeros(w.n_p, np.float32)
        ctx.rt_solve(theta, n_HI=nHI, gamma_out=g)
        out[mode] = (g.astype(np.float64), ctx.stats())
    (g0, s0), (g1, s1) = out[0], out[1]
    assert s0["rays"] == s1["rays"] and s0["hops"] == s1["hops"]
    if max_pairs:
        assert s1["chunks"] > 1
    assert np.all(np.abs(g1 - g0) <= 2e-5 * np.abs(g0) + G_ABS)
    orc = oracle.Oracle.from_workload(w, ptree_leaf=PTREE_LEAF)
    idx = np.array([0, 333, 999])
    gamma_close(g1[idx], orc.gamma(nHI, theta, targets=idx))


@pytest.mark.parametrize("mode", [0, 1])
def test_split_solves_are_result_neutral(S, cfg1, mode):
    """A solve larger than max_pairs is split: the per-ray march into chunks
    of targets (Gamma bitwise the same), the memoised march into groups of
    virtual sources, which share every chain link and leave only the
    method's boundary links outside the lists (the same rays, chain links and
    evaluations as one piece; Gamma's additions grouped differently)."""
    nHI = cfg1.n_HI()
    out = []
    for max_pairs in (0, 20000):
        ctx = S.Context(march_mode=mode, max_pairs=max_pairs)
        ctx.build_trees(cfg1.pos, cfg1.h, cfg1.src_pos, cfg1.src_L)
        g = np.zeros(cfg1.n_p, np.float32)
        ctx.rt_solve(0.5, n_HI=nHI, gamma_out=g)
        out.append((g, ctx.stats()))
    (g0, s0), (g1, s1) = out
    assert s0["chunks"] == 1 and s1["chunks"] > 10
    assert s0["rays"] == s1["rays"] and s0["hops"] == s1["hops"]
    if mode == 0:
        assert np.array_equal(g0, g1)
    else:
        assert s0["evals"] == s1["evals"]
        assert np.all(np.abs(g1.astype(np.float64) - g0) <= 2e-5 * np.abs(g0) + G_ABS)
        ctx = S.Context(march_mode=1, max_pairs=20000)      # deterministic
        ctx.build_trees(cfg1.pos, cfg1.h, cfg1.src_pos, cfg1.src_L)
        g2 = np.zeros(cfg1.n_p, np.float32)
        ctx.rt_solve(0.5, n_HI=nHI, gamma_out=g2)
        assert np.array_equal(g1, g2)


def test_grouped_diffuse_band_and_h2_match_one_piece(S):
    """Groups of virtual sources over both trees (point sources and
    emitters), with the recombination band and its photoheating carried from
    group to group, and the H2 column solve: the same rays, links and
    evaluations as one piece, results within the summation-order tolerance;
    the oracle on sampled targets."""
    w = random_workload(6001, 9, 14, diffuse=True)
    out = {}
    for max_pairs in (0, 40000):
        ctx = S.Context(max_pairs=max_pairs, T_rec=1e4, T_eff=5e4, ptree_leaf=PTREE_LEAF)
        ctx.build_trees(w.pos, w.h, w.src_pos, w.src_L, w.V, diffuse=True)
        ctx.set_state(w.n_H, w.y0)
        g = np.zeros(w.n_p, np.float32)
        ctx.rt_solve(0.6, gamma_out=g)
        st = ctx.stats()
        heat = ctx.heating()
        k = np.zeros(w.n_p, np.float32)
        ctx.h2_dissociation(np.full(w.n_p, 1e-4, np.float32), 0.6, 1e-21, k)
        out[max_pairs] = (g.astype(np.float64), heat.astype(np.float64), k.astype(np.float64), st)
    (g0, h0, k0, s0), (g1, h1, k1, s1) = out[0], out[40000]
    assert s0["chunks"] == 1 and s1["chunks"] > 3
    assert s0["rays"] == s1["rays"] and s0["hops"] == s1["hops"] and s0["evals"] == s1["evals"]
    assert np.all(np.abs(g1 - g0) <= 2e-5 * np.abs(g0) + G_ABS)
    assert np.all(np.abs(h1 - h0) <= 2e-5 * np.abs(h0) + 1e-30)
    assert np.all(np.abs(k1 - k0) <= 2e-5 * np.abs(k0) + 1e-30)
    orc = oracle.Oracle.from_workload(w, ptree_leaf=PTREE_LEAF, T_rec=1e4)
    orc.set_emitters(w.y0, w.n_H)
    idx = np.arange(0, w.n_p, 397)
    gr, hr = orc.gamma_spectral(w.n_HI(), 0.6, 5e4, targets=idx)
    gamma_close(g1[idx], gr)


def test_resident_chains_reproduce_full_solves(S, cfg1):
    """With static particles the links are reused: a resident step gives the
    Gamma of a full solve (same rays and links; tau summed in chain order)."""
    rng = np.random.default_rng(6)
    full = S.Context(link_counts=1)
    full.build_trees(cfg1.pos, cfg1.h, cfg1.src_pos, cfg1.src_L)
    res = S.Context(reuse_chains=1)
    res.build_trees(cfg1.pos, cfg1.h, cfg1.src_pos, cfg1.src_L)
    for step in range(3):
        nHI = (cfg1.n_H * rng.uniform(0.0, 1.0, cfg1.n_p)).astype(np.float32)
        a = np.zeros(cfg1.n_p, np.float32)
        b = np.zeros(cfg1.n_p, np.float32)
        full.rt_solve(0.5, n_HI=nHI, gamma_out=a)
        res.rt_solve(0.5, n_HI=nHI, gamma_out=b)
        sf, sr = full.stats(), res.stats()
        assert sf["rays"] == sr["rays"] and sf["hops"] == sr["hops"]
        if step > 0:
            assert sr["evals"] == 0          # no neighbour list evaluated
        assert np.all(np.abs(b.astype(np.float64) - a) <= 2e-5 * np.abs(a) + G_ABS), step
    # a different theta, then new geometry: full solves again, still right
    g = np.zeros(cfg1.n_p, np.float32)
    res.rt_solve(1.0, n_HI=cfg1.n_HI(), gamma_out=g)
    assert res.stats()["evals"] > 0
    w2 = lattice_workload("other", 16, 3.0, 5, 31)
    res.build_trees(w2.pos, w2.h, w2.src_pos, w2.src_L)
    orc = oracle.Oracle.from_workload(w2, ptree_leaf=PTREE_LEAF)
    for _ in range(2):
        g2 = np.zeros(w2.n_p, np.float32)
        res.rt_solve(0.5, n_HI=w2.n_HI(), gamma_out=g2)
        gamma_close(g2, orc.gamma(w2.n_HI(), 0.5))


def test_resident_coupled_steps_match_oracle(S, cfg1):
    ctx, orc = make_pair(S, cfg1, reuse_chains=1)
    ctx.set_state(cfg1.n_H, cfg1.y0)
    y_ref = cfg1.y0.copy()
    y_gpu = np.zeros(cfg1.n_p)
    for step in range(5):
        ctx.rt_solve(0.5)
        ctx.ionize(DT, y_out=y_gpu)
        _, y_ref = orc.step(y_ref, cfg1.n_H, 0.5, DT)
        assert np.max(np.abs(y_gpu - y_ref)) <= X_ABS, step


def test_single_source_theta_independent_on_gpu(S):
    w = lattice_workload("one", 12, 2.0, 1, 5)
    ctx = S.Context()
    ctx.build_trees(w.pos, w.h, w.src_pos, w.src_L)
    nHI = np.random.default_rng(0).uniform(0, 2e-3, w.n_p).astype(np.float32)
    outs = []
    for th in (0.0, 0.5, 1.0, 3.0):
        g = np.zeros(w.n_p, np.float32)
        ctx.rt_solve(th, n_HI=nHI, gamma_out=g)
        outs.append(g)
    for g in outs[1:]:
        assert np.array_equal(g, outs[0])


def test_device_and_host_pointers_agree(S, cfg1):
    import torch
    ctx = S.Context()
    ctx.build_trees(torch.from_numpy(cfg1.pos).cuda(), torch.from_numpy(cfg1.h).cuda(),
                    torch.from_numpy(cfg1.src_pos).cuda(), torch.from_numpy(cfg1.src_L).cuda())
    nHI = cfg1.n_HI()
    gd = torch.zeros(cfg1.n_p, dtype=torch.float32, device="cuda")
    ctx.rt_solve(0.5, n_HI=torch.from_numpy(nHI).cuda(), gamma_out=gd)
    torch.cuda.synchronize()
    ctx2 = S.Context()
    ctx2.build_trees(cfg1.pos, cfg1.h, cfg1.src_pos, cfg1.src_L)
    gh = np.zeros(cfg1.n_p, np.float32)
    ctx2.rt_solve(0.5, n_HI=nHI, gamma_out=gh)
    assert np.array_equal(gd.cpu().numpy(), gh)


def test_oneshot_matches_context(S, cfg1):
    nHI = cfg1.n_HI()
    a = np.zeros(cfg1.n_p, np.float32)
    S.start_rt_solve_oneshot(cfg1.pos, cfg1.h, cfg1.n_p, nHI, cfg1.src_pos, cfg1.src_L,
                             cfg1.n_s, 0.5, a)
    ctx = S.Context()
    ctx.build_trees(cfg1.pos, cfg1.h, cfg1.src_pos, cfg1.src_L)
    b = np.zeros(cfg1.n_p, np.float32)
    ctx.rt_solve(0.5, n_HI=nHI, gamma_out=b)
    assert np.array_equal(a, b)


# ------------------------------------------------------------------ ionisation
def test_ionize_parity_and_coupled_steps(S, cfg1):
    ctx, orc = make_pair(S, cfg1)
    ctx.set_state(cfg1.n_H, cfg1.y0)
    y_ref = cfg1.y0.copy()
    y_gpu = np.zeros(cfg1.n_p)
    for step in range(4):
        g = np.zeros(cfg1.n_p, np.float32)
        ctx.rt_solve(0.5, gamma_out=g)
        ctx.ionize(DT, y_out=y_gpu)
        g_ref, y_ref = orc.step(y_ref, cfg1.n_H, 0.5, DT)
        assert np.max(np.abs(y_gpu - y_ref)) <= X_ABS, step
    # open loop: the same Gamma gives the same update to rounding
    ctx.set_state(cfg1.n_H, cfg1.y0)
    ctx.rt_solve(0.5, gamma_out=g)
    ctx.ionize(DT, y_out=y_gpu)
    y_o, _ = orc.ionize(g.astype(np.float64), cfg1.n_H, cfg1.y0, DT)
    assert np.max(np.abs(y_gpu - y_o)) < 1e-12


# ------------------------------------------------------------------ diffuse
@pytest.fixture(scope="module")
def diffuse_w():
    w = lattice_workload("diffuse-12^3", 12, 2.0, 2, 17, L=3e50, diffuse=True)
    rng = np.random.default_rng(4)
    w.y0 = rng.uniform(0.0, 1.0, w.n_p)
    w.n_H = (10 ** rng.uniform(-3.5, -1.5, w.n_p)).astype(np.float32)
    return w


def test_diffuse_emitters_tree_and_gamma(S, diffuse_w):
    w = diffuse_w
    ctx, orc = make_pair(S, w)
    ctx.set_state(w.n_H, w.y0)
    orc.set_emitters(w.y0, w.n_H)
    eL = orc.emitter_L()
    assert np.array_equal(ctx.emitter_L(), (eL / 1e48).astype(np.float32))
    tg, to = ctx.tree(2), orc.tree(2)
    for k in ("level", "first", "count", "skip", "leaf"):
        assert np.array_equal(tg[k].astype(np.int64), to[k].astype(np.int64)), k
    assert np.array_equal(tg["L"], to["L"])
    assert np.array_equal(tg["cen"], to["cen"])
    nHI = w.n_HI()
    for theta in (0.0, 0.7):
        off, ent = ctx.lists(theta)
        dec, emit = decode(ent)
        for i in range(0, w.n_p, 53):
            row = slice(int(off[i]), int(off[i + 1]))
            d, e = dec[row], emit[row]
            assert d[~e].tolist() == orc.list(theta, i, which=1).tolist()
            assert d[e].tolist() == orc.list(theta, i, which=2).tolist()
        g = np.zeros(w.n_p, np.float32)
        ctx.rt_solve(theta, gamma_out=g)
        gamma_close(g, orc.gamma(nHI, theta))
    y = np.zeros(w.n_p)
    ctx.ionize(DT, y_out=y)
    y_ref, _ = orc.ionize(orc.gamma(nHI, 0.7), w.n_H, w.y0, DT)
    assert np.max(np.abs(y - y_ref)) <= X_ABS


# ------------------------------------------------------------------ edge cases
def test_edge_sizes(S):
    rng = np.random.default_rng(9)
    for n_p, n_s in ((1, 1), (2, 0), (33, 1), (40, 3)):
        pos = rng.uniform(0, 1, size=(3, n_p)).astype(np.float32)
        h = np.full(n_p, 0.4, np.float32)
        src = rng.uniform(0, 1, size=(3, n_s)).astype(np.float32)
        L = np.full(n_s, 1e48)
        ctx = S.Context(tau_cut=1e30)
        ctx.build_trees(pos, h, src, L)
        orc = oracle.Oracle(pos, h, src, L, ptree_leaf=PTREE_LEAF, **PHYS)
        nHI = np.full(n_p, 1e-3, np.float32)
        g = np.full(n_p, -1.0, np.float32)
        ctx.rt_solve(0.5, n_HI=nHI, gamma_out=g)
        gamma_close(g, orc.gamma(nHI, 0.5))
    # empty problem
    ctx = S.Context()
    ctx.build_trees(np.zeros((3, 0), np.float32), np.zeros(0, np.float32),
                    np.zeros((3, 0), np.float32), np.zeros(0))
    ctx.rt_solve(0.5, n_HI=np.zeros(0, np.float32), gamma_out=np.zeros(0, np.float32))


def test_invalid_inputs_are_rejected(S, cfg1):
    ctx = S.Context()
    with pytest.raises(S.StartError) as e:
        ctx.rt_solve(0.5, n_HI=cfg1.n_HI(), gamma_out=np.zeros(cfg1.n_p, np.float32))
    assert e.value.code == S.START_ENOTBUILT
    bad = cfg1.pos.copy()
    bad[1, 7] = np.nan
    with pytest.raises(S.StartError) as e:
        ctx.build_trees(bad, cfg1.h, cfg1.src_pos, cfg1.src_L)
    assert e.value.code == S.START_EINVAL
    hb = cfg1.h.copy()
    hb[3] = 0.0
    with pytest.raises(S.StartError) as e:
        ctx.build_trees(cfg1.pos, hb, cfg1.src_pos, cfg1.src_L)
    assert e.value.code == S.START_EINVAL
    ctx.build_trees(cfg1.pos, cfg1.h, cfg1.src_pos, cfg1.src_L)
    with pytest.raises(S.StartError) as e:
        ctx.rt_solve(-0.1, n_HI=cfg1.n_HI(), gamma_out=np.zeros(cfg1.n_p, np.float32))
    assert e.value.code == S.START_EINVAL
    nb = cfg1.n_HI()
    nb[0] = -1.0
    with pytest.raises(S.StartError) as e:
        ctx.rt_solve(0.5, n_HI=nb, gamma_out=np.zeros(cfg1.n_p, np.float32))
    assert e.value.code == S.START_EINVAL
    # the context stays usable after rejected calls
    g = np.zeros(cfg1.n_p, np.float32)
    ctx.rt_solve(0.5, n_HI=cfg1.n_HI(), gamma_out=g)
    assert np.all(np.isfinite(g)) and g.max() > 0


@pytest.mark.parametrize("mode", [0, 1])
def test_hop_cap_reports_echain(S, cfg1, mode):
    ctx = S.Context(hop_cap=2, tau_cut=1e30, march_mode=mode)
    ctx.build_trees(cfg1.pos, cfg1.h, cfg1.src_pos, cfg1.src_L)
    with pytest.raises(S.StartError) as e:
        ctx.rt_solve(0.5, n_HI=cfg1.n_HI(), gamma_out=np.zeros(cfg1.n_p, np.float32))
    assert e.value.code == S.START_ECHAIN


@pytest.mark.parametrize("diffuse", [False, True])
def test_warp_cooperative_walk_is_result_neutral(S, cfg1, diffuse):
    """One traversal per warp of 32 targets (walk_warp = 1) and one per thread
    give the same interaction lists (checksums), the same rays and chain
    links and bitwise the same Gamma, also when a split solve restricts the
    walks to groups of virtual sources."""
    w = random_workload(4001, 33, 21, diffuse=True) if diffuse else cfg1
    out = []
    for ww in (0, 1):
        for max_pairs in (0, 60000):
            ctx = S.Context(walk_warp=ww, max_pairs=max_pairs, ptree_leaf=PTREE_LEAF)
            ctx.build_trees(w.pos, w.h, w.src_pos, w.src_L, w.V if diffuse else None,
                            diffuse=diffuse)
            ctx.set_state(w.n_H, w.y0)
            g = np.zeros(w.n_p, np.float32)
            ctx.rt_solve(0.6, gamma_out=g)
            out.append((ww, max_pairs, g, ctx.stats(), ctx.list_hashes(0.6)))
    for ww, mp, g, st, (hs, cnt) in out[2:]:
        ref = out[0] if mp == 0 else out[1]
        assert np.array_equal(hs, ref[4][0]) and np.array_equal(cnt, ref[4][1])
        assert st["rays"] == ref[3]["rays"] and st["hops"] == ref[3]["hops"]
        assert np.array_equal(g, ref[2])


@pytest.mark.parametrize("which", ["cfg1", "ragged", "diffuse"])
def test_first_hop_direction_bins_are_result_neutral(S, cfg1, ragged, which):
    """The first hop scanning only its direction bin's candidate set
    (row_bins = N) or every staged neighbour (row_bins = 0) makes the same
    upstream choices: the same rays and chain links and bitwise the same
    Gamma, in one piece and split into groups of virtual sources (against
    the same split without bins: a split solve sums Gamma group by group),
    on a ragged set with duplicated positions and on the diffuse case (emitters
    inside the neighbour radius scan every neighbour).  The bins prune: the
    scanned candidates fall below a full scan, and fewer first hops need the
    FP64 re-decision."""
    w = {"cfg1": cfg1, "ragged": ragged,
         "diffuse": random_workload(4001, 33, 22, diffuse=True)}[which]
    diffuse = which == "diffuse"
    res = {}
    for nb in (0, 2, 4, 6):
        for max_pairs in (0, 60000):
            ctx = S.Context(row_bins=nb, max_pairs=max_pairs, ptree_leaf=PTREE_LEAF)
            ctx.build_trees(w.pos, w.h, w.src_pos, w.src_L, w.V if diffuse else None,
                            diffuse=diffuse)
            ctx.set_state(w.n_H, w.y0)
            g = np.zeros(w.n_p, np.float32)
            ctx.rt_solve(0.6, gamma_out=g)
            res[nb, max_pairs] = (g, ctx.stats())
            if max_pairs == 0:   # a second solve reuses the candidate sets
                g2 = np.zeros(w.n_p, np.float32)
                ctx.rt_solve(0.6, gamma_out=g2)
                assert np.array_equal(g, g2)
    assert res[0, 0][1]["rays"] > 0
    for (nb, mp), (g, st) in res.items():
        ref_g, ref_st = res[0, mp]   # a split solve sums Gamma group by group
        assert np.array_equal(g, ref_g), (nb, mp)
        assert st["rays"] == ref_st["rays"] and st["hops"] == ref_st["hops"], (nb, mp)
        assert 0 < st["first_hop_scanned"] <= st["first_hop_full"], (nb, mp)
        if nb == 0:
            assert st["first_hop_scanned"] == st["first_hop_full"]
        else:
            assert st["first_hop_scanned"] < st["first_hop_full"], (nb, mp)
            assert st["march_fallbacks"] <= res[0, mp][1]["march_fallbacks"], (nb, mp)


def _depth_and_caps(S, w, mode, theta):
    """Solve with no hop cap, then with hop_cap = the longest chain (must pass,
    bitwise the same Gamma) and one less (must report START_ECHAIN)."""
    nHI = w.n_HI()
    ctx = S.Context(tau_cut=1e30, march_mode=mode, ptree_leaf=PTREE_LEAF, link_counts=1)
    ctx.build_trees(w.pos, w.h, w.src_pos, w.src_L)
    g = np.zeros(w.n_p, np.float32)
    ctx.rt_solve(theta, n_HI=nHI, gamma_out=g)
    depth = ctx.stats()["max_hops"]
    assert depth > 2
    ctx.set_params(hop_cap=depth)
    g2 = np.zeros(w.n_p, np.float32)
    ctx.rt_solve(theta, n_HI=nHI, gamma_out=g2)
    assert np.array_equal(g, g2)
    ctx.set_params(hop_cap=depth - 1)
    with pytest.raises(S.StartError) as e:
        ctx.rt_solve(theta, n_HI=nHI, gamma_out=g2)
    assert e.value.code == S.START_ECHAIN
    return depth


@pytest.mark.parametrize("mode", [0, 1])
def test_hop_cap_at_the_longest_chain(S, cfg1, mode):
    """The limit falls where the memoised march follows chains one thread
    each (its tail kernel); both march modes agree on where it lies."""
    _depth_and_caps(S, cfg1, mode, 0.5)


# ------------------------------------------------------------------ full size, sampled
def test_config2_hop_cap_at_the_longest_chain(S):
    """64^3 particles, 1024 sources: the memoised march issues batches of
    frontier levels before its tail; hop_cap at the longest chain passes and
    one less is reported."""
    _depth_and_caps(S, config2(), 1, 1.0)


def test_config2_full_size_sampled_targets(S):
    """64^3 particles and 1024 sources at theta = 0.5 in the launch
    configuration the benchmark uses; the oracle evaluates 48 sampled
    targets one by one."""
    w = config2()
    ctx = S.Context(tau_cut=1e30)
    ctx.build_trees(w.pos, w.h, w.src_pos, w.src_L)
    nHI = w.n_HI()
    g = np.zeros(w.n_p, np.float32)
    ctx.rt_solve(0.5, n_HI=nHI, gamma_out=g)
    orc = oracle.Oracle.from_workload(w, ptree_leaf=PTREE_LEAF)
    idx = np.random.default_rng(1).choice(w.n_p, 48, replace=False)
    gamma_close(g[idx], orc.gamma(nHI, 0.5, targets=idx))
    # the per-ray march, with its early stop of opaque rays
    ctx2 = S.Context(march_mode=0)
    ctx2.build_trees(w.pos, w.h, w.src_pos, w.src_L)
    g2 = np.zeros(w.n_p, np.float32)
    ctx2.rt_solve(0.5, n_HI=nHI, gamma_out=g2)
    gamma_close(g2[idx], orc.gamma(nHI, 0.5, targets=idx))
