"""Pins of the FP64 oracle against things other than itself: numbers the
paper prints, closed forms, brute force on tiny inputs and invariants.

Each test is chosen so that a plausible mistake in the oracle (a dropped
term, a wrong sign or index, a transposed operand) fails at least one.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from start_inputs import (ALPHA_A, ALPHA_B, KPC_CM, MYR_S, SIGMA_CM2, jittered_lattice,
                          smoothing_lengths)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")
PC_CM = KPC_CM / 1000.0
PHYS = dict(sigma_cm2=SIGMA_CM2, len_unit_cm=KPC_CM, alpha_A=ALPHA_A, alpha_B=ALPHA_B)


def _random_problem(n_p, n_s, seed, box=2.0, dup=False, src_leaf=1, diffuse=False):
    rng = np.random.default_rng(seed)
    pos = rng.uniform(0, box, size=(3, n_p)).astype(np.float32)
    if dup and n_p > 4:
        pos[:, 1] = pos[:, 0]
        pos[:, 3] = pos[:, 2]
    h = smoothing_lengths(pos)
    src = rng.uniform(0, box, size=(3, n_s)).astype(np.float32)
    L = rng.lognormal(np.log(1e48), 1.0, size=n_s)
    V = np.full(n_p, box ** 3 / max(n_p, 1))
    o = oracle.Oracle(pos, h, src, L, V, diffuse=diffuse, src_leaf=src_leaf, **PHYS)
    return o, pos, h, src, L, V


# ---------------------------------------------------------------- constants
def test_paper_constants():
    g = json.load(open(GOLDEN))
    s = g["stromgren_radius"]
    R = (3 * s["N_gamma_per_s"] / (4 * math.pi * s["n_H_cm3"] ** 2 * ALPHA_B)) ** (1 / 3)
    assert round(R / KPC_CM, 1) == s["R_s_kpc"]
    m = g["mean_free_path"]
    assert round(1.0 / (m["n_H_cm3"] * SIGMA_CM2) / PC_CM, 1) == m["L_mfp_pc"]
    t = g["test4_duration"]
    t_rec = 1.0 / (t["n_H_cm3"] * ALPHA_B)
    assert abs(t["t_end_Myr"] * MYR_S / t_rec / t["t_over_trec"] - 1) < t["rel_tol"]
    for key in ("test1_optical_depth", "test2_optical_depth"):
        c = g[key]
        dx_cm = c["box_kpc"] / c["n_side"] * KPC_CM
        assert abs(c["n_H_cm3"] * SIGMA_CM2 * dx_cm / c["tau"] - 1) < c["rel_tol"]


# ---------------------------------------------------------------- keys and trees
def _decode(key):
    q = [0, 0, 0]
    for lev in range(21):
        d = (int(key) >> (3 * lev)) & 7
        q[0] |= ((d >> 2) & 1) << lev
        q[1] |= ((d >> 1) & 1) << lev
        q[2] |= (d & 1) << lev
    return q


@pytest.mark.parametrize("n_p,n_s,seed", [(1, 1, 0), (37, 5, 1), (500, 33, 2), (1000, 200, 3)])
def test_keys_locate_points(n_p, n_s, seed):
    o, pos, h, src, L, V = _random_problem(n_p, n_s, seed, dup=True)
    lo, side = o.frame()
    allp = np.concatenate([pos, src], axis=1).astype(np.float64)
    assert np.array_equal(lo, allp.min(axis=1))
    assert side == (allp.max(axis=1) - allp.min(axis=1)).max()
    cell = side / 2 ** 21
    for which, pts in ((0, pos), (1, src)):
        keys = o.keys(which)
        for i in range(pts.shape[1]):
            q = _decode(keys[i])
            for a in range(3):
                x = float(pts[a, i])
                # the key's finest cell contains the point (clamped at the top edge)
                assert lo[a] + q[a] * cell <= x + 1e-12 * side
                assert x <= lo[a] + (q[a] + 1) * cell + 1e-12 * side


@pytest.mark.parametrize("n_p,n_s,seed", [(2, 1, 0), (300, 17, 4), (2000, 64, 5)])
def test_sort_is_stable_key_order(n_p, n_s, seed):
    o, *_ = _random_problem(n_p, n_s, seed, dup=True)
    for which in (0, 1):
        keys, perm = o.keys(which), o.perm(which)
        assert sorted(perm.tolist()) == list(range(len(keys)))
        ref = np.lexsort((np.arange(len(keys)), keys))
        assert np.array_equal(perm, ref)


def _bruteforce_octree(keys_sorted, leaf):
    """Octree by recursive grouping of the decoded integer coordinates."""
    q = np.array([_decode(k) for k in keys_sorted], dtype=np.int64).reshape(-1, 3)
    nodes = []

    def rec(level, idx):
        nodes.append((level, int(idx[0]), len(idx)))
        if len(idx) <= leaf or level == 21:
            return
        sh = 21 - (level + 1)
        octant = ((q[idx, 0] >> sh) & 1) * 4 + ((q[idx, 1] >> sh) & 1) * 2 + ((q[idx, 2] >> sh) & 1)
        for d in range(8):
            sub = idx[octant == d]
            if len(sub):
                rec(level + 1, sub)

    if len(keys_sorted):
        rec(0, np.arange(len(keys_sorted)))
    return nodes, q


@pytest.mark.parametrize("n_p,n_s,seed,leaf", [(400, 40, 6, 1), (800, 100, 7, 8), (64, 3, 8, 1)])
def test_tree_matches_bruteforce_and_invariants(n_p, n_s, seed, leaf):
    o, pos, *_ = _random_problem(n_p, n_s, seed, dup=True, src_leaf=leaf)
    lo, side = o.frame()
    for which, keys, perm, pts in ((1, o.keys(1), o.perm(1), o.src_pos), (0, o.keys(0), o.perm(0), o.pos)):
        t = o.tree(which)
        ks = keys[perm]
        lf = leaf if which == 1 else 8
        ref, q = _bruteforce_octree(ks, lf)
        got = list(zip(t["level"].tolist(), t["first"].tolist(), t["count"].tolist()))
        assert got == ref
        n = len(got)
        for i in range(n):
            lev, first, cnt = got[i]
            l = side / 2 ** lev
            assert t["cube"][i, 3] == l
            # members inside the cube
            mem = pts[:, perm[first:first + cnt]].astype(np.float64)
            assert np.all(mem >= t["cube"][i, :3, None] - 1e-9 * side)
            assert np.all(mem <= t["cube"][i, :3, None] + l + 1e-9 * side)
            # skip = end of the subtree in pre-order
            j = i + 1
            while j < n and got[j][0] > lev:
                j += 1
            assert t["skip"][i] == j
            assert t["leaf"][i] == (cnt <= lf or lev == 21)
            if not t["leaf"][i]:
                c, total = i + 1, 0
                while c < t["skip"][i]:
                    total += got[c][2]
                    c = t["skip"][c]
                assert total == cnt


def test_moments():
    o, pos, h, src, L, V = _random_problem(300, 150, 9)
    t = o.tree(1)
    perm = o.perm(1)
    for n in range(len(t["level"])):
        mem = perm[t["first"][n]:t["first"][n] + t["count"][n]]
        Ls = L[mem].sum()
        assert abs(t["L"][n] / Ls - 1) < 1e-13
        c = (src[:, mem].astype(np.float64) * L[mem]).sum(axis=1) / Ls
        if t["count"][n] == 1:
            assert np.array_equal(t["cen"][n], src[:, mem[0]])
        else:
            assert np.allclose(t["cen"][n], c, rtol=0, atol=1e-6 * 2.0)
    assert abs(t["L"][0] / L.sum() - 1) < 1e-13


# ---------------------------------------------------------------- neighbours
@pytest.mark.parametrize("n_p,seed", [(1, 0), (33, 10), (700, 11)])
def test_neighbours_bruteforce(n_p, seed):
    o, pos, h, *_ = _random_problem(n_p, 3, seed, dup=True)
    off, idx = o.neighbours()
    p = pos.astype(np.float64)
    for i in range(n_p):
        d = p - p[:, i:i + 1]
        d2 = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]
        ref = [k for k in range(n_p) if k != i and d2[k] < (2.0 * float(h[i])) ** 2]
        assert idx[off[i]:off[i + 1]].tolist() == ref


# ---------------------------------------------------------------- walk
def _accept_bruteforce(t, p, theta):
    lo = t["cube"][:, :3]
    l = t["cube"][:, 3]
    hi = lo + l[:, None]
    d = np.where(p < lo, lo - p, np.where(p > hi, p - hi, 0.0))
    d2 = (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]
    return l * l <= (theta * theta) * d2


def _expected_list(t, p, theta, self_rank=-1):
    n = len(t["level"])
    acc = _accept_bruteforce(t, p, theta)
    # ancestors by pre-order containment
    out = []
    for i in range(n):
        anc_acc = any(acc[a] for a in range(i) if t["skip"][a] > i and t["first"][a] <= t["first"][i] and a != i
                      and t["level"][a] < t["level"][i])
        if anc_acc:
            continue
        if acc[i]:
            out.append((t["first"][i], 0, i))
        elif t["leaf"][i]:
            for r in range(t["first"][i], t["first"][i] + t["count"][i]):
                if r != self_rank:
                    out.append((r, 1, -(1 + r)))
    out.sort()
    return [e[2] for e in out]


@pytest.mark.parametrize("theta", [0.0, 0.3, 0.5, 1.0, 2.5])
def test_walk_bruteforce_and_partition(theta):
    o, pos, h, src, *_ = _random_problem(200, 60, 12, src_leaf=2)
    t = o.tree(1)
    for i in range(0, 200, 7):
        lst = o.list(theta, i)
        p = pos[:, i].astype(np.float64)
        assert lst.tolist() == _expected_list(t, p, np.float64(np.float32(theta)))
        covered = []
        for e in lst:
            if e >= 0:
                covered += list(range(t["first"][e], t["first"][e] + t["count"][e]))
            else:
                covered.append(-e - 1)
        assert sorted(covered) == list(range(60))
        if theta == 0.0:
            assert lst.tolist() == [-(1 + r) for r in range(60)]


def test_walk_diffuse_excludes_self():
    o, pos, *_ = _random_problem(150, 4, 13, diffuse=True)
    t = o.tree(2)
    rank = np.argsort(o.perm(0))
    for i in range(0, 150, 5):
        lst = o.list(0.7, i, which=2)
        assert lst.tolist() == _expected_list(t, pos[:, i].astype(np.float64), np.float64(np.float32(0.7)),
                                              self_rank=rank[i])
        covered = []
        for e in lst:
            covered += (list(range(t["first"][e], t["first"][e] + t["count"][e])) if e >= 0 else [-e - 1])
        assert sorted(covered) == sorted(set(range(150)) - {rank[i]})


# ---------------------------------------------------------------- march
def _lattice_problem(nside, box, seed, n_s=4):
    rng = np.random.default_rng(seed)
    pos = jittered_lattice(nside, box, rng)
    h = smoothing_lengths(pos)
    src = rng.uniform(0.1 * box, 0.9 * box, size=(3, n_s)).astype(np.float32)
    L = np.full(n_s, 5e48)
    return pos, h, src, L


def _fnv1a64(data: bytes) -> int:
    h = 14695981039346656037
    for b in data:
        h = ((h ^ b) * 1099511628211) & 0xFFFFFFFFFFFFFFFF
    return h


def test_list_hashes_are_fnv1a_of_the_lists():
    """The oracle's whole-row checksums: the 64-bit FNV-1a of the published
    test vectors, then of every row's entries (brute-force-pinned lists)
    encoded as 32-bit words, source tree then emitter tree."""
    assert _fnv1a64(b"") == 0xCBF29CE484222325
    assert _fnv1a64(b"a") == 0xAF63DC4C8601EC8C
    assert _fnv1a64(b"foobar") == 0x85944171F73967E8
    pos, h, src, L = _lattice_problem(6, 2.0, 27, n_s=9)
    n = pos.shape[1]
    V = np.full(n, (2.0 / 6) ** 3)
    for diffuse in (False, True):
        o = oracle.Oracle(pos, h, src, L, V, diffuse=diffuse, **PHYS)
        if diffuse:
            o.set_emitters(np.full(n, 0.5), np.full(n, 1e-3, np.float32))
        for theta in (0.0, 0.6):
            hs, cnt = o.list_hashes(theta)
            for i in range(0, n, 5):
                words = []
                for which in ((1, 2) if diffuse else (1,)):
                    for e in o.list(theta, i, which=which).tolist():
                        w = e if e >= 0 else (0x80000000 | (-e - 1))
                        words.append(w | (0x40000000 if which == 2 else 0))
                data = b"".join(int(w).to_bytes(4, "little") for w in words)
                assert cnt[i] == len(words)
                assert int(hs[i]) == _fnv1a64(data)


def test_march_uniform_closed_form():
    """Uniform n_HI: the trapezoids telescope to tau = sigma n |r_i - r_s|."""
    pos, h, src, L = _lattice_problem(10, 3.0, 20)
    o = oracle.Oracle(pos, h, src, L, **PHYS)
    n = 2.5e-3
    nHI = np.full(pos.shape[1], n, np.float32)
    sig = SIGMA_CM2 * KPC_CM * float(np.float32(n))
    for i in range(0, pos.shape[1], 37):
        for s in range(src.shape[1]):
            tau, hops = o.march(i, src[:, s], nHI)
            r = np.linalg.norm(pos[:, i].astype(np.float64) - src[:, s].astype(np.float64))
            assert abs(tau - sig * r) <= 1e-12 * sig * r + 1e-300
            assert hops >= 1


def test_march_linear_profile_closed_form():
    """n_HI linear in the distance to the source: every trapezoid is exact, so
    tau = sigma [a (r_i - r_e) + b (r_i^2 - r_e^2)/2 + n_e r_e] for the chain's
    end particle e, whatever path the chain takes."""
    pos, h, src, L = _lattice_problem(9, 3.0, 21, n_s=2)
    o = oracle.Oracle(pos, h, src, L, **PHYS)
    sig = SIGMA_CM2 * KPC_CM
    for s in range(2):
        rs = src[:, s].astype(np.float64)
        r = np.linalg.norm(pos.astype(np.float64) - rs[:, None], axis=0)
        a, b = 1e-3, 4e-4
        nHI = (a + b * r).astype(np.float32)
        for i in range(0, pos.shape[1], 29):
            tau, hops, chain = o.march(i, src[:, s], nHI, with_chain=True)
            e = chain[-1]
            assert chain[0] == i and len(chain) == hops
            rr = r[chain]
            assert np.all(np.diff(rr) < 0)        # strictly toward the source
            nn = a + b * rr
            ref = sig * (a * (rr[0] - rr[-1]) + 0.5 * b * (rr[0] ** 2 - rr[-1] ** 2) + nn[-1] * rr[-1])
            assert abs(tau - ref) <= 2e-6 * ref


def test_march_chain_bruteforce():
    """The upstream particle is the closer neighbour with the smallest angle to
    the ray (computed here by arccos), ties to the smaller index."""
    pos, h, src, L = _lattice_problem(7, 2.0, 22, n_s=3)
    o = oracle.Oracle(pos, h, src, L, **PHYS)
    p = pos.astype(np.float64)
    n = p.shape[1]
    nbrs = []
    for i in range(n):
        d2 = ((p - p[:, i:i + 1]) ** 2).sum(axis=0)
        nbrs.append([k for k in range(n) if k != i and d2[k] < (2.0 * float(h[i])) ** 2])
    nHI = np.full(n, 1e-3, np.float32)
    for s in range(3):
        rs = src[:, s].astype(np.float64)
        for i in range(0, n, 11):
            chain = [i]
            j = i
            while True:
                dj = np.linalg.norm(p[:, j] - rs)
                best, bphi = None, None
                for k in nbrs[j]:
                    if np.linalg.norm(p[:, k] - rs) >= dj:
                        continue
                    u, v = rs - p[:, j], p[:, k] - p[:, j]
                    phi = math.acos(max(-1.0, min(1.0, u @ v / (np.linalg.norm(u) * np.linalg.norm(v)))))
                    if best is None or phi < bphi - 1e-12:
                        best, bphi = k, phi
                if best is None:
                    break
                chain.append(best)
                j = best
            _, _, got = o.march(i, src[:, s], nHI, with_chain=True)
            assert got.tolist() == chain


def test_march_equidistant_neighbours_are_not_upstream():
    """Only neighbours strictly closer to the source can be upstream: six
    particles on a sphere around the source (exactly equidistant) each end
    their chain at once with tau = sigma n r."""
    pos = np.array([[1, -1, 0, 0, 0, 0], [0, 0, 1, -1, 0, 0], [0, 0, 0, 0, 1, -1]], np.float32)
    h = np.full(6, 1.5, np.float32)
    o = oracle.Oracle(pos, h, np.zeros((3, 1), np.float32), np.array([1e48]), **PHYS)
    nHI = np.full(6, 1e-3, np.float32)
    for i in range(6):
        tau, hops, chain = o.march(i, np.zeros(3, np.float32), nHI, with_chain=True)
        assert hops == 1 and chain.tolist() == [i]
        assert abs(tau / (SIGMA_CM2 * KPC_CM * float(nHI[0])) - 1) < 1e-15


# ---------------------------------------------------------------- Gamma
def test_gamma_optically_thin_theta0():
    pos, h, src, L = _lattice_problem(8, 2.0, 23, n_s=9)
    L = np.geomspace(1e47, 1e50, 9)
    o = oracle.Oracle(pos, h, src, L, **PHYS)
    n = pos.shape[1]
    g = o.gamma(np.zeros(n, np.float32), 0.0)
    d = pos.astype(np.float64)[:, :, None] - src.astype(np.float64)[:, None, :]
    r2 = (d ** 2).sum(axis=0) * KPC_CM ** 2
    ref = (L[None, :] / (4 * math.pi * r2)).sum(axis=1)
    assert np.allclose(g, ref, rtol=1e-12, atol=0)
    assert o.last_stats["rays"] == n * 9


def test_gamma_uniform_theta0_closed_form():
    pos, h, src, L = _lattice_problem(8, 2.0, 24, n_s=5)
    o = oracle.Oracle(pos, h, src, L, **PHYS)
    n = pos.shape[1]
    nv = np.float32(2e-3)
    g = o.gamma(np.full(n, nv, np.float32), 0.0)
    d = pos.astype(np.float64)[:, :, None] - src.astype(np.float64)[:, None, :]
    r = np.sqrt((d ** 2).sum(axis=0))
    ref = (L[None, :] * np.exp(-SIGMA_CM2 * KPC_CM * float(nv) * r) / (4 * math.pi * (r * KPC_CM) ** 2)).sum(axis=1)
    assert np.allclose(g, ref, rtol=1e-10, atol=0)


def test_gamma_single_source_is_theta_independent():
    """N_s = 1: START coincides with RSPH for every theta (Section 2.2.2)."""
    pos, h, src, L = _lattice_problem(8, 2.0, 25, n_s=1)
    o = oracle.Oracle(pos, h, src, L, **PHYS)
    rng = np.random.default_rng(0)
    nHI = rng.uniform(0, 2e-3, pos.shape[1]).astype(np.float32)
    g0 = o.gamma(nHI, 0.0)
    for th in (0.5, 1.0, 3.0):
        assert np.array_equal(o.gamma(nHI, th), g0)


def test_gamma_theta0_is_bruteforce_rsph():
    """theta = 0: every source individually (Section 2.2.2), i.e. the sum of
    per-source marches."""
    pos, h, src, L = _lattice_problem(7, 2.0, 26, n_s=6)
    o = oracle.Oracle(pos, h, src, L, **PHYS)
    rng = np.random.default_rng(1)
    nHI = rng.uniform(0, 2e-3, pos.shape[1]).astype(np.float32)
    g = o.gamma(nHI, 0.0)
    for i in range(0, pos.shape[1], 13):
        ref = 0.0
        for s in range(6):
            tau, _ = o.march(i, src[:, s], nHI)
            r2 = float(((pos[:, i].astype(np.float64) - src[:, s].astype(np.float64)) ** 2).sum())
            ref += L[s] * math.exp(-tau) / (4 * math.pi * r2 * KPC_CM ** 2)
        assert abs(g[i] / ref - 1) < 1e-12


def test_gamma_theta_error_is_small_in_thin_limit():
    """Optically thin: the virtual source is a monopole, so the error against
    brute force falls with theta (Section 2.2.2)."""
    pos, h, src, L = _lattice_problem(10, 3.0, 27, n_s=40)
    o = oracle.Oracle(pos, h, src, L, **PHYS)
    z = np.zeros(pos.shape[1], np.float32)
    g0 = o.gamma(z, 0.0)
    errs = [np.median(np.abs(o.gamma(z, th) / g0 - 1)) for th in (0.3, 0.6, 1.0)]
    assert errs[0] < errs[1] < errs[2] < 0.05
    assert errs[0] < 5e-3


# ---------------------------------------------------------------- ionisation
def _ionizer(diffuse=False, alpha_B=ALPHA_B, V=None, T_rec=0.0):
    pos = np.zeros((3, 1), np.float32)
    return oracle.Oracle(pos, np.ones(1, np.float32), np.zeros((3, 1), np.float32),
                         np.ones(1), V if V is not None else np.ones(1), sigma_cm2=SIGMA_CM2,
                         len_unit_cm=KPC_CM, alpha_A=ALPHA_A, alpha_B=alpha_B, diffuse=diffuse,
                         T_rec=T_rec)


def test_ionize_limits_and_residual():
    rng = np.random.default_rng(2)
    n = 200
    gam = 10 ** rng.uniform(-2, 8, n)
    nH = (10 ** rng.uniform(-5, 0, n)).astype(np.float32)
    y0 = rng.uniform(0, 1, n)
    dt = MYR_S
    o = _ionizer()
    y1 = np.array([o.ionize(gam[i:i + 1], nH[i:i + 1], y0[i:i + 1], dt)[0][0] for i in range(n)])
    k = SIGMA_CM2 * gam
    res = y1 - y0 - dt * (-k * y1 + ALPHA_B * nH.astype(np.float64) * (1 - y1) ** 2)
    scale = y0 + dt * (k * y1 + ALPHA_B * nH * (1 - y1) ** 2) + 1e-300
    assert np.all(np.abs(res) <= 1e-12 * scale)
    assert np.all((y1 >= 0) & (y1 <= 1))
    # no recombination: y1 = y0 / (1 + k dt)
    o0 = _ionizer(alpha_B=0.0)
    y1a, _ = o0.ionize(gam, nH, y0, dt)
    assert np.allclose(y1a, y0 / (1 + k * dt), rtol=1e-14)
    # no radiation, neutral stays neutral
    y1b, _ = o.ionize(np.zeros(n), nH, np.ones(n), dt)
    assert np.all(np.abs(y1b - 1.0) <= 4e-16)


def test_ionize_equilibrium_and_ode_convergence():
    o = _ionizer()
    nH = np.float32(1e-3)
    gam = 1e5
    k = SIGMA_CM2 * gam
    # equilibrium k y = alpha n (1 - y)^2 reached for dt >> 1/k
    y, _ = o.ionize(np.array([gam]), np.array([nH]), np.array([1.0]), 1e30)
    roots = np.roots([ALPHA_B * float(nH), -(2 * ALPHA_B * float(nH) + k), ALPHA_B * float(nH)])
    yeq = min(r.real for r in roots if 0 <= r.real <= 1)
    assert abs(y[0] / yeq - 1) < 1e-9
    # many small steps follow the exact solution of dx/dt = -alpha n x^2
    x0, T, m = 0.9, 3e15, 4000
    yv = np.array([1 - x0])
    for _ in range(m):
        yv, _ = o.ionize(np.zeros(1), np.array([nH]), yv, T / m)
    x_exact = x0 / (1 + ALPHA_B * float(nH) * x0 * T)
    assert abs((1 - yv[0]) / x_exact - 1) < 1e-3


@pytest.mark.parametrize("T_rec", [0.0, 1e4])
def test_diffuse_self_term_opaque_limit(T_rec):
    """Opaque particle: k_self per volume -> alpha_1 n_e n_p (Section 4.1),
    whether the recombination photons sit at the Lyman limit or fill the band
    of width k T / h."""
    nH = np.float32(1.0)
    y0 = 0.5
    dt = 1e9
    V = np.array([1.0])            # 1 kpc^3: tau_self ~ 1e4
    o = _ionizer(diffuse=True, V=V, T_rec=T_rec)
    y1, _ = o.ionize(np.zeros(1), np.array([nH]), np.array([y0]), dt)
    A = ALPHA_A * float(nH) * dt
    # back out k from the implicit equation
    k = (y0 - y1[0] + A * (1 - y1[0]) ** 2) / (y1[0] * dt)
    a1 = ALPHA_A - ALPHA_B
    x0 = 1 - y0
    assert abs(k * y0 * float(nH) / (a1 * x0 * x0 * float(nH) ** 2) - 1) < 1e-6


def test_diffuse_emitters_thin_theta0_bruteforce():
    pos, h, src, L = _lattice_problem(7, 2.0, 28, n_s=2)
    n = pos.shape[1]
    V = np.full(n, (2.0 / 7) ** 3)
    o = oracle.Oracle(pos, h, src, L, V, diffuse=True, **PHYS)
    rng = np.random.default_rng(3)
    y = rng.uniform(0, 1, n)
    nH = np.full(n, 1e-2, np.float32)
    o.set_emitters(y, nH)
    eL = o.emitter_L()
    a1 = ALPHA_A - ALPHA_B
    ref_L = a1 * ((1 - y) * 1e-2) ** 2 * V * KPC_CM ** 3
    assert np.allclose(eL, ref_L, rtol=1e-6)
    g = o.gamma(np.zeros(n, np.float32), 0.0)
    p = pos.astype(np.float64)
    for i in range(0, n, 17):
        r2 = ((p - p[:, i:i + 1]) ** 2).sum(axis=0) * KPC_CM ** 2
        r2s = ((src.astype(np.float64) - p[:, i:i + 1]) ** 2).sum(axis=0) * KPC_CM ** 2
        m = np.arange(n) != i
        ref = (eL[m] / (4 * math.pi * r2[m])).sum() + (L / (4 * math.pi * r2s)).sum()
        assert abs(g[i] / ref - 1) < 1e-12


def _escape_probability(pt, box, kappa, ndir=200000):
    """(1/4 pi) int exp(-kappa l(Omega)) dOmega for a point inside the cube
    [0, box]^3, l the distance to the cube's surface along Omega (Fibonacci
    directions)."""
    k = np.arange(ndir) + 0.5
    z = 1.0 - 2.0 * k / ndir
    ph = math.pi * (1.0 + 5.0 ** 0.5) * k
    rxy = np.sqrt(1.0 - z * z)
    d = np.stack([rxy * np.cos(ph), rxy * np.sin(ph), z], 1)
    with np.errstate(divide="ignore", invalid="ignore"):
        t = np.where(d > 0, (box - pt) / d, np.where(d < 0, -pt / d, np.inf))
    return float(np.exp(-kappa * t.min(1)).mean())


def diffuse_balance_ratios(nside=24, box=4.0, x=0.5, tau_dx=0.25, seed=41):
    """Radiative equilibrium of a homogeneous emitting and absorbing medium
    (Section 4.1's recombination photons, theta = 0): at an interior point the
    photons absorbed per unit volume, n_HI (sigma Gamma + k_self), equal those
    emitted per unit volume, alpha_1 n_e n_p, less the part that escapes
    through the box's surface.  Returns absorbed / (emitted (1 - P_esc)) at the
    eight particles nearest the centre, P_esc by angular quadrature."""
    dx = box / nside
    rng = np.random.default_rng(seed)
    pos = jittered_lattice(nside, box, rng)
    h = smoothing_lengths(pos)
    n = pos.shape[1]
    V = np.full(n, dx ** 3)
    n_hi = tau_dx / (SIGMA_CM2 * dx * KPC_CM)
    nH = np.full(n, n_hi / (1.0 - x), np.float32)
    y = np.full(n, 1.0 - x)
    o = oracle.Oracle(pos, h, np.zeros((3, 0), np.float32), np.zeros(0), V, diffuse=True, **PHYS)
    o.set_emitters(y, nH)
    d2 = ((pos.T.astype(np.float64) - box / 2) ** 2).sum(1)
    idx = np.argsort(d2)[:8]
    nHI = (y * nH.astype(np.float64)).astype(np.float32)
    g = o.gamma(nHI, 0.0, targets=idx)
    ks, _ = o.self_terms(nH, y)
    n_hi_cm = float(nHI[0])
    absorbed = n_hi_cm * (SIGMA_CM2 * g + ks[idx])
    n_e = x * float(nH[0])
    emitted = (ALPHA_A - ALPHA_B) * n_e * n_e          # per cm^3 and second
    kappa = n_hi_cm * SIGMA_CM2 * KPC_CM               # per length unit
    keep = np.array([1.0 - _escape_probability(pos[:, i].astype(np.float64), box, kappa)
                     for i in idx])
    return absorbed / (emitted * keep)


def test_diffuse_emitters_radiative_equilibrium():
    """Pins the emitters' luminosity N_rec = alpha_1 n_e n_p V (Section 4.1)
    through the transfer itself: a wrong coefficient (alpha_A or alpha_B for
    alpha_1), a missing volume unit, or x instead of x^2 moves the balance by
    a factor of 1.6 or more.  The lattice sum stands for the volume integral
    to about 3 % per target (one particle spacing has tau = 0.25)."""
    rel = diffuse_balance_ratios()
    assert np.all(np.abs(rel - 1.0) < 0.05), rel
    assert abs(rel.mean() - 1.0) < 0.02, rel.mean()


# ---------------------------------------------------------------- Stromgren
@pytest.mark.slow
def test_stromgren_sphere_and_ifront_law():
    """One source at the corner of a 6.6 kpc box (the geometry of Test 4 with
    the source at a corner).  The density is lowered to 1.25e-4 and the
    luminosity scaled so that R_s stays 5.4 kpc while one particle spacing
    has tau ~ 0.5, which resolves the front.  Then: the ionised octant grows
    as R_s (1 - exp(-t/t_rec))^(1/3), settles on R_s (Eq. strom), and in
    equilibrium recombinations balance the emitted photons.  The ionised
    radius is recombination weighted, (3 sum x^2 V / (4 pi/8))^(1/3), which
    is the Stromgren measure for a front of finite width."""
    box, nside = 6.6, 32
    rng = np.random.default_rng(29)
    pos = jittered_lattice(nside, box, rng)
    h = smoothing_lengths(pos)
    src = np.array([[0.0123], [0.0071], [0.0037]], np.float32)
    n = pos.shape[1]
    V = np.full(n, (box / nside) ** 3)
    n_H = 1.25e-4
    L = 5e48 * (n_H / 1e-3) ** 2
    o = oracle.Oracle(pos, h, src, np.array([L]), V, **PHYS)
    nH = np.full(n, n_H, np.float32)
    R_s = (3 * L / (4 * math.pi * n_H ** 2 * ALPHA_B)) ** (1 / 3) / KPC_CM
    assert abs(R_s - 5.39) < 0.01
    t_rec = 1.0 / (n_H * ALPHA_B)
    dt = t_rec / 20
    y = np.full(n, 1 - 1.2e-3)
    for step in range(1, 161):
        _, y = o.step(y, nH, 0.5, dt)
        if step in (40, 80, 160):
            x = 1 - y
            r_ion = (3 * 8 * np.sum(x * x * V) / (4 * math.pi)) ** (1 / 3)
            law = R_s * (1 - math.exp(-step * dt / t_rec)) ** (1 / 3)
            assert abs(r_ion / law - 1) < 0.1, (step, r_ion, law)
    assert abs(r_ion / R_s - 1) < 0.03
    rec = np.sum(ALPHA_B * (n_H * (1 - y)) ** 2 * V * KPC_CM ** 3)
    assert abs(rec / (L / 8) - 1) < 0.06


# ---------------------------------------------------------------- SPH density (Section 2.1)
def test_spline_kernel_is_normalised_with_support_2h():
    """Any SPH kernel integrates to one over its support; the cubic spline's
    support is 2h.  Checked by quadrature for two smoothing lengths."""
    quad = pytest.importorskip("scipy.integrate").quad
    for h in (1.0, 0.37):
        val, err = quad(lambda r: oracle.spline_w(r, h) * 4.0 * math.pi * r * r, 0.0, 2.0 * h,
                        points=[h], epsabs=1e-13, epsrel=1e-13)
        assert abs(val - 1.0) < 1e-10
        assert oracle.spline_w(2.0 * h, h) == 0.0 and oracle.spline_w(3.0 * h, h) == 0.0


def test_spline_kernel_shape():
    """The cubic spline's defining values: W(0) = 1/(pi h^3), W(h) = W(0)/4,
    and W, dW/dq and d2W/dq2 continuous at q = 1 (one-sided differences),
    dW/dq = 0 at q = 0 and q = 2."""
    h = 0.8
    w0 = oracle.spline_w(0.0, h)
    assert w0 == pytest.approx(1.0 / (math.pi * h ** 3), rel=1e-15)
    assert oracle.spline_w(h, h) == pytest.approx(0.25 * w0, rel=1e-15)
    f = lambda q: oracle.spline_w(q * h, h) / w0
    e = 1e-5
    d_lo = (f(1.0 - e) - f(1.0 - 2 * e)) / e
    d_hi = (f(1.0 + 2 * e) - f(1.0 + e)) / e
    assert d_lo == pytest.approx(-0.75, abs=1e-4) and d_hi == pytest.approx(-0.75, abs=1e-4)
    c_lo = (f(1.0 - e) - 2 * f(1.0 - 2 * e) + f(1.0 - 3 * e)) / e ** 2
    c_hi = (f(1.0 + 3 * e) - 2 * f(1.0 + 2 * e) + f(1.0 + e)) / e ** 2
    assert c_lo == pytest.approx(1.5, abs=1e-3) and c_hi == pytest.approx(1.5, abs=1e-3)
    assert abs(f(e) - f(0.0)) < 1e-9 and abs(f(2.0 - e)) < 1e-13


def test_sph_density_isolated_and_pair():
    """One particle alone: rho = m W(0).  Two particles closer than 2h: each
    sees itself and the other, weighted by its own h (Section 2.1)."""
    pos = np.array([[0.1, 0.9], [0.2, 0.2], [0.3, 0.3]], np.float32)
    h = np.array([0.5, 0.2], np.float32)   # 2 h_0 = 1.0 > 0.8 = r; 2 h_1 = 0.4 < r
    o = oracle.Oracle(pos, h, np.zeros((3, 0), np.float32), np.zeros(0), **PHYS)
    m = np.array([2.0, 3.0])
    rho = o.sph_density(m)
    r = float(pos[0, 1]) - float(pos[0, 0])
    q = r / float(h[0])
    w = 0.25 * (2.0 - q) ** 3 / (math.pi * float(h[0]) ** 3)
    assert rho[0] == pytest.approx(2.0 / (math.pi * float(h[0]) ** 3) + 3.0 * w, rel=1e-12)
    assert rho[1] == pytest.approx(3.0 / (math.pi * float(h[1]) ** 3), rel=1e-15)


def test_sph_density_of_a_regular_lattice():
    """On a regular cubic lattice of spacing dx with about 32 neighbours per
    kernel (h ~ 1.06 dx), the SPH estimate reproduces the mean density
    m / dx^3 to well under one per cent away from the edges."""
    pos = jittered_lattice(16, 1.0, np.random.default_rng(0), 0.0)
    h = smoothing_lengths(pos)
    o = oracle.Oracle(pos, h, np.zeros((3, 0), np.float32), np.zeros(0), **PHYS)
    rho = o.sph_density(np.full(pos.shape[1], 1.5))
    dx = 1.0 / 16
    inner = np.all((pos > 3 * dx) & (pos < 1.0 - 3 * dx), axis=0)
    ratio = rho[inner] * dx ** 3 / 1.5
    assert inner.sum() == 1000
    assert np.all(np.abs(ratio - 1.0) < 0.01)
    # mass enters linearly
    rho2 = o.sph_density(np.full(pos.shape[1], 3.0))
    assert np.allclose(rho2, 2.0 * rho, rtol=1e-15)


# ---------------------------------------------------------------- H2 photodissociation (Appendix B)
KDIS_COEF = 1.13e8


def test_h2_self_shielding_function():
    """f_sh(x) = 1 for x <= 1 and x^(-3/4) beyond (Eq. H2ss): continuous at 1."""
    for x, f in ((0.0, 1.0), (0.3, 1.0), (1.0, 1.0), (16.0, 0.125), (1e4, 1e-3), (81.0, 1.0 / 27.0)):
        assert oracle.h2_fsh(x) == pytest.approx(f, rel=1e-15)
    assert oracle.h2_fsh(1.0 + 1e-12) == pytest.approx(1.0, abs=1e-11)


def test_h2_column_is_the_trapezoid_along_a_line():
    """Ten particles on a line at x = 0..9 (2h = 1.5: each sees only its two
    neighbours), a source at x = -0.5: the chain of particle j is j, j-1, ...,
    0, so N_H2 = sum_k (n_k + n_(k-1))/2 + n_0 / 2 in length units (Eq. NH2 and
    the chain-end segment), and k_dis follows from Eq. H2ss."""
    n = 10
    pos = np.zeros((3, n), np.float32)
    pos[0] = np.arange(n, dtype=np.float32)
    h = np.full(n, 0.75, np.float32)
    src = np.array([[-0.5], [0.0], [0.0]], np.float32)
    L = np.array([3e49])
    o = oracle.Oracle(pos, h, src, L, **PHYS)
    nH2 = (1e-7 * (1.0 + np.arange(n))).astype(np.float32)
    kappa = 2.0e-22
    k = o.h2_dissociation(nH2, 0.5, kappa)
    nd = nH2.astype(np.float64)
    for j in range(n):
        col = 0.5 * nd[0] + sum(0.5 * (nd[q] + nd[q - 1]) for q in range(1, j + 1))
        N = col * KPC_CM
        r = (j + 0.5) * KPC_CM
        x = N / 1e14
        f = 1.0 if x <= 1.0 else x ** -0.75
        ref = KDIS_COEF * kappa * 3e49 / (4.0 * math.pi * r * r) * f
        assert k[j] == pytest.approx(ref, rel=1e-12), j
    assert o.last_stats["hops"] == sum(j + 1 for j in range(n))


def test_h2_dissociation_in_a_uniform_medium_and_optically_thin():
    """Uniform n_H2: every chain telescopes, N = n_H2 r (as tau = sigma n r), so
    at theta = 0 k_dis is the direct sum over sources; with n_H2 = 0 there is no
    shielding.  Both against the straight-line closed form."""
    o, pos, h, src, L, V = _random_problem(300, 7, 31, box=2.0)
    d = pos.astype(np.float64)[:, :, None] - src.astype(np.float64)[:, None, :]
    r = np.sqrt((d ** 2).sum(axis=0)) * KPC_CM
    kappa = 1e-21
    for nval in (0.0, 3e-6):
        nH2 = np.full(300, nval, np.float32)
        x = np.float64(np.float32(nval)) * r / 1e14
        f = np.where(x <= 1.0, 1.0, np.maximum(x, 1.0) ** -0.75)
        ref = (KDIS_COEF * kappa * L[None, :] / (4.0 * math.pi * r * r) * f).sum(axis=1)
        k = o.h2_dissociation(nH2, 0.0, kappa)
        assert np.allclose(k, ref, rtol=1e-10, atol=0)
        assert o.h2_dissociation(nH2, 0.0, 2 * kappa) == pytest.approx(2 * k, rel=1e-14)


def test_h2_dissociation_single_source_is_theta_independent():
    o, pos, h, src, L, V = _random_problem(400, 1, 32, box=2.0)
    nH2 = np.random.default_rng(5).uniform(0, 1e-5, 400).astype(np.float32)
    k0 = o.h2_dissociation(nH2, 0.0, 1e-21)
    k1 = o.h2_dissociation(nH2, 1.0, 1e-21)
    assert np.array_equal(k0, k1)


# ---------------------------------------------------------------- multi-frequency sources
HNU_L = 13.6 * 1.602176634e-12
K_B = 1.380649e-16


def _bb_quad(tau, T):
    """F_ion, F_heat by adaptive quadrature (scipy), independent of the
    oracle's fixed-grid rule: blackbody photon spectrum u^2/(e^(a u) - 1) over
    u = nu/nu_L >= 1, cross-section u^-3."""
    quad = pytest.importorskip("scipy.integrate").quad
    a = HNU_L / (K_B * T)
    w = lambda u: u * u / math.expm1(a * u)
    up = 1.0 + 80.0 / a
    brk = [1.0 + k / a for k in (1, 3, 10, 30)] + [max(1.0, tau ** (1.0 / 3.0))]
    brk = sorted(b for b in brk if 1.0 < b < up)
    z = quad(w, 1.0, up, points=brk, limit=400, epsabs=0, epsrel=1e-12)[0]
    fi = quad(lambda u: w(u) * u ** -3 * math.exp(-tau * u ** -3), 1.0, up, points=brk, limit=400,
              epsabs=0, epsrel=1e-12)[0]
    fh = quad(lambda u: w(u) * u ** -3 * (u - 1.0) * math.exp(-tau * u ** -3), 1.0, up,
              points=brk, limit=400, epsabs=0, epsrel=1e-12)[0]
    return fi / z, fh / z


@pytest.mark.parametrize("T", [1e5, 3e4])
def test_spectral_integrals_against_adaptive_quadrature(T):
    for tau in (0.0, 0.3, 3.0, 30.0, 300.0):
        fi, fh = oracle.bb_integrals(tau, T)
        qi, qh = _bb_quad(tau, T)
        assert fi == pytest.approx(qi, rel=1e-8) and fh == pytest.approx(qh, rel=1e-8), tau


def test_spectral_limits_and_hardening():
    """A cool source is nearly monochromatic just above the Lyman limit:
    F_ion(0) = <u^-3> is close to (below) one and F_ion(tau) / F_ion(0) ~
    exp(-tau <u^-3>) (first cumulant of a narrow spectrum); the mean excess
    energy per absorbed photon, F_heat / F_ion, grows with depth (the
    spectrum hardens)."""
    f0 = oracle.bb_integrals(0.0, 2000.0)[0]
    assert 0.9 < f0 < 1.0
    for tau in (0.5, 1.0, 2.0):
        assert oracle.bb_integrals(tau, 2000.0)[0] / f0 == pytest.approx(math.exp(-tau * f0),
                                                                          rel=2e-3)
    assert 0.0 < oracle.bb_integrals(0.0, 1e5)[0] < 1.0
    e = [oracle.bb_integrals(t, 1e5) for t in (0.0, 1.0, 10.0, 100.0, 1000.0)]
    ratio = [fh / fi for fi, fh in e]
    assert all(b > a for a, b in zip(ratio, ratio[1:]))
    assert all(b[0] < a[0] for a, b in zip(e, e[1:]))


def test_spectral_gamma_in_a_uniform_medium():
    """Uniform n_HI at theta = 0: tau_L = sigma n r on every chain, so
    Gamma_eff = sum L F_ion(sigma n r) / (4 pi r^2) and the heating per neutral
    atom sigma h nu_L sum L F_heat / (4 pi r^2), with F from adaptive quadrature."""
    pos, h, src, L = _lattice_problem(8, 2.0, 41, n_s=4)
    o = oracle.Oracle(pos, h, src, L, **PHYS)
    n = np.float32(1e-3)
    nHI = np.full(pos.shape[1], n, np.float32)
    idx = np.array([0, 77, 300, 511])
    g, hh = o.gamma_spectral(nHI, 0.0, 1e5, targets=idx)
    for q, i in enumerate(idx):
        rg, rh = 0.0, 0.0
        for s in range(4):
            r = math.sqrt(sum((float(pos[a, i]) - float(src[a, s])) ** 2 for a in range(3)))
            tau = SIGMA_CM2 * KPC_CM * float(n) * r
            fi, fh = _bb_quad(tau, 1e5)
            flux = L[s] / (4 * math.pi * (r * KPC_CM) ** 2)
            rg += flux * fi
            rh += flux * fh
        assert g[q] == pytest.approx(rg, rel=1e-7)
        assert hh[q] == pytest.approx(SIGMA_CM2 * HNU_L * rh, rel=1e-7)


# ---------------------------------------------------------------- recombination band
def _band_D(T):
    return K_B * T / HNU_L


def _band_quad(tau, T):
    """R_ion, R_heat by adaptive quadrature (scipy): photons spread evenly
    over u = nu/nu_L in [1, 1 + kT/(h nu_L)], cross-section u^-3."""
    quad = pytest.importorskip("scipy.integrate").quad
    D = _band_D(T)
    ri = quad(lambda u: u ** -3 * math.exp(-tau * u ** -3), 1.0, 1.0 + D, epsabs=0,
              epsrel=1e-13, limit=200)[0]
    rh = quad(lambda u: (u - 1.0) * u ** -3 * math.exp(-tau * u ** -3), 1.0, 1.0 + D, epsabs=0,
              epsrel=1e-13, limit=200)[0]
    return ri / D, rh / D


@pytest.mark.parametrize("T", [1e3, 1e4, 3e4])
def test_band_integrals_closed_forms_at_zero_depth(T):
    """Unattenuated: (1/D) int u^-3 du = (1 - (1+D)^-2) / (2D) and
    (1/D) int (u-1) u^-3 du = D / (2 (1+D)^2)."""
    D = _band_D(T)
    ri, rh = oracle.rec_band_integrals(0.0, T)
    assert ri == pytest.approx((1 - (1 + D) ** -2) / (2 * D), rel=1e-12)
    assert rh == pytest.approx(D / (2 * (1 + D) ** 2), rel=1e-10)


@pytest.mark.parametrize("T", [1e4, 5e4])
def test_band_integrals_against_adaptive_quadrature(T):
    for tau in (0.1, 1.0, 10.0, 100.0):
        ri, rh = oracle.rec_band_integrals(tau, T)
        qi, qh = _band_quad(tau, T)
        assert ri == pytest.approx(qi, rel=1e-8) and rh == pytest.approx(qh, rel=1e-8), tau


def test_band_narrow_limit_is_the_lyman_limit_line():
    """A band of vanishing width (T -> 0) is the line at nu_L: R_ion -> e^-tau
    and the mean excess energy per photon R_heat / R_ion -> D / 2."""
    T = 1.0
    D = _band_D(T)
    for tau in (0.0, 0.5, 2.0, 5.0):
        ri, rh = oracle.rec_band_integrals(tau, T)
        assert ri == pytest.approx(math.exp(-tau), rel=1e-4)
        assert rh / ri == pytest.approx(D / 2, rel=1e-4)


def test_band_self_terms_limits():
    """Self terms per neutral atom (Eqs. kself1, gself): an opaque particle
    absorbs its whole band, k_self n_HI -> alpha_1 n_e n_p and the heating
    n_HI -> alpha_1 n_e n_p k T / 2 (the mean excess energy of the band); a
    transparent one gives alpha_1 n_e n_p sigma R times the unattenuated
    band integrals; a narrow band is the line at nu_L."""
    a1 = ALPHA_A - ALPHA_B
    T = 2e4
    D = _band_D(T)
    y0 = np.array([0.3])
    # opaque: tau_s ~ sigma n_HI R = 6.3e-18 * 0.3 * 2e21 ~ 4e3
    o = _ionizer(diffuse=True, V=np.array([1.0]), T_rec=T)
    ks, hs = o.self_terms(np.array([1.0], np.float32), y0)
    nenp = a1 * (0.7 * 1.0) ** 2
    assert ks[0] * 0.3 == pytest.approx(nenp, rel=1e-6)
    assert hs[0] * 0.3 == pytest.approx(nenp * K_B * T / 2, rel=1e-8)
    # transparent: tau_s ~ 6.3e-18 * 0.3e-6 * 3e17 ~ 6e-7
    V = 1e-12
    o = _ionizer(diffuse=True, V=np.array([V]), T_rec=T)
    nH = np.float32(1e-6)
    ks, hs = o.self_terms(np.array([nH]), y0)
    R = (3 * V / (4 * math.pi)) ** (1 / 3) * KPC_CM
    pre = a1 * (0.7 * float(nH)) ** 2 * SIGMA_CM2 * R
    assert ks[0] == pytest.approx(pre * (1 - (1 + D) ** -2) / (2 * D), rel=1e-5)
    assert hs[0] == pytest.approx(pre * HNU_L * D / (2 * (1 + D) ** 2), rel=1e-5)
    # narrow band = line
    for V in (1e-3, 1e-1):
        k0, h0 = _ionizer(diffuse=True, V=np.array([V])).self_terms(np.array([1e-2], np.float32),
                                                                     y0)
        k1, h1 = _ionizer(diffuse=True, V=np.array([V]), T_rec=1.0).self_terms(
            np.array([1e-2], np.float32), y0)
        assert k1[0] == pytest.approx(k0[0], rel=1e-4) and h0[0] == 0.0
        assert 0 < h1[0] < 1e-4 * HNU_L * k1[0]


def test_band_gamma_in_a_uniform_medium():
    """Diffuse emitters with the band, uniform n_HI, theta = 0: every chain
    has tau_L = sigma n r, so the emitters add sum L_j R_ion(sigma n r) /
    (4 pi r^2) to Gamma_eff and sigma h nu_L sum L_j R_heat / (4 pi r^2) to the
    heating (Eq. gother), with R from adaptive quadrature; point sources at
    T_eff = 0 add L e^-tau / (4 pi r^2) and no heating."""
    T = 1e4
    pos, h, src, L = _lattice_problem(5, 1.0, 43, n_s=2)
    n = pos.shape[1]
    V = np.full(n, (1.0 / 5) ** 3)
    o = oracle.Oracle(pos, h, src, L, V, diffuse=True, T_rec=T, **PHYS)
    y = np.full(n, 0.4)
    nH = np.full(n, 2e-2, np.float32)
    o.set_emitters(y, nH)
    eL = o.emitter_L()
    nHI = (y * nH.astype(np.float64)).astype(np.float32)
    nn = float(nHI[0])
    idx = np.array([0, 62, 124])
    g, hh = o.gamma_spectral(nHI, 0.0, 0.0, targets=idx)
    p = pos.astype(np.float64)
    for q, i in enumerate(idx):
        rg, rh = 0.0, 0.0
        for s in range(src.shape[1]):
            r = math.sqrt(sum((p[a, i] - float(src[a, s])) ** 2 for a in range(3)))
            rg += L[s] * math.exp(-SIGMA_CM2 * KPC_CM * nn * r) / (4 * math.pi * (r * KPC_CM) ** 2)
        for j in range(n):
            if j == i:
                continue
            r = math.sqrt(sum((p[a, i] - p[a, j]) ** 2 for a in range(3)))
            ri, rhh = _band_quad(SIGMA_CM2 * KPC_CM * nn * r, T)
            flux = eL[j] / (4 * math.pi * (r * KPC_CM) ** 2)
            rg += flux * ri
            rh += flux * rhh
        assert g[q] == pytest.approx(rg, rel=1e-7)
        assert hh[q] == pytest.approx(SIGMA_CM2 * HNU_L * rh, rel=1e-7)


# ---------------------------------------------------------------- temperature
def _rates_golden():
    with open(os.path.join(os.path.dirname(__file__), "golden", "hydrogen_rates.json")) as f:
        return json.load(f)


def test_recombination_fits_against_published_coefficients():
    g = _rates_golden()["recombination_coefficients"]
    for T, aA, aB in zip(g["T_K"], g["alpha_A"], g["alpha_B"]):
        assert abs(oracle.rate("alpha_B", T) / aB - 1) < g["rel_tol_alpha_B"], T
        assert abs(oracle.rate("alpha_A", T) / aA - 1) < g["rel_tol_alpha_A"], T


def test_collisional_rates_carry_their_threshold_energies():
    """At low temperature a collisional rate falls as exp(-E/kT): the
    logarithmic slope against 1/T is -E/k (the power-law factors of the fits
    add a few percent here)."""
    g = _rates_golden()["threshold_energies"]
    for name, E in (("coll_ion", g["T_ionisation_K"]), ("coll_ion_cool", g["T_ionisation_K"]),
                    ("coll_exc_cool", g["T_lyman_alpha_K"])):
        T1, T2 = 3000.0, 3300.0
        slope = (math.log(oracle.rate(name, T1)) - math.log(oracle.rate(name, T2))) / \
            (1 / T1 - 1 / T2)
        assert abs(-slope / E - 1) < 0.03, (name, slope)
    # collisional-ionisation cooling removes 13.6 eV per ionisation
    assert abs(oracle.rate("coll_ion_cool", 2e4) /
               (oracle.rate("coll_ion", 2e4) * 1.380649e-16 * g["T_ionisation_K"]) - 1) < 1e-12


def test_cooling_magnitudes():
    """Free-free cooling is the classical 1.42e-27 g T^1/2 with a gaunt factor
    between 1.1 and 1.5; a recombination removes between 1/2 and 3/2 kT of
    kinetic energy on average (case B), and case A removes more than case B."""
    g = _rates_golden()["free_free"]
    kB = 1.380649e-16
    for T in (5e3, 1e4, 2e4):
        gff = oracle.rate("free_free_cool", T) / (g["prefactor"] * math.sqrt(T))
        assert g["g_ff_range"][0] <= gff <= g["g_ff_range"][1], (T, gff)
        r = oracle.rate("rec_cool_B", T) / (oracle.rate("alpha_B", T) * kB * T)
        assert 0.5 < r < 1.5, (T, r)
        assert oracle.rate("rec_cool_A", T) > oracle.rate("rec_cool_B", T)


def _thermal_oracle(diffuse=False, T_rec=0.0, n=3, V=None):
    pos, h, src, L = _lattice_problem(4, 1.0, 3, n_s=1)
    V = np.full(pos.shape[1], 1.0 / 64) if V is None else V
    return oracle.Oracle(pos, h, src, L, V, diffuse=diffuse, T_rec=T_rec, **PHYS)


def test_thermal_heating_of_neutral_gas_is_the_closed_form():
    """Neutral gas has no free electrons, so nothing cools or recombines: the
    energy equation integrates the photoheating exactly,
    T1 = T0 + (2/3) h dt / k_B (h: heating per neutral atom)."""
    o = _thermal_oracle()
    kB = 1.380649e-16
    for h, dt, T0 in ((1e-26, 3e13, 1e4), (3e-27, 1e14, 300.0), (1e-24, 1e12, 2e3)):
        y1, T1 = o.ionize_thermal(np.zeros(3), np.full(3, h), np.full(3, 1e-3, np.float32),
                                  np.ones(3), np.full(3, T0), dt)
        assert np.all(np.abs(y1 - 1.0) < 1e-12)
        assert np.allclose(T1, T0 + 2.0 * h * dt / (3.0 * kB), rtol=1e-12)


def _residuals(o, gamma, heat, nH, y0, T0, dt, y1, T1, diffuse=False):
    """The two implicit equations evaluated with the pinned coefficients."""
    kB = 1.380649e-16
    nh = float(nH)
    aR = oracle.rate("alpha_A" if diffuse else "alpha_B", T0) * nh * dt
    c = oracle.rate("coll_ion", T0) * nh * dt
    K = SIGMA_CM2 * gamma * dt
    ry = y1 - y0 - (-K * y1 - c * y1 * (1 - y1) + aR * (1 - y1) ** 2)
    x0, x1 = 1 - y0, 1 - y1
    ne, npr, nhi = x1 * nh, x1 * nh, y1 * nh
    lam = ne * npr * (oracle.rate("rec_cool_A" if diffuse else "rec_cool_B", T1) +
                      oracle.rate("free_free_cool", T1)) + \
        ne * nhi * (oracle.rate("coll_ion_cool", T1) + oracle.rate("coll_exc_cool", T1))
    du = 1.5 * kB * nh * ((1 + x1) * T1 - (1 + x0) * T0)
    rT = du - dt * (nhi * heat - lam)
    return ry, rT, abs(du) + dt * (abs(nhi * heat) + lam)


@pytest.mark.parametrize("gamma,heat,y0,T0", [(1e-13 / SIGMA_CM2, 1e-24, 1.0, 1e4),
                                              (1e-12 / SIGMA_CM2, 8e-24, 0.3, 3e4),
                                              (0.0, 0.0, 0.1, 5e4),
                                              (1e-15 / SIGMA_CM2, 1e-26, 0.7, 800.0)])
def test_thermal_step_solves_both_implicit_equations(gamma, heat, y0, T0):
    """The update is backward Euler in both y and T: the new state satisfies
    the ionisation balance at T0 and the energy balance at (T1, x1), with
    recombination, free-free, collisional excitation and ionisation cooling
    assembled from the pinned coefficients (n_e n_p and n_e n_HI)."""
    o = _thermal_oracle()
    nH = np.float32(1e-3)
    for dt in (1e11, 3.15576e13, 1e15):
        y1, T1 = o.ionize_thermal(np.full(3, gamma), np.full(3, heat), np.full(3, nH),
                                  np.full(3, y0), np.full(3, T0), dt)
        ry, rT, scale = _residuals(o, gamma, heat, nH, y0, T0, dt, y1[0], T1[0])
        assert abs(ry) < 1e-12 * max(1.0, abs(y1[0])), (dt, ry)
        if 10.0 < T1[0] < 1e9:
            assert abs(rT) < 1e-9 * scale, (dt, rT, scale)


def test_thermal_equilibrium_of_photoionised_gas():
    """Optically thin gas under a constant ionising flux whose photoelectrons
    carry 5 eV each settles where photoionisation balances recombination and
    photoheating balances the cooling; the long-step update lands there."""
    o = _thermal_oracle()
    nH = np.float32(1e-3)
    k = 1e-12
    h = k * 5.0 * 1.602176634e-12
    y, T = np.ones(1), np.full(1, 1e4)
    for _ in range(100):
        y, T = o.ionize_thermal(np.array([k / SIGMA_CM2]), np.array([h]), np.array([nH]), y, T,
                                1e16)
    ry, rT, scale = _residuals(o, k / SIGMA_CM2, h, nH, y[0], T[0], 1e16, y[0], T[0])
    x = 1 - y[0]
    aB = oracle.rate("alpha_B", T[0])
    assert abs(k * y[0] + oracle.rate("coll_ion", T[0]) * float(nH) * x * y[0] -
               aB * float(nH) * x * x) < 1e-6 * k * y[0]
    assert abs(rT) < 1e-6 * scale
    assert 1.5e4 < T[0] < 4e4 and y[0] < 1e-3


def test_thermal_emitters_use_the_local_alpha_1():
    """In the diffuse case the emitters' luminosity takes alpha_A(T) -
    alpha_B(T) at each particle's temperature (Section 4.1 with the rate
    fits), and the self term of the update does too."""
    pos, h, src, L = _lattice_problem(5, 2.0, 28, n_s=1)
    n = pos.shape[1]
    V = np.full(n, (2.0 / 5) ** 3)
    o = oracle.Oracle(pos, h, src, L, V, diffuse=True, **PHYS)
    rng = np.random.default_rng(8)
    y = rng.uniform(0.1, 0.9, n)
    T = rng.uniform(5e3, 5e4, n)
    nH = np.full(n, 1e-2, np.float32)
    o.set_emitters_T(y, nH, T)
    a1 = np.array([oracle.rate("alpha_A", t) - oracle.rate("alpha_B", t) for t in T])
    ref = a1 * ((1 - y) * nH.astype(np.float64)) ** 2 * V * KPC_CM ** 3
    assert np.allclose(o.emitter_L(), ref, rtol=1e-12)
    ks_T, _ = o.self_terms_T(nH, y, T)
    ks_c, _ = o.self_terms(nH, y)
    assert np.allclose(ks_T / ks_c, a1 / (ALPHA_A - ALPHA_B), rtol=1e-12)



# ---------------------------------------------------------------- kernel-weighted cells
def _kernel_problem(nside=12, box=3.0, seed=33, eps=None):
    pos, h, src, L = _lattice_problem(nside, box, seed, n_s=1)
    n = pos.shape[1]
    rng = np.random.default_rng(seed)
    # volumes that fill the root cube (the frame: the particles' and the
    # source's bounding cube), so that cells are filled by their members
    p = np.concatenate([pos, src], axis=1).astype(np.float64)
    side = (p.max(1) - p.min(1)).max()
    V = side ** 3 / n * rng.uniform(0.9, 1.1, n)
    nH = np.full(n, 1e-2, np.float32)
    o = oracle.Oracle(pos, h, src, L, V, diffuse=True, lum_kernel=1, **PHYS)
    if eps is None:        # the same ionisation: the same emissivity alpha_1 n_e n_p
        y = np.full(n, 0.5)
    else:
        y = eps(pos, V)
    o.set_emitters(y, nH)
    return o, pos, V, y, nH


def test_kernel_cell_luminosity_uniform_emissivity():
    """Section 2.2.2's kernel-weighted form (emissivity reading): with a
    uniform emissivity every cell of two or more members gets exactly l^3
    times it, and over a level of cells that its members fill this is their
    summed luminosity to within the lattice's discretisation; single-member
    cells keep their member's luminosity."""
    o, pos, V, y, nH = _kernel_problem()
    eL = o.emitter_L()
    e = eL / V
    assert np.allclose(e, e[0], rtol=1e-12)
    t = o.tree(2)
    perm = o.perm(0)
    for n in range(len(t["level"])):
        members = perm[t["first"][n]:t["first"][n] + t["count"][n]]
        if t["count"][n] == 1:
            assert t["L"][n] == eL[members[0]]
        else:
            l = t["cube"][n, 3]
            assert abs(t["L"][n] / (l ** 3 * e[0]) - 1) < 1e-12
    for level in (1, 2):
        sel = (t["level"] == level) & (t["count"] > 1)
        tot = sum(eL[perm[t["first"][n]:t["first"][n] + t["count"][n]]].sum()
                  for n in np.nonzero(sel)[0])
        assert abs(t["L"][sel].sum() / tot - 1) < 0.05, level


def test_kernel_cell_luminosity_bruteforce():
    """Non-uniform emissivity: each cell's value is the definition evaluated
    directly over its members (cubic spline with h = the cell's edge, the
    stored float32 centre)."""
    def eps(pos, V):
        return np.clip(0.2 + 0.6 * pos[0].astype(np.float64) / 3.0, 0.0, 1.0)
    o, pos, V, y, nH = _kernel_problem(eps=eps)
    eL = o.emitter_L()
    t = o.tree(2)
    perm = o.perm(0)
    p = pos.astype(np.float64)
    checked = 0
    for n in range(0, len(t["level"]), 7):
        if t["count"][n] < 2:
            continue
        m = perm[t["first"][n]:t["first"][n] + t["count"][n]]
        l = t["cube"][n, 3]
        d = np.sqrt(((p[:, m] - t["cen"][n].astype(np.float64)[:, None]) ** 2).sum(0))
        w = np.array([oracle.spline_w(di, l) for di in d])
        ref = l ** 3 * (eL[m] / V[m] * w).sum() / w.sum()
        assert abs(t["L"][n] / ref - 1) < 1e-12
        checked += 1
    assert checked > 20
