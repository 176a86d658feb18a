"""Full-size workloads in the launch configuration bench.py uses, checked
against the oracle on sampled targets (the oracle evaluates them one by
one): the diffuse-recombination shadowing workload (128^3 particles, all
emitting, eight clumps, one bright central source, theta = 0.7)."""
import time

import numpy as np
import pytest

import oracle
from start_inputs import MYR_S, SIGMA_CM2, config3

pytestmark = pytest.mark.gpu

G_ABS = 1e-8 / (SIGMA_CM2 * MYR_S)


def test_config3_diffuse_full_size_sampled_targets():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1005_5312_gb300 as S
    S.build()
    t0 = time.time()
    w = config3()
    t_gen = time.time() - t0
    ctx = S.Context(timing=1)
    ctx.build_trees(w.pos, w.h, w.src_pos, w.src_L, w.V, diffuse=True)
    ctx.set_state(w.n_H, w.y0)
    g = np.zeros(w.n_p, np.float32)
    t1 = time.time()
    ctx.rt_solve(0.7, gamma_out=g)
    t_solve = time.time() - t1
    st = ctx.stats()
    assert st["chunks"] >= 1 and st["rays"] > w.n_p
    orc = oracle.Oracle.from_workload(w, ptree_leaf=16)
    orc.set_emitters(w.y0, w.n_H)
    rng = np.random.default_rng(2)
    # half of the samples in the clumps (dense, shadowed), half in the background
    dense = np.nonzero(w.n_H > 1e-3)[0]
    thin = np.nonzero(w.n_H <= 1e-3)[0]
    idx = np.concatenate([rng.choice(dense, 12, replace=False), rng.choice(thin, 12, replace=False)])
    ref = orc.gamma(w.n_HI(), 0.7, targets=idx)
    err = np.abs(g[idx].astype(np.float64) - ref)
    assert np.all(err <= 1e-4 * np.abs(ref) + G_ABS), (err, ref)
    print(f"config3: gen {t_gen:.1f}s solve {t_solve:.2f}s rays {st['rays']} chunks {st['chunks']} "
          f"evals {st['evals']}")


def test_multi_chunk_request_memoised_matches_per_ray_and_oracle():
    """A served request whose pairs need several target chunks (609,707
    particles, 20,002 sources, theta = 0.5): chunks cut chains, so many links
    leave the lists and the slot capacity is retried larger; the memoised
    solve must still agree with the per-ray march and the oracle."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1005_5312_gb300 as S
    from paper_1005_5312_gb300.serve import make_request
    S.build()
    r = make_request(1, 609707, 20002, clumpy=False, theta=0.5)
    out = {}
    for mode, counts in ((1, 0), (1, 1), (0, 0)):
        ctx = S.Context(march_mode=mode, tau_cut=1e30, link_counts=counts)
        ctx.build_trees(r.pos, r.h, r.src_pos, r.src_L)
        g = np.zeros(r.n_p, np.float32)
        ctx.rt_solve(r.theta, n_HI=r.n_H, gamma_out=g)
        out[mode, counts] = (g.astype(np.float64), ctx.stats())
        ctx.close()
    (g1, s1), (gc, sc), (g0, s0) = out[1, 0], out[1, 1], out[0, 0]
    assert s1["chunks"] > 1 and s1["rays"] == s0["rays"] == sc["rays"]
    assert sc["hops"] == s0["hops"] and s1["hops"] == -1   # counted in the counting form
    assert np.all(np.abs(g1 - g0) <= 2e-5 * np.abs(g0) + G_ABS)
    assert np.all(np.abs(gc - g0) <= 2e-5 * np.abs(g0) + G_ABS)
    orc = oracle.Oracle(r.pos, r.h, r.src_pos, r.src_L, ptree_leaf=16, sigma_cm2=6.3e-18,
                        len_unit_cm=3.0857e21, alpha_A=4.18e-13, alpha_B=2.59e-13)
    idx = np.random.default_rng(4).choice(r.n_p, 12, replace=False)
    ref = orc.gamma(r.n_H, r.theta, targets=idx)
    assert np.all(np.abs(g1[idx] - ref) <= 1e-4 * np.abs(ref) + G_ABS)


def test_config5_lognormal_diffuse_full_size_sampled_targets():
    """The large diffuse run: 256^3 particles in a log-normal clumpy field
    (sigma_ln = 1.5, P(k) ~ k^-3), all emitting, plus 64 sources of 1e50/s.
    The density is recomputed by SPH summation (Section 2.1) from masses
    m = n_H V, then one solve at theta = 0.5 and one at theta = 1 run in
    target chunks; sampled densities and Gamma against the oracle."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1005_5312_gb300 as S
    from start_inputs import config5
    S.build()
    t0 = time.time()
    w = config5()
    t_gen = time.time() - t0
    ctx = S.Context(max_pairs=1 << 28)
    ctx.build_trees(w.pos, w.h, w.src_pos, w.src_L, w.V, diffuse=True)
    mass = (w.n_H.astype(np.float64) * w.V).astype(np.float32)
    rho = ctx.sph_density(mass)
    orc = oracle.Oracle.from_workload(w, ptree_leaf=16)
    rho_ref = orc.sph_density(mass.astype(np.float64))
    assert np.all(np.abs(rho - rho_ref) <= 2e-5 * rho_ref)
    n_H = rho.astype(np.float32)          # the recomputed density field, cm^-3
    ctx.set_state(n_H, w.y0)
    orc.set_emitters(w.y0, n_H)
    nHI = (w.y0 * n_H.astype(np.float64)).astype(np.float32)
    idx = np.random.default_rng(8).choice(w.n_p, 12, replace=False)
    report = [f"gen {t_gen:.1f}s"]
    for theta in (0.5, 1.0):
        g = np.zeros(w.n_p, np.float32)
        t1 = time.time()
        ctx.rt_solve(theta, gamma_out=g)
        t_solve = time.time() - t1
        st = ctx.stats()
        assert st["chunks"] > 1 and st["rays"] > 100 * w.n_p
        ref = orc.gamma(nHI, theta, targets=idx)
        err = np.abs(g[idx].astype(np.float64) - ref)
        assert np.all(err <= 1e-4 * np.abs(ref) + G_ABS), (theta, err, ref)
        report.append(f"theta {theta}: solve {t_solve:.1f}s rays {st['rays']} chunks {st['chunks']}")
    ctx.close()
    print("config5:", "; ".join(report))
