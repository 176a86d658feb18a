"""H2 photodissociation rate (Appendix B) through the C ABI against the FP64
oracle.

k_dis sums positive terms L f_sh(N_H2/1e14)/(4 pi r^2); the float32 path
carries the columns as compensated sums of float32 link terms (relative
error ~1e-6, entering f_sh with exponent -3/4) and the per-target sums in
a fixed order: the tests allow 1e-4 relative, element by element.  Ray and
chain-link counts are exact (the same chains as the Gamma solve).
"""
import math

import numpy as np
import pytest

import oracle
from start_inputs import config1, config2, lattice_workload, KPC_CM

pytestmark = pytest.mark.gpu
REL = 1e-4
KAPPA = 1.0e-21


@pytest.fixture(scope="module")
def S():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1005_5312_gb300 as S
    S.build()
    return S


def close(k, ref):
    k = np.asarray(k, np.float64)
    bad = np.nonzero(np.abs(k - ref) > REL * np.abs(ref))[0]
    assert len(bad) == 0, (len(bad), bad[:5], k[bad[:5]], ref[bad[:5]])


def lognormal_h2(n, seed):
    return np.random.default_rng(seed).lognormal(np.log(1e-4), 1.5, n).astype(np.float32)


@pytest.mark.parametrize("theta", [0.0, 0.5, 1.0])
def test_kdis_parity_config1(S, theta):
    w = config1()
    ctx = S.Context(ptree_leaf=16)
    ctx.build_trees(w.pos, w.h, w.src_pos, w.src_L)
    orc = oracle.Oracle.from_workload(w, ptree_leaf=16)
    nH2 = lognormal_h2(w.n_p, 5)
    k = ctx.h2_dissociation(nH2, theta, KAPPA)
    ref = orc.h2_dissociation(nH2, theta, KAPPA)
    close(k, ref)
    st = ctx.stats()
    assert st["rays"] == orc.last_stats["rays"] and st["hops"] in (-1, orc.last_stats["hops"])


def test_kdis_uniform_medium_closed_form(S):
    """Uniform n_H2 at theta = 0: N = n_H2 r along every chain."""
    w = lattice_workload("h2-uniform-24^3", 24, 4.0, 9, 77, L=2e49)
    ctx = S.Context()
    ctx.build_trees(w.pos, w.h, w.src_pos, w.src_L)
    nval = np.float32(2e-6)
    k = ctx.h2_dissociation(np.full(w.n_p, nval, np.float32), 0.0, KAPPA)
    d = w.pos.astype(np.float64)[:, :, None] - w.src_pos.astype(np.float64)[:, None, :]
    r = np.sqrt((d ** 2).sum(axis=0)) * KPC_CM
    x = np.float64(nval) * r / 1e14
    f = np.where(x <= 1.0, 1.0, np.maximum(x, 1.0) ** -0.75)
    ref = (1.13e8 * KAPPA * w.src_L[None, :] / (4 * math.pi * r * r) * f).sum(axis=1)
    close(k, ref)


def test_kdis_leaves_the_resident_state_alone(S):
    """Gamma, the resident chemistry and a following solve are unchanged by a
    k_dis call (the records' density slot is restored), also after an
    invalid n_H2 is rejected."""
    w = config1()
    ctx = S.Context()
    ctx.build_trees(w.pos, w.h, w.src_pos, w.src_L)
    ctx.set_state(w.n_H, w.y0)
    g0 = np.zeros(w.n_p, np.float32)
    ctx.rt_solve(0.5, gamma_out=g0)
    ctx.h2_dissociation(lognormal_h2(w.n_p, 6), 0.5, KAPPA)
    bad = lognormal_h2(w.n_p, 6)
    bad[3] = -1.0
    with pytest.raises(S.StartError):
        ctx.h2_dissociation(bad, 0.5, KAPPA)
    with pytest.raises(S.StartError):
        ctx.h2_dissociation(lognormal_h2(w.n_p, 6), 0.5, -1.0)
    y1 = np.zeros(w.n_p)
    ctx.ionize(w.dt_s, y_out=y1)      # uses the Gamma of the rt_solve above
    ref = oracle.Oracle.from_workload(w)
    gref, yref = ref.step(w.y0, w.n_H, 0.5, w.dt_s)
    assert np.all(np.abs(y1 - yref) <= 1e-3)
    g1 = np.zeros(w.n_p, np.float32)
    ctx.set_state(w.n_H, w.y0)
    ctx.rt_solve(0.5, gamma_out=g1)
    assert np.array_equal(g0, g1)


def test_kdis_ignores_the_emitters_of_a_diffuse_context(S):
    w = lattice_workload("h2-diffuse-20^3", 20, 4.0, 5, 78, L=1e49, diffuse=True)
    ctx = S.Context(ptree_leaf=16)
    ctx.build_trees(w.pos, w.h, w.src_pos, w.src_L, w.V, diffuse=True)
    ctx.set_state(w.n_H, np.full(w.n_p, 0.5))
    orc = oracle.Oracle.from_workload(w, ptree_leaf=16)
    nH2 = lognormal_h2(w.n_p, 7)
    close(ctx.h2_dissociation(nH2, 0.7, KAPPA), orc.h2_dissociation(nH2, 0.7, KAPPA))


def test_kdis_full_size_sampled_targets(S):
    w = config2()
    ctx = S.Context()
    ctx.build_trees(w.pos, w.h, w.src_pos, w.src_L)
    nH2 = lognormal_h2(w.n_p, 8)
    k = ctx.h2_dissociation(nH2, 0.5, KAPPA)
    orc = oracle.Oracle.from_workload(w, ptree_leaf=16)
    idx = np.random.default_rng(9).choice(w.n_p, 400, replace=False)
    close(k[idx], orc.h2_dissociation(nH2, 0.5, KAPPA, targets=idx))


def test_kdis_edge_cases(S):
    """No sources: k_dis = 0 everywhere; no particles: nothing to do."""
    w = lattice_workload("h2-nosrc-8^3", 8, 2.0, 0, 79)
    ctx = S.Context()
    ctx.build_trees(w.pos, w.h, w.src_pos, w.src_L)
    k = ctx.h2_dissociation(np.full(w.n_p, 1e-3, np.float32), 0.5, KAPPA)
    assert not np.any(k)
    c0 = S.Context()
    c0.build_trees(np.zeros((3, 0), np.float32), np.zeros(0, np.float32), w.src_pos, w.src_L)
    assert c0.h2_dissociation(np.zeros(0, np.float32), 0.5, KAPPA).size == 0
