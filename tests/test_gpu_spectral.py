"""Blackbody point sources (T_eff, Appendix A integrals) and diffuse
recombination photons in a band (T_rec, Section 4.1) through the C ABI
against the FP64 oracle.

The GPU interpolates ln F_ion and ln F_heat (ln R_ion, ln R_heat for the
band) from a table (spacing 2.5e-3 in s = ln(1 + tau/1e-3): interpolation
error below ~1e-5 relative where the contributions matter), on top of the float32 tau of the chains: Gamma_eff and
the heating rate are compared at 1e-4 relative plus the absolute floors
Gamma_abs = 1e-8/(sigma dt) and sigma h nu_L Gamma_abs.  Rays and chain links
are exact.
"""
import numpy as np
import pytest

import oracle
from start_inputs import KPC_CM, MYR_S, SIGMA_CM2, lattice_workload

pytestmark = pytest.mark.gpu
G_ABS = 1e-8 / (SIGMA_CM2 * MYR_S)
H_ABS = SIGMA_CM2 * 13.6 * 1.602176634e-12 * G_ABS
REL = 1e-4


@pytest.fixture(scope="module")
def S():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1005_5312_gb300 as S
    S.build()
    return S


def close(x, ref, floor):
    x = np.asarray(x, np.float64)
    bad = np.nonzero(np.abs(x - ref) > REL * np.abs(ref) + floor)[0]
    assert len(bad) == 0, (len(bad), bad[:5], x[bad[:5]], ref[bad[:5]])


@pytest.mark.parametrize("theta", [0.0, 0.6])
@pytest.mark.parametrize("T_eff", [1e5, 3e4])
def test_spectral_gamma_and_heating_parity(S, theta, T_eff):
    w = lattice_workload("bb-20^3", 20, 6.6, 16, 91, L=5e48)
    y = np.random.default_rng(2).uniform(0.0, 1.0, w.n_p)
    nHI = (y * w.n_H.astype(np.float64)).astype(np.float32)
    ctx = S.Context(T_eff=T_eff, ptree_leaf=16)
    ctx.build_trees(w.pos, w.h, w.src_pos, w.src_L)
    g = np.zeros(w.n_p, np.float32)
    ctx.rt_solve(theta, n_HI=nHI, gamma_out=g)
    heat = ctx.heating()
    orc = oracle.Oracle.from_workload(w, ptree_leaf=16)
    gref, href = orc.gamma_spectral(nHI, theta, T_eff)
    close(g, gref, G_ABS)
    close(heat, href, H_ABS)
    st = ctx.stats()
    assert st["rays"] == orc.last_stats["rays"] and st["hops"] in (-1, orc.last_stats["hops"])
    assert np.all(heat >= 0) and heat.max() > 0


def test_monochromatic_sources_heat_nothing(S):
    w = lattice_workload("mono-16^3", 16, 6.6, 4, 92)
    ctx = S.Context(reuse_chains=1)
    ctx.build_trees(w.pos, w.h, w.src_pos, w.src_L)
    ctx.set_state(w.n_H, w.y0)
    g = np.zeros(w.n_p, np.float32)
    for _ in range(2):                       # full solve, then the resident form
        ctx.rt_solve(0.5, gamma_out=g)
        assert not np.any(ctx.heating())
    # switching to blackbody sources takes the full path and heats
    ctx.set_params(T_eff=1e5, reuse_chains=1)
    ctx.rt_solve(0.5, gamma_out=g)
    assert ctx.heating().max() > 0


def test_spectral_sources_with_diffuse_emitters(S):
    """Emitters stay monochromatic at the Lyman limit and add no heating."""
    w = lattice_workload("bb-diffuse-14^3", 14, 4.0, 3, 93, L=1e49, diffuse=True)
    y = np.full(w.n_p, 0.3)
    ctx = S.Context(T_eff=1e5, ptree_leaf=16)
    ctx.build_trees(w.pos, w.h, w.src_pos, w.src_L, w.V, diffuse=True)
    ctx.set_state(w.n_H, y)
    g = np.zeros(w.n_p, np.float32)
    ctx.rt_solve(0.7, gamma_out=g)
    orc = oracle.Oracle.from_workload(w, ptree_leaf=16)
    orc.set_emitters(y, w.n_H)
    nHI = (y * w.n_H.astype(np.float64)).astype(np.float32)
    gref, href = orc.gamma_spectral(nHI, 0.7, 1e5)
    close(g, gref, G_ABS)
    close(ctx.heating(), href, H_ABS)


def test_invalid_temperature_is_rejected(S):
    with pytest.raises(S.StartError):
        S.Context(T_eff=100.0)
    with pytest.raises(S.StartError):
        S.Context(T_eff=-1.0)


def test_spectral_edge_cases(S):
    """Heating before any solve is an error; without sources Gamma and the
    heating are zero."""
    w = lattice_workload("bb-nosrc-8^3", 8, 2.0, 0, 94)
    ctx = S.Context(T_eff=1e5)
    ctx.build_trees(w.pos, w.h, w.src_pos, w.src_L)
    with pytest.raises(S.StartError):
        ctx.heating()
    ctx.set_state(w.n_H, w.y0)
    g = np.ones(w.n_p, np.float32)
    ctx.rt_solve(0.5, gamma_out=g)
    assert not np.any(g) and not np.any(ctx.heating())


@pytest.mark.parametrize("theta", [0.0, 0.7])
@pytest.mark.parametrize("T_eff", [0.0, 1e5])
def test_recombination_band_parity(S, theta, T_eff):
    """Diffuse emitters radiating the band of width k T_rec / h (Section 4.1):
    Gamma_eff, the photoheating (Eq. gother over the emitter lists plus the
    self term of Eq. gself) and the implicit update with the band-averaged
    k_self, against the oracle."""
    T_rec = 1e4
    w = lattice_workload("band-14^3", 14, 4.0, 3, 95, L=1e49, diffuse=True)
    y = np.random.default_rng(5).uniform(0.0, 1.0, w.n_p)
    ctx = S.Context(T_eff=T_eff, T_rec=T_rec, ptree_leaf=16)
    ctx.build_trees(w.pos, w.h, w.src_pos, w.src_L, w.V, diffuse=True)
    ctx.set_state(w.n_H, y)
    g = np.zeros(w.n_p, np.float32)
    ctx.rt_solve(theta, gamma_out=g)
    heat = ctx.heating()
    orc = oracle.Oracle.from_workload(w, ptree_leaf=16, T_rec=T_rec)
    orc.set_emitters(y, w.n_H)
    nHI = (y * w.n_H.astype(np.float64)).astype(np.float32)
    gref, href = orc.gamma_spectral(nHI, theta, T_eff)
    _, hself = orc.self_terms(w.n_H, y)
    close(g, gref, G_ABS)
    close(heat, href + hself, H_ABS)
    st = ctx.stats()
    assert st["rays"] == orc.last_stats["rays"] and st["hops"] in (-1, orc.last_stats["hops"])
    assert np.all(heat > 0)
    y1 = np.zeros(w.n_p)
    ctx.ionize(w.dt_s, y_out=y1)
    yref, _ = orc.ionize(gref, w.n_H, y, w.dt_s)
    assert np.max(np.abs(y1 - yref)) <= 1e-4


def test_recombination_band_needs_emitters(S):
    """Without diffuse emitters T_rec changes nothing and nothing heats."""
    w = lattice_workload("band-nodiffuse-12^3", 12, 4.0, 3, 96)
    out = []
    for T_rec in (0.0, 3e4):
        ctx = S.Context(T_rec=T_rec)
        ctx.build_trees(w.pos, w.h, w.src_pos, w.src_L)
        ctx.set_state(w.n_H, w.y0)
        g = np.zeros(w.n_p, np.float32)
        ctx.rt_solve(0.5, gamma_out=g)
        assert not np.any(ctx.heating())
        out.append(g)
    assert np.array_equal(out[0], out[1])


def test_invalid_band_temperature_is_rejected(S):
    for T_rec in (50.0, 2e5, -1.0, float("nan")):
        with pytest.raises(S.StartError):
            S.Context(T_rec=T_rec)
