"""The temperature half of the network (start_params.thermal = 1): gas
temperatures advanced by the energy equation (Section 2.1 without its
hydrodynamic terms) with photoheating from the solve, recombination
coefficients and cooling at the local temperature, against the oracle.

Tolerances: x_HII absolute 1e-3 (as for the isothermal update) and T
relative 1e-3; Gamma and the heating enter through the solve (1e-4)."""
import numpy as np
import pytest

import oracle
from start_inputs import MYR_S, config1, config3

pytestmark = pytest.mark.gpu

PTREE_LEAF = 16
X_ABS = 1e-3
T_REL = 1e-3


@pytest.fixture(scope="module")
def S():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1005_5312_gb300 as S
    S.build()
    return S


def _close(y, T, y_ref, T_ref, what):
    dy = np.abs(y - y_ref).max()
    dT = np.abs(T / T_ref - 1.0).max()
    assert dy <= X_ABS, (what, dy)
    assert dT <= T_REL, (what, dT, T[np.argmax(np.abs(T / T_ref - 1))])


def test_config1_blackbody_sources_coupled_thermal_steps(S):
    """32^3 particles and 16 sources radiating 1e5 K blackbodies: three
    coupled 1 Myr steps from neutral 1e4 K gas; photoheating raises the
    temperature of the ionised regions."""
    w = config1()
    ctx = S.Context(thermal=1, T_eff=1e5, ptree_leaf=PTREE_LEAF)
    ctx.build_trees(w.pos, w.h, w.src_pos, w.src_L)
    ctx.set_state(w.n_H, w.y0)
    T0 = np.full(w.n_p, 1e4)
    ctx.set_temperature(T0)
    orc = oracle.Oracle.from_workload(w, ptree_leaf=PTREE_LEAF)
    y_ref, T_ref = w.y0.copy(), T0.copy()
    y = np.zeros(w.n_p)
    for step in range(3):
        g = np.zeros(w.n_p, np.float32)
        ctx.rt_solve(0.5, gamma_out=g)
        ctx.ionize(MYR_S, y_out=y)
        T = ctx.temperature()
        nHI = (y_ref * w.n_H.astype(np.float64)).astype(np.float32)
        gr, hr = orc.gamma_spectral(nHI, 0.5, 1e5)
        y_ref, T_ref = orc.ionize_thermal(gr, hr, w.n_H, y_ref, T_ref, MYR_S)
        _close(y, T, y_ref, T_ref, step)
    assert T.max() > 2e4 and (1 - y).max() > 0.5


def test_diffuse_band_thermal_step_from_a_mixed_state(S):
    """Every particle emitting recombination photons in the band of width
    k T_rec / h with their photoheating, the emitters' alpha_1 at the local
    temperature, from a state with random ionisation and temperatures."""
    from test_gpu_parity import random_workload
    w = random_workload(4001, 7, 15, diffuse=True)
    rng = np.random.default_rng(16)
    T0 = rng.uniform(3e3, 5e4, w.n_p)
    ctx = S.Context(thermal=1, T_rec=1e4, T_eff=5e4, ptree_leaf=PTREE_LEAF)
    ctx.build_trees(w.pos, w.h, w.src_pos, w.src_L, w.V, diffuse=True)
    ctx.set_state(w.n_H, w.y0)
    ctx.set_temperature(T0)
    g = np.zeros(w.n_p, np.float32)
    ctx.rt_solve(0.7, gamma_out=g)
    y = np.zeros(w.n_p)
    ctx.ionize(MYR_S, y_out=y)
    T = ctx.temperature()
    orc = oracle.Oracle.from_workload(w, ptree_leaf=PTREE_LEAF, T_rec=1e4)
    orc.set_emitters_T(w.y0, w.n_H, T0)
    gr, hr = orc.gamma_spectral(w.n_HI(), 0.7, 5e4)
    _, hs = orc.self_terms_T(w.n_H, w.y0, T0)
    y_ref, T_ref = orc.ionize_thermal(gr, hr + hs, w.n_H, w.y0, T0, MYR_S)
    _close(y, T, y_ref, T_ref, "diffuse")


def test_config3_full_size_thermal_sampled_targets(S):
    """The 128^3 diffuse workload (one 3e51/s source, eight clumps, every
    particle emitting in the band) in the launch configuration the benchmark
    uses, one thermal step; the oracle on 24 sampled particles."""
    w = config3()
    T0 = np.full(w.n_p, 1e4)
    ctx = S.Context(thermal=1, T_rec=1e4)
    ctx.build_trees(w.pos, w.h, w.src_pos, w.src_L, w.V, diffuse=True)
    ctx.set_state(w.n_H, w.y0)
    ctx.set_temperature(T0)
    g = np.zeros(w.n_p, np.float32)
    ctx.rt_solve(0.7, gamma_out=g)
    y = np.zeros(w.n_p)
    ctx.ionize(MYR_S, y_out=y)
    T = ctx.temperature()
    orc = oracle.Oracle.from_workload(w, ptree_leaf=PTREE_LEAF, T_rec=1e4)
    orc.set_emitters_T(w.y0, w.n_H, T0)
    rng = np.random.default_rng(17)
    dense = np.nonzero(w.n_H > 1e-3)[0]
    thin = np.nonzero(w.n_H <= 1e-3)[0]
    idx = np.concatenate([rng.choice(dense, 12, replace=False), rng.choice(thin, 12, replace=False)])
    gr, hr = orc.gamma_spectral(w.n_HI(), 0.7, 0.0, targets=idx)
    _, hs = orc.self_terms_T(w.n_H, w.y0, T0)
    y_ref, T_ref = orc.ionize_thermal(gr, hr + hs[idx], w.n_H[idx], w.y0[idx], T0[idx], MYR_S,
                                      targets=idx)
    _close(y[idx], T[idx], y_ref, T_ref, "config3")
