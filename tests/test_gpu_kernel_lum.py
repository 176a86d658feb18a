"""The kernel-weighted luminosity of the emitter cells (start_params.
lum_kernel = 1, the alternative form of Section 2.2.2 read with the
members' emissivity): the emitter tree's luminosities against the oracle
(relative 1e-5: the GPU sums in FP32 with compensation), then Gamma at
theta = 0 and 0.7 within the usual tolerance, with the same rays and chain
links as the oracle; a clustered set puts cells of more than 2048 members
through the block-per-cell kernel."""
import numpy as np
import pytest

import oracle
from start_inputs import MYR_S, SIGMA_CM2

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


@pytest.mark.parametrize("n_p,theta", [(3001, 0.0), (20011, 0.7)])
def test_kernel_weighted_cells_match_the_oracle(S, n_p, theta):
    from test_gpu_parity import random_workload
    w = random_workload(n_p, 5, 19, diffuse=True)
    if n_p > 10000:   # a dense clump: cells of several thousand members
        w.pos[:, :8000] = (w.pos[:, :1] + np.float32(0.05) *
                           np.random.default_rng(3).uniform(0, 1, (3, 8000)).astype(np.float32))
        from start_inputs import smoothing_lengths
        w.h = smoothing_lengths(w.pos)
    ctx = S.Context(lum_kernel=1, tau_cut=1e30, ptree_leaf=PTREE_LEAF)
    ctx.build_trees(w.pos, w.h, w.src_pos, w.src_L, w.V, diffuse=True)
    ctx.set_state(w.n_H, w.y0)
    nHI = w.n_HI()
    g = np.zeros(w.n_p, np.float32)
    ctx.rt_solve(theta, gamma_out=g)
    st = ctx.stats()
    orc = oracle.Oracle.from_workload(w, ptree_leaf=PTREE_LEAF, lum_kernel=1)
    orc.set_emitters(w.y0, w.n_H)
    tg, to = ctx.tree(2), orc.tree(2)
    assert np.array_equal(tg["count"].astype(np.int64), to["count"])
    if n_p > 10000:
        assert to["count"].max() > 2048
    assert np.all(np.abs(tg["L"] - to["L"]) <= 1e-5 * np.abs(to["L"]) + 1e-300)
    assert np.array_equal(tg["cen"], to["cen"])
    idx = np.arange(w.n_p) if n_p < 10000 else np.arange(0, w.n_p, 23)
    ref = orc.gamma(nHI, theta, targets=idx)
    err = np.abs(g[idx].astype(np.float64) - ref)
    assert np.all(err <= 1e-4 * np.abs(ref) + G_ABS), float((err / (1e-4 * ref + G_ABS)).max())
    if n_p < 10000:
        assert st["rays"] == orc.last_stats["rays"] and st["hops"] in (-1, orc.last_stats["hops"])
