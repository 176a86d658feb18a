"""Batches of independent problems in one context (start_build_batch): every
kernel of the solve runs once over all of them, each target walking only its
own problem's tree and marching through its own particles.  Each problem's
Gamma, update and counts must be bitwise those of the same calls on it alone;
two coupled steps; a problem without sources and a one-particle problem in
the batch; the per-ray march too."""
import numpy as np
import pytest

import oracle
from start_inputs import MYR_S, SIGMA_CM2, lattice_workload

pytestmark = pytest.mark.gpu

G_ABS = 1e-8 / (SIGMA_CM2 * MYR_S)


@pytest.fixture(scope="module")
def S():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1005_5312_gb300 as S
    S.build()
    return S


def _problems():
    from paper_1005_5312_gb300.serve import make_request
    reqs = [make_request(r, n_p, n_s, clumpy=bool(r % 2), theta=0.6)
            for r, (n_p, n_s) in enumerate([(3000, 40), (5001, 1), (2048, 300), (1, 3),
                                             (4000, 0), (7777, 77)])]
    return reqs


@pytest.mark.parametrize("mode,counts", [(1, 0), (1, 1), (0, 0)])
def test_batch_is_bitwise_the_problems_alone(S, mode, counts):
    reqs = _problems()
    ctx = S.Context(march_mode=mode, tau_cut=1e30, link_counts=counts)
    ctx.build_batch([(r.pos, r.h, r.src_pos, r.src_L) for r in reqs])
    off = np.cumsum([0] + [r.n_p for r in reqs])
    nH = np.concatenate([r.n_H for r in reqs])
    y = np.concatenate([r.y0 for r in reqs])
    ctx.set_state(nH, y)
    alone = [S.Context(march_mode=mode, tau_cut=1e30, link_counts=counts) for _ in reqs]
    for a, r in zip(alone, reqs):
        a.build_trees(r.pos, r.h, r.src_pos, r.src_L)
        a.set_state(r.n_H, r.y0)
    for step in range(2):
        g = np.zeros(off[-1], np.float32)
        yb = np.zeros(off[-1])
        ctx.rt_solve(0.6, gamma_out=g)
        st = ctx.stats()
        ctx.ionize(MYR_S, y_out=yb)
        rays = hops = 0
        for b, (a, r) in enumerate(zip(alone, reqs)):
            ga = np.zeros(r.n_p, np.float32)
            ya = np.zeros(r.n_p)
            a.rt_solve(0.6, gamma_out=ga)
            sa = a.stats()
            rays += sa["rays"]
            hops += sa["hops"]
            a.ionize(MYR_S, y_out=ya)
            assert np.array_equal(g[off[b]:off[b + 1]], ga), (step, b)
            assert np.array_equal(yb[off[b]:off[b + 1]], ya), (step, b)
        assert st["rays"] == rays
        if mode == 1 and counts == 0:   # chain links are counted in the counting form only
            assert st["hops"] == -1
        else:
            assert st["hops"] == hops
    # and the oracle on one problem of the batch
    r, b = reqs[2], 2
    orc = oracle.Oracle(r.pos, r.h, r.src_pos, r.src_L, ptree_leaf=16, sigma_cm2=SIGMA_CM2,
                        len_unit_cm=3.0857e21, alpha_A=4.18e-13, alpha_B=2.59e-13)
    nHI = (y[off[b]:off[b + 1]] * r.n_H.astype(np.float64)).astype(np.float32)
    ctx2 = S.Context(march_mode=mode, tau_cut=1e30)
    ctx2.build_batch([(q.pos, q.h, q.src_pos, q.src_L) for q in reqs])
    g2 = np.zeros(off[-1], np.float32)
    ctx2.rt_solve(0.6, n_HI=np.concatenate([(q.y0 * q.n_H.astype(np.float64)).astype(np.float32)
                                             for q in reqs]), gamma_out=g2)
    ref = orc.gamma(nHI, 0.6)
    err = np.abs(g2[off[b]:off[b + 1]].astype(np.float64) - ref)
    assert np.all(err <= 1e-4 * np.abs(ref) + G_ABS)
