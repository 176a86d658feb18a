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
