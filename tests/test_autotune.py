"""Autotuner: the search itself (CPU, with a synthetic cost) and, on the GPU,
that tuned knobs leave every result bitwise unchanged."""
import numpy as np
import pytest

from paper_1005_5312_gb300.autotune import (DEFAULTS, SEARCH_SPACE, Tuner, coordinate_descent,
                                            problem_class)


def test_coordinate_descent_finds_the_separable_minimum():
    target = {"march_group": 4, "ptree_leaf": 32, "row_warps": 4, "walk_warp": 1, "row_bins": 6}
    calls = []

    def cost(p):
        calls.append(p)
        return sum((np.log2(p[k] + 1) - np.log2(target[k] + 1)) ** 2 for k in target) + 1.0

    best, t, tried = coordinate_descent(cost)
    assert best == target and t == 1.0
    assert len(calls) == len(tried) <= 1 + sum(len(v) for v in SEARCH_SPACE.values())


def test_problem_classes_and_cache():
    assert problem_class(262144, 1024, 0.5) == (18, 10, 0.5, False)
    assert problem_class(300000, 1000, 0.5) == problem_class(262144, 1024, 0.5)
    t = Tuner()
    assert t.params_for(1 << 18, 1 << 10, 0.5) == DEFAULTS
    t.cache[problem_class(1 << 18, 1 << 10, 0.5)] = dict(DEFAULTS, march_group=8)
    assert t.params_for(262000, 1030, 0.5)["march_group"] == 8


@pytest.mark.gpu
def test_tuned_knobs_are_result_neutral():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1005_5312_gb300 as S
    from start_inputs import lattice_workload
    S.build()
    w = lattice_workload("tune-24^3", 24, 4.0, 40, 9)
    nHI = w.n_HI()
    tuner = Tuner()
    best = tuner.tune(w.pos, w.h, w.src_pos, w.src_L, 0.5, nHI, repeats=1)
    assert set(best) == set(DEFAULTS)
    out = []
    for p in (DEFAULTS, best, {"march_group": 8, "ptree_leaf": 8, "row_warps": 4,
                               "walk_warp": 1, "row_bins": 0}):
        ctx = S.Context(**p)
        ctx.build_trees(w.pos, w.h, w.src_pos, w.src_L)
        g = np.zeros(w.n_p, np.float32)
        ctx.rt_solve(0.5, n_HI=nHI, gamma_out=g)
        out.append(g)
    assert np.array_equal(out[0], out[1]) and np.array_equal(out[0], out[2])
