"""Autotuner of the knobs that do not change any result.

* ``ptree_leaf``  -- particle-tree leaf size (neighbour search),
* ``march_group`` -- lanes cooperating on one neighbour-list evaluation of
  the later chain levels (the warp-per-target grouping of the march),
* ``row_warps``   -- the first hop's tile shape: target rows per block,
* ``walk_warp``   -- one tree walk per warp of 32 targets, or per thread,
* ``row_bins``    -- the first hop's direction bins (candidate sets per bin,
  or a scan of every neighbour).

Each knob is varied in turn around the current best (coordinate descent),
timing one full step (build + solve) per candidate with CUDA events, and the
fastest setting is kept.  The memory bound of a solve (max_pairs) is not a
knob here: it decides how a large solve is split, which regroups Gamma's
additions.  Results are cached per problem class (powers of
two of N_p and N_s, theta, diffuse), so a server tunes a class once.  The
source-tree leaf size is *not* tuned: it changes the method's result (one
source per cell is the paper's choice).
"""
from __future__ import annotations

import math

SEARCH_SPACE = {
    "march_group": (1, 2, 4, 8),
    "ptree_leaf": (8, 16, 32),
    "row_warps": (4, 8),
    "walk_warp": (0, 1),
    "row_bins": (0, 4, 6),
}
DEFAULTS = {"march_group": 2, "ptree_leaf": 16, "row_warps": 8, "walk_warp": 0, "row_bins": 4}


def problem_class(n_p: int, n_s: int, theta: float, diffuse: bool = False) -> tuple:
    return (int(round(math.log2(max(n_p, 1)))), int(round(math.log2(max(n_s, 1)))),
            round(float(theta), 3), bool(diffuse))


def coordinate_descent(time_fn, space=None, start=None, rounds: int = 1) -> tuple:
    """Minimise time_fn(params) knob by knob.  Returns (best params, best
    time, every (params, time) tried)."""
    space = space or SEARCH_SPACE
    best = dict(start or DEFAULTS)
    tried = {}

    def t(p):
        key = tuple(sorted(p.items()))
        if key not in tried:
            tried[key] = time_fn(dict(p))
        return tried[key]

    best_t = t(best)
    for _ in range(rounds):
        for knob, values in space.items():
            for v in values:
                cand = dict(best, **{knob: v})
                tc = t(cand)
                if tc < best_t:
                    best, best_t = cand, tc
    return best, best_t, [(dict(k), v) for k, v in tried.items()]


class Tuner:
    """Per-class cache of tuned parameters."""

    def __init__(self):
        self.cache = {}

    def params_for(self, n_p, n_s, theta, diffuse=False):
        return dict(self.cache.get(problem_class(n_p, n_s, theta, diffuse), DEFAULTS))

    def tune(self, pos, h, src_pos, src_L, theta, n_HI, repeats: int = 2, V=None,
             diffuse=False, stream=None) -> dict:
        """Tune on one problem (host or device arrays); returns the params."""
        import torch

        from . import Context
        dev = torch.device("cuda", torch.cuda.current_device())
        st = stream or torch.cuda.current_stream(dev)
        n_p = int(h.shape[0])

        def time_fn(p):
            ctx = Context(stream=st, **p)
            g = torch.zeros(n_p, dtype=torch.float32, device=dev)
            # first call grows the buffers; time the following ones
            ctx.build_trees(pos, h, src_pos, src_L, V, diffuse=diffuse)
            ctx.rt_solve(theta, n_HI=n_HI, gamma_out=g)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            for _ in range(repeats):
                ctx.build_trees(pos, h, src_pos, src_L, V, diffuse=diffuse)
                ctx.rt_solve(theta, n_HI=n_HI, gamma_out=g)
            e1.record(st)
            torch.cuda.synchronize(dev)
            ctx.close()
            return e0.elapsed_time(e1) / repeats

        best, _, _ = coordinate_descent(time_fn)
        self.cache[problem_class(n_p, int(src_L.shape[0]), theta, diffuse)] = best
        return best

    def tune_requests(self, requests, max_classes: int = 24, repeats: int = 2) -> list:
        """Tune the problem classes of a request stream (the most frequent
        first, at most max_classes), each on its first request; returns the
        classes tuned."""
        counts = {}
        first = {}
        for r in requests:
            k = problem_class(r.n_p, r.n_s, r.theta)
            counts[k] = counts.get(k, 0) + 1
            first.setdefault(k, r)
        done = []
        for k in sorted(counts, key=lambda q: -counts[q])[:max_classes]:
            if k in self.cache:
                continue
            r = first[k]
            nHI = (r.y0 * r.n_H.astype("float64")).astype("float32")
            self.tune(r.pos, r.h, r.src_pos, r.src_L, r.theta, nHI, repeats=repeats)
            done.append(k)
        return done
