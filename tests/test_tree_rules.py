"""The octree level census, checked on the CPU against the oracle's trees.

The GPU counts every level's cells from the sorted Morton keys alone before
it builds the levels: a cell of level l starts at sorted key k iff k is the
first key of its level-l prefix and the parent cell holds more than `leaf`
keys (a cell of at most `leaf` keys, or of the deepest level, is a leaf).
This file states that rule in plain Python and checks it against the level
sizes of the oracle's recursive construction (Section 2.2.2), on random,
duplicated and tightly clustered inputs; the GPU trees themselves are
compared with the oracle's bit for bit by the GPU tests.
"""
import bisect

import numpy as np
import pytest

import oracle
from start_inputs import smoothing_lengths
from test_oracle_pins import PHYS

LEVELS = 21


def census(keys, leaf):
    n = len(keys)
    hist = [0] * (LEVELS + 1)
    for k in range(n):
        key = keys[k]
        lvl = 0
        if k > 0:
            x = keys[k - 1] ^ key
            lcp = (63 - x.bit_length()) // 3 if x else LEVELS
            lvl = lcp + 1
            if lvl <= LEVELS:   # the cell holding keys k - 1 and k must be split
                sh = 3 * (LEVELS - lcp)
                p = key >> sh
                lo = bisect.bisect_left(keys, p << sh, 0, k)
                hi = bisect.bisect_left(keys, (p + 1) << sh, k, n)
                if hi - lo <= leaf:
                    lvl = LEVELS + 1
        while lvl <= LEVELS:
            hist[lvl] += 1
            if lvl == 0:
                c = n
            else:
                sh = 3 * (LEVELS - lvl)
                c = bisect.bisect_left(keys, ((key >> sh) + 1) << sh, k, n) - k
            if c <= leaf or lvl == LEVELS:
                break
            lvl += 1
    return hist


def _problem(seed, n_p, n_s, kind):
    rng = np.random.default_rng(seed)
    pos = rng.uniform(0, 2.0, size=(3, n_p)).astype(np.float32)
    src = rng.uniform(0, 2.0, size=(3, n_s)).astype(np.float32)
    if kind in ("dup", "clustered"):
        pos[:, 1:20:2] = pos[:, 0:19:2]            # identical positions: level-21 leaves
    if kind == "clustered":
        pos[:, 100:160] = pos[:, 100:101] + np.float32(1e-4) * rng.uniform(
            0, 1, (3, 60)).astype(np.float32)
        src[:, 1::2] = src[:, 0::2] + np.float32(3e-5) * rng.uniform(
            0.1, 1, (3, n_s // 2)).astype(np.float32)
    h = smoothing_lengths(pos)
    L = rng.lognormal(np.log(1e48), 1.0, size=n_s)
    return pos, h, src, L


@pytest.mark.parametrize("kind", ["random", "dup", "clustered"])
@pytest.mark.parametrize("ptree_leaf", [1, 8, 16])
def test_level_census_matches_the_recursive_construction(kind, ptree_leaf):
    pos, h, src, L = _problem(7, 700, 64, kind)
    o = oracle.Oracle(pos, h, src, L, ptree_leaf=ptree_leaf, src_leaf=1, **PHYS)
    for which, leaf in ((0, ptree_leaf), (1, 1)):
        keys = sorted(int(v) for v in o.keys(which))
        levels = o.tree(which)["level"]
        ref = np.bincount(levels, minlength=LEVELS + 1).tolist()
        assert census(keys, leaf) == ref, (kind, which)
