"""SPH density (Section 2.1) through the C ABI against the FP64 oracle.

Tolerance: every term m_k W(r_ik, h_i) is positive and carries a few
float32 roundings (offsets, root, q = r/h, the spline), the sum of ~33 such
terms and the 1/(pi h^3) factor add some more: a relative error of a few
1e-6.  The tests allow 2e-5 relative, element by element.
"""
import math

import numpy as np
import pytest

import oracle
from start_inputs import KPC_CM, SIGMA_CM2, ALPHA_A, ALPHA_B, config1, config2, smoothing_lengths

pytestmark = pytest.mark.gpu
REL = 2e-5
PHYS = dict(sigma_cm2=SIGMA_CM2, len_unit_cm=KPC_CM, alpha_A=ALPHA_A, alpha_B=ALPHA_B)


@pytest.fixture(scope="module")
def S():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1005_5312_gb300 as S
    S.build()
    return S


def pair(S, pos, h, src=None, L=None):
    src = np.zeros((3, 0), np.float32) if src is None else src
    L = np.zeros(0) if L is None else L
    ctx = S.Context(ptree_leaf=16)
    ctx.build_trees(pos, h, src, L)
    orc = oracle.Oracle(pos, h, src, L, ptree_leaf=16, **PHYS)
    return ctx, orc


def close(rho, ref):
    rho = np.asarray(rho, np.float64)
    err = np.abs(rho - ref)
    bad = np.nonzero(err > REL * np.abs(ref))[0]
    assert len(bad) == 0, (len(bad), bad[:5], rho[bad[:5]], ref[bad[:5]])


def test_density_parity_config1_lognormal_masses(S):
    w = config1()
    ctx, orc = pair(S, w.pos, w.h, w.src_pos, w.src_L)
    m = np.random.default_rng(3).lognormal(0.0, 1.0, w.n_p).astype(np.float32)
    close(ctx.sph_density(m), orc.sph_density(m.astype(np.float64)))


def test_density_parity_random_with_duplicates_and_wide_kernels(S):
    """Random positions (a ragged count), two coincident pairs, every third
    particle with a 2x smoothing length (~250 neighbours)."""
    rng = np.random.default_rng(21)
    pos = rng.uniform(0, 2.0, size=(3, 4099)).astype(np.float32)
    pos[:, 1] = pos[:, 0]
    pos[:, 3] = pos[:, 2]
    h = smoothing_lengths(pos)
    h[::3] *= np.float32(2.0)
    ctx, orc = pair(S, pos, h)
    m = rng.uniform(0.0, 3.0, pos.shape[1]).astype(np.float32)
    m[7] = 0.0
    close(ctx.sph_density(m), orc.sph_density(m.astype(np.float64)))


def test_density_device_buffers_and_single_particle(S):
    import torch
    w = config1()
    ctx, orc = pair(S, w.pos, w.h)
    m = torch.full((w.n_p,), 0.75, dtype=torch.float32, device="cuda")
    out = torch.zeros(w.n_p, dtype=torch.float32, device="cuda")
    ctx.sph_density(m, out)
    torch.cuda.synchronize()
    close(out.cpu().numpy(), orc.sph_density(np.full(w.n_p, 0.75)))
    # one particle: only itself, W(0, h) = 1 / (pi h^3)
    p1 = np.array([[0.5], [0.5], [0.5]], np.float32)
    h1 = np.array([0.3], np.float32)
    c1 = S.Context()
    c1.build_trees(p1, h1, np.zeros((3, 0), np.float32), np.zeros(0))
    r1 = c1.sph_density(np.array([2.0], np.float32))
    assert r1[0] == pytest.approx(2.0 / (math.pi * 0.3 ** 3), rel=REL)


def test_density_rejects_bad_input(S):
    w = config1()
    ctx = S.Context()
    with pytest.raises(S.StartError):
        ctx.sph_density(np.ones(w.n_p, np.float32))      # trees not built
    ctx.build_trees(w.pos, w.h, w.src_pos, w.src_L)
    m = np.ones(w.n_p, np.float32)
    m[5] = -1.0
    with pytest.raises(S.StartError):
        ctx.sph_density(m)
    m[5] = np.nan
    with pytest.raises(S.StartError):
        ctx.sph_density(m)
    m[5] = 1.0
    assert np.all(np.isfinite(ctx.sph_density(m)))      # usable after the errors
    ctx.set_state(w.n_H, w.y0)                           # no stale input error left


def test_density_full_size_multisource_workload(S):
    """The 64^3 benchmark workload, every particle."""
    w = config2()
    ctx, orc = pair(S, w.pos, w.h, w.src_pos, w.src_L)
    m = np.random.default_rng(4).uniform(0.5, 1.5, w.n_p).astype(np.float32)
    close(ctx.sph_density(m), orc.sph_density(m.astype(np.float64)))


def test_density_without_particles(S):
    ctx = S.Context()
    ctx.build_trees(np.zeros((3, 0), np.float32), np.zeros(0, np.float32),
                    np.zeros((3, 1), np.float32), np.ones(1))
    assert ctx.sph_density(np.zeros(0, np.float32)).size == 0
