"""Seeded synthetic workloads for the START radiative-transfer hot path.

This module only draws inputs: particle positions, smoothing lengths,
densities, emitter volumes, source positions and luminosities, and the
physical parameters a run is configured with.  It holds none of the
method's arithmetic (no trees, no optical depths, no rates), so both the
CUDA path and the FP64 oracle can consume what it produces.

The workloads stand in for the paper's test problems, which are not public
data (positions of the sources in Tests 1-6 are not given):

* ``config1`` / ``config2``: static uniform hydrogen with many point sources,
  shaped like Test 1 (Section 3.1.1, multiple sources in an optically thick
  uniform medium) but in a 6.6 kpc box.
* ``config3``: background gas with dense clumps, a central bright source and
  every particle emitting recombination photons, shaped like Test 6
  (Section 4.2.3, shadowing by a clump) with eight clumps.
* ``config4_requests``: a Poisson stream of solves of mixed size for the
  serving loop.
* ``config5``: a log-normal clumpy field with all particles emitting plus 64
  point sources.

Particles sit on a jittered lattice, coordinate = (i + 1/2 + U(-1/4, 1/4)) dx
per axis, and carry equal volume V = dx^3.  The smoothing length is chosen so
that each particle has exactly 32 neighbours inside 2h: 2h is set half-way
between the distances of the 32nd and 33rd nearest other particles.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

KPC_CM = 3.0857e21          # one kiloparsec in cm (length unit of every workload)
MYR_S = 3.15576e13          # one megayear in s

# Physical parameters of the monochromatic 13.6 eV, T = 1e4 K problem.  They
# are configuration values handed to both implementations, not derived here.
SIGMA_CM2 = 6.3e-18         # HI cross-section at the Lyman limit
ALPHA_B = 2.59e-13          # case-B recombination coefficient at 1e4 K, cm^3/s
ALPHA_A = 4.18e-13          # case-A recombination coefficient at 1e4 K, cm^3/s

N_NGB = 32                  # neighbours per smoothing kernel


@dataclass
class Workload:
    """One radiative-transfer problem in SoA float32 layout.

    pos      (3, N_p) float32, kpc
    h        (N_p,)   float32, kpc; neighbours are the particles within 2h
    n_H      (N_p,)   float32, cm^-3
    y0       (N_p,)   float64, initial neutral fraction y = 1 - x_HII
    V        (N_p,)   float64, particle volume in kpc^3
    src_pos  (3, N_s) float32, kpc
    src_L    (N_s,)   float64, ionising photons per second
    """
    name: str
    pos: np.ndarray
    h: np.ndarray
    n_H: np.ndarray
    y0: np.ndarray
    V: np.ndarray
    src_pos: np.ndarray
    src_L: np.ndarray
    box_kpc: float
    dx_kpc: float
    diffuse: bool = False
    thetas: tuple = (0.0, 0.5, 1.0)
    dt_s: float = MYR_S
    steps: int = 1
    params: dict = field(default_factory=dict)

    @property
    def n_p(self) -> int:
        return int(self.pos.shape[1])

    @property
    def n_s(self) -> int:
        return int(self.src_pos.shape[1])

    def n_HI(self) -> np.ndarray:
        """Neutral density n_H * y rounded to float32 (the solver's input)."""
        return (self.y0 * self.n_H.astype(np.float64)).astype(np.float32)


def default_params(diffuse: bool = False) -> dict:
    return dict(sigma_cm2=SIGMA_CM2, len_unit_cm=KPC_CM, alpha_A=ALPHA_A,
                alpha_B=ALPHA_B, diffuse=bool(diffuse), src_leaf=1)


def jittered_lattice(nside: int, box: float, rng: np.random.Generator,
                     jitter: float = 0.25) -> np.ndarray:
    """(3, nside^3) float32 positions (i + 1/2 + U(-jitter, jitter)) * dx."""
    dx = box / nside
    i = np.arange(nside, dtype=np.float64)
    gx, gy, gz = np.meshgrid(i, i, i, indexing="ij")
    g = np.stack([gx.ravel(), gy.ravel(), gz.ravel()])
    g = g + 0.5 + rng.uniform(-jitter, jitter, size=g.shape)
    return (g * dx).astype(np.float32)


def smoothing_lengths(pos: np.ndarray, n_ngb: int = N_NGB) -> np.ndarray:
    """h with 2h half-way between the n_ngb-th and (n_ngb+1)-th neighbour.

    Distances are taken between the float32 positions promoted to float64.
    Particles with fewer than n_ngb+1 others get 2h beyond the farthest one.
    """
    from scipy.spatial import cKDTree

    p = pos.T.astype(np.float64)
    n = p.shape[0]
    if n <= 1:
        return np.full(n, 1.0, dtype=np.float32)
    k = min(n_ngb + 2, n)
    tree = cKDTree(p)
    d, _ = tree.query(p, k=k, workers=-1)
    d = np.atleast_2d(d)
    if k == n_ngb + 2:
        two_h = 0.5 * (d[:, n_ngb] + d[:, n_ngb + 1])
    else:
        two_h = 1.01 * d[:, -1] + 1e-6
    h = (0.5 * two_h).astype(np.float32)
    return h


def uniform_sources(n_s: int, box: float, rng: np.random.Generator,
                    pos: np.ndarray, min_sep: float) -> np.ndarray:
    """(3, n_s) float32 positions uniform in the box, at least min_sep from
    every particle (redrawn until they are)."""
    from scipy.spatial import cKDTree

    tree = cKDTree(pos.T.astype(np.float64))
    out = np.empty((3, n_s), dtype=np.float32)
    filled = 0
    while filled < n_s:
        cand = rng.uniform(0.0, box, size=(n_s - filled, 3)).astype(np.float32)
        d, _ = tree.query(cand.astype(np.float64), k=1)
        ok = cand[d >= min_sep]
        out[:, filled:filled + len(ok)] = ok.T
        filled += len(ok)
    return out


def lattice_workload(name: str, nside: int, box: float, n_s: int, seed: int,
                     n_H: float = 1e-3, L=5e48, y0: float = 1.0,
                     diffuse: bool = False, jitter: float = 0.25) -> Workload:
    """Uniform-density jittered lattice with n_s uniform point sources.

    L is either a number (all sources equal) or a callable rng -> (n_s,) array.
    """
    rng = np.random.default_rng(seed)
    pos = jittered_lattice(nside, box, rng, jitter)
    dx = box / nside
    h = smoothing_lengths(pos)
    n = pos.shape[1]
    src = uniform_sources(n_s, box, rng, pos, 1e-3 * dx) if n_s else np.zeros((3, 0), np.float32)
    if callable(L):
        src_L = np.asarray(L(rng), dtype=np.float64)
    else:
        src_L = np.full(n_s, float(L), dtype=np.float64)
    return Workload(name=name, pos=pos, h=h,
                    n_H=np.full(n, n_H, dtype=np.float32),
                    y0=np.full(n, y0, dtype=np.float64),
                    V=np.full(n, dx ** 3, dtype=np.float64),
                    src_pos=src, src_L=src_L, box_kpc=box, dx_kpc=dx,
                    diffuse=diffuse, params=default_params(diffuse))


def config1(seed: int = 53121) -> Workload:
    """32^3 particles, 6.6 kpc box, n_H = 1e-3, neutral, 16 sources of 5e48/s;
    one solve plus a 1 Myr step at theta in {0, 0.5, 1}."""
    w = lattice_workload("plain-32^3-16src", 32, 6.6, 16, seed, L=5e48)
    w.thetas = (0.0, 0.5, 1.0)
    w.steps = 1
    return w


def config2(seed: int = 53122, nside: int = 64) -> Workload:
    """64^3 particles, 6.6 kpc box, n_H = 1e-3, 1024 sources with log-normal
    L (median 1e48/s, sigma_ln = 1); 20 coupled 1 Myr steps.  A smaller
    nside gives the same recipe on fewer particles (profiling cases)."""
    def lum(rng):
        return 1e48 * np.exp(rng.normal(0.0, 1.0, size=1024))
    w = lattice_workload(f"multisource-{nside}^3-1024src", nside, 6.6, 1024, seed, L=lum)
    w.thetas = (0.0, 0.5, 1.0)
    w.steps = 20
    return w


def _clump_density(pos: np.ndarray, centres: np.ndarray, r_c: float,
                   n_bg: float, n_c: float) -> np.ndarray:
    p = pos.T.astype(np.float64)
    n = np.full(p.shape[0], n_bg)
    for c in centres:
        inside = np.sum((p - c) ** 2, axis=1) < r_c * r_c
        n[inside] = n_c
    return n.astype(np.float32)


def config3(seed: int = 53123, nside: int = 128) -> Workload:
    """Diffuse recombination shadowing: background 2e-4 cm^-3, eight clumps of
    radius 0.8 kpc at 200x overdensity, one 3e51/s source at the box centre,
    every particle an emitter; theta = 0.7.  The box is 6.6 kpc."""
    box = 6.6
    rng = np.random.default_rng(seed)
    pos = jittered_lattice(nside, box, rng)
    dx = box / nside
    h = smoothing_lengths(pos)
    centres = rng.uniform(0.8, box - 0.8, size=(8, 3))
    n_H = _clump_density(pos, centres, 0.8, 2e-4, 0.04)
    n = pos.shape[1]
    # the central source is nudged off the lattice site it could coincide with
    src = np.array([[box / 2 + 0.123 * dx], [box / 2 + 0.071 * dx], [box / 2 + 0.037 * dx]],
                   dtype=np.float32)
    w = Workload(name=f"diffuse-{nside}^3-8clumps", pos=pos, h=h, n_H=n_H,
                 y0=np.full(n, 1.0 - 1.2e-3), V=np.full(n, dx ** 3),
                 src_pos=src, src_L=np.array([3e51]), box_kpc=box, dx_kpc=dx,
                 diffuse=True, thetas=(0.7,), params=default_params(True))
    return w


def gaussian_random_field(nside: int, rng: np.random.Generator, slope: float = -3.0) -> np.ndarray:
    """Unit-variance Gaussian field on nside^3 with power spectrum P(k) ~ k^slope."""
    white = rng.standard_normal((nside, nside, nside))
    fk = np.fft.rfftn(white)
    kx = np.fft.fftfreq(nside)[:, None, None]
    ky = np.fft.fftfreq(nside)[None, :, None]
    kz = np.fft.rfftfreq(nside)[None, None, :]
    k = np.sqrt(kx * kx + ky * ky + kz * kz)
    amp = np.zeros_like(k)
    amp[k > 0] = k[k > 0] ** (slope / 2.0)
    g = np.fft.irfftn(fk * amp, s=(nside, nside, nside), axes=(0, 1, 2))
    g -= g.mean()
    g /= g.std()
    return g


def config5(seed: int = 53125, nside: int = 256) -> Workload:
    """Log-normal clumpy field (sigma_ln rho = 1.5, P(k) ~ k^-3, mean n_H =
    1e-3 in a 6.6 kpc box), all particles emitting plus 64 point sources of
    1e50/s; theta in {0.5, 1}."""
    box = 6.6
    rng = np.random.default_rng(seed)
    pos = jittered_lattice(nside, box, rng)
    dx = box / nside
    h = smoothing_lengths(pos)
    g = gaussian_random_field(nside, rng).ravel()
    s = 1.5
    n_H = np.exp(s * g - 0.5 * s * s)
    n_H *= 1e-3 / n_H.mean()
    n = pos.shape[1]
    src = uniform_sources(64, box, rng, pos, 1e-3 * dx)
    return Workload(name=f"diffuse-lognormal-{nside}^3-64src", pos=pos, h=h,
                    n_H=n_H.astype(np.float32), y0=np.full(n, 1.0 - 1.2e-3),
                    V=np.full(n, dx ** 3), src_pos=src,
                    src_L=np.full(64, 1e50), box_kpc=box, dx_kpc=dx,
                    diffuse=True, thetas=(0.5, 1.0), steps=10,
                    params=default_params(True))


@dataclass
class Request:
    """One served solve: arrival time (s) and the recipe of its inputs."""
    rid: int
    t_arrive: float
    n_p: int
    n_s: int
    clumpy: bool
    theta: float
    seed: int

    def workload(self) -> Workload:
        rng = np.random.default_rng(self.seed)
        box = 6.6
        nside = int(math.ceil(self.n_p ** (1.0 / 3.0) - 1e-9))
        full = jittered_lattice(nside, box, rng)
        keep = np.sort(rng.choice(full.shape[1], size=self.n_p, replace=False))
        pos = np.ascontiguousarray(full[:, keep])
        dx = box / nside
        h = smoothing_lengths(pos)
        if self.clumpy:
            centres = rng.uniform(0.8, box - 0.8, size=(8, 3))
            n_H = _clump_density(pos, centres, 0.8, 2e-4, 0.04)
        else:
            n_H = np.full(self.n_p, 1e-3, dtype=np.float32)
        src = uniform_sources(self.n_s, box, rng, pos, 1e-3 * dx)
        src_L = 1e48 * np.exp(rng.normal(0.0, 1.0, size=self.n_s))
        return Workload(name=f"req{self.rid}", pos=pos, h=h, n_H=n_H,
                        y0=np.ones(self.n_p), V=np.full(self.n_p, dx ** 3),
                        src_pos=src, src_L=src_L, box_kpc=box, dx_kpc=dx,
                        thetas=(self.theta,), params=default_params(False))


def config4_requests(n_req: int = 256, rate_hz: float = 50.0, seed: int = 53124,
                     log2_np=(15.0, 21.0)) -> list:
    """Poisson stream of solves: exponential inter-arrivals (mean 1/rate),
    N_p = round(2^U(a, b)), N_s = round(exp(U(0, ln N_p))), uniform or clumpy
    density (coin flip), theta in {0.5, 1}."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate_hz, size=n_req))
    out = []
    for r in range(n_req):
        n_p = int(round(2.0 ** rng.uniform(*log2_np)))
        n_s = max(1, int(round(math.exp(rng.uniform(0.0, math.log(n_p))))))
        out.append(Request(rid=r, t_arrive=float(t[r]), n_p=n_p, n_s=n_s,
                           clumpy=bool(rng.integers(0, 2)),
                           theta=float(rng.choice([0.5, 1.0])),
                           seed=int(seed * 1000 + r)))
    return out


CONFIGS = {1: config1, 2: config2, 3: config3, 5: config5}
