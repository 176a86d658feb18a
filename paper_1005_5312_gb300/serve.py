"""Continuous batching of radiative-transfer solves on one GPU.

Requests (particles, sources, theta, steps) arrive over time.  A request is
admitted, in arrival order, as soon as a worker slot is free and its
estimated device memory fits the remaining budget; each worker owns a
library context on its own CUDA stream, so the kernels of admitted requests
overlap on the GPU while their host threads wait in the library (ctypes
releases the GIL).  Library buffers come from a stream-ordered pool, so one
request growing its buffers never synchronises the others.  A worker keeps
its context (and therefore its grown buffers) from request to request,
unless the library's memory in use then exceeds the trim threshold: the
worker's context is then recreated, returning its buffers.  A request that
runs out of device memory is retried once on a fresh context.

`serve(requests, workers=1)` is the plain baseline: one solve at a time.
Every request's results are the same whether it runs alone or in a mix
(the solve is deterministic).

With batch_small > 1, a worker that takes a small request (at most
small_n_p particles) also takes the small requests that have already
arrived and share its theta, time step and step count, up to batch_small of
them, and solves them as one batch (start_build_batch): every kernel of the
solve then runs once for the whole batch, and each request's results are
bitwise those of solving it alone.
"""
from __future__ import annotations

import math
import threading
import time
from dataclasses import dataclass, field

import numpy as np

from . import Context, lib

# device bytes per particle (records, h, n_H, y, V, Gamma, trees, neighbour
# lists) and per interaction pair (entry, target, contribution, memoised
# chain state and its hash-table share), with headroom
BYTES_PER_PARTICLE = 480
BYTES_PER_PAIR = 150


def list_length_estimate(n_s: int, theta: float) -> float:
    """Expected interaction-list length per target (fit to measurements on
    uniform workloads: 321 at N_s = 1024, theta = 0.5; 146 at theta = 1)."""
    if n_s <= 0:
        return 0.0
    return min(float(n_s), 14.0 * math.log2(n_s + 1) / max(theta, 0.05) ** 1.2 + 8.0)


def memory_estimate(n_p: int, n_s: int, theta: float, max_pairs: int) -> int:
    pairs = min(n_p * list_length_estimate(n_s, theta), float(max_pairs))
    return int(BYTES_PER_PARTICLE * (n_p + n_s) + BYTES_PER_PAIR * pairs) + (64 << 20)


@dataclass
class SolveRequest:
    rid: int
    t_arrive: float          # seconds after the start of the stream
    pos: np.ndarray          # (3, n_p) float32
    h: np.ndarray
    src_pos: np.ndarray
    src_L: np.ndarray
    n_H: np.ndarray
    y0: np.ndarray
    theta: float
    dt: float
    steps: int = 1

    @property
    def n_p(self):
        return int(self.h.shape[0])

    @property
    def n_s(self):
        return int(self.src_L.shape[0])


@dataclass
class SolveResult:
    rid: int
    t_arrive: float
    t_admit: float
    t_done: float
    gamma: np.ndarray
    y: np.ndarray
    rays: int
    mem_estimate: int

    @property
    def latency(self):
        return self.t_done - self.t_arrive


@dataclass
class _Worker:
    ctx: Context
    stream: object
    busy: bool = False


def request_knobs(req, reuse_fixed: bool = False, tuner=None) -> dict:
    """Parameters a worker sets before serving req: resident chains only for
    a request of several coupled steps (unless the server fixed them), and
    the tuner's knobs of the request's problem class."""
    knobs = {} if reuse_fixed else {"reuse_chains": int(req.steps > 1)}
    if tuner is not None:
        knobs.update(tuner.params_for(req.n_p, req.n_s, req.theta))
    return knobs


class Server:
    """FIFO admission by worker slots and a device-memory budget."""

    def __init__(self, workers: int = 4, budget_bytes: float = 150e9, max_pairs: int = 1 << 27,
                 tuner=None, trim_bytes: float = None, batch_small: int = 0,
                 small_n_p: int = 1 << 16, **params):
        import torch
        self.torch = torch
        self.budget = float(budget_bytes)
        self.trim_bytes = 0.5 * self.budget if trim_bytes is None else float(trim_bytes)
        self.retries = 0
        self.trims = 0
        self.max_pairs = int(max_pairs)
        # resident chains pay off over several coupled steps of one request;
        # unless fixed here, each request sets them by its step count
        self.reuse_fixed = "reuse_chains" in params
        self.params = dict(dict(reuse_chains=1), **params, max_pairs=self.max_pairs)
        self.workers = []
        for _ in range(max(1, workers)):
            st = torch.cuda.Stream()
            self.workers.append(_Worker(Context(stream=st, **self.params), st))
        self.tuner = tuner
        self.batch_small = int(batch_small)
        self.small_n_p = int(small_n_p)
        self.batches = 0
        self.cv = threading.Condition()
        self.reserved = 0.0
        self.results = []
        self.errors = []

    def close(self):
        for w in self.workers:
            w.ctx.close()

    def _fresh_context(self, w: _Worker):
        """Recreate a worker's context: its grown buffers go back to the pool."""
        w.ctx.close()
        w.ctx = Context(stream=w.stream, **self.params)

    def _run(self, ctx, req: SolveRequest):
        knobs = request_knobs(req, self.reuse_fixed, self.tuner)
        if knobs:
            ctx.set_params(**knobs)
        ctx.build_trees(req.pos, req.h, req.src_pos, req.src_L)
        y = np.ascontiguousarray(req.y0, dtype=np.float64).copy()
        g = np.zeros(req.n_p, np.float32)
        rays = 0
        for _ in range(req.steps):
            ctx.set_state(req.n_H, y)
            ctx.rt_solve(req.theta, gamma_out=g)
            ctx.ionize(req.dt, y_out=y)
            rays += ctx.stats()["rays"]
        return g, y, rays

    def _run_batch(self, ctx, reqs):
        """Several small requests as one batch; returns [(g, y, rays)] per request."""
        r0 = reqs[0]
        ctx.build_batch([(r.pos, r.h, r.src_pos, r.src_L) for r in reqs])
        off = np.cumsum([0] + [r.n_p for r in reqs])
        nH = np.concatenate([np.asarray(r.n_H, np.float32) for r in reqs])
        y = np.concatenate([np.asarray(r.y0, np.float64) for r in reqs])
        g = np.zeros(int(off[-1]), np.float32)
        rays = 0
        for _ in range(r0.steps):
            ctx.set_state(nH, y)
            ctx.rt_solve(r0.theta, gamma_out=g)
            ctx.ionize(r0.dt, y_out=y)
            rays += ctx.stats()["rays"]
        share = [r.n_p / max(1, int(off[-1])) for r in reqs]
        return [(g[off[b]:off[b + 1]].copy(), y[off[b]:off[b + 1]].copy(), int(rays * share[b]))
                for b in range(len(reqs))]

    def _solve(self, w: _Worker, reqs, t0: float, t_admit: float, est: int):
        from . import START_ENOMEM, StartError
        if not isinstance(reqs, list):
            reqs = [reqs]
        try:
            def run():
                if len(reqs) == 1:
                    return [self._run(w.ctx, reqs[0])]
                return self._run_batch(w.ctx, reqs)
            try:
                outs = run()
            except StartError as e:
                if e.code != START_ENOMEM:
                    raise
                self._fresh_context(w)            # out of memory: once more, from scratch
                with self.cv:
                    self.retries += 1
                outs = run()
            t_done = time.perf_counter() - t0
            with self.cv:
                if len(reqs) > 1:
                    self.batches += 1
                for req, (g, y, rays) in zip(reqs, outs):
                    self.results.append(SolveResult(req.rid, req.t_arrive, t_admit, t_done, g, y,
                                                    rays, est))
            if memory_in_use() > self.trim_bytes:
                self._fresh_context(w)
                with self.cv:
                    self.trims += 1
        except Exception as e:  # reported by serve()
            with self.cv:
                self.errors.append((reqs[0].rid, repr(e)))
        finally:
            with self.cv:
                w.busy = False
                self.reserved -= est
                self.cv.notify_all()

    def serve(self, requests, realtime: bool = True) -> list:
        """Replay the requests at their arrival times (realtime) or back to
        back, admit them FIFO, and return the results in request order."""
        reqs = sorted(requests, key=lambda r: (r.t_arrive, r.rid))
        self.results, self.errors = [], []
        threads = []
        t0 = time.perf_counter()
        i = 0
        while i < len(reqs):
            req = reqs[i]
            i += 1
            if realtime:
                wait = req.t_arrive - (time.perf_counter() - t0)
                if wait > 0:
                    time.sleep(wait)
            est = memory_estimate(req.n_p, req.n_s, req.theta, self.max_pairs)
            with self.cv:
                while True:
                    free = [w for w in self.workers if not w.busy]
                    fits = self.reserved + est <= self.budget or self.reserved == 0.0
                    if free and fits:
                        w = free[0]
                        w.busy = True
                        self.reserved += est
                        break
                    self.cv.wait()
                batch = [req]
                if self.batch_small > 1 and req.n_p <= self.small_n_p:
                    # the compatible small requests that have arrived meanwhile
                    now = time.perf_counter() - t0 if realtime else float("inf")
                    while (i < len(reqs) and len(batch) < self.batch_small and
                           reqs[i].t_arrive <= now and reqs[i].n_p <= self.small_n_p and
                           reqs[i].theta == req.theta and reqs[i].dt == req.dt and
                           reqs[i].steps == req.steps):
                        e = memory_estimate(reqs[i].n_p, reqs[i].n_s, reqs[i].theta,
                                            self.max_pairs)
                        if self.reserved + e > self.budget:
                            break
                        self.reserved += e
                        est += e
                        batch.append(reqs[i])
                        i += 1
            t_admit = time.perf_counter() - t0
            th = threading.Thread(target=self._solve, args=(w, batch, t0, t_admit, est),
                                  daemon=True)
            th.start()
            threads.append(th)
        for th in threads:
            th.join()
        if self.errors:
            raise RuntimeError(f"{len(self.errors)} requests failed: {self.errors[:3]}")
        return sorted(self.results, key=lambda r: r.rid)


def summarize(results, t_first_arrival: float = 0.0) -> dict:
    lat = np.array([r.latency for r in results])
    span = max(r.t_done for r in results) - t_first_arrival
    return {"solves_per_s": len(results) / span, "p50_ms": 1e3 * float(np.percentile(lat, 50)),
            "p99_ms": 1e3 * float(np.percentile(lat, 99)), "makespan_s": span,
            "rays_per_s": sum(r.rays for r in results) / span, "n": len(results)}


def make_request(rid: int, n_p: int, n_s: int, clumpy: bool, theta: float, t_arrive: float = 0.0,
                 seed: int = 53124, steps: int = 1, dt: float = 3.15576e13) -> SolveRequest:
    """One request: particles on a jittered lattice of the requested size in
    a 6.6 kpc box with 2h = 2.04 spacings (about 33 neighbours), uniform
    n_H = 1e-3 or eight 200x clumps on 2e-4, sources uniform with
    L = 1e48 exp(N(0, 1)).  The arrays depend only on (seed, rid)."""
    rng = np.random.default_rng((seed, rid))
    box = 6.6
    nside = int(math.ceil(n_p ** (1.0 / 3.0) - 1e-9))
    dx = box / nside
    keep = np.sort(rng.choice(nside ** 3, size=n_p, replace=False))
    ijk = np.stack(np.unravel_index(keep, (nside, nside, nside))).astype(np.float64)
    pos = ((ijk + 0.5 + rng.uniform(-0.25, 0.25, size=ijk.shape)) * dx).astype(np.float32)
    h = np.full(n_p, 1.02 * dx, np.float32)
    if clumpy:
        n_H = np.full(n_p, 2e-4)
        for c in rng.uniform(0.8, box - 0.8, size=(8, 3)):
            inside = np.sum((pos.T.astype(np.float64) - c) ** 2, axis=1) < 0.64
            n_H[inside] = 0.04
        n_H = n_H.astype(np.float32)
    else:
        n_H = np.full(n_p, 1e-3, np.float32)
    src = rng.uniform(0.0, box, size=(3, n_s)).astype(np.float32)
    src_L = 1e48 * np.exp(rng.normal(0.0, 1.0, size=n_s))
    return SolveRequest(rid, float(t_arrive), np.ascontiguousarray(pos), h, src, src_L, n_H,
                        np.ones(n_p), float(theta), dt, steps)


def make_requests(n_req: int = 256, rate_hz: float = 50.0, log2_np=(15.0, 21.0), seed: int = 53124,
                  steps: int = 1, dt: float = 3.15576e13) -> list:
    """Config-4-shaped stream: exponential inter-arrivals, N_p = 2^U(a, b),
    N_s = exp(U(0, ln N_p)), uniform or clumpy density (coin flip), theta in
    {0.5, 1}; request r's recipe and arrays do not depend on n_req."""
    t = np.cumsum(np.random.default_rng(seed).exponential(1.0 / rate_hz, size=n_req))
    out = []
    for r in range(n_req):
        rng = np.random.default_rng((seed, r, 1))
        n_p = int(round(2.0 ** rng.uniform(*log2_np)))
        n_s = max(1, int(round(math.exp(rng.uniform(0.0, math.log(n_p))))))
        clumpy = bool(rng.integers(0, 2))
        theta = float(rng.choice([0.5, 1.0]))
        out.append(make_request(r, n_p, n_s, clumpy, theta, float(t[r]), seed, steps, dt))
    return out


def memory_in_use() -> int:
    return int(lib().start_memory_in_use())
