#!/usr/bin/env python3
"""Benchmark of the START hot path on one GB300 (or N replicas under torchrun).

The headline workload is the large diffuse run: 256^3 = 16777216 particles
on a jittered lattice in a 6.6 kpc box, log n_H a Gaussian random field
(P(k) ~ k^-3, sigma_ln = 1.5, mean 1e-3 cm^-3), every particle emitting
recombination photons plus 64 point sources of 1e50 photons/s.  A step is
one pass of the whole path: frame, Morton keys, sorts, source, particle and
emitter octrees, moments, neighbour lists, the SPH density recompute from
the particle masses (Section 2.1), the emitters' luminosities and moments,
the walk, the memoised ray march, Gamma, and the implicit 1 Myr ionisation
update with the diffuse self term, coupled from step to step.  The metric
is rays per second (a ray is one (target, virtual source) pair whose
optical depth is evaluated and added to Gamma); theta_crit = 0.5 is the
headline and 1.0 is reported beside it.  The 64^3 multiple-source set, the
128^3 diffuse set and the served request stream are reported as extra keys.

Prints one JSON line.  --impl reference times the FP64 oracle on the host
cores on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# algorithmic bytes of the march (per neighbour-list evaluation: 32 u32
# indices + 32 float3 positions + 1 float n_HI), per ray (virtual-source
# record) and per target (Gamma out)
ALGO_BYTES_PER_EVAL = 516
ALGO_BYTES_PER_RAY = 16
ALGO_BYTES_PER_TARGET = 8
L2_FLUSH_BYTES = 512 << 20
G_REL = 1e-4


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--theta", type=float, default=0.5)
    ap.add_argument("--theta2", type=float, default=1.0)
    ap.add_argument("--march-group", type=int, default=2)
    ap.add_argument("--row-bins", type=int, default=4,
                    help="first-hop direction bins per cube-face edge (0: scan every neighbour)")
    ap.add_argument("--max-pairs", type=int, default=3_000_000_000,
                    help="interaction pairs per group of the large run (device memory of the "
                         "march about 60 B per pair)")
    ap.add_argument("--nside", type=int, default=256,
                    help="lattice side of the headline workload (256: the benchmark; "
                         "smaller: profiling cases)")
    ap.add_argument("--side-steps", type=int, default=3,
                    help="timed steps of the theta2 and end-to-end lines")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-theta2", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0,
                    help="oracle work per CPU-baseline measurement")
    ap.add_argument("--ref-targets", type=int, default=256,
                    help="targets per step of the reference arm")
    ap.add_argument("--no-extras", action="store_true",
                    help="only the headline workload (no 64^3, 128^3 or serving lines)")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-resident", action="store_true")
    ap.add_argument("--no-diffuse", action="store_true")
    ap.add_argument("--no-next", action="store_true",
                    help="skip the SPH density, H2 photodissociation, blackbody-source and "
                         "recombination-band lines")
    ap.add_argument("--no-method-error", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=256)
    ap.add_argument("--serve-rate", type=float, default=50.0)
    ap.add_argument("--serve-low-rate", type=float, default=8.0)
    ap.add_argument("--serve-low-requests", type=int, default=96)
    ap.add_argument("--serve-workers", type=int, default=4)
    ap.add_argument("--serve-log2np", default="15,21")
    ap.add_argument("--serve-small-log2np", default="11,15",
                    help="particle counts of the small-request stream (log2 range)")
    ap.add_argument("--serve-small-rate", type=float, default=2000.0)
    ap.add_argument("--serve-small-requests", type=int, default=512)
    ap.add_argument("--serve-small-workers", type=int, default=8)
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reduce_over_ranks(seconds, units):
    """Whole-job figures of independent replicas: the slowest rank's time and
    the units all ranks processed (an initialised process group, any backend;
    one rank: unchanged)."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return seconds, units
    gathered = [None] * dist.get_world_size()
    dist.all_gather_object(gathered, (seconds, units))
    return max(x[0] for x in gathered), sum(x[1] for x in gathered)


class ClockSampler:
    """nvidia-smi clock/throttle samples while the timed region runs."""

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in self.rows if len(r) > 2 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) > 2 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            for k, nm in enumerate(names):
                if len(r) > 5 + k and r[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(self.rows)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def sources_sha() -> str:
    """sha256 (16 hex digits) of every CUDA source of the library: recorded
    DRAM traffic stays valid only while none of the kernels has changed."""
    import hashlib
    d = os.path.join(ROOT, "paper_1005_5312_gb300", "csrc")
    h = hashlib.sha256()
    for name in sorted(os.listdir(d)):
        if name.endswith((".cu", ".cuh")):
            with open(os.path.join(d, name), "rb") as f:
                h.update(name.encode() + b"\0" + f.read())
    return h.hexdigest()[:16]


def traffic_record(key: str):
    """DRAM bytes per step from a committed ncu summary, if it was taken on
    the current kernels (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f).get(key)
    if not d or d.get("sources_sha") != sources_sha():
        return None
    return d


def rel_errors(g, ref, g_abs):
    """Relative deviation of the GPU Gamma from the oracle's where the oracle
    is above the absolute floor, and the count outside the tolerance."""
    g = np.asarray(g, np.float64)
    ref = np.asarray(ref, np.float64)
    err = np.abs(g - ref)
    over = int(np.sum(err > G_REL * np.abs(ref) + g_abs))
    m = ref > g_abs
    rel = err[m] / ref[m]
    if rel.size == 0:
        rel = np.zeros(1)
    return {"targets": int(len(ref)), "above_floor": int(m.sum()),
            "max_rel": float(rel.max()), "p99_rel": float(np.percentile(rel, 99)),
            "median_rel": float(np.median(rel)), "outside_tolerance": over,
            "tolerance": f"|dG| <= {G_REL:g} G_oracle + {g_abs:.3g}"}


# ---------------------------------------------------------------- reference arm
def run_reference(args):
    """The FP64 oracle as it stands, on the host cores, on a bounded sample of
    the headline workload: Gamma at random targets each step (the trees and
    neighbour lists built once, outside the timed steps)."""
    import oracle
    from start_inputs import config5
    ws, rank, _ = dist_env()
    if rank != 0:
        return None
    oracle.build()
    w = config5(nside=args.nside)
    orc = oracle.Oracle.from_workload(w, ptree_leaf=16)
    orc.set_emitters(w.y0, w.n_H)
    nHI = w.n_HI()
    rng = np.random.default_rng(7)
    per_step = min(w.n_p, args.ref_targets)
    times, rays = [], []
    for s in range(args.warmup + args.steps):
        idx = rng.choice(w.n_p, per_step, replace=False)
        t0 = time.perf_counter()
        orc.gamma(nHI, args.theta, targets=idx)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            times.append(dt)
            rays.append(orc.last_stats["rays"])
    v = sum(rays) / sum(times)
    cores = oracle.threads()
    return {"impl": "reference", "metric": f"RT rays/s at theta_crit={args.theta}",
            "value": v, "unit": "rays/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": w.name, "n_p": w.n_p, "n_s": w.n_s, "emitters": w.n_p,
                       "theta": args.theta, "sample": f"{per_step} random targets per step"},
            "cpu_baseline": {"value": v, "unit": "rays/s", "cores": cores, "kind": "oracle",
                             "sample": f"Gamma at {per_step} random targets of {w.n_p} per step "
                                       f"(all emitters and point sources, neutral start)"},
            "e2e": {"value": v, "unit": "rays/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def oracle_sample(w, theta, seconds, seed=5, chunk=None):
    """The oracle as it stands on the host cores: Gamma at random targets of
    the workload's starting state, in chunks until `seconds` of work.
    Returns (targets, Gamma, rays, seconds, threads)."""
    import oracle
    oracle.build()
    orc = oracle.Oracle.from_workload(w, ptree_leaf=16)
    if w.diffuse:
        orc.set_emitters(w.y0, w.n_H)
    nHI = w.n_HI()
    order = np.random.default_rng(seed).permutation(w.n_p)
    chunk = chunk or max(64, 4 * oracle.threads())
    done, rays, t = 0, 0, 0.0
    parts = []
    while t < seconds and done < w.n_p:
        idx = order[done:done + chunk]
        t0 = time.perf_counter()
        parts.append(orc.gamma(nHI, theta, targets=idx))
        t += time.perf_counter() - t0
        rays += orc.last_stats["rays"]
        done += len(idx)
    return order[:done], np.concatenate(parts), rays, t, oracle.threads()


# Per-phase models of the algorithmic bytes of a step (each phase's
# compulsory traffic: what its kernels must read and write once), from the
# step's own counts.  st: summed counters of the step; w: the workload.
def phase_models(st, n_p, n_s, diffuse, chunk_count):
    rays, links = st["rays"], st["evals"]
    off = max(0, links - rays)          # chain links outside the interaction lists
    nb = st["nbr_total"]
    nodes = st["nodes_part"] + st["nodes_src"] + (st["nodes_emit"] if diffuse else 0)
    return {
        # frame, keys, 8 radix passes (key + index in and out), octree records,
        # neighbour search (its CSR written) and the records of the particles
        "build": {"kernels": "k_bbox, k_morton, k_rs_*, k_level_census, octree levels, "
                             "k_moments_*, k_neighbours, k_nb_compact",
                  "bytes": n_p * (12 + 4 + 8 + 8 * 24 + 16 + 8) + nb * 4 + nodes * 64,
                  "model": "per particle: position, h, key, 8 radix passes x 24 B, record, CSR "
                           "offsets; 4 B per neighbour; 64 B per octree node"},
        "density": {"kernels": "k_mass_to_morton, k_sph_density",
                    "bytes": n_p * 36 + nb * 24,
                    "model": "per particle 36 B (mass gather, record, h, offsets, result); "
                             "per neighbour 24 B (index, record, mass)"},
        "emit": {"kernels": "k_emitters, k_moments_level",
                 "bytes": (n_p * 32 + st["nodes_emit"] * 64) if diffuse else 0,
                 "model": "per particle 32 B (y, n_H, V, L out); 64 B per emitter-tree node"},
        "walk": {"kernels": "k_walk (count, fill; or one walk into scratch rows and "
                            "k_walk_compact; the fill writes the order keys), k_walk_hist, "
                            "k_row_bins",
                 "bytes": rays * 12 + n_p * 16 * chunk_count,
                 "model": "per pair 12 B (canonical id written, read, order key written); per "
                          "target and walk its 16 B record"},
        "hops": {"kernels": "k_memo_hop_rows, k_memo_hop_hard, k_memo_hop<G>, k_memo_tail",
                 "bytes": links * 32 + off * ALGO_BYTES_PER_EVAL + n_p * chunk_count * 676,
                 "model": "per chain link 32 B (id, order key and its direction bin's candidate "
                          "mask read; state (next, d_tau), length and next written); per link "
                          "outside the lists its neighbour list (516 B); per target and chunk its "
                          "staged neighbour list (33 x 20 B + 16 B)"},
        "link": {"kernels": "k_memo_link, k_memo_resolve",
                 "bytes": off * 56 + rays * 8,
                 "model": "per link outside the lists 56 B (upstream, id, key, table entry, "
                          "claimed slot, next written); per pair 8 B (row search)"},
        "jump": {"kernels": "k_memo_jump8<3, 12>",
                 "bytes": st["jump_bytes"],
                 "model": "8 B own state (next, FP32 sum) per slot and round; 16 B per slot "
                          "that advances (first successor read and the write); 8 B per further "
                          "successor read; 8 B per closed chain copied once"},
        "gamma": {"kernels": "k_memo_gamma",
                  "bytes": rays * 12 + n_p * 8,
                  "model": "per pair 12 B (8-byte chain state, id); per target 8 B"},
        "ionize": {"kernels": "k_ionize",
                   "bytes": n_p * (36 if diffuse else 28),
                   "model": "per particle: y read and written (16), Gamma (4), n_H (4), n_HI "
                            "(4), V (8, diffuse)"},
    }


def kernel_table(phase_ms, models, step_ms, peak):
    rows = []
    for name, m in models.items():
        ms = phase_ms.get(name)
        if ms is None or ms < 0:
            continue
        gbs = m["bytes"] / (ms * 1e-3) / 1e9 if ms > 0 else 0.0
        rows.append({"phase": name, "kernels": m["kernels"], "ms_per_step": ms,
                     "share_of_step": ms / step_ms, "algorithmic_bytes_per_step": m["bytes"],
                     "achieved_GB_per_s": gbs, "frac_of_measured_hbm": gbs / peak,
                     "bytes_model": m["model"]})
    rows.sort(key=lambda r: -r["ms_per_step"])
    return rows


def headline(S, w, dev, args, T, clk_index):
    """The headline workload: W untimed and K timed coupled steps at theta,
    then the theta2 line; per-step CUDA events on the context's stream."""
    import torch
    stream = torch.cuda.current_stream(dev)
    ctx = S.Context(timing=1, march_group=args.march_group, row_bins=args.row_bins, stream=stream,
                    max_pairs=args.max_pairs)
    pos, h, sp, sL, V = T(w.pos), T(w.h), T(w.src_pos), T(w.src_L), T(w.V)
    mass = T((w.n_H.astype(np.float64) * w.V).astype(np.float32))
    rho = torch.zeros(w.n_p, dtype=torch.float32, device=dev)
    y0 = T(w.y0)
    y = y0.clone()
    g = torch.zeros(w.n_p, dtype=torch.float32, device=dev)

    def step(theta):
        ctx.build_trees(pos, h, sp, sL, V, diffuse=True)
        ctx.sph_density(mass, rho)
        ctx.set_state(rho, y)
        ctx.rt_solve(theta, gamma_out=g)
        ctx.ionize(w.dt_s, y_out=y)

    def run(theta, steps, warmup, clock=None):
        y.copy_(y0)
        for _ in range(warmup):
            step(theta)
        torch.cuda.synchronize(dev)
        ctx.timings()                       # reset the phase sums
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        stats, phases = [], []
        l0 = ctx.stats()["launches"]
        if args.gpus > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize(dev)
        if clock:
            clock.__enter__()
        t_wall = time.perf_counter()
        for e0, e1 in ev:
            e0.record(stream)
            step(theta)
            e1.record(stream)
            phases.append(ctx.timings())     # synchronises
            stats.append(ctx.stats())
        if args.gpus > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize(dev)
        t_wall = time.perf_counter() - t_wall
        if clock:
            clock.__exit__()
        step_ms = [a.elapsed_time(b) for a, b in ev]
        launches = ctx.stats()["launches"] - l0
        return dict(step_ms=step_ms, stats=stats, phases=phases, launches=launches, wall=t_wall)

    clk = ClockSampler(clk_index)
    r1 = run(args.theta, args.steps, args.warmup, clk)
    r2 = None if args.no_theta2 else run(args.theta2, args.side_steps, 1)
    # the starting state once more, for the parity check against the oracle
    g_start = None
    if not args.no_cpu:
        ctx.build_trees(pos, h, sp, sL, V, diffuse=True)
        ctx.set_state(T(w.n_H), y0)
        g0 = torch.zeros(w.n_p, dtype=torch.float32, device=dev)
        ctx.rt_solve(args.theta, gamma_out=g0)
        g_start = g0.cpu().numpy()
    ctx.close()
    return r1, r2, clk.summary(), g_start


def headline_e2e(S, w, args):
    """The same step through the C ABI with host buffers (numpy arrays): every
    step copies its inputs to the device and Gamma and y back."""
    ctx = S.Context(march_group=args.march_group, row_bins=args.row_bins, max_pairs=args.max_pairs)
    mass = (w.n_H.astype(np.float64) * w.V).astype(np.float32)
    rho = np.zeros(w.n_p, np.float32)
    y = w.y0.copy()
    g = np.zeros(w.n_p, np.float32)

    def step():
        ctx.build_trees(w.pos, w.h, w.src_pos, w.src_L, w.V, diffuse=True)
        ctx.sph_density(mass, rho)
        ctx.set_state(rho, y)
        ctx.rt_solve(args.theta, gamma_out=g)
        ctx.ionize(w.dt_s, y_out=y)

    step()
    y[:] = w.y0
    rays = 0
    t0 = time.perf_counter()
    for _ in range(args.side_steps):
        step()
        rays += ctx.stats()["rays"]
    te, rays = reduce_over_ranks(time.perf_counter() - t0, rays)
    ctx.close()
    h2d = w.pos.nbytes + w.h.nbytes + w.src_pos.nbytes + w.src_L.nbytes + w.V.nbytes + \
        mass.nbytes + rho.nbytes + y.nbytes
    d2h = rho.nbytes + g.nbytes + y.nbytes
    return {"value": rays / te, "unit": "rays/s", "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "ms_per_step": 1e3 * te / args.side_steps,
            "steps": args.side_steps,
            "note": "numpy host buffers through the C ABI: positions, h, sources, V, masses "
                    "and y copied in, the density, Gamma and y copied out, every step"}


def resident_steps(S, w, dev, args, T):
    """Coupled steps of the same problem with resident trees and chain links
    (the geometry is static): after one full solve, each step recomputes the
    optical depths from the current n_HI, sums them along the stored chains
    (one replayed CUDA graph) and applies the implicit update."""
    import torch
    stream = torch.cuda.current_stream(dev)
    ctx = S.Context(reuse_chains=1, march_group=args.march_group, row_bins=args.row_bins, stream=stream)
    ctx.build_trees(T(w.pos), T(w.h), T(w.src_pos), T(w.src_L))
    ctx.set_state(T(w.n_H), T(w.y0))
    g = torch.zeros(w.n_p, dtype=torch.float32, device=dev)
    y = torch.zeros(w.n_p, dtype=torch.float64, device=dev)
    ctx.rt_solve(args.theta, gamma_out=g)        # full solve: finds and keeps the links
    ctx.ionize(w.dt_s, y_out=y)
    for _ in range(args.warmup):
        ctx.rt_solve(args.theta, gamma_out=g)
        ctx.ionize(w.dt_s, y_out=y)
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    rays = 0
    e0.record(stream)
    for _ in range(args.steps):
        ctx.rt_solve(args.theta, gamma_out=g)
        ctx.ionize(w.dt_s, y_out=y)
        rays += ctx.stats()["rays"]
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1)
    ctx.close()
    return {"value": rays / (ms * 1e-3), "unit": "rays/s", "ms_per_step": ms / args.steps,
            "note": "links of the first full solve reused; per step: d_tau, chain sums, Gamma, "
                    "implicit update (no tree build, walk or neighbour search)"}


# algorithmic bytes of one particle's SPH density: its record, h and CSR
# offsets, then per neighbour its index, record and mass (33 neighbours in
# this recipe), the mass gather and the scattered result
DENSITY_BYTES_PER_NEIGHBOUR = 4 + 16 + 4
DENSITY_BYTES_PER_PARTICLE = 16 + 4 + 8 + 4 + 4 + 4 + 4


def sph_density(S, w, dev, args, T, flush):
    """SPH density (Section 2.1) of the benchmark particles from device masses,
    L2 flushed before every timed call."""
    import torch
    stream = torch.cuda.current_stream(dev)
    ctx = S.Context(stream=stream)
    ctx.build_trees(T(w.pos), T(w.h), T(w.src_pos), T(w.src_L))
    m = torch.ones(w.n_p, dtype=torch.float32, device=dev)
    rho = torch.zeros(w.n_p, dtype=torch.float32, device=dev)
    for _ in range(args.warmup):
        ctx.sph_density(m, rho)
    torch.cuda.synchronize(dev)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    for e0, e1 in evs:
        flush.zero_()
        e0.record(stream)
        ctx.sph_density(m, rho)
        e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = sum(a.elapsed_time(b) for a, b in evs) / args.steps
    nbr = ctx.stats()["nbr_total"]
    ctx.close()
    algo = DENSITY_BYTES_PER_PARTICLE * w.n_p + DENSITY_BYTES_PER_NEIGHBOUR * nbr
    return {"value": w.n_p / (ms * 1e-3), "unit": "particles/s", "ms_per_call": ms,
            "neighbours_per_particle": nbr / w.n_p,
            "algorithmic_GB_per_s": algo / (ms * 1e-3) / 1e9,
            "note": "two kernels (mass gather to Morton order, density); gathers L2-served"}


def h2_dissociation(S, w, dev, args, T, flush):
    """H2 photodissociation rates (Appendix B) of the benchmark particles: the
    same walk and memoised chains as the Gamma solve, carrying the H2 column
    (log-normal n_H2) and the self-shielding function; L2 flushed before every
    timed call."""
    import numpy as np
    import torch
    stream = torch.cuda.current_stream(dev)
    ctx = S.Context(stream=stream, march_group=args.march_group, row_bins=args.row_bins)
    ctx.build_trees(T(w.pos), T(w.h), T(w.src_pos), T(w.src_L))
    nH2 = T(np.random.default_rng(5).lognormal(np.log(1e-4), 1.5, w.n_p).astype(np.float32))
    k = torch.zeros(w.n_p, dtype=torch.float32, device=dev)
    for _ in range(args.warmup):
        ctx.h2_dissociation(nH2, args.theta, 1e-21, k)
    torch.cuda.synchronize(dev)
    ms, rays = 0.0, 0
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.h2_dissociation(nH2, args.theta, 1e-21, k)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms += e0.elapsed_time(e1)
        rays += ctx.stats()["rays"]
    ctx.close()
    return {"value": rays / (ms * 1e-3), "unit": "rays/s", "ms_per_call": ms / args.steps,
            "theta": args.theta, "note": "walk + memoised chains carrying N_H2 + self-shielded "
                                         "LW flux per pair (no tree build)"}


def method_error(S, w, dev, args, T):
    """The method's own error (Section 2.2.2): Gamma at theta = 0.5 and 1.0
    against theta = 0 (every source individually, the brute-force RSPH sum)
    on the benchmark particles, for the neutral start and optically thin
    (n_HI = 0); relative deviations over the particles whose brute-force Gamma
    exceeds the absolute floor 1e-8 / (sigma dt)."""
    import numpy as np
    import torch
    stream = torch.cuda.current_stream(dev)
    ctx = S.Context(stream=stream, march_group=args.march_group, row_bins=args.row_bins, reuse_chains=0)
    ctx.build_trees(T(w.pos), T(w.h), T(w.src_pos), T(w.src_L))
    floor = 1e-8 / (w.params["sigma_cm2"] * w.dt_s)
    out = {"floor": floor}
    for name, nhi in (("neutral", w.n_HI()), ("thin", np.zeros(w.n_p, np.float32))):
        n_t = T(nhi)
        g = {}
        for th in (0.0, 0.5, 1.0):
            gd = torch.zeros(w.n_p, dtype=torch.float32, device=dev)
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            ctx.rt_solve(th, n_HI=n_t, gamma_out=gd)
            torch.cuda.synchronize(dev)
            dt = time.perf_counter() - t0
            g[th] = gd.double().cpu().numpy()
            if th == 0.0 and name == "neutral":
                out["brute_force_rays_per_s"] = ctx.stats()["rays"] / dt
        ok = g[0.0] > floor
        res = {"particles": int(ok.sum())}
        for th in (0.5, 1.0):
            rel = np.abs(g[th][ok] / g[0.0][ok] - 1.0)
            res[f"theta_{th}"] = {"median": float(np.median(rel)),
                                  "p90": float(np.percentile(rel, 90)), "max": float(rel.max())}
        out[name] = res
    ctx.close()
    return out


def blackbody_sources(S, w, dev, args, T, flush):
    """The benchmark workload with blackbody point sources (T_eff = 1e5 K, as
    in Test 1): full solves from built trees, Gamma_eff and the photoheating
    rate per pair from the spectral tables; L2 flushed before every call."""
    import torch
    stream = torch.cuda.current_stream(dev)
    ctx = S.Context(stream=stream, march_group=args.march_group, row_bins=args.row_bins, T_eff=1e5)
    ctx.build_trees(T(w.pos), T(w.h), T(w.src_pos), T(w.src_L))
    ctx.set_state(T(w.n_H), T(w.y0))
    g = torch.zeros(w.n_p, dtype=torch.float32, device=dev)
    for _ in range(args.warmup):
        ctx.rt_solve(args.theta, gamma_out=g)
    torch.cuda.synchronize(dev)
    ms, rays = 0.0, 0
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.rt_solve(args.theta, gamma_out=g)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms += e0.elapsed_time(e1)
        rays += ctx.stats()["rays"]
    ctx.close()
    return {"value": rays / (ms * 1e-3), "unit": "rays/s", "ms_per_call": ms / args.steps,
            "theta": args.theta, "T_eff": 1e5,
            "note": "walk + memoised chains + spectral Gamma and heating per pair (no tree build)"}


def diffuse_workload(S, dev, args, T, T_rec=0.0):
    """The diffuse-recombination shadowing workload at full size: 128^3
    particles (all emitting), eight 200x clumps, one 3e51/s central source,
    theta = 0.7; coupled full-path steps (emitter moments, walk over both
    trees, memoised march in target chunks, Gamma, update with k_self).
    T_rec > 0: the recombination photons fill the band of width k T_rec / h
    (band tables per emitter pair, photoheating with its self term)."""
    import torch
    from start_inputs import config3
    w = config3()
    stream = torch.cuda.current_stream(dev)
    ctx = S.Context(timing=1, march_group=args.march_group, row_bins=args.row_bins, stream=stream, max_pairs=1 << 29,
                    T_rec=T_rec)
    y = T(w.y0)
    g = torch.zeros(w.n_p, dtype=torch.float32, device=dev)
    pos, h, sp, sL, V, nH = T(w.pos), T(w.h), T(w.src_pos), T(w.src_L), T(w.V), T(w.n_H)

    def step():
        ctx.build_trees(pos, h, sp, sL, V, diffuse=True)
        ctx.set_state(nH, y)
        ctx.rt_solve(0.7, gamma_out=g)
        ctx.ionize(w.dt_s, y_out=y)

    step()
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    steps, rays = 2, 0
    e0.record(stream)
    for _ in range(steps):
        step()
        rays += ctx.stats()["rays"]
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1)
    st = ctx.stats()
    ctx.close()
    return {"value": rays / (ms * 1e-3), "unit": "rays/s", "ms_per_step": ms / steps,
            "rays_per_step": rays / steps, "chunks": st["chunks"],
            "evaluations_per_ray": st["evals"] / max(1, st["rays"]), "workload": w.name,
            "theta": 0.7, "T_rec": T_rec}


def serving(args):
    """Continuous batching vs one solve at a time on the same Poisson stream
    of requests of mixed size (real-time replay, 150 GB budget), at an
    arrival rate above one GPU's capacity and at one below it; and a stream
    of small requests, where a solve is bound by launches and host round
    trips, served by more workers with the autotuned knobs of each problem
    class (tuned before the stream starts)."""
    from paper_1005_5312_gb300.autotune import SEARCH_SPACE, Tuner
    from paper_1005_5312_gb300.serve import Server, make_requests, summarize
    lo, hi = (float(x) for x in args.serve_log2np.split(","))
    slo, shi = (float(x) for x in args.serve_small_log2np.split(","))
    out = {"workers": args.serve_workers, "budget_gb": 150}
    small = make_requests(args.serve_small_requests, rate_hz=args.serve_small_rate,
                          log2_np=(slo, shi), seed=53125)
    tuner = Tuner()
    t0 = time.perf_counter()
    tuned = tuner.tune_requests(small, max_classes=24)
    tune_s = time.perf_counter() - t0
    for key, reqs, workers_served, tnr in (
            ("saturated", make_requests(args.serve_requests, rate_hz=args.serve_rate,
                                        log2_np=(lo, hi)), args.serve_workers, None),
            ("below_capacity", make_requests(args.serve_low_requests,
                                             rate_hz=args.serve_low_rate, log2_np=(lo, hi)),
             args.serve_workers, None),
            ("small_requests", small, args.serve_small_workers, tuner)):
        res = {}
        arms = [("plain", 1, 0), ("served", workers_served, 0)]
        if key == "small_requests":
            arms.append(("served_batched", workers_served, 16))
        for name, workers, bsz in arms:
            srv = Server(workers=workers, budget_bytes=150e9,
                         tuner=tnr if name != "plain" else None, batch_small=bsz,
                         small_n_p=1 << 16)
            # warm the workers' contexts and pools on a small request
            srv.serve(make_requests(workers, rate_hz=1e9, log2_np=(14, 14), seed=1),
                      realtime=False)
            r = srv.serve(reqs, realtime=True)
            srv.close()
            res[name] = summarize(r)
            res[name]["context_trims"] = srv.trims
            res[name]["oom_retries"] = srv.retries
            if bsz:
                res[name]["batches"] = srv.batches
        n_p = [r.n_p for r in reqs]
        rate = len(reqs) / max(r.t_arrive for r in reqs)
        a, b = (slo, shi) if key == "small_requests" else (lo, hi)
        out[key] = {"workload": f"{len(reqs)} requests, Poisson {rate:.3g}/s, "
                                f"N_p=2^U({a:g},{b:g}), N_s=e^U(0,ln N_p), uniform|clumpy, "
                                f"theta in {{0.5,1}}, 1 step each",
                    "mean_n_p": float(np.mean(n_p)), "workers": workers_served,
                    "served": res["served"], "plain": res["plain"],
                    "solves_per_s_vs_plain": res["served"]["solves_per_s"] /
                    res["plain"]["solves_per_s"]}
        if "served_batched" in res:
            out[key]["served_batched"] = res["served_batched"]
            out[key]["batched_solves_per_s_vs_plain"] = (res["served_batched"]["solves_per_s"] /
                                                         res["plain"]["solves_per_s"])
    out["small_requests"]["autotuner"] = {"classes_tuned": len(tuned), "tuning_s": tune_s,
                                          "knobs": ", ".join(sorted(SEARCH_SPACE)),
                                          "tuned_outside_the_stream": True}
    return out


def multisource_lines(S, dev, args, T, flush, w2, peak):
    """The 64^3 multiple-source workload (1024 point sources): coupled full
    steps at theta and theta2 with L2 flushed between timed steps, the
    resident-chain steps, the method's own error and the next-row lines."""
    import torch
    stream = torch.cuda.current_stream(dev)
    ctx = S.Context(timing=1, march_group=args.march_group, row_bins=args.row_bins, stream=stream)
    pos, h, spos, sL = T(w2.pos), T(w2.h), T(w2.src_pos), T(w2.src_L)
    nH, y0 = T(w2.n_H), T(w2.y0)
    y = y0.clone()
    g = torch.zeros(w2.n_p, dtype=torch.float32, device=dev)

    def step(theta):
        ctx.build_trees(pos, h, spos, sL)
        ctx.set_state(nH, y)
        ctx.rt_solve(theta, gamma_out=g)
        ctx.ionize(w2.dt_s, y_out=y)

    out = {"workload": w2.name, "n_p": w2.n_p, "n_s": w2.n_s,
           "l2": "512 MB buffer written between timed steps"}
    steps = max(3, args.steps)
    for theta in (args.theta, args.theta2):
        y.copy_(y0)
        for _ in range(3):
            step(theta)
        torch.cuda.synchronize(dev)
        ctx.timings()
        ms, rays, evals, phases = [], [], [], {}
        for _ in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step(theta)
            e1.record(stream)
            tm = ctx.timings()
            st = ctx.stats()
            ms.append(e0.elapsed_time(e1))
            rays.append(st["rays"])
            evals.append(st["evals"])
            for k, v in tm.items():
                if v is not None and v >= 0:
                    phases[k] = phases.get(k, 0.0) + v / steps
        t = sum(ms)
        algo = (ALGO_BYTES_PER_EVAL * sum(evals) + ALGO_BYTES_PER_RAY * sum(rays) +
                ALGO_BYTES_PER_TARGET * w2.n_p * steps) / steps
        out[f"theta_{theta}"] = {
            "value": sum(rays) / (t * 1e-3), "unit": "rays/s", "ms_per_step": t / steps,
            "rays_per_step": sum(rays) / steps, "evaluations_per_ray": sum(evals) / sum(rays),
            "phase_ms_per_step": phases,
            "roofline_step": {"algorithmic_bytes_per_step": algo,
                              "achieved_GB_per_s": algo / (t / steps * 1e-3) / 1e9,
                              "frac_of_measured_hbm": algo / (t / steps * 1e-3) / 1e9 / peak}}
    ctx.close()
    if not args.no_resident:
        out["resident_steps"] = resident_steps(S, w2, dev, args, T)
    if not args.no_method_error:
        out["method_error"] = method_error(S, w2, dev, args, T)
    if not args.no_next:
        out["sph_density"] = sph_density(S, w2, dev, args, T, flush)
        out["h2_dissociation"] = h2_dissociation(S, w2, dev, args, T, flush)
        out["blackbody_sources"] = blackbody_sources(S, w2, dev, args, T, flush)
    # Gamma at the neutral start, for the parity check against the oracle
    ctx = S.Context(march_group=args.march_group, row_bins=args.row_bins, stream=stream)
    ctx.build_trees(pos, h, spos, sL)
    g0 = torch.zeros(w2.n_p, dtype=torch.float32, device=dev)
    ctx.rt_solve(args.theta, n_HI=T(w2.n_HI()), gamma_out=g0)
    g_start = g0.cpu().numpy()
    ctx.close()
    return out, g_start


# ---------------------------------------------------------------- GPU arm
def run_gpu(args):
    import torch
    import paper_1005_5312_gb300 as S
    from start_inputs import config2, config5

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    S.build()
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    peak, peak_kind = measured_peaks()

    w = config5(nside=args.nside)
    r1, r2, clocks, g5_start = headline(S, w, dev, args, T, local)

    tot_ms, rays = reduce_over_ranks(sum(r1["step_ms"]), sum(s["rays"] for s in r1["stats"]))
    value = rays / (tot_ms * 1e-3)
    K = args.steps
    step_ms = tot_ms / K
    st_sum = {k: sum(s[k] for s in r1["stats"]) / K
              for k in ("rays", "evals", "hops", "jump_bytes", "march_fallbacks", "chunks")}
    last = r1["stats"][-1]
    for k in ("nbr_total", "nodes_part", "nodes_src", "nodes_emit"):
        st_sum[k] = last[k]
    phase_ms = {}
    for ph in r1["phases"]:
        for k, v in ph.items():
            if v is not None and v >= 0:
                phase_ms[k] = phase_ms.get(k, 0.0) + v / K
    # the march phase holds the walk's fill, hops, link and jump; report the
    # fill as part of the walk
    if "march" in phase_ms:
        rest = phase_ms["march"] - sum(phase_ms.get(k, 0.0) for k in ("hops", "link", "jump"))
        phase_ms["walk"] = phase_ms.get("walk", 0.0) + max(0.0, rest)
    models = phase_models(st_sum, w.n_p, w.n_s, True, max(1, round(st_sum["chunks"])))
    kernels = kernel_table(phase_ms, models, step_ms, peak)

    # whole-step roofline: the march's algorithmic traffic per step
    algo = (ALGO_BYTES_PER_EVAL * st_sum["evals"] + ALGO_BYTES_PER_RAY * st_sum["rays"] +
            ALGO_BYTES_PER_TARGET * w.n_p)
    achieved = algo / (step_ms * 1e-3) / 1e9
    tr = traffic_record("step_" + w.name)
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "peak_source": f"{peak_kind} (copy bandwidth)",
            "traffic": tr["dram_bytes_per_step"] if tr else None,
            "kernel": "whole step (every kernel of build, density, walk, march, Gamma, update)",
            "launch_ms": step_ms, "algorithmic_bytes_per_launch": algo,
            "model": "516 B per neighbour-list evaluation (32 u32 indices, 32 float3 positions, "
                     "one float n_HI) + 16 B per ray + 8 B per target",
            "evaluations_per_step": st_sum["evals"], "rays_per_step": st_sum["rays"]}

    out = {"metric": f"RT rays/s at theta_crit={args.theta}", "value": value, "unit": "rays/s",
           "n_gpus": ws, "steps": K, "warmup": args.warmup, "ms_per_step": step_ms,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
           "data": "synthetic",
           "config": {"workload": w.name, "n_p": w.n_p, "n_s": w.n_s, "emitters": w.n_p,
                      "theta": args.theta, "dt_s": w.dt_s, "march_group": args.march_group,
                      "max_pairs": args.max_pairs, "row_bins": args.row_bins, "march": "memoised",
                      "l2": "no flush: every step streams inputs and buffers far larger than "
                            "L2 (particles 16.7M x 60 B, neighbour lists 2.1 GB, chain slots "
                            "tens of GB)",
                      "step": "build_trees + sph_density + set_state + rt_solve + ionize, "
                              "coupled"},
           "gpu_launches": r1["launches"],
           "rays_per_step": st_sum["rays"] / 1.0,
           "evaluations_per_ray": st_sum["evals"] / max(1.0, st_sum["rays"]),
           "chain_links_per_ray": (st_sum["hops"] / max(1.0, st_sum["rays"])
                                   if st_sum["hops"] >= 0 else None),
           "chunks_per_step": st_sum["chunks"],
           "march_fallbacks_per_step": st_sum["march_fallbacks"],
           "roofline": roof, "kernels": kernels, "clocks": clocks}
    if r2 is not None:
        t2 = sum(r2["step_ms"])
        out[f"theta_{args.theta2}"] = {
            "value": sum(s["rays"] for s in r2["stats"]) / (t2 * 1e-3), "unit": "rays/s",
            "ms_per_step": t2 / len(r2["step_ms"]), "steps": len(r2["step_ms"]),
            "rays_per_step": sum(s["rays"] for s in r2["stats"]) / len(r2["step_ms"])}
    if not args.no_e2e:
        out["e2e"] = headline_e2e(S, w, args)

    parity = {}
    g2_start = None
    if not args.no_extras:
        w2 = config2()
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
        out["multisource_64cubed"], g2_start = multisource_lines(S, dev, args, T, flush, w2, peak)
        if not args.no_diffuse:
            out["diffuse_128cubed"] = diffuse_workload(S, dev, args, T)
            if not args.no_next:
                out["diffuse_128cubed_recombination_band"] = diffuse_workload(S, dev, args, T,
                                                                               T_rec=1e4)
        if ws == 1 and not args.no_serve:
            out["serving"] = serving(args)

    if rank == 0 and ws == 1 and not args.no_cpu:
        g_abs = 1e-8 / (w.params["sigma_cm2"] * w.dt_s)
        idx, ref, orays, osec, cores = oracle_sample(w, args.theta, args.cpu_seconds)
        out["cpu_baseline"] = {
            "value": orays / osec, "unit": "rays/s", "cores": cores, "kind": "oracle",
            "sample": f"Gamma at {len(idx)} random targets of {w.n_p} (theta={args.theta}, "
                      f"starting state, all emitters and point sources): {orays} rays in "
                      f"{osec:.1f} s"}
        parity[f"{w.name}_theta{args.theta}"] = rel_errors(g5_start[idx], ref, g_abs)
        if g2_start is not None:
            idx2, ref2, _, _, _ = oracle_sample(w2, args.theta, 10.0)
            parity[f"{w2.name}_theta{args.theta}"] = rel_errors(g2_start[idx2], ref2, g_abs)
        out["parity"] = parity
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return out if rank == 0 else None


def main():
    args = parse()
    res = run_reference(args) if args.impl == "reference" else run_gpu(args)
    if res is not None:
        print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
