#!/usr/bin/env python3
"""Benchmark of the START hot path on one GB300 (or N replicas under torchrun).

A step is one pass of the whole path over the multiple-source workload
(64^3 = 262144 particles on a jittered lattice, 1024 sources with
log-normal luminosity, uniform n_H = 1e-3 in a 6.6 kpc box): frame, Morton
keys, sorts, source and particle octrees, moments, neighbour lists, walk,
ray march, Gamma and the implicit 1 Myr ionisation update, coupled from step
to step.  The metric is rays per second (a ray is one (target, virtual
source) pair whose optical depth is evaluated); theta_crit = 0.5 is the
headline and 1.0 is reported beside it.

Prints one JSON line.  --impl reference times the FP64 oracle on the host
cores on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json

import numpy as np
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

ALGO_BYTES_PER_HOP = 516     # 32 u32 neighbour indices + 32 float3 positions + 1 float n_HI
ALGO_BYTES_PER_RAY = 16      # virtual source record
ALGO_BYTES_PER_TARGET = 8    # Gamma out, target record
# memoised march, per evaluated chain link: the neighbour list (516 B) plus
# the link's source record (16 B), its hash-table entry (16 B) and its slot
# state (virtual source, particle, next, tau, links: 16 B)
L2_FLUSH_BYTES = 512 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--theta", type=float, default=0.5)
    ap.add_argument("--theta2", type=float, default=1.0)
    ap.add_argument("--march-group", type=int, default=2)
    ap.add_argument("--march-mode", type=int, default=1, choices=[0, 1],
                    help="1 memoised march (default), 0 per-ray march")
    ap.add_argument("--nside", type=int, default=64,
                    help="lattice side of the multiple-source workload (64: the benchmark; "
                         "smaller: profiling cases)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-theta2", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=10.0,
                    help="oracle work per CPU-baseline measurement")
    ap.add_argument("--ref-targets", type=int, default=16384,
                    help="targets per step of the reference arm")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-resident", action="store_true")
    ap.add_argument("--no-diffuse", action="store_true")
    ap.add_argument("--no-next", action="store_true",
                    help="skip the SPH density, H2 photodissociation, blackbody-source and "
                         "recombination-band lines")
    ap.add_argument("--no-method-error", action="store_true")
    ap.add_argument("--lognormal256", action="store_true",
                    help="add the 256^3 log-normal diffuse workload (about a minute)")
    ap.add_argument("--serve-requests", type=int, default=256)
    ap.add_argument("--serve-rate", type=float, default=50.0)
    ap.add_argument("--serve-workers", type=int, default=4)
    ap.add_argument("--serve-log2np", default="15,21")
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


def kernel_source_sha(source: str, kernel: str) -> str:
    """sha256 (16 hex digits) of a kernel's definition text (from its
    `__global__` line to the matching closing brace) together with the
    file's constexpr definitions (tile shapes, template arguments)."""
    import hashlib
    import re
    text = open(os.path.join(ROOT, "paper_1005_5312_gb300", "csrc", source)).read()
    m = re.search(r"__global__[^;{]*?\b" + re.escape(kernel) + r"\s*\(", text)
    if not m:
        return ""
    consts = "\n".join(re.findall(r"^constexpr [^\n]*;", text, flags=re.M))
    i = text.index("{", m.end())
    depth = 0
    for j in range(i, len(text)):
        depth += {"{": 1, "}": -1}.get(text[j], 0)
        if depth == 0:
            return hashlib.sha256((consts + "\n" + text[m.start():j + 1]).encode()).hexdigest()[:16]
    return ""


def traffic_record(kernel: str):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on
    the kernel's current definition (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f).get(kernel)
    if not d:
        return None
    return d if d.get("kernel_sha") == kernel_source_sha(d["source"], kernel) else None


# ---------------------------------------------------------------- reference arm
def run_reference(args, w):
    import numpy as np
    import oracle
    ws, rank, _ = dist_env()
    if rank != 0:
        return None
    oracle.build()
    orc = oracle.Oracle.from_workload(w, ptree_leaf=16)
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
            "config": {"workload": w.name, "n_p": w.n_p, "n_s": w.n_s, "theta": args.theta,
                       "sample": f"{per_step} random targets per step"},
            "cpu_baseline": {"value": v, "unit": "rays/s", "cores": cores, "kind": "oracle",
                             "sample": f"{per_step} random targets of {w.n_p} per step"},
            "e2e": {"value": v, "unit": "rays/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def cpu_baseline(w, theta, seconds):
    """The oracle as it stands on the host cores: Gamma at random targets of
    the same workload (neutral start), in chunks until `seconds` of work."""
    import numpy as np
    import oracle
    oracle.build()
    orc = oracle.Oracle.from_workload(w, ptree_leaf=16)
    order = np.random.default_rng(5).permutation(w.n_p)
    nHI = w.n_HI()
    done, rays, t = 0, 0, 0.0
    chunk = 1024
    while t < seconds and done < w.n_p:
        idx = order[done:done + chunk]
        t0 = time.perf_counter()
        orc.gamma(nHI, theta, targets=idx)
        t += time.perf_counter() - t0
        rays += orc.last_stats["rays"]
        done += len(idx)
    return {"value": rays / t, "unit": "rays/s", "cores": oracle.threads(), "kind": "oracle",
            "sample": f"Gamma at {done} random targets of {w.n_p} (theta={theta}, neutral "
                      f"start): {rays} rays in {t:.1f} s"}


def resident_steps(S, w, dev, args, T):
    """Coupled steps of the same problem with resident trees and chain links
    (the geometry is static): after one full solve, each step recomputes the
    optical depths from the current n_HI, sums them along the stored chains
    (one replayed CUDA graph) and applies the implicit update."""
    import torch
    stream = torch.cuda.current_stream(dev)
    ctx = S.Context(reuse_chains=1, march_group=args.march_group, stream=stream)
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
    ctx = S.Context(stream=stream, march_group=args.march_group)
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
    ctx = S.Context(stream=stream, march_group=args.march_group, reuse_chains=0)
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
    ctx = S.Context(stream=stream, march_group=args.march_group, T_eff=1e5)
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
    ctx = S.Context(timing=1, march_group=args.march_group, stream=stream, max_pairs=1 << 29,
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


def lognormal_256(S, dev, args, T):
    """The large diffuse run at full size (opt-in): 256^3 particles in a
    log-normal field (sigma_ln = 1.5, P(k) ~ k^-3), every particle emitting
    plus 64 sources of 1e50/s; per theta in {0.5, 1}: SPH density recompute
    from masses, then a full coupled step (build, walk over both trees,
    memoised march in target chunks, Gamma, implicit update)."""
    import numpy as np
    import torch
    from start_inputs import config5
    w = config5()
    stream = torch.cuda.current_stream(dev)
    ctx = S.Context(timing=1, march_group=args.march_group, stream=stream, max_pairs=1 << 29)
    pos, h, sp, sL, V = T(w.pos), T(w.h), T(w.src_pos), T(w.src_L), T(w.V)
    mass = T((w.n_H.astype(np.float64) * w.V).astype(np.float32))
    rho = torch.zeros(w.n_p, dtype=torch.float32, device=dev)
    y = T(w.y0)
    g = torch.zeros(w.n_p, dtype=torch.float32, device=dev)
    out = {"workload": w.name, "n_p": w.n_p}
    for theta in (0.5, 1.0):
        y.copy_(T(w.y0))
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.build_trees(pos, h, sp, sL, V, diffuse=True)
        ctx.sph_density(mass, rho)
        ctx.set_state(rho, y)
        ctx.rt_solve(theta, gamma_out=g)
        ctx.ionize(w.dt_s, y_out=y)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1)
        st = ctx.stats()
        out[f"theta_{theta}"] = {"value": st["rays"] / (ms * 1e-3), "unit": "rays/s",
                                 "ms_per_step": ms, "rays_per_step": st["rays"],
                                 "chunks": st["chunks"]}
    ctx.close()
    return out


def serving(args):
    """Continuous batching vs one solve at a time on the same Poisson stream
    of requests of mixed size (real-time replay, 150 GB budget)."""
    from paper_1005_5312_gb300.serve import Server, make_requests, summarize
    lo, hi = (float(x) for x in args.serve_log2np.split(","))
    reqs = make_requests(args.serve_requests, rate_hz=args.serve_rate, log2_np=(lo, hi))
    res = {}
    for name, workers in (("plain", 1), ("served", args.serve_workers)):
        srv = Server(workers=workers, budget_bytes=150e9)
        # warm the workers' contexts and pools on a small request
        srv.serve(make_requests(workers, rate_hz=1e9, log2_np=(14, 14), seed=1), realtime=False)
        r = srv.serve(reqs, realtime=True)
        srv.close()
        res[name] = summarize(r)
        res[name]["context_trims"] = srv.trims
        res[name]["oom_retries"] = srv.retries
    sp = res["served"]["solves_per_s"] / res["plain"]["solves_per_s"]
    n_p = [r.n_p for r in reqs]
    return {"workload": f"{len(reqs)} requests, Poisson {args.serve_rate:g}/s, N_p=2^U({lo:g},{hi:g}),"
                        " N_s=e^U(0,ln N_p), uniform|clumpy, theta in {0.5,1}, 1 step each",
            "workers": args.serve_workers, "budget_gb": 150, "mean_n_p": float(np.mean(n_p)),
            "served": res["served"], "plain": res["plain"],
            "solves_per_s_vs_plain": sp}


# ---------------------------------------------------------------- GPU arm
def run_gpu(args, w):
    import numpy as np
    import torch
    import paper_1005_5312_gb300 as S

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    S.build()
    stream = torch.cuda.current_stream(dev)
    ctx = S.Context(timing=1, march_group=args.march_group, march_mode=args.march_mode,
                    stream=stream)
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    pos, h, spos, sL = T(w.pos), T(w.h), T(w.src_pos), T(w.src_L)
    nH, y0 = T(w.n_H), T(w.y0)
    y = y0.clone()
    g = torch.zeros(w.n_p, dtype=torch.float32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def step(theta):
        ctx.build_trees(pos, h, spos, sL)
        ctx.set_state(nH, y)
        ctx.rt_solve(theta, gamma_out=g)
        ctx.ionize(w.dt_s, y_out=y)

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize(dev)

    def timed(theta, steps, warmup):
        y.copy_(y0)
        for _ in range(warmup):
            step(theta)
        torch.cuda.synchronize(dev)
        ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        march_ms, hop_ms, rays, hops, evals, fbs = [], [], [], [], [], []
        link_ms, jump_ms, jump_bytes, jump_rounds = [], [], [], []
        l0 = ctx.stats()["launches"]
        barrier()
        t_wall = time.perf_counter()
        for k in range(steps):
            flush.zero_()                      # evict L2 between timed steps
            ev0[k].record(stream)
            step(theta)
            ev1[k].record(stream)
            tm = ctx.timings()
            st = ctx.stats()
            march_ms.append(tm["march"])
            hop_ms.append(tm["hops"])
            link_ms.append(tm["link"])
            jump_ms.append(tm["jump"])
            jump_bytes.append(st["jump_bytes"])
            jump_rounds.append(st["jump_rounds"])
            rays.append(st["rays"])
            hops.append(st["hops"])
            evals.append(st["evals"])
            fbs.append(st["march_fallbacks"])
        barrier()
        t_wall = time.perf_counter() - t_wall
        launches = ctx.stats()["launches"] - l0
        step_ms = [a.elapsed_time(b) for a, b in zip(ev0, ev1)]
        return dict(step_ms=step_ms, march_ms=march_ms, hop_ms=hop_ms, rays=rays, hops=hops,
                    evals=evals, fbs=fbs, launches=launches, wall=t_wall, link_ms=link_ms,
                    jump_ms=jump_ms, jump_bytes=jump_bytes, jump_rounds=jump_rounds)

    with ClockSampler(local) as clk:
        r1 = timed(args.theta, args.steps, args.warmup)
    r2 = None if args.no_theta2 else timed(args.theta2, max(2, args.steps // 2), 1)

    tot_ms, rays = reduce_over_ranks(sum(r1["step_ms"]), sum(r1["rays"]))
    value = rays / (tot_ms * 1e-3)

    # roofline of the dominant kernel
    peak, peak_kind = measured_peaks()
    if args.march_mode == 1:
        # memoised march: the pointer-jumping rounds (its largest share of a
        # step); bytes and durations summed over the timed steps' rounds
        kern = "k_memo_jump"
        n_launch = sum(r1["jump_rounds"])
        per_launch = sum(r1["jump_bytes"]) / n_launch
        avg_ms = sum(r1["jump_ms"]) / n_launch
    else:
        kern = "k_march"
        algo_l = [ALGO_BYTES_PER_HOP * hp + ALGO_BYTES_PER_RAY * r + ALGO_BYTES_PER_TARGET * w.n_p
                  for r, hp in zip(r1["rays"], r1["evals"])]
        per_launch = sum(algo_l) / len(algo_l)
        avg_ms = sum(r1["march_ms"]) / len(r1["march_ms"])
    achieved = per_launch / (avg_ms * 1e-3) / 1e9
    tr = traffic_record(kern)
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "peak_source": peak_kind,
            "traffic": tr["dram_bytes_per_launch"] if tr else None,
            "kernel": kern, "launch_ms": avg_ms, "algorithmic_bytes_per_launch": per_launch}
    if args.march_mode == 1:
        roof["launches_per_step"] = sum(r1["jump_rounds"]) / args.steps

    out = {"metric": f"RT rays/s at theta_crit={args.theta}", "value": value, "unit": "rays/s",
           "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": tot_ms / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": w.name, "n_p": w.n_p, "n_s": w.n_s, "theta": args.theta,
                      "dt_s": w.dt_s, "march_group": args.march_group,
                      "march": "memoised" if args.march_mode == 1 else "per-ray",
                      "l2": "512 MB buffer written between timed steps",
                      "step": "build_trees + set_state + rt_solve + ionize, coupled"},
           "rays_per_step": rays / args.steps / ws,
           "chain_links_per_ray": sum(r1["hops"]) / max(1, sum(r1["rays"])),
           "evaluations_per_ray": sum(r1["evals"]) / max(1, sum(r1["rays"])),
           "march_ms_per_step": sum(r1["march_ms"]) / len(r1["march_ms"]),
           "march_fallbacks_per_step": sum(r1["fbs"]) / args.steps,
           "memo_kernels_ms_per_step": ({
               "hops": sum(r1["hop_ms"]) / args.steps, "link": sum(r1["link_ms"]) / args.steps,
               "jump": sum(r1["jump_ms"]) / args.steps} if args.march_mode == 1 else None),
           "gpu_launches": r1["launches"],
           "roofline": roof, "clocks": clk.summary()}
    if r2 is not None:
        t2 = sum(r2["step_ms"])
        out[f"theta_{args.theta2}"] = {"value": sum(r2["rays"]) / (t2 * 1e-3), "unit": "rays/s",
                                       "ms_per_step": t2 / len(r2["step_ms"]),
                                       "rays_per_step": sum(r2["rays"]) / len(r2["rays"]),
                                       "march_ms": sum(r2["march_ms"]) / len(r2["march_ms"])}
    phases = ctx.timings()
    out["phase_ms_last_step"] = phases

    if not args.no_resident:
        out["resident_steps"] = resident_steps(S, w, dev, args, T)
    if not args.no_method_error:
        out["method_error"] = method_error(S, w, dev, args, T)
    if not args.no_next:
        out["sph_density"] = sph_density(S, w, dev, args, T, flush)
        out["h2_dissociation"] = h2_dissociation(S, w, dev, args, T, flush)
        out["blackbody_sources"] = blackbody_sources(S, w, dev, args, T, flush)
    if not args.no_diffuse:
        out["diffuse_128cubed"] = diffuse_workload(S, dev, args, T)
        if not args.no_next:
            out["diffuse_128cubed_recombination_band"] = diffuse_workload(S, dev, args, T,
                                                                           T_rec=1e4)
    if args.lognormal256:
        out["lognormal_256cubed"] = lognormal_256(S, dev, args, T)

    if not args.no_e2e:
        # end to end through the C ABI with host buffers: H2D copies of the
        # step's inputs and D2H of Gamma and y inside the timed region
        hpos, hh, hsp, hsL = w.pos, w.h, w.src_pos, w.src_L
        hnH = w.n_H
        hy = w.y0.copy()
        hg = np.zeros(w.n_p, np.float32)
        ctx_h = S.Context(march_group=args.march_group, march_mode=args.march_mode)

        def hstep():
            ctx_h.build_trees(hpos, hh, hsp, hsL)
            ctx_h.set_state(hnH, hy)
            ctx_h.rt_solve(args.theta, gamma_out=hg)
            ctx_h.ionize(w.dt_s, y_out=hy)

        for _ in range(args.warmup):
            hstep()
        hy[:] = w.y0
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        e_rays = 0
        for _ in range(args.steps):
            hstep()
            e_rays += ctx_h.stats()["rays"]
        te, e_rays = reduce_over_ranks(time.perf_counter() - t0, e_rays)
        h2d = hpos.nbytes + hh.nbytes + hsp.nbytes + hsL.nbytes + hnH.nbytes + hy.nbytes
        d2h = hg.nbytes + hy.nbytes
        out["e2e"] = {"value": e_rays / te, "unit": "rays/s", "h2d_bytes_per_step": h2d,
                      "d2h_bytes_per_step": d2h, "ms_per_step": 1e3 * te / args.steps}
        ctx_h.close()

    if ws == 1 and not args.no_serve:
        out["serving"] = serving(args)

    if rank == 0 and ws == 1 and not args.no_cpu:
        out["cpu_baseline"] = cpu_baseline(w, args.theta, args.cpu_seconds)
    ctx.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return out if rank == 0 else None


def main():
    args = parse()
    from start_inputs import config2
    w = config2(nside=args.nside)
    res = run_reference(args, w) if args.impl == "reference" else run_gpu(args, w)
    if res is not None:
        print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
