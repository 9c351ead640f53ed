#!/usr/bin/env python
"""Benchmark of the adaptive MG-CG solver on one GB300 (or N replicas).

Workload (default "L128_b6_massweep"): 128 x 128 quenched U(1) lattice at
beta = 6 (seeded Metropolis, 200 sweeps), three levels (4x4 then 2x2 blocks,
Nv = 8 per chirality, 8 setup relaxation sweeps), one Gaussian source chi,
b = D^dagger chi, tol 1e-10.  One step = the setup at the near-critical mass
(lambda_min(A) < 1e-5) followed by the mass sweep {m_nc, -0.05, 0.0, 0.1},
reusing the setup's vectors: for each mass, rebuild the Galerkin hierarchy
and coarsest inverse (except for m_nc), form b = D^dagger chi, and solve to
true FP64 relative residual 1e-10 -- 4 solves per step.

Arms:
  (default)          the CUDA library, mixed-precision MG-CG (value), plus the
                     same step with plain FP64 MG-CG, an end-to-end leg with
                     host buffers, roofline of the dominant kernel family and
                     the CPU oracle timed on a bounded sample.
  --impl reference   the CPU oracle on the same workload (bounded sample per
                     step, scaled to whole solves with the oracle's own
                     iteration counts).
Multi-GPU: replicas only (each rank solves the same workload independently);
value sums the solves of all ranks over the max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

METRIC = "MG-CG solves/s & p50/p99 latency at rel.res 1e-10 vs plain FP64; stencil GB/s"
UNIT = "solves/s"


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return {"hbm_gbs": d["hbm_gbs"], "bf16_tflops": d["bf16_tflops"],
                "bf16_tflops_sustained": d.get("bf16_tflops_sustained", d["bf16_tflops"]),
                "src": "measured", "sm_max_mhz": d.get("sm_max_mhz", 2070.0)}
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "src": "fallback", "sm_max_mhz": 2070.0}


def max_over_ranks(x, device=None):
    """The largest value of x over the ranks of the job (the slowest rank's
    time); x itself when no process group is running."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, world, slowest_seconds):
    """Whole-job throughput of independent replicas: the units all ranks
    processed over the slowest rank's time."""
    return units_per_rank * world / slowest_seconds


def workload_inputs(name):
    wl = W.BENCH_WORKLOADS[name]
    crit = json.load(open(os.path.join(ROOT, "workloads", "critical_masses.json")))[wl["critical_key"]]
    theta = W.quenched_u1_angles(wl["Lx"], wl["Lt"], wl["beta"], wl["sweeps"], wl["seed"])
    plaq = W.mean_plaquette(theta)
    if abs(plaq - crit["plaquette"]) > 1e-12:
        raise RuntimeError(f"regenerated gauge field differs from the stored one (plaquette {plaq})")
    U = W.links_from_angles(theta)
    noise = W.setup_noise(wl["Lx"], wl["Lt"], wl["blocks"], wl["Nv"], wl["noise_seed"])
    chi = W.gaussian_field((wl["Lt"], wl["Lx"], 2), wl["chi_seed"])
    masses = [crit["m_nc"]] + list(wl["heavy_masses"])
    return wl, crit, U, noise, chi, masses


# ---------------------------------------------------------------------------
# serving workload: Poisson arrivals over 8 configurations
# ---------------------------------------------------------------------------
# (key, L, beta, sweeps, seed, blocks, Nv, plan): 64^2 beta 3, 128^2 beta 6,
# 256^2 and 512^2 beta 10, two seeds each.  Hierarchies end at a 16 x 16 x 16
# coarsest level (4096 unknowns): three levels at 64^2 and 128^2, four at
# 256^2, five at 512^2.  On 256^2 and 512^2 the set-up (at the near-critical
# mass) adds two adaptive passes (Sec. 3), on levels 1 and 2, 30 V-cycles each.
SERVING_CONFIGS = [
    ("L64_b3_s1", 64, 3.0, 200, 1, [(4, 4), (2, 2)], [8, 8], ()),
    ("L64_b3_s2", 64, 3.0, 200, 2, [(4, 4), (2, 2)], [8, 8], ()),
    ("L128_b6_s1", 128, 6.0, 200, 1, [(4, 4), (2, 2)], [8, 8], ()),
    ("L128_b6_s2", 128, 6.0, 200, 2, [(4, 4), (2, 2)], [8, 8], ()),
    ("L256_b10_s1", 256, 10.0, 500, 1, [(4, 4), (2, 2), (2, 2)], [8, 8, 8], (1, 2)),
    ("L256_b10_s2", 256, 10.0, 500, 2, [(4, 4), (2, 2), (2, 2)], [8, 8, 8], (1, 2)),
    ("L512_b10_s1", 512, 10.0, 500, 1, [(4, 4), (2, 2), (2, 2), (2, 2)], [8, 8, 8, 8], (1, 2)),
    ("L512_b10_s2", 512, 10.0, 500, 2, [(4, 4), (2, 2), (2, 2), (2, 2)], [8, 8, 8, 8], (1, 2)),
]
SERVE_CYCLES = 30


# Mixed-precision solver of every leg: "reliable" = MG_SOLVER_MGCG_RELIABLE
# (FP32 Krylov iteration, FP64 reliable updates), "mixed" = MG_SOLVER_MGCG_MIXED
# (FP64 Krylov recursion); both use the FP32 V-cycle with BF16 coarse blocks.
SOLVER_CODES = {"mixed": 1, "reliable": 3}
MIXED_SOLVER = SOLVER_CODES["mixed"]


def _gauge_angles(args):
    L, beta, sweeps, seed = args
    return W.quenched_u1_angles(L, L, beta, sweeps, seed)


def critical_table():
    out = {}
    for f in ("critical_masses.json", "critical_masses_serving.json"):
        p = os.path.join(ROOT, "workloads", f)
        if os.path.exists(p):
            out.update(json.load(open(p)))
    return out


def _pct(v, q):
    v = sorted(v)
    return v[min(len(v) - 1, max(0, int(math.ceil(q * len(v))) - 1))]


def serving_leg(args, mg, torch, dev):
    """Serving stream over the 8 configurations through the serving engine
    (continuous batching per configuration and mass, 4 workers, max 16
    right-hand sides per batch).  A request draws its configuration uniformly,
    its mass uniformly from {0.05, 0.0, m_nc} and 1-16 Gaussian right-hand
    sides; tol 1e-10, mixed solver.  After a warm-up that builds every
    (configuration, mass) hierarchy:
    * one at a time, one right-hand side per (configuration, mass) group with
      the mixed solver and with plain FP64 MG-CG: the single-RHS service
      times, from which the single-RHS throughput of each solver on the same
      request mix follows (right-hand sides / sum of their service times);
    * the saturation point: all requests of the stream submitted at once; its
      right-hand sides per second is the capacity;
    * Poisson points at each fraction of that capacity in --serve-loads.
    Each point reports right-hand sides per second, submit-to-completion
    latency p50/p99 and the same split by (configuration, mass) group."""
    import multiprocessing as mp
    crit = critical_table()
    with mp.get_context("spawn").Pool(min(8, os.cpu_count() or 1)) as pool:
        thetas = pool.map(_gauge_angles, [(c[1], c[2], c[3], c[4]) for c in SERVING_CONFIGS])
    gen = torch.Generator(device=dev).manual_seed(2024)
    masses, missing, labels = [], [], []
    t_build = time.perf_counter()
    with mg.Server(budget_bytes=args.serve_budget_gb << 30, max_rhs=16, workers=4) as srv:
        ids = []
        for (key, L, beta, sw, seed, blocks, Nv, plan), th in zip(SERVING_CONFIGS, thetas):
            ms, lab = [0.05, 0.0], ["0.05", "0.0"]
            if key in crit and abs(W.mean_plaquette(th) - crit[key]["plaquette"]) <= 1e-12:
                ms.append(crit[key]["m_nc"])
                lab.append("m_nc")
            else:
                missing.append(key)
            masses.append(ms)
            labels.append(lab)
            U = torch.from_numpy(W.links_from_angles(th)).to(dev)
            noise = torch.from_numpy(W.setup_noise(L, L, blocks, Nv, 7,
                                                   refine_levels=[p - 1 for p in plan])).to(dev)
            kw = dict(setup_sweeps=8)
            if plan:
                kw.update(refine_levels=list(plan), refine_cycles=SERVE_CYCLES)
            ids.append(srv.add_config(U, mg.make_params(L, L, blocks, Nv, **kw), min(ms), noise=noise))

        def rhs(c, n):
            L = SERVING_CONFIGS[c][1]
            return torch.randn((n, L, L, 2), dtype=torch.complex128, device=dev, generator=gen)

        def one_at_a_time(solver):
            out = {}
            for c in range(len(SERVING_CONFIGS)):
                for m, lab in zip(masses[c], labels[c]):
                    b = rhs(c, 1)
                    x = torch.empty_like(b)
                    torch.cuda.synchronize()
                    st, infos, ms = srv.wait(srv.submit(ids[c], m, b, x, 1, 1e-10, solver), 1)
                    if st != 0:
                        raise RuntimeError(f"serving warm-up solve failed ({st})")
                    out[(c, lab)] = ms / 1000.0
            return out
        one_at_a_time(MIXED_SOLVER)          # builds every hierarchy
        build_s = time.perf_counter() - t_build
        single_mixed = one_at_a_time(MIXED_SOLVER)
        single_fp64 = one_at_a_time(mg.SOLVER_MGCG_FP64)

        def stream(seed, n_req):
            rng = np.random.default_rng(seed)
            reqs = []
            for _ in range(n_req):
                c = int(rng.integers(len(SERVING_CONFIGS)))
                k = int(rng.integers(len(masses[c])))
                reqs.append((c, k, int(rng.integers(1, 17))))
            return rng, reqs

        def run_point(seed, rate):
            rng, reqs = stream(seed, args.serve_requests)
            gaps = rng.exponential(1.0 / rate, size=len(reqs)) if rate else np.zeros(len(reqs))
            bufs = [rhs(c, n) for c, _, n in reqs]
            bufs = [(b, torch.empty_like(b)) for b in bufs]
            s0 = srv.stats()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            submit_t, rids = [], []
            for (c, k, n), (b, x), gap in zip(reqs, bufs, gaps):
                t0 += gap
                delay = t0 - time.perf_counter()
                if delay > 0:
                    time.sleep(delay)
                submit_t.append(time.perf_counter())
                rids.append(srv.submit(ids[c], masses[c][k], b, x, n, 1e-10, MIXED_SOLVER))
            lat, worst, failed = [], 0.0, 0
            for r, (c, k, n) in zip(rids, reqs):
                st, infos, ms = srv.wait(r, n)
                failed += st != 0
                lat.append(ms)
                worst = max([worst] + [i.true_residual for i in infos])
            wall = max(t + l / 1000.0 for t, l in zip(submit_t, lat)) - submit_t[0]
            s1 = srv.stats()
            total_rhs = sum(n for _, _, n in reqs)
            groups = {}
            for (c, k, n), l in zip(reqs, lat):
                groups.setdefault(f"{SERVING_CONFIGS[c][0]}@{labels[c][k]}", []).append((l, n))
            by_group = {g: {"requests": len(v), "rhs": sum(n for _, n in v),
                            "p50_ms": round(_pct([l for l, _ in v], 0.5), 1),
                            "p99_ms": round(_pct([l for l, _ in v], 0.99), 1)}
                        for g, v in sorted(groups.items())}
            p99 = _pct(lat, 0.99)
            tail = [g for g, v in by_group.items() if v["p99_ms"] >= 0.5 * p99]
            nb = s1.batches - s0.batches
            return {"requests": len(reqs), "rhs": total_rhs,
                    "arrival_rate_per_s": round(rate, 4) if rate else None,
                    "value": round(total_rhs / wall, 3), "wall_s": round(wall, 2),
                    "p50_ms": round(_pct(lat, 0.5), 1), "p99_ms": round(p99, 1),
                    "failed": failed, "max_true_residual": worst,
                    "mean_batch_rhs": round((s1.batched_rhs - s0.batched_rhs) / max(nb, 1), 2),
                    "groups_with_p99_above_half_of_overall": tail, "by_group": by_group}

        # saturation, then Poisson points at fractions of the measured capacity
        sat = run_point(2024, None)
        mean_rhs = sat["rhs"] / sat["requests"]
        points = [dict(sat, offered_load="all at once")]
        for j, load in enumerate(float(v) for v in args.serve_loads.split(",") if v):
            p = run_point(2025 + j, load * sat["value"] / mean_rhs)
            points.append(dict(p, offered_load=load))
        stats = srv.stats()

    # single-RHS throughput of each solver over the saturation stream's mix
    _, reqs = stream(2024, args.serve_requests)
    tot = sum(n for _, _, n in reqs)
    one = lambda t: round(tot / sum(n * t[(c, labels[c][k])] for c, k, n in reqs), 3)   # noqa: E731
    fp64_rate, mixed_rate = one(single_fp64), one(single_mixed)
    return {"configs": [c[0] for c in SERVING_CONFIGS],
            "hierarchies": {c[0]: {"levels": len(c[5]) + 1, "blocks": c[5], "Nv": c[6],
                                   "adaptive_passes": list(c[7]), "cycles": SERVE_CYCLES if c[7] else 0}
                            for c in SERVING_CONFIGS},
            "unit": "solves/s (right-hand sides)",
            "value": sat["value"], "p50_ms": sat["p50_ms"], "p99_ms": sat["p99_ms"],
            "capacity_rhs_per_s": sat["value"], "points": points,
            "single_rhs_one_at_a_time": {
                "plain_fp64_mgcg": fp64_rate, "mixed_mgcg": mixed_rate,
                "note": "per-(configuration, mass) single-RHS service times on the same resident "
                        "hierarchies, weighted by the saturation stream's right-hand-side counts"},
            "capacity_vs_plain_fp64_single_rhs": round(sat["value"] / fp64_rate, 2),
            "service_ms_single_rhs": {f"{SERVING_CONFIGS[c][0]}@{lab}": {
                "mixed": round(single_mixed[(c, lab)] * 1e3, 1), "plain_fp64": round(single_fp64[(c, lab)] * 1e3, 1)}
                for c, lab in sorted(single_mixed)},
            "build_and_warmup_s": round(build_s, 1),
            "builds": stats.builds, "clones": stats.clones, "evictions": stats.evictions,
            "remasses": stats.remasses, "peak_resident_gb": round(stats.peak_resident_bytes / 2 ** 30, 2),
            "budget_gb": args.serve_budget_gb, "masses_without_m_nc": missing}


# ---------------------------------------------------------------------------
# clocks sampler
# ---------------------------------------------------------------------------
class Clocks:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                rows.append(f)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def gpu_bench(args):
    import torch
    import torch.distributed as dist
    from paper_0710_3612_gb300 import mg

    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    if args.serving_only:
        mg.lib()
        serving = serving_leg(args, mg, torch, dev)
        if rank == 0:
            print(json.dumps({"metric": "serving stream: right-hand sides solved per second at "
                              "saturation, latency p50/p99 per offered load",
                              "value": serving["value"], "unit": serving["unit"], "n_gpus": world,
                              "higher_is_better": True, "data": "synthetic", "serving": serving}))
        return

    # gauge fields of the batched workloads, generated on the host meanwhile
    import multiprocessing as mp
    cfg_names = [c for c in args.config_legs.split(",") if c]
    have = critical_table()
    cfg_gen = [c for c in cfg_names if W.BATCHED_WORKLOADS[c]["critical_key"] in have]
    cfg_pool = mp.get_context("spawn").Pool(len(cfg_gen)) if cfg_gen else None
    cfg_theta = {c: cfg_pool.apply_async(_gauge_angles, ((W.BATCHED_WORKLOADS[c]["Lx"],
                                                            W.BATCHED_WORKLOADS[c]["beta"],
                                                            W.BATCHED_WORKLOADS[c]["sweeps"],
                                                            W.BATCHED_WORKLOADS[c]["seed"]),))
                 for c in cfg_gen}
    wl, crit, U, noise, chi, masses = workload_inputs(args.workload)
    mg.lib()
    stream = torch.cuda.current_stream()
    U_d = torch.from_numpy(U).to(dev)
    noise_d = torch.from_numpy(noise).to(dev)
    chi_d = torch.from_numpy(chi).to(dev)
    b_d = torch.empty_like(chi_d)
    x_d = torch.empty_like(chi_d)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > L2
    tol = wl["tol"]
    params = mg.make_params(wl["Lx"], wl["Lt"], wl["blocks"], wl["Nv"], noise_d,
                            setup_sweeps=wl["setup_sweeps"], coarsest_reuse=args.coarsest_reuse)
    ev = lambda: torch.cuda.Event(enable_timing=True)   # noqa: E731

    def step(solver, record=None, profile=False, phases=None):
        p = params
        if profile:                        # per-kernel-family event timing from the setup on
            p = type(params).from_buffer_copy(params)
            p.profile = 1
        h = mg.mg_setup(U_d, masses[0], p, stream)
        mark = (lambda what: phases.append((what, mg.mg_kernel_launches()))) if phases is not None \
            else (lambda what: None)
        mark("setup")
        try:
            for m in masses:
                if m != masses[0]:
                    mg.mg_set_mass(h, m)
                    mark(f"set_mass {m}")
                mg.mg_apply_D(h, chi_d, b_d, 1, 1, mg.PREC_F64)
                e0, e1 = ev(), ev()
                e0.record(stream)
                st, info = mg.mg_solve(h, b_d, x_d, 1, tol, 200000, solver)
                e1.record(stream)
                if st != 0 or not info[0].true_residual <= tol:
                    raise RuntimeError(f"solve failed at m={m}: status {st}, "
                                       f"residual {info[0].true_residual}: {mg.mg_last_error(h)}")
                if record is not None:
                    record.append((m, e0, e1, info[0]))
                mark(f"solve {m}")
            prof = None
            if profile:
                prof = {f: mg.mg_profile_read(h, f) for f in range(mg.KF_COUNT)}
            return prof
        finally:
            mg.mg_destroy(h)

    def timed(solver, K, clocks=None, phases=None):
        recs, steps = [], []
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        if clocks:
            clocks.start()
        launches0 = mg.mg_kernel_launches()
        for i in range(K):
            flush.zero_()                      # L2 flush between timed steps
            s0, s1 = ev(), ev()
            s0.record(stream)
            step(solver, recs, phases=phases if i == 0 else None)
            s1.record(stream)
            steps.append((s0, s1))
        torch.cuda.synchronize()
        launches = mg.mg_kernel_launches() - launches0
        if world > 1:
            dist.barrier()
        ck = clocks.stop() if clocks else None
        step_ms = [a.elapsed_time(b) for a, b in steps]
        total = sum(step_ms)
        total = max_over_ranks(total, dev)
        solve_ms = [a.elapsed_time(b) for _, a, b, _ in recs]
        per_mass = {}
        for (m, a, b, info), t in zip(recs, solve_ms):
            d = per_mass.setdefault(repr(m), {"ms": [], "iterations": info.iterations,
                                              "fine_applies": info.fine_applies,
                                              "refinements": info.refinements,
                                              "true_residual": info.true_residual})
            d["ms"].append(t)
        for d in per_mass.values():
            d["median_ms"] = round(statistics.median(d.pop("ms")), 3)
        return {"total_ms": total, "step_ms": step_ms, "solve_ms": solve_ms, "per_mass": per_mass,
                "launches": launches, "clocks": ck}

    # warm-up
    for _ in range(args.warmup):
        step(MIXED_SOLVER)
    clocks = Clocks(local) if rank == 0 else None
    phases = [] if args.phase_launches else None
    base = mg.mg_kernel_launches()
    res = timed(MIXED_SOLVER, args.steps, clocks, phases)
    value = job_rate(len(masses) * args.steps, world, res["total_ms"] / 1000.0)

    if args.timed_only:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": round(value, 3), "unit": UNIT,
                              "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                              "ms_per_step": round(res["total_ms"] / args.steps, 3),
                              "per_mass": res["per_mass"], "gpu_launches": int(res["launches"]),
                              "phase_launches": [(w, n - base) for w, n in phases] if phases else None,
                              "note": "timed-only profiling run"}))
        return
    # plain FP64 MG-CG, same step
    kp = max(1, min(args.steps, args.plain_steps))
    step(mg.SOLVER_MGCG_FP64)
    plain = timed(mg.SOLVER_MGCG_FP64, kp)
    plain_value = job_rate(len(masses) * kp, world, plain["total_ms"] / 1000.0)
    # the other mixed-precision variant, same step
    other = [k for k in SOLVER_CODES if SOLVER_CODES[k] != MIXED_SOLVER][0]
    step(SOLVER_CODES[other])
    alt = timed(SOLVER_CODES[other], kp)
    alt_line = {"solver": other, "value": round(job_rate(len(masses) * kp, world, alt["total_ms"] / 1000.0), 3),
                "unit": UNIT, "steps": kp, "ms_per_step": round(alt["total_ms"] / kp, 3),
                "per_mass": alt["per_mass"]}

    # batched mixed-precision MG-CG: many right-hand sides of the same
    # configuration at the near-critical mass in one Krylov loop
    batched = batched_leg(args, mg, torch, dev, stream, wl, U_d, noise_d, masses, world)

    # adaptive refinement by V-cycles at the near-critical mass
    adaptive = adaptive_leg(args, mg, torch, dev, stream, wl, U_d, noise_d, masses, world)

    # batched workloads at their near-critical masses (256^2 x 64 RHS, 1024^2 x 16 RHS)
    config_legs = []
    for c in cfg_names:
        if c in cfg_theta:
            config_legs.append(batched_config_leg(args, mg, torch, dev, stream, c, cfg_theta[c].get(),
                                                  world))
        else:
            config_legs.append({"workload": c, "unavailable": "no near-critical mass from the "
                                "oracle's finder for this configuration"})
    if cfg_pool is not None:
        cfg_pool.close()

    # smoothed aggregation near the critical mass (NEXT-3)
    smoothed = smoothed_leg(args, mg, torch, dev, stream) if args.smoothed_leg else None

    # roofline: one profiled step, dominant kernel family by device time
    prof = step(MIXED_SOLVER, profile=True)
    roof = roofline(prof, wl, load_peaks())

    # end-to-end through the public API with host buffers
    e2e = e2e_leg(args, mg, torch, dev, stream, wl, U, noise, chi, masses, params, world)

    # serving: Poisson request stream over 8 configurations through the serving engine
    serving = serving_leg(args, mg, torch, dev) if args.serve_requests > 0 else None

    if rank == 0:
        sm = sorted(res["solve_ms"])
        pct = lambda q: sm[min(len(sm) - 1, int(math.ceil(q * len(sm))) - 1)]   # noqa: E731
        psm = sorted(plain["solve_ms"])
        ppct = lambda q: psm[min(len(psm) - 1, int(math.ceil(q * len(psm))) - 1)]   # noqa: E731
        cpu = None if (args.no_cpu_baseline or world > 1) else cpu_baseline(args)
        line = {
            "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(res["total_ms"] / args.steps, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": ("f32+bf16 (V-cycle), f32 (Krylov iteration) / f64 (reliable updates, solution, "
                      "true residual, coarsest)" if args.solver == "reliable" else
                      "f32+bf16 (V-cycle) / f64 (outer, residual, coarsest)"),
            "data": "synthetic: seeded quenched U(1) Metropolis configuration, Gaussian source",
            "config": {"workload": args.workload, "lattice": [wl["Lx"], wl["Lt"]], "beta": wl["beta"],
                       "levels": len(wl["blocks"]) + 1, "blocks": wl["blocks"], "Nv": wl["Nv"],
                       "masses": [round(m, 12) for m in masses], "m_crit": crit["m_crit"],
                       "tol": wl["tol"], "rhs_per_solve": 1, "solves_per_step": len(masses),
                       "step": "setup at m_nc + 4 x (re-Galerkin/coarsest inverse, b = D^dag chi, solve)",
                       "coarsest_reuse": args.coarsest_reuse,
                       "parallelism": f"replicas x{world}",
                       "l2": "flushed between timed steps (256 MiB write)"},
            "latency_ms": {"p50": round(pct(0.5), 3), "p99": round(pct(0.99), 3),
                           "per_mass": res["per_mass"]},
            "plain_fp64": {"value": round(plain_value, 3), "unit": UNIT, "steps": kp,
                           "ms_per_step": round(plain["total_ms"] / kp, 3),
                           "p50_ms": round(ppct(0.5), 3), "p99_ms": round(ppct(0.99), 3),
                           "per_mass": plain["per_mass"]},
            "mixed_vs_plain_fp64": round(value / plain_value, 3),
            "solver": args.solver,
            "other_mixed_solver": alt_line,
            "batched": batched,
            "batched_configs": config_legs,
            "smoothed_aggregation": smoothed,
            "adaptive": adaptive,
            "serving": serving,
            "roofline": roof,
            "stencil": stencil_gbs(mg, torch, dev, stream),
            "stencil_multi_rhs": stencil_multi_rhs(mg, torch, dev, stream),
            "autotune": mg.stencil_tunings(),
            "gauge_gen": gauge_gen_leg(mg, torch, dev, stream),
            "e2e": e2e,
            "gpu_launches": int(res["launches"]),
            "clocks": res["clocks"],
            "cpu_baseline": cpu,
        }
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


FAM_NAMES = ["fine_A_f32", "coarse_apply_f32_bf16", "transfer", "coarsest_solve",
             "coarsest_inverse", "galerkin", "fine_A_f64", "coarsest_gemv_tiles", "gj_update",
             "coarse_apply_f64"]

def ncu_traffic():
    """DRAM bytes (read + write) per launch of each roofline candidate from the
    ncu captures recorded in profiles/ncu_traffic.json, each with the SHA-256
    of the CUDA source file it was captured from; a candidate whose source has
    changed since its capture gets None."""
    import hashlib
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(p):
        return {}
    out = {}
    for name, rec in json.load(open(p)).items():
        src = os.path.join(ROOT, rec["source"])
        ok = os.path.exists(src) and hashlib.sha256(open(src, "rb").read()).hexdigest() == rec["source_sha256"]
        out[name] = rec["dram_bytes_per_launch"] if ok else None
    return out


def roofline(prof, wl, peaks):
    """Roofline of the dominant kernel of one profiled (eager) step, and of
    the other candidates.  The candidates are the profiling families that time
    one kind of kernel each (CUDA events recorded on the library's stream
    around each launch, set-up included): the tensor-core Gauss-Jordan update
    of the coarsest inverse, the fused FP32 and FP64 fine stencils, the tile
    kernel of the packed Hermitian GEMV and the BF16 coarse apply; achieved =
    algorithmic bytes (or flops) per launch / average launch duration."""
    Lx, Lt = wl["Lx"], wl["Lt"]
    V = Lx * Lt
    Nv1, Nv2 = wl["Nv"]
    b1, b2 = wl["blocks"]
    V2 = V // (b1[0] * b1[1])
    V3 = V2 // (b2[0] * b2[1])
    N3 = V3 * 2 * Nv2
    ld = (N3 + 63) // 64 * 64
    nt = ld // 64
    ntiles = nt * (nt + 1) // 2
    cand = {8: "gj_update", 7: "coarsest_gemv_tiles", 1: "coarse_apply_bf16", 0: "fine_A_f32",
            6: "fine_A_f64"}
    traffic = ncu_traffic()
    total = sum(prof[f][0] for f in cand)

    def one(fam):
        ms, calls = prof[fam]
        per_call_s = ms / 1000.0 / max(calls, 1)
        o = {"kernel": cand[fam], "launches": calls, "avg_us": round(per_call_s * 1e6, 3),
             "ms_in_step": round(ms, 3)}
        if fam == 8:
            # complex rank-64 update of the lower 64 x 64 tiles outside the pivot
            # row and column: 64^3 complex multiply-adds (8 real flops) per tile
            flops = (ntiles - nt) * 64.0 ** 3 * 8.0
            peak = peaks["bf16_tflops_sustained"] * 1.1 / 2.25   # nominal TF32 / BF16 ratio
            o.update({"bound": "tensor", "achieved": round(flops / per_call_s / 1e12, 3),
                      "peak": round(peak, 1), "unit": "TFLOP/s", "flops_per_launch": flops,
                      "peak_note": f"of {peaks['src']}: sustained bf16 x nominal tf32/bf16 1.1/2.25",
                      "tensor_flops_issued_per_launch": 3 * flops,
                      "note": "mma.sync m16n8k8 TF32, three products per FP32-accurate product",
                      "traffic": traffic.get("gj_update")})
        else:
            if fam == 0:
                byts = 48.0 * V                          # psi in/out + links, FP32
            elif fam == 6:
                byts = 96.0 * V
            elif fam == 1:      # level-2 BF16 blocks + FP32 input and output vectors
                byts = V2 * (9 * (2 * Nv1) ** 2 * 4.0 + 2 * 2 * Nv1 * 8.0)
            else:               # packed lower tiles of the inverse + per-tile partial sums
                byts = ntiles * 64 * 64 * 8.0 + ntiles * 2 * 64 * 8.0
            o.update({"bound": "hbm", "achieved": round(byts / per_call_s / 1e9, 1),
                      "peak": peaks["hbm_gbs"], "unit": "GB/s", "bytes_per_launch": int(byts),
                      "peak_note": f"of {peaks['src']}", "traffic": traffic.get(cand[fam])})
        o["frac"] = round(o["achieved"] / o["peak"], 4)
        o["share_of_candidates"] = round(ms / total, 3) if total else None
        return o

    fam = max(cand, key=lambda f: prof[f][0])
    out = one(fam)
    out["timing"] = "CUDA events on the library stream around each launch, one eager step"
    out["family_ms_in_step"] = {FAM_NAMES[f]: round(prof[f][0], 3) for f in prof}
    out["other_candidates"] = [one(f) for f in cand if f != fam]
    return out


def stencil_gbs(mg, torch, dev, stream):
    """Fused A = D^dagger D (FP32) on a 4096 x 4096 lattice (above L2): algorithmic
    48 B/site over CUDA-event time, median of 50 after 10 warm-ups."""
    L = 4096
    U = torch.polar(torch.ones(2, L, L, dtype=torch.float64, device=dev),
                    torch.rand(2, L, L, dtype=torch.float64, device=dev) * 0.5).contiguous()
    params = mg.make_params(L, L, [], [])          # nlevels = 1: fine operator only
    h = mg.mg_setup(U, 0.1, params, stream)
    try:
        x = torch.randn(L * L * 2, dtype=torch.complex64, device=dev)
        y = torch.empty_like(x)
        for _ in range(10):
            mg.mg_apply_A(h, x, y, 1, mg.PREC_F32)
        ts = []
        for _ in range(50):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            mg.mg_apply_A(h, x, y, 1, mg.PREC_F32)
            b.record(stream)
            ts.append((a, b))
        torch.cuda.synchronize()
        med = statistics.median(a.elapsed_time(b) for a, b in ts)
        gbs = 48.0 * L * L / (med / 1000.0) / 1e9
        peaks = load_peaks()
        return {"lattice": [L, L], "precision": "f32", "median_us": round(med * 1000, 2),
                "gbs": round(gbs, 1), "frac_hbm": round(gbs / peaks["hbm_gbs"], 4),
                "bytes_per_site": 48}
    finally:
        mg.mg_destroy(h)


def stencil_multi_rhs(mg, torch, dev, stream, L=1024, nrhs=16):
    """Fused FP32 A on nrhs vectors of an L x L lattice (the 1024^2 x 16
    workload's shape, about 550 MB per launch, above L2): algorithmic
    32 nrhs + 16 bytes per site over CUDA-event time, median of 20 after 5
    warm-ups (the autotuned launch shape)."""
    U = torch.polar(torch.ones(2, L, L, dtype=torch.float64, device=dev),
                    torch.rand(2, L, L, dtype=torch.float64, device=dev) * 0.5).contiguous()
    p = mg.make_params(L, L, [], [], max_rhs=nrhs)
    h = mg.mg_setup(U, 0.1, p, stream)
    try:
        x = torch.randn(nrhs * L * L * 2, dtype=torch.complex64, device=dev)
        y = torch.empty_like(x)
        for _ in range(5):
            mg.mg_apply_A(h, x, y, nrhs, mg.PREC_F32)
        ts = []
        for _ in range(20):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            mg.mg_apply_A(h, x, y, nrhs, mg.PREC_F32)
            b.record(stream)
            ts.append((a, b))
        torch.cuda.synchronize()
        med = statistics.median(a.elapsed_time(b) for a, b in ts)
        byt = (32.0 * nrhs + 16.0) * L * L
        peaks = load_peaks()
        return {"lattice": [L, L], "nrhs": nrhs, "precision": "f32", "median_us": round(med * 1000, 2),
                "gbs": round(byt / (med / 1000.0) / 1e9, 1),
                "frac_hbm": round(byt / (med / 1000.0) / 1e9 / peaks["hbm_gbs"], 4),
                "bytes_per_site": 32 * nrhs + 16, "peak_note": f"of {peaks['src']}"}
    finally:
        mg.mg_destroy(h)


def gauge_gen_leg(mg, torch, dev, stream):
    """Quenched U(1) field of the largest serving lattice on the device
    (checkerboard Metropolis, counter-based uniforms): 512 x 512, beta = 10,
    500 sweeps from a cold start, CUDA-event time."""
    L, beta, sweeps = 512, 10.0, 500
    th = torch.zeros((2, L, L), dtype=torch.float64, device=dev)
    mg.gauge_metropolis(th, beta, 5, 1, stream=stream)            # warm-up (discarded)
    th.zero_()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    acc = mg.gauge_metropolis(th, beta, sweeps, 1, stream=stream)
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    return {"lattice": [L, L], "beta": beta, "sweeps": sweeps, "ms": round(ms, 2),
            "link_updates_per_s": round(2 * L * L * sweeps / (ms / 1000.0), 1),
            "acceptance": round(acc / (2 * L * L * sweeps), 4),
            "mean_plaquette": round(float(torch.cos(th[0] + torch.roll(th[1], -1, 1)
                                                    - torch.roll(th[0], -1, 0) - th[1]).mean()), 6)}


def batched_leg(args, mg, torch, dev, stream, wl, U_d, noise_d, masses, world):
    """nrhs Gaussian sources chi_k (seeds chi_seed + 1000 + k), b_k = D^dagger chi_k,
    solved together at the near-critical mass with the mixed solver (BF16 coarse
    blocks on the tensor cores); solves/s against plain FP64 single-RHS MG-CG on
    the same right-hand sides (first two of them)."""
    nrhs = args.batch_rhs
    if nrhs < 1:
        return None
    chis = np.stack([W.gaussian_field((wl["Lt"], wl["Lx"], 2), wl["chi_seed"] + 1000 + k)
                     for k in range(nrhs)])
    chi_d = torch.from_numpy(chis).to(dev)
    b_d = torch.empty_like(chi_d)
    x_d = torch.empty_like(chi_d)
    tol = wl["tol"]
    out = {"nrhs": nrhs, "mass": masses[0]}
    with mg.Multigrid(U_d, masses[0], wl["blocks"], wl["Nv"], noise_d,
                      setup_sweeps=wl["setup_sweeps"], max_rhs=nrhs) as s:
        mg.mg_apply_D(s.h, chi_d, b_d, nrhs, 1, mg.PREC_F64)
        mg.mg_solve(s.h, b_d, x_d, nrhs, tol, 200000, MIXED_SOLVER)     # warm-up
        reps = []
        for _ in range(max(1, args.batch_reps)):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st, info = mg.mg_solve(s.h, b_d, x_d, nrhs, tol, 200000, MIXED_SOLVER)
            e1.record(stream)
            torch.cuda.synchronize()
            if st != 0 or max(i.true_residual for i in info) > tol:
                raise RuntimeError("batched solve did not converge")
            reps.append(e0.elapsed_time(e1))
        ms = max_over_ranks(statistics.median(reps), dev)
        out.update({"value": round(job_rate(nrhs, world, ms / 1000.0), 3), "unit": UNIT,
                    "ms_per_batch": round(ms, 3),
                    "iterations_max": max(i.iterations for i in info),
                    "max_true_residual": max(i.true_residual for i in info)})
    with mg.Multigrid(U_d, masses[0], wl["blocks"], wl["Nv"], noise_d,
                      setup_sweeps=wl["setup_sweeps"]) as s:
        ts = []
        for k in range(2):
            bk = b_d[k].contiguous()
            xk = torch.empty_like(bk)
            mg.mg_solve(s.h, bk, xk, 1, tol, 200000, mg.SOLVER_MGCG_FP64)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            mg.mg_solve(s.h, bk, xk, 1, tol, 200000, mg.SOLVER_MGCG_FP64)
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        out["plain_fp64_single_rhs"] = round(1000.0 / statistics.median(ts), 3)
        out["vs_plain_fp64_single_rhs"] = round(out["value"] / world / out["plain_fp64_single_rhs"], 2)
    return out


def adaptive_leg(args, mg, torch, dev, stream, wl, U_d, noise_d, masses, world):
    """Adaptive refinement by V-cycles (Sec. 3) on the workload's hierarchy at
    the near-critical mass: `plan` lists the level refined by each pass
    (args.adaptive_cycles V-cycles on a Gaussian error, seeds noise_seed + 100 + p;
    coarser levels set up again from setup noise of seed noise_seed + 1 + p).
    Reports the refinement time, and the single-RHS and batched mixed solves
    at m_nc before and after it (the headline step keeps the relaxation-only
    set-up of the workload definition)."""
    plan = [int(c) for c in args.adaptive_plan]
    if not plan:
        return None
    L, Lt, blocks, tol, m = wl["Lx"], wl["Lt"], wl["blocks"], wl["tol"], masses[0]
    nrhs = max(1, args.batch_rhs)
    chis = np.stack([W.gaussian_field((Lt, L, 2), wl["chi_seed"] + 1000 + k) for k in range(nrhs)])
    chi_d = torch.from_numpy(chis).to(dev)
    b_d = torch.empty_like(chi_d)
    x_d = torch.empty_like(chi_d)
    ev = lambda: torch.cuda.Event(enable_timing=True)   # noqa: E731

    def timed_solve(h, n):
        mg.mg_solve(h, b_d, x_d, n, tol, 200000, MIXED_SOLVER)       # warm-up
        reps = []
        for _ in range(3):
            e0, e1 = ev(), ev()
            e0.record(stream)
            st, info = mg.mg_solve(h, b_d, x_d, n, tol, 200000, MIXED_SOLVER)
            e1.record(stream)
            torch.cuda.synchronize()
            if st != 0 or max(i.true_residual for i in info) > tol:
                raise RuntimeError("adaptive leg: solve did not converge")
            reps.append(e0.elapsed_time(e1))
        ms = max_over_ranks(statistics.median(reps), dev)
        return {"iterations_max": max(i.iterations for i in info), "ms": round(ms, 3),
                "max_true_residual": max(i.true_residual for i in info)}

    Nv = list(wl["Nv"])
    out = {"plan": args.adaptive_plan, "ncycles": args.adaptive_cycles, "mass": m}
    with mg.Multigrid(U_d, m, blocks, Nv, noise_d, setup_sweeps=wl["setup_sweeps"],
                      max_rhs=nrhs) as s:
        mg.mg_apply_D(s.h, chi_d, b_d, nrhs, 1, mg.PREC_F64)
        before1, beforeB = timed_solve(s.h, 1), timed_solve(s.h, nrhs)
        rhos, keep = [], []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for p, lvl in enumerate(plan):
            Nv[lvl - 1] += 1
            Lx_l, Lt_l, n_l, _ = mg.mg_get_level(s.h, lvl)
            e0 = torch.from_numpy(W.gaussian_field((Lt_l, Lx_l, n_l), wl["noise_seed"] + 100 + p)).to(dev)
            nz = torch.from_numpy(W.refine_noise(L, Lt, blocks, Nv, lvl - 1, wl["noise_seed"] + 1 + p)).to(dev)
            keep.append(nz)
            rhos.append(round(s.refine(lvl, e0, args.adaptive_cycles, nz), 4))
        torch.cuda.synchronize()
        refine_ms = max_over_ranks((time.perf_counter() - t0) * 1e3, dev)
        after1, afterB = timed_solve(s.h, 1), timed_solve(s.h, nrhs)
        coarsest = mg.mg_get_level(s.h, len(blocks) + 1)
    out.update({"Nv_after": Nv, "rho_per_pass": rhos, "refine_ms": round(refine_ms, 1),
                "coarsest_unknowns": coarsest[0] * coarsest[1] * coarsest[2],
                "single_rhs": {"relaxation_only": before1, "refined": after1,
                               "speedup": round(before1["ms"] / after1["ms"], 2)},
                "batched": {"nrhs": nrhs,
                            "relaxation_only": dict(beforeB, value=round(job_rate(nrhs, world, beforeB["ms"] / 1e3), 3)),
                            "refined": dict(afterB, value=round(job_rate(nrhs, world, afterB["ms"] / 1e3), 3)),
                            "unit": UNIT,
                            "speedup": round(beforeB["ms"] / afterB["ms"], 2)},
                "breakeven_solves": round(refine_ms / max(1e-9, before1["ms"] - after1["ms"]), 1)})
    return out


def batched_config_leg(args, mg, torch, dev, stream, name, theta, world):
    """One batched workload of workloads.BATCHED_WORKLOADS at its near-critical
    mass (the oracle's finder, workloads/critical_masses.json): nrhs Gaussian
    sources chi_k (seeds chi_seed + k), b_k = D^dagger chi_k, solved together
    with the mixed solver.  Reported: set-up time; solves/s over `config_reps`
    batches and the per-batch latency percentiles; plain FP64 single-RHS MG-CG
    on b_0 (time-capped: its rate is then iterations done / time); the
    multi-RHS BF16 coarse apply of level 2 and the fused FP32 fine stencil on
    nrhs vectors, each over its CUDA-event time, against the HBM roofline."""
    wl = W.BATCHED_WORKLOADS[name]
    Lx, Lt, nrhs, tol = wl["Lx"], wl["Lt"], wl["nrhs"], wl["tol"]
    out = {"workload": name, "lattice": [Lx, Lt], "beta": wl["beta"], "levels": len(wl["blocks"]) + 1,
           "blocks": wl["blocks"], "Nv": wl["Nv"], "nrhs": nrhs}
    crit = critical_table().get(wl["critical_key"])
    if crit is None:
        out["unavailable"] = "no near-critical mass from the oracle's finder for this configuration"
        return out
    if abs(W.mean_plaquette(theta) - crit["plaquette"]) > 1e-12:
        out["unavailable"] = "regenerated gauge field differs from the one the finder used"
        return out
    m = crit["m_nc"]
    out.update({"mass": m, "m_crit": crit["m_crit"], "lambda_min": crit["lambda_min"]})
    ev = lambda: torch.cuda.Event(enable_timing=True)   # noqa: E731
    U_d = torch.from_numpy(W.links_from_angles(theta)).to(dev)
    noise_d = torch.from_numpy(W.setup_noise(Lx, Lt, wl["blocks"], wl["Nv"], wl["noise_seed"])).to(dev)
    chi_d = torch.from_numpy(np.stack([W.gaussian_field((Lt, Lx, 2), wl["chi_seed"] + k)
                                       for k in range(nrhs)])).to(dev)
    b_d = torch.empty_like(chi_d)
    x_d = torch.empty_like(chi_d)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s = mg.Multigrid(U_d, m, wl["blocks"], wl["Nv"], noise_d, stream=stream,
                     setup_sweeps=wl["setup_sweeps"], max_rhs=nrhs, **wl.get("params", {}))
    torch.cuda.synchronize()
    out["setup_ms"] = round((time.perf_counter() - t0) * 1e3, 1)
    try:
        dense, steps, tres = mg.mg_get_coarsest_info(s.h)
        Lc = mg.mg_get_level(s.h, len(wl["blocks"]) + 1)
        out["coarsest"] = {"unknowns": Lc[0] * Lc[1] * Lc[2], "solver": "fp32 inverse + fp64 refinement"
                           if dense else "fp64 cg", "steps": steps, "test_residual": tres}
        out["device_gb"] = round(mg.mg_device_bytes(s.h) / 2 ** 30, 2)
        mg.mg_apply_D(s.h, chi_d, b_d, nrhs, 1, mg.PREC_F64)
        mg.mg_solve(s.h, b_d, x_d, nrhs, tol, 30, MIXED_SOLVER)   # warm-up: graphs built
        lat = []
        for _ in range(max(1, min(args.config_reps, wl.get("reps", args.config_reps)))):
            e0, e1 = ev(), ev()
            e0.record(stream)
            st, info = mg.mg_solve(s.h, b_d, x_d, nrhs, tol, 100000, MIXED_SOLVER)
            e1.record(stream)
            torch.cuda.synchronize()
            if st != 0 or max(i.true_residual for i in info) > tol:
                raise RuntimeError(f"{name}: batched solve failed (status {st})")
            lat.append(e0.elapsed_time(e1))
        ms = max_over_ranks(statistics.median(lat), dev)
        ls = sorted(lat)
        pct = lambda q: ls[min(len(ls) - 1, int(math.ceil(q * len(ls))) - 1)]   # noqa: E731
        out.update({"value": round(job_rate(nrhs, world, ms / 1000.0), 3), "unit": UNIT,
                    "batches": len(lat), "ms_per_batch": round(ms, 2),
                    "latency_ms": {"p50": round(pct(0.5), 2), "p99": round(pct(0.99), 2),
                                   "note": f"per batch of {nrhs}, over {len(lat)} batches"},
                    "iterations_max": max(i.iterations for i in info),
                    "max_true_residual": max(i.true_residual for i in info)})
        # where the time of an iteration goes (50 eager iterations, CUDA events
        # per kernel family; eager launches add a few microseconds per kernel)
        mg.mg_profile_enable(s.h, 1)
        mg.mg_solve(s.h, b_d, x_d, nrhs, tol, 50, MIXED_SOLVER)
        out["family_ms_per_iteration"] = {FAM_NAMES[f]: round(mg.mg_profile_read(s.h, f)[0] / 50, 3)
                                          for f in range(mg.KF_COUNT)}
        mg.mg_profile_enable(s.h, 0)
        # plain FP64 single-RHS MG-CG on b_0, capped in time
        b0 = b_d[0].contiguous()
        x0 = torch.empty_like(b0)
        cap = max(1, args.plain_iter_cap)
        e0, e1 = ev(), ev()
        e0.record(stream)
        st, info1 = mg.mg_solve(s.h, b0, x0, 1, tol, cap, mg.SOLVER_MGCG_FP64)
        e1.record(stream)
        torch.cuda.synchronize()
        t1 = e0.elapsed_time(e1)
        it1 = info1[0].iterations
        conv = st == 0 and info1[0].true_residual <= tol
        mixed_iters = max(i.iterations for i in info)
        plain = {"iterations": it1, "ms": round(t1, 2), "converged": bool(conv),
                 "true_residual": info1[0].true_residual}
        if conv:
            plain["value"] = round(job_rate(1, world, t1 / 1000.0), 4)
        else:   # the same per-iteration cost over the mixed solver's iteration count (labelled)
            plain["value_extrapolated"] = round(job_rate(1, world, t1 / 1000.0 * mixed_iters / max(it1, 1)), 4)
            plain["note"] = (f"stopped at {cap} iterations; rate extrapolated to the mixed batch's "
                             f"{mixed_iters} iterations at the measured cost per iteration")
        out["plain_fp64_single_rhs"] = plain
        pv = plain.get("value", plain.get("value_extrapolated"))
        out["vs_plain_fp64_single_rhs"] = round(out["value"] / world / pv, 2) if pv else None
        # level-2 multi-RHS BF16 coarse apply (tcgen05) and fine stencil on nrhs vectors
        Lx2, Lt2, n2, _ = mg.mg_get_level(s.h, 2)
        xc = torch.randn((nrhs, Lt2, Lx2, n2), dtype=torch.complex64, device=dev)
        yc = torch.empty_like(xc)
        xf = torch.randn((nrhs, Lt, Lx, 2), dtype=torch.complex64, device=dev)
        yf = torch.empty_like(xf)

        def kernel_us(fn, reps=20):
            for _ in range(3):
                fn()
            e0, e1 = ev(), ev()
            e0.record(stream)
            for _ in range(reps):
                fn()
            e1.record(stream)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) * 1e3 / reps
        peaks = load_peaks()
        us_c = kernel_us(lambda: mg.mg_apply_coarse(s.h, 2, xc, yc, nrhs, mg.PREC_BF16))
        byt_c = Lx2 * Lt2 * (9 * n2 * n2 * 4.0 + 2 * n2 * nrhs * 8.0)
        fl_c = 8.0 * 9 * n2 * n2 * nrhs * Lx2 * Lt2
        out["coarse_apply_level2"] = {
            "kernel": "tcgen05 multi-RHS BF16 coarse apply", "sites": Lx2 * Lt2, "dof": n2, "nrhs": nrhs,
            "us": round(us_c, 2), "bytes": int(byt_c), "achieved_gbs": round(byt_c / us_c / 1e3, 1),
            "frac_hbm": round(byt_c / us_c / 1e3 / peaks["hbm_gbs"], 4),
            "tflops": round(fl_c / us_c / 1e6, 2), "peak_note": f"of {peaks['src']}",
            "timing": "20 back-to-back launches between CUDA events on the library stream"}
        us_f = kernel_us(lambda: mg.mg_apply_A(s.h, xf, yf, nrhs, mg.PREC_F32))
        byt_f = Lx * Lt * (32.0 * nrhs + 16.0)
        out["fine_stencil"] = {"precision": "f32", "nrhs": nrhs, "us": round(us_f, 2),
                               "bytes_per_site": 32 * nrhs + 16, "achieved_gbs": round(byt_f / us_f / 1e3, 1),
                               "frac_hbm": round(byt_f / us_f / 1e3 / peaks["hbm_gbs"], 4),
                               "peak_note": f"of {peaks['src']}",
                               "working_set_mb": round(Lx * Lt * (32.0 * nrhs + 16.0) / 2 ** 20, 1)}
    finally:
        s.close()
    return out


def smoothed_leg(args, mg, torch, dev, stream):
    """Smoothed aggregation (Sec. 3) near the critical mass: 64 x 64, beta = 3
    (200 sweeps, seed 1) at its near-critical mass (the oracle's finder), 4 x 4
    blocks, Nv = 8.  omega from the condition-number search on the two-level
    hierarchy; the same omega on three levels (4 x 4 then 2 x 2 blocks; the
    first level's vectors are the same, so is the optimal omega).  FP64 and
    mixed MG-CG iterations and CUDA-event times on one Gaussian source, with
    the smoothed and with the tentative prolongator."""
    crit = critical_table().get("L64_b3_s1")
    L = 64
    th = W.quenched_u1_angles(L, L, 3.0, 200, 1)
    if crit is None or abs(W.mean_plaquette(th) - crit["plaquette"]) > 1e-12:
        return {"unavailable": "no near-critical mass for the 64 x 64 beta 3 configuration"}
    m = crit["m_nc"]
    U = torch.from_numpy(W.links_from_angles(th)).to(dev)
    b = torch.from_numpy(W.gaussian_field((L, L, 2), 303)).to(dev)
    out = {"lattice": [L, L], "beta": 3.0, "mass": m, "m_crit": crit["m_crit"], "Nv": 8}
    ev = lambda: torch.cuda.Event(enable_timing=True)   # noqa: E731

    def run(blocks, Nv, **kw):
        noise = torch.from_numpy(W.setup_noise(L, L, blocks, Nv, 7)).to(dev)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with mg.Multigrid(U, m, blocks, Nv, noise, stream=stream, **kw) as s:
            torch.cuda.synchronize()
            setup_ms = (time.perf_counter() - t0) * 1e3
            om, cond = mg.mg_get_smoothing(s.h)
            bd = torch.empty_like(b)
            mg.mg_apply_D(s.h, b, bd, 1, 1, mg.PREC_F64)
            r = {"setup_ms": round(setup_ms, 1), "omega": om}
            if cond:
                r["cond_level2"] = round(cond, 3)
            for name, solver in (("fp64", mg.SOLVER_MGCG_FP64), ("mixed", MIXED_SOLVER)):
                x = torch.empty_like(bd)
                mg.mg_solve(s.h, bd, x, 1, 1e-10, 100000, solver)
                e0, e1 = ev(), ev()
                e0.record(stream)
                st, info = mg.mg_solve(s.h, bd, x, 1, 1e-10, 100000, solver)
                e1.record(stream)
                torch.cuda.synchronize()
                if st != 0 or info[0].true_residual > 1e-10:
                    raise RuntimeError("smoothed leg: solve failed")
                r[name] = {"iterations": info[0].iterations, "ms": round(e0.elapsed_time(e1), 2)}
            return r
    two = [(4, 4)]
    three = [(4, 4), (2, 2)]
    sm2 = run(two, [8], smooth_omega=-1.0)
    out["two_levels"] = {"smoothed": sm2, "tentative": run(two, [8])}
    out["three_levels"] = {"smoothed": run(three, [8, 8], smooth_omega=sm2["omega"]),
                           "tentative": run(three, [8, 8])}
    return out


def e2e_leg(args, mg, torch, dev, stream, wl, U, noise, chi, masses, params, world):
    """Same step through the public API with pinned host buffers copied in and
    the solutions copied out inside the timed region."""
    Uh = torch.from_numpy(U).pin_memory()
    nh = torch.from_numpy(noise).pin_memory()
    ch = torch.from_numpy(chi).pin_memory()
    xh = torch.empty_like(ch).pin_memory()
    K = max(1, min(args.steps, args.e2e_steps))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(K):
        Ud = Uh.to(dev, non_blocking=True)
        nd = nh.to(dev, non_blocking=True)
        cd = ch.to(dev, non_blocking=True)
        with mg.Multigrid(Ud, masses[0], wl["blocks"], wl["Nv"], nd,
                          setup_sweeps=wl["setup_sweeps"], coarsest_reuse=args.coarsest_reuse) as s:
            b = torch.empty_like(cd)
            for m in masses:
                if m != masses[0]:
                    s.set_mass(m)
                mg.mg_apply_D(s.h, cd, b, 1, 1, mg.PREC_F64)
                x, info = s.solve(b, tol=wl["tol"], maxiter=200000, solver=MIXED_SOLVER)
                xh.copy_(x, non_blocking=True)
                torch.cuda.synchronize()
                if not info[0].true_residual <= wl["tol"]:
                    raise RuntimeError("e2e solve did not converge")
    torch.cuda.synchronize()
    dt = max_over_ranks(time.perf_counter() - t0, dev)
    return {"value": round(job_rate(len(masses) * K, world, dt), 3), "unit": UNIT, "steps": K,
            "h2d_bytes_per_step": int(Uh.nbytes + nh.nbytes + ch.nbytes),
            "d2h_bytes_per_step": int(len(masses) * xh.nbytes)}


# ---------------------------------------------------------------------------
# CPU oracle: bounded sample, scaled to whole solves
# ---------------------------------------------------------------------------
def oracle_sample(name, nc_iters_sample):
    """Runs in a subprocess with one BLAS thread: setup at m_nc, re-mass + solve at
    the heaviest mass, and nc_iters_sample MG-CG iterations at m_nc.  Returns
    per-phase seconds."""
    from oracle import krylov, multigrid, wilson
    wl, crit, U, noise, chi, masses = workload_inputs(name)
    t0 = time.perf_counter()
    H = multigrid.setup(U, masses[0], wl["blocks"], wl["Nv"], noise, sweeps=wl["setup_sweeps"])
    t_setup = time.perf_counter() - t0
    b = wilson.apply_D(U, masses[0], chi, dagger=True)
    t0 = time.perf_counter()
    krylov.mgcg(H, b, 1e-300, nc_iters_sample)
    t_nc = (time.perf_counter() - t0) / nc_iters_sample
    t0 = time.perf_counter()
    multigrid.set_mass(H, masses[-1])
    t_mass = time.perf_counter() - t0
    b = wilson.apply_D(U, masses[-1], chi, dagger=True)
    t0 = time.perf_counter()
    _, it_heavy, _ = krylov.mgcg(H, b, wl["tol"], 20000)
    t_heavy = time.perf_counter() - t0
    return {"setup_s": t_setup, "nc_iter_s": t_nc, "set_mass_s": t_mass,
            "heavy_solve_s": t_heavy, "heavy_iters": it_heavy}


def scale_oracle(name, s):
    """Seconds of one full 4-mass step from the sample, using the oracle's own
    iteration counts (workloads/oracle_iterations.json)."""
    its = json.load(open(os.path.join(ROOT, "workloads", "oracle_iterations.json")))[name]["masses"]
    wl, crit, *_ = (W.BENCH_WORKLOADS[name], json.load(open(os.path.join(
        ROOT, "workloads", "critical_masses.json")))[W.BENCH_WORKLOADS[name]["critical_key"]])
    n_nc = its[repr(crit["m_nc"])]["iterations"]
    heavy = [its[repr(m)]["iterations"] for m in wl["heavy_masses"]]
    per_heavy_iter = s["heavy_solve_s"] / max(s["heavy_iters"], 1)
    step_s = (s["setup_s"] + n_nc * s["nc_iter_s"] + 3 * s["set_mass_s"]
              + sum(heavy) * per_heavy_iter)
    return step_s, n_nc


def run_oracle_subprocess(name, iters):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    code = ("import json,sys; sys.path.insert(0, %r); import bench; "
            "print(json.dumps(bench.oracle_sample(%r, %d)))" % (ROOT, name, iters))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                       cwd=ROOT, timeout=900)
    if r.returncode != 0:
        raise RuntimeError("oracle sample failed: " + r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def host_cpu():
    """Model name and logical core count of the host."""
    model = None
    try:
        for line in open("/proc/cpuinfo"):
            k = line.split(":")[0].strip().lower()
            if k in ("model name", "cpu model", "hardware"):
                model = line.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    if model is None:
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True).stdout
            for line in out.splitlines():
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except OSError:
            pass
    return model or "unknown", os.cpu_count() or 1


def cpu_baseline(args):
    """The oracle on one host core, and the same sample run on every core at
    once (independent processes, one BLAS thread each: the host's whole-CPU
    rate for independent solves, the sum of the per-process rates)."""
    from concurrent.futures import ThreadPoolExecutor
    model, cores = host_cpu()
    t0 = time.perf_counter()
    s = run_oracle_subprocess(args.workload, args.oracle_iters)
    wall = time.perf_counter() - t0
    step_s, n_nc = scale_oracle(args.workload, s)
    out = {"value": round(4.0 / step_s, 5), "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": (f"numpy FP64 oracle, 1 thread: setup at m_nc, {args.oracle_iters} MG-CG "
                      f"iterations at m_nc, re-mass + full solve at m=0.1; scaled to the 4-mass "
                      f"step with the oracle's iteration counts (m_nc: {n_nc})"),
           "sample_wall_s": round(wall, 1), "scaled_step_s": round(step_s, 2),
           "host_cpu": model, "host_cores": cores}
    if args.cpu_all_cores:
        t0 = time.perf_counter()
        with ThreadPoolExecutor(cores) as ex:
            samples = list(ex.map(lambda _: run_oracle_subprocess(args.workload, args.oracle_iters),
                                  range(cores)))
        wall_all = time.perf_counter() - t0
        rate = sum(4.0 / scale_oracle(args.workload, q)[0] for q in samples)
        out["all_cores"] = {"value": round(rate, 5), "unit": UNIT, "cores": cores,
                            "processes": cores, "sample_wall_s": round(wall_all, 1),
                            "note": "one oracle process per core, each the 1-thread sample above"}
    return out


def reference_arm(args):
    rank = int(os.environ.get("RANK", 0))
    if rank != 0:
        return
    for _ in range(args.warmup):
        run_oracle_subprocess(args.workload, 2)
    vals, walls = [], []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        s = run_oracle_subprocess(args.workload, args.oracle_iters)
        walls.append(time.perf_counter() - t0)
        step_s, n_nc = scale_oracle(args.workload, s)
        vals.append(step_s)
    value = 4.0 * len(vals) / sum(vals)
    wl = W.BENCH_WORKLOADS[args.workload]
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 5), "unit": UNIT,
            "n_gpus": int(os.environ.get("WORLD_SIZE", 1)), "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(1000 * sum(vals) / len(vals), 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic: seeded quenched U(1) Metropolis configuration, Gaussian source",
            "config": {"workload": args.workload, "lattice": [wl["Lx"], wl["Lt"]],
                       "levels": len(wl["blocks"]) + 1, "Nv": wl["Nv"], "solves_per_step": 4},
            "cpu_baseline": {"value": round(value, 5), "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": (f"per step: setup at m_nc, {args.oracle_iters} MG-CG iterations "
                                        f"at m_nc, re-mass + solve at m=0.1; scaled to the 4-mass "
                                        f"step with the oracle's iteration counts (m_nc: {n_nc})"),
                             "sample_wall_s_per_step": round(sum(walls) / len(walls), 1)},
            "e2e": {"value": round(value, 5), "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def ncu_case(args):
    """Small cases for kernel-level ncu captures (a few launches of one kernel):
    stencil -- fused FP32 A on a 2048 x 2048 lattice (about 200 MB per launch,
               above L2); coarse -- BF16 coarse apply on level 2 of the
               benchmark workload, one right-hand side; coarse_mma -- the same
               with 64 right-hand sides (tensor cores); coarsest -- the
               coarsest solve (packed FP32 GEMV + FP64 refinement) of the
               benchmark workload; vcycle -- one FP32 V-cycle; setup -- the
               set-up of the benchmark workload alone (its Gauss-Jordan
               inverse of the 4096-unknown coarsest operator included)."""
    import torch
    from paper_0710_3612_gb300 import mg
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    if args.ncu_case == "stencil":
        L = 2048
        U = torch.polar(torch.ones(2, L, L, dtype=torch.float64, device=dev),
                        torch.rand(2, L, L, dtype=torch.float64, device=dev)).contiguous()
        h = mg.mg_setup(U, 0.1, mg.make_params(L, L, [], []), stream)
        x = torch.randn(L * L * 2, dtype=torch.complex64, device=dev)
        y = torch.empty_like(x)
        for _ in range(4):
            mg.mg_apply_A(h, x, y, 1, mg.PREC_F32)
    else:
        wl, crit, U, noise, chi, masses = workload_inputs(args.workload)
        nd = torch.from_numpy(noise).to(dev)
        h = mg.mg_setup(torch.from_numpy(U).to(dev), masses[0],
                        mg.make_params(wl["Lx"], wl["Lt"], wl["blocks"], wl["Nv"], nd,
                                       setup_sweeps=wl["setup_sweeps"],
                                       coarsest_gj_tcgen05=int(args.gj_tcgen05)), stream)
        if args.ncu_case in ("coarse", "coarse_mma"):
            nrhs = 64 if args.ncu_case == "coarse_mma" else 1
            Lx, Lt, n, _ = mg.mg_get_level(h, 2)
            x = torch.randn(nrhs * Lx * Lt * n, dtype=torch.complex64, device=dev)
            y = torch.empty_like(x)
            for _ in range(4):
                mg.mg_apply_coarse(h, 2, x, y, nrhs, mg.PREC_BF16)
        elif args.ncu_case == "setup":
            pass
        elif args.ncu_case == "coarsest":
            Lx, Lt, n, _ = mg.mg_get_level(h, len(wl["blocks"]) + 1)
            x = torch.randn(Lx * Lt * n, dtype=torch.complex128, device=dev)
            y = torch.empty_like(x)
            for _ in range(4):
                mg.mg_coarsest_solve(h, x, y)
        else:
            x = torch.randn(wl["Lx"] * wl["Lt"] * 2, dtype=torch.complex64, device=dev)
            y = torch.empty_like(x)
            for _ in range(4):
                mg.mg_vcycle(h, x, y, mg.PREC_F32)
    torch.cuda.synchronize()
    mg.mg_destroy(h)
    print(json.dumps({"ncu_case": args.ncu_case, "ok": True}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--coarsest-reuse", type=int, default=12,
                    help="mg_params.coarsest_reuse of the mass-sweep step (0: invert at every mass)")
    ap.add_argument("--solver", default="mixed", choices=list(SOLVER_CODES),
                    help="mixed-precision MG-CG variant of every leg")
    ap.add_argument("--workload", default="L128_b6_massweep", choices=list(W.BENCH_WORKLOADS))
    ap.add_argument("--plain-steps", type=int, default=3)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--oracle-iters", type=int, default=20)
    ap.add_argument("--batch-rhs", type=int, default=64,
                    help="right-hand sides of the batched leg (0 skips it)")
    ap.add_argument("--batch-reps", type=int, default=3)
    ap.add_argument("--config-legs", default="L256_b10_nc64,L1024_b10_nc16_l5",
                    help="batched workloads at their near-critical mass ('' skips them)")
    ap.add_argument("--config-reps", type=int, default=3)
    ap.add_argument("--smoothed-leg", type=int, default=1, help="1: run the smoothed-aggregation leg")
    ap.add_argument("--plain-iter-cap", type=int, default=400,
                    help="iteration cap of the plain FP64 single-RHS solve of the batched workloads")
    ap.add_argument("--adaptive-plan", default="112222",
                    help="levels refined by the adaptive passes of the adaptive leg ('' skips it)")
    ap.add_argument("--adaptive-cycles", type=int, default=30)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-all-cores", type=int, default=1,
                    help="1: also time the oracle sample on every host core at once")
    ap.add_argument("--serve-requests", type=int, default=48,
                    help="requests per point of the serving leg (0 skips the serving leg)")
    ap.add_argument("--serve-loads", default="0.3",
                    help="Poisson points of the serving leg, as fractions of the measured capacity")
    ap.add_argument("--serving-only", action="store_true",
                    help="run the serving leg alone and print it as the JSON line")
    ap.add_argument("--serve-budget-gb", type=int, default=128)
    ap.add_argument("--timed-only", action="store_true",
                    help="skip the plain-FP64, roofline, stencil and end-to-end legs (profiling runs)")
    ap.add_argument("--gj-tcgen05", action="store_true",
                    help="with --ncu-case: coarsest inverse updates on tcgen05 tensor cores")
    ap.add_argument("--phase-launches", action="store_true",
                    help="with --timed-only: library kernel launches counted at the end of each "
                         "phase (setup, re-mass, solve) of the first timed step")
    ap.add_argument("--ncu-case", choices=["stencil", "coarse", "coarse_mma", "coarsest", "vcycle",
                                           "setup"],
                    help="run a small kernel case for an ncu capture and exit")
    args = ap.parse_args()
    global MIXED_SOLVER
    MIXED_SOLVER = SOLVER_CODES[args.solver]
    if args.ncu_case:
        ncu_case(args)
    elif args.impl == "reference":
        reference_arm(args)
    else:
        gpu_bench(args)


if __name__ == "__main__":
    main()
