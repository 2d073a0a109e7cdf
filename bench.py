"""Benchmark of one particle-in-cell field step: cloud-in-cell deposit onto
every level -> AMR multigrid V-cycles to relative residual 1e-10 -> E
gathered to the particles, FP64, by default on the five-bunch workload:
base 128^3 with two density-tagged refinement levels (rho > 0.1 max) and
10^7 particles in five Gaussian bunches (sigma 0.04, 0.15 apart along x).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Beside the FP64 step it reports the
mixed-precision form on the same workload (its error against the FP64
result of every timed step, and against the oracle), the 256^3 + 3 levels
roofline instance, per-kernel device times from a profiled copy of the
solve graph, and the oracle timed on the host cores.  With N > 1
(torchrun) every rank solves its own seeded replica of the workload (no
collective on the data path) and the value is the total solves/s over all
ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "V-cycle HBM GB/s + solves/s to 1e-10 residual; served p50/p99 solve latency"
WORKLOAD = "c3_bunches"
FALLBACK_HBM_GBS = 6800.0
# FP64 arithmetic peak from unit counts and clock: 152 SMs x 2 FP64 FMA
# lanes per SM per clock x 2 flops x 2.07 GHz; the FP64 rooflines divide by
# the rate amr_probe_fp64_fma measures in the same run (about 529 G FMA/s)
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
EPS = 1e-10


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--bottom-cycles", type=int, default=2)
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--robin-d", type=float, default=None,
                    help="Robin domain faces d phi/dn + phi/d = 0 with this d (default: Dirichlet)")
    ap.add_argument("--periodic", action="store_true", help="periodic domain faces (default: Dirichlet)")
    ap.add_argument("--form", default="step", choices=["step", "batched", "served", "pic", "sphere"],
                    help="step: one deposit/solve/gather step; batched: many hierarchies per launch")
    ap.add_argument("--batch", type=int, default=256)
    ap.add_argument("--pic-particles", type=int, default=1_000_000, help="pic: particles of the five bunches")
    ap.add_argument("--pic-n0", type=int, default=64, help="pic: base grid")
    ap.add_argument("--requests", type=int, default=2000, help="served: requests taken from the stream")
    ap.add_argument("--sequential-prefix", type=int, default=100,
                    help="served: requests of the prefix also solved one at a time")
    ap.add_argument("--slots", type=int, default=16, help="served: concurrent slots")
    ap.add_argument("--budget-gb", type=float, default=150.0, help="served: HBM budget")
    ap.add_argument("--max-n0", type=int, default=256, help="served: cap of the base grid")
    ap.add_argument("--max-particles", type=float, default=1e7, help="served: cap of the particle count")
    ap.add_argument("--mode", default="graph", choices=["graph", "persistent", "eager"],
                    help="solve as one captured graph, one persistent kernel, or host-driven launches")
    ap.add_argument("--no-mixed", action="store_true", help="skip the mixed-precision form of the step")
    ap.add_argument("--no-roofline-instance", action="store_true", help="skip the 256^3 + 3 levels instance")
    ap.add_argument("--launch-list", action="store_true",
                    help="only hierarchy creation, W warm-up and K timed steps (for a profiler's launch list)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def job_rate(local_s, units_per_rank, world, device="cuda"):
    """Whole-job throughput of `world` ranks that each processed
    units_per_rank units in local_s seconds: all ranks' units over the
    slowest rank's time (the maximum over ranks, one all-reduce).  Returns
    (units per second, the slowest time in seconds)."""
    t = float(local_s)
    if world > 1:
        import torch
        import torch.distributed as dist
        x = torch.tensor([t], dtype=torch.float64, device=device)
        dist.all_reduce(x, op=dist.ReduceOp.MAX)
        t = float(x.item())
    return world * units_per_rank / t, t


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            return json.load(open(p)), "measured"
        except Exception:
            pass
    return None, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        self.f.flush()
        rows = []
        for line in open(self.f.name):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


class OracleSample:
    """The oracle (plain FP64 C, OpenMP over independent loops) on a bounded
    sample of the workload: each sample step deposits every particle, runs
    ONE V-cycle of Alg. 2 from the previous step's potential (warm start;
    Alg. 1 residuals, average-down and E come with it) and gathers E to every
    particle.  Per solve: t_deposit + V t_vcycle + t_gather, with V the number
    of V-cycles the oracle needs to reach the stopping tolerance on this
    workload (counted over the sample steps: their V-cycles continue one
    solve)."""

    def __init__(self, w, parts, robin_d=None, periodic=False):
        import oracle
        self.cores = oracle.set_threads()
        t0 = time.perf_counter()
        self.O = oracle.OracleHierarchy(w.n0, w.lmax, particles=parts, tag_mode=w.tag_mode,
                                        tag_lambda=w.tag_lambda, boxes=w.boxes or None, robin_d=robin_d or 0.0,
                                        periodic=periodic)
        self.create_s = time.perf_counter() - t0
        self.parts = parts
        self.t = {"deposit": [], "vcycle": [], "gather": []}
        self.cycles = 0
        self.converged_at = None
        self.rel = None

    def step(self):
        O, parts = self.O, self.parts
        t0 = time.perf_counter()
        O.deposit(*parts)
        t1 = time.perf_counter()
        it, rel = O.solve(eps=EPS, max_iter=1, bottom_rtol=1e-12, warm=self.cycles > 0)
        t2 = time.perf_counter()
        O.gather(*parts[:3])
        t3 = time.perf_counter()
        self.cycles += it
        self.rel = rel
        if self.converged_at is None and float(np.max(rel)) <= EPS:
            self.converged_at = self.cycles
        self.t["deposit"].append(t1 - t0)
        self.t["vcycle"].append(t2 - t1)
        self.t["gather"].append(t3 - t2)
        return t3 - t0

    def per_solve_s(self, vcycles):
        m = {k: statistics.mean(v) for k, v in self.t.items()}
        return m["deposit"] + vcycles * m["vcycle"] + m["gather"], m

    def report(self, w, vcycles, source):
        sec, m = self.per_solve_s(vcycles)
        return {"value": 1.0 / sec, "unit": "solves/s", "cores": self.cores, "kind": "oracle",
                "sample": (f"{len(self.t['vcycle'])} sample step(s) of {w.name}, each: deposit of all "
                           f"{len(self.parts[0])} particles (serial, particle order) + ONE V-cycle (warm start) "
                           f"+ gather to all particles; per solve = deposit {m['deposit']:.3f} s + {vcycles} "
                           f"V-cycles x {m['vcycle']:.3f} s ({source}) + gather {m['gather']:.3f} s; hierarchy "
                           f"creation ({self.create_s:.2f} s) excluded"),
                "oracle_vcycles_done": self.cycles, "oracle_rel_res": [float(x) for x in self.rel]}


def run_reference(args, rank, world):
    """The oracle timed on this host's cores on the same workload, metric and
    unit; each step is one bounded sample step (see OracleSample)."""
    if rank != 0:
        return
    from paper_1812_03689_gb300 import inputs
    w = inputs.workload(args.workload)
    parts = w.particles()
    S = OracleSample(w, parts, robin_d=args.robin_d, periodic=args.periodic)
    for _ in range(args.warmup):
        S.step()
    for k in S.t:
        S.t[k].clear()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        S.step()
    dt = time.perf_counter() - t0
    if S.converged_at is not None:
        vc, src = S.converged_at, "the oracle's own count to 1e-10 over these steps"
    else:
        vc, src = S.cycles, f"a lower bound: {S.cycles} V-cycles done without reaching 1e-10"
    cb = S.report(w, vc, src)
    v = cb["value"]
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / v,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "n0": w.n0, "max_level": w.lmax, "particles": w.n_particles,
                   "bc": bc_name(args)},
        "cpu_baseline": cb,
        "sample_wall_s": dt,
        "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def bc_name(args):
    if args.periodic:
        return "periodic"
    return "dirichlet" if args.robin_d is None else f"robin d={args.robin_d:g}"


def run_batched(args, rank, world, local):
    """Batched form: independent uneven hierarchies solved to 1e-10 by ONE
    graph launch per batch (amr_batch_solve; the library's default batch
    holds every hierarchy's solve as an independent branch of one captured
    graph), against the same hierarchies solved one after another (one
    captured graph each), the persistent cluster program and the
    lock-step-rounds program (both also one launch per batch), and the
    concurrent graphs of amr_solve_many."""
    import torch
    from paper_1812_03689_gb300 import amrmg, inputs
    torch.cuda.set_device(local)
    reqs = inputs.batched_requests(args.batch)
    t0 = time.perf_counter()
    hs = []
    for r in reqs:
        parts = [torch.from_numpy(a).cuda() for a in r.particles(3)]
        hs.append(amrmg.Hierarchy(r.n0, r.lmax, particles=parts, precision=args.precision))
    create_s = time.perf_counter() - t0
    opts = dict(eps=EPS, bottom_cycles=args.bottom_cycles)
    stream = torch.cuda.current_stream()

    def timed(fn, steps):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        ms = []
        for _ in range(steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        return statistics.median(ms)

    def phis():
        return [h.get(h.nlevels - 1, "phi") for h in hs[:16]]

    # one at a time, one graph each (the reference for every other form)
    ts = timed(lambda: [h.solve(**opts) for h in hs], max(1, args.steps // 2))
    phi_s = phis()
    forms = {}
    for mode in ("graphs", "clusters", "rounds"):
        os.environ["AMR_BATCH"] = mode
        B = amrmg.Batch(hs, **opts)
        os.environ.pop("AMR_BATCH", None)
        launches0 = sum(h.kernel_launches() for h in hs)
        holder = {}
        tb = timed(lambda: holder.__setitem__("st", B.solve()), args.steps)
        launches = (sum(h.kernel_launches() for h in hs) - launches0) / (args.steps + args.warmup)
        same = all(np.array_equal(a, b) for a, b in zip(phis(), phi_s))
        st = holder["st"]
        forms[mode] = {"value": len(hs) / (tb / 1e3), "unit": "solves/s", "ms": tb,
                       "speedup_vs_sequential": ts / tb, "bitwise_equal_to_sequential": same,
                       "gpu_launches_per_batch": launches,
                       "iters": {"min": min(x["iters"] for x in st), "max": max(x["iters"] for x in st),
                                 "mean": statistics.mean(x["iters"] for x in st)},
                       "max_rel_res": max(float(x["rel_res"].max()) for x in st)}
        B.close()
    # the same hierarchies side by side: their graphs on 16 streams
    amrmg.solve_many(hs, n_streams=16, **opts)
    torch.cuda.synchronize()
    ms_c = []
    for _ in range(max(1, args.steps // 2)):
        t0c = time.perf_counter()
        amrmg.solve_many(hs, n_streams=16, **opts)
        ms_c.append(1e3 * (time.perf_counter() - t0c))
    same_c = all(np.array_equal(a, b) for a, b in zip(phis(), phi_s))
    tc = statistics.median(ms_c)
    g = forms["graphs"]
    out = {
        "metric": "batched solves/s to 1e-10 residual (one graph launch per batch)",
        "value": g["value"], "unit": "solves/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": g["ms"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32+f64", "data": "synthetic",
        "config": {"workload": "batched_uneven", "hierarchies": len(hs), "precision": args.precision,
                   "n0_range": [min(r.n0 for r in reqs), max(r.n0 for r in reqs)],
                   "levels": [sum(1 for h in hs if h.nlevels == k) for k in (1, 2, 3)],
                   "particles_range": [min(r.n_particles for r in reqs), max(r.n_particles for r in reqs)],
                   "creation_s": create_s},
        "gpu_launches": g["gpu_launches_per_batch"],
        "speedup_vs_sequential": g["speedup_vs_sequential"],
        "bitwise_equal_to_sequential": g["bitwise_equal_to_sequential"],
        "sequential_graph": {"value": len(hs) / (ts / 1e3), "unit": "solves/s", "ms": ts},
        "forms": forms,
        "concurrent_graphs": {"value": len(hs) / (tc / 1e3), "unit": "solves/s", "ms": tc, "streams": 16,
                              "timing": "host wall clock around amr_solve_many (returns when all are done)",
                              "bitwise_equal_to_sequential": same_c},
    }
    print(json.dumps(out), flush=True)


def run_pic(args, rank, world, local):
    """Multi-step form (the paper's neighbouring-bunch runs, Sec. 6.3): five
    Gaussian bunches in particle space (spacing 1, sigma 0.267 of it, as the
    5-bunch workload in the cube), each step maps them into the cube
    (delta = 20 %), deposits, solves to 1e-10, rescales phi and E to particle
    space, gathers and pushes (kick-drift); the hierarchy is regridded by
    density every 10 steps (amr_regrid_boxes, new hierarchy, warm start)."""
    import torch
    from paper_1812_03689_gb300 import amrmg
    torch.cuda.set_device(local)
    nb, npb = 5, args.pic_particles // 5
    g = np.random.default_rng(1812036890 + 7)
    pos_h = [np.concatenate([g.normal(c, 0.267, npb) for c in (-2.0, -1.0, 0.0, 1.0, 2.0)])]
    pos_h += [g.normal(0.0, 0.267, nb * npb) for _ in range(2)]
    n = nb * npb
    pos = [torch.from_numpy(a).cuda() for a in pos_h]
    mom = [torch.zeros(n, dtype=torch.float64, device="cuda") for _ in range(3)]
    q = torch.full((n,), 1.0 / n, dtype=torch.float64, device="cuda")
    qm, dt = 40.0, 0.02
    state = {"H": None, "k": 0}
    opts = dict(eps=EPS, bottom_cycles=args.bottom_cycles)

    def step():
        u, v, w, S = amrmg.domain_transform(*pos, delta=0.2)
        H = state["H"]
        if H is None:
            H = amrmg.Hierarchy(args.pic_n0, 2, particles=(u, v, w, q), tag_mode="rel", tag_lambda=0.1,
                                precision=args.precision)
        elif state["k"] % 10 == 0:
            N = amrmg.Hierarchy(args.pic_n0, 2, boxes=H.regrid_boxes("rel", 0.1, 2), precision=args.precision)
            N.transfer_phi_from(H)
            H = N
        state["H"] = H
        state["k"] += 1
        H.deposit(u, v, w, q)
        st = H.solve(**opts)
        H.rescale_fields(S)
        E = H.gather(u, v, w)
        amrmg.push(pos, mom, E, qm, dt)
        return st

    centre = slice(2 * npb, 3 * npb)
    m0 = amrmg.moments(*[t[centre].contiguous() for t in pos])
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    iters = []
    for _ in range(args.steps):
        iters.append(step()["iters"])
    torch.cuda.synchronize()
    dt_s = time.perf_counter() - t0
    m1 = amrmg.moments(*[t[centre].contiguous() for t in pos])
    H = state["H"]
    out = {
        "metric": "PIC steps/s (transform, deposit, solve to 1e-10, rescale, gather, push; regrid every 10)",
        "value": args.steps / dt_s, "unit": "steps/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * dt_s / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.precision == "fp64" else "f32+f64", "data": "synthetic",
        "config": {"workload": "five_bunches", "particles": n, "n0": args.pic_n0, "max_level": 2,
                   "levels": H.nlevels, "valid_cells": [H.level_box(l)[2] for l in range(H.nlevels)],
                   "q_over_m": qm, "dt": dt, "delta": 0.2, "regrid_every": 10, "precision": args.precision},
        "iters_per_solve": statistics.mean(iters),
        "centre_bunch": {"sigma_start": m0["sigma"].tolist(), "sigma_end": m1["sigma"].tolist(),
                         "xi_start": m0["xi"].tolist(), "xi_end": m1["xi"].tolist()},
        "timing": "host wall clock around the steps, synchronised on both sides (the step reads the transform "
                  "scale and the regrid boxes on the host)",
    }
    print(json.dumps(out), flush=True)


def run_sphere(args, rank, world, local):
    """The paper's uniformly charged sphere (Sec. 6.2: R = 0.2, Q = 1,
    centred in the unit cube, base 32^3 with one refined level on the
    central 16^3 coarse cells) with Robin domain faces over a sweep of the
    distance d (Eq. robin_bc) and with homogeneous Dirichlet faces: the error
    of phi against the free-space closed form, GPU and oracle on the same
    density, and their difference."""
    import torch
    import oracle
    from paper_1812_03689_gb300 import amrmg, inputs
    torch.cuda.set_device(local)
    oracle.set_threads()
    w = inputs.workload("c1_small")
    R = 0.2
    rows = []
    for d in [None, 0.05, 0.1, 0.25, 0.5, 0.85, 1.7, 5.0]:
        G = amrmg.Hierarchy(w.n0, w.lmax, boxes=w.boxes, robin_d=d)
        O = oracle.OracleHierarchy(w.n0, w.lmax, boxes=w.boxes, robin_d=d or 0.0)
        rhos = []
        for l in range(G.nlevels):
            lo, hi, _ = G.level_box(l)
            rho = inputs.sphere_density(lo, hi, G.h(l), radius=R) * (G.mask(l) > 0)
            G.set(l, "rho", rho)
            O.set(l, "rho", rho)
            rhos.append(rho)
        t0 = time.perf_counter()
        st = G.solve(eps=1e-12)
        gpu_ms = 1e3 * (time.perf_counter() - t0)
        O.solve(eps=1e-12, bottom_rtol=1e-14)
        err, diff = [], []
        for l in range(G.nlevels):
            X, Y, Z = O.centres(l)
            r = np.sqrt((X - 0.5) ** 2 + (Y - 0.5) ** 2 + (Z - 0.5) ** 2)
            exact = np.where(r > R, 1 / (4 * np.pi * r), (3 - r * r / (R * R)) / (8 * np.pi * R))
            m = G.mask(l) > 0
            g, o = G.get(l, "phi"), O.get(l, "phi")
            err.append(float(np.abs(g - exact)[m].max() / exact[m].max()))
            diff.append(float(np.linalg.norm((g - o)[m]) / np.linalg.norm(o[m])))
        rows.append({"bc": "dirichlet" if d is None else "robin", "d": d, "iters": st["iters"],
                     "max_rel_error_vs_closed_form": err, "gpu_vs_oracle_phi_rel_l2": diff,
                     "gpu_solve_ms": gpu_ms})
        G.close()
    best = min((r for r in rows if r["d"] is not None), key=lambda r: max(r["max_rel_error_vs_closed_form"]))
    out = {"metric": "uniformly charged sphere: max |phi - closed form| / max phi per level, Robin d sweep",
           "value": max(best["max_rel_error_vs_closed_form"]), "unit": "relative error", "n_gpus": 1,
           "steps": len(rows), "warmup": 0, "ms_per_step": statistics.mean(r["gpu_solve_ms"] for r in rows),
           "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": "sphere_robin_sweep", "n0": w.n0, "max_level": w.lmax, "radius": R,
                      "refined_box": "central 16^3 coarse cells", "eps": 1e-12,
                      "density": "cell volume fraction (8^3 samples) x 3Q / (4 pi R^3)"},
           "best_d": best["d"], "rows": rows}
    print(json.dumps(out), flush=True)


def run_served(args, rank, world, local):
    """Served form: a Poisson stream of uneven requests through the
    continuous-batching loop (admission by HBM budget, overlapping slots), at
    the workload's arrival rate (2000/s, faster than the loop serves them:
    the latency then includes the backlog) and again, with the same requests,
    at half the measured service rate (the latency is then the service
    time); a prefix of the requests also one at a time (one slot)."""
    import torch
    from paper_1812_03689_gb300 import amrmg, inputs
    torch.cuda.set_device(local)
    rate = 2000.0
    stream_reqs = inputs.served_requests(10_000, rate, max_n0=args.max_n0, max_particles=args.max_particles)
    sample = stream_reqs[:args.requests]
    budget = int(args.budget_gb * (1 << 30))
    opts = dict(eps=EPS, bottom_cycles=args.bottom_cycles)

    def make(scale):
        return [amrmg.make_request(r.n0, r.lmax, r.n_particles, r.sigma, seed=1812036890 + r.index,
                                   arrival_s=r.arrival_s * scale, precision=args.precision) for r in sample]

    def stats(res):
        ok = [r for r in res if r["status"] in (0, 3)]
        lat = np.array([r["done_s"] - r["arrival_s"] for r in ok])
        span = max(r["done_s"] for r in res) - min(r["arrival_s"] for r in res)
        return ok, lat, span

    warm = make(1.0)[:4]
    amrmg.serve(warm, budget, args.slots, realtime=False, **opts)  # warm-up (allocator, caches)
    t0 = time.perf_counter()
    res = amrmg.serve(make(1.0), budget, args.slots, realtime=True, **opts)
    wall1 = time.perf_counter() - t0
    ok, lat, span = stats(res)
    served_rate = len(ok) / span
    low_rate = 0.5 * served_rate
    print(json.dumps({"progress": "arrivals at 2000/s done", "solves_per_s": served_rate, "wall_s": wall1,
                      "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
                      "refused": sum(1 for r in res if r["status"] == 2)}), file=sys.stderr, flush=True)
    t0 = time.perf_counter()
    res2 = amrmg.serve(make(rate / low_rate), budget, args.slots, realtime=True, **opts)
    wall2 = time.perf_counter() - t0
    ok2, lat2, span2 = stats(res2)
    print(json.dumps({"progress": "arrivals below the service rate done", "wall_s": wall2}), file=sys.stderr,
          flush=True)
    nseq = min(len(sample), args.sequential_prefix)
    seq = amrmg.serve(make(1.0)[:nseq], budget, 1, realtime=False, **opts)
    seq_span = max(r["done_s"] for r in seq)
    # the mix's requests against the same requests alone (one slot):
    # checksums of the gathered field, relative to the largest
    diffs = [float(np.abs(a["checksum"] - b["checksum"]).max() / max(np.abs(b["checksum"]).max(), 1e-300))
             for a, b in zip(res[:nseq], seq) if a["status"] == 0 and b["status"] == 0]
    over = [r["device_bytes"] for r in res if r["status"] == 0]
    out = {
        "metric": "served solves/s and p50/p99 latency (continuous batching, Poisson arrivals)",
        "value": served_rate, "unit": "solves/s", "n_gpus": 1, "steps": len(sample), "warmup": len(warm),
        "ms_per_step": 1e3 * span / max(len(ok), 1), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32+f64", "data": "synthetic",
        "config": {"workload": "served_poisson", "requests": len(sample), "of_stream": 10_000,
                   "rate_per_s": rate, "n0_cap": args.max_n0, "particles_cap": args.max_particles,
                   "slots": args.slots, "budget_gb": args.budget_gb, "precision": args.precision,
                   "levels": "0-3", "n0_range": [min(r.n0 for r in sample), max(r.n0 for r in sample)],
                   "particles_range": [min(r.n_particles for r in sample), max(r.n_particles for r in sample)]},
        "latency_s": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                      "max": float(lat.max()), "note": "arrivals at 2000/s outpace the loop: backlog included"},
        "wall_s": wall1,
        "below_service_rate": {"rate_per_s": low_rate, "value": len(ok2) / span2, "unit": "solves/s",
                               "latency_s": {"p50": float(np.percentile(lat2, 50)),
                                             "p99": float(np.percentile(lat2, 99)), "max": float(lat2.max())},
                               "wall_s": wall2,
                               "note": "the same requests, arrival times stretched to half the measured service "
                                       "rate: the latency is the service time of a request among the others"},
        "one_at_a_time": {"requests": nseq, "value": nseq / seq_span, "unit": "solves/s",
                          "vs_same_prefix_served": None},
        "refused": sum(1 for r in res if r["status"] == 2),
        "failed": sum(1 for r in res if r["status"] not in (0, 2, 3)),
        "max_rel_res": max(r["rel_res_max"] for r in ok),
        "max_checksum_rel_diff_vs_alone": max(diffs) if diffs else None,
        "device_gb": {"max_request": max(over) / 2 ** 30 if over else None,
                      "mean_request": float(np.mean(over)) / 2 ** 30 if over else None},
    }
    print(json.dumps(out), flush=True)


class StepRunner:
    """One hierarchy of a workload and its deposit -> solve -> gather step."""

    def __init__(self, amrmg, w, dev, precision, args, stream):
        import torch
        self.amrmg, self.dev, self.stream = amrmg, dev, stream
        self.n = dev[0].numel()
        t0 = time.perf_counter()
        self.H = amrmg.Hierarchy(w.n0, w.lmax, particles=dev, tag_mode=w.tag_mode, tag_lambda=w.tag_lambda,
                                 boxes=w.boxes or None, stream=stream, precision=precision,
                                 robin_d=args.robin_d, periodic=args.periodic)
        self.create_s = time.perf_counter() - t0
        self.E = [torch.empty(self.n, dtype=torch.float64, device="cuda") for _ in range(3)]
        self.opts = dict(eps=EPS, bottom_cycles=args.bottom_cycles, use_graph=args.mode == "graph",
                         persistent=args.mode == "persistent")
        self.ops = {}

    def step(self):
        a = self.amrmg
        H = self.H
        H.deposit(*self.dev)
        st = H.solve(**self.opts)
        a._check(a._lib.amr_gather(H._h, *[a._dev(t, "p") for t in self.dev[:3]], self.n,
                                   *[a._dev(t, "e") for t in self.E], None))
        return st

    def timed(self, steps, warmup, flush, after=None):
        """Warm-up steps, then `steps` timed steps (CUDA events on the
        hierarchy's stream, L2 flushed before each, outside the events);
        after(k) runs after timed step k, outside the timed region."""
        import torch
        for _ in range(warmup):
            self.step()
        torch.cuda.synchronize()
        ms, iters = [], []
        for k in range(steps):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(self.stream)
            st = self.step()
            e1.record(self.stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
            iters.append(st["iters"])
            if after:
                after(k)
        torch.cuda.synchronize()
        return ms, iters

    def levels(self, field="phi"):
        return [self.H.get(l, field) for l in range(self.H.nlevels)]


def rel_l2(a, b):
    na = float(np.sqrt(sum(float(np.sum((x - y) ** 2)) for x, y in zip(a, b))))
    nb = float(np.sqrt(sum(float(np.sum(y ** 2)) for y in b)))
    return na / nb if nb > 0 else na


def kernel_profile(R, steps, flush, mode):
    """Per-kind device times of `steps` more steps with the library's
    per-launch timers: mode "graph" times the kernels of a profiled copy of
    the solve graph (same kernels and grouped launches, unrolled to the timed
    V-cycle count, event-record nodes around each kernel node)."""
    import torch
    R.H.profile(True, mode=mode)
    for _ in range(steps):
        flush.fill_(1.0)
        R.step()
    torch.cuda.synchronize()
    prof = R.H.profile_read()
    R.ops = R.H.profile_read_ops()
    R.H.profile(False)
    return prof


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.form == "batched":
        return run_batched(args, rank, world, local)
    if args.form == "served":
        return run_served(args, rank, world, local)
    if args.form == "pic":
        return run_pic(args, rank, world, local)
    if args.form == "sphere":
        return run_sphere(args, rank, world, local)
    import torch
    from paper_1812_03689_gb300 import amrmg, inputs

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    w = inputs.workload(args.workload)
    parts_host = w.particles(request_index=rank)
    n = len(parts_host[0])
    dev = [torch.from_numpy(a).cuda() for a in parts_host]
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")  # 512 MB > L2
    R = StepRunner(amrmg, w, dev, args.precision, args, stream)
    H = R.H
    # the FP64 FMA rate of this device now (the FP64 roofline's denominator):
    # best of three probe launches of ~60 ms
    fp64 = None
    if not args.launch_list:
        with ClockSampler(local) as pclk:
            rates = [amrmg.probe_fp64_fma(16384, stream=stream) for _ in range(5)]
        g = max(r[0] for r in rates)
        pc = pclk.summary()
        sms = torch.cuda.get_device_properties(local).multi_processor_count
        fp64 = {"gfma_per_s": g, "tflops": 2.0 * g / 1e3, "ms": [r[1] for r in rates],
                "probe": "amr_probe_fp64_fma: 8 independent FMA chains per thread, every resident block",
                "clocks": pc, "sms": sms,
                "fma_per_sm_per_clock": (g * 1e9 / (sms * pc["sm_mhz"] * 1e6)) if pc.get("sm_mhz") else None}
    if args.launch_list:
        ms, _ = R.timed(args.steps, args.warmup, flush)
        if rank == 0:
            print(json.dumps({"launch_list_run": w.name, "ms_per_step": statistics.mean(ms)}), flush=True)
        return
    for _ in range(args.warmup):
        R.step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    launches0 = H.kernel_launches()
    with ClockSampler(local) as clocks:
        ms_steps, iters = R.timed(args.steps, 0, flush)
    launches = H.kernel_launches() - launches0
    value, slow_s = job_rate(sum(ms_steps) / 1e3, args.steps, world)
    total_ms = 1e3 * slow_s
    E64 = [t.clone() for t in R.E]
    phi64 = R.levels() if rank == 0 else None

    # per-kernel device times from a profiled copy of the step
    prof_mode = "graph" if args.mode == "graph" else "eager"
    prof = kernel_profile(R, args.steps, flush, prof_mode)

    # end to end through the C ABI with host buffers (pinned), copies timed
    pin = [torch.from_numpy(a).pin_memory() for a in parts_host]
    pout = [torch.empty(n, dtype=torch.float64).pin_memory() for _ in range(3)]
    o = amrmg.solve_opts(**R.opts)
    ptrs = [ctypes_ptr(t) for t in pin]
    optrs = [ctypes_ptr(t) for t in pout]
    for _ in range(3):
        H.step_ptrs(*ptrs, n, *optrs, o)
    torch.cuda.synchronize()
    # at least 20 steps: a single host-side stall of a few ten ms weighs
    # less in the mean (every step's time is reported too)
    e2e_steps = max(args.steps, 20)
    t0 = time.perf_counter()
    e2e_ms = []
    for _ in range(e2e_steps):
        t1 = time.perf_counter()
        H.step_ptrs(*ptrs, n, *optrs, o)
        e2e_ms.append(1e3 * (time.perf_counter() - t1))
    e2e_s = time.perf_counter() - t0
    e2e_value, _ = job_rate(e2e_s, e2e_steps, world)

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    peaks, peak_src = measured_peaks()
    hbm_peak = float(peaks.get("hbm_gbs", FALLBACK_HBM_GBS)) if peaks else FALLBACK_HBM_GBS
    dom_name, (dom_ms, dom_n, dom_bytes, dom_flops) = max(prof.items(), key=lambda kv: kv[1][0])
    total_prof_ms = sum(v[0] for v in prof.values())
    vcycle_kinds = ("rbgs", "residual", "restrict", "prolong", "finish", "cf_correct", "flux", "norms",
                    "mg_restrict", "mg_prolong", "coarse_solve", "elementwise", "coarse_part", "check",
                    "sine_transform", "tridiagonal")
    vc_ms = sum(prof[k][0] for k in vcycle_kinds if k in prof)
    vc_bytes = sum(prof[k][2] for k in vcycle_kinds if k in prof)
    # DRAM bytes per launch of the dominant kernel from one ncu capture of
    # this workload (profiles/traffic_<kernel>_<workload>[_mixed].md, line
    # "bytes_per_launch: N"), else null
    traffic = None
    suffix = "" if args.precision == "fp64" else "_mixed"
    tfile = os.path.join(ROOT, "profiles", f"traffic_{dom_name}_{w.name}{suffix}.md")
    if os.path.exists(tfile):
        for line in open(tfile):
            if line.strip().startswith("bytes_per_launch:"):
                try:
                    traffic = float(line.split(":", 1)[1])
                except ValueError:
                    traffic = None
    out = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32+f64",
        "data": "synthetic",
        "config": {"workload": w.name, "precision": args.precision, "n0": w.n0, "max_level": w.lmax,
                   "bc": bc_name(args), "levels": H.nlevels,
                   "valid_cells": [H.level_box(l)[2] for l in range(H.nlevels)], "particles": n,
                   "eps": EPS, "smoother": "RB-GS 2+2", "bottom": ("exact: sine transforms x, y + tridiagonal z" if H.bottom_solver() == "exact"
                              else f"GMG {args.bottom_cycles} cycles"), "mode": args.mode,
                   "l2": "flushed between timed steps (512 MB write)",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "iters_per_solve": statistics.mean(iters),
        "gpu_launches": launches,
        "roofline": roofline(args.precision, dom_name, dom_ms, dom_n, dom_bytes, dom_flops, hbm_peak, peak_src,
                             traffic, total_prof_ms, fp64, R.ops.get(dom_name, 0.0)),
        "fp64_peak": fp64,
        "vcycle": {"alg_gbs": vc_bytes / (vc_ms / 1e3) / 1e9 if vc_ms else None, "ms_per_solve": vc_ms / args.steps},
        "kernels": {k: {"ms": v[0], "launches": v[1], "alg_gbs": v[2] / (v[0] / 1e3) / 1e9 if v[0] else None,
                        **({"alg_tflops": v[3] / (v[0] / 1e3) / 1e12} if v[3] and v[0] else {})}
                    for k, v in sorted(prof.items(), key=lambda kv: -kv[1][0])},
        "kernel_timing": (f"{args.steps} more steps; " + (
            "the solve as a profiled copy of its captured graph (same kernels and grouped launches, unrolled "
            "to the timed V-cycle count) with event-record nodes around each kernel node; a grouped launch's "
            "time is split over its operations by their algorithmic bytes; deposit and gather bracketed by "
            "events on the stream" if prof_mode == "graph" else "host-driven launches, each bracketed by events")),
        "e2e": {"value": e2e_value, "unit": "solves/s", "ms_per_step": [round(x, 3) for x in e2e_ms],
                "h2d_bytes_per_step": 32 * n,
                "d2h_bytes_per_step": 24 * n},
        "clocks": clocks.summary(),
    }
    out["kernels_ms_per_step"] = total_prof_ms / args.steps

    # the mixed-precision form on the same workload: its own timed steps and
    # the error of every timed result against the FP64 result
    Rm = None
    if args.precision == "fp64" and not args.no_mixed and world == 1:
        Rm = StepRunner(amrmg, w, dev, "mixed", args, stream)
        errs = []

        def mixed_error(k):
            e = rel_l2([t.cpu().numpy() for t in Rm.E], [t.cpu().numpy() for t in E64])
            ph = rel_l2(Rm.levels(), phi64)
            errs.append({"phi_rel_l2": ph, "e_rel_l2": e})

        ms_m, it_m = Rm.timed(args.steps, args.warmup, flush, after=mixed_error)
        out["mixed"] = {
            "value": args.steps / (sum(ms_m) / 1e3), "unit": "solves/s", "ms_per_step": sum(ms_m) / args.steps,
            "iters_per_solve": statistics.mean(it_m), "dtype": "f32+f64",
            "error_vs_fp64_per_result": errs,
            "max_error_vs_fp64": {"phi_rel_l2": max(x["phi_rel_l2"] for x in errs),
                                  "e_rel_l2": max(x["e_rel_l2"] for x in errs)},
            "note": "FP32 V-cycle on the correction inside FP64 iterative refinement (FP64 residual, interface "
                    "corrections and coarsest solve); errors are relative L2 over all levels (phi) and all "
                    "particles (gathered E) against the FP64 step's result",
        }
    if not args.no_cpu_baseline and world == 1:
        S = OracleSample(w, parts_host, robin_d=args.robin_d, periodic=args.periodic)
        S.step()
        vc = int(round(statistics.mean(iters)))
        out["cpu_baseline"] = S.report(w, vc, "the GPU solve's V-cycle count")
        # the oracle's solve carried on to the stopping tolerance (untimed):
        # the FP64 and mixed results of the last timed steps against it
        more, rel = S.O.solve(eps=EPS, max_iter=100, bottom_rtol=1e-12, warm=True)
        oe = S.O.gather(*parts_host[:3])
        ophi = [S.O.get(l, "phi") for l in range(S.O.nlevels)]
        ev = {"oracle_vcycles": S.cycles + more, "oracle_rel_res": [float(x) for x in rel],
              "fp64": {"phi_rel_l2": rel_l2(phi64, ophi),
                       "e_rel_l2": rel_l2([t.cpu().numpy() for t in E64], list(oe))}}
        if Rm is not None:
            ev["mixed"] = {"phi_rel_l2": rel_l2(Rm.levels(), ophi),
                           "e_rel_l2": rel_l2([t.cpu().numpy() for t in Rm.E], list(oe))}
        ev["note"] = ("both sides stop at relative residual 1e-10, so these differences are the solve tolerance's "
                      "(the parity tests solve both sides tighter)")
        out["error_vs_oracle"] = ev
        del S
    # the roofline instance (256^3 + 3 levels, 10^7 particles in five
    # bunches), FP64 and mixed, a few timed steps each
    if args.workload == "c3_bunches" and not args.no_roofline_instance and world == 1:
        del Rm
        wr = inputs.workload("roofline")
        pr = wr.particles()
        dr = [torch.from_numpy(a).cuda() for a in pr]
        ri = {}
        for prec in ("fp64", "mixed"):
            Rr = StepRunner(amrmg, wr, dr, prec, args, stream)
            ms_r, it_r = Rr.timed(3, 2, flush)
            pr_r = kernel_profile(Rr, 1, flush, prof_mode)
            vk = [k for k in vcycle_kinds if k in pr_r]
            vms = sum(pr_r[k][0] for k in vk)
            vby = sum(pr_r[k][2] for k in vk)
            top = max(pr_r.items(), key=lambda kv: kv[1][0])
            ri[prec] = {"value": 3 / (sum(ms_r) / 1e3), "unit": "solves/s", "ms_per_step": sum(ms_r) / 3,
                        "iters_per_solve": statistics.mean(it_r), "creation_s": Rr.create_s,
                        "valid_cells": [Rr.H.level_box(l)[2] for l in range(Rr.H.nlevels)],
                        "vcycle_alg_gbs": vby / (vms / 1e3) / 1e9 if vms else None,
                        "vcycle_ms_per_solve": vms,
                        "top_kernel": {"kind": top[0], "ms_per_solve": top[1][0],
                                       "alg_gbs": top[1][2] / (top[1][0] / 1e3) / 1e9 if top[1][0] else None,
                                       **({"alg_tflops": top[1][3] / (top[1][0] / 1e3) / 1e12}
                                          if top[1][3] and top[1][0] else {})}}
            del Rr
            torch.cuda.synchronize()
        out["roofline_instance"] = {"workload": "roofline (n0 256, 3 refinement levels, 1e7 particles, five "
                                                "bunches)", **ri}
    print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def roofline(precision, name, ms, n, alg_bytes, alg_flops, hbm_peak, peak_src, traffic, total_ms, fp64=None,
             alg_ops=0.0):
    """Roofline of the dominant kernel.  An FP64 kernel is bound by the FP64
    pipe (about two lanes per SM on this part): it is reported as the rate of
    its algorithmic FP64 instructions (an FMA counts 1, an add or a multiply
    1) against the FP64 instruction rate the library's probe measured in this
    run, with the flop view (against 2 flops per probe FMA) and the HBM view
    beside it; FP32 kernels against HBM."""
    gbs = alg_bytes / (ms / 1e3) / 1e9
    hbm = {"achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
           "peak_source": "of measured" if peak_src == "measured" else "of fallback"}
    base = {"kernel": name, "traffic": traffic, "launches": n, "avg_launch_us": 1e3 * ms / n,
            "share": ms / total_ms}
    if precision == "fp64" and alg_flops:
        tf = alg_flops / (ms / 1e3) / 1e12
        fpeak = fp64["tflops"] if fp64 else FP64_PEAK_TFLOPS
        src = ("of measured: FP64 FMA probe (amr_probe_fp64_fma) in this run" if fp64
               else "of derived: 152 SMs x 2 FP64 FMA/clk x 2.07 GHz")
        flop_view = {"achieved": tf, "peak": fpeak, "unit": "TFLOP/s", "frac": tf / fpeak}
        if alg_ops:
            top = alg_ops / (ms / 1e3) / 1e12
            opeak = fpeak / 2.0  # one FP64 instruction per probe FMA
            return {"bound": "alu", "achieved": top, "peak": opeak, "unit": "T FP64 instr/s", "frac": top / opeak,
                    "peak_source": src, **base, "flops": flop_view, "hbm": hbm}
        return {"bound": "alu", **flop_view, "peak_source": src, **base, "hbm": hbm}
    return {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
            "peak_source": hbm["peak_source"], **base}


def ctypes_ptr(t):
    import ctypes
    return ctypes.c_void_p(t.data_ptr())


if __name__ == "__main__":
    main()
