"""Benchmark of one particle-in-cell field step: cloud-in-cell deposit onto
every level -> AMR multigrid V-cycles to relative residual 1e-10 -> E
gathered to the particles, FP64, on the base-64^3 hierarchy with two tagged
refinement levels (rho > 0.1 max) and 1e6 anisotropic-Gaussian particles.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  With N > 1 (torchrun) every rank solves its
own seeded replica of the workload (no collective on the data path) and
the value is the total solves/s over all ranks.
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
WORKLOAD = "c2_fp64"
FALLBACK_HBM_GBS = 6800.0
# FP64 arithmetic peak from unit counts and clock: 152 SMs x 2 FP64 FMA
# lanes per SM per clock x 2 flops x 2.07 GHz (a probe measured 598 GFMA/s)
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
    ap.add_argument("--form", default="step", choices=["step", "batched", "served", "pic"],
                    help="step: one deposit/solve/gather step; batched: many hierarchies per launch")
    ap.add_argument("--batch", type=int, default=256)
    ap.add_argument("--pic-particles", type=int, default=1_000_000, help="pic: particles of the five bunches")
    ap.add_argument("--pic-n0", type=int, default=64, help="pic: base grid")
    ap.add_argument("--requests", type=int, default=300, help="served: requests taken from the stream")
    ap.add_argument("--slots", type=int, default=16, help="served: concurrent slots")
    ap.add_argument("--budget-gb", type=float, default=150.0, help="served: HBM budget")
    ap.add_argument("--max-n0", type=int, default=96, help="served: cap of the base grid (bounded sample)")
    ap.add_argument("--max-particles", type=float, default=1e6, help="served: cap of the particle count")
    ap.add_argument("--mode", default="graph", choices=["graph", "persistent", "eager"],
                    help="solve as one captured graph, one persistent kernel, or host-driven launches")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


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


def run_reference(args, rank, world):
    """The oracle (plain FP64 CPU C) timed on this host's cores on the same
    workload, one full deposit + solve + gather per step."""
    if rank != 0:
        return
    import oracle
    from paper_1812_03689_gb300 import inputs
    w = inputs.workload(args.workload)
    parts = w.particles()
    O = oracle.OracleHierarchy(w.n0, w.lmax, particles=parts, tag_mode=w.tag_mode, tag_lambda=w.tag_lambda,
                               boxes=w.boxes or None, robin_d=args.robin_d or 0.0, periodic=args.periodic)

    def step():
        O.deposit(*parts)
        O.solve(eps=EPS, bottom_rtol=1e-12)
        O.gather(*parts[:3])

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    v = args.steps / dt
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "n0": w.n0, "max_level": w.lmax, "particles": w.n_particles,
                   "bc": bc_name(args)},
        "cpu_baseline": {"value": v, "unit": "solves/s", "cores": 1, "kind": "oracle",
                         "sample": "every step is the full workload (deposit + solve to 1e-10 + gather)"},
        "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def bc_name(args):
    if args.periodic:
        return "periodic"
    return "dirichlet" if args.robin_d is None else f"robin d={args.robin_d:g}"


def cpu_baseline(w, parts, budget_s=25.0, robin_d=None, periodic=False):
    import oracle
    t0 = time.perf_counter()
    O = oracle.OracleHierarchy(w.n0, w.lmax, particles=parts, tag_mode=w.tag_mode, tag_lambda=w.tag_lambda,
                               boxes=w.boxes or None, robin_d=robin_d or 0.0, periodic=periodic)
    t1 = time.perf_counter()
    n = 0
    while True:
        O.deposit(*parts)
        O.solve(eps=EPS, bottom_rtol=1e-12)
        O.gather(*parts[:3])
        n += 1
        if time.perf_counter() - t1 > budget_s / 2 or n >= 3:
            break
    dt = time.perf_counter() - t1
    return {"value": n / dt, "unit": "solves/s", "cores": 1, "kind": "oracle",
            "sample": f"{n} full step(s) of {w.name} (deposit + solve to 1e-10 + gather), "
                      f"hierarchy creation ({t1 - t0:.2f} s) excluded"}


def run_batched(args, rank, world, local):
    """Batched form: independent uneven hierarchies solved to 1e-10 by one
    persistent kernel launch per solve, against the same hierarchies solved
    one after another (one captured graph each)."""
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
    B = amrmg.Batch(hs, **opts)
    stream = torch.cuda.current_stream()
    launches0 = sum(h.kernel_launches() for h in hs)
    for _ in range(args.warmup):
        B.solve()
    torch.cuda.synchronize()
    ms_b = []
    for _ in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        stats = B.solve()
        e1.record(stream)
        e1.synchronize()
        ms_b.append(e0.elapsed_time(e1))
    launches_b = (sum(h.kernel_launches() for h in hs) - launches0) / args.steps
    phi_b = [h.get(h.nlevels - 1, "phi") for h in hs[:16]]
    # one at a time, one graph each
    for h in hs:
        h.solve(**opts)
    torch.cuda.synchronize()
    ms_s = []
    for _ in range(max(1, args.steps // 2)):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for h in hs:
            h.solve(**opts)
        e1.record(stream)
        e1.synchronize()
        ms_s.append(e0.elapsed_time(e1))
    phi_s = [h.get(h.nlevels - 1, "phi") for h in hs[:16]]
    same = all(np.array_equal(a, b) for a, b in zip(phi_b, phi_s))
    # the same hierarchies side by side: their graphs on 16 streams
    amrmg.solve_many(hs, n_streams=16, **opts)
    torch.cuda.synchronize()
    ms_c = []
    for _ in range(max(1, args.steps // 2)):
        t0c = time.perf_counter()
        amrmg.solve_many(hs, n_streams=16, **opts)
        ms_c.append(1e3 * (time.perf_counter() - t0c))
    phi_c = [h.get(h.nlevels - 1, "phi") for h in hs[:16]]
    same_c = all(np.array_equal(a, b) for a, b in zip(phi_c, phi_s))
    tc = statistics.median(ms_c)
    tb = statistics.median(ms_b)
    ts = statistics.median(ms_s)
    out = {
        "metric": "batched solves/s to 1e-10 residual (one persistent launch per batch)",
        "value": len(hs) / (tb / 1e3), "unit": "solves/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tb, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32+f64", "data": "synthetic",
        "config": {"workload": "batched_uneven", "hierarchies": len(hs), "precision": args.precision,
                   "n0_range": [min(r.n0 for r in reqs), max(r.n0 for r in reqs)],
                   "levels": [sum(1 for h in hs if h.nlevels == k) for k in (1, 2, 3)],
                   "particles_range": [min(r.n_particles for r in reqs), max(r.n_particles for r in reqs)],
                   "creation_s": create_s},
        "gpu_launches": launches_b,
        "sequential_graph": {"value": len(hs) / (ts / 1e3), "unit": "solves/s", "ms": ts},
        "concurrent_graphs": {"value": len(hs) / (tc / 1e3), "unit": "solves/s", "ms": tc, "streams": 16,
                              "timing": "host wall clock around amr_solve_many (returns when all are done)",
                              "bitwise_equal_to_sequential": same_c},
        "speedup_vs_sequential": ts / tb,
        "iters": {"min": min(s["iters"] for s in stats), "max": max(s["iters"] for s in stats),
                  "mean": statistics.mean(s["iters"] for s in stats)},
        "max_rel_res": max(float(s["rel_res"].max()) for s in stats),
        "bitwise_equal_to_sequential": same,
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


def run_served(args, rank, world, local):
    """Served form: a Poisson stream of uneven requests through the
    continuous-batching loop (admission by HBM budget, overlapping slots),
    against the same requests one at a time."""
    import torch
    from paper_1812_03689_gb300 import amrmg, inputs
    torch.cuda.set_device(local)
    stream_reqs = inputs.served_requests(10_000, 2000.0, max_n0=args.max_n0, max_particles=args.max_particles)
    sample = stream_reqs[:args.requests]
    reqs = [amrmg.make_request(r.n0, r.lmax, r.n_particles, r.sigma, seed=1812036890 + r.index,
                               arrival_s=r.arrival_s, precision=args.precision) for r in sample]
    budget = int(args.budget_gb * (1 << 30))
    opts = dict(eps=EPS, bottom_cycles=args.bottom_cycles)
    amrmg.serve(reqs[:4], budget, args.slots, realtime=False, **opts)  # warm-up (allocator, caches)
    res = amrmg.serve(reqs, budget, args.slots, realtime=True, **opts)
    ok = [r for r in res if r["status"] in (0, 3)]
    lat = np.array([r["done_s"] - r["arrival_s"] for r in ok])
    span = max(r["done_s"] for r in res) - min(r["arrival_s"] for r in res)
    seq = amrmg.serve(reqs, budget, 1, realtime=False, **opts)
    seq_span = max(r["done_s"] for r in seq)
    seq_lat = np.array([r["done_s"] for r in seq])
    diffs = [float(np.abs(a["checksum"] - b["checksum"]).max() / max(np.abs(b["checksum"]).max(), 1e-300))
             for a, b in zip(res, seq) if a["status"] == 0 and b["status"] == 0]
    out = {
        "metric": "served solves/s and p50/p99 latency (continuous batching, Poisson arrivals)",
        "value": len(ok) / span, "unit": "solves/s", "n_gpus": 1, "steps": len(reqs), "warmup": 4,
        "ms_per_step": 1e3 * span / max(len(ok), 1), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32+f64", "data": "synthetic",
        "config": {"workload": "served_poisson", "requests": len(reqs), "of_stream": 10_000,
                   "rate_per_s": 2000.0, "n0_cap": args.max_n0, "particles_cap": args.max_particles,
                   "slots": args.slots, "budget_gb": args.budget_gb, "precision": args.precision},
        "latency_s": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                      "max": float(lat.max())},
        "one_at_a_time": {"value": len(reqs) / seq_span, "unit": "solves/s",
                          "latency_s_if_arriving_together": {"p50": float(np.percentile(seq_lat, 50)),
                                                             "p99": float(np.percentile(seq_lat, 99))}},
        "refused": sum(1 for r in res if r["status"] == 2),
        "max_rel_res": max(r["rel_res_max"] for r in ok),
        "max_checksum_rel_diff_vs_alone": max(diffs) if diffs else None,
        "peak_reserved_gb": None,
    }
    print(json.dumps(out), flush=True)


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
    H = amrmg.Hierarchy(w.n0, w.lmax, particles=dev, tag_mode=w.tag_mode, tag_lambda=w.tag_lambda,
                        boxes=w.boxes or None, stream=stream, precision=args.precision, robin_d=args.robin_d,
                        periodic=args.periodic)
    ex, ey, ez = (torch.empty(n, dtype=torch.float64, device="cuda") for _ in range(3))
    opts = dict(eps=EPS, bottom_cycles=args.bottom_cycles, use_graph=args.mode == "graph",
                persistent=args.mode == "persistent")
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")  # 512 MB > L2

    def step():
        H.deposit(*dev)
        st = H.solve(**opts)
        amrmg._check(amrmg._lib.amr_gather(H._h, *[amrmg._dev(t, "p") for t in dev[:3]], n,
                                           amrmg._dev(ex, "ex"), amrmg._dev(ey, "ey"), amrmg._dev(ez, "ez"), None))
        return st

    for _ in range(args.warmup):
        st = step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    launches0 = H.kernel_launches()
    iters = []
    ms_steps = []
    with ClockSampler(local) as clocks:
        torch.cuda.synchronize()
        for _ in range(args.steps):
            flush.fill_(1.0)  # L2 flush between timed steps, outside the events
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st = step()
            e1.record(stream)
            e1.synchronize()
            ms_steps.append(e0.elapsed_time(e1))
            iters.append(st["iters"])
        torch.cuda.synchronize()
    launches = H.kernel_launches() - launches0
    total_ms = sum(ms_steps)
    if world > 1:
        t = torch.tensor([total_ms], dtype=torch.float64, device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    value = world * args.steps / (total_ms / 1e3)

    # per-kernel device times: the same K steps again with per-launch events
    H.profile(True)
    for _ in range(args.steps):
        flush.fill_(1.0)
        step()
    torch.cuda.synchronize()
    prof = H.profile_read()
    H.profile(False)

    # end to end through the C ABI with host buffers (pinned), copies timed
    pin = [torch.from_numpy(a).pin_memory() for a in parts_host]
    pout = [torch.empty(n, dtype=torch.float64).pin_memory() for _ in range(3)]
    o = amrmg.solve_opts(**opts)
    ptrs = [ctypes_ptr(t) for t in pin]
    optrs = [ctypes_ptr(t) for t in pout]
    H.step_ptrs(*ptrs, n, *optrs, o)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        H.step_ptrs(*ptrs, n, *optrs, o)
    e2e_s = time.perf_counter() - t0
    e2e_value = world * args.steps / e2e_s if world == 1 else None
    if world > 1:
        t = torch.tensor([e2e_s], dtype=torch.float64, device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        e2e_value = world * args.steps / float(t.item())

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    peaks, peak_src = measured_peaks()
    hbm_peak = float(peaks.get("hbm_gbs", FALLBACK_HBM_GBS)) if peaks else FALLBACK_HBM_GBS
    dom = max(prof.items(), key=lambda kv: kv[1][0])
    dom_name, (dom_ms, dom_n, dom_bytes, dom_flops) = dom
    achieved = dom_bytes / (dom_ms / 1e3) / 1e9
    total_prof_ms = sum(v[0] for v in prof.values())
    vcycle_kinds = ("rbgs", "residual", "restrict", "prolong", "finish", "cf_correct", "flux", "norms",
                    "mg_restrict", "mg_prolong", "coarse_solve", "elementwise")
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
                             traffic, total_prof_ms),
        "vcycle": {"alg_gbs": vc_bytes / (vc_ms / 1e3) / 1e9 if vc_ms else None, "ms_per_solve": vc_ms / args.steps},
        "kernels": {k: {"ms": v[0], "launches": v[1], "alg_gbs": v[2] / (v[0] / 1e3) / 1e9 if v[0] else None,
                        **({"alg_tflops": v[3] / (v[0] / 1e3) / 1e12} if v[3] and v[0] else {})}
                    for k, v in sorted(prof.items(), key=lambda kv: -kv[1][0])},
        "e2e": {"value": e2e_value, "unit": "solves/s", "h2d_bytes_per_step": 32 * n,
                "d2h_bytes_per_step": 24 * n},
        "clocks": clocks.summary(),
    }
    if not args.no_cpu_baseline and world == 1:
        out["cpu_baseline"] = cpu_baseline(w, parts_host, robin_d=args.robin_d, periodic=args.periodic)
    print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def roofline(precision, name, ms, n, alg_bytes, alg_flops, hbm_peak, peak_src, traffic, total_ms):
    """Roofline of the dominant kernel.  An FP64 smoother is bound by the
    FP64 pipe (about two lanes per SM), so it is reported against the FP64
    arithmetic peak, with its HBM view beside it; FP32 kernels against HBM."""
    gbs = alg_bytes / (ms / 1e3) / 1e9
    hbm = {"achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
           "peak_source": "of measured" if peak_src == "measured" else "of fallback"}
    base = {"kernel": name, "traffic": traffic, "launches": n, "avg_launch_us": 1e3 * ms / n,
            "share": ms / total_ms}
    if precision == "fp64" and alg_flops:
        tf = alg_flops / (ms / 1e3) / 1e12
        return {"bound": "alu", "achieved": tf, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": tf / FP64_PEAK_TFLOPS,
                "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk x 2 flops x 2.07 GHz", **base, "hbm": hbm}
    return {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
            "peak_source": hbm["peak_source"], **base}


def ctypes_ptr(t):
    import ctypes
    return ctypes.c_void_p(t.data_ptr())


if __name__ == "__main__":
    main()
