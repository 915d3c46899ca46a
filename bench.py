#!/usr/bin/env python
"""Throughput benchmark of the DPD-CGMD engine on synthetic systems.

Default workload (N = 1): the DPD-only throughput system -- 1,000,000 plasma
particles at rho = 3 in a 69.336^3 box with frozen walls in y and a
Poiseuille body force g = 0.02, velocity-Verlet at dt = 0.01 (one reduced time
unit = 166.4 ns, so a step is 1.664 ns), Verlet skin 0.3.  One "step" is one
fluid step of the whole hot path: kick-drift + rebuild check, (conditional)
cell sort + list build, DPD pair forces.

Prints ONE JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle
instead, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

NS_PER_TAU = 166.4          # 1 tau = 166.4 ns (dt_f = 0.01 tau = 1.664 ns)
METRIC = "simulated ns/day & particle-steps/s, AI-MTS vs fine-step STS on 1 GB300"
L2_BYTES = 126 * 2 ** 20
FALLBACK_HBM_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", default="msm", choices=["msm", "reference"])
    ap.add_argument("--workload", default="dpd1m", choices=["dpd1m"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--direct", action="store_true",
                    help="launch every kernel from the host instead of replaying the captured graph "
                         "(profilers cannot see kernels inside conditional graphs)")
    return ap.parse_args()


def workload(name, seed):
    import synth
    if name == "dpd1m":
        s = synth.config_dpd_throughput(seed=seed)
        return s, dict(dt=0.01, skin=0.3, mode="sts")
    raise ValueError(name)


def ns_per_day(steps, seconds, dt):
    return steps * dt * NS_PER_TAU / seconds * 86400.0


def cpu_count():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def oracle_sample(seed, target_s=10.0, max_steps=200):
    """The FP64 oracle (as it stands) on a 65,536-particle sample of the same
    workload (same density, walls, body force, dt): particle-steps/s."""
    import oracle as O
    import synth
    s = synth.plasma_box(n=65536, walls=True, body_force=0.02, seed=seed)
    p = O.system_params(s)
    x, v, f = O.run_respa(p, s.x, s.v, s.tag, dt_f=0.01, n_outer=1)
    steps, t0 = 0, time.perf_counter()
    n0 = 1
    while steps < max_steps and time.perf_counter() - t0 < target_s:
        x, v, f = O.run_respa(p, x, v, s.tag, dt_f=0.01, n_outer=1, n0=n0, t0=n0 * 0.01, forces=f)
        steps += 1
        n0 += 1
    el = time.perf_counter() - t0
    return s.n * steps / el, steps, s.n, el


class ClockSampler:
    def __init__(self, path):
        self.path = path
        self.proc = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=self.fh, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self, gpu_index):
        if self.proc is None or not os.path.exists(self.path):
            return None
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [c.strip() for c in line.split(",")]
            if len(f) < 9:
                continue
            try:
                if int(f[0]) != gpu_index:
                    continue
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        for k in ("hbm_gbs", "hbm_GBps", "hbm"):
            if k in d:
                return float(d[k]), "measured"
    except Exception:
        pass
    return FALLBACK_HBM_GBS, "fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    for fn in ("forces.cu", "msm_internal.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2205_14121_gb300", "csrc", fn), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(workload_name):
    """DRAM bytes per launch of the fluid DPD kernel from a committed ncu
    summary, if it was taken on the current kernel source."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        d = json.load(open(path))
        e = d.get(workload_name)
        if e and e.get("source_hash") == kernel_source_hash():
            return float(e["dram_bytes_per_launch"])
    except Exception:
        pass
    return None


def whole_job_rate(units_local, seconds_local, world, device="cpu"):
    """Replicas: units processed by all ranks / the slowest rank's time.
    Returns (units_total, seconds_max); collective only when world > 1."""
    if world <= 1:
        return float(units_local), float(seconds_local)
    import torch
    import torch.distributed as dist
    u = torch.tensor([float(units_local)], dtype=torch.float64, device=device)
    t = torch.tensor([float(seconds_local)], dtype=torch.float64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(u.item()), float(t.item())


def run_reference(args, rank, world):
    if rank != 0:
        return
    s_ps, steps, n, el = None, 0, 0, 0.0
    per_step = []
    import oracle as O
    import synth
    s = synth.plasma_box(n=65536, walls=True, body_force=0.02, seed=20220528)
    p = O.system_params(s)
    x, v, f = O.run_respa(p, s.x, s.v, s.tag, dt_f=0.01, n_outer=1)
    n0 = 1
    for it in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        x, v, f = O.run_respa(p, x, v, s.tag, dt_f=0.01, n_outer=1, n0=n0, t0=n0 * 0.01, forces=f)
        n0 += 1
        if it >= args.warmup:
            per_step.append(time.perf_counter() - t0)
    el = float(np.sum(per_step))
    s_ps = s.n * args.steps / el
    # the sample's particle-steps/s, expressed for the full workload's particle count
    n_full = workload(args.workload, seed=20220528)[0].n
    value = s_ps / n_full * 0.01 * NS_PER_TAU * 86400.0
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "ns/day", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "particle_steps_per_s": s_ps,
            "config": {"workload": "dpd-only throughput, 65,536-particle sample (rho=3, walls, g=0.02, dt=0.01)",
                       "sample_of": args.workload},
            "cpu_baseline": {"value": value, "unit": "ns/day", "cores": cpu_count(), "kind": "oracle",
                             "sample": f"{args.steps} STS steps of a {s.n}-particle sample, scaled to "
                                       f"{n_full} particles by particle-steps/s"},
            "e2e": {"value": value, "unit": "ns/day", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    import torch.distributed as dist

    import paper_2205_14121_gb300 as M
    from paper_2205_14121_gb300 import build as B

    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    B.build()

    s, wl = workload(args.workload, seed=20220528 + rank)
    n = s.n
    g = M.System(s.box, s.x, s.v, s.tag, X0=s.X0, bonds=s.bonds, r0=s.r0, walls=s.walls, wall=s.wall,
                 shear_rate=s.shear_rate, body_force=s.body_force, dt=wl["dt"], skin=wl["skin"])
    stream = g.stream

    # warm-up (first list build, first forces, clocks)
    g.mts_step(args.warmup, direct=args.direct)
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # ---- timed region --------------------------------------------------
    g.profile_read(reset=True)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    clk_path = os.path.join(ROOT, "gpurun_out", f"clocks_rank{rank}.csv")
    os.makedirs(os.path.dirname(clk_path), exist_ok=True)
    with ClockSampler(clk_path) as clk:
        barrier()
        ev0.record(stream)
        g.mts_step(args.steps, direct=args.direct)
        ev1.record(stream)
        barrier()
    ms = ev0.elapsed_time(ev1)
    prof_plain = g.profile_read(reset=True)
    # whole job: every rank's particle-steps over the slowest rank's time
    units, sec = whole_job_rate(n * args.steps, ms / 1e3, world, device="cuda")
    ms = sec * 1e3
    ps = units / sec
    value = ns_per_day(args.steps, sec, wl["dt"]) * (units / (n * args.steps))

    # ---- roofline pass: same K steps with per-class CUDA events ----------
    g.profile_enable(True)
    g.mts_step(args.steps)
    prof = g.profile_read(reset=True)
    g.profile_enable(False)
    obs = g.observables()
    n_half = len(g.neighbor_pairs(M.MD_LIST_FLUID)) / n
    fl_launch = prof["launches"]["fluid_dpd"]
    fl_ms = prof["ms"]["fluid_dpd"] / max(fl_launch, 1)
    bytes_per_particle = 16 + 16 + 4 * n_half + 16      # x32 + v + list + f
    achieved = n * bytes_per_particle / (fl_ms * 1e-3) / 1e9
    peak, peak_kind = measured_peak()
    traffic = ncu_traffic(args.workload)

    # ---- end to end through the C ABI with host buffers ------------------
    e2e = None
    if args.e2e_steps > 0:
        xh = torch.from_numpy(np.ascontiguousarray(s.x)).pin_memory().numpy()
        vh = torch.from_numpy(np.ascontiguousarray(s.v)).pin_memory().numpy()
        th = torch.from_numpy(np.ascontiguousarray(s.tag)).pin_memory().numpy()
        barrier()
        t0 = time.perf_counter()
        for k in range(args.e2e_steps):
            g.set_particles(xh, vh, th, s.X0, step0=k)
            g.mts_step(1)
            g.observables()
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        e2e = {"value": ns_per_day(args.e2e_steps, el, wl["dt"]) * world, "unit": "ns/day",
               "h2d_bytes_per_step": int(xh.nbytes + vh.nbytes + th.nbytes),
               "d2h_bytes_per_step": 3 * (16 * 4 + 64) + 16 * 8 + 9 * 8,
               "note": "per step: state upload, forced list rebuild + forces, one step, observables"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        ps_cpu, st_cpu, n_cpu, el_cpu = oracle_sample(seed=20220528)
        cpu = {"value": ps_cpu / n * wl["dt"] * NS_PER_TAU * 86400.0, "unit": "ns/day", "cores": cpu_count(),
               "kind": "oracle", "particle_steps_per_s": ps_cpu,
               "sample": f"{st_cpu} STS steps of a {n_cpu}-particle sample of the same workload ({el_cpu:.1f} s), "
                         f"scaled to {n} particles by particle-steps/s"}

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    clocks = clk.summary(local)
    line = {
        "metric": METRIC, "value": value, "unit": "ns/day", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "particle_steps_per_s": ps,
        "config": {"workload": "dpd-only throughput: 1,000,000 plasma particles, rho=3, 69.336^3 box, walls in y, "
                               "g=0.02, STS velocity-Verlet dt=0.01, skin 0.3",
                   "n_particles": n, "mode": "replicas" if world > 1 else "single",
                   "l2": "inputs larger than L2 (about 2e8 B touched per step vs 1.3e8 B L2); no flush"},
        "roofline": {"bound": "hbm", "kernel": "k_dpd (fluid level pair forces)", "achieved": achieved,
                     "peak": peak, "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                     "peak_source": peak_kind,
                     "bytes_per_particle": bytes_per_particle, "n_half": n_half, "launch_ms": fl_ms},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": prof_plain["total_launches"],
        "clocks": clocks,
        "kernel_ms_per_step": {k: v / max(args.steps, 1) for k, v in prof["ms"].items()},
        "n_builds": obs["n_builds"],
        "temperature": obs["temperature"],
    }
    print(json.dumps(line), flush=True)
    g.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
