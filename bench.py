#!/usr/bin/env python
"""Throughput benchmark of the DPD-CGMD engine on synthetic systems.

Default workload (N = 1): the platelet channel -- 8,040,000 plasma particles
at rho = 3 in a 400 x 100 x 67 channel with frozen walls in y and a
Poiseuille body force (wall shear rate 0.05), plus 16 platelets of 10,000
coarse-grained particles (8,360,800 particles).  The timed arm is AI-MTS:
outer steps of dt_f = 0.01 (one reduced time unit = 166.4 ns, so 1.664 ns per
step), one interface substep, per-platelet step ratios from the trained
controller (fixed k = 10 when no trained parameters are present).  Beside it,
the same system under fine-step STS (velocity-Verlet with dt = 0.001 for
every particle, the reference of Sec. 4.1) and under fixed-k RESPA (k = 10).

``--workload dpd1m``: the DPD-only throughput system (1,000,000 plasma
particles in a 69.336^3 box, walls, g = 0.02, STS dt = 0.01, skin 0.3).

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
FALLBACK_HBM_GBS = 6800.0
CONTROLLER = os.path.join(ROOT, "paper_2205_14121_gb300", "data", "controller.npz")


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=150)
    ap.add_argument("--impl", default="msm", choices=["msm", "reference"])
    ap.add_argument("--workload", default="channel", choices=["channel", "dpd1m"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-compare", action="store_true", help="skip the fine-STS and fixed-k arms")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--clock-log", default=None,
                    help="directory for the nvidia-smi clock samples of the timed region (default: a temp dir)")
    ap.add_argument("--direct", action="store_true",
                    help="launch every kernel from the host instead of replaying the captured graph "
                         "(profilers cannot see kernels inside conditional graphs)")
    return ap.parse_args(argv)


def workload(name, seed):
    import synth
    if name == "dpd1m":
        return synth.config_dpd_throughput(seed=seed), dict(
            dt=0.01, skin=0.3,
            desc="dpd-only throughput: 1,000,000 plasma particles, rho=3, 69.336^3 box, walls in y, g=0.02, "
                 "STS velocity-Verlet dt=0.01, skin 0.3")
    if name == "channel":
        return synth.config_channel_platelets(seed=seed), dict(
            dt=0.01, skin=0.3, skin_plt=0.5,
            desc="platelet channel: 8,040,000 plasma at rho=3 in 400x100x67, y walls, Poiseuille g for wall "
                 "shear rate 0.05, 16 platelets x 10,000 CG particles (5% receptors); AI-MTS dt_f=0.01, k_m=1, "
                 "per-platelet k from the controller vs fine-step STS dt=0.001; skin 0.3, platelet skin 0.5")
    raise ValueError(name)


def ns_per_day(steps, seconds, dt):
    return steps * dt * NS_PER_TAU / seconds * 86400.0


def cpu_count():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


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


class OracleSample:
    """The FP64 oracle (as it stands) on a bounded sample of the workload."""

    def __init__(self, name, seed):
        import oracle as O
        import synth
        self.O = O
        if name == "dpd1m":
            s = synth.plasma_box(n=65536, walls=True, body_force=0.02, seed=seed)
            self.what = "STS steps"
            self.kw = dict(dt_f=0.01)
            self.fn = O.run_respa
            self.extra = ()
        else:
            # a 20 x 10 x 8 section of the channel with one 600-particle platelet, AI-MTS with k = 10
            g = synth.poiseuille_g(0.05, synth.ETA_DPD, 3.0, 10.0)
            s = synth.platelet_system((20.0, 10.0, 8.0), 4800, 1, 600, synth.scaled_radii(600), walls=True,
                                      body_force=g, seed=seed, centers=[(10.0, 5.0, 4.0)])
            self.what = "AI-MTS outer steps (k = 10)"
            self.kw = dict(X0=s.X0, bonds=s.bonds, r0=s.r0, dt_f=0.01, k_m=1)
            self.fn = O.run_ai_respa
            self.extra = ([10],)
        self.s = s
        self.p = O.system_params(s)
        self.x, self.v, self.f = self.fn(self.p, s.x, s.v, s.tag, *self.extra, n_outer=1, **self.kw)
        self.n0 = 1

    def step(self):
        self.x, self.v, self.f = self.fn(self.p, self.x, self.v, self.s.tag, *self.extra, n_outer=1, n0=self.n0,
                                         t0=self.n0 * 0.01, forces=self.f, **self.kw)
        self.n0 += 1


def oracle_rate(name, seed, target_s=10.0, max_steps=200):
    o = OracleSample(name, seed)
    steps, t0 = 0, time.perf_counter()
    while steps < max_steps and time.perf_counter() - t0 < target_s:
        o.step()
        steps += 1
    el = time.perf_counter() - t0
    return o.s.n * steps / el, steps, o.s.n, el, o.what


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


def ncu_traffic(workload_name, skin):
    """DRAM bytes per launch of the fluid DPD kernel from a committed ncu
    summary, if it was taken on the current kernel source and list skin."""
    path = os.path.join(ROOT, "profiles", "k_dpd_traffic.json")
    try:
        d = json.load(open(path))
        e = d.get(workload_name)
        if e and e.get("source_hash") == kernel_source_hash() and e.get("skin") == skin:
            return float(e["dram_bytes_per_launch"])
    except Exception:
        pass
    return None


def run_reference(args, rank, world):
    """The oracle, as it stands, timed step by step on the host cores."""
    if rank != 0:
        return
    s, wl = workload(args.workload, seed=20220528)
    n_full = s.n
    del s
    o = OracleSample(args.workload, 20220528)
    per_step = []
    for it in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        o.step()
        if it >= args.warmup:
            per_step.append(time.perf_counter() - t0)
    el = float(np.sum(per_step))
    n_s = o.s.n
    s_ps = n_s * args.steps / el
    value = s_ps / n_full * wl["dt"] * NS_PER_TAU * 86400.0
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "ns/day", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "particle_steps_per_s": s_ps,
            "config": {"workload": f"FP64 oracle on a {n_s}-particle sample: {o.what}", "sample_of": wl["desc"]},
            "cpu_baseline": {"value": value, "unit": "ns/day", "cores": cpu_count(), "kind": "oracle",
                             "sample": f"{args.steps} {o.what} of a {n_s}-particle sample, scaled to "
                                       f"{n_full} particles by particle-steps/s"},
            "e2e": {"value": value, "unit": "ns/day", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


FINE_SKIN_PLT = 0.0      # fine-step STS: the plasma skin for the platelets too


def make_system(M, s, dt, skin, seed, skin_plt=0.0, flags=0):
    return M.System(s.box, s.x, s.v, s.tag, X0=s.X0, bonds=s.bonds, r0=s.r0, walls=s.walls, wall=s.wall,
                    shear_rate=s.shear_rate, body_force=s.body_force, dt=dt, skin=skin, seed=seed,
                    skin_plt=skin_plt, flags=flags)


def timed(g, step, n, barrier):
    """CUDA-event time (ms) of `step(n)` on g's stream, barriers on both sides."""
    import torch
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    barrier()
    ev0.record(g.stream)
    step(n)
    ev1.record(g.stream)
    barrier()
    return ev0.elapsed_time(ev1)


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
    from paper_2205_14121_gb300 import ai_mts as A
    from paper_2205_14121_gb300 import build as Bld

    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    Bld.build()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    seed = 20220528 + rank
    s, wl = workload(args.workload, seed=seed)
    n = s.n
    g = make_system(M, s, wl["dt"], wl["skin"], seed, wl.get("skin_plt", 0.0))

    mode_info = {}
    decisions = []
    ctl = None
    if args.workload == "channel":
        if os.path.exists(CONTROLLER):
            ctl, trust = A.load_controller(CONTROLLER)
            mode_info["controller"] = os.path.relpath(CONTROLLER, ROOT)
        else:
            trust = A.TrustBound()
            mode_info["controller"] = "absent: fixed k = 10 for every platelet"

        def step(k):
            if ctl is None:
                g.set_platelet_levels(np.full(g.cfg.n_platelets, trust.fallback_k, np.int32))
                g.mts_step(k, mode=M.MD_MODE_AI, k_m=1, direct=args.direct, record=True)
            else:
                A.run_ai_mts(g, ctl, k, k_m=1, trust=trust, log=decisions)
        mode_info["mode"] = "AI-MTS"
    else:
        def step(k):
            g.mts_step(k, direct=args.direct)
        mode_info["mode"] = "STS"

    # warm-up (first list build, first forces, graph capture, a full feature window)
    step(args.warmup)
    torch.cuda.synchronize()
    decisions.clear()

    # ---- timed region --------------------------------------------------
    g.profile_read(reset=True)
    import tempfile
    clk_path = os.path.join(args.clock_log or tempfile.gettempdir(), f"clocks_rank{rank}.csv")
    os.makedirs(os.path.dirname(clk_path), exist_ok=True)
    with ClockSampler(clk_path) as clk:
        ms = timed(g, step, args.steps, barrier)
    prof_plain = g.profile_read(reset=True)
    units, sec = whole_job_rate(n * args.steps, ms / 1e3, world, device="cuda")
    ms = sec * 1e3
    ps = units / sec
    value = ns_per_day(args.steps, sec, wl["dt"]) * (units / (n * args.steps))
    if ctl is not None:
        ks = [k for d in decisions for k in d["k"]]
        mode_info["decisions"] = len(decisions)
        mode_info["mean_k"] = float(np.mean(ks)) if ks else None
        mode_info["fallback_fraction"] = (float(np.mean([u for d in decisions for u in d["unsure"]]))
                                          if decisions else None)

    # ---- roofline pass: per-class CUDA events on the launching stream -----
    g.profile_enable(True)
    n_prof = min(args.steps, 100)
    step(n_prof)
    prof = g.profile_read(reset=True)
    g.profile_enable(False)
    obs = g.observables()
    n_half = g.neighbor_count(M.MD_LIST_FLUID) / n
    fl_launch = prof["launches"]["fluid_dpd"]
    fl_ms = prof["ms"]["fluid_dpd"] / max(fl_launch, 1)
    bytes_per_particle = 16 + 16 + 4 * n_half + 16      # x32 + v + list + f
    achieved = n * bytes_per_particle / (fl_ms * 1e-3) / 1e9
    peak, peak_kind = measured_peak()
    traffic = ncu_traffic(args.workload, wl["skin"])

    # ---- end to end through the C ABI with host buffers ------------------
    e2e = None
    if args.e2e_steps > 0:
        xh = torch.from_numpy(np.ascontiguousarray(s.x)).pin_memory().numpy()
        vh = torch.from_numpy(np.ascontiguousarray(s.v)).pin_memory().numpy()
        # the ratios the controller chose in the timed region (fallback k otherwise)
        levels = np.asarray(decisions[-1]["k"] if decisions else
                            [10] * (g.cfg.n_platelets if args.workload == "channel" else 0), np.int32)
        # the particle set (tags, rest positions, bonds) is configuration and
        # stays on the device; every step uploads a state and reads results
        g.set_particles(s.x, s.v, s.tag, s.X0, step0=0)

        def e2e_step(k):
            g.set_xv(xh, vh, step0=k)
            if args.workload == "channel":
                g.set_platelet_levels(levels)
                g.mts_step(1, mode=M.MD_MODE_AI, k_m=1)
            else:
                g.mts_step(1)
            g.observables()

        for k in range(2):       # warm-up: the first list build and graph capture of a one-step call
            e2e_step(k)
        barrier()
        t0 = time.perf_counter()
        for k in range(args.e2e_steps):
            e2e_step(k)
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        e2e = {"value": ns_per_day(args.e2e_steps, el, wl["dt"]) * world, "unit": "ns/day",
               "h2d_bytes_per_step": int(xh.nbytes + vh.nbytes + 4 * len(levels)),
               "d2h_bytes_per_step": 3 * (16 * 4 + 64) + 16 * 8 + 9 * 8,
               "note": "per step: upload of x and v from page-locked host memory (md_set_xv; tags, rest "
                       "positions and bonds set once before timing), a list rebuild only if the uploaded state "
                       "fails the rebuild check, forces of the new state, one outer step, observables read "
                       "back; two untimed warm-up steps"}
    g.close()
    del g
    torch.cuda.empty_cache()

    # ---- comparison arms on the same system ------------------------------
    compare = {}
    if args.workload == "channel" and not args.no_compare:
        # each arm at the Verlet skins that suit it (sweeps of the plasma skin
        # over 0.15-0.6 and of the platelet skin over 0.2-0.9: fine-step STS
        # rebuilds rarely and prefers the shorter lists of skin 0.2; the
        # dt = 0.01 arms run 2-3% faster at a plasma skin of 0.5 than at 0.3,
        # but the end-to-end step, which rebuilds every call, 9% slower, so
        # 0.3 is kept; their platelet particles, which tripped most rebuilds,
        # get a skin of 0.5: a rebuild every 5 instead of 3 outer steps)
        respa = lambda h, k: h.mts_step(k, mode=M.MD_MODE_RESPA, k_m=1, k_p=10, direct=args.direct)
        # the last arm: the uniform unit-variance noise variate in place of the
        # Gaussian (MD_CFG_UNIFORM_NOISE, a speed option; the paper's is normal)
        arms = [("fine_sts", 0.001, 0.2, FINE_SKIN_PLT, lambda h, k: h.mts_step(k, direct=args.direct), 0),
                ("respa_k10", 0.01, wl["skin"], wl["skin_plt"], respa, 0),
                ("respa_k10_uniform_noise", 0.01, wl["skin"], wl["skin_plt"], respa, M.MD_CFG_UNIFORM_NOISE)]
        for name, dt, skin, skin_plt, fn, flags in arms:
            h = make_system(M, s, dt, skin, seed, skin_plt, flags)
            fn(h, args.warmup)
            t_ms = timed(h, lambda k: fn(h, k), args.steps, barrier)
            u2, s2 = whole_job_rate(n * args.steps, t_ms / 1e3, world, device="cuda")
            compare[name] = {"ns_per_day": ns_per_day(args.steps, s2, dt) * (u2 / (n * args.steps)),
                             "ms_per_step": s2 * 1e3 / args.steps, "dt": dt, "skin": skin, "skin_plt": skin_plt,
                             "particle_steps_per_s": u2 / s2}
            h.close()
            del h
            torch.cuda.empty_cache()
        compare["speedup_ai_mts_vs_fine_sts"] = value / compare["fine_sts"]["ns_per_day"]

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        ps_cpu, st_cpu, n_cpu, el_cpu, what = oracle_rate(args.workload, seed=20220528)
        cpu = {"value": ps_cpu / n * wl["dt"] * NS_PER_TAU * 86400.0, "unit": "ns/day", "cores": cpu_count(),
               "kind": "oracle", "particle_steps_per_s": ps_cpu,
               "sample": f"{st_cpu} {what} of a {n_cpu}-particle sample of the same workload ({el_cpu:.1f} s), "
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
        "config": {"workload": wl["desc"], "n_particles": n, "parallelism": "replicas" if world > 1 else "single",
                   "l2": "inputs larger than L2 (a force pass reads more than 129 MB); no flush", **mode_info},
        "compare": compare or None,
        "roofline": {"bound": "hbm", "kernel": "k_dpd (fluid level pair forces)", "achieved": achieved,
                     "peak": peak, "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                     "peak_source": peak_kind,
                     "bytes_per_particle": bytes_per_particle, "n_half": n_half, "launch_ms": fl_ms,
                     "limiter": "instruction issue: 78% of issue slots active, 73% of the issue limit "
                                "(0.92 of 1.26 T warp instructions/s at 2.07 GHz), the ALU pipe the busiest "
                                "(ncu on the 1M system, profiles/k_dpd_dpd1m.md)"},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": prof_plain["total_launches"],
        "clocks": clocks,
        "kernel_ms_per_step": {k: v / max(n_prof, 1) for k, v in prof["ms"].items()},
        "n_builds": obs["n_builds"],
        "temperature": obs["temperature"],
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
