#!/usr/bin/env python
"""Throughput benchmark of the DPD-CGMD engine on synthetic systems.

Default workload (N = 1): the paper-scale clot channel -- about 101 M
particles in a 1,100 x 300 x 93 channel with frozen walls in y and a
Poiseuille body force (wall shear rate 0.05): 250 platelets of 40,000
coarse-grained particles (two wall-attached aggregates of 90 on opposite
walls at the same x, 70 in the flow) and plasma at rho = 3 around and inside
them.  The system is first relaxed from its synthetic start and a full
feature window recorded, untimed; the timed arm is AI-MTS: outer steps of
dt_f = 0.01 (one reduced time unit = 166.4 ns, so 1.664 ns per step), two
interface substeps, per-platelet step ratios from the trained controller
(decided on the device).  Beside it, from the same relaxed state, fine-step
STS (velocity-Verlet with dt = 0.001 for every particle, the reference of
Sec. 4.1) and fixed-k RESPA (k = 10).

``--workload channel``: the 8.3 M-particle platelet channel (400 x 100 x 67,
16 platelets of 10,000).  ``--workload dpd1m``: the DPD-only throughput
system (1,000,000 plasma particles in a 69.336^3 box, walls, g = 0.02, STS
dt = 0.01, skin 0.3).

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
K_M = 2                     # interface substeps per fluid step (Table 1), the ratio the controller was trained at
PAPER_LJ_RC = 0.8 * 2.0 ** (1.0 / 6.0)


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=150)
    ap.add_argument("--impl", default="msm", choices=["msm", "reference"])
    ap.add_argument("--workload", default="paper", choices=["paper", "channel", "dpd1m"])
    ap.add_argument("--relax", type=int, default=400,
                    help="untimed outer steps that relax the synthetic start before the feature window")
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
    if name == "paper":
        from paper_2205_14121_gb300._binding import MD_CFG_MORSE_STANDARD
        # Inter-platelet terms of the 40,000-particle shells (23 particles
        # per unit area, spacing 0.21 against sigma = 0.8): LJ cut at its
        # minimum, 2^(1/6) sigma (excluded volume only; with the 2.5 sigma
        # cut-off the summed attraction of two such membranes zips the
        # aggregates' shells together and their LJ rows grow past 800), and
        # the receptor Morse term in its standard form with range alpha = 2
        # (with the printed form's range alpha / (2 r0) = 1 the aggregates'
        # shells overlap within about 100 outer steps).
        return synth.config_paper_scale(seed=seed), dict(
            dt=0.01, skin=0.3, skin_plt=0.5, flags=MD_CFG_MORSE_STANDARD, params=dict(lj_rc=PAPER_LJ_RC),
            desc="paper-scale clot channel: ~101M particles, plasma at rho=3 in 1100x300x93, y walls, Poiseuille g "
                 "for wall shear rate 0.05, 250 platelets x 40,000 CG particles (5% receptors; LJ eps=1, "
                 "sigma=0.8 cut at 2^(1/6) sigma; standard-form Morse D=2, alpha=2, r0=1; two wall-attached "
                 "aggregates of 90 at the same x on opposite walls, 70 in the flow); AI-MTS dt_f=0.01, "
                 f"k_m={K_M}, per-platelet k from the controller vs fine-step STS dt=0.001; skin 0.3, "
                 "platelet skin 0.5")
    if name == "channel":
        return synth.config_channel_platelets(seed=seed), dict(
            dt=0.01, skin=0.3, skin_plt=0.5,
            desc="platelet channel: 8,040,000 plasma at rho=3 in 400x100x67, y walls, Poiseuille g for wall "
                 "shear rate 0.05, 16 platelets x 10,000 CG particles (5% receptors); AI-MTS dt_f=0.01, "
                 f"k_m={K_M}, "
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
            self.kw = dict(X0=s.X0, bonds=s.bonds, r0=s.r0, dt_f=0.01, k_m=K_M)
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


def make_system(M, s, dt, skin, seed, skin_plt=0.0, flags=0, params=None):
    return M.System(s.box, s.x, s.v, s.tag, X0=s.X0, bonds=s.bonds, r0=s.r0, angles=s.angles,
                    theta0=s.theta0, walls=s.walls, wall=s.wall,
                    shear_rate=s.shear_rate, body_force=s.body_force, dt=dt, skin=skin, seed=seed,
                    skin_plt=skin_plt, flags=flags, **(params or {}))


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


def traffic_entry(workload_name, skin, n):
    """DRAM bytes per launch of the fluid DPD kernel from a committed ncu
    summary taken on the current kernel source and list skin: the workload's
    own capture, else the platelet channel's scaled by the rows (a capture of
    the paper-scale system would hold more device memory than an ncu replay
    should).  Returns (bytes, note) or (None, reason)."""
    path = os.path.join(ROOT, "profiles", "k_dpd_traffic.json")
    try:
        d = json.load(open(path))
    except Exception:
        return None, "no committed capture"
    e = d.get(workload_name)
    scaled = False
    if e is None and workload_name == "paper":
        e, scaled = d.get("channel"), True
    if not e or e.get("source_hash") != kernel_source_hash() or e.get("skin") != skin:
        return None, "the committed capture predates the current kernel source"
    b = float(e["dram_bytes_per_launch"])
    if scaled:
        return b * n / float(e["rows"]), f"channel capture ({e['rows']} rows) scaled to {n} rows"
    return b, "ncu capture of this workload"


def issue_limiter(workload_name, launch_ms, n, sm_mhz):
    """The fluid DPD pass against its two on-chip limits at the sampled SM
    clock: warp-instruction issue (152 SMs x 4 schedulers x 1 per cycle) and
    the L1 data pipe (152 SMs x 1 LSU wavefront per cycle), with the per-row
    counts of a committed ncu capture of the current kernel source (the
    channel's); None without one."""
    path = os.path.join(ROOT, "profiles", "k_dpd_traffic.json")
    try:
        d = json.load(open(path))
        e = d.get("instructions")
        if not e or e.get("source_hash") != kernel_source_hash() or not sm_mhz:
            return None
        per_row = float(e["warp_inst_per_row"])
        sec = launch_ms * 1e-3
        out = {"warp_inst_per_row": per_row,
               "issue_fraction": per_row * n / sec / (152 * 4 * sm_mhz * 1e6),
               "source": e.get("command", "")}
        c = d.get("channel", {})
        if c.get("source_hash") == kernel_source_hash() and c.get("l1_wavefronts_per_launch"):
            wf = float(c["l1_wavefronts_per_launch"]) / float(c["rows"])
            out["l1_wavefronts_per_row"] = wf
            out["l1_wavefront_fraction"] = wf * n / sec / (152 * sm_mhz * 1e6)
        return out
    except Exception:
        return None


_T0 = time.time()


def progress(msg):
    """Phase marks on stderr (the JSON line goes to stdout)."""
    print(f"[bench {time.time() - _T0:7.1f} s] {msg}", file=sys.stderr, flush=True)


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
    t_gen = time.perf_counter()
    s, wl = workload(args.workload, seed=seed)
    t_gen = time.perf_counter() - t_gen
    n = s.n
    progress(f"generated {args.workload}: {n} particles in {t_gen:.1f} s")
    platelets = args.workload != "dpd1m"
    g = make_system(M, s, wl["dt"], wl["skin"], seed, wl.get("skin_plt", 0.0), wl.get("flags", 0), wl.get("params"))

    mode_info = {"generation_s": t_gen}
    decisions = []
    ctl = None
    if platelets:
        if os.path.exists(CONTROLLER):
            ctl, trust = A.load_controller(CONTROLLER)
            mode_info["controller"] = os.path.relpath(CONTROLLER, ROOT)
        else:
            trust = A.TrustBound()
            mode_info["controller"] = "absent: fixed k = 10 for every platelet"

        def step(k):
            if ctl is None:
                g.set_platelet_levels(np.full(g.cfg.n_platelets, trust.fallback_k, np.int32))
                g.mts_step(k, mode=M.MD_MODE_AI, k_m=K_M, direct=args.direct, record=True)
            else:
                A.run_ai_mts(g, ctl, k, k_m=K_M, trust=trust, log=decisions, direct=args.direct)

        # an equilibrated start independent of --warmup: relax the synthetic
        # state at the fallback ratio, then record one full feature window
        g.set_platelet_levels(np.full(g.cfg.n_platelets, trust.fallback_k, np.int32))
        t_rel = time.perf_counter()
        g.mts_step(args.relax, mode=M.MD_MODE_AI, k_m=K_M, direct=args.direct)
        if ctl is not None:
            A.run_ai_mts(g, ctl, 128, k_m=K_M, trust=trust, direct=args.direct)        # fills the window, no decision yet
        torch.cuda.synchronize()
        mode_info["relax"] = {"steps": args.relax + (128 if ctl is not None else 0),
                              "s": time.perf_counter() - t_rel, "temperature": g.observables()["temperature"]}
    else:
        def step(k):
            g.mts_step(k, direct=args.direct)
        g.mts_step(args.relax, direct=args.direct)
    progress(f"relaxed: {mode_info.get('relax')}")
    # the relaxed state every comparison arm starts from
    x_rel, v_rel, _ = g.read_particles()

    # warm-up (graph capture of the timed call shape)
    step(args.warmup)
    torch.cuda.synchronize()
    decisions.clear()

    progress("warm-up done")
    # ---- timed region --------------------------------------------------
    g.profile_read(reset=True)
    builds0 = g.observables()["n_builds"]
    import tempfile
    clk_path = os.path.join(args.clock_log or tempfile.gettempdir(), f"clocks_rank{rank}.csv")
    os.makedirs(os.path.dirname(clk_path), exist_ok=True)
    with ClockSampler(clk_path) as clk:
        ms = timed(g, step, args.steps, barrier)
    prof_plain = g.profile_read(reset=True)
    obs_t = g.observables()
    units, sec = whole_job_rate(n * args.steps, ms / 1e3, world, device="cuda")
    ms = sec * 1e3
    ps = units / sec
    value = ns_per_day(args.steps, sec, wl["dt"]) * (units / (n * args.steps))
    mode_info["timed_builds"] = obs_t["n_builds"] - builds0
    if platelets:
        ks = [k for d in decisions for k in d["k"]]
        mode_info["decisions"] = len(decisions)
        mode_info["mean_k"] = float(np.mean(ks)) if ks else None
        mode_info["fallback_fraction"] = (float(np.mean([u for d in decisions for u in d["unsure"]]))
                                          if decisions else None)
        mode_info["mode"] = "AI-MTS" if decisions else "fixed-k fallback (no controller decision in the timed steps)"
    else:
        mode_info["mode"] = "STS"

    progress(f"timed: {ms / args.steps:.2f} ms per step, {mode_info.get('decisions')} decisions")
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
    traffic, traffic_note = traffic_entry(args.workload, wl["skin"], n)

    # ---- the controller's cost: one decision for every platelet ----------
    ctl_info = None
    if ctl is not None:
        for _ in range(2):
            ctl.decide_system(g, trust)
        t0 = time.perf_counter()
        reps = 10
        for _ in range(reps):
            ctl.decide_system(g, trust)
        us = (time.perf_counter() - t0) / reps * 1e6
        holds = [h for d in decisions for h in d["hold"]]
        hold_min = float(np.mean([min(d["hold"]) for d in decisions])) if decisions else None
        ctl_info = {"us_per_decision": us, "platelets_per_decision": g.cfg.n_platelets,
                    "note": "md_ai_decide_system: ring gather, denoise, GRU autoencoder, heads, trust bound and "
                            "ratio map on the device, P decisions copied back; wall clock per call",
                    "share_of_step_at_mean_hold": (us * 1e-3 / hold_min) / (ms / args.steps) if hold_min else None,
                    "mean_hold": float(np.mean(holds)) if holds else None}

    progress("roofline pass and controller timing done")
    # ---- end to end through the C ABI with host buffers ------------------
    e2e = None
    if args.e2e_steps > 0:
        levels = np.asarray(decisions[-1]["k"] if decisions else
                            [10] * (g.cfg.n_platelets if platelets else 0), np.int32)
        # the particle set (tags, rest positions, bonds) is configuration and
        # stays on the device; every step uploads a state and reads results
        g.set_particles(s.x, s.v, s.tag, s.X0, step0=0)

        def one_step():
            if platelets:
                g.set_platelet_levels(levels)
                g.mts_step(1, mode=M.MD_MODE_AI, k_m=K_M)
            else:
                g.mts_step(1)

        # states that change from step to step: the relaxed state and the
        # state one outer step later, uploaded in turn from page-locked memory
        g.set_xv(x_rel, v_rel, step0=0)
        one_step()
        x2, v2, _ = g.read_particles()
        states = [(torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy(),
                   torch.from_numpy(np.ascontiguousarray(b)).pin_memory().numpy())
                  for a, b in ((x_rel, v_rel), (x2, v2))]
        del x2, v2

        def e2e_step(k):
            xh, vh = states[k % 2]
            g.set_xv(xh, vh, step0=k)
            one_step()
            return g.observables()

        for k in range(2):       # warm-up: the first list build and graph capture of a one-step call
            e2e_step(k)
        barrier()
        b0 = g.observables()["n_builds"]
        t0 = time.perf_counter()
        for k in range(args.e2e_steps):
            o_last = e2e_step(k)
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        xh, vh = states[0]
        e2e = {"value": ns_per_day(args.e2e_steps, el, wl["dt"]) * world, "unit": "ns/day",
               "h2d_bytes_per_step": int(xh.nbytes + vh.nbytes + 4 * len(levels)),
               "d2h_bytes_per_step": 3 * (16 * 4 + 64) + 16 * 8 + 9 * 8,
               "builds_in_timed_steps": int(o_last["n_builds"] - b0),
               "note": "per step: upload of x and v (the relaxed state and the state one step later, in turn) from "
                       "page-locked host memory (md_set_xv; tags, rest positions and bonds set once before timing), "
                       "a list rebuild when the uploaded state fails the rebuild check, forces of the new state, one "
                       "outer step, observables read back; two untimed warm-up steps"}
        del states
    g.close()
    del g
    torch.cuda.empty_cache()

    progress(f"e2e done: {e2e['value'] if e2e else None}")
    # ---- comparison arms on the same system, from the relaxed state -------
    compare = {}
    if platelets and not args.no_compare:
        # each arm at the Verlet skins that suit it (sweeps of the plasma skin
        # over 0.15-0.6 and of the platelet skin over 0.2-0.9 on the channel:
        # fine-step STS rebuilds rarely and prefers the shorter lists of skin
        # 0.2; the dt = 0.01 arms' platelet particles, which tripped most
        # rebuilds, get a skin of 0.5)
        respa = lambda h, k: h.mts_step(k, mode=M.MD_MODE_RESPA, k_m=K_M, k_p=10, direct=args.direct)
        fl = wl.get("flags", 0)
        arms = [("fine_sts", 0.001, 0.2, FINE_SKIN_PLT, lambda h, k: h.mts_step(k, direct=args.direct), fl),
                ("respa_k10", 0.01, wl["skin"], wl["skin_plt"], respa, fl)]
        rel = type(s)(box=s.box, x=x_rel, v=v_rel, tag=s.tag, X0=s.X0, bonds=s.bonds, r0=s.r0, angles=s.angles,
                      theta0=s.theta0, walls=s.walls,
                      wall=s.wall, shear_rate=s.shear_rate, body_force=s.body_force, n_platelets=s.n_platelets)
        for name, dt, skin, skin_plt, fn, flags in arms:
            h = make_system(M, rel, dt, skin, seed, skin_plt, flags, wl.get("params"))
            fn(h, max(args.warmup, 3))
            t_ms = timed(h, lambda k: fn(h, k), args.steps, barrier)
            u2, s2 = whole_job_rate(n * args.steps, t_ms / 1e3, world, device="cuda")
            compare[name] = {"ns_per_day": ns_per_day(args.steps, s2, dt) * (u2 / (n * args.steps)),
                             "ms_per_step": s2 * 1e3 / args.steps, "dt": dt, "skin": skin, "skin_plt": skin_plt,
                             "particle_steps_per_s": u2 / s2}
            h.close()
            del h
            torch.cuda.empty_cache()
            progress(f"arm {name}: {compare[name]['ms_per_step']:.2f} ms per step")
        compare["speedup_vs_fine_sts"] = value / compare["fine_sts"]["ns_per_day"]
        compare["speedup_vs_respa_k10"] = value / compare["respa_k10"]["ns_per_day"]
        compare["note"] = ("every arm starts from the same relaxed state; speed-ups are of the timed arm "
                           f"({mode_info['mode']})")

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
    limiter = issue_limiter(args.workload, fl_ms, n, clocks["sm_mhz"] if clocks else None)
    line = {
        "metric": METRIC, "value": value, "unit": "ns/day", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "particle_steps_per_s": ps,
        "config": {"workload": wl["desc"], "n_particles": n, "parallelism": "replicas" if world > 1 else "single",
                   "l2": "inputs larger than L2 (a force pass reads more than 129 MB); no flush", **mode_info},
        "compare": compare or None,
        "controller": ctl_info,
        "roofline": {"bound": "hbm", "kernel": "k_dpd (fluid level pair forces)", "achieved": achieved,
                     "peak": peak, "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                     "traffic_note": traffic_note, "peak_source": peak_kind,
                     "bytes_per_particle": bytes_per_particle, "n_half": n_half, "launch_ms": fl_ms,
                     "rows": n, "limiter": limiter},
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
