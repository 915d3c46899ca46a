"""AI-MTS (Sec. 3.3, Table 2): the controller-driven time stepping loop and
the pipeline that trains the controller on trajectories of this code.

Every step of the simulation and of the network runs in libmsm (md_mts_step,
the per-platelet measurements, md_ai_*); this module only sequences those
calls and keeps the bookkeeping: which windows were recorded, which step
ratio each one earned, when to ask the controller again.

Labels ("trial and error" made a procedure): from the state at the end of a
window, fixed-k continuations are run for every k of the class set and
compared with the finest one (k = 20) over the next `horizon` outer steps;
the label is the coarsest k (the largest platelet step dt_m / k) whose mean
principal stresses stay within 3% and whose mean centre-of-mass velocity
stays within 1% of the finest run (the tolerances of Sec. 4.2).  The hold
label is how long that label stays unchanged along the trajectory, clipped to
[100, 2000] steps.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np

from . import _binding as B
from .controller import K_SET, TRAIN_AE, TRAIN_HEADS, Controller, default_config, param_layout

GATE_STRESS = 0.03
GATE_VCOM = 0.01
HOLD_RANGE = (100.0, 2000.0)
F_VCOM = slice(0, 3)       # measurement columns: centre-of-mass velocity
F_STRESS = slice(6, 9)     # principal stresses
F_STRAIN = 9               # largest bond strain


@dataclass
class TrustBound:
    """Fallback to a fixed ratio when the controller is unsure (Table 2): the
    top class probability is low, or the window lies outside the training
    data (reconstruction error or bond strain beyond their 99th percentiles
    over the training windows).  Applied on the device by md_ai_decide."""
    p_min: float = 0.6           # smallest accepted top class probability
    rec_max: float = math.inf    # largest accepted reconstruction error
    strain_max: float = 0.2      # largest accepted bond strain in the window
    fallback_k: int = 10
    strain_col: int = F_STRAIN
    hold_range: tuple = HOLD_RANGE


def init_params(cfg, seed=0):
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights, zero biases."""
    rng = np.random.default_rng(seed)
    parts = []
    for name, shape in param_layout(cfg):
        if name.endswith(".W") or ".W_" in name:
            bound = 1.0 / math.sqrt(shape[-1])
            parts.append(rng.uniform(-bound, bound, size=shape).astype(np.float32).ravel())
        else:
            parts.append(np.zeros(int(np.prod(shape)), np.float32))
    return np.concatenate(parts)


def decide(controller, windows, trust):
    """Per-platelet ratio, hold and unsure flags for raw windows (Table 2
    steps 1-6, all on the device)."""
    d = controller.decide(windows, trust)
    return d["k"], d["hold"], d["unsure"]


def run_ai_mts(system, controller, n_steps, k_m=1, trust=None, T=128, log=None, direct=False):
    """Advance n_steps outer steps under AI-MTS: the measurements of the T
    steps before each decision go to the feature ring from inside the step
    graph; with a full window the controller sets each platelet's ratio and
    is asked again after the shortest predicted hold.  direct: launch every
    kernel from the host instead of replaying the step graph."""
    trust = trust or TrustBound()
    P = system.cfg.n_platelets
    # the ratios and the count of consecutive records at the end of the ring
    # carry over from one call to the next on the same system
    state = getattr(system, "_ai_mts_state", None)
    if state is None:
        system.set_platelet_levels(np.full(P, trust.fallback_k, np.int32))
        state = {"fresh": 0}
        system._ai_mts_state = state
    done = 0
    fresh = state["fresh"]
    while done < n_steps:
        count = system.feature_count()
        fresh = min(fresh, count)          # new particles restart the ring
        if fresh >= T:
            d = controller.decide_system(system, trust)
            k, hold, unsure = d["k"], d["hold"], d["unsure"]
            system.set_platelet_levels(k)
            run = int(hold.min())
            if log is not None:
                log.append(dict(step=done, k=k.tolist(), hold=hold.tolist(), unsure=unsure.tolist(),
                                why=d["why"].tolist()))
        else:
            run = T - fresh
        run = max(1, min(run, n_steps - done))
        # only the T steps before the next decision need recording
        quiet = max(0, run - T)
        if quiet:
            system.mts_step(quiet, mode=B.MD_MODE_AI, k_m=k_m, direct=direct)
            fresh = 0
        system.mts_step(run - quiet, mode=B.MD_MODE_AI, k_m=k_m, record=True, direct=direct)
        fresh += run - quiet
        done += run
    state["fresh"] = fresh
    return log


# ---------------------------------------------------------------------------
# training data
# ---------------------------------------------------------------------------

def training_system(seed, box=(36.0, 18.0, 16.0), n_shell=2000, shear_rate=0.05):
    """A walled channel with four platelets: two close to each other near the
    lower wall (in contact range, fast dynamics) and two placed at random in
    the flow."""
    import synth
    rng = np.random.default_rng(seed)
    Lx, Ly, Lz = box
    radii = synth.scaled_radii(n_shell)
    a = radii[0]
    x0 = rng.uniform(a + 1.0, Lx - 3 * a - 3.0)
    gap = rng.uniform(1.0, 1.8)
    centers = [(x0, a + 1.0, Lz / 2), (x0 + 2 * a + gap, a + 1.0 + rng.uniform(-0.3, 0.3), Lz / 2)]
    n_pl = int(round(3.0 * Lx * Ly * Lz))
    g = synth.poiseuille_g(shear_rate, synth.ETA_DPD, 3.0, Ly)
    return synth.platelet_system(box, n_pl, 4, n_shell, radii, walls=True, body_force=g, seed=seed,
                                 centers=centers)


def make_system(s, **kw):
    return B.System(s.box, s.x, s.v, s.tag, X0=s.X0, bonds=s.bonds, r0=s.r0, angles=s.angles,
                    theta0=s.theta0, walls=s.walls, wall=s.wall,
                    shear_rate=s.shear_rate, body_force=s.body_force, **kw)


def _means(records):
    return records[:, :, F_STRESS].mean(1), records[:, :, F_VCOM].mean(1)


def continuation_errors(system, horizon, k_m=1):
    """Relative errors [P][len(K_SET)] of each fixed-k continuation from the
    current state against the finest, for the mean principal stresses and
    the mean centre-of-mass velocity over `horizon` outer steps.  The state
    is restored afterwards."""
    blob = system.get_state()
    means = {}
    for k in K_SET:
        system.set_state(blob)
        try:
            system.mts_step(horizon, mode=B.MD_MODE_RESPA, k_m=k_m, k_p=k, record=True)
        except B.MdError as e:      # a ratio too coarse for these dynamics
            if e.code not in (-4, -5):
                raise
            means[k] = None
            continue
        rec, _ = system.read_feature_ring()
        means[k] = _means(rec[:, -horizon:])
    system.set_state(blob)
    if means[K_SET[-1]] is None:
        return None, None
    s_ref, v_ref = means[K_SET[-1]]
    for k in K_SET:
        if means[k] is None:
            means[k] = (np.full_like(s_ref, np.inf), np.full_like(v_ref, np.inf))
    v_scale = np.linalg.norm(v_ref, axis=1) + 0.05
    s_scale = np.linalg.norm(s_ref, axis=1) + 1e-6
    es = np.stack([np.linalg.norm(means[k][0] - s_ref, axis=1) / s_scale for k in K_SET], 1)
    ev = np.stack([np.linalg.norm(means[k][1] - v_ref, axis=1) / v_scale for k in K_SET], 1)
    return es, ev


def label_from_errors(es, ev):
    """Class of the coarsest k within both tolerances (the finest when none is)."""
    ok = (es <= GATE_STRESS) & (ev <= GATE_VCOM)
    ok[:, -1] = True
    return ok.argmax(1).astype(np.int32)


def hold_labels(classes, stride):
    """Steps for which each window's label stays unchanged along the
    trajectory: classes [W][P] -> hold [W][P]."""
    W, P = classes.shape
    hold = np.zeros((W, P))
    for p in range(P):
        run = 0
        for w in range(W - 1, -1, -1):
            run = run + 1 if (w + 1 < W and classes[w + 1, p] == classes[w, p]) else 1
            hold[w, p] = run * stride
    return np.clip(hold, *HOLD_RANGE)


@dataclass
class Dataset:
    windows: list = field(default_factory=list)    # [P][T][F] raw windows
    classes: list = field(default_factory=list)    # [P]
    holds: list = field(default_factory=list)      # [P]
    err_s: list = field(default_factory=list)      # [P][len(K_SET)]
    err_v: list = field(default_factory=list)

    def arrays(self):
        cat = lambda xs: np.concatenate(xs, 0)
        return (cat(self.windows).astype(np.float32), cat(self.classes), cat(self.holds), cat(self.err_s),
                cat(self.err_v))


def generate(seeds, n_windows=8, warmup=50, horizon=50, k_m=1, k_record=10, T=128, n_shell=2000, progress=None,
             system_kw=None):
    """Windows of per-platelet measurements under fixed-k RESPA (k_record),
    each labelled from the continuations at its end.  system_kw: further
    System configuration (force-field fields and flags)."""
    data = Dataset()
    for seed in seeds:
        # platelets in contact: long LJ rows
        sys = make_system(training_system(seed, n_shell=n_shell), seed=int(seed), caps={"lj": 4096},
                          **(system_kw or {}))
        try:
            sys.mts_step(warmup, mode=B.MD_MODE_RESPA, k_m=k_m, k_p=k_record)
        except B.MdError as e:
            if e.code not in (-4, -5):
                raise
            sys.close()
            continue
        wins, cls, es_all, ev_all = [], [], [], []
        for w in range(n_windows):
            blob = sys.get_state()
            sys.set_state(blob)                      # restart the ring at this window
            try:
                sys.mts_step(T, mode=B.MD_MODE_RESPA, k_m=k_m, k_p=k_record, record=True)
            except B.MdError as e:
                if e.code not in (-4, -5):
                    raise
                break                                # this trajectory went unstable
            win, cnt = sys.read_feature_ring()
            es, ev = continuation_errors(sys, horizon, k_m=k_m)
            if es is None:
                break
            wins.append(win)
            cls.append(label_from_errors(es, ev))
            es_all.append(es)
            ev_all.append(ev)
        sys.close()
        if not cls:
            continue
        classes = np.stack(cls)
        holds = hold_labels(classes, T)
        for w in range(len(cls)):
            data.windows.append(wins[w])
            data.classes.append(classes[w])
            data.holds.append(holds[w])
            data.err_s.append(es_all[w])
            data.err_v.append(ev_all[w])
        if progress:
            progress(seed, classes)
    return data


# ---------------------------------------------------------------------------
# training
# ---------------------------------------------------------------------------

def _batches(n, size, rng):
    idx = rng.permutation(n)
    for b in range(0, n, size):
        yield idx[b:b + size]


def train(windows, classes, holds, epochs_ae=40, epochs_heads=80, batch=128, lr_ae=2e-3, lr_heads=3e-3, seed=0,
          progress=None):
    """Autoencoder first (reconstruction), then the heads on its latent
    (Sec. 3.3 trains them separately).  Returns (controller, artefacts)."""
    cfg = default_config(batch_max=batch)
    ctl = Controller(cfg)
    ctl.set_params(init_params(cfg, seed))
    n = windows.shape[0]
    den = np.concatenate([ctl.prepare(windows[b:b + batch]) for b in range(0, n, batch)])
    mean = den.reshape(-1, cfg.F).mean(0)
    std = den.reshape(-1, cfg.F).std(0) + 1e-6
    ctl.set_norm(mean, std)
    x = np.concatenate([ctl.prepare(windows[b:b + batch]) for b in range(0, n, batch)])
    rng = np.random.default_rng(seed)
    hist = {"ae": [], "heads": []}
    for ep in range(epochs_ae):
        losses = [ctl.train_step(x[i], TRAIN_AE, lr_ae) for i in _batches(n, batch, rng)]
        hist["ae"].append(float(np.mean(losses)))
        if progress:
            progress("ae", ep, hist["ae"][-1])
    log_hold = np.log(holds).astype(np.float32)
    for ep in range(epochs_heads):
        losses = [ctl.train_step(x[i], TRAIN_HEADS, lr_heads, k_class=classes[i], log_hold=log_hold[i])
                  for i in _batches(n, batch, rng)]
        hist["heads"].append(float(np.mean(losses)))
        if progress:
            progress("heads", ep, hist["heads"][-1])
    rec = np.concatenate([ctl.predict(windows[b:b + batch])["rec_err"] for b in range(0, n, batch)])
    art = dict(params=ctl.get_params(), mean=mean.astype(np.float32), std=std.astype(np.float32),
               rec_p99=np.float32(np.percentile(rec, 99)),
               strain_p99=np.float32(np.percentile(windows[:, :, F_STRAIN].max(1), 99)), history=hist)
    return ctl, art


def load_controller(path, batch=256):
    """Controller with the parameters, normalisation and trust bound saved by `save`."""
    d = np.load(path)
    ctl = Controller(default_config(batch_max=batch))
    ctl.set_params(d["params"])
    ctl.set_norm(d["mean"], d["std"])
    strain = float(d["strain_p99"]) if "strain_p99" in d.files else TrustBound.strain_max
    p_min = float(d["p_min"]) if "p_min" in d.files else TrustBound.p_min
    return ctl, TrustBound(rec_max=float(d["rec_p99"]), strain_max=strain, p_min=p_min)


def save(path, art):
    np.savez(path, params=art["params"], mean=art["mean"], std=art["std"], rec_p99=art["rec_p99"],
             strain_p99=art["strain_p99"], p_min=art.get("p_min", TrustBound.p_min))


def gains(c, fb):
    """A policy's gain over another: strictly better on one of (violations,
    mean ratio) and no worse on the other."""
    return ((c["violations"] <= fb["violations"] and c["mean_k"] < fb["mean_k"]) or
            (c["violations"] < fb["violations"] and c["mean_k"] <= fb["mean_k"]))


P_MIN_GRID = (0.4, 0.45, 0.5, 0.55, 0.6, 0.65, 0.7, 0.8)


def gain_margin(c, fb):
    """The larger of the policy's two ratios to the other's (violations, mean
    ratio): below 1 on both axes means a gain on both, and the smaller the
    value, the wider the gain on the weaker axis."""
    if fb["violations"] > 0:
        rv = c["violations"] / fb["violations"]
    else:
        rv = 0.0 if c["violations"] == 0 else math.inf
    return max(rv, c["mean_k"] / fb["mean_k"])


def select_trust(ctl, trust, windows, err_s, err_v, grid=P_MIN_GRID):
    """The top-probability bound of the trust test chosen on training windows:
    among the bounds whose policy gains over fixed-k at the fallback ratio,
    the one with the widest gain on its weaker axis (smallest gain_margin);
    the given bound when none gains.  Returns (trust, evaluations per bound)."""
    best, table = None, {}
    for p in grid:
        t = replace(trust, p_min=float(p))
        r = evaluate(ctl, windows, err_s, err_v, t)
        c, fb = r["controller"], r[f"fixed_k{t.fallback_k}"]
        m = gain_margin(c, fb)
        table[float(p)] = dict(c, gain=gains(c, fb), margin=m)
        if gains(c, fb) and (best is None or m < best[0]):
            best = (m, t)
    return (best[1] if best else trust), table


def evaluate(ctl, windows, err_s, err_v, trust, batch=128):
    """Policies on labelled windows: the violation rate of the tolerances and
    the mean step ratio (cost of the platelet level) of the controller and of
    every fixed ratio."""
    n = windows.shape[0]
    ks, unsure = [], []
    for b in range(0, n, batch):
        k, _, u = decide(ctl, windows[b:b + batch], trust)
        ks.append(k)
        unsure.append(u)
    k = np.concatenate(ks)
    unsure = np.concatenate(unsure)
    col = np.searchsorted(np.array(K_SET), k)
    viol = lambda c: float(np.mean((err_s[np.arange(n), c] > GATE_STRESS) | (err_v[np.arange(n), c] > GATE_VCOM)))
    out = {"controller": {"violations": viol(col), "mean_k": float(k.mean()),
                          "fallback_fraction": float(unsure.mean()),
                          "k_counts": [int((k == kk).sum()) for kk in K_SET]}}
    for j, kk in enumerate(K_SET):
        out[f"fixed_k{kk}"] = {"violations": viol(np.full(n, j)), "mean_k": float(kk)}
    return out


# ---------------------------------------------------------------------------
# the paper's own variant (Sec. 3.3): LSTM autoencoder + FCN on log k
# ---------------------------------------------------------------------------

def lstm_windows(windows, T=50):
    """The variant's input from recorded windows: the last T steps of its six
    measurement columns (controller.LSTM_COLUMNS)."""
    from .controller import LSTM_COLUMNS
    return np.ascontiguousarray(windows[:, -T:, list(LSTM_COLUMNS)], np.float32)


def train_lstm(windows, classes, epochs_ae=60, epochs_fcn=120, batch=128, lr_ae=3e-3, lr_fcn=3e-3, seed=0):
    """The variant trained on the same labelled windows: the autoencoder
    first, then the FCN on log k of the label (Sec. 3.3 trains them
    separately).  Returns (model, artefacts)."""
    from .controller import LSTMController, lstm_config, lstm_param_layout
    cfg = lstm_config(batch_max=batch)
    m = LSTMController(cfg)
    rng = np.random.default_rng(seed)
    parts = []
    for name, shape in lstm_param_layout(cfg):
        if ".W" in name:
            bound = 1.0 / math.sqrt(shape[-1])
            parts.append(rng.uniform(-bound, bound, size=shape).astype(np.float32).ravel())
        else:
            parts.append(np.zeros(int(np.prod(shape)), np.float32))
    m.set_params(np.concatenate(parts))
    raw = lstm_windows(windows)
    n = raw.shape[0]
    den = np.concatenate([m.prepare(raw[b:b + batch]) for b in range(0, n, batch)])
    mean = den.reshape(-1, cfg.F).mean(0)
    std = den.reshape(-1, cfg.F).std(0) + 1e-6
    m.set_norm(mean, std)
    x = np.concatenate([m.prepare(raw[b:b + batch]) for b in range(0, n, batch)])
    lk = np.log(np.asarray(K_SET, np.float64)[classes]).astype(np.float32)
    hist = {"ae": [], "fcn": []}
    for _ in range(epochs_ae):
        hist["ae"].append(float(np.mean([m.train_step(x[i], TRAIN_AE, lr_ae) for i in _batches(n, batch, rng)])))
    for _ in range(epochs_fcn):
        hist["fcn"].append(float(np.mean([m.train_step(x[i], TRAIN_HEADS, lr_fcn, log_k=lk[i])
                                          for i in _batches(n, batch, rng)])))
    return m, dict(params=m.get_params(), mean=mean.astype(np.float32), std=std.astype(np.float32), history=hist)


def evaluate_lstm(m, windows, err_s, err_v, batch=128):
    """The variant's policy on labelled windows (the class nearest its log k;
    the paper describes no trust bound for it)."""
    n = windows.shape[0]
    raw = lstm_windows(windows)
    k = np.concatenate([m.predict(raw[b:b + batch])["k"] for b in range(0, n, batch)])
    col = np.searchsorted(np.array(K_SET), k)
    bad = (err_s[np.arange(n), col] > GATE_STRESS) | (err_v[np.arange(n), col] > GATE_VCOM)
    return {"violations": float(bad.mean()), "mean_k": float(k.mean()),
            "k_counts": [int((k == kk).sum()) for kk in K_SET]}
