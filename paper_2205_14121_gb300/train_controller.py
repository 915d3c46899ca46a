"""Train the AI-MTS controller (Sec. 3.3) on trajectories of this code.

    python -m paper_2205_14121_gb300.train_controller --out paper_2205_14121_gb300/data/controller.npz

Generates labelled windows of per-platelet measurements (see ai_mts), trains
the autoencoder and the heads on the GPU, evaluates the controller against
fixed step ratios on held-out trajectories and writes the parameters plus a
JSON summary next to them.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=os.path.join(ROOT, "paper_2205_14121_gb300", "data", "controller.npz"))
    ap.add_argument("--train-seeds", type=int, default=24)
    ap.add_argument("--test-seeds", type=int, default=6)
    ap.add_argument("--windows", type=int, default=8)
    ap.add_argument("--horizon", type=int, default=50)
    ap.add_argument("--n-shell", type=int, default=2000)
    ap.add_argument("--k-m", type=int, default=2, help="interface substeps per fluid step (Table 1 k_m)")
    ap.add_argument("--epochs-ae", type=int, default=40)
    ap.add_argument("--epochs-heads", type=int, default=80)
    ap.add_argument("--dataset", default=None, help="save / reuse the labelled windows here (.npz)")
    ap.add_argument("--lj-rc", type=float, default=None,
                    help="inter-platelet LJ cut-off of the training systems (default: the configuration's 2.0)")
    ap.add_argument("--morse-standard", action="store_true",
                    help="receptor Morse term in its standard form (MD_CFG_MORSE_STANDARD)")
    ap.add_argument("--select-only", action="store_true",
                    help="keep the trained parameters in --out; choose the trust bound again on --dataset")
    args = ap.parse_args(argv)

    from paper_2205_14121_gb300 import ai_mts as A
    from paper_2205_14121_gb300 import build as Bld
    from paper_2205_14121_gb300._binding import MD_CFG_MORSE_STANDARD
    Bld.build()

    if args.select_only:
        return reselect(args, A)
    t0 = time.time()
    seeds_train = list(range(1000, 1000 + args.train_seeds))
    seeds_test = list(range(5000, 5000 + args.test_seeds))

    def progress(seed, classes):
        print(f"seed {seed}: classes per window {classes.tolist()}  ({time.time() - t0:.0f} s)", flush=True)

    if args.dataset and os.path.exists(args.dataset):
        d = np.load(args.dataset)
        tr = [d[f"train_{k}"] for k in ("w", "c", "h", "es", "ev")]
        te = [d[f"test_{k}"] for k in ("w", "c", "h", "es", "ev")]
    else:
        system_kw = {}
        if args.lj_rc is not None:
            system_kw["lj_rc"] = args.lj_rc
        if args.morse_standard:
            system_kw["flags"] = MD_CFG_MORSE_STANDARD
        kw = dict(n_windows=args.windows, horizon=args.horizon, n_shell=args.n_shell, progress=progress, k_m=args.k_m,
                  system_kw=system_kw)
        tr = A.generate(seeds_train, **kw).arrays()
        te = A.generate(seeds_test, **kw).arrays()
        if args.dataset:
            np.savez(args.dataset, **{f"train_{k}": a for k, a in zip(("w", "c", "h", "es", "ev"), tr)},
                     **{f"test_{k}": a for k, a in zip(("w", "c", "h", "es", "ev"), te)})
    t_data = time.time() - t0
    w_tr, c_tr, h_tr, es_tr, ev_tr = tr
    w_te, c_te, h_te, es_te, ev_te = te
    print(f"{len(c_tr)} training windows, {len(c_te)} held out; class counts "
          f"{np.bincount(c_tr, minlength=5).tolist()} / {np.bincount(c_te, minlength=5).tolist()}", flush=True)

    def prog(what, ep, loss):
        if ep % 10 == 0:
            print(f"{what} epoch {ep}: loss {loss:.4f}", flush=True)

    ctl, art = A.train(w_tr, c_tr, h_tr, epochs_ae=args.epochs_ae, epochs_heads=args.epochs_heads, progress=prog)
    t_train = time.time() - t0 - t_data
    trust = A.TrustBound(rec_max=float(art["rec_p99"]), strain_max=float(art["strain_p99"]))
    trust, p_table = A.select_trust(ctl, trust, w_tr, es_tr, ev_tr)
    art["p_min"] = trust.p_min
    ev_train = A.evaluate(ctl, w_tr, es_tr, ev_tr, trust)
    ev_test = A.evaluate(ctl, w_te, es_te, ev_te, trust)
    pred_te = np.concatenate([ctl.predict(w_te[b:b + 128])["cls"] for b in range(0, len(c_te), 128)])
    # the paper's own LSTM variant on the same windows, for comparison
    lstm, lart = A.train_lstm(w_tr, c_tr)
    lstm_test = A.evaluate_lstm(lstm, w_te, es_te, ev_te)
    os.makedirs(os.path.dirname(args.out), exist_ok=True)
    A.save(args.out, art)
    np.savez(os.path.splitext(args.out)[0] + "_lstm.npz", params=lart["params"], mean=lart["mean"], std=lart["std"])
    np.savez(os.path.splitext(args.out)[0] + "_heldout.npz", w=w_te, c=c_te, h=h_te, es=es_te, ev=ev_te)
    summary = dict(train_windows=int(len(c_tr)), test_windows=int(len(c_te)),
                   class_counts_train=np.bincount(c_tr, minlength=5).tolist(),
                   class_counts_test=np.bincount(c_te, minlength=5).tolist(),
                   test_class_accuracy=float(np.mean(pred_te == c_te)),
                   eval_train=ev_train, eval_test=ev_test, lstm_variant_test=lstm_test,
                   lstm_loss_ae=lart["history"]["ae"][-1], lstm_loss_fcn=lart["history"]["fcn"][-1],
                   p_min=trust.p_min, p_min_table_train=p_table,
                   rec_p99=float(art["rec_p99"]),
                   strain_p99=float(art["strain_p99"]),
                   loss_ae=art["history"]["ae"][-1], loss_heads=art["history"]["heads"][-1],
                   seconds_data=t_data, seconds_train=t_train,
                   horizon=args.horizon, windows_per_trajectory=args.windows, n_shell=args.n_shell, k_m=args.k_m,
                   lj_rc=args.lj_rc, morse_standard=bool(args.morse_standard),
                   strain_p50_train=float(np.median(w_tr[:, :, A.F_STRAIN].max(1))))
    with open(os.path.splitext(args.out)[0] + "_training.json", "w") as f:
        json.dump(summary, f, indent=1)
    print(json.dumps(summary), flush=True)


def reselect(args, A):
    """Choose the trust bound of a trained controller again (its parameters
    unchanged) and refresh the evaluations of its summary."""
    d = np.load(args.dataset)
    ctl, trust = A.load_controller(args.out)
    trust, p_table = A.select_trust(ctl, trust, d["train_w"], d["train_es"], d["train_ev"])
    saved = dict(np.load(args.out))
    saved["p_min"] = trust.p_min
    A.save(args.out, saved)
    js = os.path.splitext(args.out)[0] + "_training.json"
    summary = json.load(open(js)) if os.path.exists(js) else {}
    summary.update(p_min=trust.p_min, p_min_table_train=p_table,
                   eval_train=A.evaluate(ctl, d["train_w"], d["train_es"], d["train_ev"], trust),
                   eval_test=A.evaluate(ctl, d["test_w"], d["test_es"], d["test_ev"], trust))
    with open(js, "w") as f:
        json.dump(summary, f, indent=1)
    print(json.dumps(summary), flush=True)


if __name__ == "__main__":
    main()
