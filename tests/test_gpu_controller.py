"""The trained step-ratio controller (Table 2) against the method without it
(fixed-k RESPA at the fallback ratio) and against every fixed ratio:
fixed ratios on held-out labelled windows of this code's own trajectories
(the labels and the per-ratio errors come from fixed-k continuations)."""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

DATA = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2205_14121_gb300", "data")


def test_trained_controller_against_fixed_ratios():
    from paper_2205_14121_gb300 import ai_mts as A
    ctl, trust = A.load_controller(os.path.join(DATA, "controller.npz"))
    d = np.load(os.path.join(DATA, "controller_heldout.npz"))
    res = A.evaluate(ctl, d["w"], d["es"], d["ev"], trust)
    print(res)
    c = res["controller"]
    fb = res[f"fixed_k{trust.fallback_k}"]
    # what the network gains over the method without it (fixed-k RESPA at the
    # fallback ratio): strictly better on one axis -- fewer tolerance
    # violations, or a lower mean ratio (cheaper platelet level) -- and no
    # worse on the other
    assert ((c["violations"] <= fb["violations"] and c["mean_k"] < fb["mean_k"]) or
            (c["violations"] < fb["violations"] and c["mean_k"] <= fb["mean_k"])), (c, fb)
    # the network's own choices are used, and they vary with the window
    assert c["fallback_fraction"] < 0.5
    assert sum(1 for n in c["k_counts"] if n > 0) >= 2
    # more accurate than the cheapest ratio, and no fixed ratio is both at
    # least as accurate and at least as cheap (strictly better in one)
    assert c["violations"] < res["fixed_k1"]["violations"]
    for f in (res[f"fixed_k{k}"] for k in A.K_SET):
        dominated = (f["violations"] <= c["violations"] and f["mean_k"] <= c["mean_k"]
                     and (f["violations"] < c["violations"] or f["mean_k"] < c["mean_k"]))
        assert not dominated, (f, c)
