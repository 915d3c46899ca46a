"""The trained step-ratio controller (Table 2) against the method without it:
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
    fixed = [res[f"fixed_k{k}"] for k in A.K_SET]
    # more accurate than the cheapest ratio, and no fixed ratio is both at
    # least as accurate and at least as cheap (strictly better in one)
    assert c["violations"] < res["fixed_k1"]["violations"]
    for f in fixed:
        dominated = (f["violations"] <= c["violations"] and f["mean_k"] <= c["mean_k"]
                     and (f["violations"] < c["violations"] or f["mean_k"] < c["mean_k"]))
        assert not dominated, (f, c)
