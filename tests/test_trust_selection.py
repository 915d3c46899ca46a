"""Host logic of the controller's trust-bound choice (Table 2 step 5): the
gain test against the fallback ratio and the choice of the top-probability
bound on training windows.  The device evaluation is replaced by a table, so
these run without a GPU."""
import math

import pytest

from paper_2205_14121_gb300 import ai_mts as A


def pol(v, k):
    return {"violations": v, "mean_k": k, "fallback_fraction": 0.0, "k_counts": [0] * 5}


def test_gain_needs_strictly_better_on_one_axis_and_no_worse_on_the_other():
    fb = pol(0.30, 10.0)
    assert A.gains(pol(0.20, 10.0), fb)          # fewer violations, same cost
    assert A.gains(pol(0.30, 8.0), fb)           # same violations, cheaper
    assert A.gains(pol(0.10, 5.0), fb)
    assert not A.gains(pol(0.30, 10.0), fb)      # identical to the fallback
    assert not A.gains(pol(0.10, 11.0), fb)      # more accurate but dearer
    assert not A.gains(pol(0.31, 5.0), fb)       # cheaper but less accurate


def test_gain_margin_is_the_weaker_axis_ratio():
    fb = pol(0.30, 10.0)
    assert A.gain_margin(pol(0.15, 9.0), fb) == pytest.approx(0.9)
    assert A.gain_margin(pol(0.27, 5.0), fb) == pytest.approx(0.9)
    assert A.gain_margin(pol(0.0, 4.0), pol(0.0, 10.0)) == pytest.approx(0.4)
    assert A.gain_margin(pol(0.1, 4.0), pol(0.0, 10.0)) == math.inf


def fake_evaluate(table, fb=pol(0.30, 10.0)):
    def evaluate(ctl, windows, err_s, err_v, trust, batch=128):
        return {"controller": dict(table[round(trust.p_min, 2)]), f"fixed_k{trust.fallback_k}": dict(fb)}
    return evaluate


def test_select_trust_takes_the_widest_gain(monkeypatch):
    table = {p: pol(0.5, 12.0) for p in A.P_MIN_GRID}
    table[0.4] = pol(0.20, 7.3)       # margin 0.73
    table[0.45] = pol(0.21, 7.2)      # margin 0.72 -- the widest
    table[0.55] = pol(0.11, 9.7)      # fewest violations, margin 0.97
    monkeypatch.setattr(A, "evaluate", fake_evaluate(table))
    t, tab = A.select_trust(None, A.TrustBound(), None, None, None)
    assert t.p_min == pytest.approx(0.45)
    assert tab[0.55]["gain"] and not tab[0.6]["gain"]
    assert tab[0.45]["margin"] == pytest.approx(0.72)


def test_select_trust_keeps_the_given_bound_without_a_gain(monkeypatch):
    table = {p: pol(0.4, 11.0) for p in A.P_MIN_GRID}
    monkeypatch.setattr(A, "evaluate", fake_evaluate(table))
    given = A.TrustBound(p_min=0.6)
    t, tab = A.select_trust(None, given, None, None, None)
    assert t is given
    assert not any(v["gain"] for v in tab.values())
