"""The paper's LSTM controller variant (Sec. 3.3) on the device against its
FP64 oracle (oracle/lstm.py).  The device computes in FP32 (no tensor cores
at these widths), so outputs agree to about 1e-5 of their scale and every
parameter block's gradient to 1e-3 relative; training lowers both losses."""
import numpy as np
import pytest

from oracle import ai as A
from oracle import lstm as OL

pytestmark = pytest.mark.gpu


def named(p):
    out = {}
    for k in ("enc1", "enc2", "dec1", "dec2"):
        for q in ("W_ih", "W_hh", "b_ih", "b_hh"):
            out[f"{k}.{q}"] = p[k][q]
    out["out.W"], out["out.b"] = p["out"]["W"], p["out"]["b"]
    for i, layer in enumerate(p["fcn"]):
        out[f"fcn.{i}.W"], out[f"fcn.{i}.b"] = layer["W"], layer["b"]
    return out


def flat(p, cfg, Ctl):
    n = named(p)
    return np.concatenate([np.asarray(n[name], np.float32).reshape(-1) for name, _ in Ctl.lstm_param_layout(cfg)])


def blocks(vec, cfg, Ctl):
    out, o = {}, 0
    for name, shape in Ctl.lstm_param_layout(cfg):
        k = int(np.prod(shape))
        out[name] = vec[o:o + k].reshape(shape)
        o += k
    return out


@pytest.fixture(scope="module")
def setup():
    from paper_2205_14121_gb300 import controller as Ctl
    cfg = Ctl.lstm_config(batch_max=32)
    m = Ctl.LSTMController(cfg)
    p = OL.init_params(seed=7)
    m.set_params(flat(p, cfg, Ctl))
    return Ctl, cfg, m, p


def windows(B, seed, T=50, F=6):
    rng = np.random.default_rng(seed)
    t = np.arange(T)[None, :, None]
    return np.sin(0.08 * t * (1 + rng.random((B, 1, F)))) + 0.3 * rng.standard_normal((B, T, F))


def test_lstm_predict_matches_oracle(setup):
    """Denoise, normalise, LSTM autoencoder and FCN: log k and the
    reconstruction error of every window; the class of log k."""
    Ctl, cfg, m, p = setup
    raw = 1.5 + windows(20, 1)
    mean, std = np.full(6, 1.5), np.full(6, 0.8)
    m.set_norm(mean, std)
    out = m.predict(raw.astype(np.float32))
    ref = OL.predict(p, raw.astype(np.float32).astype(np.float64), mean, std)
    scale = np.abs(ref["log_k"]).max() + 1e-12
    assert np.abs(out["log_k"] - ref["log_k"]).max() < 2e-5 * scale + 1e-6
    assert np.abs(out["rec_err"] - ref["rec_err"]).max() < 2e-5 * ref["rec_err"].max()


@pytest.mark.parametrize("what", ["ae", "fcn"])
def test_lstm_gradients_match_oracle(setup, what):
    """Backpropagation through time on the device: every parameter block of
    the trained part against the FP64 oracle (relative error < 1e-3), the
    other part's gradient zero."""
    Ctl, cfg, m, p = setup
    rng = np.random.default_rng(2)
    x = rng.standard_normal((12, 50, 6)).astype(np.float32)
    xd = x.astype(np.float64)
    if what == "ae":
        loss, g = m.grads(x, Ctl.TRAIN_AE)
        lo, go = OL.ae_loss_and_grads(p, xd)
    else:
        lk = np.log(rng.choice([1, 2, 5, 10, 20], 12)).astype(np.float32)
        loss, g = m.grads(x, Ctl.TRAIN_HEADS, log_k=lk)
        z, _ = OL.encode(p, xd)
        lo, go = OL.fcn_loss_and_grads(p, z, lk.astype(np.float64))
    assert loss == pytest.approx(lo, rel=1e-4)
    gb = blocks(g, cfg, Ctl)
    if what == "ae":
        ref = {f"{k}.{q}": go[k][q] for k in ("enc1", "enc2", "dec1", "dec2") for q in ("W_ih", "W_hh", "b_ih")}
        ref.update({"out.W": go["out"]["W"], "out.b": go["out"]["b"]})
    else:
        ref = {f"fcn.{i}.{k}": go["fcn"][i][k] for i in range(4) for k in ("W", "b")}
    for name, r in ref.items():
        if name.endswith("b_hh"):
            continue                     # the same gradient as b_ih
        d = gb[name]
        assert np.linalg.norm(d - r) <= 1e-3 * np.linalg.norm(r) + 1e-7, name
    other = [n for n in gb if (n.startswith("fcn") if what == "ae" else not n.startswith("fcn"))]
    assert all(np.all(gb[n] == 0) for n in other)


def test_lstm_training_lowers_both_losses(setup):
    """Adam on the device: the autoencoder's reconstruction loss and then the
    FCN's log k loss fall over a few epochs on fixed windows."""
    Ctl, cfg, m, p = setup
    m2 = Ctl.LSTMController(cfg)
    m2.set_params(flat(OL.init_params(seed=9), cfg, Ctl))
    rng = np.random.default_rng(5)
    x = (A.denoise(windows(32, 3)) - 0.0).astype(np.float32)
    lk = np.log(np.where(x[:, :, 0].mean(1) > 0, 10.0, 2.0)).astype(np.float32)
    ae = [m2.train_step(x, Ctl.TRAIN_AE, 5e-3) for _ in range(120)]
    hd = [m2.train_step(x, Ctl.TRAIN_HEADS, 5e-3, log_k=lk) for _ in range(150)]
    assert np.mean(ae[-10:]) < 0.7 * np.mean(ae[:5])
    assert np.mean(hd[-10:]) < 0.5 * np.mean(hd[:5])
