"""Pins of the FP64 controller oracle (Table 2): GRU forward against
torch.nn.GRU, every backward against central finite differences, Adam against
torch.optim.Adam, the filters against closed forms."""
import math

import numpy as np
import pytest

from oracle import ai as A


def small_params(seed=1, f_in=3, h=5, latent=4):
    return A.init_params(seed=seed, f_in=f_in, h=h, latent=latent, head_layers=(6, 4, 3), n_classes=5)


def test_moving_average_closed_form():
    x = np.arange(10.0)[:, None] * np.ones((1, 2))
    y = A.moving_average(x, 5)
    assert np.allclose(y[4:, 0], np.arange(4, 10) - 2.0)
    assert np.allclose(y[:4, 0], [0.0, 0.5, 1.0, 1.5])


def test_haar_keeps_constants_and_pair_averages_a_ramp():
    c = np.full((16, 3), 2.5)
    assert np.allclose(A.haar_denoise(c), c)
    ramp = np.arange(16.0)[:, None]
    y = A.haar_denoise(ramp)
    pair_mean = (ramp[0::2] + ramp[1::2]) / 2
    assert np.allclose(y[0::2], pair_mean) and np.allclose(y[1::2], pair_mean)


def test_denoise_reduces_noise():
    rng = np.random.default_rng(0)
    t = np.linspace(0, 4 * np.pi, 128)
    clean = np.stack([np.sin(t), np.cos(0.5 * t)], axis=1)
    noisy = clean + 0.3 * rng.standard_normal(clean.shape)
    err_noisy = np.mean((noisy - clean) ** 2)
    err_den = np.mean((A.denoise(noisy) - clean) ** 2)
    assert err_den < 0.5 * err_noisy


def test_gru_forward_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(2)
    layer = A._gru_layer(rng, 3, 5)
    xs = rng.standard_normal((7, 4, 3))
    hs, _ = A.gru_forward(layer, xs)
    g = torch.nn.GRU(3, 5).double()
    with torch.no_grad():
        g.weight_ih_l0.copy_(torch.from_numpy(layer["W_ih"]))
        g.weight_hh_l0.copy_(torch.from_numpy(layer["W_hh"]))
        g.bias_ih_l0.copy_(torch.from_numpy(layer["b_ih"]))
        g.bias_hh_l0.copy_(torch.from_numpy(layer["b_hh"]))
        out, _ = g(torch.from_numpy(xs))
    assert np.allclose(hs, out.numpy(), rtol=0, atol=1e-13)


def _fd_check(loss_fn, params, grads, names, eps=1e-6, rtol=1e-6, samples=6, seed=0):
    rng = np.random.default_rng(seed)
    flat = dict(A.flatten(params))
    gflat = dict(A.flatten(grads))
    for name in names:
        arr = flat[name]
        g = gflat[name]
        for _ in range(samples):
            idx = tuple(rng.integers(0, s) for s in arr.shape)
            old = arr[idx]
            arr[idx] = old + eps
            lp = loss_fn()
            arr[idx] = old - eps
            lm = loss_fn()
            arr[idx] = old
            fd = (lp - lm) / (2 * eps)
            assert g[idx] == pytest.approx(fd, rel=rtol, abs=1e-9), (name, idx, g[idx], fd)


def test_autoencoder_backward_matches_finite_differences():
    p = small_params()
    x = np.random.default_rng(3).standard_normal((2, 6, 3))
    _, g = A.ae_loss_and_grads(p, x)
    names = [n for n, _ in A.flatten({k: p[k] for k in ("enc1", "enc2", "lat", "dec1", "dec2", "out")})]
    _fd_check(lambda: A.ae_loss_and_grads(p, x)[0],
              {k: p[k] for k in ("enc1", "enc2", "lat", "dec1", "dec2", "out")}, g, names)


def test_heads_backward_matches_finite_differences():
    p = small_params()
    rng = np.random.default_rng(4)
    zl = rng.standard_normal((8, 4))
    kc = rng.integers(0, 5, 8)
    lh = rng.standard_normal(8)
    _, g, _ = A.heads_loss_and_grads(p, zl, kc, lh)
    names = [n for n, _ in A.flatten({"khead": p["khead"], "lhead": p["lhead"]})]
    _fd_check(lambda: A.heads_loss_and_grads(p, zl, kc, lh)[0], {"khead": p["khead"], "lhead": p["lhead"]}, g,
              names)


def test_adam_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(5)
    w = rng.standard_normal((4, 3))
    p = {"w": w.copy()}
    opt = A.Adam(p, lr=1e-2)
    tw = torch.nn.Parameter(torch.from_numpy(w.copy()))
    topt = torch.optim.Adam([tw], lr=1e-2)
    for it in range(5):
        g = rng.standard_normal((4, 3))
        opt.step(p, {"w": g})
        topt.zero_grad()
        tw.grad = torch.from_numpy(g.copy())
        topt.step()
    assert np.allclose(p["w"], tw.detach().numpy(), rtol=0, atol=1e-12)


def test_predict_trust_bound():
    p = small_params()
    rng = np.random.default_rng(6)
    raw = rng.standard_normal((3, 8, 3))
    out = A.predict(p, raw, 0.0, 1.0, rec_threshold=np.inf, p_min=0.0)
    assert out["trusted"].all() and set(out["k"]) <= set(A.K_SET)
    out = A.predict(p, raw, 0.0, 1.0, rec_threshold=-1.0, p_min=0.0)
    assert not out["trusted"].any()
    assert np.all((out["hold"] >= 100) & (out["hold"] <= 2000))


def test_trust_decision_reasons_and_fallback():
    """Table 2 steps 5-6 on hand-made outputs: a confident window keeps its
    class's ratio; low top probability, a reconstruction error above the
    bound and a bond strain above the bound (at a single step of the raw
    window) each give the fallback ratio with their own reason bit; the hold
    is exp(log hold) clipped to [100, 2000] and truncated, a NaN gives the
    lower end."""
    prob = np.array([[0.05, 0.05, 0.8, 0.05, 0.05],    # class 2 -> k = 5
                     [0.3, 0.3, 0.2, 0.1, 0.1],         # top 0.3 < 0.6
                     [0.0, 0.0, 0.0, 0.9, 0.1],         # rec too large
                     [0.0, 0.0, 0.0, 0.0, 1.0],         # strain too large
                     [np.nan, 0.0, 0.0, 0.0, 0.0]])
    rec = np.array([0.1, 0.1, 5.0, 0.1, 0.1])
    raw = np.zeros((5, 4, 12))
    raw[3, 2, 9] = 0.9
    log_hold = np.log([50.0, 150.7, 1e4, 999.9, 1.0])
    log_hold[4] = np.nan
    k, hold, why = A.trust_decision(prob, rec, log_hold, raw, p_min=0.6, rec_threshold=1.0, strain_max=0.5,
                                    strain_col=9, fallback_k=10)
    assert k.tolist() == [5, 10, 10, 10, 10]
    assert why.tolist() == [0, A.UNSURE_PROB, A.UNSURE_REC, A.UNSURE_STRAIN, A.UNSURE_PROB]
    assert hold.tolist() == [100, 150, 2000, 999, 100]


# ---------------------------------------------------------------------------
# the paper's LSTM variant (Sec. 3.3)
# ---------------------------------------------------------------------------

def test_lstm_forward_matches_torch():
    """The oracle's LSTM layer equals torch.nn.LSTM with the same weights
    (gate order i, f, g, o; zero initial state)."""
    torch = pytest.importorskip("torch")
    from oracle import lstm as L
    rng = np.random.default_rng(21)
    layer = L._lstm(rng, 6, 16)
    xs = rng.standard_normal((7, 5, 6))
    hs, cs, _ = L.lstm_forward(layer, xs)
    m = torch.nn.LSTM(6, 16).double()
    with torch.no_grad():
        m.weight_ih_l0.copy_(torch.from_numpy(layer["W_ih"]))
        m.weight_hh_l0.copy_(torch.from_numpy(layer["W_hh"]))
        m.bias_ih_l0.copy_(torch.from_numpy(layer["b_ih"]))
        m.bias_hh_l0.copy_(torch.from_numpy(layer["b_hh"]))
        out, (hT, cT) = m(torch.from_numpy(xs))
    assert np.abs(hs - out.numpy()).max() < 1e-12
    assert np.abs(cs[-1] - cT.numpy()[0]).max() < 1e-12


def _fd_check(loss_fn, p, g, names, n=6, seed=0, h=1e-6):
    rng = np.random.default_rng(seed)
    for name in names:
        blocks = name.split(".")
        arr = p
        garr = g
        for b in blocks:
            arr = arr[int(b)] if isinstance(arr, list) else arr[b]
            garr = garr[int(b)] if isinstance(garr, list) else garr[b]
        for _ in range(n):
            idx = tuple(rng.integers(0, s) for s in arr.shape)
            old = arr[idx]
            arr[idx] = old + h
            lp = loss_fn()
            arr[idx] = old - h
            lm = loss_fn()
            arr[idx] = old
            assert garr[idx] == pytest.approx((lp - lm) / (2 * h), rel=1e-5, abs=1e-9), (name, idx)


def test_lstm_autoencoder_and_fcn_gradients_match_finite_differences():
    """Backpropagation through time of the LSTM autoencoder (latent = last
    hidden and cell state of the 4-unit layer) and of the FCN on log k, against
    FP64 central differences, every parameter block."""
    from oracle import lstm as L
    p = L.init_params(seed=3)
    rng = np.random.default_rng(4)
    x = rng.standard_normal((3, 9, 6))
    loss, g = L.ae_loss_and_grads(p, x)
    names = [f"{blk}.{w}" for blk in ("enc1", "enc2", "dec1", "dec2") for w in ("W_ih", "W_hh", "b_ih")]
    _fd_check(lambda: L.ae_loss_and_grads(p, x)[0], p, g, names + ["out.W", "out.b"])
    z, _ = L.encode(p, x)
    t = np.log([2.0, 5.0, 10.0])
    loss, g = L.fcn_loss_and_grads(p, z, t)
    _fd_check(lambda: L.fcn_loss_and_grads(p, z, t)[0], p, g, [f"fcn.{i}.W" for i in range(4)] + ["fcn.3.b"])


def test_lstm_categorise_to_nearest_level():
    """Table 2 step 5: log k to the nearest class of {1, 2, 5, 10, 20} in log space."""
    from oracle import lstm as L
    lk = np.log([1.0, 1.4, 1.5, 3.2, 3.1, 7.0, 7.1, 14.0, 14.2, 100.0, 0.01])
    assert L.categorise(lk).tolist() == [0, 0, 1, 2, 1, 2, 3, 3, 4, 4, 0]
