"""FP64 numpy oracle of the paper's own controller variant -- TEST INFRASTRUCTURE.

Only tests/ use it.  Sec. 3.3 describes it: the most recent 50 steps of six
per-platelet measurements, denoised (Table 2 step 2, the same filter as
oracle.ai), go through a two-layer LSTM autoencoder of 16 and 4 units that
yields 8 latent features, and a four-layer FCN of 32, 16, 8 and 1 neurons
gives the platelet time step (Table 2 step 4), categorised to an integration
level (step 5).  Readings of the garbled passage: the 8 latent features are
the final hidden and cell states of the 4-unit layer (4 + 4); the decoder
mirrors the encoder (LSTM 8 -> 4, LSTM 4 -> 16, linear 16 -> 6 at every
step, fed the repeated latent); the FCN's one output is log k, the ratio of
the fluid step to the platelet step, categorised to the nearest class of
{1, 2, 5, 10, 20} in log space.

LSTM cell (Hochreiter and Schmidhuber, 1997, with forget gate), gates
stacked (i, f, g, o) along the first axis of W_ih [4H, in], W_hh [4H, H],
b_ih [4H], b_hh [4H]:
  i = s(W_ii x + b_ii + W_hi h + b_hi), f = s(...), g = tanh(...), o = s(...)
  c' = f * c + i * g,  h' = o * tanh(c')
Backward passes are written out step by step and pinned by finite
differences; the forward pass against torch.nn.LSTM.
"""
from __future__ import annotations

import math

import numpy as np

from .ai import K_SET, denoise, sigmoid

T_WIN = 50
F_IN = 6
H1, H2 = 16, 4
LATENT = 2 * H2
FCN = (32, 16, 8)


def _lstm(rng, n_in, h):
    k = 1.0 / math.sqrt(h)
    return dict(W_ih=rng.uniform(-k, k, (4 * h, n_in)), W_hh=rng.uniform(-k, k, (4 * h, h)),
                b_ih=rng.uniform(-k, k, 4 * h), b_hh=rng.uniform(-k, k, 4 * h))


def _linear(rng, n_in, n_out):
    k = 1.0 / math.sqrt(n_in)
    return dict(W=rng.uniform(-k, k, (n_out, n_in)), b=rng.uniform(-k, k, n_out))


def init_params(seed=0, f_in=F_IN, h1=H1, h2=H2, fcn=FCN):
    rng = np.random.default_rng(seed)
    lat = 2 * h2
    dims = (lat,) + tuple(fcn) + (1,)
    return dict(enc1=_lstm(rng, f_in, h1), enc2=_lstm(rng, h1, h2), dec1=_lstm(rng, lat, h2),
                dec2=_lstm(rng, h2, h1), out=_linear(rng, h1, f_in),
                fcn=[_linear(rng, dims[i], dims[i + 1]) for i in range(len(dims) - 1)])


# ---------------------------------------------------------------------------
# LSTM forward / backward
# ---------------------------------------------------------------------------

def lstm_forward(layer, xs):
    """xs [T, B, in] -> hs [T, B, H], cs [T, B, H] and the cache for backward
    (zero initial state)."""
    T, B, _ = xs.shape
    H = layer["W_hh"].shape[1]
    h = np.zeros((B, H))
    c = np.zeros((B, H))
    hs, cs, cache = [], [], []
    for t in range(T):
        a = xs[t] @ layer["W_ih"].T + layer["b_ih"] + h @ layer["W_hh"].T + layer["b_hh"]
        i = sigmoid(a[:, 0:H])
        f = sigmoid(a[:, H:2 * H])
        g = np.tanh(a[:, 2 * H:3 * H])
        o = sigmoid(a[:, 3 * H:4 * H])
        c_new = f * c + i * g
        tc = np.tanh(c_new)
        h_new = o * tc
        cache.append((xs[t], h, c, i, f, g, o, tc))
        h, c = h_new, c_new
        hs.append(h)
        cs.append(c)
    return np.stack(hs), np.stack(cs), cache


def lstm_backward(layer, cache, dhs, dh_last=None, dc_last=None):
    """Gradients of a loss given dL/dh_t (dhs [T, B, H], may be None) plus
    dL/dh_T and dL/dc_T of the last step.  Returns (grads, dxs)."""
    T = len(cache)
    B, H = cache[0][1].shape
    g_out = {k: np.zeros_like(v) for k, v in layer.items()}
    dxs = np.zeros((T, B, layer["W_ih"].shape[1]))
    dh = np.zeros((B, H)) if dh_last is None else dh_last.copy()
    dc = np.zeros((B, H)) if dc_last is None else dc_last.copy()
    for t in range(T - 1, -1, -1):
        x, h_prev, c_prev, i, f, g, o, tc = cache[t]
        if dhs is not None:
            dh = dh + dhs[t]
        do = dh * tc
        dct = dc + dh * o * (1.0 - tc * tc)
        di = dct * g
        df = dct * c_prev
        dg = dct * i
        dc = dct * f
        da = np.concatenate([di * i * (1 - i), df * f * (1 - f), dg * (1 - g * g), do * o * (1 - o)], axis=1)
        g_out["W_ih"] += da.T @ x
        g_out["W_hh"] += da.T @ h_prev
        g_out["b_ih"] += da.sum(0)
        g_out["b_hh"] += da.sum(0)
        dxs[t] = da @ layer["W_ih"]
        dh = da @ layer["W_hh"]
    return g_out, dxs


# ---------------------------------------------------------------------------
# autoencoder and FCN
# ---------------------------------------------------------------------------

def encode(p, x):
    """x [B, T, F] (denoised, normalised) -> latent [B, 2 H2] = [h_T, c_T] of
    the second layer, and the caches."""
    xs = np.transpose(x, (1, 0, 2))
    h1, _, c1 = lstm_forward(p["enc1"], xs)
    h2, s2, c2 = lstm_forward(p["enc2"], h1)
    z = np.concatenate([h2[-1], s2[-1]], axis=1)
    return z, (xs, h1, c1, h2, c2)


def decode(p, z, T):
    zs = np.repeat(z[None], T, axis=0)
    d1, _, k1 = lstm_forward(p["dec1"], zs)
    d2, _, k2 = lstm_forward(p["dec2"], d1)
    y = d2 @ p["out"]["W"].T + p["out"]["b"]
    return np.transpose(y, (1, 0, 2)), (zs, d1, k1, d2, k2)


def ae_loss_and_grads(p, x):
    """Reconstruction MSE over B*T*F and its gradient (autoencoder part)."""
    B, T, F = x.shape
    z, (xs, h1, c1, h2, c2) = encode(p, x)
    y, (zs, d1, k1, d2, k2) = decode(p, z, T)
    e = y - x
    loss = float(np.mean(e * e))
    dy = np.transpose(2.0 * e / e.size, (1, 0, 2))            # [T, B, F]
    g = {}
    g["out"] = dict(W=np.einsum("tbf,tbh->fh", dy, d2), b=dy.sum((0, 1)))
    dd2 = dy @ p["out"]["W"]
    g["dec2"], dd1 = lstm_backward(p["dec2"], k2, dd2)
    g["dec1"], dzs = lstm_backward(p["dec1"], k1, dd1)
    dz = dzs.sum(0)
    H = p["enc2"]["W_hh"].shape[1]
    g["enc2"], dh1 = lstm_backward(p["enc2"], c2, None, dh_last=dz[:, :H], dc_last=dz[:, H:])
    g["enc1"], _ = lstm_backward(p["enc1"], c1, dh1)
    return loss, g


def fcn_forward(layers, z):
    acts = [z]
    a = z
    for li, l in enumerate(layers):
        a = a @ l["W"].T + l["b"]
        if li + 1 < len(layers):
            a = np.maximum(a, 0.0)
        acts.append(a)
    return a, acts


def fcn_loss_and_grads(p, z, log_k):
    """Mean squared error of the FCN's log k against targets [B], and its
    gradient (FCN part)."""
    out, acts = fcn_forward(p["fcn"], z)
    e = out[:, 0] - log_k
    loss = float(np.mean(e * e))
    d = (2.0 * e / len(e))[:, None]
    grads = [None] * len(p["fcn"])
    for li in range(len(p["fcn"]) - 1, -1, -1):
        l = p["fcn"][li]
        grads[li] = dict(W=d.T @ acts[li], b=d.sum(0))
        d = d @ l["W"]
        if li > 0:
            d = d * (acts[li] > 0)
    return loss, dict(fcn=grads)


def categorise(log_k, k_set=K_SET):
    """Table 2 step 5: the class of k nearest the prediction in log space."""
    lk = np.log(np.asarray(k_set, np.float64))
    return np.abs(np.asarray(log_k)[:, None] - lk[None, :]).argmin(1)


def predict(p, raw, mean, std, w=5):
    """raw [B, 50, 6] -> dict(log_k, k, rec_err)."""
    x = (denoise(raw, w) - mean) / std
    z, _ = encode(p, x)
    y, _ = decode(p, z, x.shape[1])
    rec = np.mean((y - x) ** 2, axis=(1, 2))
    out, _ = fcn_forward(p["fcn"], z)
    cls = categorise(out[:, 0])
    return dict(log_k=out[:, 0], cls=cls, k=np.asarray(K_SET)[cls], rec_err=rec)
