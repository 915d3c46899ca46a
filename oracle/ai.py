"""FP64 numpy oracle of the learned step-size controller -- TEST INFRASTRUCTURE.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg use it.
It restates the AI inference pipeline of Table 2 (Sec. 3.3):

  1. raw time series X (window of T steps x F per-platelet measurements)
  2. denoise: moving average, then a one-level Haar wavelet transform with
     soft thresholding of the detail coefficients (Donoho-Johnstone
     universal threshold, sigma from the median absolute detail)
  3. autoencoder: 2-layer GRU encoder -> latent vector (16), 2-layer GRU
     decoder fed the repeated latent -> reconstruction (trained on MSE)
  4. FCN heads on the latent: step-ratio class k in {1,2,5,10,20} (softmax)
     and hold length l (regression on log l)
  5. categorise to integration levels; 6. export (level, hold) per platelet

The GRU cell (Cho et al., 2014) in the convention with the reset gate on the
recurrent candidate term:
  r = s(W_ir x + b_ir + W_hr h + b_hr),  z = s(W_iz x + b_iz + W_hz h + b_hz)
  n = tanh(W_in x + b_in + r * (W_hn h + b_hn)),  h' = (1 - z) * n + z * h
Gates are stacked (r, z, n) along the first axis of W_ih [3H, in],
W_hh [3H, H], b_ih [3H], b_hh [3H].

Backward passes are written out step by step (backpropagation through time)
and pinned by finite differences; the forward pass is pinned against
torch.nn.GRU; Adam against torch.optim.Adam.
"""
from __future__ import annotations

import math

import numpy as np

K_SET = (1, 2, 5, 10, 20)
F_IN = 12
H = 64
LATENT = 16
HEAD_LAYERS = (32, 16, 8)


def sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


# ---------------------------------------------------------------------------
# Table 2, step 2: denoising filter
# ---------------------------------------------------------------------------

def moving_average(x, w=5):
    """Causal moving average over the time axis (axis -2): y_t = mean(x_{t-w+1..t}),
    shorter windows at the start."""
    x = np.asarray(x, dtype=np.float64)
    c = np.cumsum(x, axis=-2)
    out = np.empty_like(x)
    T = x.shape[-2]
    for t in range(T):
        lo = t - w
        s = c[..., t, :] - (c[..., lo, :] if lo >= 0 else 0.0)
        out[..., t, :] = s / min(w, t + 1)
    return out


def haar_denoise(x):
    """One-level Haar transform along time, soft-threshold the details with
    lambda = sigma sqrt(2 ln T), sigma = median|d| / 0.6745, inverse transform.
    T must be even.  Works on [..., T, F]."""
    x = np.asarray(x, dtype=np.float64)
    T = x.shape[-2]
    assert T % 2 == 0
    s2 = math.sqrt(2.0)
    ev, od = x[..., 0::2, :], x[..., 1::2, :]
    a = (ev + od) / s2
    d = (ev - od) / s2
    sigma = np.median(np.abs(d), axis=-2, keepdims=True) / 0.6745
    lam = sigma * math.sqrt(2.0 * math.log(T))
    d = np.sign(d) * np.maximum(np.abs(d) - lam, 0.0)
    out = np.empty_like(x)
    out[..., 0::2, :] = (a + d) / s2
    out[..., 1::2, :] = (a - d) / s2
    return out


def denoise(x, w=5):
    return haar_denoise(moving_average(x, w))


# ---------------------------------------------------------------------------
# parameters
# ---------------------------------------------------------------------------

def _gru_layer(rng, n_in, h):
    k = 1.0 / math.sqrt(h)
    return dict(W_ih=rng.uniform(-k, k, (3 * h, n_in)), W_hh=rng.uniform(-k, k, (3 * h, h)),
                b_ih=rng.uniform(-k, k, 3 * h), b_hh=rng.uniform(-k, k, 3 * h))


def _linear(rng, n_in, n_out):
    k = 1.0 / math.sqrt(n_in)
    return dict(W=rng.uniform(-k, k, (n_out, n_in)), b=rng.uniform(-k, k, n_out))


def init_params(seed=0, f_in=F_IN, h=H, latent=LATENT, head_layers=HEAD_LAYERS, n_classes=len(K_SET)):
    rng = np.random.default_rng(seed)
    p = dict(enc1=_gru_layer(rng, f_in, h), enc2=_gru_layer(rng, h, h), lat=_linear(rng, h, latent),
             dec1=_gru_layer(rng, latent, h), dec2=_gru_layer(rng, h, h), out=_linear(rng, h, f_in))
    for name, n_out in (("khead", n_classes), ("lhead", 1)):
        dims = (latent,) + tuple(head_layers) + (n_out,)
        p[name] = [_linear(rng, dims[i], dims[i + 1]) for i in range(len(dims) - 1)]
    return p


def zeros_like(p):
    if isinstance(p, dict):
        return {k: zeros_like(v) for k, v in p.items()}
    if isinstance(p, list):
        return [zeros_like(v) for v in p]
    return np.zeros_like(p)


def flatten(p, prefix=""):
    """(name, array) pairs in a fixed order (the order of the weight file)."""
    out = []
    if isinstance(p, dict):
        for k in sorted(p):
            out += flatten(p[k], f"{prefix}{k}.")
    elif isinstance(p, list):
        for i, v in enumerate(p):
            out += flatten(v, f"{prefix}{i}.")
    else:
        out.append((prefix[:-1], p))
    return out


# ---------------------------------------------------------------------------
# GRU forward / backward
# ---------------------------------------------------------------------------

def gru_forward(layer, xs, h0=None):
    """xs [T, B, in] -> hs [T, B, H] and the cache for backward."""
    T, B, _ = xs.shape
    h3 = layer["W_hh"].shape[0]
    Hh = h3 // 3
    h = np.zeros((B, Hh)) if h0 is None else h0
    hs = np.empty((T, B, Hh))
    cache = []
    for t in range(T):
        gi = xs[t] @ layer["W_ih"].T + layer["b_ih"]
        gh = h @ layer["W_hh"].T + layer["b_hh"]
        r = sigmoid(gi[:, :Hh] + gh[:, :Hh])
        z = sigmoid(gi[:, Hh:2 * Hh] + gh[:, Hh:2 * Hh])
        ghn = gh[:, 2 * Hh:]
        n = np.tanh(gi[:, 2 * Hh:] + r * ghn)
        h_new = (1.0 - z) * n + z * h
        cache.append((xs[t], h, r, z, n, ghn))
        h = h_new
        hs[t] = h
    return hs, cache


def gru_backward(layer, cache, dhs, dh_last=None):
    """dhs [T, B, H]: dL/dh_t from above (per step).  Returns grads of the layer
    and dL/dx [T, B, in]."""
    g = {k: np.zeros_like(v) for k, v in layer.items()}
    T = len(cache)
    B, Hh = dhs.shape[1], dhs.shape[2]
    dxs = np.empty((T, B, layer["W_ih"].shape[1]))
    dh = np.zeros((B, Hh)) if dh_last is None else dh_last.copy()
    for t in range(T - 1, -1, -1):
        x, h_prev, r, z, n, ghn = cache[t]
        dh = dh + dhs[t]
        dn = dh * (1.0 - z)
        dz = dh * (h_prev - n)
        dh_prev = dh * z
        dan = dn * (1.0 - n * n)            # through tanh
        dr = dan * ghn
        dghn = dan * r
        daz = dz * z * (1.0 - z)
        dar = dr * r * (1.0 - r)
        dgi = np.concatenate([dar, daz, dan], axis=1)
        dgh = np.concatenate([dar, daz, dghn], axis=1)
        g["W_ih"] += dgi.T @ x
        g["b_ih"] += dgi.sum(0)
        g["W_hh"] += dgh.T @ h_prev
        g["b_hh"] += dgh.sum(0)
        dxs[t] = dgi @ layer["W_ih"]
        dh = dh_prev + dgh @ layer["W_hh"]
    return g, dxs


def linear_forward(l, x):
    return x @ l["W"].T + l["b"]


def linear_backward(l, x, dy):
    return dict(W=dy.T @ x, b=dy.sum(0)), dy @ l["W"]


# ---------------------------------------------------------------------------
# autoencoder (Table 2 step 3)
# ---------------------------------------------------------------------------

def encode(p, x):
    """x [B, T, F] (filtered, normalised) -> latent [B, LATENT], cache."""
    xs = np.transpose(x, (1, 0, 2))
    h1, c1 = gru_forward(p["enc1"], xs)
    h2, c2 = gru_forward(p["enc2"], h1)
    zl = linear_forward(p["lat"], h2[-1])
    return zl, (xs, h1, c1, h2, c2)


def decode(p, zl, T):
    zs = np.repeat(zl[None], T, axis=0)
    d1, k1 = gru_forward(p["dec1"], zs)
    d2, k2 = gru_forward(p["dec2"], d1)
    y = d2 @ p["out"]["W"].T + p["out"]["b"]          # [T, B, F]
    return np.transpose(y, (1, 0, 2)), (zs, d1, k1, d2, k2)


def ae_loss_and_grads(p, x):
    """Reconstruction MSE (mean over B, T, F) and its gradient for the AE parts."""
    B, T, F = x.shape
    zl, (xs, h1, c1, h2, c2) = encode(p, x)
    y, (zs, d1, k1, d2, k2) = decode(p, zl, T)
    diff = y - x
    loss = float(np.mean(diff * diff))
    dy = 2.0 * diff / diff.size                        # [B, T, F]
    dyt = np.transpose(dy, (1, 0, 2))                  # [T, B, F]
    g = zeros_like({k: p[k] for k in ("enc1", "enc2", "lat", "dec1", "dec2", "out")})
    g["out"]["W"] = np.einsum("tbf,tbh->fh", dyt, d2)
    g["out"]["b"] = dyt.sum((0, 1))
    dd2 = dyt @ p["out"]["W"]
    gd2, dd1 = gru_backward(p["dec2"], k2, dd2)
    gd1, dzs = gru_backward(p["dec1"], k1, dd1)
    g["dec2"], g["dec1"] = gd2, gd1
    dzl = dzs.sum(0)
    gl, dh2_last = linear_backward(p["lat"], h2[-1], dzl)
    g["lat"] = gl
    dh2 = np.zeros_like(h2)
    dh2[-1] = dh2_last
    ge2, dh1 = gru_backward(p["enc2"], c2, dh2)
    ge1, _ = gru_backward(p["enc1"], c1, dh1)
    g["enc2"], g["enc1"] = ge2, ge1
    return loss, g


# ---------------------------------------------------------------------------
# FCN heads (Table 2 step 4)
# ---------------------------------------------------------------------------

def mlp_forward(layers, x):
    acts = [x]
    for i, l in enumerate(layers):
        x = linear_forward(l, x)
        if i + 1 < len(layers):
            x = np.maximum(x, 0.0)
        acts.append(x)
    return x, acts


def mlp_backward(layers, acts, dy):
    grads = [None] * len(layers)
    for i in range(len(layers) - 1, -1, -1):
        if i + 1 < len(layers):
            dy = dy * (acts[i + 1] > 0.0)
        grads[i], dy = linear_backward(layers[i], acts[i], dy)
    return grads, dy


def softmax(z):
    z = z - z.max(axis=1, keepdims=True)
    e = np.exp(z)
    return e / e.sum(axis=1, keepdims=True)


def heads_loss_and_grads(p, zl, k_class, log_hold, w_hold=1.0):
    """Cross-entropy of the k class + w_hold * MSE of log hold, mean over the batch."""
    B = zl.shape[0]
    logits, ak = mlp_forward(p["khead"], zl)
    pr = softmax(logits)
    ce = float(-np.mean(np.log(pr[np.arange(B), k_class] + 1e-300)))
    dlog = pr.copy()
    dlog[np.arange(B), k_class] -= 1.0
    dlog /= B
    gk, _ = mlp_backward(p["khead"], ak, dlog)
    lh, al = mlp_forward(p["lhead"], zl)
    e = lh[:, 0] - log_hold
    mse = float(np.mean(e * e))
    gl, _ = mlp_backward(p["lhead"], al, (w_hold * 2.0 * e / B)[:, None])
    return ce + w_hold * mse, dict(khead=gk, lhead=gl), dict(ce=ce, mse=mse)


# ---------------------------------------------------------------------------
# inference (Table 2 steps 1-6) and the trust bound
# ---------------------------------------------------------------------------

UNSURE_PROB, UNSURE_REC, UNSURE_STRAIN = 1, 2, 4


def trust_decision(prob, rec, log_hold, raw, p_min=0.6, rec_threshold=np.inf, strain_max=np.inf, strain_col=None,
                   fallback_k=10, hold_range=(100, 2000), k_set=K_SET):
    """Table 2 steps 5-6: the most probable class's ratio, or fallback_k when
    the window is unsure -- top probability below p_min, reconstruction error
    above rec_threshold, or the raw window's strain column above strain_max at
    any step (NaN fails each test) -- and the hold exp(log_hold) clipped to
    hold_range, truncated to whole steps.  Returns (k, hold, why bits)."""
    prob = np.asarray(prob, np.float64)
    why = np.zeros(prob.shape[0], np.int32)
    why |= np.where(~(prob.max(1) >= p_min), UNSURE_PROB, 0).astype(np.int32)
    why |= np.where(~(np.asarray(rec) <= rec_threshold), UNSURE_REC, 0).astype(np.int32)
    if strain_col is not None:
        smax = np.asarray(raw)[:, :, strain_col].max(1)
        why |= np.where(~(smax <= strain_max), UNSURE_STRAIN, 0).astype(np.int32)
    k = np.where(why != 0, fallback_k, np.asarray(k_set)[prob.argmax(1)]).astype(np.int32)
    h = np.exp(np.asarray(log_hold, np.float64))
    hold = np.floor(np.where(np.isnan(h), hold_range[0], np.clip(h, hold_range[0], hold_range[1])))
    return k, hold.astype(np.int32), why


def predict(p, raw, mean, std, rec_threshold=np.inf, p_min=0.6, hold_range=(100, 2000), w=5, strain_max=np.inf,
            strain_col=None, fallback_k=10):
    """raw [B, T, F] -> dict(k, hold, prob, rec_err, trusted, k_final, why):
    Table 2 steps 1-4, then the trust bound and ratio map of steps 5-6."""
    x = (denoise(raw, w) - mean) / std
    zl, _ = encode(p, x)
    y, _ = decode(p, zl, x.shape[1])
    rec = np.mean((y - x) ** 2, axis=(1, 2))
    logits, _ = mlp_forward(p["khead"], zl)
    pr = softmax(logits)
    cls = pr.argmax(1)
    lh, _ = mlp_forward(p["lhead"], zl)
    hold = np.clip(np.exp(lh[:, 0]), hold_range[0], hold_range[1])
    k_final, _, why = trust_decision(pr, rec, lh[:, 0], raw, p_min, rec_threshold, strain_max, strain_col, fallback_k,
                                     hold_range)
    return dict(k=np.array(K_SET)[cls], cls=cls, hold=hold, prob=pr, rec_err=rec, trusted=why == 0,
                k_final=k_final, why=why, log_hold=lh[:, 0])


# ---------------------------------------------------------------------------
# Adam (Kingma & Ba, 2015)
# ---------------------------------------------------------------------------

class Adam:
    def __init__(self, params, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.lr, self.b1, self.b2, self.eps = lr, b1, b2, eps
        self.m = zeros_like(params)
        self.v = zeros_like(params)
        self.t = 0

    def step(self, params, grads):
        self.t += 1
        c1 = 1.0 - self.b1 ** self.t
        c2 = 1.0 - self.b2 ** self.t

        def upd(p, g, m, v):
            if isinstance(p, dict):
                for k in p:
                    if k in g:
                        upd(p[k], g[k], m[k], v[k])
            elif isinstance(p, list):
                for a, b, c, d in zip(p, g, m, v):
                    upd(a, b, c, d)
            else:
                m *= self.b1
                m += (1.0 - self.b1) * g
                v *= self.b2
                v += (1.0 - self.b2) * g * g
                p -= self.lr * (m / c1) / (np.sqrt(v / c2) + self.eps)

        upd(params, grads, self.m, self.v)
