"""Binding of the learned step-size controller (Table 2) in libmsm.

Argument marshalling only: denoising, the GRU autoencoder, the heads, the
losses, backpropagation and Adam all run in libmsm's CUDA kernels.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from ._binding import MdError, lib

K_SET = (1, 2, 5, 10, 20)
AI_HOST, AI_DEVICE = 0, 1
TRAIN_AE, TRAIN_HEADS = 1, 2


class md_ai_trust(C.Structure):
    _fields_ = [("p_min", C.c_float), ("rec_max", C.c_float), ("strain_max", C.c_float), ("strain_col", C.c_int32),
                ("fallback_k", C.c_int32), ("hold_min", C.c_float), ("hold_max", C.c_float)]


UNSURE_PROB, UNSURE_REC, UNSURE_STRAIN = 1, 2, 4


class md_ai_config(C.Structure):
    _fields_ = [("T", C.c_int32), ("F", C.c_int32), ("hidden", C.c_int32), ("latent", C.c_int32),
                ("n_classes", C.c_int32), ("head_hidden", C.c_int32 * 3), ("batch_max", C.c_int32)]


_bound = False


def _bind():
    global _bound
    if _bound:
        return lib()
    L = lib()
    vp, fp, ip = C.c_void_p, C.POINTER(C.c_float), C.POINTER(C.c_int32)
    cfgp = C.POINTER(md_ai_config)
    L.md_ai_config_defaults.argtypes = [cfgp]
    L.md_ai_param_count.argtypes = [cfgp, C.POINTER(C.c_int64)]
    L.md_ai_workspace_size.argtypes = [cfgp, C.POINTER(C.c_size_t)]
    L.md_ai_init.argtypes = [cfgp, vp, C.c_size_t, vp, C.POINTER(vp)]
    L.md_ai_destroy.argtypes = [vp]
    L.md_ai_destroy.restype = None
    L.md_ai_last_error.argtypes = [vp]
    L.md_ai_last_error.restype = C.c_char_p
    L.md_ai_set_params.argtypes = [vp, fp, C.c_int64]
    L.md_ai_get_params.argtypes = [vp, fp, C.c_int64]
    L.md_ai_set_norm.argtypes = [vp, fp, fp]
    L.md_ai_predict.argtypes = [vp, vp, C.c_int32, C.c_int32, fp]
    L.md_ai_encode.argtypes = [vp, fp, C.c_int32, fp, fp]
    L.md_ai_prepare.argtypes = [vp, vp, C.c_int32, C.c_int32, fp]
    L.md_ai_grads.argtypes = [vp, fp, ip, fp, C.c_int32, C.c_int32, fp, fp]
    L.md_ai_train_step.argtypes = [vp, fp, ip, fp, C.c_int32, C.c_int32, C.c_float, fp]
    tp = C.POINTER(md_ai_trust)
    L.md_ai_decide.argtypes = [vp, vp, C.c_int32, C.c_int32, tp, ip, ip, ip, ip]
    L.md_ai_decide_system.argtypes = [vp, vp, tp, ip, ip, ip, ip]
    for n in ("md_ai_decide", "md_ai_decide_system"):
        getattr(L, n).restype = C.c_int
    for n in ("md_ai_config_defaults", "md_ai_param_count", "md_ai_workspace_size", "md_ai_init", "md_ai_set_params",
              "md_ai_get_params", "md_ai_set_norm", "md_ai_predict", "md_ai_encode", "md_ai_grads", "md_ai_prepare",
              "md_ai_train_step"):
        getattr(L, n).restype = C.c_int
    _bound = True
    return L


def default_config(batch_max=256, T=128, F=12, latent=16, head_hidden=(32, 16, 8), n_classes=5):
    c = md_ai_config()
    _bind().md_ai_config_defaults(C.byref(c))
    c.T, c.F, c.latent, c.n_classes, c.batch_max = T, F, latent, n_classes, batch_max
    for k in range(3):
        c.head_hidden[k] = head_hidden[k]
    return c


def param_layout(cfg):
    """(name, shape) of every parameter block in the flat layout of msm.h."""
    H, F, L, Cn = cfg.hidden, cfg.F, cfg.latent, cfg.n_classes
    hh = list(cfg.head_hidden)
    out = []

    def gru(name, nin):
        out.extend([(f"{name}.W_ih", (3 * H, nin)), (f"{name}.W_hh", (3 * H, H)), (f"{name}.b_ih", (3 * H,)),
                    (f"{name}.b_hh", (3 * H,))])

    gru("enc1", F)
    gru("enc2", H)
    out.extend([("lat.W", (L, H)), ("lat.b", (L,))])
    gru("dec1", L)
    gru("dec2", H)
    out.extend([("out.W", (F, H)), ("out.b", (F,))])
    for head, last in (("khead", Cn), ("lhead", 1)):
        dims = [L] + hh + [last]
        for l in range(4):
            out.extend([(f"{head}.{l}.W", (dims[l + 1], dims[l])), (f"{head}.{l}.b", (dims[l + 1],))])
    return out


def flatten(params_by_name, cfg):
    """Concatenate named arrays (dict name -> array) in the flat layout."""
    parts = []
    for name, shape in param_layout(cfg):
        a = np.asarray(params_by_name[name], np.float32)
        assert a.shape == tuple(shape), (name, a.shape, shape)
        parts.append(a.ravel())
    return np.concatenate(parts)


def unflatten(vec, cfg):
    out, o = {}, 0
    for name, shape in param_layout(cfg):
        n = int(np.prod(shape))
        out[name] = np.asarray(vec[o:o + n]).reshape(shape)
        o += n
    return out


class Controller:
    """The Table 2 pipeline over a torch-allocated device workspace."""

    def __init__(self, cfg=None, stream=None):
        import torch
        L = _bind()
        self.cfg = cfg if cfg is not None else default_config()
        n = C.c_int64()
        nb = C.c_size_t()
        if L.md_ai_param_count(C.byref(self.cfg), C.byref(n)) or L.md_ai_workspace_size(C.byref(self.cfg),
                                                                                        C.byref(nb)):
            raise MdError(-1, "invalid controller configuration")
        self.n_params = n.value
        self.workspace = torch.empty(nb.value, dtype=torch.uint8, device="cuda")
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = C.c_void_p()
        rc = L.md_ai_init(C.byref(self.cfg), C.c_void_p(self.workspace.data_ptr()), nb.value,
                          C.c_void_p(self.stream.cuda_stream), C.byref(h))
        if rc:
            raise MdError(rc, "md_ai_init")
        self.h = h

    def _check(self, rc, what):
        if rc:
            raise MdError(rc, f"{what}: {_bind().md_ai_last_error(self.h).decode()}")

    def close(self):
        if getattr(self, "h", None):
            _bind().md_ai_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _f(a):
        a = np.ascontiguousarray(a, np.float32)
        return a, a.ctypes.data_as(C.POINTER(C.c_float))

    def set_params(self, vec):
        vec, p = self._f(vec)
        self._check(_bind().md_ai_set_params(self.h, p, vec.size), "md_ai_set_params")

    def get_params(self):
        out = np.zeros(self.n_params, np.float32)
        self._check(_bind().md_ai_get_params(self.h, out.ctypes.data_as(C.POINTER(C.c_float)), self.n_params),
                    "md_ai_get_params")
        return out

    def set_norm(self, mean, std):
        m, mp = self._f(mean)
        s, sp = self._f(std)
        self._check(_bind().md_ai_set_norm(self.h, mp, sp), "md_ai_set_norm")

    def predict(self, raw):
        raw, rp = self._f(raw)
        B = raw.shape[0]
        out = np.zeros((B, self.cfg.n_classes + 2), np.float32)
        self._check(_bind().md_ai_predict(self.h, C.cast(rp, C.c_void_p), B, AI_HOST,
                                          out.ctypes.data_as(C.POINTER(C.c_float))), "md_ai_predict")
        probs = out[:, :self.cfg.n_classes]
        return dict(prob=probs, cls=probs.argmax(1), k=np.array(K_SET)[probs.argmax(1)],
                    log_hold=out[:, self.cfg.n_classes], rec_err=out[:, self.cfg.n_classes + 1])

    @staticmethod
    def _trust(trust):
        t = md_ai_trust(float(trust.p_min), float(min(trust.rec_max, 3.0e38)), float(min(trust.strain_max, 3.0e38)),
                        int(trust.strain_col), int(trust.fallback_k), float(trust.hold_range[0]),
                        float(trust.hold_range[1]))
        kv = np.ascontiguousarray(K_SET, np.int32)
        return t, kv

    def _decisions(self, B):
        k = np.zeros(B, np.int32)
        hold = np.zeros(B, np.int32)
        why = np.zeros(B, np.int32)
        ptr = lambda a: a.ctypes.data_as(C.POINTER(C.c_int32))
        return k, hold, why, ptr

    def decide(self, raw, trust):
        """Table 2 steps 1-6 on the device: per-window ratio, hold length and
        unsure-reason bits (0: the controller's own class was kept)."""
        raw, rp = self._f(raw)
        B = raw.shape[0]
        t, kv = self._trust(trust)
        k, hold, why, ptr = self._decisions(B)
        self._check(_bind().md_ai_decide(self.h, C.cast(rp, C.c_void_p), B, AI_HOST, C.byref(t), ptr(kv), ptr(k),
                                         ptr(hold), ptr(why)), "md_ai_decide")
        return dict(k=k, hold=hold, why=why, unsure=why != 0)

    def decide_system(self, system, trust):
        """md_ai_decide on the system's own feature ring (one window per
        platelet, gathered on the device)."""
        B = system.cfg.n_platelets
        t, kv = self._trust(trust)
        k, hold, why, ptr = self._decisions(B)
        self._check(_bind().md_ai_decide_system(self.h, system.h, C.byref(t), ptr(kv), ptr(k), ptr(hold), ptr(why)),
                    "md_ai_decide_system")
        return dict(k=k, hold=hold, why=why, unsure=why != 0)

    def prepare(self, raw):
        """Denoised, normalised windows [B][T][F] (Table 2 steps 1-2, on the device)."""
        raw, rp = self._f(raw)
        B = raw.shape[0]
        out = np.zeros((B, self.cfg.T, self.cfg.F), np.float32)
        self._check(_bind().md_ai_prepare(self.h, C.cast(rp, C.c_void_p), B, AI_HOST,
                                          out.ctypes.data_as(C.POINTER(C.c_float))), "md_ai_prepare")
        return out

    def encode(self, x):
        x, xp = self._f(x)
        B = x.shape[0]
        z = np.zeros((B, self.cfg.latent), np.float32)
        y = np.zeros((self.cfg.T, B, self.cfg.F), np.float32)
        self._check(_bind().md_ai_encode(self.h, xp, B, z.ctypes.data_as(C.POINTER(C.c_float)),
                                         y.ctypes.data_as(C.POINTER(C.c_float))), "md_ai_encode")
        return z, np.transpose(y, (1, 0, 2))

    def _labels(self, k_class, log_hold, B):
        if k_class is None:
            return None, None, None, None
        kc = np.ascontiguousarray(k_class, np.int32)
        lh = np.ascontiguousarray(log_hold, np.float32)
        return kc, lh, kc.ctypes.data_as(C.POINTER(C.c_int32)), lh.ctypes.data_as(C.POINTER(C.c_float))

    def grads(self, x, what, k_class=None, log_hold=None):
        x, xp = self._f(x)
        B = x.shape[0]
        kc, lh, kp, lp = self._labels(k_class, log_hold, B)
        g = np.zeros(self.n_params, np.float32)
        loss = C.c_float()
        self._check(_bind().md_ai_grads(self.h, xp, kp, lp, B, what, g.ctypes.data_as(C.POINTER(C.c_float)),
                                        C.byref(loss)), "md_ai_grads")
        return loss.value, g

    def train_step(self, x, what, lr, k_class=None, log_hold=None):
        x, xp = self._f(x)
        B = x.shape[0]
        kc, lh, kp, lp = self._labels(k_class, log_hold, B)
        loss = C.c_float()
        self._check(_bind().md_ai_train_step(self.h, xp, kp, lp, B, what, float(lr), C.byref(loss)),
                    "md_ai_train_step")
        return loss.value


# ---------------------------------------------------------------------------
# the paper's own controller variant (Sec. 3.3): LSTM autoencoder + FCN
# ---------------------------------------------------------------------------

class md_lstm_config(C.Structure):
    _fields_ = [("T", C.c_int32), ("F", C.c_int32), ("H1", C.c_int32), ("H2", C.c_int32), ("fcn", C.c_int32 * 3),
                ("batch_max", C.c_int32)]


_lstm_bound = False

# measurement columns the variant reads (of the 12 recorded per platelet):
# angular velocity (3), centre-of-mass velocity along the flow, plasma flow
# speed at the centre of mass, largest bond strain
LSTM_COLUMNS = (3, 4, 5, 0, 11, 9)


def _bind_lstm():
    global _lstm_bound
    L = lib()
    if _lstm_bound:
        return L
    vp, fp = C.c_void_p, C.POINTER(C.c_float)
    cp = C.POINTER(md_lstm_config)
    L.md_lstm_config_defaults.argtypes = [cp]
    L.md_lstm_param_count.argtypes = [cp, C.POINTER(C.c_int64)]
    L.md_lstm_workspace_size.argtypes = [cp, C.POINTER(C.c_size_t)]
    L.md_lstm_init.argtypes = [cp, vp, C.c_size_t, vp, C.POINTER(vp)]
    L.md_lstm_destroy.argtypes = [vp]
    L.md_lstm_destroy.restype = None
    L.md_lstm_last_error.argtypes = [vp]
    L.md_lstm_last_error.restype = C.c_char_p
    L.md_lstm_set_params.argtypes = [vp, fp, C.c_int64]
    L.md_lstm_get_params.argtypes = [vp, fp, C.c_int64]
    L.md_lstm_set_norm.argtypes = [vp, fp, fp]
    L.md_lstm_predict.argtypes = [vp, vp, C.c_int32, C.c_int32, fp]
    L.md_lstm_prepare.argtypes = [vp, vp, C.c_int32, C.c_int32, fp]
    L.md_lstm_grads.argtypes = [vp, fp, fp, C.c_int32, C.c_int32, fp, fp]
    L.md_lstm_train_step.argtypes = [vp, fp, fp, C.c_int32, C.c_int32, C.c_float, fp]
    for n in ("md_lstm_config_defaults", "md_lstm_param_count", "md_lstm_workspace_size", "md_lstm_init",
              "md_lstm_set_params", "md_lstm_get_params", "md_lstm_set_norm", "md_lstm_predict", "md_lstm_grads",
              "md_lstm_train_step", "md_lstm_prepare"):
        getattr(L, n).restype = C.c_int
    _lstm_bound = True
    return L


def lstm_config(batch_max=256):
    c = md_lstm_config()
    _bind_lstm().md_lstm_config_defaults(C.byref(c))
    c.batch_max = batch_max
    return c


def lstm_param_layout(cfg):
    """(name, shape) of every parameter block in the flat layout of msm.h."""
    H1, H2, F = cfg.H1, cfg.H2, cfg.F
    out = []
    for name, nin, h in (("enc1", F, H1), ("enc2", H1, H2), ("dec1", 2 * H2, H2), ("dec2", H2, H1)):
        out += [(f"{name}.W_ih", (4 * h, nin)), (f"{name}.W_hh", (4 * h, h)), (f"{name}.b_ih", (4 * h,)),
                (f"{name}.b_hh", (4 * h,))]
    out += [("out.W", (F, H1)), ("out.b", (F,))]
    dims = (2 * H2,) + tuple(cfg.fcn) + (1,)
    for i in range(4):
        out += [(f"fcn.{i}.W", (dims[i + 1], dims[i])), (f"fcn.{i}.b", (dims[i + 1],))]
    return out


class LSTMController:
    """The paper's LSTM autoencoder + FCN (Sec. 3.3) over a torch-allocated
    device workspace: argument marshalling only."""

    def __init__(self, cfg=None, stream=None):
        import torch
        L = _bind_lstm()
        self.cfg = cfg if cfg is not None else lstm_config()
        n = C.c_int64()
        nb = C.c_size_t()
        if L.md_lstm_param_count(C.byref(self.cfg), C.byref(n)) or L.md_lstm_workspace_size(C.byref(self.cfg),
                                                                                            C.byref(nb)):
            raise MdError(-1, "invalid LSTM controller configuration")
        self.n_params = n.value
        self.workspace = torch.empty(nb.value, dtype=torch.uint8, device="cuda")
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = C.c_void_p()
        rc = L.md_lstm_init(C.byref(self.cfg), C.c_void_p(self.workspace.data_ptr()), nb.value,
                            C.c_void_p(self.stream.cuda_stream), C.byref(h))
        if rc:
            raise MdError(rc, "md_lstm_init")
        self.h = h

    def _check(self, rc, what):
        if rc:
            raise MdError(rc, f"{what}: {_bind_lstm().md_lstm_last_error(self.h).decode()}")

    def close(self):
        if getattr(self, "h", None):
            _bind_lstm().md_lstm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    _f = staticmethod(Controller._f)

    def set_params(self, vec):
        vec, p = self._f(vec)
        self._check(_bind_lstm().md_lstm_set_params(self.h, p, vec.size), "md_lstm_set_params")

    def get_params(self):
        out = np.zeros(self.n_params, np.float32)
        self._check(_bind_lstm().md_lstm_get_params(self.h, out.ctypes.data_as(C.POINTER(C.c_float)), self.n_params),
                    "md_lstm_get_params")
        return out

    def set_norm(self, mean, std):
        m, mp = self._f(mean)
        s, sp = self._f(std)
        self._check(_bind_lstm().md_lstm_set_norm(self.h, mp, sp), "md_lstm_set_norm")

    def predict(self, raw):
        """raw [B][T][F] -> dict(log_k, cls, k, rec_err); cls the nearest
        class of log k (Table 2 step 5)."""
        raw, rp = self._f(raw)
        B = raw.shape[0]
        out = np.zeros((B, 2), np.float32)
        self._check(_bind_lstm().md_lstm_predict(self.h, C.cast(rp, C.c_void_p), B, AI_HOST,
                                                 out.ctypes.data_as(C.POINTER(C.c_float))), "md_lstm_predict")
        lk = np.log(np.asarray(K_SET, np.float64))
        cls = np.abs(out[:, 0:1].astype(np.float64) - lk[None, :]).argmin(1)
        return dict(log_k=out[:, 0], cls=cls, k=np.asarray(K_SET)[cls], rec_err=out[:, 1])

    def prepare(self, raw):
        """Denoised, normalised windows [B][T][F] (Table 2 steps 1-2, on the device)."""
        raw, rp = self._f(raw)
        B = raw.shape[0]
        out = np.zeros((B, self.cfg.T, self.cfg.F), np.float32)
        self._check(_bind_lstm().md_lstm_prepare(self.h, C.cast(rp, C.c_void_p), B, AI_HOST,
                                                 out.ctypes.data_as(C.POINTER(C.c_float))), "md_lstm_prepare")
        return out

    def grads(self, x, what, log_k=None):
        x, xp = self._f(x)
        B = x.shape[0]
        lk = None if log_k is None else np.ascontiguousarray(log_k, np.float32)
        g = np.zeros(self.n_params, np.float32)
        loss = C.c_float()
        self._check(_bind_lstm().md_lstm_grads(self.h, xp, None if lk is None else lk.ctypes.data_as(
            C.POINTER(C.c_float)), B, what, g.ctypes.data_as(C.POINTER(C.c_float)), C.byref(loss)), "md_lstm_grads")
        return float(loss.value), g

    def train_step(self, x, what, lr, log_k=None):
        x, xp = self._f(x)
        B = x.shape[0]
        lk = None if log_k is None else np.ascontiguousarray(log_k, np.float32)
        loss = C.c_float()
        self._check(_bind_lstm().md_lstm_train_step(self.h, xp, None if lk is None else lk.ctypes.data_as(
            C.POINTER(C.c_float)), B, what, float(lr), C.byref(loss)), "md_lstm_train_step")
        return float(loss.value)
