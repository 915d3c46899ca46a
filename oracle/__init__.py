"""FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA path.

ctypes wrappers over ``msm_oracle.c`` (forces of Eq. 1-4, the FP32 neighbour
predicate, the Table 1 RESPA / velocity-Verlet loop, Sec. 4.2 observables) and,
in :mod:`oracle.ai`, the numpy FP64 learned controller (Table 2).

Parity status of each function is stated in its docstring; every function
here is pinned by ``tests/test_oracle_*.py`` against closed forms, invariants
or brute force.
"""
from __future__ import annotations

import ctypes as C
import math

import numpy as np

from . import build as _build

LVL_FLUID, LVL_IFACE, LVL_PLT = 1, 2, 4
LVL_ALL = 7

_lib = None


class Params(C.Structure):
    _fields_ = [
        ("L", C.c_double * 3),
        ("walls", C.c_int32),
        ("le", C.c_int32),
        ("le_rate", C.c_double),
        ("le_offset", C.c_double),
        ("g", C.c_double),
        ("rc", C.c_double), ("a_ff", C.c_double), ("a_fw", C.c_double), ("a_fp", C.c_double),
        ("gamma", C.c_double), ("sigma", C.c_double),
        ("lj_eps", C.c_double), ("lj_sigma", C.c_double), ("lj_rc", C.c_double),
        ("lj_excl", C.c_double),
        ("m_D", C.c_double), ("m_alpha", C.c_double), ("m_r0", C.c_double),
        ("m_rc", C.c_double), ("f_A", C.c_double),
        ("k_b", C.c_double),
        ("seed_lo", C.c_uint32), ("seed_hi", C.c_uint32),
        ("plt_k", C.POINTER(C.c_int32)), ("lvl_k", C.c_int32),
        ("iface_lj", C.c_int32),
        ("uniform_noise", C.c_int32),
        ("n_angles", C.c_int32),
        ("angles", C.POINTER(C.c_int32)),
        ("theta0", C.POINTER(C.c_double)),
        ("k_a", C.c_double),
    ]


DEFAULTS = dict(rc=1.0, a_ff=25.0, a_fw=25.0, a_fp=50.0, gamma=4.5, sigma=3.0,
                lj_eps=1.0, lj_sigma=0.8, lj_rc=2.0, lj_excl=1e30,
                m_D=2.0, m_alpha=2.0, m_r0=1.0, m_rc=5.0, f_A=0.0, k_b=100.0, k_a=5.0)


def make_params(box, walls=False, le_rate=0.0, le_offset=0.0, g=0.0, seed=20220528, angles=None, theta0=None,
                **kw):
    """Oracle parameters; angles [na, 3] particle rows (i, vertex j, k) with
    rest angles theta0 [na] for the Eq. 2 angle term (kept alive on p)."""
    p = Params()
    for k in range(3):
        p.L[k] = float(box[k])
    p.walls = int(bool(walls))
    p.le = int(le_rate != 0.0 and not walls)
    p.le_rate = float(le_rate)
    p.le_offset = float(le_offset)
    p.g = float(g)
    d = dict(DEFAULTS)
    d.update(kw)
    p.iface_lj = int(bool(d.pop("iface_lj", False)))
    p.uniform_noise = int(bool(d.pop("uniform_noise", False)))
    for k, v in d.items():
        setattr(p, k, float(v))
    p.seed_lo = seed & 0xFFFFFFFF
    p.seed_hi = (seed >> 32) & 0xFFFFFFFF
    set_angles(p, angles, theta0)
    return p


def set_angles(p, angles, theta0):
    """Attach (or with None, detach) the angle triplets of the Eq. 2 angle term."""
    if angles is None or len(angles) == 0:
        p.n_angles = 0
        p._angles = p._theta0 = None
        p.angles = C.cast(None, C.POINTER(C.c_int32))
        p.theta0 = C.cast(None, C.POINTER(C.c_double))
        return p
    a = np.ascontiguousarray(angles, dtype=np.int32).reshape(-1, 3)
    t = np.ascontiguousarray(theta0, dtype=np.float64).reshape(-1)
    assert a.shape[0] == t.shape[0]
    p._angles, p._theta0 = a, t
    p.n_angles = a.shape[0]
    p.angles = a.ctypes.data_as(C.POINTER(C.c_int32))
    p.theta0 = t.ctypes.data_as(C.POINTER(C.c_double))
    return p


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        dp = C.POINTER(C.c_double)
        ip = C.POINTER(C.c_int32)
        up = C.POINTER(C.c_uint32)
        fp = C.POINTER(C.c_float)
        P = C.POINTER(Params)
        L.orc_philox4x32_10.argtypes = [up, up, up]
        L.orc_gauss_from_bits.argtypes = [C.c_uint32, C.c_uint32]
        L.orc_gauss_from_bits.restype = C.c_double
        L.orc_zeta.argtypes = [P, C.c_int32, C.c_int32, C.c_uint32, C.c_uint32]
        L.orc_zeta.restype = C.c_double
        L.orc_forces_brute.argtypes = [P, C.c_int32, dp, dp, ip, ip, dp, C.c_int32, ip, dp,
                                       C.c_uint32, C.c_uint32, C.c_uint32, C.c_double,
                                       C.c_uint32, C.c_uint32, C.c_double, dp, dp]
        L.orc_forces_cells.argtypes = [P, C.c_int32, dp, dp, ip, ip, dp, ip, ip, dp,
                                       C.c_uint32, C.c_uint32, C.c_uint32, C.c_double,
                                       C.c_uint32, C.c_uint32, C.c_double,
                                       C.c_int32, ip, dp, dp]
        L.orc_pair_forces.argtypes = [P, C.c_int32, dp, dp, ip, ip, dp, C.c_uint32, C.c_uint32, C.c_uint32,
                                      C.c_double, C.c_uint32, C.c_uint32, C.c_double, C.c_int64, ip, ip, dp]
        L.orc_r2_f32.argtypes = [fp, fp, fp, C.c_int32, C.c_int32, C.c_float]
        L.orc_r2_f32.restype = C.c_float
        L.orc_pairs_f32.argtypes = [C.c_int32, fp, ip, fp, fp, C.c_int32, C.c_int32, C.c_float,
                                    C.c_int32, C.c_float, C.c_float, C.c_int64, ip]
        L.orc_pairs_f32.restype = C.c_int64
        L.orc_run_respa.argtypes = [P, C.c_int32, C.c_int32, dp, dp, ip, ip, dp, ip, dp,
                                    C.c_double, C.c_int32, C.c_int32, C.c_int32,
                                    C.c_uint32, C.c_double, C.c_int32, dp, dp, dp]
        L.orc_kinetics.argtypes = [P, C.c_int32, dp, dp, ip, C.c_int32, dp, dp, dp]
        L.orc_run_sts.argtypes = [P, C.c_int32, C.c_int32, dp, dp, ip, ip, dp, ip, dp,
                                  C.c_double, C.c_int32, C.c_uint32, C.c_double, C.c_int32, dp]
        L.orc_run_nested.argtypes = [P, C.c_int32, C.c_int32, dp, dp, ip, ip, dp, ip, dp, ip, C.c_int32, ip,
                                     C.c_int32, C.c_double, C.c_int32, C.c_int32, C.c_uint32, C.c_double, dp, dp]
        L.orc_run_ai_respa.argtypes = [P, C.c_int32, C.c_int32, dp, dp, ip, ip, dp, ip, dp, ip, C.c_int32, C.c_int32,
                                       C.c_double, C.c_int32, C.c_int32, C.c_uint32, C.c_double, C.c_int32,
                                       dp, dp, dp]
        _lib = L
    return _lib


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(C.POINTER(C.c_double))


def _i(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(C.POINTER(C.c_int32))


def _f(a):
    a = np.ascontiguousarray(a, dtype=np.float32)
    return a, a.ctypes.data_as(C.POINTER(C.c_float))


def philox4x32_10(ctr, key):
    """Philox4x32-10 block (SC'11): 4 counter words, 2 key words -> 4 words."""
    c = (C.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (C.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (C.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def gauss_from_bits(r0, r1):
    return lib().orc_gauss_from_bits(int(r0) & 0xFFFFFFFF, int(r1) & 0xFFFFFFFF)


def zeta(p, id_i, id_j, n_time, c_sub=0):
    return lib().orc_zeta(C.byref(p), int(id_i), int(id_j), int(n_time), int(c_sub))


def forces_brute(p, x, v, tag, X0=None, bonds=None, r0=None, ids=None, level_mask=LVL_ALL,
                 n_time=0, c_sub=0, dt=0.01, n_time_m=None, c_sub_m=None, dt_m=None):
    """Forces (Eq. 1-4) on every particle by the all-pairs sum.

    Returns (f[n,3], acc) with acc = dict(epot, vir[3,3], vir_c[3,3])."""
    n = x.shape[0]
    x, xp = _d(x)
    v, vp = _d(v)
    tag, tp = _i(tag)
    ids, idp = _i(np.arange(n) if ids is None else ids)
    X0, X0p = _d(x if X0 is None else X0)
    if bonds is None or len(bonds) == 0:
        bonds = np.zeros((0, 2), np.int32)
        r0 = np.zeros(0)
    bonds, bp = _i(bonds)
    r0, rp = _d(r0)
    f = np.zeros((n, 3))
    acc = np.zeros(19)
    lib().orc_forces_brute(C.byref(p), n, xp, vp, idp, tp, X0p, bonds.shape[0], bp, rp,
                           level_mask, n_time, c_sub, dt,
                           n_time if n_time_m is None else n_time_m,
                           c_sub if c_sub_m is None else c_sub_m,
                           dt if dt_m is None else dt_m,
                           f.ctypes.data_as(C.POINTER(C.c_double)),
                           acc.ctypes.data_as(C.POINTER(C.c_double)))
    return f, dict(epot=acc[0], vir=acc[1:10].reshape(3, 3), vir_c=acc[10:19].reshape(3, 3))


def pair_forces(p, x, v, tag, pairs, X0=None, ids=None, level_mask=LVL_ALL, n_time=0, c_sub=0, dt=0.01,
                n_time_m=None, c_sub_m=None, dt_m=None):
    """F_ij of Eq. 1-4 for listed pairs [npair, 2] of rows (zero where the
    pair does not interact); the same pair force the all-pairs sum adds up."""
    n = x.shape[0]
    x, xp = _d(x)
    v, vp = _d(v)
    tag, tp = _i(tag)
    ids, idp = _i(np.arange(n) if ids is None else ids)
    X0, X0p = _d(x if X0 is None else X0)
    pairs = np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1, 2)
    pi, pip = _i(pairs[:, 0])
    pj, pjp = _i(pairs[:, 1])
    F = np.zeros((pairs.shape[0], 3))
    lib().orc_pair_forces(C.byref(p), n, xp, vp, idp, tp, X0p, level_mask, n_time, c_sub, dt,
                          n_time if n_time_m is None else n_time_m, c_sub if c_sub_m is None else c_sub_m,
                          dt if dt_m is None else dt_m, pairs.shape[0], pip, pjp,
                          F.ctypes.data_as(C.POINTER(C.c_double)))
    return F


def bond_csr(n, bonds, r0):
    bonds = np.asarray(bonds, dtype=np.int64).reshape(-1, 2)
    a = np.concatenate([bonds[:, 0], bonds[:, 1]])
    b = np.concatenate([bonds[:, 1], bonds[:, 0]])
    rr = np.concatenate([r0, r0])
    order = np.lexsort((b, a))
    a, b, rr = a[order], b[order], rr[order]
    off = np.zeros(n + 1, np.int64)
    np.add.at(off, a + 1, 1)
    return np.cumsum(off).astype(np.int32), b.astype(np.int32), rr.astype(np.float64)


def forces_cells(p, x, v, tag, X0=None, bonds=None, r0=None, ids=None, level_mask=LVL_ALL,
                 n_time=0, c_sub=0, dt=0.01, n_time_m=None, c_sub_m=None, dt_m=None,
                 sample=None, with_acc=False):
    """Forces on ``sample`` (default: all) particles via a cell list; same
    definition and summation order as :func:`forces_brute`.  with_acc: also
    return dict(epot, vir, vir_c) of the pair terms (bonds excluded), which
    are the system's totals when every particle is in the sample."""
    n = x.shape[0]
    x, xp = _d(x)
    v, vp = _d(v)
    tag, tp = _i(tag)
    ids, idp = _i(np.arange(n) if ids is None else ids)
    X0, X0p = _d(x if X0 is None else X0)
    ip = C.POINTER(C.c_int32)
    if bonds is not None and len(bonds):
        off, nbr, rr = bond_csr(n, bonds, r0)
        off, offp = _i(off)
        nbr, nbrp = _i(nbr)
        rr, rrp = _d(rr)
    else:
        offp = C.cast(None, ip)
        nbrp = C.cast(None, ip)
        rrp = C.cast(None, C.POINTER(C.c_double))
    if sample is None:
        ns = n
        sp = C.cast(None, ip)
    else:
        sample, sp = _i(sample)
        ns = sample.shape[0]
    f = np.zeros((ns, 3))
    acc = np.zeros(19)
    lib().orc_forces_cells(C.byref(p), n, xp, vp, idp, tp, X0p, offp, nbrp, rrp, level_mask,
                           n_time, c_sub, dt,
                           n_time if n_time_m is None else n_time_m,
                           c_sub if c_sub_m is None else c_sub_m,
                           dt if dt_m is None else dt_m,
                           ns, sp, f.ctypes.data_as(C.POINTER(C.c_double)),
                           acc.ctypes.data_as(C.POINTER(C.c_double)))
    if with_acc:
        return f, dict(epot=acc[0], vir=acc[1:10].reshape(3, 3), vir_c=acc[10:19].reshape(3, 3))
    return f


def r2_f32(xi, xj, box_f32, walls=False, le=False, delta=0.0):
    xi, xip = _f(xi)
    xj, xjp = _f(xj)
    Lf, Lp = _f(box_f32)
    return lib().orc_r2_f32(xip, xjp, Lp, int(walls), int(le), float(np.float32(delta)))


KIND_FLUID, KIND_IFACE, KIND_LJ, KIND_MORSE = 0, 1, 2, 3


def pairs_f32(x32, tag, box_f32, kind, cut2, X0f=None, excl2=0.0, walls=False, le=False,
              delta=0.0):
    """Unordered index pairs (i<j) of list ``kind`` with r2 < cut2 under the FP32
    predicate (brute force).  Returns int32 array (m, 2) sorted."""
    n = x32.shape[0]
    x32, xp = _f(x32)
    tag, tp = _i(tag)
    X0f, X0p = _f(x32 if X0f is None else X0f)
    Lf, Lp = _f(box_f32)
    cnt = lib().orc_pairs_f32(n, xp, tp, X0p, Lp, int(walls), int(le), float(np.float32(delta)),
                              kind, float(np.float32(cut2)), float(np.float32(excl2)), 0,
                              C.cast(None, C.POINTER(C.c_int32)))
    out = np.zeros((max(cnt, 1), 2), np.int32)
    lib().orc_pairs_f32(n, xp, tp, X0p, Lp, int(walls), int(le), float(np.float32(delta)),
                        kind, float(np.float32(cut2)), float(np.float32(excl2)), cnt,
                        out.ctypes.data_as(C.POINTER(C.c_int32)))
    return out[:cnt]


def run_respa(p, x, v, tag, X0=None, bonds=None, r0=None, ids=None, dt_f=0.01, k_m=1, k_p=1,
              n_outer=1, n0=0, t0=0.0, forces=None):
    """Table 1 RESPA (k_m = k_p = 1: velocity-Verlet).  Returns (x, v, (f_f, f_m, f_p)).

    ``forces``: level forces at entry; None -> evaluated first."""
    n = x.shape[0]
    x = np.array(x, dtype=np.float64, order="C")
    v = np.array(v, dtype=np.float64, order="C")
    tag, tp = _i(tag)
    ids, idp = _i(np.arange(n) if ids is None else ids)
    X0, X0p = _d(x.copy() if X0 is None else X0)
    if bonds is None or len(bonds) == 0:
        bonds = np.zeros((0, 2), np.int32)
        r0 = np.zeros(0)
    bonds, bp = _i(bonds)
    r0, rp = _d(r0)
    if forces is None:
        ff, fm, fpl = np.zeros((n, 3)), np.zeros((n, 3)), np.zeros((n, 3))
        init = 1
    else:
        ff, fm, fpl = (np.array(a, dtype=np.float64, order="C") for a in forces)
        init = 0
    dp = C.POINTER(C.c_double)
    lib().orc_run_respa(C.byref(p), n, bonds.shape[0], x.ctypes.data_as(dp), v.ctypes.data_as(dp),
                        idp, tp, X0p, bp, rp, dt_f, k_m, k_p, n_outer, n0, t0, init,
                        ff.ctypes.data_as(dp), fm.ctypes.data_as(dp), fpl.ctypes.data_as(dp))
    return x, v, (ff, fm, fpl)


def run_ai_respa(p, x, v, tag, plt_k, X0=None, bonds=None, r0=None, ids=None, dt_f=0.01, k_m=1, n_outer=1,
                 n0=0, t0=0.0, forces=None):
    """AI-MTS: Table 1 with per-platelet step ratios plt_k[P].  Returns (x, v, (f_f, f_m, J)),
    J the platelet-level impulse of the last evaluation point (every term due)."""
    import math
    n = x.shape[0]
    x = np.array(x, dtype=np.float64, order="C")
    v = np.array(v, dtype=np.float64, order="C")
    tag, tp = _i(tag)
    ids, idp = _i(np.arange(n) if ids is None else ids)
    X0, X0p = _d(x.copy() if X0 is None else X0)
    if bonds is None or len(bonds) == 0:
        bonds = np.zeros((0, 2), np.int32)
        r0 = np.zeros(0)
    bonds, bp = _i(bonds)
    r0, rp = _d(r0)
    pk, pkp = _i(plt_k)
    tg = np.asarray(tag)
    if (tg >= 0).any() and len(pk) < int((tg[tg >= 0] & ~(1 << 30)).max() + 1):
        raise ValueError("run_ai_respa: one ratio per platelet")
    K = 1
    for k in pk:
        K = K * int(k) // math.gcd(K, int(k))
    if forces is None:
        ff, fm, fpl = np.zeros((n, 3)), np.zeros((n, 3)), np.zeros((n, 3))
        init = 1
    else:
        ff, fm, fpl = (np.array(a, dtype=np.float64, order="C") for a in forces)
        init = 0
    dp = C.POINTER(C.c_double)
    lib().orc_run_ai_respa(C.byref(p), n, bonds.shape[0], x.ctypes.data_as(dp), v.ctypes.data_as(dp), idp, tp,
                           X0p, bp, rp, pkp, len(pk), K, dt_f, k_m, n_outer, n0, t0, init, ff.ctypes.data_as(dp),
                           fm.ctypes.data_as(dp), fpl.ctypes.data_as(dp))
    return x, v, (ff, fm, fpl)


def run_nested(p, x, v, tag, plt_level, ratios, X0=None, bonds=None, r0=None, ids=None, dt_f=0.01, k_m=1,
               n_outer=1, n0=0, t0=0.0):
    """Table 1 as printed: platelets in nested sublevels (plt_level[P] in
    1..C, level 1 one step per interface substep, level l ratios[l - 1]
    steps per step of level l - 1; ratios[0] = 1), the innermost level
    drifting every particle.  Forces evaluated at entry.  Returns (x, v)."""
    n = x.shape[0]
    x = np.array(x, dtype=np.float64, order="C")
    v = np.array(v, dtype=np.float64, order="C")
    tag, tp = _i(tag)
    ids, idp = _i(np.arange(n) if ids is None else ids)
    X0, X0p = _d(x.copy() if X0 is None else X0)
    if bonds is None or len(bonds) == 0:
        bonds = np.zeros((0, 2), np.int32)
        r0 = np.zeros(0)
    bonds, bp = _i(bonds)
    r0, rp = _d(r0)
    lv, lvp = _i(plt_level)
    kr, krp = _i(ratios)
    tg = np.asarray(tag)
    P = int(((tg[tg >= 0] & ~(1 << 30)).max() + 1)) if (tg >= 0).any() else 0
    if len(lv) < P or kr[0] != 1 or lv.min(initial=1) < 1 or lv.max(initial=1) > len(kr):
        raise ValueError("run_nested: one level in 1..len(ratios) per platelet, ratios[0] = 1")
    ff, fm = np.zeros((n, 3)), np.zeros((n, 3))
    dp = C.POINTER(C.c_double)
    lib().orc_run_nested(C.byref(p), n, bonds.shape[0], x.ctypes.data_as(dp), v.ctypes.data_as(dp), idp, tp, X0p,
                         bp, rp, lvp, len(lv), krp, len(kr), dt_f, k_m, n_outer, n0, t0, ff.ctypes.data_as(dp),
                         fm.ctypes.data_as(dp))
    return x, v


def run_sts(p, x, v, tag, X0=None, bonds=None, r0=None, ids=None, dt=0.01, n_steps=1, n0=0, t0=0.0,
            force=None):
    """Single-time-step velocity-Verlet (all forces in one pass).  Returns (x, v, f)."""
    n = x.shape[0]
    x = np.array(x, dtype=np.float64, order="C")
    v = np.array(v, dtype=np.float64, order="C")
    tag, tp = _i(tag)
    ids, idp = _i(np.arange(n) if ids is None else ids)
    X0, X0p = _d(x.copy() if X0 is None else X0)
    if bonds is None or len(bonds) == 0:
        bonds = np.zeros((0, 2), np.int32)
        r0 = np.zeros(0)
    bonds, bp = _i(bonds)
    r0, rp = _d(r0)
    f = np.zeros((n, 3)) if force is None else np.array(force, dtype=np.float64, order="C")
    dp = C.POINTER(C.c_double)
    lib().orc_run_sts(C.byref(p), n, bonds.shape[0], x.ctypes.data_as(dp), v.ctypes.data_as(dp), idp, tp, X0p,
                      bp, rp, dt, n_steps, n0, t0, int(force is None), f.ctypes.data_as(dp))
    return x, v, f


def kinetics(p, x, v, tag, nbins=0):
    """Momentum, kinetic energy, peculiar temperature and y-profiles (Sec. 4.2)."""
    n = x.shape[0]
    x, xp = _d(x)
    v, vp = _d(v)
    tag, tp = _i(tag)
    out = np.zeros(14)
    pv = np.zeros(max(nbins, 1))
    pr = np.zeros(max(nbins, 1))
    dp = C.POINTER(C.c_double)
    lib().orc_kinetics(C.byref(p), n, xp, vp, tp, nbins, out.ctypes.data_as(dp),
                       pv.ctypes.data_as(dp), pr.ctypes.data_as(dp))
    return dict(momentum=out[0:3].copy(), ke=out[3], T=out[4], K=out[5:14].reshape(3, 3).copy(),
                prof_vx=pv[:nbins].copy(), prof_rho=pr[:nbins].copy())


def pressure(p, kin, acc, volume=None):
    """P = [sum m|v-u|^2 + sum_pairs r.F^C] / (3V)  (conservative virial)."""
    V = volume if volume is not None else p.L[0] * p.L[1] * p.L[2]
    return (np.trace(kin["K"]) + np.trace(acc["vir_c"])) / (3.0 * V)


def system_params(sysm, seed=20220528, le_offset=0.0, **kw):
    """Oracle parameters for a :class:`synth.System` (its angle triplets included)."""
    kw.setdefault("angles", getattr(sysm, "angles", None))
    kw.setdefault("theta0", getattr(sysm, "theta0", None))
    return make_params(sysm.box, walls=sysm.walls, le_rate=sysm.shear_rate, le_offset=le_offset,
                       g=sysm.body_force, seed=seed, **kw)
