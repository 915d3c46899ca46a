"""ctypes binding of libmsm (include/msm.h): argument marshalling only.

Every computation runs inside libmsm.so; PyTorch provides the device
workspace and the CUDA stream.  There is no fallback: if the library is
missing, :func:`lib` raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))

MD_OK = 0
MD_LEVEL_FLUID, MD_LEVEL_IFACE, MD_LEVEL_PLT, MD_LEVEL_ALL = 1, 2, 4, 7
MD_CFG_WALLS, MD_CFG_LEES_EDWARDS, MD_CFG_MORSE_STANDARD, MD_CFG_IFACE_LJ = 1, 2, 4, 8
MD_CFG_UNIFORM_NOISE = 16
MD_LIST_FLUID, MD_LIST_IFACE, MD_LIST_LJ, MD_LIST_MORSE = 0, 1, 2, 3
MD_FORCE_VIRIAL = 1
MD_FORCE_DETERMINISTIC = 2
MD_MODE_STS, MD_MODE_RESPA, MD_MODE_AI = 0, 1, 2
MD_SCHED_DIRECT, MD_SCHED_RECORD, MD_SCHED_DETERMINISTIC = 1, 2, 4
RECEPTOR_BIT = 1 << 30

ERRORS = {-1: "MD_EINVAL", -2: "MD_ENOMEM", -3: "MD_ECUDA", -4: "MD_ENBR_OVERFLOW", -5: "MD_EUNSTABLE",
          -6: "MD_ETIMEOUT", -7: "MD_ENOTRAINED", -8: "MD_ETOOLARGE"}
MD_PHILOX_STATIC_MAX = 16384


class MdError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class md_config(C.Structure):
    _fields_ = [
        ("n", C.c_int64), ("n_bonds", C.c_int64), ("n_plt_particles", C.c_int64), ("n_receptors", C.c_int64),
        ("n_platelets", C.c_int32), ("flags", C.c_int32),
        ("box", C.c_double * 3), ("wall", C.c_double), ("shear_rate", C.c_double), ("body_force", C.c_double),
        ("dt", C.c_double), ("skin", C.c_double),
        ("rc", C.c_double), ("a_ff", C.c_double), ("a_fw", C.c_double), ("a_fp", C.c_double),
        ("gamma", C.c_double), ("sigma", C.c_double),
        ("lj_eps", C.c_double), ("lj_sigma", C.c_double), ("lj_rc", C.c_double), ("lj_excl", C.c_double),
        ("morse_D", C.c_double), ("morse_alpha", C.c_double), ("morse_r0", C.c_double), ("morse_rc", C.c_double),
        ("f_A", C.c_double), ("k_bond", C.c_double),
        ("seed", C.c_uint64),
        ("cap_fluid", C.c_int32), ("cap_iface", C.c_int32), ("cap_lj", C.c_int32), ("cap_morse", C.c_int32),
        ("skin_plt", C.c_double),
        ("n_angles", C.c_int64), ("k_angle", C.c_double),
    ]


class md_buffers(C.Structure):
    _fields_ = [("workspace", C.c_void_p), ("workspace_bytes", C.c_size_t)]


class md_mts_schedule(C.Structure):
    _fields_ = [("mode", C.c_int32), ("k_m", C.c_int32), ("k_p", C.c_int32), ("flags", C.c_int32)]


class md_observables_t(C.Structure):
    _fields_ = [
        ("step", C.c_int64), ("time", C.c_double), ("momentum", C.c_double * 3), ("kinetic", C.c_double),
        ("temperature", C.c_double), ("kin_tensor", C.c_double * 9), ("virial_c", C.c_double * 9),
        ("pressure", C.c_double), ("n_builds", C.c_int64), ("max_rows", C.c_int64 * 4),
    ]


MD_PROF_CLASSES = 6
PROF_NAMES = ("fluid_dpd", "iface_dpd", "platelet", "integrate", "rebuild", "other")


class md_profile_t(C.Structure):
    _fields_ = [("launches", C.c_int64 * MD_PROF_CLASSES), ("ms", C.c_double * MD_PROF_CLASSES),
                ("total_launches", C.c_int64)]


_lib = None


def md_philox(ctr, key, use_library=False):
    """Philox4x32-10 blocks on the device (own kernel or cuRAND): ctr (n,4) uint32."""
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    key = np.ascontiguousarray(key, dtype=np.uint32).reshape(2)
    out = np.zeros_like(ctr)
    u32p = C.POINTER(C.c_uint32)
    rc = lib().md_philox(ctr.ctypes.data_as(u32p), key.ctypes.data_as(u32p), ctr.shape[0],
                         out.ctypes.data_as(u32p), int(use_library))
    if rc:
        raise MdError(rc, "md_philox")
    return out


def md_philox_static(ctr, key, use_library=False):
    """md_philox with the library's static device scratch (no allocation);
    at most MD_PHILOX_STATIC_MAX blocks per call."""
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    key = np.ascontiguousarray(key, dtype=np.uint32).reshape(2)
    out = np.zeros_like(ctr)
    u32p = C.POINTER(C.c_uint32)
    rc = lib().md_philox_static(ctr.ctypes.data_as(u32p), key.ctypes.data_as(u32p), ctr.shape[0],
                                out.ctypes.data_as(u32p), int(use_library))
    if rc:
        raise MdError(rc, f"md_philox_static: {ctr.shape[0]} blocks (static scratch holds "
                          f"{MD_PHILOX_STATIC_MAX})")
    return out


def library_path():
    return os.path.join(HERE, "_lib", "libmsm.so")


def lib():
    """Load libmsm.so (built by ``__graft_entry__.build()``); raise if absent."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"libmsm.so is not built ({path}); run __graft_entry__.build()")
    L = C.CDLL(path)
    vp, i64, i32, u32 = C.c_void_p, C.c_int64, C.c_int32, C.c_uint32
    dp = C.POINTER(C.c_double)
    ip = C.POINTER(C.c_int32)
    fp = C.POINTER(C.c_float)
    L.md_config_defaults.argtypes = [C.POINTER(md_config)]
    L.md_workspace_size.argtypes = [C.POINTER(md_config), C.POINTER(C.c_size_t)]
    L.md_init.argtypes = [C.POINTER(md_config), C.POINTER(md_buffers), vp, C.POINTER(vp)]
    L.md_destroy.argtypes = [vp]
    L.md_destroy.restype = None
    L.md_last_error.argtypes = [vp]
    L.md_last_error.restype = C.c_char_p
    L.md_set_particles.argtypes = [vp, dp, dp, ip, dp, i64]
    L.md_set_xv.argtypes = [vp, dp, dp, i64]
    L.md_set_bonds.argtypes = [vp, ip, dp, i64]
    L.md_set_angles.argtypes = [vp, ip, dp, i64]
    L.md_neighbor_build.argtypes = [vp, u32, C.c_int]
    L.md_forces.argtypes = [vp, u32, u32]
    L.md_read_forces.argtypes = [vp, u32, dp]
    L.md_read_particles.argtypes = [vp, dp, dp, fp]
    L.md_mts_step.argtypes = [vp, i64, C.POINTER(md_mts_schedule)]
    L.md_set_platelet_levels.argtypes = [vp, ip]
    L.md_observables.argtypes = [vp, C.POINTER(md_observables_t)]
    L.md_flow_profile.argtypes = [vp, C.c_int32, dp]
    L.md_neighbor_pairs.argtypes = [vp, i32, ip, i64, C.POINTER(C.c_int64)]
    L.md_get_state.argtypes = [vp, vp, C.POINTER(C.c_size_t)]
    L.md_set_state.argtypes = [vp, vp, C.c_size_t]
    L.md_profile_enable.argtypes = [vp, C.c_int]
    L.md_profile_read.argtypes = [vp, C.POINTER(md_profile_t), C.c_int]
    L.md_philox.argtypes = [C.POINTER(C.c_uint32), C.POINTER(C.c_uint32), i64, C.POINTER(C.c_uint32), C.c_int]
    L.md_philox_static.argtypes = L.md_philox.argtypes
    L.md_platelet_features.argtypes = [vp, dp]
    L.md_record_features.argtypes = [vp]
    L.md_read_feature_ring.argtypes = [vp, fp, C.POINTER(C.c_int64)]
    for name in ("md_platelet_features", "md_record_features", "md_read_feature_ring"):
        getattr(L, name).restype = C.c_int
    for name in ("md_config_defaults", "md_workspace_size", "md_init", "md_set_particles", "md_set_xv", "md_set_bonds",
                 "md_set_angles",
                 "md_neighbor_build", "md_forces", "md_read_forces", "md_read_particles", "md_mts_step",
                 "md_set_platelet_levels", "md_flow_profile",
                 "md_observables", "md_neighbor_pairs", "md_get_state", "md_set_state", "md_profile_enable",
                 "md_profile_read", "md_philox", "md_philox_static"):
        getattr(L, name).restype = C.c_int
    _lib = L
    return L


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


def config_for(n, box, tag=None, n_bonds=0, walls=False, wall=1.0, shear_rate=0.0, body_force=0.0, dt=0.01,
               skin=0.3, seed=20220528, caps=None, flags=0, n_angles=0, **params):
    """md_config for n particles (counts of platelet / receptor particles from tag);
    flags: extra MD_CFG_* bits (MD_CFG_MORSE_STANDARD, MD_CFG_IFACE_LJ,
    MD_CFG_UNIFORM_NOISE)."""
    cfg = md_config()
    cfg.n = int(n)
    for k in range(3):
        cfg.box[k] = float(box[k])
    rc = lib().md_config_defaults(C.byref(cfg))
    if rc:
        raise MdError(rc, "md_config_defaults")
    cfg.n_bonds = int(n_bonds)
    cfg.n_angles = int(n_angles)
    if tag is not None:
        t = np.asarray(tag)
        plt = t >= 0
        cfg.n_plt_particles = int(plt.sum())
        cfg.n_receptors = int((plt & ((t & RECEPTOR_BIT) != 0)).sum())
        cfg.n_platelets = int(((t[plt] & ~RECEPTOR_BIT).max() + 1) if plt.any() else 0)
    cfg.flags = ((MD_CFG_WALLS if walls else 0) | (MD_CFG_LEES_EDWARDS if (shear_rate and not walls) else 0) |
                 int(flags))
    cfg.wall = float(wall)
    cfg.shear_rate = float(shear_rate)
    cfg.body_force = float(body_force)
    cfg.dt = float(dt)
    cfg.skin = float(skin)
    cfg.seed = int(seed)
    for k, val in params.items():
        setattr(cfg, k, float(val))
    if caps:
        for k, val in caps.items():
            setattr(cfg, "cap_" + k, int(val))
    return cfg


class System:
    """One md_system over a torch-allocated device workspace."""

    def __init__(self, box, x, v, tag, X0=None, bonds=None, r0=None, walls=False, wall=1.0, shear_rate=0.0,
                 body_force=0.0, dt=0.01, skin=0.3, seed=20220528, step0=0, caps=None, stream=None, angles=None,
                 theta0=None, **params):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("System needs a CUDA device")
        L = lib()
        x = np.ascontiguousarray(x, dtype=np.float64)
        n = x.shape[0]
        bonds = np.zeros((0, 2), np.int32) if bonds is None else np.ascontiguousarray(bonds, dtype=np.int32)
        angles = np.zeros((0, 3), np.int32) if angles is None else np.ascontiguousarray(angles, dtype=np.int32)
        self.cfg = config_for(n, box, tag=tag, n_bonds=len(bonds), walls=walls, wall=wall, shear_rate=shear_rate,
                              body_force=body_force, dt=dt, skin=skin, seed=seed, caps=caps, n_angles=len(angles),
                              **params)
        nbytes = C.c_size_t()
        self._check(L.md_workspace_size(C.byref(self.cfg), C.byref(nbytes)), "md_workspace_size", None)
        self.workspace = torch.empty(int(nbytes.value), dtype=torch.uint8, device="cuda")
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        bufs = md_buffers(self.workspace.data_ptr(), int(nbytes.value))
        h = C.c_void_p()
        rc = L.md_init(C.byref(self.cfg), C.byref(bufs), C.c_void_p(self.stream.cuda_stream), C.byref(h))
        if rc:
            raise MdError(rc, L.md_last_error(None).decode())
        self.h = h
        self.n = n
        self.set_particles(x, v, tag, X0, step0)
        if len(bonds):
            self.set_bonds(bonds, r0)
        if len(angles):
            self.set_angles(angles, theta0)

    # -- plumbing ---------------------------------------------------------
    def _check(self, rc, what, h="self"):
        if rc:
            msg = lib().md_last_error(self.h if h == "self" else None).decode()
            raise MdError(rc, f"{what}: {msg}")

    def close(self):
        if getattr(self, "h", None):
            lib().md_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- C ABI, same names --------------------------------------------------
    def set_particles(self, x, v, tag, X0=None, step0=0):
        x = np.ascontiguousarray(x, dtype=np.float64)
        v = np.ascontiguousarray(v, dtype=np.float64)
        tag = np.ascontiguousarray(tag, dtype=np.int32)
        X0p = None
        if X0 is not None:
            X0 = np.ascontiguousarray(X0, dtype=np.float64)
            X0p = _dp(X0)
        self._check(lib().md_set_particles(self.h, _dp(x), _dp(v), _ip(tag), X0p, int(step0)), "md_set_particles")

    md_set_particles = set_particles

    def set_xv(self, x, v, step0=0):
        """New positions and velocities of the same particle set (tags, rest
        positions and bonds kept on the device)."""
        x = np.ascontiguousarray(x, dtype=np.float64)
        v = np.ascontiguousarray(v, dtype=np.float64)
        self._check(lib().md_set_xv(self.h, _dp(x), _dp(v), int(step0)), "md_set_xv")

    md_set_xv = set_xv

    def set_bonds(self, bonds, r0):
        bonds = np.ascontiguousarray(bonds, dtype=np.int32)
        r0 = np.ascontiguousarray(r0, dtype=np.float64)
        self._check(lib().md_set_bonds(self.h, _ip(bonds), _dp(r0), len(r0)), "md_set_bonds")

    md_set_bonds = set_bonds

    def set_angles(self, angles, theta0):
        """Angle triplets (i, vertex j, k) and rest angles of the Eq. 2 angle term."""
        a = np.ascontiguousarray(angles, dtype=np.int32).reshape(-1, 3)
        t = np.ascontiguousarray(theta0, dtype=np.float64).reshape(-1)
        self._check(lib().md_set_angles(self.h, _ip(a), _dp(t), a.shape[0]), "md_set_angles")

    md_set_angles = set_angles

    def neighbor_build(self, list_mask=0xF, force=True):
        self._check(lib().md_neighbor_build(self.h, list_mask, int(force)), "md_neighbor_build")

    md_neighbor_build = neighbor_build

    def forces(self, level_mask=MD_LEVEL_ALL, virial=False, deterministic=False):
        flags = (MD_FORCE_VIRIAL if virial else 0) | (MD_FORCE_DETERMINISTIC if deterministic else 0)
        self._check(lib().md_forces(self.h, level_mask, flags), "md_forces")

    md_forces = forces

    def read_forces(self, level_mask=MD_LEVEL_ALL):
        f = np.zeros((self.n, 3))
        self._check(lib().md_read_forces(self.h, level_mask, _dp(f)), "md_read_forces")
        return f

    md_read_forces = read_forces

    def read_particles(self):
        x = np.zeros((self.n, 3))
        v = np.zeros((self.n, 3))
        x32 = np.zeros((self.n, 3), np.float32)
        self._check(lib().md_read_particles(self.h, _dp(x), _dp(v), x32.ctypes.data_as(C.POINTER(C.c_float))),
                    "md_read_particles")
        return x, v, x32

    md_read_particles = read_particles

    def mts_step(self, n_outer, mode=MD_MODE_STS, k_m=1, k_p=1, direct=False, record=False, deterministic=False):
        sched = md_mts_schedule(mode, k_m, k_p,
                                (1 if direct else 0) | (2 if record else 0) | (4 if deterministic else 0))
        self._check(lib().md_mts_step(self.h, int(n_outer), C.byref(sched)), "md_mts_step")

    md_mts_step = mts_step

    def set_platelet_levels(self, k):
        """Per-platelet step ratios k_p for MD_MODE_AI (Sec. 3.3)."""
        k = np.ascontiguousarray(k, dtype=np.int32)
        self._check(lib().md_set_platelet_levels(self.h, k.ctypes.data_as(C.POINTER(C.c_int32))),
                    "md_set_platelet_levels")

    md_set_platelet_levels = set_platelet_levels

    def flow_profile(self, nbins=20):
        """(mean plasma v_x, plasma number density) per slab of y (Sec. 4.2)."""
        out = np.zeros(2 * nbins)
        self._check(lib().md_flow_profile(self.h, int(nbins), _dp(out)), "md_flow_profile")
        return out[:nbins], out[nbins:]

    md_flow_profile = flow_profile

    def observables(self):
        o = md_observables_t()
        self._check(lib().md_observables(self.h, C.byref(o)), "md_observables")
        return dict(step=o.step, time=o.time, momentum=np.array(o.momentum[:]), kinetic=o.kinetic,
                    temperature=o.temperature, kin_tensor=np.array(o.kin_tensor[:]).reshape(3, 3),
                    virial_c=np.array(o.virial_c[:]).reshape(3, 3), pressure=o.pressure, n_builds=o.n_builds,
                    max_rows=list(o.max_rows))

    md_observables = observables

    def neighbor_pairs(self, kind):
        cnt = C.c_int64()
        self._check(lib().md_neighbor_pairs(self.h, kind, None, 0, C.byref(cnt)), "md_neighbor_pairs")
        out = np.zeros((max(cnt.value, 1), 2), np.int32)
        self._check(lib().md_neighbor_pairs(self.h, kind, _ip(out), cnt.value, C.byref(cnt)), "md_neighbor_pairs")
        return out[:cnt.value]

    md_neighbor_pairs = neighbor_pairs

    def neighbor_count(self, kind):
        """Number of pairs in list `kind` (row counts only, no pair download)."""
        cnt = C.c_int64()
        self._check(lib().md_neighbor_pairs(self.h, kind, None, 0, C.byref(cnt)), "md_neighbor_pairs")
        return cnt.value

    def get_state(self):
        nb = C.c_size_t()
        self._check(lib().md_get_state(self.h, None, C.byref(nb)), "md_get_state")
        blob = (C.c_char * nb.value)()
        self._check(lib().md_get_state(self.h, blob, C.byref(nb)), "md_get_state")
        return bytes(blob)

    md_get_state = get_state

    def set_state(self, blob):
        buf = C.create_string_buffer(blob, len(blob))
        self._check(lib().md_set_state(self.h, buf, len(blob)), "md_set_state")

    md_set_state = set_state

    def platelet_features(self):
        P = self.cfg.n_platelets
        out = np.zeros((P, 12))
        self._check(lib().md_platelet_features(self.h, _dp(out)), "md_platelet_features")
        return out

    md_platelet_features = platelet_features

    def record_features(self):
        self._check(lib().md_record_features(self.h), "md_record_features")

    md_record_features = record_features

    def read_feature_ring(self):
        P = self.cfg.n_platelets
        out = np.zeros((P, 128, 12), np.float32)
        cnt = C.c_int64()
        self._check(lib().md_read_feature_ring(self.h, out.ctypes.data_as(C.POINTER(C.c_float)), C.byref(cnt)),
                    "md_read_feature_ring")
        return out[:, :min(cnt.value, 128)], cnt.value

    md_read_feature_ring = read_feature_ring

    def feature_count(self):
        """Records appended to the feature ring so far (no ring copy)."""
        cnt = C.c_int64()
        self._check(lib().md_read_feature_ring(self.h, None, C.byref(cnt)), "md_read_feature_ring")
        return cnt.value

    def profile_enable(self, on=True):
        self._check(lib().md_profile_enable(self.h, int(on)), "md_profile_enable")

    md_profile_enable = profile_enable

    def profile_read(self, reset=True):
        p = md_profile_t()
        self._check(lib().md_profile_read(self.h, C.byref(p), int(reset)), "md_profile_read")
        return dict(launches={n: p.launches[k] for k, n in enumerate(PROF_NAMES)},
                    ms={n: p.ms[k] for k, n in enumerate(PROF_NAMES)}, total_launches=p.total_launches)

    md_profile_read = profile_read
