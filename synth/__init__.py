"""Seeded synthetic inputs shaped like the paper's DPD-CGMD systems (Sec. 3.1, Fig. 1).

This module is shared by the CUDA path's tests/benchmarks and by the CPU
oracle's tests.  It only draws *inputs* -- particle positions, velocities,
platelet shells, bond topology, receptor flags, wall layers -- and holds none
of the method's arithmetic (no forces, no integrator, no observables).

Recipe (all draws from ``numpy.random.Generator(Philox(seed))``):

* plasma: uniform positions in the fluid region, number density rho = 3;
* velocities: Maxwell-Boltzmann at kT = 1 (m = 1), net momentum removed;
* walls (when present): frozen layers of thickness ``wall`` at rho = 3 just
  outside y in [0, Ly], velocity 0 (the no-slip vessel walls of Sec. 3.1);
* platelets: Fibonacci-spiral points on a spheroid shell with radii (a, b, b),
  random orientation, bonds = union of each particle's 6 nearest shell
  neighbours with r0 = initial length, receptors = a seeded 5 % subset;
  placements are rejected when any particle comes closer than 1.0 to an
  already placed particle of another platelet.

Particle tag encoding (int32), shared by every consumer of these arrays:
    -1 plasma, -2 wall, p >= 0 platelet id p, receptor flag in bit 30.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

TAG_FLUID = -1
TAG_WALL = -2
RECEPTOR_BIT = 1 << 30

DEFAULT_SEED = 20220528


def rng_for(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(seed))


@dataclass
class System:
    """Arrays of one synthetic system, in particle-id order (id = row)."""

    box: tuple                      # (Lx, Ly, Lz) of the fluid region
    x: np.ndarray                   # (N, 3) float64 positions
    v: np.ndarray                   # (N, 3) float64 velocities
    tag: np.ndarray                 # (N,) int32, encoding above
    X0: np.ndarray                  # (N, 3) float64 rest positions (platelets; copy of x elsewhere)
    bonds: np.ndarray               # (nb, 2) int32 particle ids
    r0: np.ndarray                  # (nb,) float64 rest lengths
    walls: bool = False
    wall: float = 1.0               # wall layer thickness
    shear_rate: float = 0.0         # Lees-Edwards rate (periodic y only)
    body_force: float = 0.0         # g along +x
    n_platelets: int = 0
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.x.shape[0])


# ----------------------------------------------------------------------------
# building blocks
# ----------------------------------------------------------------------------

def uniform_box(rng, n, lo, hi):
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    return lo + (hi - lo) * rng.random((n, 3))


def maxwell(rng, n, kT=1.0):
    v = rng.standard_normal((n, 3)) * math.sqrt(kT)
    if n > 0:
        v -= v.mean(axis=0, keepdims=True)
    return v


def fibonacci_sphere(n):
    k = np.arange(n, dtype=np.float64) + 0.5
    z = 1.0 - 2.0 * k / n
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    phi = k * (math.pi * (3.0 - math.sqrt(5.0)))
    return np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)


def random_rotation(rng):
    q = rng.standard_normal(4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


def spheroid_shell(n, radii):
    """Shell points on a spheroid with semi-axes ``radii`` (body frame)."""
    return fibonacci_sphere(n) * np.asarray(radii, dtype=np.float64)[None, :]


def knn_bonds(points, k=6):
    """Union of each point's k nearest neighbours: (i<j) pairs + rest lengths."""
    from scipy.spatial import cKDTree

    tree = cKDTree(points)
    _, nb = tree.query(points, k=k + 1)
    i = np.repeat(np.arange(points.shape[0]), k)
    j = nb[:, 1:].reshape(-1)
    a = np.minimum(i, j)
    b = np.maximum(i, j)
    pairs = np.unique(np.stack([a, b], axis=1), axis=0)
    r0 = np.linalg.norm(points[pairs[:, 0]] - points[pairs[:, 1]], axis=1)
    return pairs.astype(np.int32), r0


def scaled_radii(n_shell, base_n=2000, base=(4.0, 2.0, 2.0)):
    """Radii keeping the 2,000-particle (4,2,2) shell's areal density."""
    s = math.sqrt(n_shell / base_n)
    return tuple(r * s for r in base)


class _Occupancy:
    """Voxel occupancy (edge 1.0) used to reject overlapping placements."""

    def __init__(self, lo, hi):
        self.lo = np.floor(np.asarray(lo, dtype=np.float64)) - 2.0
        self.shape = tuple(int(s) for s in (np.ceil(np.asarray(hi) - self.lo) + 3))
        self.grid = np.zeros(self.shape, dtype=bool)

    def _vox(self, pts):
        return np.floor(pts - self.lo).astype(np.int64)

    def free(self, pts):
        v = self._vox(pts)
        if (v < 0).any() or (v >= np.asarray(self.shape)).any():
            return False
        return not self.grid[v[:, 0], v[:, 1], v[:, 2]].any()

    def mark(self, pts):
        v = self._vox(pts)
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dz in (-1, 0, 1):
                    w = v + np.array([dx, dy, dz])
                    w = np.clip(w, 0, np.asarray(self.shape) - 1)
                    self.grid[w[:, 0], w[:, 1], w[:, 2]] = True


def _place_platelets(rng, n_plt, n_shell, radii, lo, hi, centers_fn=None,
                     max_tries=20000, occ=None, periodic_xz=None):
    """Random non-overlapping placements; returns list of (points, center, rotation)."""
    body = spheroid_shell(n_shell, radii)
    occ = occ or _Occupancy(lo, hi)
    out = []
    tries = 0
    rmax = max(radii)
    while len(out) < n_plt:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("could not place platelets without overlap")
        if centers_fn is not None:
            c = centers_fn(rng)
        else:
            c = lo + rmax + 1.0 + (np.asarray(hi) - np.asarray(lo) - 2 * rmax - 2.0) * rng.random(3)
        rot = random_rotation(rng)
        pts = body @ rot.T + c
        if (pts < np.asarray(lo) + 0.5).any() or (pts > np.asarray(hi) - 0.5).any():
            continue
        if not occ.free(pts):
            continue
        occ.mark(pts)
        out.append((pts, c, rot))
    return out


def _assemble(box, fluid_x, wall_x, plts, rng, n_shell, receptor_frac, kT=1.0):
    nf = fluid_x.shape[0]
    nw = wall_x.shape[0]
    npl = len(plts)
    xs = [fluid_x, wall_x] + [p[0] for p in plts]
    x = np.concatenate(xs, axis=0) if xs else np.zeros((0, 3))
    n = x.shape[0]
    tag = np.empty(n, dtype=np.int32)
    tag[:nf] = TAG_FLUID
    tag[nf:nf + nw] = TAG_WALL
    bonds = []
    r0s = []
    base = nf + nw
    for p in range(npl):
        off = base + p * n_shell
        t = np.full(n_shell, p, dtype=np.int32)
        nrec = int(round(receptor_frac * n_shell))
        rec = rng.permutation(n_shell)[:nrec]
        t[rec] |= RECEPTOR_BIT
        tag[off:off + n_shell] = t
        b, r0 = knn_bonds(plts[p][0])
        bonds.append(b + off)
        r0s.append(r0)
    v = maxwell(rng, n, kT)
    v[nf:nf + nw] = 0.0
    mob = tag != TAG_WALL
    if mob.any():
        v[mob] -= v[mob].mean(axis=0, keepdims=True)
    bonds = np.concatenate(bonds, axis=0).astype(np.int32) if bonds else np.zeros((0, 2), np.int32)
    r0 = np.concatenate(r0s) if r0s else np.zeros((0,), np.float64)
    return x, v, tag, bonds, r0


def _fill_platelets(rng, fx, plts, radii, box, gap, rho=3.0):
    """Plasma around and inside the shells: positions inside a spheroid or
    closer than `gap` to its membrane are dropped, and each interior gets
    1.1 rho x (the volume of the spheroid shrunk by `gap`) positions drawn
    uniformly in that shrunken spheroid.  A plasma particle on top of the
    dense membrane would start under the summed repulsion of dozens of
    membrane particles, and a shell without its interior fluid collapses
    under the outer pressure (it has no bending stiffness); a slightly denser
    interior keeps it inflated."""
    from scipy.spatial import cKDTree
    L = np.asarray(box, dtype=np.float64)
    a = np.asarray(radii, dtype=np.float64)
    keep = np.ones(len(fx), dtype=bool)
    tree = cKDTree(fx % L, boxsize=L)
    interiors = []
    for pts, c, rot in plts:
        near = np.asarray(tree.query_ball_point(np.asarray(c) % L, a.max() + gap), dtype=np.int64)
        if len(near):
            d = fx[near] - c
            d -= L * np.round(d / L)
            y = d @ rot                                   # body frame
            inside = ((y / a) ** 2).sum(1) < 1.0
            dm, _ = cKDTree(pts).query(c + d, distance_upper_bound=gap)
            keep[near[inside | np.isfinite(dm)]] = False
        b = np.maximum(a - gap, 0.05)
        n_in = int(round(1.1 * rho * 4.0 / 3.0 * np.pi * b.prod()))
        u = rng.standard_normal((n_in, 3))
        u /= np.linalg.norm(u, axis=1, keepdims=True)
        u *= rng.random((n_in, 1)) ** (1.0 / 3.0)
        interiors.append((u * b) @ rot.T + c)
    out = np.concatenate([fx[keep]] + interiors, axis=0)
    return out % L if len(out) else out


def wall_layers(rng, box, wall, rho=3.0):
    Lx, Ly, Lz = box
    nw1 = int(round(rho * Lx * Lz * wall))
    lo = uniform_box(rng, nw1, (0, -wall, 0), (Lx, 0, Lz))
    hi = uniform_box(rng, nw1, (0, Ly, 0), (Lx, Ly + wall, Lz))
    return np.concatenate([lo, hi], axis=0)


# ----------------------------------------------------------------------------
# systems
# ----------------------------------------------------------------------------

def plasma_box(n=None, box=None, rho=3.0, walls=False, wall=1.0, body_force=0.0,
               shear_rate=0.0, seed=DEFAULT_SEED, kT=1.0):
    """Plasma-only periodic box (optionally with y-walls)."""
    rng = rng_for(seed)
    if box is None:
        L = (n / rho) ** (1.0 / 3.0)
        L = float(np.float32(L))   # binary32-exact edge: FP32 and FP64 images agree
        box = (L, L, L)
    if n is None:
        n = int(round(rho * box[0] * box[1] * box[2]))
    fx = uniform_box(rng, n, (0, 0, 0), box)
    wx = wall_layers(rng, box, wall, rho) if walls else np.zeros((0, 3))
    x, v, tag, bonds, r0 = _assemble(box, fx, wx, [], rng, 0, 0.0, kT)
    return System(box=tuple(box), x=x, v=v, tag=tag, X0=x.copy(), bonds=bonds, r0=r0,
                  walls=walls, wall=wall, shear_rate=shear_rate, body_force=body_force,
                  meta=dict(kind="plasma", seed=seed))


def platelet_system(box, n_plasma, n_plt, n_shell, radii, walls=False, wall=1.0,
                    shear_rate=0.0, body_force=0.0, receptor_frac=0.05,
                    seed=DEFAULT_SEED, centers=None, clusters=None, kT=1.0, plasma_gap=0.8, developed_flow=False):
    """Plasma + spheroid platelet shells (Fig. 1 shapes, synthetic sizes).

    n_plasma plasma positions are drawn uniformly; see _fill_platelets for
    how the plasma meets the membranes.  developed_flow (walls and a body
    force): mobile particles start on the steady Poiseuille profile
    u_x(y) = rho g y (Ly - y) / (2 eta) with eta = ETA_DPD, which the flow would
    otherwise take about rho Ly^2 / eta time units to develop."""
    rng = rng_for(seed)
    box = tuple(float(b) for b in box)
    lo = np.zeros(3)
    hi = np.asarray(box)
    occ = _Occupancy(lo - 2, hi + 2)
    plts = []
    if centers is not None:
        body = spheroid_shell(n_shell, radii)
        for c in centers:
            rot = random_rotation(rng)
            pts = body @ rot.T + np.asarray(c, dtype=np.float64)
            occ.mark(pts)
            plts.append((pts, np.asarray(c, dtype=np.float64), rot))
    if clusters:
        for (cx, cy, cz, spread, count) in clusters:
            def cfn(r, cx=cx, cy=cy, cz=cz, spread=spread):
                return np.array([cx, cy, cz]) + spread * r.standard_normal(3) * np.array([1.0, 0.5, 1.0])
            plts += _place_platelets(rng, count, n_shell, radii, lo, hi, centers_fn=cfn, occ=occ)
    rest = n_plt - len(plts)
    if rest > 0:
        plts += _place_platelets(rng, rest, n_shell, radii, lo, hi, occ=occ)
    fx = uniform_box(rng, n_plasma, (0, 0, 0), box)
    if plts and len(fx):
        fx = _fill_platelets(rng, fx, plts, radii, box, plasma_gap)
    wx = wall_layers(rng, box, wall) if walls else np.zeros((0, 3))
    x, v, tag, bonds, r0 = _assemble(box, fx, wx, plts, rng, n_shell, receptor_frac, kT)
    if developed_flow and walls and body_force:
        mob = tag != TAG_WALL
        y = x[mob, 1]
        v[mob, 0] += 3.0 * body_force * y * (box[1] - y) / (2.0 * ETA_DPD)
    return System(box=box, x=x, v=v, tag=tag, X0=x.copy(), bonds=bonds, r0=r0,
                  walls=walls, wall=wall, shear_rate=shear_rate, body_force=body_force,
                  n_platelets=n_plt, meta=dict(kind="platelets", seed=seed, n_shell=n_shell,
                                               radii=tuple(radii)))


def config_couette_platelet(seed=DEFAULT_SEED, scale=1.0):
    """Plain STS parity system: 20^3 periodic box, rho = 3 plasma (24,000),
    Lees-Edwards shear 0.05, one 2,000-particle (4,2,2) shell at the centre.
    ``scale`` < 1 shrinks the box edge and the shell count proportionally."""
    L = 20.0 * scale
    n_pl = int(round(3.0 * L ** 3))
    n_shell = max(50, int(round(2000 * scale ** 2)))
    radii = scaled_radii(n_shell)
    return platelet_system((L, L, L), n_pl, 1, n_shell, radii, walls=False,
                           shear_rate=0.05, seed=seed, centers=[(L / 2, L / 2, L / 2)])


def config_dpd_throughput(n=1_000_000, seed=DEFAULT_SEED):
    """DPD-only throughput system: n plasma particles in an (n/3)^(1/3) cube,
    frozen walls in y, Poiseuille body force g = 0.02 along x."""
    return plasma_box(n=n, walls=True, wall=1.0, body_force=0.02, seed=seed)


def poiseuille_g(shear_rate, eta, rho, Ly):
    """Body force whose Poiseuille profile has wall shear rate ``shear_rate``."""
    return 2.0 * eta * shear_rate / (rho * Ly)


ETA_DPD = 0.86  # viscosity estimate for a=25, gamma=4.5, rho=3 (replaced by a measured value when available)


def config_channel_platelets(box=(400.0, 100.0, 67.0), n_plt=16, n_shell=10_000,
                             seed=DEFAULT_SEED, shear_rate=0.05, eta=ETA_DPD):
    """Fixed-k RESPA system: plasma at rho = 3 in a y-walled channel + n_plt shells
    of n_shell particles (areal density of the (4,2,2)/2,000 shell)."""
    Lx, Ly, Lz = box
    n_pl = int(round(3.0 * Lx * Ly * Lz))
    g = poiseuille_g(shear_rate, eta, 3.0, Ly)
    return platelet_system(box, n_pl, n_plt, n_shell, scaled_radii(n_shell), walls=True,
                           body_force=g, seed=seed)


def config_paper_scale(box=(1100.0, 300.0, 93.0), n_flow=70, n_clot=90, n_shell=40_000,
                       seed=DEFAULT_SEED, shear_rate=0.05, eta=ETA_DPD):
    """Paper-sized single-GPU system: two wall-attached clusters of n_clot shells at
    the same x on opposite walls plus n_flow flowing shells in a walled channel."""
    Lx, Ly, Lz = box
    radii = scaled_radii(n_shell)
    n_pl = int(round(3.0 * Lx * Ly * Lz))
    g = poiseuille_g(shear_rate, eta, 3.0, Ly)
    b = radii[1]
    clusters = [(Lx / 2, b + 1.5, Lz / 2, 3.0 * radii[0], n_clot),
                (Lx / 2, Ly - b - 1.5, Lz / 2, 3.0 * radii[0], n_clot)]
    return platelet_system(box, n_pl, n_flow + 2 * n_clot, n_shell, radii, walls=True,
                           body_force=g, seed=seed, clusters=clusters)
