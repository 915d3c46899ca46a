"""Seeded synthetic inputs shaped like the paper's DPD-CGMD systems (Sec. 3.1, Fig. 1).

This module is shared by the CUDA path's tests/benchmarks and by the CPU
oracle's tests.  It only draws *inputs* -- particle positions, velocities,
platelet shells, bond topology, receptor flags, wall layers -- and holds none
of the method's arithmetic (no forces, no integrator, no observables).

Recipe (all draws from ``numpy.random.Generator(Philox(seed))``):

* plasma: uniform positions in the fluid region, number density rho = 3
  (with platelets: drawn voxel by voxel, a multinomial count per voxel and
  uniform positions inside it, which is the same distribution);
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
    angles: np.ndarray = None       # (na, 3) int32 particle ids (i, vertex j, k) of the Eq. 2 angle term
    theta0: np.ndarray = None       # (na,) float64 rest angles
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


# Bending triplets: at each vertex j, every bonded neighbour i paired with
# the bonded neighbour k across from it (the largest angle i-j-k, if above
# 150 degrees) -- three nearly straight lines through each vertex of the
# membrane, as in a triangulated sheet -- with their rest angles as the
# reference, so that a shell starts without bending stress.
ANGLE_MIN = 5.0 * math.pi / 6.0


def angle_triplets(points, pairs, min_angle=ANGLE_MIN):
    """Bending triplets (i, j, k) of a bonded shell, j the vertex and i < k,
    and their rest angles (rounded to binary32)."""
    n = points.shape[0]
    nb = [[] for _ in range(n)]
    for a, b in pairs:
        nb[a].append(b)
        nb[b].append(a)
    tri = set()
    for j in range(n):
        ns = nb[j]
        if len(ns) < 2:
            continue
        u = points[ns] - points[j]
        u /= np.linalg.norm(u, axis=1, keepdims=True)
        c = u @ u.T
        np.fill_diagonal(c, 2.0)
        for a in range(len(ns)):
            b = int(np.argmin(c[a]))
            if np.arccos(np.clip(c[a, b], -1.0, 1.0)) > min_angle:
                i, k = sorted((ns[a], ns[b]))
                tri.add((i, j, k))
    if not tri:
        return np.zeros((0, 3), np.int32), np.zeros(0)
    t = np.asarray(sorted(tri), np.int32)
    return t, _f32(triplet_angles(points, t.astype(np.int64)))


def _f32(a):
    """Rest values rounded to binary32 (the precision the device stores), so
    that the device and the FP64 checks read the same numbers."""
    return np.asarray(a, np.float32).astype(np.float64)


def triplet_angles(points, t):
    a = points[t[:, 0]] - points[t[:, 1]]
    b = points[t[:, 2]] - points[t[:, 1]]
    c = (a * b).sum(1) / (np.linalg.norm(a, axis=1) * np.linalg.norm(b, axis=1))
    return np.arccos(np.clip(c, -1.0, 1.0))


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


def small_rotation(rng, angle):
    """Rotation by a uniform random angle in [0, angle] about a random axis."""
    u = rng.standard_normal(3)
    u /= np.linalg.norm(u)
    t = angle * rng.random()
    K = np.array([[0.0, -u[2], u[1]], [u[2], 0.0, -u[0]], [-u[1], u[0], 0.0]])
    return np.eye(3) + math.sin(t) * K + (1.0 - math.cos(t)) * (K @ K)


def _lattice_platelets(rng, count, n_shell, radii, x0, y_wall, up, Lz, lo, hi, occ, gap=2.5, jitter=0.03):
    """A wall-attached aggregate: `count` shells lying with their long axis
    along the flow (x), packed on a lattice that fills layer by layer away
    from the wall at y = y_wall (`up` = +1 for the lower wall, -1 for the
    upper), neighbours `gap` apart at their closest points (within the
    receptor Morse range, so that the aggregate starts bound), each turned by
    a small random rotation."""
    a, b, _ = radii
    sx, sy, sz = 2 * a + gap, 2 * b + gap, 2 * b + gap
    nz = max(1, int((Lz - 2 * b - 1.0) // sz) + 1)
    per_layer_x = max(1, int(math.ceil(count / (nz * max(1, int(math.ceil(count / (nz * 5))))))))
    body = spheroid_shell(n_shell, radii)
    out = []
    k = 0
    layer = 0
    while len(out) < count:
        yc = y_wall + up * (b + 1.5 + layer * sy)
        for ix in range(per_layer_x):
            for iz in range(nz):
                if len(out) >= count:
                    break
                c = np.array([x0 + (ix - (per_layer_x - 1) / 2) * sx, yc, Lz / 2 + (iz - (nz - 1) / 2) * sz])
                rot = small_rotation(rng, jitter)
                pts = body @ rot.T + c
                k += 1
                if (pts < np.asarray(lo) + 0.5).any() or (pts > np.asarray(hi) - 0.5).any() or not occ.free(pts):
                    raise RuntimeError("aggregate lattice does not fit the channel")
                occ.mark(pts)
                out.append((pts, c, rot))
        layer += 1
    return out


def _assemble(box, fluid_x, wall_x, plts, rng, n_shell, receptor_frac, kT=1.0, body=None):
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
    angs = []
    th0s = []
    base = nf + nw
    # every shell is a rigid motion of the same body-frame points: one
    # neighbour search gives every shell's bond and angle topology
    topo = knn_bonds(body)[0] if (npl and body is not None) else None
    atopo = angle_triplets(body, topo)[0] if topo is not None else None
    for p in range(npl):
        off = base + p * n_shell
        t = np.full(n_shell, p, dtype=np.int32)
        nrec = int(round(receptor_frac * n_shell))
        rec = rng.permutation(n_shell)[:nrec]
        t[rec] |= RECEPTOR_BIT
        tag[off:off + n_shell] = t
        pts = plts[p][0]
        if topo is None:
            b, r0 = knn_bonds(pts)
            at, th0 = angle_triplets(pts, b)
        else:
            b = topo
            r0 = np.linalg.norm(pts[b[:, 0]] - pts[b[:, 1]], axis=1)
            at = atopo
            th0 = _f32(triplet_angles(pts, at.astype(np.int64)))
        bonds.append(b + off)
        r0s.append(r0)
        angs.append(at + off)
        th0s.append(th0)
    v = maxwell(rng, n, kT)
    v[nf:nf + nw] = 0.0
    n_mob = n - nw
    if n_mob > 0:               # net momentum of the mobile particles removed
        v -= v.sum(axis=0, keepdims=True) / n_mob
        v[nf:nf + nw] = 0.0
    bonds = np.concatenate(bonds, axis=0).astype(np.int32) if bonds else np.zeros((0, 2), np.int32)
    r0 = np.concatenate(r0s) if r0s else np.zeros((0,), np.float64)
    angles = np.concatenate(angs, axis=0).astype(np.int32) if angs else np.zeros((0, 3), np.int32)
    theta0 = np.concatenate(th0s) if th0s else np.zeros((0,), np.float64)
    return x, v, tag, bonds, r0, angles, theta0


class VoxelPlasma:
    """Uniform plasma positions drawn voxel by voxel: the box is cut into
    nv[0] x nv[1] x nv[2] equal voxels, the counts per voxel are one
    multinomial draw with equal probabilities and each voxel's positions are
    uniform inside it -- together exactly n independent uniform positions in
    the box, stored grouped by voxel (start[v] .. start[v + 1]) so that the
    plasma near a point is a few contiguous slices."""

    def __init__(self, rng, n, box, cell):
        self.L = np.asarray(box, dtype=np.float64)
        self.nv = np.maximum(np.floor(self.L / cell).astype(np.int64), 1)
        self.h = self.L / self.nv
        nvox = int(self.nv.prod())
        counts = rng.multinomial(n, np.full(nvox, 1.0 / nvox))
        self.start = np.concatenate([[0], np.cumsum(counts)])
        x = rng.random((n, 3))
        vid = np.repeat(np.arange(nvox, dtype=np.int64), counts)
        ny_nz = self.nv[1] * self.nv[2]
        x[:, 0] += vid // ny_nz
        x[:, 1] += (vid // self.nv[2]) % self.nv[1]
        x[:, 2] += vid % self.nv[2]
        del vid
        x *= self.h
        self.x = x

    def near(self, c):
        """Plasma rows in the 27 voxels around point c (periodic wrap): a
        superset of those within one voxel edge of c."""
        cv = np.minimum(np.floor((np.asarray(c) % self.L) / self.h).astype(np.int64), self.nv - 1)
        offs = np.array([(i, j, k) for i in (-1, 0, 1) for j in (-1, 0, 1) for k in (-1, 0, 1)])
        w = (cv[None, :] + offs) % self.nv
        vs = np.unique((w[:, 0] * self.nv[1] + w[:, 1]) * self.nv[2] + w[:, 2])
        return np.concatenate([np.arange(self.start[v], self.start[v + 1]) for v in vs])


def _fill_platelets(rng, plasma, plts, radii, box, gap, rho=3.0, body=None):
    """Plasma around and inside the shells: positions inside a spheroid or
    closer than `gap` to its membrane are dropped, and each interior gets
    1.1 rho x (the volume of the spheroid shrunk by `gap`) positions drawn
    uniformly in that shrunken spheroid.  A plasma particle on top of the
    dense membrane would start under the summed repulsion of dozens of
    membrane particles, and a shell without its interior fluid collapses
    under the outer pressure; a slightly denser interior keeps it inflated.
    `plasma` is a VoxelPlasma with voxels at least a.max() + gap wide."""
    from scipy.spatial import cKDTree
    L = np.asarray(box, dtype=np.float64)
    a = np.asarray(radii, dtype=np.float64)
    fx = plasma.x
    keep = np.ones(len(fx), dtype=bool)
    reach = a.max() + gap
    # every shell is a rigid motion of the same body-frame points, so the
    # distance to a membrane is measured in the body frame against one tree
    tree = cKDTree(body)
    interiors = []
    for pts, c, rot in plts:
        cand = plasma.near(c)
        d = fx[cand] - c
        for k in range(3):                                # minimum image
            dk = d[:, k]
            dk[dk > 0.5 * L[k]] -= L[k]
            dk[dk < -0.5 * L[k]] += L[k]
        close = (d * d).sum(1) <= reach * reach
        near, d = cand[close], d[close]
        if len(near):
            y = d @ rot                                   # body frame
            er = np.sqrt(((y / a) ** 2).sum(1))           # ellipsoidal radius: the membrane is er = 1
            inside = er < 1.0
            # a point at er >= 1 lies on the shell scaled by er, at least
            # (er - 1) times the smallest semi-axis from the membrane
            band = ~inside & ((er - 1.0) * a.min() <= gap)
            dm, _ = tree.query(y[band], distance_upper_bound=gap)
            drop = inside.copy()
            drop[np.nonzero(band)[0][np.isfinite(dm)]] = True
            keep[near[drop]] = False
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
    x, v, tag, bonds, r0, angles, theta0 = _assemble(box, fx, wx, [], rng, 0, 0.0, kT)
    return System(box=tuple(box), x=x, v=v, tag=tag, X0=x.copy(), bonds=bonds, r0=r0, angles=angles, theta0=theta0,
                  walls=walls, wall=wall, shear_rate=shear_rate, body_force=body_force,
                  meta=dict(kind="plasma", seed=seed))


def platelet_system(box, n_plasma, n_plt, n_shell, radii, walls=False, wall=1.0,
                    shear_rate=0.0, body_force=0.0, receptor_frac=0.05,
                    seed=DEFAULT_SEED, centers=None, clusters=None, kT=1.0, plasma_gap=0.8, developed_flow=False,
                    aggregates=None):
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
    for (x0, y_wall, up, count) in (aggregates or ()):
        plts += _lattice_platelets(rng, count, n_shell, radii, x0, y_wall, up, box[2], lo, hi, occ)
    if clusters:
        for (cx, cy, cz, spread, count) in clusters:
            def cfn(r, cx=cx, cy=cy, cz=cz, spread=spread):
                return np.array([cx, cy, cz]) + spread * r.standard_normal(3) * np.array([1.0, 0.5, 1.0])
            plts += _place_platelets(rng, count, n_shell, radii, lo, hi, centers_fn=cfn, occ=occ)
    rest = n_plt - len(plts)
    if rest > 0:
        plts += _place_platelets(rng, rest, n_shell, radii, lo, hi, occ=occ)
    body = spheroid_shell(n_shell, radii) if plts else None
    if plts and n_plasma:
        plasma = VoxelPlasma(rng, n_plasma, box, max(radii) + plasma_gap)
        fx = _fill_platelets(rng, plasma, plts, radii, box, plasma_gap, body=body)
        del plasma
    else:
        fx = uniform_box(rng, n_plasma, (0, 0, 0), box)
    wx = wall_layers(rng, box, wall) if walls else np.zeros((0, 3))
    x, v, tag, bonds, r0, angles, theta0 = _assemble(box, fx, wx, plts, rng, n_shell, receptor_frac, kT, body=body)
    del fx
    if developed_flow and walls and body_force:
        mob = tag != TAG_WALL
        y = x[mob, 1]
        v[mob, 0] += 3.0 * body_force * y * (box[1] - y) / (2.0 * ETA_DPD)
    return System(box=box, x=x, v=v, tag=tag, X0=x.copy(), bonds=bonds, r0=r0, angles=angles, theta0=theta0,
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
    """Paper-sized single-GPU system (Sec. 3.1: a clot of about 102 M
    particles): two wall-attached aggregates of n_clot shells at the same x on
    opposite walls (packed from the wall outwards, neighbours within the
    receptor Morse range) plus n_flow shells placed at random in the walled
    channel; plasma at rho = 3 around and inside them."""
    Lx, Ly, Lz = box
    radii = scaled_radii(n_shell)
    n_pl = int(round(3.0 * Lx * Ly * Lz))
    g = poiseuille_g(shear_rate, eta, 3.0, Ly)
    aggregates = [(Lx / 2, 0.0, 1, n_clot), (Lx / 2, Ly, -1, n_clot)]
    return platelet_system(box, n_pl, n_flow + 2 * n_clot, n_shell, radii, walls=True,
                           body_force=g, seed=seed, aggregates=aggregates)
