"""FP64 numpy oracle of the per-platelet measurements -- TEST INFRASTRUCTURE.

Sec. 3.3: each platelet's dynamics is characterised by time series of
physics measurements computed during the simulation (angular velocity
components, kinetic energies, flow speed at the centre of mass); the build
records twelve per platelet and step:

  0-2  centre-of-mass velocity V = mean v_i
  3-5  angular velocity w = I^-1 L, L = sum r_i x (v_i - V), I = sum(|r_i|^2 1 - r_i r_i^T),
       r_i = minimum-image position relative to the centre of mass
  6-8  principal values (ascending) of the platelet stress
       S = -1/2 sum_i (r_i F_i^T + F_i r_i^T)  (moment of the total forces F_i)
  9    largest bond strain |r_b - r0_b| / r0_b over the platelet's bonds
  10   contacts: receptor pairs with another platelet closer than 1.5 r0 (Morse r0)
  11   plasma flow speed: mean |v| of plasma particles within 2 of the centre of mass
"""
from __future__ import annotations

import numpy as np

RECEPTOR_BIT = 1 << 30
N_FEATURES = 12


def _min_image(d, box, walls):
    d = d.copy()
    for k in range(3):
        if k == 1 and walls:
            continue
        d[..., k] -= box[k] * np.round(d[..., k] / box[k])
    return d


def platelet_features(x, v, f, tag, bonds, r0, box, walls=False, morse_r0=1.0, flow_radius=2.0):
    """x, v, f [n, 3] (positions, velocities, total forces), tag [n], bonds [nb, 2],
    r0 [nb] -> features [P, 12] in platelet-id order."""
    x = np.asarray(x, np.float64)
    v = np.asarray(v, np.float64)
    f = np.asarray(f, np.float64)
    tag = np.asarray(tag)
    plt = tag >= 0
    pid = np.where(plt, tag & ~RECEPTOR_BIT, -1)
    P = int(pid.max() + 1) if plt.any() else 0
    out = np.zeros((P, N_FEATURES))
    rec = plt & ((tag & RECEPTOR_BIT) != 0)
    fluid = tag == -1
    bonds = np.asarray(bonds).reshape(-1, 2)
    for p in range(P):
        idx = np.nonzero(pid == p)[0]
        ref = x[idx[0]]
        rel = _min_image(x[idx] - ref, box, walls)
        com = ref + rel.mean(axis=0)
        r = rel - rel.mean(axis=0)
        V = v[idx].mean(axis=0)
        out[p, 0:3] = V
        u = v[idx] - V
        L = np.cross(r, u).sum(axis=0)
        I = np.eye(3) * (r * r).sum() - r.T @ r
        out[p, 3:6] = np.linalg.solve(I, L)
        S = -0.5 * (r.T @ f[idx] + f[idx].T @ r)
        out[p, 6:9] = np.linalg.eigvalsh(S)
        if len(bonds):
            mine = pid[bonds[:, 0]] == p
            if mine.any():
                b = bonds[mine]
                d = _min_image(x[b[:, 0]] - x[b[:, 1]], box, walls)
                strain = np.abs(np.linalg.norm(d, axis=1) - r0[mine]) / r0[mine]
                out[p, 9] = strain.max()
        mine_rec = np.nonzero(rec & (pid == p))[0]
        other_rec = np.nonzero(rec & (pid != p))[0]
        if len(mine_rec) and len(other_rec):
            d = _min_image(x[mine_rec][:, None, :] - x[other_rec][None, :, :], box, walls)
            out[p, 10] = float((np.linalg.norm(d, axis=2) < 1.5 * morse_r0).sum())
        fl = np.nonzero(fluid)[0]
        d = _min_image(x[fl] - com, box, walls)
        near = np.linalg.norm(d, axis=1) < flow_radius
        out[p, 11] = float(np.linalg.norm(v[fl][near], axis=1).mean()) if near.any() else 0.0
    return out


def flow_profile(x, v, tag, box, nbins=20):
    """Sec. 4.2 (Fig. 4): the flow across the channel -- nbins equal slabs of y
    in [0, Ly), positions outside counted in the edge slabs; per slab the mean
    v_x of its plasma particles (0 when empty) and their number density."""
    x = np.asarray(x, np.float64)
    v = np.asarray(v, np.float64)
    plasma = np.asarray(tag) == -1
    Lx, Ly, Lz = (float(b) for b in box)
    b = np.clip(np.floor(x[plasma, 1] * nbins / Ly).astype(np.int64), 0, nbins - 1)
    n = np.bincount(b, minlength=nbins).astype(np.float64)
    s = np.bincount(b, weights=v[plasma, 0], minlength=nbins)
    mean = np.where(n > 0, s / np.maximum(n, 1.0), 0.0)
    return mean, n / (Lx * Lz * Ly / nbins)
