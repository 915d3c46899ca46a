"""Pins of the per-platelet measurement oracle (Sec. 3.3) against closed forms."""
import numpy as np
import pytest

from oracle import features as F

REC = F.RECEPTOR_BIT
BOX = (30.0, 30.0, 30.0)


def tetra(center, scale=1.0):
    base = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], float) * scale
    return base + np.asarray(center)


def test_rigid_motion_gives_com_and_angular_velocity():
    """v_i = V + w x r_i (rigid body) is recovered exactly: V and w = I^-1 L."""
    rng = np.random.default_rng(0)
    x = tetra((10, 10, 10)) + 0.1 * rng.standard_normal((4, 3))
    V = np.array([0.3, -0.2, 0.1])
    w = np.array([0.5, 1.5, -0.7])
    r = x - x.mean(0)
    v = V + np.cross(w, r)
    out = F.platelet_features(x, v, np.zeros((4, 3)), np.zeros(4, np.int32), np.zeros((0, 2), int), np.zeros(0),
                              BOX)
    assert np.allclose(out[0, 0:3], V, atol=1e-12)
    assert np.allclose(out[0, 3:6], w, atol=1e-12)


def test_stress_of_a_repulsive_pair():
    """Two members pushed apart along x by +-F at separation d: S has the
    principal values -dF, 0, 0 (force moment -1/2 sum(rF + Fr))."""
    x = np.array([[10.0, 10, 10], [12.0, 10, 10], [11.0, 11.5, 10], [11.0, 10.5, 11.5]])
    f = np.zeros((4, 3))
    f[0, 0], f[1, 0] = -3.0, 3.0       # d = 2 along x, repulsive F = 3
    out = F.platelet_features(x, np.zeros((4, 3)), f, np.zeros(4, np.int32), np.zeros((0, 2), int), np.zeros(0),
                              BOX)
    assert np.allclose(out[0, 6:9], [-6.0, 0.0, 0.0], atol=1e-12)


def test_bond_strain_contacts_and_flow_speed():
    xa = tetra((10, 10, 10))
    xb = tetra((10, 8, 13.2))       # its vertex 2 sits 1.2 above vertex 3 of the first
    fluid = np.array([[10.0, 10.0, 10.5], [10.0, 11.0, 10.0], [10.0, 10.0, 12.5]])
    x = np.concatenate([xa, xb, fluid])
    v = np.zeros_like(x)
    v[8] = [3.0, 4.0, 0.0]            # speed 5, 0.5 from the COM of platelet 0
    v[9] = [0.0, 0.0, 1.0]            # speed 1, 1.0 away
    v[10] = [9.0, 0.0, 0.0]           # 2.5 away: outside the radius of 2
    tag = np.array([0, 0, 0 | REC, 0 | REC, 1 | REC, 1, 1 | REC, 1, -1, -1, -1], np.int32)
    bonds = np.array([[0, 1], [4, 5]])
    d01 = np.linalg.norm(xa[0] - xa[1])
    r0 = np.array([d01 / 1.1, np.linalg.norm(xb[0] - xb[1])])
    out = F.platelet_features(x, v, np.zeros_like(x), tag, bonds, r0, BOX)
    assert out[0, 9] == pytest.approx(0.1, rel=1e-12)
    assert out[1, 9] == pytest.approx(0.0, abs=1e-12)
    # receptor pairs between the platelets closer than 1.5
    d = np.linalg.norm(x[[2, 3]][:, None] - x[[4, 6]][None], axis=2)
    n_close = int((d < 1.5).sum())
    assert n_close == 1
    assert out[0, 10] == 1 and out[1, 10] == 1
    assert out[0, 11] == pytest.approx((5.0 + 1.0) / 2, rel=1e-12)


def test_minimum_image_across_the_box():
    """A platelet straddling the periodic x face measures like an unwrapped one."""
    x = tetra((0.2, 10, 10), 0.5)
    xw = x.copy()
    xw[:, 0] %= BOX[0]
    v = np.random.default_rng(1).standard_normal((4, 3))
    a = F.platelet_features(x + [5, 0, 0], v, np.zeros((4, 3)), np.zeros(4, np.int32), np.zeros((0, 2), int),
                            np.zeros(0), BOX)
    b = F.platelet_features(xw, v, np.zeros((4, 3)), np.zeros(4, np.int32), np.zeros((0, 2), int), np.zeros(0), BOX)
    assert np.allclose(a[:, :10], b[:, :10], atol=1e-12)


def test_flow_profile_of_a_linear_shear_field():
    """Sec. 4.2 flow profile: particles at the slab centres moving with
    v_x = a + b y give back a + b y_c in every slab and the density count /
    slab volume; wall and platelet particles do not count."""
    box = (4.0, 10.0, 5.0)
    nb = 5
    yc = (np.arange(nb) + 0.5) * 2.0
    rng = np.random.default_rng(3)
    pts, vel, tags = [], [], []
    for k, y in enumerate(yc):
        m = k + 2                                   # slab k holds k + 2 plasma particles
        p = np.column_stack([rng.uniform(0, 4, m), np.full(m, y), rng.uniform(0, 5, m)])
        pts.append(p)
        vel.append(np.column_stack([0.3 + 0.05 * p[:, 1], rng.normal(size=m), rng.normal(size=m)]))
        tags.append(np.full(m, -1))
    # walls and a platelet with velocities that would spoil the profile
    pts.append(np.array([[1.0, -0.5, 1.0], [1.0, 5.0, 1.0]]))
    vel.append(np.array([[9.0, 0, 0], [-9.0, 0, 0]]))
    tags.append(np.array([-2, 0]))
    x, v, tag = np.concatenate(pts), np.concatenate(vel), np.concatenate(tags)
    mean, dens = F.flow_profile(x, v, tag, box, nb)
    assert np.allclose(mean, 0.3 + 0.05 * yc, rtol=0, atol=1e-14)
    assert np.allclose(dens, (np.arange(nb) + 2) / (4.0 * 5.0 * 2.0), rtol=1e-14)
