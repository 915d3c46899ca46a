"""Pins of the FP64 oracle against closed forms, invariants, physics and brute force.

Each test names the passage of the paper (or the textbook fact) that fixes the
expected value; none of them re-types the oracle's own formula.
"""
import math

import numpy as np
import pytest

import oracle as O
import synth


def two_body(r, v_rel=(0.0, 0.0, 0.0), tags=(-1, -1), box=(10.0, 10.0, 10.0)):
    x = np.array([[5.0 + r, 5.0, 5.0], [5.0, 5.0, 5.0]])
    v = np.array([list(v_rel), [0.0, 0.0, 0.0]])
    return x, v, np.array(tags, np.int32)


# --------------------------------------------------------------------------
# Eq. 1 -- DPD
# --------------------------------------------------------------------------

@pytest.mark.parametrize("r", [0.1, 0.5, 0.93])
def test_dpd_conservative_matches_eq1_at_points(r):
    """Eq. 1: F^C = a (1 - r/rc) e_ij, zero beyond rc; a=25, rc=1."""
    p = O.make_params((10, 10, 10), gamma=0.0, sigma=0.0)
    x, v, tag = two_body(r)
    f, acc = O.forces_brute(p, x, v, tag)
    assert f[0, 0] == pytest.approx(25.0 * (1.0 - r), rel=1e-13)
    assert abs(f[0, 1]) < 1e-14 and abs(f[0, 2]) < 1e-14
    assert f[1, 0] == -f[0, 0]
    x, v, tag = two_body(1.0001)
    f, _ = O.forces_brute(p, x, v, tag)
    assert np.all(f == 0.0)


@pytest.mark.parametrize("r", [0.7, 0.85, 0.95])
def test_interface_lj_variant_is_repulsive_lj(r):
    """Eq. 3 read with an LJ conservative term (the selectable variant): the
    plasma-platelet conservative force is 24 eps [2 (s/r)^12 - (s/r)^6] / r
    (eps 1, s 0.8) below the LJ minimum 2^(1/6) s and zero beyond it, and its
    energy the LJ potential shifted up by eps; the default reading gives
    a_fp (1 - r/rc) with a_fp = 50."""
    x, v, tag = two_body(r, tags=(-1, 0))
    p = O.make_params((10, 10, 10), gamma=0.0, sigma=0.0, iface_lj=True)
    f, acc = O.forces_brute(p, x, v, tag, X0=x)
    s6 = (0.8 / r) ** 6
    inside = r < 2.0 ** (1.0 / 6.0) * 0.8
    assert f[0, 0] == pytest.approx(24.0 * (2.0 * s6 * s6 - s6) / r if inside else 0.0, rel=1e-12, abs=1e-14)
    assert f[1, 0] == -f[0, 0]
    assert acc["epot"] == pytest.approx(4.0 * (s6 * s6 - s6) + 1.0 if inside else 0.0, rel=1e-12, abs=1e-14)
    p0 = O.make_params((10, 10, 10), gamma=0.0, sigma=0.0)
    f0, _ = O.forces_brute(p0, x, v, tag, X0=x)
    assert f0[0, 0] == pytest.approx(50.0 * (1.0 - r), rel=1e-13)


def test_dpd_conservative_is_minus_gradient_of_energy():
    """F^C = -dU/dr with U = (a rc / 2)(1 - r/rc)^2 -- central difference of the
    oracle's potential energy, a separate code path from its force."""
    p = O.make_params((10, 10, 10), gamma=0.0, sigma=0.0)
    for r in (0.2, 0.6, 0.9):
        h = 1e-6
        up = O.forces_brute(p, *two_body(r + h))[1]["epot"]
        um = O.forces_brute(p, *two_body(r - h))[1]["epot"]
        f = O.forces_brute(p, *two_body(r))[0][0, 0]
        assert f == pytest.approx(-(up - um) / (2 * h), rel=1e-7)


def test_dpd_dissipative_opposes_relative_motion():
    """Eq. 1: F^D = -gamma w^D (e.v) e with w^D = (1 - r)^2 (fluctuation-dissipation
    reading): particles approaching each other are pushed apart, receding pulled."""
    p = O.make_params((10, 10, 10), a_ff=0.0, sigma=0.0)
    r = 0.4
    # particle 0 at +r moving towards particle 1 (v_x < 0): e.v < 0 -> repulsive (+x on 0)
    f, _ = O.forces_brute(p, *two_body(r, v_rel=(-2.0, 0, 0)))
    assert f[0, 0] == pytest.approx(4.5 * (1 - r) ** 2 * 2.0, rel=1e-13)
    f, _ = O.forces_brute(p, *two_body(r, v_rel=(2.0, 0, 0)))
    assert f[0, 0] == pytest.approx(-4.5 * (1 - r) ** 2 * 2.0, rel=1e-13)
    # motion perpendicular to e gives no central dissipative force
    f, _ = O.forces_brute(p, *two_body(r, v_rel=(0.0, 3.0, 0)))
    assert abs(f[0, 0]) < 1e-14


def test_random_force_symmetric_gaussian_scaled_by_inverse_sqrt_dt():
    """Eq. 1 (Groot-Warren reading of the sqrt(dt) term): F^R = sigma w zeta / sqrt(dt),
    zeta symmetric in (i, j); halving dt multiplies F^R by sqrt(2)."""
    p = O.make_params((10, 10, 10), a_ff=0.0, gamma=0.0)
    x, v, tag = two_body(0.3)
    f1, _ = O.forces_brute(p, x, v, tag, dt=0.01, n_time=7)
    f2, _ = O.forces_brute(p, x, v, tag, dt=0.005, n_time=7)
    assert f2[0, 0] == pytest.approx(f1[0, 0] * math.sqrt(2.0), rel=1e-13)
    z = O.zeta(p, 0, 1, 7, 0)
    assert O.zeta(p, 1, 0, 7, 0) == z
    assert f1[0, 0] == pytest.approx(3.0 * 0.7 * z / math.sqrt(0.01), rel=1e-13)
    assert f1[1, 0] == -f1[0, 0]


def test_zeta_moments_are_standard_normal():
    """zeta ~ N(0,1) (Eq. 1): mean 0, variance 1, kurtosis 3 within 4 standard errors,
    over 40,000 pair/time counters."""
    p = O.make_params((10, 10, 10))
    z = np.array([O.zeta(p, i, i + 1 + (i % 7), t, 0) for i in range(4000) for t in range(10)])
    n = z.size
    assert abs(z.mean()) < 4.0 / math.sqrt(n)
    assert abs(z.var() - 1.0) < 4.0 * math.sqrt(2.0 / n)
    assert abs((z ** 4).mean() - 3.0) < 4.0 * math.sqrt(96.0 / n)
    # distinct counters give distinct draws; keys change the stream
    p2 = O.make_params((10, 10, 10), seed=12345)
    assert O.zeta(p2, 0, 1, 7, 0) != O.zeta(p, 0, 1, 7, 0)
    assert O.zeta(p, 0, 1, 7, 1) != O.zeta(p, 0, 1, 7, 0)


def test_uniform_noise_variant_moments():
    """The speed option's zeta: a uniform variate on [-sqrt(3), sqrt(3)] has mean
    0, variance 1 and fourth moment 9/5; within 4 standard errors over 40,000
    pair/time counters, bounded by sqrt(3), and flat over 12 equal bins."""
    p = O.make_params((10, 10, 10), uniform_noise=True)
    z = np.array([O.zeta(p, i, i + 1 + (i % 7), t, 0) for i in range(4000) for t in range(10)])
    n = z.size
    assert abs(z.mean()) < 4.0 / math.sqrt(n)
    assert abs((z ** 2).mean() - 1.0) < 4.0 * math.sqrt(0.8 / n)
    assert abs((z ** 4).mean() - 1.8) < 4.0 * math.sqrt((9.0 - 1.8 ** 2) / n)
    assert np.abs(z).max() < math.sqrt(3.0)
    counts, _ = np.histogram(z, bins=12, range=(-math.sqrt(3.0), math.sqrt(3.0)))
    e = n / 12.0
    assert ((counts - e) ** 2 / e).sum() < 40.0          # chi-square, 11 dof: p ~ 4e-5
    # the same counters as the Gaussian draw, only the transform differs
    g = O.make_params((10, 10, 10))
    assert O.zeta(p, 3, 9, 4, 0) != O.zeta(g, 3, 9, 4, 0)
    assert O.zeta(p, 9, 3, 4, 0) == O.zeta(p, 3, 9, 4, 0)


def test_uniform_noise_variant_thermalises_to_kT():
    """Fluctuation-dissipation (Eq. 1 with sigma^2 = 2 gamma kT) needs only the
    noise's first two moments: the DPD fluid driven by the uniform variate
    settles at kT = 1 as well."""
    s = synth.plasma_box(n=3 * 8 ** 3, seed=11)
    p = O.system_params(s, uniform_noise=True)
    x, v, f = s.x, s.v, None
    n0 = 0
    Ts = []
    for block in range(24):
        x, v, f = O.run_respa(p, x, v, s.tag, dt_f=0.01, n_outer=25, n0=n0, t0=n0 * 0.01, forces=f)
        n0 += 25
        if block >= 14:
            Ts.append(O.kinetics(p, x, v, s.tag)["T"])
    assert np.mean(Ts) == pytest.approx(1.0, abs=0.03)


# Known-answer vectors of Philox4x32-10 published with the SC'11 generator
# (Salmon, Moraes, Dror and Shaw, "Parallel random numbers: as easy as 1, 2,
# 3"; the Random123 distribution's known-answer file): counter, key, output.
PHILOX4X32_10_KAT = [
    ((0x00000000, 0x00000000, 0x00000000, 0x00000000), (0x00000000, 0x00000000),
     (0x6627e8d5, 0xe169c58d, 0xbc57ac4c, 0x9b00dbd8)),
    ((0xffffffff, 0xffffffff, 0xffffffff, 0xffffffff), (0xffffffff, 0xffffffff),
     (0x408f276d, 0x41c83b0e, 0xa20bc7c6, 0x6d5451fd)),
    ((0x243f6a88, 0x85a308d3, 0x13198a2e, 0x03707344), (0xa4093822, 0x299f31d0),
     (0xd16cfe09, 0x94fdcceb, 0x5001e420, 0x24126ea1)),
]


@pytest.mark.parametrize("ctr,key,out", PHILOX4X32_10_KAT)
def test_philox4x32_10_known_answers(ctr, key, out):
    """Philox4x32-10 (the generator of Eq. 1's zeta_ij) reproduces the published
    known-answer vectors bit for bit: a wrong multiplier, Weyl constant, round
    count or word order fails here."""
    assert O.philox4x32_10(ctr, key) == list(out)


def test_philox_words_are_uniform_and_avalanche():
    """Philox4x32-10 (SC'11) output words: uniform top bytes (chi-square) and a
    single flipped counter bit changes about half of the 128 output bits."""
    words = np.array([O.philox4x32_10([i, 0, 0, 0], [1, 2]) for i in range(20000)], dtype=np.uint64)
    top = (words >> 24).ravel()
    counts = np.bincount(top.astype(np.int64), minlength=256)
    exp = top.size / 256
    chi2 = ((counts - exp) ** 2 / exp).sum()
    assert chi2 < 255 + 5 * math.sqrt(2 * 255)
    flips = []
    for i in range(200):
        a = O.philox4x32_10([i, 5, 6, 7], [9, 9])
        b = O.philox4x32_10([i ^ 1, 5, 6, 7], [9, 9])
        flips.append(sum(bin(x ^ y).count("1") for x, y in zip(a, b)))
    assert abs(np.mean(flips) - 64.0) < 3.0


def test_gaussian_transform_tails():
    """Box-Muller: u1 = 1 gives zeta = 0; the smallest u1 = 2^-24 gives the largest
    magnitude sqrt(2 ln 2^24) = 5.768."""
    assert O.gauss_from_bits(0xFFFFFF00, 0) == 0.0
    assert O.gauss_from_bits(0, 0) == pytest.approx(math.sqrt(2 * 24 * math.log(2)), rel=1e-14)


# --------------------------------------------------------------------------
# Eq. 2 / Eq. 4 -- LJ, Morse, bonds
# --------------------------------------------------------------------------

def plt_pair(r, rec=True, same=False, X0_far=True):
    x = np.array([[5.0 + r, 5.0, 5.0], [5.0, 5.0, 5.0]])
    v = np.zeros((2, 3))
    bit = O_REC if rec else 0
    tag = np.array([0 | bit, (0 if same else 1) | bit], np.int32)
    X0 = x.copy()
    if X0_far:
        X0[0, 0] += 10.0
    return x, v, tag, X0


O_REC = synth.RECEPTOR_BIT


def test_lj_zero_crossing_and_minimum():
    """Eq. 2 LJ: F = 0 at r = 2^(1/6) sigma, repulsive inside, attractive outside
    (sigma = 0.8), zero beyond the cut-off 2.5 sigma = 2.0."""
    p = O.make_params((20, 20, 20), m_D=0.0)
    rmin = 2 ** (1 / 6) * 0.8
    x, v, tag, X0 = plt_pair(rmin, rec=False)
    f, _ = O.forces_brute(p, x, v, tag, X0=X0)
    assert abs(f[0, 0]) < 1e-12
    f, _ = O.forces_brute(p, *plt_pair(0.85, rec=False)[:3], X0=plt_pair(0.85, rec=False)[3])
    assert f[0, 0] > 0
    f, _ = O.forces_brute(p, *plt_pair(1.2, rec=False)[:3], X0=plt_pair(1.2, rec=False)[3])
    assert f[0, 0] < 0
    f, _ = O.forces_brute(p, *plt_pair(2.01, rec=False)[:3], X0=plt_pair(2.01, rec=False)[3])
    assert np.all(f == 0)
    # the LJ well depth at r_min is -eps (+ the cut-off shift 4 eps [(s/rc)^12 - (s/rc)^6])
    _, acc = O.forces_brute(p, *plt_pair(rmin, rec=False)[:3], X0=plt_pair(rmin, rec=False)[3])
    s = 0.8 / 2.0
    assert acc["epot"] == pytest.approx(-1.0 - 4 * (s ** 12 - s ** 6), rel=1e-12)


@pytest.mark.parametrize("kind", ["lj", "morse", "bond"])
def test_force_is_minus_gradient(kind):
    """Eq. 2: each force equals -dU/dr of the oracle's separately coded energy."""
    p = O.make_params((20, 20, 20), f_A=0.0)
    for r in (0.8, 0.95, 1.3, 1.9, 3.0):
        if kind == "lj" and r > 1.95:
            continue

        def ef(rr):
            x, v, tag, X0 = plt_pair(rr, rec=(kind == "morse"))
            if kind == "lj":
                pp = O.make_params((20, 20, 20), m_D=0.0)
                f, acc = O.forces_brute(pp, x, v, tag, X0=X0)
            elif kind == "morse":
                pp = O.make_params((20, 20, 20), lj_eps=0.0)
                f, acc = O.forces_brute(pp, x, v, tag, X0=X0)
            else:
                tag = np.array([0, 0], np.int32)
                X0 = x.copy()  # same platelet at rest distance < 2.5: LJ excluded
                f, acc = O.forces_brute(p, x, v, tag, X0=X0, bonds=np.array([[0, 1]]),
                                        r0=np.array([1.1]))
            return f[0, 0], acc["epot"]

        h = 1e-6
        f0, _ = ef(r)
        up = ef(r + h)[1]
        um = ef(r - h)[1]
        assert f0 == pytest.approx(-(up - um) / (2 * h), rel=1e-6, abs=1e-9)


def test_morse_printed_form_equals_standard_form():
    """Eq. 2's Morse U = D[e^{a(1-r/r0)} - 2 e^{a(1-r/r0)/2}] is the textbook
    D[(1 - e^{-b(r-re)})^2 - 1] with b = a/(2 r0), re = r0 (same minimum -D at r0)."""
    p = O.make_params((20, 20, 20), lj_eps=0.0, m_rc=50.0)
    for r in (0.7, 1.0, 1.6, 3.0):
        x, v, tag, X0 = plt_pair(r)
        _, acc = O.forces_brute(p, x, v, tag, X0=X0)
        b = 2.0 / 2.0
        std = 2.0 * ((1 - math.exp(-b * (r - 1.0))) ** 2 - 1.0)
        shift = 2.0 * ((1 - math.exp(-b * (50.0 - 1.0))) ** 2 - 1.0)
        assert acc["epot"] == pytest.approx(std - shift, rel=1e-12, abs=1e-12)


def test_morse_only_between_receptors_of_different_platelets():
    """Eq. 4: the inter-platelet Morse acts between receptor sites of different
    platelets; same-platelet or non-receptor pairs feel no Morse."""
    p = O.make_params((20, 20, 20), lj_eps=0.0)
    for rec, same, expect in ((True, False, True), (False, False, False), (True, True, False)):
        x, v, tag, X0 = plt_pair(1.5, rec=rec, same=same)
        f, _ = O.forces_brute(p, x, v, tag, X0=X0)
        assert (abs(f[0, 0]) > 0) == expect


def test_receptor_term_fA():
    """Eq. 4: the receptor term adds f_A (1 - r/r0) along e_ij."""
    p0 = O.make_params((20, 20, 20), lj_eps=0.0)
    p1 = O.make_params((20, 20, 20), lj_eps=0.0, f_A=3.0)
    x, v, tag, X0 = plt_pair(1.4)
    d = O.forces_brute(p1, x, v, tag, X0=X0)[0][0, 0] - O.forces_brute(p0, x, v, tag, X0=X0)[0][0, 0]
    assert d == pytest.approx(3.0 * (1 - 1.4), rel=1e-12)


def test_lj_rest_distance_exclusion():
    """With an exclusion radius of 2.5, same-platelet pairs closer than that at
    rest feel no LJ and far-at-rest pairs do; the default radius excludes every
    pair of one platelet."""
    pd = O.make_params((20, 20, 20), m_D=0.0)
    x, v, tag, X0 = plt_pair(1.0, rec=False, same=True, X0_far=True)
    assert np.all(O.forces_brute(pd, x, v, tag, X0=X0)[0] == 0)
    p = O.make_params((20, 20, 20), m_D=0.0, lj_excl=2.5)
    x, v, tag, X0 = plt_pair(1.0, rec=False, same=True, X0_far=False)
    assert np.all(O.forces_brute(p, x, v, tag, X0=X0)[0] == 0)
    x, v, tag, X0 = plt_pair(1.0, rec=False, same=True, X0_far=True)
    assert O.forces_brute(p, x, v, tag, X0=X0)[0][0, 0] != 0


# --------------------------------------------------------------------------
# sums, images, invariants
# --------------------------------------------------------------------------

def small_platelet_system(seed=3):
    return synth.config_couette_platelet(seed=seed, scale=0.4)


def test_cells_equal_brute_force_all_levels():
    """The cell-list path sums exactly the pairs the all-pairs path sums."""
    s = small_platelet_system()
    p = O.system_params(s, le_offset=1.37)
    fb, _ = O.forces_brute(p, s.x, s.v, s.tag, X0=s.X0, bonds=s.bonds, r0=s.r0, n_time=3)
    fc = O.forces_cells(p, s.x, s.v, s.tag, X0=s.X0, bonds=s.bonds, r0=s.r0, n_time=3)
    scale = np.abs(fb).max()
    assert np.abs(fb - fc).max() <= 1e-12 * scale


def test_momentum_conserved_without_walls_or_body_force():
    """Newton's third law holds pair by pair (F^R antisymmetric by the symmetric
    zeta key): the net force vanishes to rounding, Lees-Edwards images included."""
    s = small_platelet_system()
    p = O.system_params(s, le_offset=2.9)
    f, _ = O.forces_brute(p, s.x, s.v, s.tag, X0=s.X0, bonds=s.bonds, r0=s.r0)
    assert np.abs(f.sum(axis=0)).max() <= 1e-12 * np.abs(f).sum()


def test_minimum_image_across_periodic_faces():
    """A pair straddling the x face interacts exactly like the unwrapped pair."""
    p = O.make_params((10, 10, 10), sigma=0.0)
    x = np.array([[0.1, 5, 5], [9.7, 5, 5]])
    f, _ = O.forces_brute(p, x, np.zeros((2, 3)), np.array([-1, -1], np.int32))
    assert f[0, 0] == pytest.approx(25.0 * (1 - 0.4), rel=1e-12)


def test_lees_edwards_image_shift():
    """Lees-Edwards: the image of a particle across y is displaced by delta in x and
    by shear_rate*Ly in v_x; a pair that only touches through the shifted image."""
    p = O.make_params((10, 10, 10), le_rate=0.1, le_offset=3.0, sigma=0.0, gamma=0.0)
    # i near the top at x=5.0, j near the bottom at x=2.2: image of j at x=5.2, y+10
    x = np.array([[5.0, 9.8, 5.0], [2.2, 0.1, 5.0]])
    f, _ = O.forces_brute(p, x, np.zeros((2, 3)), np.array([-1, -1], np.int32))
    r = math.hypot(0.2, 0.3)
    assert f[0, 0] == pytest.approx(25 * (1 - r) * (-0.2 / r), rel=1e-12)
    assert f[0, 1] == pytest.approx(25 * (1 - r) * (-0.3 / r), rel=1e-12)
    # dissipative force sees the image velocity offset shear_rate*Ly = 1 in v_x
    pd = O.make_params((10, 10, 10), le_rate=0.1, le_offset=3.0, sigma=0.0, a_ff=0.0)
    f, _ = O.forces_brute(pd, x, np.zeros((2, 3)), np.array([-1, -1], np.int32))
    ex, ey = -0.2 / r, -0.3 / r
    edotv = ex * (0.0 - 1.0)  # v_i - (v_j + 1 x^)
    assert f[0, 0] == pytest.approx(-4.5 * (1 - r) ** 2 * edotv * ex, rel=1e-12)


def test_walls_are_not_periodic_in_y():
    p = O.make_params((10, 10, 10), walls=True, sigma=0.0)
    x = np.array([[5.0, 9.9, 5.0], [5.0, 0.1, 5.0]])
    f, _ = O.forces_brute(p, x, np.zeros((2, 3)), np.array([-1, -1], np.int32))
    assert np.all(f == 0)


# --------------------------------------------------------------------------
# FP32 neighbour predicate vs FP64 distances
# --------------------------------------------------------------------------

@pytest.mark.parametrize("le", [False, True])
def test_pairs_f32_agree_with_fp64_sets(le):
    """The FP32 list predicate selects the same pairs as exact distances, except
    pairs within 1e-5 of the cut-off."""
    rng = np.random.default_rng(5)
    L = np.float32(7.0)
    n = 600
    x = (rng.random((n, 3)) * L).astype(np.float32)
    tag = np.full(n, -1, np.int32)
    delta = np.float32(2.345) if le else np.float32(0.0)
    cut = 1.3
    pr = O.pairs_f32(x, tag, np.array([L, L, L], np.float32), O.KIND_FLUID, np.float32(cut * cut),
                     le=le, delta=delta)
    got = set(map(tuple, pr.tolist()))
    xd = x.astype(np.float64)
    exact = set()
    near = set()
    for i in range(n):
        d = xd[i] - xd[i + 1:]
        if le:
            up = d[:, 1] > L / 2
            dn = d[:, 1] < -L / 2
            d[up, 1] -= L
            d[up, 0] -= float(delta)
            d[dn, 1] += L
            d[dn, 0] += float(delta)
        else:
            d[:, 1] -= L * np.round(d[:, 1] / L)
        d[:, 0] -= L * np.round(d[:, 0] / L)
        d[:, 2] -= L * np.round(d[:, 2] / L)
        r = np.sqrt((d * d).sum(1))
        for k in np.nonzero(r < cut)[0]:
            exact.add((i, i + 1 + int(k)))
        for k in np.nonzero(np.abs(r - cut) < 1e-5)[0]:
            near.add((i, i + 1 + int(k)))
    assert (got ^ exact) <= near
    assert len(got) > 1000


def test_pairs_f32_kinds_partition_dpd_pairs():
    """Kinds 0 and 1 split the DPD pairs by level; wall-wall pairs are in neither."""
    s = small_platelet_system()
    x32 = s.x.astype(np.float32)
    box = np.array(s.box, np.float32)
    cut2 = np.float32(1.3 ** 2)
    k0 = O.pairs_f32(x32, s.tag, box, O.KIND_FLUID, cut2, le=True)
    k1 = O.pairs_f32(x32, s.tag, box, O.KIND_IFACE, cut2, le=True)
    t = s.tag
    assert np.all((t[k0[:, 0]] < 0) & (t[k0[:, 1]] < 0))
    assert np.all((t[k1[:, 0]] >= 0) != (t[k1[:, 1]] >= 0))
    assert len(k1) > 0


# --------------------------------------------------------------------------
# Table 1 integrators
# --------------------------------------------------------------------------

def shell_only(n_shell=300, seed=11):
    s = synth.platelet_system((30.0, 30.0, 30.0), 0, 1, n_shell, synth.scaled_radii(n_shell),
                              seed=seed, centers=[(15.0, 15.0, 15.0)])
    return s


def total_energy(p, x, v, s):
    _, acc = O.forces_brute(p, x, v, s.tag, X0=s.X0, bonds=s.bonds, r0=s.r0,
                            level_mask=O.LVL_PLT)
    return 0.5 * (v * v).sum() + acc["epot"]


def test_velocity_verlet_time_reversible():
    """Velocity-Verlet / RESPA are time-reversible for conservative forces: run n
    steps, reverse velocities, run n steps, and the start state returns."""
    s = shell_only()
    p = O.system_params(s)
    v0 = s.v * 0.5
    x1, v1, _ = O.run_respa(p, s.x, v0, s.tag, X0=s.X0, bonds=s.bonds, r0=s.r0, dt_f=0.002,
                            k_m=1, k_p=3, n_outer=40)
    x2, v2, _ = O.run_respa(p, x1, -v1, s.tag, X0=s.X0, bonds=s.bonds, r0=s.r0, dt_f=0.002,
                            k_m=1, k_p=3, n_outer=40)
    assert np.abs(x2 - s.x).max() < 1e-9
    assert np.abs(v2 + v0).max() < 1e-8


def test_nve_energy_error_scales_as_dt_squared():
    """Velocity-Verlet is second order: the energy fluctuation of a bonded shell
    (bonds and angles) shrinks ~4x when dt is halved, and stays small."""
    s = shell_only()
    p = O.system_params(s)
    e0 = total_energy(p, s.x, s.v, s)
    errs = []
    for dt, n in ((0.002, 100), (0.001, 200)):
        x, v, _ = O.run_respa(p, s.x, s.v, s.tag, X0=s.X0, bonds=s.bonds, r0=s.r0, dt_f=dt,
                              n_outer=n)
        errs.append(abs(total_energy(p, x, v, s) - e0))
    assert errs[1] < errs[0] / 2.5
    assert errs[1] < 1e-3 * abs(e0) + 1e-2


def test_respa_inner_steps_match_fine_verlet_for_platelet_only():
    """With only platelet forces, RESPA(k_p) over dt_f equals velocity-Verlet with
    dt_f/k_p (the outer and middle levels carry no force)."""
    s = shell_only()
    p = O.system_params(s)
    x1, v1, _ = O.run_respa(p, s.x, s.v, s.tag, X0=s.X0, bonds=s.bonds, r0=s.r0, dt_f=0.004,
                            k_m=2, k_p=2, n_outer=5)
    x2, v2, _ = O.run_respa(p, s.x, s.v, s.tag, X0=s.X0, bonds=s.bonds, r0=s.r0, dt_f=0.001,
                            n_outer=20)
    assert np.abs(x1 - x2).max() < 1e-11
    assert np.abs(v1 - v2).max() < 1e-9


def test_sts_is_respa_k1_with_one_level():
    """With only the fluid level populated, the single-pass velocity-Verlet and
    Table 1 at k_m = k_p = 1 perform the same arithmetic (bitwise)."""
    s = synth.plasma_box(n=3 * 6 ** 3, seed=4, walls=True, body_force=0.02)
    p = O.system_params(s)
    x1, v1, _ = O.run_sts(p, s.x, s.v, s.tag, dt=0.01, n_steps=4)
    x2, v2, _ = O.run_respa(p, s.x, s.v, s.tag, dt_f=0.01, n_outer=4)
    assert np.array_equal(x1, x2) and np.array_equal(v1, v2)


def test_sts_time_reversible():
    """Single-pass velocity-Verlet is time-reversible for the conservative shell."""
    s = shell_only()
    p = O.system_params(s)
    x1, v1, _ = O.run_sts(p, s.x, s.v, s.tag, X0=s.X0, bonds=s.bonds, r0=s.r0, dt=0.002, n_steps=60)
    x2, v2, _ = O.run_sts(p, x1, -v1, s.tag, X0=s.X0, bonds=s.bonds, r0=s.r0, dt=0.002, n_steps=60)
    assert np.abs(x2 - s.x).max() < 1e-9
    assert np.abs(v2 + s.v).max() < 1e-8


def test_walls_bounce_back():
    """No-slip bounce-back (Sec. 3.1 walls): a particle crossing y = 0 is mirrored
    and its velocity reversed."""
    p = O.make_params((10, 10, 10), walls=True, a_ff=0.0, gamma=0.0, sigma=0.0)
    x = np.array([[5.0, 0.05, 5.0]])
    v = np.array([[1.0, -10.0, 0.5]])
    x1, v1, _ = O.run_respa(p, x, v, np.array([-1], np.int32), dt_f=0.01, n_outer=1)
    assert x1[0, 1] == pytest.approx(0.05, abs=1e-12)
    assert np.allclose(v1[0], [-1.0, 10.0, -0.5])
    # the 0.005 spent beyond the wall is retraced in x and z as well
    assert x1[0, 0] == pytest.approx(5.0, abs=1e-12)
    assert x1[0, 2] == pytest.approx(5.0, abs=1e-12)


def test_bounce_back_independent_of_substeps():
    """Table 1 drifts at the innermost level; a walled plasma particle that
    feels no inner force must end at the same place however the drift is split."""
    p = O.make_params((10, 10, 10), walls=True, a_ff=0.0, gamma=0.0, sigma=0.0)
    x = np.array([[5.0, 0.03, 5.0]])
    v = np.array([[2.0, -7.0, -1.0]])
    tag = np.array([-1], np.int32)
    xa, va, _ = O.run_respa(p, x, v, tag, dt_f=0.01, n_outer=1)
    xb, vb, _ = O.run_respa(p, x, v, tag, dt_f=0.01, k_m=2, k_p=5, n_outer=1)
    assert np.allclose(xa, xb, atol=1e-14) and np.allclose(va, vb, atol=1e-14)


# --------------------------------------------------------------------------
# thermodynamics (Groot & Warren 1997) on the oracle
# --------------------------------------------------------------------------

@pytest.mark.slow
def test_dpd_temperature_and_equation_of_state():
    """sigma^2 = 2 gamma kT fixes kT = 1: within 1.5% at dt = 0.01 (the
    discretisation leaves the measured kT about 1% high).  Pressure: the C virial sum equals an independent numpy sum over pair
    distances, and the excess-pressure coefficient alpha = (p - rho kT)/(a rho^2)
    lies between 0.088 and Groot & Warren's high-density fit 0.101 (their fit
    overshoots at rho = 3, where alpha is ~0.092)."""
    s = synth.plasma_box(n=3 * 8 ** 3, seed=7)
    p = O.system_params(s)
    L = s.box[0]
    x, v, f = s.x, s.v, None
    n0 = 0
    Ts, Ps, Pex_c, Pex_np = [], [], [], []
    for block in range(138):   # 4.5 tau of relaxation from random positions, then 30 tau
        x, v, f = O.run_respa(p, x, v, s.tag, dt_f=0.01, n_outer=25, n0=n0, t0=n0 * 0.01,
                              forces=f)
        n0 += 25
        if block < 18:
            continue
        kin = O.kinetics(p, x, v, s.tag)
        Ts.append(kin["T"])
        if block % 10:
            continue
        _, acc = O.forces_cells(p, x, v, s.tag, n_time=n0, with_acc=True)
        Ps.append(O.pressure(p, kin, acc))
        Pex_c.append(np.trace(acc["vir_c"]) / (3 * L ** 3))
        d = x[:, None, :] - x[None, :, :]
        d -= L * np.round(d / L)
        r = np.sqrt((d * d).sum(-1))[np.triu_indices(len(x), 1)]
        r = r[r < 1.0]
        Pex_np.append((25.0 * (1.0 - r) * r).sum() / (3 * L ** 3))
    # 120 samples 0.25 tau apart: the standard error of the mean is about 0.2%
    assert np.mean(Ts) == pytest.approx(1.0, rel=0.015)
    assert np.mean(Pex_c) == pytest.approx(np.mean(Pex_np), rel=1e-10)
    alpha = (np.mean(Ps) - 3.0 * np.mean(Ts)) / (25.0 * 9.0)
    assert 0.088 < alpha < 0.101


def test_ideal_gas_pressure():
    """a = 0: the DPD thermostat alone gives the ideal-gas law p = rho kT."""
    s = synth.plasma_box(n=3 * 6 ** 3, seed=8)
    p = O.system_params(s, a_ff=0.0)
    x, v, f, n0 = s.x, s.v, None, 0
    Ps, Ts = [], []
    for block in range(16):
        x, v, f = O.run_respa(p, x, v, s.tag, dt_f=0.01, n_outer=25, n0=n0, t0=n0 * 0.01, forces=f)
        n0 += 25
        _, acc = O.forces_brute(p, x, v, s.tag, n_time=n0)
        kin = O.kinetics(p, x, v, s.tag)
        Ps.append(O.pressure(p, kin, acc))
        Ts.append(kin["T"])
    n = s.n
    assert np.mean(Ps) == pytest.approx(np.mean(Ts) * (3 * n - 3) / (3 * s.box[0] ** 3), rel=1e-12)
    assert np.mean(Ts) == pytest.approx(1.0, abs=0.03)


def test_wall_temperature_hand_built_slabs():
    """Walls: the peculiar velocity is taken against the mean v_x of the mobile
    particles in each slab of y.  Each of 4 slabs holds two particles at
    u_b +- a_b in x plus (0, c, 0): K_xx = sum 2 a_b^2 and K_yy = 8 c^2 whatever
    the stream u_b; a wall particle (any velocity) and a particle above Ly (out
    of every slab mean, but peculiar against the top slab) complete the set."""
    p = O.make_params((4.0, 8.0, 4.0), walls=True)
    u = [0.3, 1.1, -0.7, 2.0]
    a = [0.1, 0.25, 0.4, 0.05]
    c = 0.2
    x, v, tag = [], [], []
    for b in range(4):
        for sgn in (1.0, -1.0):
            x.append((1.0, 2.0 * b + 0.5 + 0.5 * (sgn > 0), 1.0))
            v.append((u[b] + sgn * a[b], c, 0.0))
            tag.append(synth.TAG_FLUID)
    x.append((2.0, 4.0, 2.0)); v.append((50.0, -30.0, 9.0)); tag.append(synth.TAG_WALL)
    x.append((2.0, 8.3, 2.0)); v.append((u[3] + 0.5, 0.0, 0.0)); tag.append(synth.TAG_FLUID)
    x, v, tag = np.array(x), np.array(v), np.array(tag, np.int32)
    kin = O.kinetics(p, x, v, tag, nbins=4)
    Kxx = 2.0 * sum(ai * ai for ai in a) + 0.25
    assert kin["K"][0, 0] == pytest.approx(Kxx, rel=1e-14)
    assert kin["K"][1, 1] == pytest.approx(8 * c * c, rel=1e-14)
    assert kin["K"][0, 1] == pytest.approx(0.0, abs=1e-15)
    assert kin["T"] == pytest.approx((Kxx + 8 * c * c) / (3 * 9), rel=1e-14)
    assert kin["ke"] == pytest.approx(0.5 * (v[tag != synth.TAG_WALL] ** 2).sum(), rel=1e-14)


COUETTE_RATE = 0.5


def couette_run(n_blocks=55, rate=COUETTE_RATE, seed=9):
    """An 8^3 Lees-Edwards box sheared at `rate` from the linear profile:
    the y-binned v_x and the xy shear stress (kinetic + every pair force)
    sampled every 0.3 tau after 3 tau."""
    s = synth.plasma_box(n=3 * 8 ** 3, seed=seed, shear_rate=rate)
    p = O.system_params(s)
    v = s.v.copy()
    v[:, 0] += rate * (s.x[:, 1] - s.box[1] / 2)
    x, f, n0 = s.x, None, 0
    V = s.box[0] * s.box[1] * s.box[2]
    profs, sxy = [], []
    for block in range(n_blocks):
        x, v, f = O.run_respa(p, x, v, s.tag, dt_f=0.01, n_outer=30, n0=n0, t0=n0 * 0.01, forces=f)
        n0 += 30
        if block < 10:
            continue
        kin = O.kinetics(p, x, v, s.tag, nbins=8)
        profs.append(kin["prof_vx"])
        p.le_offset = (rate * s.box[1] * n0 * 0.01) % s.box[0]
        _, acc = O.forces_cells(p, x, v, s.tag, n_time=n0, with_acc=True)
        sxy.append((kin["K"][0, 1] + acc["vir"][0, 1]) / V)
    return s, np.array(profs), np.array(sxy)


@pytest.fixture(scope="module")
def couette():
    return couette_run()


@pytest.mark.slow
def test_couette_linear_profile_under_lees_edwards(couette):
    """Lees-Edwards shear gives a linear v_x(y) with the imposed slope: within 5%
    and R^2 > 0.99, at a shear rate of 0.5 over 13.5 tau.  (At the
    channel's 0.05 the thermal noise of the slope in this box is about 15% after 30 tau;
    the tenfold rate keeps the pin within seconds.)"""
    s, profs, _ = couette
    prof = profs.mean(0)
    yc = (np.arange(8) + 0.5) * s.box[1] / 8
    slope, icpt = np.polyfit(yc, prof, 1)
    assert slope == pytest.approx(COUETTE_RATE, rel=0.05)
    pred = slope * yc + icpt
    r2 = 1 - ((prof - pred) ** 2).sum() / ((prof - prof.mean()) ** 2).sum()
    assert r2 > 0.99


def block_mean(a, nb=9):
    a = np.asarray(a)
    b = a[:len(a) // nb * nb].reshape(nb, -1).mean(1)
    return b.mean(), b.std(ddof=1) / np.sqrt(nb)


@pytest.mark.slow
def test_poiseuille_viscosity_consistent_with_couette_stress(couette):
    """Two independent measurements of the plasma viscosity agree within their
    error bars: eta = -<sigma_xy> / shear rate from the Lees-Edwards stress,
    and eta from the curvature of the Poiseuille profile of a walled channel
    under a body force g, u(y) = rho g y (Ly - y) / (2 eta) (no-slip walls of
    Sec. 3.1, started on the profile of a guess and averaged for 20 tau)."""
    _, _, sxy = couette
    eta_c, se_c = block_mean(-sxy / COUETTE_RATE)
    box, g = (6.0, 12.0, 6.0), 0.05
    s = synth.plasma_box(box=box, walls=True, body_force=g, seed=31)
    p = O.system_params(s)
    mob = s.tag == synth.TAG_FLUID
    v = s.v.copy()
    y = s.x[mob, 1]
    v[mob, 0] += 3.0 * g * y * (box[1] - y) / (2.0 * 0.85)
    x, f, n0 = s.x, None, 0
    nb = 12
    yc = (np.arange(nb) + 0.5) * box[1] / nb
    etas = []
    for block in range(75):
        x, v, f = O.run_respa(p, x, v, s.tag, dt_f=0.01, n_outer=40, n0=n0, t0=n0 * 0.01, forces=f)
        n0 += 40
        if block < 25:
            continue
        u = O.kinetics(p, x, v, s.tag, nbins=nb)["prof_vx"]
        c = np.polyfit(yc, u, 2)
        etas.append(-3.0 * g / (2.0 * c[0]))
    eta_p, se_p = block_mean(etas, nb=10)
    assert 0.6 < eta_c < 1.1
    assert abs(eta_p - eta_c) < 3.0 * np.hypot(se_c, se_p) + 0.02 * eta_c


@pytest.mark.slow
def test_nve_energy_drift_of_bonded_shells_with_lj():
    """CGMD in NVE (no fluid, no thermostat): two bonded 200-particle shells
    that start within the LJ range of each other (Eq. 2 bonds and LJ; the
    receptor Morse and the angle term switched off), velocity-Verlet at
    dt = 0.001 for 10^4 steps.
    The total energy stays within 1e-4 of its start, and its linear drift
    over the run (the fitted slope times the duration) is below 1e-4 of it."""
    n_shell, gap = 200, 1.2
    r = synth.scaled_radii(n_shell)
    s = synth.platelet_system((30.0, 30.0, 30.0), 0, 2, n_shell, r, seed=23,
                              centers=[(15.0 - r[0] - gap / 2, 15.0, 15.0), (15.0 + r[0] + gap / 2, 15.0, 15.0)])
    p = O.system_params(s, m_D=0.0, m_rc=2.0, k_a=0.0)
    v = 0.5 * s.v

    def energy(x, v):
        _, acc = O.forces_brute(p, x, v, s.tag, X0=s.X0, bonds=s.bonds, r0=s.r0, level_mask=O.LVL_PLT)
        return 0.5 * (v * v).sum() + acc["epot"]

    d = np.linalg.norm(s.x[:n_shell, None] - s.x[None, n_shell:], axis=-1)
    assert (d < 2.0).sum() > 10          # the LJ acts between the shells at the start
    x, f, n0 = s.x, None, 0
    es = [energy(x, v)]
    for block in range(10):
        x, v, f = O.run_respa(p, x, v, s.tag, X0=s.X0, bonds=s.bonds, r0=s.r0, dt_f=0.001, n_outer=1000,
                              forces=f, n0=n0)
        n0 += 1000
        es.append(energy(x, v))
    es = np.array(es)
    e = abs(es.mean())
    assert np.abs(es - es[0]).max() < 1e-4 * e
    assert abs(np.polyfit(np.arange(11), es, 1)[0] * 10) < 1e-4 * e


# --------------------------------------------------------------------------
# Sec. 3.3 -- AI-MTS: per-platelet step ratios
# --------------------------------------------------------------------------

def two_isolated_shells(n_shell=200, seed=17):
    """Two platelets 14 apart in a 30^3 box (beyond every platelet-level cutoff),
    no plasma: the levels do not couple them."""
    s = synth.platelet_system((30.0, 30.0, 30.0), 0, 2, n_shell, synth.scaled_radii(n_shell), seed=seed,
                              centers=[(8.0, 15.0, 15.0), (22.0, 15.0, 15.0)])
    rng = np.random.default_rng(seed)
    s.x += 0.03 * rng.standard_normal(s.x.shape)
    return s


def test_ai_mts_equal_ratios_is_fixed_k_respa():
    """Sec. 3.3: when the controller gives every platelet the same k, AI-MTS is
    Table 1's RESPA with k_p = k (plasma, walls and interface levels included)."""
    s = synth.platelet_system((8.0, 8.0, 8.0), 1200, 2, 120, synth.scaled_radii(120), walls=True,
                              body_force=0.02, seed=5, centers=[(2.7, 4.0, 4.0), (5.4, 4.0, 4.0)])
    p = O.system_params(s)
    xa, va, _ = O.run_respa(p, s.x, s.v, s.tag, X0=s.X0, bonds=s.bonds, r0=s.r0, dt_f=0.01, k_m=2, k_p=3,
                            n_outer=3)
    xb, vb, _ = O.run_ai_respa(p, s.x, s.v, s.tag, [3, 3], X0=s.X0, bonds=s.bonds, r0=s.r0, dt_f=0.01, k_m=2,
                               n_outer=3)
    assert np.abs(xa - xb).max() < 1e-11
    assert np.abs(va - vb).max() < 1e-9


def test_ai_mts_isolated_platelets_follow_their_own_ratio():
    """Sec. 3.3: each platelet moves with its own k.  Two platelets that share no
    force each follow the fixed-k RESPA trajectory of their own ratio."""
    s = two_isolated_shells()
    p = O.system_params(s)
    kw = dict(X0=s.X0, bonds=s.bonds, r0=s.r0, dt_f=0.004, k_m=2, n_outer=4)
    xa, va, _ = O.run_ai_respa(p, s.x, s.v, s.tag, [2, 5], **kw)
    p0 = s.tag == 0
    p1 = s.tag == 1
    for k, sel in ((2, p0), (5, p1)):
        xr, vr, _ = O.run_respa(p, s.x, s.v, s.tag, k_p=k, **kw)
        assert np.abs(xa[sel] - xr[sel]).max() < 1e-11
        assert np.abs(va[sel] - vr[sel]).max() < 1e-9
    # and the two ratios give visibly different trajectories
    x1, _, _ = O.run_respa(p, s.x, s.v, s.tag, k_p=1, **kw)
    assert np.abs(xa[p1] - x1[p1]).max() > 1e-9



def interacting_shells(n_shell=200, seed=17):
    """Two platelets 3 apart (closest particles about 1.5 apart): LJ and receptor
    Morse pairs between them."""
    s = two_isolated_shells(n_shell, seed)
    s.x[s.tag >= 0] = np.where((s.tag[s.tag >= 0] & ~synth.RECEPTOR_BIT)[:, None] == 1,
                               s.x[s.tag >= 0] - np.array([11.0, 0.0, 0.0]), s.x[s.tag >= 0])
    return s


def test_ai_mts_mixed_ratios_conserve_momentum():
    """Each cross-platelet pair is integrated on the finer grid for both of its
    ends, so its impulses cancel: with no plasma, walls or body force the total
    momentum is conserved exactly (rounding only) for any ratios."""
    s = interacting_shells()
    p = O.system_params(s)
    kw = dict(X0=s.X0, bonds=s.bonds, r0=s.r0, dt_f=0.004, k_m=2, n_outer=5)
    _, acc = O.forces_brute(p, s.x, s.v, s.tag, X0=s.X0, bonds=s.bonds, r0=s.r0, level_mask=O.LVL_PLT)
    x1, v1, _ = O.run_ai_respa(p, s.x, s.v, s.tag, [1, 5], **kw)
    assert np.abs(x1 - s.x).max() > 1e-3                # the shells did move
    pid = s.tag & ~synth.RECEPTOR_BIT
    a, b = s.x[pid == 0], s.x[pid == 1]                   # and they touch (LJ range 2.0)
    assert np.sqrt(((a[:, None, :] - b[None, :, :]) ** 2).sum(-1)).min() < 2.0
    scale = np.abs(v1 - s.v).sum()
    assert np.abs(v1.sum(0) - s.v.sum(0)).max() < 1e-12 * max(scale, 1.0)


def test_ai_mts_time_reversible_with_mixed_ratios():
    """The kick/drift pattern of every grid is symmetric within the interface
    step, so the mixed-ratio loop is time-reversible for conservative forces."""
    s = interacting_shells()
    p = O.system_params(s)
    v0 = 0.5 * s.v
    kw = dict(X0=s.X0, bonds=s.bonds, r0=s.r0, dt_f=0.004, k_m=1, n_outer=20)
    x1, v1, _ = O.run_ai_respa(p, s.x, v0, s.tag, [1, 2], **kw)
    x2, v2, _ = O.run_ai_respa(p, x1, -v1, s.tag, [1, 2], **kw)
    assert np.abs(x2 - s.x).max() < 1e-9
    assert np.abs(v2 + v0).max() < 1e-8


# --------------------------------------------------------------------------
# Eq. 2 -- angle term k_a (theta - theta0)^2
# --------------------------------------------------------------------------

def three_body(theta, r1=0.3, r2=0.25, box=(10.0, 10.0, 10.0), shift=(5.0, 5.0, 5.0)):
    """i at r1 along x from the vertex j, k at r2 in the xy plane at angle theta."""
    j = np.array(shift)
    x = np.array([j + [r1, 0.0, 0.0], j, j + [r2 * math.cos(theta), r2 * math.sin(theta), 0.0]])
    return x, np.zeros((3, 3)), np.zeros(3, np.int32)


@pytest.mark.parametrize("theta,theta0", [(2.6, 2.8), (2.9, 2.7), (1.4, 1.0)])
def test_angle_force_closed_form(theta, theta0):
    """Eq. 2 angle term as printed, U = k_a (theta - theta0)^2: the energy, and
    the force on each arm's end, 2 k_a |theta - theta0| / r perpendicular to
    its arm in the plane, turning the angle back toward theta0; the vertex
    takes the opposite of their sum."""
    k_a = 20.0
    x, v, tag = three_body(theta)
    p = O.make_params((10, 10, 10), k_a=k_a, angles=[[0, 1, 2]], theta0=[theta0])
    f, acc = O.forces_brute(p, x, v, tag, level_mask=O.LVL_PLT)
    assert acc["epot"] == pytest.approx(k_a * (theta - theta0) ** 2, rel=1e-12)
    mag = 2.0 * k_a * (theta - theta0)
    # on i (arm along +x): along +y when the angle must shrink (theta > theta0)
    assert f[0] == pytest.approx([0.0, mag / 0.3, 0.0], abs=1e-12)
    # on k (arm at angle theta): along the inward normal (sin t, -cos t) times the same sign
    assert f[2] == pytest.approx([mag / 0.25 * math.sin(theta), -mag / 0.25 * math.cos(theta), 0.0], abs=1e-12)
    assert f[1] == pytest.approx(-(f[0] + f[2]), abs=1e-12)


def test_angle_force_is_minus_gradient():
    """F = -grad U for triplets in general position, one of them across the
    periodic x face, by central differences of the oracle's energy."""
    rng = np.random.default_rng(12)
    x = rng.uniform(4.0, 6.0, (6, 3))
    x[3:] = x[:3] * 0.2 + np.array([9.85, 3.0, 3.0])       # a triplet straddling x = 10
    x[3, 0] = 0.1
    x %= 10.0
    tag = np.zeros(6, np.int32)
    p = O.make_params((10, 10, 10), k_a=20.0, angles=[[0, 1, 2], [3, 4, 5]], theta0=[2.5, 2.0])
    f, _ = O.forces_brute(p, x, np.zeros_like(x), tag, level_mask=O.LVL_PLT)
    h = 1e-6
    for a in range(6):
        for d in range(3):
            xp, xm = x.copy(), x.copy()
            xp[a, d] += h
            xm[a, d] -= h
            up = O.forces_brute(p, xp, np.zeros_like(x), tag, level_mask=O.LVL_PLT)[1]["epot"]
            um = O.forces_brute(p, xm, np.zeros_like(x), tag, level_mask=O.LVL_PLT)[1]["epot"]
            assert f[a, d] == pytest.approx(-(up - um) / (2 * h), rel=1e-6, abs=1e-6)


def test_angle_forces_conserve_momentum_and_angular_momentum():
    """The angle term depends on relative positions and on nothing that turns
    with the body: its forces sum to zero and exert no net torque."""
    rng = np.random.default_rng(13)
    x = 5.0 + rng.standard_normal((3, 3)) * 0.3
    p = O.make_params((10, 10, 10), k_a=20.0, angles=[[0, 1, 2]], theta0=[2.0])
    f, _ = O.forces_brute(p, x, np.zeros_like(x), np.zeros(3, np.int32), level_mask=O.LVL_PLT)
    assert np.abs(f.sum(0)).max() < 1e-12
    assert np.abs(np.cross(x - x.mean(0), f).sum(0)).max() < 1e-11


def test_shell_angles_bend_straight_through_vertices_and_rest_at_theta0():
    """The synthetic shells' angle triplets: both arms bonded to the vertex,
    each the straight continuation across it (rest angle above 150 degrees),
    every vertex in at least one triplet, reference angle the rest angle (so
    the undeformed shell feels no angle force); and a flat triangular sheet,
    where those triplets are straight, feels none either."""
    s = synth.platelet_system((20.0, 20.0, 20.0), 0, 1, 400, synth.scaled_radii(400), seed=3,
                              centers=[(10.0, 10.0, 10.0)])
    bonded = set(map(tuple, np.sort(s.bonds, 1).tolist()))
    for i, j, k in s.angles.tolist():
        assert tuple(sorted((i, j))) in bonded and tuple(sorted((j, k))) in bonded
    assert synth.triplet_angles(s.x, s.angles.astype(np.int64)).min() > np.radians(150.0)
    assert np.abs(s.theta0 - synth.triplet_angles(s.x, s.angles.astype(np.int64))).max() < 1e-6
    assert set(s.angles[:, 1].tolist()) == set(range(s.n))
    p = O.system_params(s, k_b=0.0)
    f, acc = O.forces_brute(p, s.x, s.v, s.tag, X0=s.X0, level_mask=O.LVL_PLT)
    assert np.abs(f).max() < 1e-3 and acc["epot"] < 1e-9     # theta0 rounded to binary32
    # a flat triangular patch (spacing 0.22) and its own bending triplets
    pts = np.array([[0.22 * (i + 0.5 * (j % 2)), 0.22 * math.sqrt(3) / 2 * j, 0.0]
                    for j in range(6) for i in range(6)]) + 5.0
    d = np.linalg.norm(pts[:, None] - pts[None], axis=-1)
    pairs = np.argwhere(np.triu(np.abs(d - 0.22) < 1e-9, 1))      # the lattice's nearest neighbours
    tri, th0 = synth.angle_triplets(pts, pairs)
    assert len(tri) > 20
    p = O.make_params((20, 20, 20), k_a=20.0, k_b=0.0, angles=tri, theta0=th0)
    f, acc = O.forces_brute(p, pts, np.zeros_like(pts), np.zeros(len(pts), np.int32), level_mask=O.LVL_PLT)
    assert np.abs(f).max() < 1e-9 and abs(acc["epot"]) < 1e-9      # theta0 = pi rounded to binary32


@pytest.mark.slow
def test_nve_energy_of_a_shell_with_bonds_and_angles_is_second_order():
    """CGMD in NVE: one bonded 200-particle shell with the Eq. 2 angle term on
    its bending triplets (k = 5, rest angles as reference), velocity-Verlet
    from Maxwell velocities at kT = 1 over 5 time units.  The printed form
    has a cone point at theta = pi, which the nearly straight triplets cross
    under thermal bending (the force direction turns over there), so the
    energy drifts; the drift is an integration error of second order: it
    falls about fourfold when dt is halved (0.001 -> 0.0005), and stays
    below 1e-3 of the energy at the smaller step."""
    s = synth.platelet_system((30.0, 30.0, 30.0), 0, 1, 200, synth.scaled_radii(200), seed=11,
                              centers=[(15.0, 15.0, 15.0)])
    p = O.system_params(s, m_rc=2.0)
    assert p.n_angles == len(s.angles) > 400 and p.k_a == 5.0

    def energy(x, v):
        _, acc = O.forces_brute(p, x, v, s.tag, X0=s.X0, bonds=s.bonds, r0=s.r0, level_mask=O.LVL_PLT)
        return 0.5 * (v * v).sum() + acc["epot"]

    drift = []
    for dt in (0.001, 0.0005):
        x, v, f, n0 = s.x, s.v, None, 0
        es = [energy(x, v)]
        steps = int(round(0.5 / dt))
        for block in range(10):
            x, v, f = O.run_respa(p, x, v, s.tag, X0=s.X0, bonds=s.bonds, r0=s.r0, dt_f=dt, n_outer=steps,
                                  forces=f, n0=n0)
            n0 += steps
            es.append(energy(x, v))
        es = np.array(es)
        drift.append(abs(np.polyfit(np.arange(11), es, 1)[0] * 10) / abs(es.mean()))
    assert drift[1] < drift[0] / 2.5
    assert drift[1] < 1e-3


def test_listed_pair_forces_add_up_to_the_all_pairs_sum():
    """The oracle's per-pair forces F_ij over every pair (both orders) sum to
    the all-pairs forces, and F_ji = -F_ij (Eq. 1 noise symmetric in i, j)."""
    s = small_platelet_system(seed=5)
    p = O.system_params(s, le_offset=0.7)
    n = s.n
    ii, jj = np.triu_indices(n, 1)
    pairs = np.stack([ii, jj], 1)
    F = O.pair_forces(p, s.x, s.v, s.tag, pairs, X0=s.X0, n_time=2)
    Fr = O.pair_forces(p, s.x, s.v, s.tag, pairs[:, ::-1], X0=s.X0, n_time=2)
    assert np.array_equal(F, -Fr)
    f = np.zeros((n, 3))
    np.add.at(f, ii, F)
    np.add.at(f, jj, -F)
    f[s.tag != synth.TAG_WALL, 0] += p.g
    # bonds and angles are not pairs of this kind: compare with them switched off
    p0 = O.system_params(s, le_offset=0.7, k_b=0.0, k_a=0.0)
    fb0, _ = O.forces_brute(p0, s.x, s.v, s.tag, X0=s.X0, n_time=2)
    assert np.abs(f - fb0).max() < 1e-10 * (np.abs(fb0).max() + 1)


def three_contact_shells(seed=8):
    """Three 120-particle platelets in plasma, close enough for LJ and Morse
    between neighbours, in a walled box."""
    s = synth.platelet_system((12.0, 8.0, 8.0), 2300, 3, 120, synth.scaled_radii(120), walls=True,
                              body_force=0.02, seed=seed, centers=[(2.8, 4.0, 4.0), (5.6, 4.0, 4.0), (8.4, 4.1, 4.0)])
    rng = np.random.default_rng(seed)
    plt = s.tag >= 0
    s.x[plt] += 0.03 * rng.standard_normal((int(plt.sum()), 3))
    return s


@pytest.mark.parametrize("levels,ratios", [([1, 2, 2], [1, 4]), ([1, 2, 3], [1, 2, 5]), ([3, 1, 2], [1, 2, 2])])
def test_table1_nested_sublevels_equal_the_ratio_grid(levels, ratios):
    """Table 1 as printed -- flowing platelets on level 1 (one step per
    interface substep), finer levels nested inside it, the innermost
    (aggregating) level drifting every particle -- performs the kicks and
    drifts of the per-platelet ratio grid (each platelet's k = dt_m / dt of
    its level, a term on the finer platelet's grid): the same trajectory to
    rounding, with interface substeps (k_m = 2), plasma, walls and the
    inter-platelet LJ and Morse terms between levels."""
    s = three_contact_shells()
    p = O.system_params(s)
    K = np.cumprod(ratios)
    plt_k = [int(K[l - 1]) for l in levels]
    kw = dict(X0=s.X0, bonds=s.bonds, r0=s.r0, dt_f=0.01, k_m=2, n_outer=3)
    xa, va = O.run_nested(p, s.x, s.v, s.tag, levels, ratios, **kw)
    xb, vb, _ = O.run_ai_respa(p, s.x, s.v, s.tag, plt_k, **kw)
    assert np.abs(xa - s.x).max() > 1e-3            # the particles moved
    assert np.abs(xa - xb).max() < 1e-11
    assert np.abs(va - vb).max() < 1e-9
