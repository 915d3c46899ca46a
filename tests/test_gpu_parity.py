"""GPU path (libmsm through the C ABI) against the FP64 oracle.

Tolerances:
 * neighbour sets: bit-exact (the oracle evaluates the same binary32 predicate);
 * per-step forces: |F_gpu - F_orc|_inf <= 1e-5 (|F_orc,i| + F_rms) per particle,
   the oracle fed the GPU's FP32 snapshot (positions, velocities, box, offset);
 * FP64 reductions: 1e-10 relative on identical inputs;
 * short trajectories: derived from FP32 force rounding (see each test).
"""
import numpy as np
import pytest

import oracle as O
import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5


def f32(a):
    return np.asarray(a, np.float32).astype(np.float64)


def make_gpu(s, step0=0, x=None, v=None, **kw):
    import paper_2205_14121_gb300 as M
    return M.System(s.box, s.x if x is None else x, s.v if v is None else v, s.tag, X0=s.X0, angles=s.angles, theta0=s.theta0, bonds=s.bonds,
                    r0=s.r0, walls=s.walls, wall=s.wall, shear_rate=s.shear_rate, body_force=s.body_force,
                    step0=step0, **kw)


def le_offset_f32(s, step, dt=0.01):
    if s.walls or not s.shear_rate:
        return 0.0
    return float(np.float32((s.shear_rate * s.box[1] * step * dt) % s.box[0]))


def oracle_forces(s, x32, v, step, level_mask=O.LVL_ALL, dt=0.01, dt_m=None, **kw):
    p = O.system_params(s, le_offset=le_offset_f32(s, step, dt), **kw)
    f, acc = O.forces_brute(p, f32(x32), f32(v), s.tag, X0=f32(s.X0), bonds=s.bonds, r0=f32(s.r0),
                            level_mask=level_mask, n_time=step, dt=dt, dt_m=dt_m)
    return f, acc


def assert_force_parity(f_gpu, f_orc, tol=TOL):
    mag = np.sqrt((f_orc ** 2).sum(1))
    frms = np.sqrt((mag ** 2).mean())
    err = np.abs(f_gpu - f_orc).max(1)
    bound = tol * (mag + frms)
    worst = np.argmax(err / bound)
    assert np.all(err <= bound), (f"particle {worst}: err {err[worst]:.3e} > {bound[worst]:.3e}; "
                                  f"F_orc {f_orc[worst]}, F_gpu {f_gpu[worst]}")


@pytest.fixture(scope="module")
def plt_sys():
    """12^3 Lees-Edwards box, 5,184 plasma + two 400-particle shells 4.0 apart
    (LJ and receptor pairs between them), shells jittered by 0.02 so that the
    bonds carry load."""
    s = synth.platelet_system((12.0, 12.0, 12.0), 5184, 2, 400, synth.scaled_radii(400), shear_rate=0.05,
                              seed=11, centers=[(4.0, 6.0, 6.0), (8.0, 6.0, 6.0)])
    rng = np.random.default_rng(21)
    plt = s.tag >= 0
    s.x[plt] += 0.02 * rng.standard_normal((plt.sum(), 3))
    return s


@pytest.fixture(scope="module")
def plt_wall_sys():
    """The two-shell system in a y-walled channel with a body force (Lees-Edwards
    images move a plasma particle that crosses y by the offset of the crossing
    time, which RESPA's once-per-substep fluid drift does not resolve; walls
    bounce exactly alike)."""
    s = synth.platelet_system((12.0, 12.0, 12.0), 5184, 2, 400, synth.scaled_radii(400), walls=True,
                              body_force=0.02, seed=13, centers=[(4.0, 6.0, 6.0), (8.0, 6.0, 6.0)])
    rng = np.random.default_rng(22)
    plt = s.tag >= 0
    s.x[plt] += 0.02 * rng.standard_normal((plt.sum(), 3))
    return s


@pytest.fixture(scope="module")
def wall_sys():
    return synth.plasma_box(box=(9.0, 8.0, 7.0), walls=True, body_force=0.02, seed=12)


@pytest.mark.parametrize("excl,skin_plt", [(2.5, None), (None, None), (None, 0.7)])
@pytest.mark.parametrize("kind", [0, 1, 2, 3])
def test_neighbor_sets_bit_exact(plt_sys, kind, excl, skin_plt):
    """Every list kind equals the oracle's brute-force FP32 pair set: with an LJ
    exclusion radius of 2.5 (far-at-rest pairs of one platelet kept), with the
    default (no same-platelet LJ; the bounding-sphere prefilter active), and
    with a platelet skin of 0.7 (interface reach rc + (0.3 + 0.7) / 2, LJ and
    Morse reaches cut-off + 0.7)."""
    s = plt_sys
    kw = {} if excl is None else {"lj_excl": excl}
    if skin_plt is not None:
        kw["skin_plt"] = skin_plt
    g = make_gpu(s, step0=17, **kw)
    g.neighbor_build(force=True)
    got = g.neighbor_pairs(kind)
    _, _, x32 = g.read_particles()
    sp = 0.3 if skin_plt is None else skin_plt
    cut = [1.3, 1.0 + 0.5 * (0.3 + sp), 2.0 + sp, 5.0 + sp][kind]
    excl2 = np.float32(np.inf) if excl is None else np.float32(excl * excl)
    ref = O.pairs_f32(x32, s.tag, np.array(s.box, np.float32), kind, np.float32(cut * cut),
                      X0f=s.X0.astype(np.float32), excl2=excl2, le=True,
                      delta=le_offset_f32(s, 17))
    gs = set(map(tuple, got.tolist()))
    rs = set(map(tuple, ref.tolist()))
    assert len(got) == len(gs), "duplicate pairs in the GPU list"
    assert gs == rs, (len(gs - rs), len(rs - gs))
    assert len(rs) > 0


def test_plasma_list_bit_exact_with_walls(wall_sys):
    """Plasma list in a walled box (no periodic y): bit-exact set equality."""
    s = wall_sys
    g = make_gpu(s, step0=3)
    g.neighbor_build(force=True)
    got = g.neighbor_pairs(0)
    _, _, x32 = g.read_particles()
    ref = O.pairs_f32(x32, s.tag, np.array(s.box, np.float32), 0, np.float32(1.3 * 1.3), walls=True)
    gs = set(map(tuple, got.tolist()))
    assert len(got) == len(gs)
    assert gs == set(map(tuple, ref.tolist()))


@pytest.mark.parametrize("box,walls", [((7.9, 9.1, 8.3), False), ((10.4, 6.0, 9.75), True)])
def test_plasma_list_bit_exact_uneven_cells(box, walls):
    """The plasma list without Lees-Edwards images: a fully periodic box with
    uneven cell counts per axis, and a walled box whose cells span the list
    reach with little to spare."""
    s = synth.plasma_box(box=box, walls=walls, body_force=0.02 if walls else 0.0, seed=14)
    g = make_gpu(s, step0=2)
    g.neighbor_build(force=True)
    got = g.neighbor_pairs(0)
    _, _, x32 = g.read_particles()
    ref = O.pairs_f32(x32, s.tag, np.array(s.box, np.float32), 0, np.float32(1.3 * 1.3), walls=walls)
    gs = set(map(tuple, got.tolist()))
    assert len(got) == len(gs)
    assert gs == set(map(tuple, ref.tolist()))
    assert len(gs) > 0


@pytest.mark.parametrize("kind", [0, 1])
def test_neighbor_sets_bit_exact_walls_platelets(plt_wall_sys, kind):
    """Plasma and interface lists of the walled two-shell channel: platelet
    particles have no plasma-list row and are no plasma-list partner."""
    s = plt_wall_sys
    g = make_gpu(s, step0=4)
    g.neighbor_build(force=True)
    got = g.neighbor_pairs(kind)
    _, _, x32 = g.read_particles()
    cut = [1.3, 1.3][kind]
    ref = O.pairs_f32(x32, s.tag, np.array(s.box, np.float32), kind, np.float32(cut * cut), walls=True)
    gs = set(map(tuple, got.tolist()))
    assert len(got) == len(gs)
    assert gs == set(map(tuple, ref.tolist()))
    assert len(gs) > 0


def test_forces_match_oracle_all_levels(plt_sys):
    s = plt_sys
    import paper_2205_14121_gb300 as M
    g = make_gpu(s, step0=5)
    _, _, x32 = g.read_particles()
    for mask in (M.MD_LEVEL_FLUID, M.MD_LEVEL_IFACE, M.MD_LEVEL_PLT, M.MD_LEVEL_ALL):
        g.forces(mask)
        fg = g.read_forces(mask)
        fo, _ = oracle_forces(s, x32, s.v, 5, level_mask=mask)
        assert_force_parity(fg, fo)


def test_force_variants_match_oracle(plt_sys):
    """The readings' selectable variants: Eq. 3 with the repulsive LJ as the
    interface's conservative term (MD_CFG_IFACE_LJ), and the Morse term of
    Eq. 2 given by the standard form's range a = 1.5 (MD_CFG_MORSE_STANDARD:
    the printed form with alpha = 2 a r0 = 3)."""
    import paper_2205_14121_gb300 as M
    from paper_2205_14121_gb300._binding import MD_CFG_IFACE_LJ, MD_CFG_MORSE_STANDARD
    s = plt_sys
    g = make_gpu(s, step0=5, flags=MD_CFG_IFACE_LJ | MD_CFG_MORSE_STANDARD, morse_alpha=1.5)
    _, _, x32 = g.read_particles()
    g.forces()
    fo_i, _ = oracle_forces(s, x32, s.v, 5, level_mask=O.LVL_IFACE, iface_lj=True)
    assert_force_parity(g.read_forces(M.MD_LEVEL_IFACE), fo_i)
    fo_p, _ = oracle_forces(s, x32, s.v, 5, level_mask=O.LVL_PLT, m_alpha=3.0)
    assert_force_parity(g.read_forces(M.MD_LEVEL_PLT), fo_p)
    # the variants change the forces: not the default's
    fd_i, _ = oracle_forces(s, x32, s.v, 5, level_mask=O.LVL_IFACE)
    assert np.abs(fd_i - fo_i).max() > 1.0


@pytest.mark.parametrize("det", [False, True])
def test_uniform_noise_variant_matches_oracle(plt_sys, det):
    """MD_CFG_UNIFORM_NOISE: zeta_ij of Eq. 1 and Eq. 3 as the unit-variance
    uniform variate; plasma and interface levels against the oracle's
    uniform_noise reading, in the ordinary and the deterministic modes."""
    import paper_2205_14121_gb300 as M
    from paper_2205_14121_gb300._binding import MD_CFG_UNIFORM_NOISE
    s = plt_sys
    g = make_gpu(s, step0=7, flags=MD_CFG_UNIFORM_NOISE)
    _, _, x32 = g.read_particles()
    g.forces(deterministic=det)
    for lvl, mask in ((O.LVL_FLUID, M.MD_LEVEL_FLUID), (O.LVL_IFACE, M.MD_LEVEL_IFACE)):
        fo, _ = oracle_forces(s, x32, s.v, 7, level_mask=lvl, uniform_noise=True)
        fg = g.read_forces(mask)
        assert_force_parity(fg, fo)
        # not the Gaussian draw
        fd, _ = oracle_forces(s, x32, s.v, 7, level_mask=lvl)
        assert np.abs(fd - fo).max() > 1.0


def test_forces_walls_body_force(wall_sys):
    s = wall_sys
    g = make_gpu(s, step0=2)
    g.forces()
    fg = g.read_forces()
    _, _, x32 = g.read_particles()
    fo, _ = oracle_forces(s, x32, s.v, 2)
    assert_force_parity(fg, fo)


def test_net_force_vanishes(plt_sys):
    """Pairwise antisymmetry (Eq. 1 noise keyed symmetrically): sum F ~ 0 up to
    FP32 accumulation."""
    g = make_gpu(plt_sys, step0=9)
    g.forces()
    f = g.read_forces()
    assert np.abs(f.sum(0)).max() < 1e-5 * np.abs(f).sum()


@pytest.mark.parametrize("which", ["le", "walls"])
def test_deterministic_forces(plt_sys, plt_wall_sys, which):
    """MD_FORCE_DETERMINISTIC: the forces of every level equal the oracle's,
    are bit-identical between two systems built from the same state (their
    particle orders differ: the cell sort places particles by atomics), and,
    without walls or body force, add up to exactly zero (every pair term
    cancels in 64-bit fixed point)."""
    s = plt_sys if which == "le" else plt_wall_sys
    g1 = make_gpu(s, step0=5)
    g2 = make_gpu(s, step0=5)
    _, _, x32 = g1.read_particles()
    g1.forces(deterministic=True)
    g2.forces(deterministic=True)
    f1, f2 = g1.read_forces(), g2.read_forces()
    assert np.array_equal(f1, f2)
    fo, _ = oracle_forces(s, x32, s.v, 5)
    assert_force_parity(f1, fo)
    if which == "le":
        assert np.all(f1.sum(0) == 0.0), f1.sum(0)
    # the default mode agrees to FP32 summation order
    g1.forces()
    assert_force_parity(g1.read_forces(), fo)


def test_virial_and_kinetics_match_oracle(plt_sys):
    s = plt_sys
    g = make_gpu(s, step0=4)
    g.forces(virial=True)
    o = g.observables()
    _, v, x32 = g.read_particles()
    _, acc = oracle_forces(s, x32, v, 4)
    p = O.system_params(s, le_offset=le_offset_f32(s, 4))
    kin = O.kinetics(p, s.x, v, s.tag)
    assert np.allclose(o["momentum"], kin["momentum"], rtol=0, atol=1e-9 * np.abs(v).sum())
    assert o["kinetic"] == pytest.approx(kin["ke"], rel=1e-10)
    assert np.allclose(o["virial_c"], acc["vir_c"], rtol=1e-4, atol=1e-4 * np.abs(acc["vir_c"]).max())
    assert o["temperature"] == pytest.approx(kin["T"], rel=1e-10)
    assert np.allclose(o["kin_tensor"], kin["K"], rtol=1e-10, atol=1e-10 * np.abs(kin["K"]).max())


def test_wall_temperature_subtracts_local_flow(plt_wall_sys):
    """With walls the peculiar velocity is relative to the 20-slab mean v_x of
    the mobile particles (Sec. 4.2): a parabolic stream of amplitude 0.5 laid on
    the thermal velocities leaves the temperature near its thermal value, and
    the GPU's FP64 sums equal the oracle's on the GPU's own state."""
    s = plt_wall_sys
    Ly = s.box[1]
    v0 = f32(s.v)
    y = s.x[:, 1]
    mob = s.tag != synth.TAG_WALL
    v0[mob, 0] += (2.0 * y[mob] * (Ly - y[mob]) / Ly ** 2).astype(np.float32)
    g = make_gpu(s, x=f32(s.x), v=v0)
    g.mts_step(2)
    o = g.observables()
    x, v, _ = g.read_particles()
    kin = O.kinetics(O.system_params(s), x, v, s.tag, nbins=20)
    assert o["temperature"] == pytest.approx(kin["T"], rel=1e-10)
    assert np.allclose(o["kin_tensor"], kin["K"], rtol=1e-10, atol=1e-10 * np.abs(kin["K"]).max())
    assert o["kinetic"] == pytest.approx(kin["ke"], rel=1e-10)
    assert abs(kin["T"] - 1.0) < 0.1
    # the stream itself is not temperature: without the subtraction the sum
    # would exceed 3 N_mobile T by the stream's kinetic energy
    stream = 2.0 * kin["ke"] - np.trace(kin["K"])
    assert stream > 0.01 * mob.sum()


@pytest.mark.parametrize("which", ["walls", "le"])
def test_fast_particles_keep_the_lists_and_every_pair(plt_wall_sys, plt_sys, which):
    """Plasma that moved beyond skin/2 but within the skin keeps the lists:
    40 plasma particles next to the shells are launched at speed 7 toward
    their platelet's centre; after three STS steps they are 0.15-0.3 from their
    build positions, no rebuild has run, and the forces of every level equal
    the oracle's brute-force forces on the GPU's state -- the pairs the lists
    lack (plasma and interface) come from the fast-particle pass.  With walls
    and with Lees-Edwards images (whose offset moves between the build and
    the check)."""
    import paper_2205_14121_gb300 as M
    s = plt_wall_sys if which == "walls" else plt_sys
    x0, v0 = f32(s.x), f32(s.v)
    plt = np.flatnonzero(s.tag >= 0)
    plasma = np.flatnonzero(s.tag == synth.TAG_FLUID)
    rng = np.random.default_rng(31)
    d = np.sqrt(((x0[plasma, None, :] - x0[None, plt[::7], :]) ** 2).sum(-1)).min(1)
    near = plasma[(d > 1.2) & (d < 2.0)]
    pick = rng.choice(near, 40, replace=False)
    for k in pick:
        p = s.tag[plt[np.argmin(((x0[plt] - x0[k]) ** 2).sum(1))]] & ~(1 << 30)
        c = x0[s.tag == p].mean(0) if (s.tag == p).any() else x0[plt].mean(0)
        u = c - x0[k]
        v0[k] = 7.0 * u / np.linalg.norm(u)
    g = make_gpu(s, x=x0, v=v0, step0=3)
    g.mts_step(3)
    o = g.observables()
    x, v, x32 = g.read_particles()
    dx = x - x0
    L = np.array(s.box)
    if which == "le":       # an image across y carries the offset in x
        cross = np.round(dx[:, 1] / L[1])
        dx[:, 1] -= L[1] * cross
        dx[:, 0] -= cross * (s.shear_rate * L[1] * 0.01 * 6)   # the offset at the end, within 0.02 of the crossing's
    for ax in (0, 2):
        dx[:, ax] -= L[ax] * np.round(dx[:, ax] / L[ax])
    moved = np.sqrt((dx ** 2).sum(1))
    assert o["n_builds"] == 1, "a rebuild ran: the fast particles did not stay within the skin"
    assert 10 <= (moved[pick] > 0.15).sum() and moved.max() < 0.3, np.sort(moved)[-5:]
    g.forces()
    fg = g.read_forces()
    fo, _ = oracle_forces(s, x32, v, 6)
    assert_force_parity(fg, fo)
    if which == "le":
        assert le_offset_f32(s, 6) != le_offset_f32(s, 3)
    for lvl in (M.MD_LEVEL_FLUID, M.MD_LEVEL_IFACE):
        assert_force_parity(g.read_forces(lvl), oracle_forces(s, x32, v, 6, level_mask=lvl)[0])


def test_sts_trajectory_tracks_oracle(plt_sys):
    """Five velocity-Verlet steps from identical FP32-exact states: positions
    agree to 1e-4 (FP32 force rounding ~1e-5 F times dt^2 growth) and
    velocities to 5e-3 of their rms."""
    s = plt_sys
    x0, v0 = f32(s.x), f32(s.v)
    g = make_gpu(s, step0=0, x=x0, v=v0)
    g.mts_step(5)
    xg, vg, _ = g.read_particles()
    p = O.system_params(s)
    xo, vo, _ = O.run_sts(p, x0, v0, s.tag, X0=f32(s.X0), bonds=s.bonds, r0=f32(s.r0), dt=0.01, n_steps=5)
    dx = xg - xo
    L = np.array(s.box)
    dx -= L * np.round(dx / L)
    assert np.abs(dx).max() < 1e-4
    assert np.abs(vg - vo).max() < 5e-3 * np.sqrt((vo ** 2).mean())


def test_respa_k1_is_sts_without_platelets(wall_sys):
    """With only the fluid level populated, Table 1 with k_m = k_p = 1 is plain
    velocity-Verlet: the two GPU schedules agree to FP32 atomic-order noise."""
    import paper_2205_14121_gb300 as M
    s = wall_sys
    x0, v0 = f32(s.x), f32(s.v)
    a = make_gpu(s, x=x0, v=v0)
    a.mts_step(3)
    b = make_gpu(s, x=x0, v=v0)
    b.mts_step(3, mode=M.MD_MODE_RESPA, k_m=1, k_p=1)
    xa, va, _ = a.read_particles()
    xb, vb, _ = b.read_particles()
    assert np.abs(xa - xb).max() < 1e-6
    assert np.abs(va - vb).max() < 1e-4


def test_respa_platelet_substeps_track_oracle(plt_wall_sys):
    """Fixed-k RESPA (k_m = 2, k_p = 4) against the oracle's Table 1 loop."""
    import paper_2205_14121_gb300 as M
    s = plt_wall_sys
    x0, v0 = f32(s.x), f32(s.v)
    g = make_gpu(s, x=x0, v=v0)
    g.mts_step(3, mode=M.MD_MODE_RESPA, k_m=2, k_p=4)
    xg, vg, _ = g.read_particles()
    p = O.system_params(s)
    xo, vo, _ = O.run_respa(p, x0, v0, s.tag, X0=f32(s.X0), bonds=s.bonds, r0=f32(s.r0), dt_f=0.01, k_m=2,
                            k_p=4, n_outer=3)
    dx = xg - xo
    L = np.array(s.box)
    dx -= L * np.round(dx / L)
    assert np.abs(dx).max() < 1e-4
    assert np.abs(vg - vo).max() < 5e-3 * np.sqrt((vo ** 2).mean())


@pytest.mark.parametrize("mode,k_m,k_p", [(0, 1, 1), (1, 2, 3)])
def test_graph_replay_matches_direct_launches(plt_wall_sys, mode, k_m, k_p):
    """The captured WHILE/IF graph performs the same steps, list rebuilds
    included, as launching every kernel from the host."""
    s = plt_wall_sys
    x0, v0 = f32(s.x), f32(s.v)
    a = make_gpu(s, x=x0, v=v0)
    a.mts_step(25, mode=mode, k_m=k_m, k_p=k_p)
    b = make_gpu(s, x=x0, v=v0)
    b.mts_step(25, mode=mode, k_m=k_m, k_p=k_p, direct=True)
    oa, ob = a.observables(), b.observables()
    assert oa["n_builds"] == ob["n_builds"] and oa["n_builds"] >= 2
    assert oa["step"] == ob["step"] == 25
    xa, va, _ = a.read_particles()
    xb, vb, _ = b.read_particles()
    dx = xa - xb
    dx -= np.array(s.box) * np.round(dx / np.array(s.box))
    assert np.abs(dx).max() < 1e-3   # chaotic growth of FP32 atomic-order noise over 25 steps


def test_ai_mts_mixed_ratios_track_oracle(plt_wall_sys):
    """AI-MTS (Sec. 3.3) with per-platelet ratios k = (2, 5) on the fine grid
    K = 10 against the oracle's per-platelet loop; same bound as fixed-k RESPA."""
    import paper_2205_14121_gb300 as M
    s = plt_wall_sys
    x0, v0 = f32(s.x), f32(s.v)
    g = make_gpu(s, x=x0, v=v0)
    g.set_platelet_levels([2, 5])
    g.mts_step(3, mode=M.MD_MODE_AI, k_m=2)
    xg, vg, _ = g.read_particles()
    p = O.system_params(s)
    xo, vo, _ = O.run_ai_respa(p, x0, v0, s.tag, [2, 5], X0=f32(s.X0), bonds=s.bonds, r0=f32(s.r0), dt_f=0.01,
                               k_m=2, n_outer=3)
    dx = xg - xo
    L = np.array(s.box)
    dx -= L * np.round(dx / L)
    assert np.abs(dx).max() < 1e-4
    assert np.abs(vg - vo).max() < 5e-3 * np.sqrt((vo ** 2).mean())
    # the two platelets really moved on different grids: k = (5, 2) differs
    h = make_gpu(s, x=x0, v=v0)
    h.set_platelet_levels([5, 2])
    h.mts_step(3, mode=M.MD_MODE_AI, k_m=2)
    xh, _, _ = h.read_particles()
    plt = s.tag >= 0
    d2 = xh[plt] - xg[plt]
    d2 -= L * np.round(d2 / L)
    assert np.abs(d2).max() > 1e-6


def test_ai_mts_platelets_apart_drift_on_their_own_grids():
    """Two platelets with no LJ or receptor pair between them (7.7 apart at
    their closest, beyond every platelet list reach) and ratios k = (2, 5):
    on the K = 10 grid each moves only at its own grid points (drift strides
    5 and 2), and the trajectory matches the oracle's, which drifts every
    platelet particle at every substep."""
    import paper_2205_14121_gb300 as M
    s = synth.platelet_system((16.0, 16.0, 16.0), 12288, 2, 400, synth.scaled_radii(400), walls=True,
                              body_force=0.02, seed=17, centers=[(4.0, 8.0, 4.0), (12.0, 8.0, 12.0)])
    x0, v0 = f32(s.x), f32(s.v)
    g = make_gpu(s, x=x0, v=v0)
    g.set_platelet_levels([2, 5])
    g.mts_step(3, mode=M.MD_MODE_AI, k_m=2)
    assert g.neighbor_count(M.MD_LIST_LJ) == 0 and g.neighbor_count(M.MD_LIST_MORSE) == 0
    xg, vg, _ = g.read_particles()
    p = O.system_params(s)
    xo, vo, _ = O.run_ai_respa(p, x0, v0, s.tag, [2, 5], X0=f32(s.X0), bonds=s.bonds, r0=f32(s.r0), dt_f=0.01,
                               k_m=2, n_outer=3)
    dx = xg - xo
    L = np.array(s.box)
    dx -= L * np.round(dx / L)
    assert np.abs(dx).max() < 1e-4
    assert np.abs(vg - vo).max() < 5e-3 * np.sqrt((vo ** 2).mean())


def test_ai_mts_contact_pair_skips_rows_between_its_stride_points():
    """Three platelets, k = (1, 2, 5) on the K = 10 grid: the first two touch
    (LJ and receptor pairs between them) and share the drift stride
    10 / lcm(1, 2) = 5, so their LJ and Morse rows are not read at the
    substeps in between, where none of their terms is due; the third lies
    apart (stride 2).  The trajectory matches the oracle's, which evaluates
    every pair at every substep and scales it by whether it is due."""
    import paper_2205_14121_gb300 as M
    s = synth.platelet_system((16.0, 16.0, 16.0), 12288, 3, 400, synth.scaled_radii(400), walls=True,
                              body_force=0.02, seed=19, centers=[(4.0, 8.0, 4.0), (8.0, 8.0, 4.0), (12.0, 8.0, 12.0)])
    x0, v0 = f32(s.x), f32(s.v)
    g = make_gpu(s, x=x0, v=v0)
    g.set_platelet_levels([1, 2, 5])
    g.mts_step(3, mode=M.MD_MODE_AI, k_m=2)
    assert g.neighbor_count(M.MD_LIST_LJ) > 0 and g.neighbor_count(M.MD_LIST_MORSE) > 0
    xg, vg, _ = g.read_particles()
    p = O.system_params(s)
    xo, vo, _ = O.run_ai_respa(p, x0, v0, s.tag, [1, 2, 5], X0=f32(s.X0), bonds=s.bonds, r0=f32(s.r0), dt_f=0.01,
                               k_m=2, n_outer=3)
    dx = xg - xo
    L = np.array(s.box)
    dx -= L * np.round(dx / L)
    assert np.abs(dx).max() < 1e-4
    assert np.abs(vg - vo).max() < 5e-3 * np.sqrt((vo ** 2).mean())


def test_ai_mts_tracks_table1_nested_sublevels(plt_wall_sys):
    """Table 1's nested sublevels as printed (oracle: a flowing platelet on
    level 1, one step per interface substep; an aggregating one on level 2,
    five steps inside each; the inner level drifting every particle) against
    the device's per-platelet ratio grid with k = (1, 5): the same
    trajectory within the fixed-k RESPA bound."""
    import paper_2205_14121_gb300 as M
    s = plt_wall_sys
    x0, v0 = f32(s.x), f32(s.v)
    g = make_gpu(s, x=x0, v=v0)
    g.set_platelet_levels([1, 5])
    g.mts_step(3, mode=M.MD_MODE_AI, k_m=2)
    xg, vg, _ = g.read_particles()
    p = O.system_params(s)
    xo, vo = O.run_nested(p, x0, v0, s.tag, [1, 2], [1, 5], X0=f32(s.X0), bonds=s.bonds, r0=f32(s.r0), dt_f=0.01,
                          k_m=2, n_outer=3)
    dx = xg - xo
    L = np.array(s.box)
    dx -= L * np.round(dx / L)
    assert np.abs(dx).max() < 1e-4
    assert np.abs(vg - vo).max() < 5e-3 * np.sqrt((vo ** 2).mean())


def test_ai_mts_equal_ratios_match_respa_on_gpu(plt_wall_sys):
    """With every k_p = 4 the AI-MTS kernels take the fixed-k RESPA steps."""
    import paper_2205_14121_gb300 as M
    s = plt_wall_sys
    x0, v0 = f32(s.x), f32(s.v)
    a = make_gpu(s, x=x0, v=v0)
    a.set_platelet_levels([4, 4])
    a.mts_step(4, mode=M.MD_MODE_AI, k_m=2)
    b = make_gpu(s, x=x0, v=v0)
    b.mts_step(4, mode=M.MD_MODE_RESPA, k_m=2, k_p=4)
    xa, va, _ = a.read_particles()
    xb, vb, _ = b.read_particles()
    dx = xa - xb
    dx -= np.array(s.box) * np.round(dx / np.array(s.box))
    assert np.abs(dx).max() < 1e-4
    assert np.abs(va - vb).max() < 1e-2


def test_ai_mts_graph_replay_and_level_validation(plt_wall_sys):
    """Graph replay of the AI-MTS step equals direct launches; a new ratio set
    with another lcm recaptures; bad ratios are rejected."""
    import paper_2205_14121_gb300 as M
    s = plt_wall_sys
    x0, v0 = f32(s.x), f32(s.v)
    a = make_gpu(s, x=x0, v=v0)
    with pytest.raises(M.MdError):
        a.mts_step(2, mode=M.MD_MODE_AI)          # no ratios yet
    for bad in ([0, 1], [1, 65], [7, 11]):
        with pytest.raises(M.MdError):
            a.set_platelet_levels(bad)
    b = make_gpu(s, x=x0, v=v0)
    for g in (a, b):
        g.set_platelet_levels([1, 2])
    a.mts_step(10, mode=M.MD_MODE_AI, k_m=1)
    b.mts_step(10, mode=M.MD_MODE_AI, k_m=1, direct=True)
    for g in (a, b):
        g.set_platelet_levels([10, 20])
    a.mts_step(10, mode=M.MD_MODE_AI, k_m=1)
    b.mts_step(10, mode=M.MD_MODE_AI, k_m=1, direct=True)
    oa, ob = a.observables(), b.observables()
    assert oa["step"] == ob["step"] == 20 and oa["n_builds"] == ob["n_builds"]
    xa, _, _ = a.read_particles()
    xb, _, _ = b.read_particles()
    dx = xa - xb
    dx -= np.array(s.box) * np.round(dx / np.array(s.box))
    assert np.abs(dx).max() < 1e-3


@pytest.mark.parametrize("which", ["le", "walls"])
def test_platelet_features_match_oracle(plt_sys, plt_wall_sys, which):
    """K8 per-platelet measurements (FP64 device reductions) against the oracle on
    the GPU's own FP32 snapshot and forces."""
    from oracle import features as OF
    s = plt_sys if which == "le" else plt_wall_sys
    g = make_gpu(s, step0=2)
    g.mts_step(3)
    feat = g.platelet_features()
    _, v, x32 = g.read_particles()
    f = g.read_forces()
    ref = OF.platelet_features(f32(x32), f32(v), f, s.tag, s.bonds, f32(s.r0), np.array(s.box, np.float32),
                               walls=s.walls)
    assert feat.shape == ref.shape == (2, 12)
    cols = [0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 11]
    scale = np.abs(ref[:, cols]).max(0) + 1e-12
    assert np.all(np.abs(feat[:, cols] - ref[:, cols]) <= 1e-6 * scale + 1e-9), (feat, ref)
    assert np.all(np.abs(feat[:, 10] - ref[:, 10]) <= 1)   # pairs on the 1.5 r0 boundary may flip (FP32 test)
    # ring buffer: chronological records
    g.record_features()
    g.mts_step(1)
    g.record_features()
    ring, cnt = g.read_feature_ring()
    assert cnt == 2 and ring.shape == (2, 2, 12)
    assert np.allclose(ring[:, 0], feat.astype(np.float32))


@pytest.mark.parametrize("mode", ["respa", "ai"])
def test_step_graph_records_features_every_step(plt_wall_sys, mode):
    """MD_SCHED_RECORD appends the measurements of every outer step from inside
    the (replayed) step graph: the records equal those of one-step calls
    followed by md_record_features; in AI-MTS they use plain platelet forces."""
    import paper_2205_14121_gb300 as M
    s = plt_wall_sys
    x0, v0 = f32(s.x), f32(s.v)
    kw = dict(mode=M.MD_MODE_RESPA, k_m=1, k_p=2) if mode == "respa" else dict(mode=M.MD_MODE_AI, k_m=1)
    a = make_gpu(s, x=x0, v=v0)
    b = make_gpu(s, x=x0, v=v0)
    if mode == "ai":
        a.set_platelet_levels([2, 2])
        b.set_platelet_levels([2, 2])
    a.mts_step(6, record=True, **kw)
    for _ in range(6):
        b.mts_step(1, **kw)
        b.record_features()
    ra, ca = a.read_feature_ring()
    rb, cb = b.read_feature_ring()
    assert ca == cb == 6 and ra.shape == (2, 6, 12)
    scale = np.abs(rb).max(axis=(0, 1)) + 1e-9
    assert np.all(np.abs(ra - rb) <= 2e-3 * scale + 1e-6), np.abs(ra - rb).max(axis=(0, 1)) / scale
    if mode == "ai":   # the same step under fixed-k RESPA records the same measurements
        c = make_gpu(s, x=x0, v=v0)
        c.mts_step(6, record=True, mode=M.MD_MODE_RESPA, k_m=1, k_p=2)
        rc_, _ = c.read_feature_ring()
        assert np.all(np.abs(ra - rc_) <= 2e-3 * scale + 1e-6)


@pytest.mark.parametrize("which", ["walls", "le"])
def test_flow_profile_matches_oracle(wall_sys, plt_sys, which):
    """Sec. 4.2 flow profile (FP64 device sums) against the oracle on the GPU's
    own state."""
    from oracle import features as OF
    s = wall_sys if which == "walls" else plt_sys
    g = make_gpu(s)
    g.mts_step(5)
    mean, dens = g.flow_profile(20)
    x, v, _ = g.read_particles()
    ref_mean, ref_dens = OF.flow_profile(x, v, s.tag, s.box, 20)
    assert np.allclose(mean, ref_mean, rtol=1e-12, atol=1e-13)
    assert np.allclose(dens, ref_dens, rtol=1e-12)
    assert abs(dens.mean() - 3.0) < 0.5


@pytest.mark.parametrize("shift,pinned", [(0.0, False), (1.7, False), (0.0, True)])
def test_set_xv_equals_full_upload(plt_wall_sys, shift, pinned):
    """md_set_xv (positions and velocities only, tags and rest positions kept
    on the device) leaves the same state as md_set_particles with the same
    tags: two RESPA steps from it agree to FP32 atomic-order noise (a wrong
    tag, rest position or stale list would move particles by orders more).
    Near the state of the last build (shift 0) it keeps the lists and the
    cell order; the whole system moved by 1.7 along x trips the rebuild check.
    From page-locked host arrays the two uploads take a side stream."""
    import paper_2205_14121_gb300 as M
    s = plt_wall_sys
    rng = np.random.default_rng(5)
    mob = (s.tag != synth.TAG_WALL)[:, None]
    x1 = s.x + 0.01 * rng.standard_normal(s.x.shape) * mob
    x1[:, 0] = (x1[:, 0] + shift) % s.box[0]
    x1 = f32(x1)
    v1 = f32(s.v * 0.9)
    a = make_gpu(s, x=x1, v=v1, step0=7)
    b = make_gpu(s, step0=0)
    b.mts_step(1)
    builds = b.observables()["n_builds"]
    if pinned:
        import torch
        b.set_xv(torch.from_numpy(np.ascontiguousarray(x1, np.float64)).pin_memory().numpy(),
                 torch.from_numpy(np.ascontiguousarray(v1, np.float64)).pin_memory().numpy(), step0=7)
    else:
        b.set_xv(x1, v1, step0=7)
    for g in (a, b):
        g.mts_step(2, mode=M.MD_MODE_RESPA, k_m=1, k_p=5)
    xa, va, _ = a.read_particles()
    xb, vb, _ = b.read_particles()
    assert np.abs(xa - xb).max() < 1e-5
    assert np.abs(va - vb).max() < 1e-3 * np.sqrt((va ** 2).mean())
    assert a.observables()["step"] == b.observables()["step"] == 9
    if shift == 0.0:
        assert b.observables()["n_builds"] == builds, "a rebuild ran on a state within the skin"


def test_checkpoint_roundtrip(plt_sys):
    s = plt_sys
    g = make_gpu(s)
    g.mts_step(2)
    blob = g.get_state()
    x1, v1, _ = g.read_particles()
    h = make_gpu(s)
    h.set_state(blob)
    x2, v2, _ = h.read_particles()
    assert np.array_equal(x1, x2) and np.array_equal(v1, v2)
    g.mts_step(2)
    h.mts_step(2)
    xa, _, _ = g.read_particles()
    xb, _, _ = h.read_particles()
    assert np.abs(xa - xb).max() < 1e-5


def test_full_size_dpd_throughput_system_sampled():
    """The 1,000,000-particle walled plasma system in the benchmark's launch
    configuration: forces of 3,000 sampled particles against the oracle."""
    s = synth.config_dpd_throughput()
    g = make_gpu(s, step0=1)
    g.forces()
    fg = g.read_forces()
    _, _, x32 = g.read_particles()
    rng = np.random.default_rng(1)
    sample = rng.choice(s.n, 3000, replace=False).astype(np.int32)
    p = O.system_params(s)
    fo = O.forces_cells(p, f32(x32), f32(s.v), s.tag, n_time=1, dt=0.01, sample=sample)
    mag = np.sqrt((fo ** 2).sum(1))
    frms = np.sqrt((mag ** 2).mean())
    err = np.abs(fg[sample] - fo).max(1)
    assert np.all(err <= TOL * (mag + frms))


def test_full_size_channel_sampled():
    """The 8,330,178-particle platelet channel in the benchmark's launch
    configuration (plasma skin 0.3, platelet skin 0.5): forces of every level
    on 2,000 sampled plasma and 1,000 sampled platelet particles against the
    oracle.  The shells are jittered by 0.02 so that their bonds carry load
    (at rest length a bond force is pure FP32 cancellation)."""
    import paper_2205_14121_gb300 as M
    s = synth.config_channel_platelets(seed=20220528)
    rng = np.random.default_rng(2)
    x = s.x.copy()
    plt = s.tag >= 0
    x[plt] += rng.normal(0.0, 0.02, size=(int(plt.sum()), 3))
    g = make_gpu(s, step0=3, x=x, skin=0.3, skin_plt=0.5)
    g.forces()
    _, _, x32 = g.read_particles()
    sample = np.concatenate([rng.choice(np.flatnonzero(s.tag == -1), 2000, replace=False),
                             rng.choice(np.flatnonzero(s.tag >= 0), 1000, replace=False)]).astype(np.int32)
    p = O.system_params(s)
    for lvl, mask in ((O.LVL_FLUID, M.MD_LEVEL_FLUID), (O.LVL_IFACE, M.MD_LEVEL_IFACE),
                      (O.LVL_PLT, M.MD_LEVEL_PLT)):
        fo = O.forces_cells(p, f32(x32), f32(s.v), s.tag, X0=f32(s.X0), bonds=s.bonds, r0=f32(s.r0),
                            level_mask=lvl, n_time=3, dt=0.01, sample=sample)
        fg = g.read_forces(mask)[sample]
        assert np.abs(fo).max() > 0.0
        assert_force_parity(fg, fo)
    g.close()


def test_philox_matches_curand_and_oracle():
    """The device Philox4x32-10 equals cuRAND's Philox4_32_10 (a library
    implementation of the same SC'11 generator) block for block, and the
    oracle's CPU implementation bit for bit."""
    from paper_2205_14121_gb300._binding import md_philox
    rng = np.random.default_rng(3)
    ctr = rng.integers(0, 2 ** 32, size=(4096, 4), dtype=np.uint64).astype(np.uint32)
    ctr[:, 1] &= (1 << 30) - 1      # keep 4*counter inside cuRAND's 64-bit offset
    ctr[:8] = 0
    ctr[8:16, 0] = np.arange(8)
    key = np.array([20220528, 0], np.uint32)
    own = md_philox(ctr, key)
    lib = md_philox(ctr, key, use_library=True)
    assert np.array_equal(own, lib)
    orc = np.array([O.philox4x32_10(c, key) for c in ctr[:512]], dtype=np.uint32)
    assert np.array_equal(own[:512], orc)
