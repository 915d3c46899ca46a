"""Failure paths of the C ABI, each made on the host: a list capacity too
small, a non-finite state handed in, an inconsistent configuration, and a
checkpoint resumed into a fresh system.  None of them faults or stalls the
device -- the library turns each into a status code and stays usable -- and
the resumed run is compared bit for bit with an uninterrupted one in the
deterministic step mode."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def small_shells(seed=51):
    import synth
    return synth.platelet_system((14.0, 12.0, 12.0), 3 * 14 * 12 * 12, 2, 300, synth.scaled_radii(300), walls=True,
                                 body_force=0.01, seed=seed, centers=[(4.0, 6.0, 6.0), (10.0, 6.0, 6.0)])


def make(s, **kw):
    import paper_2205_14121_gb300 as M
    return M.System(s.box, s.x, s.v, s.tag, X0=s.X0, bonds=s.bonds, r0=s.r0, angles=s.angles,
                    theta0=s.theta0, walls=s.walls, wall=s.wall,
                    body_force=s.body_force, **kw)


def test_list_overflow_reported_then_retry_at_default_capacity():
    """A plasma list capacity of 4 (rows hold about 13 entries) makes the build
    return MD_ENBR_OVERFLOW (-4) instead of writing past the rows; the same
    system at the default capacity builds, steps and reports its longest row."""
    import paper_2205_14121_gb300 as M
    s = small_shells()
    g = make(s, caps={"fluid": 4})
    with pytest.raises(M.MdError) as e:
        g.neighbor_build(force=True)
    assert e.value.code == -4
    with pytest.raises(M.MdError) as e:          # a later call reports it again, nothing was stepped
        g.mts_step(1)
    assert e.value.code == -4
    g.close()
    h = make(s)
    h.mts_step(5, mode=M.MD_MODE_RESPA, k_p=2)
    obs = h.observables()
    assert np.isfinite(obs["temperature"]) and 4 < obs["max_rows"][0] <= 96
    h.close()


def test_non_finite_velocity_is_unstable():
    """A NaN written into the host velocity array of md_set_xv: the placed
    state fails the check of the kick-drift and the call returns
    MD_EUNSTABLE (-5); loading a finite state afterwards steps again."""
    import paper_2205_14121_gb300 as M
    s = small_shells()
    g = make(s)
    g.mts_step(3)                                  # lists built: md_set_xv checks the placed state
    x, v, _ = g.read_particles()
    bad = v.copy()
    bad[17, 1] = np.nan
    with pytest.raises(M.MdError) as e:
        g.set_xv(x, bad)
    assert e.value.code == -5
    g.set_xv(x, v)
    g.mts_step(2)
    assert np.isfinite(g.observables()["temperature"])
    g.close()


def test_non_finite_velocity_before_the_first_build_stops_the_step():
    """The same NaN loaded before any list exists (md_set_particles): the first
    step's integrator raises the unstable flag and md_mts_step returns
    MD_EUNSTABLE."""
    import paper_2205_14121_gb300 as M
    s = small_shells()
    v = s.v.copy()
    v[5, 0] = np.inf
    g = make(s)
    g.set_particles(s.x, v, s.tag, s.X0)
    with pytest.raises(M.MdError) as e:
        g.mts_step(1)
    assert e.value.code == -5
    g.close()


@pytest.mark.parametrize("bad", ["dt", "walls_and_le", "receptors", "tag"])
def test_corrupt_configuration_is_rejected(bad):
    """Inconsistent configurations return MD_EINVAL (-1) from md_init or
    md_set_particles: a negative step, walls together with Lees-Edwards
    images, more receptors than platelet particles, a tag below -2."""
    import paper_2205_14121_gb300 as M
    s = small_shells()
    with pytest.raises(M.MdError) as e:
        if bad == "dt":
            make(s, dt=-0.01)
        elif bad == "walls_and_le":
            M.System(s.box, s.x, s.v, s.tag, X0=s.X0, bonds=s.bonds, r0=s.r0, angles=s.angles,
                     theta0=s.theta0, walls=True, wall=s.wall, flags=M.MD_CFG_LEES_EDWARDS)
        elif bad == "receptors":
            tag = s.tag.copy()
            tag[tag >= 0] |= 1 << 30             # every platelet particle a receptor: the counts no longer match
            g = make(s)
            g.set_particles(s.x, s.v, tag, s.X0)
        else:
            tag = s.tag.copy()
            tag[0] = -7
            g = make(s)
            g.set_particles(s.x, s.v, tag, s.X0)
    assert e.value.code == -1


def test_deterministic_steps_resume_bitwise_from_a_checkpoint():
    """Deterministic step mode (MD_SCHED_DETERMINISTIC): a RESPA run of 5 and
    then 7 outer steps on one system equals, bit for bit, 5 steps,
    md_get_state, a fresh system restored by md_set_state, and 7 more steps
    -- positions, velocities and forces (the counter-based pair noise resumes
    at the restored time index, and fixed-point force sums do not depend on
    the particle order the new system's lists give).  Both runs end a call
    after step 5: a call closes its last step's fluid-level half kick
    separately, where consecutive steps inside one call fuse it with the next
    opening half kick."""
    import paper_2205_14121_gb300 as M
    s = small_shells(seed=53)
    a = make(s)
    a.mts_step(5, mode=M.MD_MODE_RESPA, k_p=4, deterministic=True)
    a.mts_step(7, mode=M.MD_MODE_RESPA, k_p=4, deterministic=True)
    xa, va, _ = a.read_particles()
    fa = a.read_forces(M.MD_LEVEL_ALL)
    b = make(s)
    b.mts_step(5, mode=M.MD_MODE_RESPA, k_p=4, deterministic=True)
    blob = b.get_state()
    b.close()
    c = make(s)
    c.set_state(blob)
    c.mts_step(7, mode=M.MD_MODE_RESPA, k_p=4, deterministic=True)
    xc, vc, _ = c.read_particles()
    fc = c.read_forces(M.MD_LEVEL_ALL)
    assert np.array_equal(xa, xc)
    assert np.array_equal(va, vc)
    assert np.array_equal(fa, fc)
    with pytest.raises(M.MdError) as e:           # AI-MTS has no deterministic step mode
        c.set_platelet_levels(np.array([10, 10], np.int32))
        c.mts_step(1, mode=M.MD_MODE_AI, deterministic=True)
    assert e.value.code == -1
    a.close()
    c.close()


def test_deterministic_steps_repeat_bitwise():
    """Two deterministic STS runs from the same state agree bit for bit (the
    default mode's float atomics may not)."""
    import paper_2205_14121_gb300 as M
    s = small_shells(seed=55)
    out = []
    for _ in range(2):
        g = make(s)
        g.mts_step(20, deterministic=True)
        out.append(g.read_particles()[:2])
        g.close()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
