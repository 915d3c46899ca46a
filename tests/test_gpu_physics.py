"""Physics of the GPU path over longer runs than the oracle can afford:
the plasma in the walled channel carries the parabolic Poiseuille profile of
its body force (Sec. 4.2, Fig. 4), at the temperature of the thermostat."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_poiseuille_profile_in_the_walled_channel():
    """Starting on the steady profile of the viscosity estimate, the time-
    averaged plasma v_x(y) stays parabolic (R^2 > 0.98) with the curvature of
    rho g / (2 eta) for an eta within 25% of the estimate, and kT stays 1."""
    import paper_2205_14121_gb300 as M
    import synth
    box = (30.0, 24.0, 20.0)
    g = 0.005
    # plasma only: a walled box started on the steady profile of the estimate
    s = synth.plasma_box(box=box, walls=True, body_force=g, seed=77)
    mob = s.tag == -1
    y = s.x[mob, 1]
    s.v[mob, 0] += 3.0 * g * y * (box[1] - y) / (2.0 * synth.ETA_DPD)
    sysm = M.System(s.box, s.x, s.v, s.tag, walls=True, wall=s.wall, body_force=g)
    sysm.mts_step(200)
    prof, temps = [], []
    for _ in range(40):
        sysm.mts_step(25)
        prof.append(sysm.flow_profile(24)[0])
        temps.append(sysm.observables()["temperature"])
    u = np.mean(prof, 0)
    yc = (np.arange(24) + 0.5) * box[1] / 24
    c = np.polyfit(yc, u, 2)
    fit = np.polyval(c, yc)
    r2 = 1.0 - ((u - fit) ** 2).sum() / ((u - u.mean()) ** 2).sum()
    eta = -3.0 * g / (2.0 * c[0])          # u = rho g y (Ly - y) / (2 eta): leading coefficient -rho g / (2 eta)
    print(dict(r2=r2, eta=eta, umax=u.max(), T=np.mean(temps)))
    assert r2 > 0.98
    assert abs(eta / synth.ETA_DPD - 1.0) < 0.25
    assert abs(np.mean(temps) - 1.0) < 0.03
