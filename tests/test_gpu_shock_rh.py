"""Pin P10 on the GPU: the M = 8 normal shock at full size (64x4x4 hex, p = 2,
32^3 velocities, F and G) for its 2000 mixed-form SSP-RK3 steps.

The far field must stay at the Rankine--Hugoniot states the Dirichlet ends
impose (section "Results", low-altitude conditions, normal-shock physics).
What those ends impose is the Maxwellian of each state sampled on the
velocity grid; on this grid the upstream Maxwellian (thermal speed 1) is
sampled at a spacing of 1.94 thermal speeds along the first axis, so its
discrete moments differ from the continuous state by 0.8% in density and 1.7%
in temperature (the downstream one, at theta = 13.4, by 3e-4).  So the
solution is held, at 1e-3, to the discrete states the ends impose (computed by
the oracle from the sampled Maxwellians); and to the continuous
Rankine--Hugoniot states within that measured quadrature difference plus
1e-3.  The mass flux rho U_1 at the two ends is compared with the same
allowance.  After 2000 steps (t = 0.33 mean free times) the shock has not
settled, so the ends' flux balance is not asserted beyond that."""
import numpy as np
import pytest

from oracle import bgk as obgk
from oracle.velocity import VelocityGrid
from paper_2312_06567_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib(libbgk, cuda_device):
    from paper_2312_06567_gb300 import bgk
    return bgk


def _discrete_state(wl, vg, gas, s):
    rho, u, th = s
    F = obgk.maxwellian(vg, np.array([rho]), np.array([[u, 0.0, 0.0]]), np.array([th]))
    m = obgk.raw_moments(F, 0.5 * wl.delta * th * F, vg)
    r, U, E, t, _, _ = obgk.macroscopic(m, gas)
    return np.array([r[0], U[0, 0], t[0]])


def test_normal_shock_far_field_keeps_the_rankine_hugoniot_states(lib):
    wl = W.normal_shock_tube()
    vg = VelocityGrid(wl.vel_n, wl.vel_lo, wl.vel_hi)
    gas = obgk.Gas(delta=wl.delta, Pr=wl.Pr, mu_ref=wl.mu_ref, theta_ref=wl.theta_ref, theta_S=wl.theta_S)
    s1, s2 = W.normal_shock_states(8.0, 1.4)
    d1, d2 = _discrete_state(wl, vg, gas, s1), _discrete_state(wl, vg, gas, s2)
    c1, c2 = np.array(s1), np.array(s2)
    x = W.node_positions(wl).reshape(-1, 3)
    rho, U, theta = wl.init(x)
    q = np.zeros((x.shape[0], 5))
    q[:, 0] = rho
    q[:, 1:4] = U
    q[:, 4] = theta
    n1 = wl.mesh_n[0]
    e1 = np.repeat(np.arange(wl.n_elem) % n1, wl.n_sol)
    i1 = np.tile(np.arange(wl.n_sol) % (wl.p + 1), wl.n_elem)
    lo = (e1 == 0) & (i1 == 0)                         # nodes nearest x = -20
    hi = (e1 == n1 - 1) & (i1 == wl.p)                 # nodes nearest x = 40
    with lib.Solver(wl, lib.BGK_MIXED) as s:
        s.set_maxwellian(q)
        s.set_graphs(True)
        dt = wl.dt()
        s.tune_stage(dt, reps=1)
        assert s.step(dt, wl.steps) == lib.BGK_OK
        m = s.macro()
    for sel, dstate, cstate in ((lo, d1, c1), (hi, d2, c2)):
        got = np.stack([m[sel, 0], m[sel, 1], m[sel, 4]], axis=1)          # rho, U1, theta
        assert np.all(np.isfinite(got))
        rel_d = np.abs(got - dstate[None, :]) / np.abs(dstate[None, :])
        assert np.max(rel_d) <= 1e-3, (cstate, np.max(rel_d, axis=0))
        quad = np.abs(dstate - cstate) / np.abs(cstate)                   # the grid's quadrature difference
        rel_c = np.abs(got - cstate[None, :]) / np.abs(cstate[None, :])
        assert np.all(rel_c <= quad[None, :] + 1e-3), (cstate, np.max(rel_c, axis=0), quad)
    flux_lo = np.mean(m[lo, 0] * m[lo, 1])
    flux_hi = np.mean(m[hi, 0] * m[hi, 1])
    quad_flux = abs(d1[0] * d1[1] - d2[0] * d2[1]) / (c1[0] * c1[1])
    assert abs(flux_lo - flux_hi) / (c1[0] * c1[1]) <= quad_flux + 1e-3
