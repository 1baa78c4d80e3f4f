"""GPU (CUDA, through the C-ABI) vs the FP64 CPU oracle, element by element.

Tolerances: FP64 path within 1e-12 relative.  "Relative" for a state-shaped
array is per velocity slab: max over (e, s) of |gpu - oracle| divided by the
slab's max |oracle| (or, for a residual R, by the slab's max |f| times the
fastest rate in it, sum_d 2|u_d|/h_d + max 1/tau, i.e. the error of
f + dt R at the largest stable dt).  Moments and Q' are compared per point,
scaled by rho, rho sqrt(theta) and E.
"""
import numpy as np
import pytest

from oracle import bgk as obgk
from oracle import stage as ostage
from paper_2312_06567_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def lib(libbgk, cuda_device):
    from paper_2312_06567_gb300 import bgk
    return bgk


def slab_err(a, b):
    C, Nu = b.shape[:2]
    d = np.abs(a - b).reshape(C * Nu, -1).max(axis=1)
    s = np.abs(b).reshape(C * Nu, -1).max(axis=1)
    return float(np.max(d / np.maximum(s, 1e-300)))


def rhs_err(r_gpu, r_ora, f, wl, tau_min):
    C, Nu = f.shape[:2]
    u = W.velocity_nodes(wl)
    h = np.array([(wl.mesh_hi[d] - wl.mesh_lo[d]) / wl.mesh_n[d] for d in range(3)])
    rate = np.sum(2 * np.abs(u) / h, axis=1) + 1.0 / tau_min           # [Nu]
    scale = np.abs(f).reshape(C, Nu, -1).max(axis=2) * rate[None, :]
    d = np.abs(r_gpu - r_ora).reshape(C, Nu, -1).max(axis=2)
    return float(np.max(d / np.maximum(scale, 1e-300)))


def moment_err(m_gpu, m_ora, delta=0.0):
    gas = obgk.Gas(delta=delta)
    rho, U, E, th, P, Pi = obgk.macroscopic(m_ora, gas)
    sc = np.stack([rho, rho * np.sqrt(th), rho * np.sqrt(th), rho * np.sqrt(th),
                   rho * th, rho * th, rho * th, rho * th, rho * th, rho * th,
                   np.maximum(m_ora[:, 10], rho * th)], axis=1)
    return float(np.max(np.abs(m_gpu - m_ora) / sc))


def _mild_es_box(mesh_n=(3, 2, 2), p=3, vel_n=(10, 9, 8)):
    """Taylor--Green physics (ES-BGK Pr=2/3) at a size the oracle handles,
    with a ragged velocity grid."""
    return W.reduced(W.taylor_green_box(), mesh_n=mesh_n, vel_n=vel_n).replace(p=p)


def _mild_shock(mesh_n=(6, 1, 1), vel_n=(16, 10, 9), mach=3.0):
    """Polyatomic (F, G) normal shock with Dirichlet x-ends at M=3, on a velocity
    box narrowed to the M=3 states so a small grid still resolves them."""
    wl = W.reduced(W.normal_shock_tube(mach=mach), mesh_n=mesh_n, vel_n=vel_n)
    return wl.replace(vel_lo=(-9.0, -8.0, -8.0), vel_hi=(11.0, 8.0, 8.0))


CASES = {
    "sine_box_p1": lambda: W.periodic_sine_box(),
    "tgv_es_p3_ragged": lambda: _mild_es_box(),
    "shock_fg_p2_dirichlet": lambda: _mild_shock(),
    "tiny_p4_single_element": lambda: _mild_es_box(mesh_n=(1, 1, 1), p=4, vel_n=(9, 8, 10)),
    "ragged_p1_dirichlet_x": lambda: _mild_shock(mesh_n=(3, 1, 2), vel_n=(13, 9, 11)).replace(
        p=1),
}


@pytest.mark.parametrize("name", list(CASES))
def test_moments_and_rhs_match_oracle(lib, name):
    wl = CASES[name]()
    pb = ostage.problem_from_workload(wl)
    f = W.random_anisotropic_state(wl, seed=11)
    with lib.Solver(wl) as s:
        s.set_state(f)
        m_gpu = s.moments()
        r_gpu = s.rhs(f)
    m_ora = obgk.raw_moments(f[0].reshape(wl.n_vel, -1), f[1].reshape(wl.n_vel, -1)
                             if wl.n_comp == 2 else None, pb.vg)
    assert moment_err(m_gpu, m_ora, wl.delta) <= 1e-13
    r_ora, info = pb.rhs(f)
    assert np.all(info["converged"])
    assert rhs_err(r_gpu, r_ora, f, wl, info["tau"].min()) <= TOL


@pytest.mark.parametrize("name", ["sine_box_p1", "tgv_es_p3_ragged", "shock_fg_p2_dirichlet"])
def test_one_step_matches_oracle(lib, name):
    wl = CASES[name]()
    pb = ostage.problem_from_workload(wl)
    f = W.random_anisotropic_state(wl, seed=5)
    dt = wl.dt()
    with lib.Solver(wl) as s:
        s.set_state(f)
        assert s.step(dt, 1) == lib.BGK_OK
        f_gpu = s.get_state()
    f_ora, _ = pb.step(f, dt)
    assert slab_err(f_gpu, f_ora) <= TOL


def test_full_small_config_ten_steps_and_conservation(lib):
    """The 4^3, p=1, 8^3-velocity periodic sine box for its 10 SSP-RK3 steps:
    element-wise parity with the oracle and totals kept to round-off."""
    wl = W.periodic_sine_box()
    pb = ostage.problem_from_workload(wl)
    f0 = W.maxwellian_state(wl)
    dt = wl.dt()
    with lib.Solver(wl) as s:
        s.set_state(f0)
        t_prev = s.totals()
        drift = 0.0
        for _ in range(wl.steps):
            assert s.step(dt, 1) == lib.BGK_OK
            t = s.totals()
            scale = np.array([t_prev[0]] * 4 + [t_prev[4]])
            drift = max(drift, float(np.max(np.abs(t - t_prev) / scale)))
            t_prev = t
        f_gpu = s.get_state()
        mean_it, max_it, res = s.stats()
    f = f0
    for _ in range(wl.steps):
        f, _ = pb.step(f, dt)
    assert slab_err(f_gpu, f) <= TOL
    assert drift <= 1e-12
    assert max_it <= 50 and res <= 1e-13


@pytest.mark.parametrize("delta,Pr", [(0.0, 2 / 3), (2.0, 0.72), (0.0, 1.0)])
def test_qprime_matches_oracle(lib, delta, Pr):
    wl = _mild_es_box(mesh_n=(2, 1, 1), p=2, vel_n=(14, 12, 13)).replace(delta=delta, Pr=Pr)
    f = W.random_anisotropic_state(wl, seed=3)
    pb = ostage.problem_from_workload(wl)
    F = f[0].reshape(wl.n_vel, -1)
    G = f[1].reshape(wl.n_vel, -1) if wl.n_comp == 2 else None
    m = obgk.raw_moments(F, G, pb.vg)
    qp_o, it_o, conv, res = obgk.solve_qprime(m, pb.gas, pb.vg)
    assert np.all(conv)
    with lib.Solver(wl) as s:
        qp_g, it_g, st = s.qprime(m)
    assert st == lib.BGK_OK
    th = qp_o[:, 4]
    assert np.max(np.abs(qp_g[:, 0] - qp_o[:, 0]) / qp_o[:, 0]) <= TOL
    assert np.max(np.abs(qp_g[:, 1:4] - qp_o[:, 1:4]) / np.sqrt(th)[:, None]) <= TOL
    assert np.max(np.abs(qp_g[:, 4] - th) / th) <= TOL
    assert np.all(np.abs(it_g - it_o) <= 1)


def test_set_maxwellian_matches_generator(lib):
    wl = _mild_shock()
    x = W.node_positions(wl)
    rho, U, theta = wl.init(x)
    q = np.concatenate([rho.reshape(-1, 1), U.reshape(-1, 3), theta.reshape(-1, 1)], axis=1)
    with lib.Solver(wl) as s:
        assert np.allclose(s.node_coords(), x, rtol=0, atol=1e-13)
        s.set_maxwellian(q)
        f_gpu = s.get_state()
    assert slab_err(f_gpu, W.maxwellian_state(wl)) <= TOL


def test_newton_nonconvergence_is_reported_not_trapped(lib):
    """max_iter = 0 on a non-equilibrium state: the device status word reports
    BGK_ENOCONV through the return code; the context stays usable."""
    wl = _mild_es_box(mesh_n=(2, 1, 1), p=1, vel_n=(8, 8, 8))
    f = W.random_anisotropic_state(wl, seed=2)
    with lib.Solver(wl) as s:
        s.set_state(f)
        s.set_newton(1e-13, 0)
        assert s.step(wl.dt(), 1) == lib.BGK_ENOCONV
        s.set_newton(1e-13, 50)
        s.set_state(f)
        assert s.step(wl.dt(), 1) == lib.BGK_OK


def test_degenerate_and_rejected_calls_leave_the_context_usable(lib):
    """Zero steps leave the state and totals bit for bit; a non-positive dt, a
    negative step count and an empty Q' batch are rejected with BGK_EINVAL
    before any launch; the context then steps and matches the oracle."""
    wl = CASES["sine_box_p1"]()
    f = W.random_anisotropic_state(wl, seed=5)           # the state of test_one_step_matches_oracle
    dt = wl.dt()
    with lib.Solver(wl) as s:
        s.set_state(f)
        t0 = s.totals()
        assert s.step(dt, 0) == lib.BGK_OK
        assert np.array_equal(s.get_state(), f)
        assert np.array_equal(s.totals(), t0)
        for bad_dt, n in ((0.0, 1), (-dt, 1), (float("nan"), 1), (dt, -1)):
            with pytest.raises(lib.BGKError) as ei:
                s.step(bad_dt, n)
            assert ei.value.status == lib.BGK_EINVAL
        with pytest.raises(lib.BGKError) as ei:
            s.qprime(np.zeros((0, 11)))
        assert ei.value.status == lib.BGK_EINVAL
        assert np.array_equal(s.get_state(), f)
        assert s.step(dt, 1) == lib.BGK_OK
        f_gpu = s.get_state()
    f_ora, _ = ostage.problem_from_workload(wl).step(f, dt)
    assert slab_err(f_gpu, f_ora) <= TOL
