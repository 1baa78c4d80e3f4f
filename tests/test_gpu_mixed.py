"""Mixed-precision form (FP32 state and FR, FP64 moments and Q' solve) against
the FP64 oracle, through the C-ABI.

Bars: moments within 1e-5 relative of the oracle per point (scaled by rho,
rho sqrt(theta), rho theta); the residual within 1e-5 of the slab scale used
by the FP64 parity tests; the instantaneous rate of change of the totals
under the mixed residual within 1e-12 (the FP32 advection and the corrected
FP32 equilibrium are discretely conservative up to rounding); mean
conservation drift per step <= 1e-10 relative on the 2.3e8-DOF Taylor--Green
physics.  The only non-conservation left is the one rounding of each stored
FP32 value (the update is formed with a single rounding at the level of f):
a stage's totals equal those of the oracle's exact stage rounded once to FP32,
to 2e-10 of the totals.  On the sine box, whose 512 points hold only 8
distinct states, that rounding does not average out over points: one FP32
rounding per stage of the oracle's own exact stages already drifts by 1e-10
to 3e-9 per step there (tests/test_oracle_storage_floor.py), so the bar on the
10-step mean is 2e-9.
"""
import numpy as np
import pytest

from oracle import bgk as obgk
from oracle import stage as ostage
from paper_2312_06567_gb300 import workloads as W

from test_gpu_parity import CASES, moment_err, rhs_err, slab_err

pytestmark = pytest.mark.gpu

TOL_MIXED = 1e-5


@pytest.fixture(scope="module")
def lib(libbgk, cuda_device):
    from paper_2312_06567_gb300 import bgk
    return bgk


def _oracle_moments(f, wl, pb):
    return obgk.raw_moments(f[0].reshape(wl.n_vel, -1),
                            f[1].reshape(wl.n_vel, -1) if wl.n_comp == 2 else None, pb.vg)


@pytest.mark.parametrize("name", ["sine_box_p1", "tgv_es_p3_ragged", "shock_fg_p2_dirichlet",
                                  "ragged_p1_dirichlet_x"])
def test_mixed_rhs_and_step_match_oracle(lib, name):
    wl = CASES[name]()
    pb = ostage.problem_from_workload(wl)
    f32 = W.random_anisotropic_state(wl, seed=11).astype(np.float32)
    f = f32.astype(np.float64)
    with lib.Solver(wl, lib.BGK_MIXED) as s:
        s.set_state(f32)
        m_gpu = s.moments()
        r_gpu = s.rhs(f32)
        assert s.step(wl.dt(), 1) == lib.BGK_OK
        f1_gpu = s.get_state()
        m1_gpu = s.moments()
    assert moment_err(m_gpu, _oracle_moments(f, wl, pb), wl.delta) <= 1e-13
    r_ora, info = pb.rhs(f)
    assert rhs_err(r_gpu.astype(np.float64), r_ora, f, wl, info["tau"].min()) <= TOL_MIXED
    f1_ora, _ = pb.step(f, wl.dt())
    assert slab_err(f1_gpu.astype(np.float64), f1_ora) <= TOL_MIXED
    assert moment_err(m1_gpu, _oracle_moments(f1_ora, wl, pb), wl.delta) <= TOL_MIXED


def _true_totals(s):
    """Totals of the stored state with FP64 accumulation (not the stage's own
    moment epilogue): re-setting the state invalidates the cached moments."""
    s.set_state(s.get_state())
    return s.totals()


def test_mixed_small_config_ten_steps(lib):
    """Sine box, 10 steps: moments within 1e-5 of the FP64 oracle; mean drift
    per step at the FP32 storage-rounding floor of this field."""
    wl = W.periodic_sine_box()
    pb = ostage.problem_from_workload(wl)
    f0 = W.maxwellian_state(wl).astype(np.float32)
    dt = wl.dt()
    with lib.Solver(wl, lib.BGK_MIXED) as s:
        s.set_state(f0)
        t0 = s.totals()
        assert s.step(dt, wl.steps) == lib.BGK_OK
        m_gpu = s.moments()
        t1 = _true_totals(s)
    f = f0.astype(np.float64)
    for _ in range(wl.steps):
        f, _ = pb.step(f, dt)
    assert moment_err(m_gpu, _oracle_moments(f, wl, pb)) <= TOL_MIXED
    scale = np.array([t0[0]] * 4 + [t0[4]])
    assert np.all(np.abs(t1 - t0) / scale / wl.steps <= 2e-9)


@pytest.mark.parametrize("a,b,c_dt", [(0.0, 1.0, 1.0), (0.75, 0.25, 0.25), (1.0 / 3.0, 2.0 / 3.0, 2.0 / 3.0)])
def test_mixed_stage_totals_at_the_fp32_storage_floor(lib, a, b, c_dt):
    """Sine box, each Runge--Kutta stage from the state after one stage: the
    totals of the stored FP32 output equal those of the exact combination
    a f^n + b f + c R of the same FP32 inputs and the context's own residual R
    (bgk_rhs, the same kernels), rounded once to FP32, to 2e-11 of the
    totals; they differ from the unrounded combination's by up to ~1e-9 there,
    so what is left is the rounding of the stored state and nothing else (a
    second rounding of the f^n combination had added 2e-8)."""
    wl = W.periodic_sine_box()
    pb = ostage.problem_from_workload(wl)
    dt = wl.dt()
    f0 = W.maxwellian_state(wl).astype(np.float32)
    f0d = f0.astype(np.float64)
    o1, _ = pb.stage(f0d, f0d, 0.0, 1.0, dt)
    fs = o1.astype(np.float32)
    with lib.Solver(wl, lib.BGK_MIXED) as s:
        out = np.empty_like(fs)
        s.stage(f0, fs, out, a, b, c_dt * dt)
        R = s.rhs(fs).astype(np.float64)
    fa, fab, fc = np.float32(a), np.float32(a + b), np.float32(c_dt * dt)
    exact = float(fa) * f0d + (float(fab) - float(fa)) * fs.astype(np.float64) + float(fc) * R
    t_ref = pb.totals(f0d)
    scale = np.array([t_ref[0]] * 4 + [t_ref[4]])
    t_gpu = pb.totals(out.astype(np.float64))
    t_once = pb.totals(exact.astype(np.float32).astype(np.float64))
    t_exact = pb.totals(exact)
    assert np.all(np.abs(t_gpu - t_once) / scale <= 2e-11), (t_gpu - t_once) / scale
    assert np.max(np.abs(t_once - t_exact) / scale) >= 1e-11       # the rounding is what is measured


def test_mixed_residual_is_conservative(lib):
    """Totals of the mixed residual R(f) (FP64 sums of its FP32 values) vanish
    to 1e-12 of the totals times 1/dt: FP32 advection in deviation form with
    telescoping trace weights and the moment-corrected FP32 equilibrium."""
    wl = W.reduced(W.taylor_green_box(), mesh_n=(4, 4, 2))
    pb = ostage.problem_from_workload(W.reduced(wl, mesh_n=(1, 1, 1)))
    Wq = np.einsum("i,j,k->ijk", pb.fr.wq, pb.fr.wq, pb.fr.wq).reshape(-1)
    with lib.Solver(wl, lib.BGK_MIXED) as s:
        x = s.node_coords()
        rho, U, theta = wl.init(x)
        q = np.concatenate([rho.reshape(-1, 1), U.reshape(-1, 3), theta.reshape(-1, 1)], axis=1)
        s.set_maxwellian(q)
        f = s.get_state()
        r = s.rhs(f).astype(np.float64)
    w, u = pb.vg.w, pb.vg.u
    fd = f.astype(np.float64)
    for psi in (np.ones(len(w)), u[:, 0], 0.5 * np.sum(u * u, axis=1)):
        rate = np.einsum("k,kes,s->", w * psi, r[0], Wq)
        tot = np.einsum("k,kes,s->", w * np.abs(psi), fd[0], Wq)
        assert abs(rate) * wl.dt() <= 1e-12 * tot


def test_mixed_conservation_drift_at_scale(lib):
    """2.3e8 DOF of the Taylor--Green physics (8x8x4 hex, p=3, 24^3 velocities):
    total mass, momentum and energy drift <= 1e-10 relative per step, on the
    mean over 4 steps of the FP64 totals of the stored FP32 state."""
    wl = W.reduced(W.taylor_green_box(), mesh_n=(8, 8, 4))
    n = 4
    with lib.Solver(wl, lib.BGK_MIXED) as s:
        x = s.node_coords()
        rho, U, theta = wl.init(x)
        q = np.concatenate([rho.reshape(-1, 1), U.reshape(-1, 3), theta.reshape(-1, 1)], axis=1)
        s.set_maxwellian(q)
        t0 = s.totals()
        assert s.step(wl.dt(), n) == lib.BGK_OK
        t1 = _true_totals(s)
    scale = np.array([t0[0]] * 4 + [t0[4]])
    assert np.all(np.abs(t1 - t0) / scale / n <= 1e-10), (t1 - t0) / scale / n


def test_mixed_matches_fp64_form_after_steps(lib):
    """Mixed vs FP64 GPU forms on the ES Taylor--Green physics after 3 steps:
    moments within 1e-5."""
    wl = CASES["tgv_es_p3_ragged"]()
    f = W.random_anisotropic_state(wl, seed=4)
    out = {}
    for prec in (lib.BGK_FP64, lib.BGK_MIXED):
        with lib.Solver(wl, prec) as s:
            s.set_state(f if prec == lib.BGK_FP64 else f.astype(np.float32))
            assert s.step(wl.dt(), 3) == lib.BGK_OK
            out[prec] = s.moments()
    assert moment_err(out[lib.BGK_MIXED], out[lib.BGK_FP64]) <= TOL_MIXED


def test_mixed_set_maxwellian(lib):
    wl = CASES["shock_fg_p2_dirichlet"]()
    x = W.node_positions(wl)
    rho, U, theta = wl.init(x)
    q = np.concatenate([rho.reshape(-1, 1), U.reshape(-1, 3), theta.reshape(-1, 1)], axis=1)
    with lib.Solver(wl, lib.BGK_MIXED) as s:
        s.set_maxwellian(q)
        f_gpu = s.get_state()
    assert f_gpu.dtype == np.float32
    assert slab_err(f_gpu.astype(np.float64), W.maxwellian_state(wl)) <= 1e-6


def test_mixed_fp32_and_fp64_newton_sums_agree(lib):
    """The mixed form with the Q' velocity sums on the FP32 pipe (default) and
    with FP64 sums: moments within 1e-5 after 3 steps, both conservative."""
    wl = CASES["tgv_es_p3_ragged"]()
    f = W.random_anisotropic_state(wl, seed=6).astype(np.float32)
    out = {}
    for fp32 in (True, False):
        with lib.Solver(wl, lib.BGK_MIXED) as s:
            s.set_qprime_engine(fp32)
            s.set_state(f)
            t0 = s.totals()
            assert s.step(wl.dt(), 3) == lib.BGK_OK
            out[fp32] = s.moments()
            t1 = _true_totals(s)
            scale = np.array([t0[0]] * 4 + [t0[4]])
            assert np.all(np.abs(t1 - t0) / scale / 3 <= 1e-8)
    assert moment_err(out[True], out[False]) <= TOL_MIXED


def test_fp32_newton_sums_rejected_for_fp64_form(lib):
    wl = CASES["sine_box_p1"]()
    with lib.Solver(wl, lib.BGK_FP64) as s:
        with pytest.raises(lib.BGKError) as ei:
            s.set_qprime_engine(True)
        assert ei.value.status == lib.BGK_EINVAL
