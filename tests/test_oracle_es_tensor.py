"""Pins of the tensor variant of the discrete ES equilibrium (monatomic):
brute-force discrete moments, the analytic Jacobian, the Maxwellian fixed
point on a symmetric grid, exact conservation of a full step, and the
property it exists for -- the discrete stress of the source relaxes exactly
toward the ES target, which the d+2 solve does not do."""
import math

import numpy as np
import pytest

from oracle import bgk, stage
from oracle.velocity import VelocityGrid
from paper_2312_06567_gb300 import workloads as W


def _state(seed, P=6, vel=(9, 8, 10), lo=(-6.0, -5.0, -6.5), hi=(6.5, 5.5, 6.0)):
    vg = VelocityGrid(vel, lo, hi)
    rng = np.random.default_rng(seed)
    F = np.zeros((vg.size, P))
    for part in range(2):
        U = 0.4 * rng.standard_normal((P, 3))
        a = 0.35 * rng.standard_normal((P, 3, 3))
        cov = np.eye(3)[None] * (0.8 + 0.4 * rng.uniform(size=(P, 1, 1))) + np.einsum("pij,pkj->pik", a, a)
        F += (0.7 if part == 0 else 0.3) * bgk.gaussian(vg.u, 1.0 + 0.2 * rng.uniform(size=P), U, cov)
    return vg, F


@pytest.mark.parametrize("Pr", [2.0 / 3.0, 0.72, 1.0])
def test_tensor_equilibrium_has_the_target_discrete_moments(Pr):
    """fsum over the velocity grid: sum w g = rho, sum w u g = rho U,
    sum w (u-U)(u-U)^T g = rho T with T the ES target tensor, to 1e-13."""
    vg, F = _state(1)
    gas = bgk.Gas(Pr=Pr, es_tensor=True)
    m = bgk.raw_moments(F, None, vg)
    b, U, it, conv, res = bgk.solve_qprime_tensor(m, gas, vg)
    assert np.all(conv)
    g = bgk.tensor_equilibrium(b, U, vg)
    rho, Uf, E, theta, pres, Pi = bgk.macroscopic(m, gas)
    T = bgk.temperature_tensor(theta, Pi / rho[:, None, None], Pr)
    for p in range(F.shape[1]):
        w = vg.w
        assert abs(math.fsum(w * g[:, p]) - rho[p]) <= 1e-13 * rho[p]
        for d in range(3):
            assert abs(math.fsum(w * vg.u[:, d] * g[:, p]) - rho[p] * Uf[p, d]) <= 1e-13 * rho[p] * math.sqrt(theta[p]) * 10
        c = vg.u - Uf[p]
        for i in range(3):
            for j in range(3):
                s = math.fsum(w * c[:, i] * c[:, j] * g[:, p])
                assert abs(s - rho[p] * T[p, i, j]) <= 1e-13 * rho[p] * theta[p] * 10
        # energy is the trace: conserved
        e = math.fsum(w * 0.5 * np.sum(vg.u * vg.u, axis=1) * g[:, p])
        assert abs(e - E[p]) <= 1e-13 * E[p] * 10


def test_tensor_jacobian_equals_central_differences():
    vg, F = _state(2, P=3)
    gas = bgk.Gas(Pr=0.72, es_tensor=True)
    m = bgk.raw_moments(F, None, vg)
    t, U, rho, theta = bgk.tensor_targets(m, gas)
    b, _, _, _, _ = bgk.solve_qprime_tensor(m, gas, vg, max_iter=1)
    R, J, _ = bgk.tensor_residual(b, t, U, vg)
    h = 1e-6
    for a in range(10):
        bp, bm = b.copy(), b.copy()
        bp[:, a] += h
        bm[:, a] -= h
        Rp, _, _ = bgk.tensor_residual(bp, t, U, vg)
        Rm, _, _ = bgk.tensor_residual(bm, t, U, vg)
        fd = (Rp - Rm) / (2 * h)
        assert np.max(np.abs(fd - J[:, :, a])) <= 1e-6 * np.max(np.abs(J))


def test_symmetric_maxwellian_is_a_fixed_point_and_agrees_with_the_d_plus_2_solve():
    """U = 0 on a grid symmetric in every axis, Pr = 1: the sampled
    Maxwellian's discrete covariance is isotropic, so both solves return it."""
    vg = VelocityGrid((9, 9, 9), (-6.0, -6.0, -6.0), (6.0, 6.0, 6.0))
    rho = np.array([1.0, 0.7, 1.6])
    theta = np.array([1.0, 0.6, 1.7])
    F = bgk.maxwellian(vg, rho, np.zeros((3, 3)), theta)
    m = bgk.raw_moments(F, None, vg)
    gt = bgk.Gas(Pr=1.0, es_tensor=True)
    b, U, it, conv, res = bgk.solve_qprime_tensor(m, gt, vg)
    g = bgk.tensor_equilibrium(b, U, vg)
    assert np.max(np.abs(g - F)) <= 1e-13 * np.max(F)
    qp, _, _, _ = bgk.solve_qprime(m, bgk.Gas(Pr=1.0), vg)
    g5, _ = bgk.equilibrium(qp, m, bgk.Gas(Pr=1.0), vg)
    assert np.max(np.abs(g - g5)) <= 1e-13 * np.max(F)


def test_tensor_step_conserves_totals():
    wl = W.reduced(W.taylor_green_box(), mesh_n=(2, 2, 2), vel_n=(10, 9, 8)).replace(p=2, es_tensor=True)
    pb = stage.problem_from_workload(wl)
    f = W.random_anisotropic_state(wl, seed=9)
    t0 = pb.totals(f)
    f1, infos = pb.step(f, wl.dt())
    assert all(np.all(i["converged"]) for i in infos)
    t1 = pb.totals(f1)
    scale = np.max(np.abs(pb.totals(np.abs(f))))
    assert np.all(np.abs(t1 - t0) <= 1e-13 * scale)


def test_source_relaxes_the_discrete_stress_exactly_toward_the_es_target():
    """sum w (u-U)(u-U)^T S = (rho T - Pi)/tau exactly with the tensor variant;
    the d+2 solve misses it on a coarse grid by far more than rounding."""
    vg, F = _state(3, P=4, vel=(7, 6, 8))
    out = {}
    for tensor in (True, False):
        gas = bgk.Gas(Pr=0.72, es_tensor=tensor)
        S, _, info = bgk.bgk_source(F, None, gas, vg)
        m = info["m"]
        rho, U, E, theta, pres, Pi = bgk.macroscopic(m, gas)
        T = bgk.temperature_tensor(theta, Pi / rho[:, None, None], gas.Pr)
        target = (rho[:, None, None] * T - Pi) / info["tau"][:, None, None]
        c = vg.u[:, None, :] - U[None, :, :]
        got = np.einsum("k,kpi,kpj,kp->pij", vg.w, c, c, S)
        out[tensor] = np.max(np.abs(got - target) / np.abs(target).max())
    assert out[True] <= 1e-11
    assert out[False] >= 1e-6
