"""Pins of the macroscopic post-processing reference (oracle/diagnostics.py):
the FR density gradient is exact for fields that are polynomials of degree <= p
and continuous across faces (including Dirichlet faces holding the field's
value), converges at order >= p on a smooth periodic field, and carries the
central common value at a jump; Mach, lambda and Kn_GLL follow their
definitions."""
import numpy as np

from oracle import bgk, diagnostics
from oracle.mesh import BoxMesh
from oracle.stage import Problem
from oracle.velocity import VelocityGrid


def _moments(rho, U, theta, delta=0.0):
    """Raw moments m[P, 11] of the fields (a Maxwellian's, in closed form)."""
    P = len(rho)
    m = np.zeros((P, 11))
    m[:, 0] = rho
    m[:, 1:4] = rho[:, None] * U
    for i in range(3):
        m[:, 4 + i] = rho * (U[:, i] ** 2 + theta)
    m[:, 7] = rho * U[:, 0] * U[:, 1]
    m[:, 8] = rho * U[:, 0] * U[:, 2]
    m[:, 9] = rho * U[:, 1] * U[:, 2]
    m[:, 10] = 0.5 * delta * rho * theta
    return m


def _problem(n, p, lo, hi, periodic, dirichlet=None, delta=0.0):
    mesh = BoxMesh(n, lo, hi, periodic)
    gas = bgk.Gas(delta=delta, Pr=2.0 / 3.0, mu_ref=0.05, theta_ref=1.0, theta_S=0.5)
    return Problem(mesh, p, VelocityGrid((4, 4, 4), (-3, -3, -3), (3, 3, 3)), gas, dirichlet=dirichlet)


def test_gradient_exact_for_continuous_polynomial_with_dirichlet_ends():
    b = 0.3
    for p in (1, 2, 3):
        dirichlet = {(0, -1): (1.0 + b * 0.0, (0, 0, 0), 1.0), (0, 1): (1.0 + b * 2.0, (0, 0, 0), 1.0)}
        pb = _problem((3, 2, 2), p, (0, 0, 0), (2, 1, 1), (False, True, True), dirichlet)
        x = pb.mesh.node_coords(pb.fr.xi).reshape(-1, 3)
        rho = 1.0 + b * x[:, 0]
        out = diagnostics.macro_fields(pb, _moments(rho, np.zeros((len(rho), 3)), np.ones(len(rho))))
        assert np.allclose(out[:, 0], rho, rtol=1e-14)
        assert np.allclose(out[:, 8], b, rtol=1e-12)


def test_gradient_converges_on_a_periodic_sine():
    errs = []
    for n in (4, 8, 16):
        pb = _problem((n, 1, 1), 2, (0, 0, 0), (2 * np.pi, 1, 1), (True, True, True))
        x = pb.mesh.node_coords(pb.fr.xi).reshape(-1, 3)
        rho = 1.0 + 0.1 * np.sin(x[:, 0])
        out = diagnostics.macro_fields(pb, _moments(rho, np.zeros((len(rho), 3)), np.ones(len(rho))))
        errs.append(np.max(np.abs(out[:, 8] - np.abs(0.1 * np.cos(x[:, 0])))))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates >= 2.0), rates


def test_jump_gets_the_central_common_value():
    """Piecewise-constant density (1 on the left element, 3 on the right,
    periodic): the FR gradient inside each element is the correction
    derivative times half the jump, with the sign of the side it sits on."""
    p = 2
    pb = _problem((2, 1, 1), p, (0, 0, 0), (2, 1, 1), (True, True, True))
    q = p + 1
    rho = np.repeat([1.0, 3.0], q ** 3)
    out = diagnostics.macro_fields(pb, _moments(rho, np.zeros((len(rho), 3)), np.ones(len(rho))))
    h = 1.0
    # left element: right face common 2 (jump +1), left face (periodic) common 2 (jump +1)
    g_left = (2.0 / h) * (1.0 * pb.fr.dgR + 1.0 * pb.fr.dgL)
    i1 = np.arange(q ** 3) % q
    assert np.allclose(out[: q ** 3, 8], np.abs(g_left[i1]), atol=1e-13)
    g_right = (2.0 / h) * (-1.0 * pb.fr.dgR - 1.0 * pb.fr.dgL)
    assert np.allclose(out[q ** 3:, 8], np.abs(g_right[i1]), atol=1e-13)


def test_mach_lambda_and_knudsen_definitions():
    pb = _problem((2, 1, 1), 1, (0, 0, 0), (2 * np.pi, 1, 1), (True, True, True), delta=2.0)
    x = pb.mesh.node_coords(pb.fr.xi).reshape(-1, 3)
    P = len(x)
    rho = 1.0 + 0.2 * np.sin(x[:, 0])
    U = np.column_stack([np.full(P, 0.4), np.full(P, -0.1), np.zeros(P)])
    th = np.full(P, 0.8)
    out = diagnostics.macro_fields(pb, _moments(rho, U, th, delta=2.0))
    gamma = 7.0 / 5.0
    assert np.allclose(out[:, 4], th, rtol=1e-13)
    assert np.allclose(out[:, 5], rho * th, rtol=1e-13)
    assert np.allclose(out[:, 6], np.sqrt(0.17 / (gamma * 0.8)), rtol=1e-13)
    lam = pb.gas.viscosity(th) / rho * np.sqrt(np.pi / (2 * th))
    assert np.allclose(out[:, 7], lam, rtol=1e-13)
    assert np.allclose(out[:, 9], lam * out[:, 8] / rho, rtol=1e-13)
