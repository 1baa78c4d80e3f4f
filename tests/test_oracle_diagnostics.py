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


# ---- curvilinear meshes ----------------------------------------------------
def test_curved_fields_on_an_axis_aligned_box_equal_the_box_oracle():
    """A box given as node coordinates (Dirichlet x-ends, F and G): the
    chain-rule gradient with the curl-form metrics is the box's (2/h) d/dxi,
    so every field equals macro_fields on discontinuous random data."""
    from oracle import curved, stage
    from paper_2312_06567_gb300 import workloads as W
    wl = W.reduced(W.normal_shock_tube(), mesh_n=(4, 2, 2), vel_n=(4, 4, 4)).replace(p=2)
    x = W.node_positions(wl)
    P = wl.n_elem * wl.n_sol
    rng = np.random.default_rng(3)
    m = _moments(1 + 0.3 * rng.uniform(size=P), 0.2 * rng.standard_normal((P, 3)), 1 + 0.3 * rng.uniform(size=P),
                 delta=wl.delta)
    box = diagnostics.macro_fields(stage.problem_from_workload(wl), m)
    curv = diagnostics.macro_fields_curved(curved.problem_from_workload(wl, x), m)
    assert np.max(np.abs(curv - box) / np.abs(box)) <= 1e-12


def test_curved_gradient_is_exact_for_linear_density_on_trilinear_elements():
    """Trilinear elements of a sphere shell (azimuth periodic, closed radial and
    polar faces), p = 2: a density linear in x is a polynomial of degree 1 per
    reference direction, continuous across faces, and the curl-form metrics are
    exact (S^d / J = grad xi_d), so grad rho = a at every node."""
    from oracle import curved
    from oracle.fr import FR1D
    from paper_2312_06567_gb300 import workloads as W
    p, n = 2, (2, 3, 4)
    ogrid = W.sphere_ogrid(n=n, p=1)
    xi = FR1D(p).xi
    q = p + 1
    g3, g2, g1 = np.meshgrid(xi, xi, xi, indexing="ij")
    loc = np.stack([g1.ravel(), g2.ravel(), g3.ravel()], axis=1)
    x = np.zeros((ogrid.n_elem, q ** 3, 3))
    for e in range(ogrid.n_elem):
        c = np.array([e % n[0], (e // n[0]) % n[1], e // (n[0] * n[1])], dtype=np.float64)
        for a in (0, 1):
            for b in (0, 1):
                for cc in (0, 1):
                    v = ogrid.mapping((c + np.array([a, b, cc])) / np.asarray(n, dtype=np.float64))
                    s = ((1 + (2 * a - 1) * loc[:, 0]) * (1 + (2 * b - 1) * loc[:, 1]) * (1 + (2 * cc - 1) * loc[:, 2]) / 8)
                    x[e] += s[:, None] * v
    mesh = curved.CurvedMesh(n, (False, False, True), x, p)
    pb = curved.CurvedProblem(mesh, VelocityGrid((3, 3, 3), (-3.0,) * 3, (3.0,) * 3), bgk.Gas(),
                              closed=[(0, -1), (0, 1), (1, -1), (1, 1)])
    a = np.array([0.3, -0.5, 0.2])
    xs = x.reshape(-1, 3)
    rho = 2.0 + xs @ a
    f = diagnostics.macro_fields_curved(pb, _moments(rho, np.zeros((len(rho), 3)), np.ones(len(rho))))
    assert np.max(np.abs(f[:, 8] - np.linalg.norm(a))) <= 1e-12 * np.linalg.norm(a)


def test_curved_gradient_converges_on_a_warped_mesh():
    """Smooth periodic density on the warped periodic box: the gradient's
    max-norm error falls at order ~p (p = 2, 3; at p = 1 the trilinear
    geometry's metric error dominates)."""
    from oracle import curved
    from paper_2312_06567_gb300 import workloads as W
    for p in (2, 3):
        errs = []
        for nn in (4, 8, 16):
            wl = W.wavy_periodic_box(p=p, n=(nn, nn, nn), vel_n=(3, 3, 3))
            xx = W.node_positions(wl)
            x = xx.reshape(-1, 3)
            rho = 1 + 0.2 * np.sin(2 * np.pi * x[:, 0]) * np.cos(2 * np.pi * x[:, 1])
            g = np.stack([0.4 * np.pi * np.cos(2 * np.pi * x[:, 0]) * np.cos(2 * np.pi * x[:, 1]),
                          -0.4 * np.pi * np.sin(2 * np.pi * x[:, 0]) * np.sin(2 * np.pi * x[:, 1]),
                          np.zeros(len(x))], axis=1)
            f = diagnostics.macro_fields_curved(curved.problem_from_workload(wl, xx),
                                                _moments(rho, np.zeros((len(rho), 3)), np.ones(len(rho))))
            errs.append(float(np.max(np.abs(f[:, 8] - np.linalg.norm(g, axis=1)))))
        assert errs[0] > errs[1] > errs[2], (p, errs)
        assert np.log2(errs[1] / errs[2]) >= p - 0.6, (p, errs)
