"""Pins of the shock / sonic-surface post-processing on fields whose answers
are closed forms (no GPU)."""
import numpy as np

from paper_2312_06567_gb300 import postprocess as pp
from paper_2312_06567_gb300 import workloads as W


def test_first_axis_lines_run_through_the_mesh():
    wl = W.reduced(W.normal_shock_tube(), mesh_n=(5, 2, 3)).replace(p=2)
    lines = pp.first_axis_lines(wl)
    x = W.node_positions(wl).reshape(-1, 3)
    assert lines.shape == (2 * 3 * 9, 5 * 3)
    assert len(np.unique(lines)) == wl.n_elem * wl.n_sol            # every node once
    for pts in lines[:7]:
        assert np.all(np.diff(x[pts, 0]) > 0)                      # ordered along x
        assert np.ptp(x[pts, 1]) == 0 and np.ptp(x[pts, 2]) == 0   # one (y, z) each


def test_mach_crossing_of_a_linear_field_is_exact():
    x = np.zeros((6, 3))
    x[:, 0] = np.linspace(0.0, 5.0, 6)
    mach = 2.2 - 0.4 * x[:, 0]                                      # Mach = 1 at x = 3
    cr = pp.mach_crossings(x, mach, [np.arange(6)])
    assert len(cr) == 1 and abs(cr[0][1][0] - 3.0) < 1e-14


def test_max_gradient_of_a_tanh_shock_and_its_thickness():
    """rho = a + b tanh((s - s0)/w): the gradient peaks at s0 (the parabola
    refinement finds it to the grid's curvature error), and the max-slope
    thickness (rho_2 - rho_1) / (b/w) is 2 w."""
    a, b, w, s0 = 3.0, 2.0, 0.7, 1.234
    s = np.linspace(-5.0, 5.0, 401)
    x = np.zeros((len(s), 3))
    x[:, 0] = s
    g = b / w / np.cosh((s - s0) / w) ** 2
    pos, pt = pp.max_gradient_position(x, g, np.arange(len(s)))
    assert abs(pos - (s0 + 5.0)) < 1e-4 and abs(pt[0] - s0) < 1e-4
    assert abs(pp.max_slope_thickness(a - b, a + b, b / w) - 2 * w) < 1e-14
