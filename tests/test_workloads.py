"""Pins of the synthetic workload definitions (input generators)."""
import math
import os

import numpy as np
import pytest

from paper_2312_06567_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_normal_shock_states_match_naca_1135_table():
    ref = {}
    for line in open(os.path.join(GOLDEN, "normal_shock_m8_g14.txt")):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()
            ref[k] = float(v)
    (r1, u1, t1), (r2, u2, t2) = W.normal_shock_states(8.0, 1.4)
    assert r2 / r1 == pytest.approx(ref["rho2_over_rho1"], rel=2e-4)
    assert (r2 * t2) / (r1 * t1) == pytest.approx(ref["p2_over_p1"], rel=2e-4)
    assert t2 / t1 == pytest.approx(ref["T2_over_T1"], rel=5e-4)
    assert u2 / math.sqrt(1.4 * t2) == pytest.approx(ref["M2"], rel=2e-4)
    # mass flux continuity across the shock
    assert r1 * u1 == pytest.approx(r2 * u2, rel=1e-14)


def test_workload_sizes():
    a, b, c = W.periodic_sine_box(), W.taylor_green_box(), W.normal_shock_tube()
    assert (a.n_elem, a.n_sol, a.n_vel, a.dof) == (64, 8, 512, 262144)
    assert (b.n_elem, b.n_sol, b.n_vel) == (4096, 64, 13824) and b.dof == 3623878656
    assert (c.n_elem, c.n_sol, c.n_vel, c.n_comp) == (1024, 27, 32768, 2)
    assert a.dt() == pytest.approx(0.1 * 0.25 / (6 * 3))
    assert W.mu_from_knudsen(0.1) == pytest.approx(0.0797884560802865, rel=1e-14)


def test_node_and_velocity_layout():
    wl = W.reduced(W.periodic_sine_box(), mesh_n=(3, 2, 2), vel_n=(2, 3, 4))
    x = W.node_positions(wl)
    # element e = e1 + n1 (e2 + n2 e3), node s = i1 + q (i2 + q i3)
    e = 1 + 3 * (1 + 2 * 1)
    s = 1 + 2 * (0 + 2 * 1)
    r = 1 / math.sqrt(3)
    h = np.array([1 / 3, 1 / 2, 1 / 2])
    exp = np.array([1, 1, 1]) * h + (np.array([r, -r, r]) + 1) / 2 * h
    assert np.allclose(x[e, s], exp)
    u = W.velocity_nodes(wl)
    k = 1 + 2 * (2 + 3 * 3)
    assert np.allclose(u[k], [6, 6, 6])
    assert np.allclose(u[0], [-6, -6, -6])


def test_initial_maxwellian_state_shapes_and_g_factor():
    wl = W.reduced(W.normal_shock_tube(), mesh_n=(4, 1, 1), vel_n=(6, 4, 4))
    f = W.maxwellian_state(wl)
    assert f.shape == (2, 96, 4, 27)
    x = W.node_positions(wl)
    _, _, theta = wl.init(x)
    assert np.allclose(f[1], (theta.reshape(1, 4, 27)) * f[0])   # delta/2 = 1
    assert np.all(f >= 0) and np.all(f.max(axis=1) > 0)
