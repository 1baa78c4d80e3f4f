"""Pins of the discrete velocity grid (oracle/velocity.py): the trapezoid rule
on a uniform box integrates constants and linear functions exactly, a Gaussian
to its closed form (the rule converges spectrally for smooth decaying
integrands), and nodes are ordered k = k1 + n1 (k2 + n2 k3)."""
import numpy as np

from oracle.velocity import VelocityGrid


def test_trapezoid_is_exact_for_constants_and_linear_functions():
    lo, hi = np.array([-3.0, -1.5, 0.5]), np.array([5.0, 2.5, 4.0])
    vg = VelocityGrid((7, 5, 9), lo, hi)
    vol = np.prod(hi - lo)
    assert abs(np.sum(vg.w) - vol) <= 1e-13 * vol
    for d in range(3):
        exact = vol * 0.5 * (hi[d] + lo[d])                    # integral of u_d over the box
        assert abs(np.sum(vg.w * vg.u[:, d]) - exact) <= 1e-13 * vol * np.max(np.abs(hi))
    # end nodes carry half weight along each axis
    w1 = (hi[0] - lo[0]) / 6
    assert abs(vg.w1d[0][0] - 0.5 * w1) <= 1e-15 and abs(vg.w1d[0][3] - w1) <= 1e-15


def test_trapezoid_integrates_a_gaussian_to_its_closed_form():
    vg = VelocityGrid((41, 41, 41), (-10.0,) * 3, (10.0,) * 3)
    g = np.exp(-0.5 * np.sum(vg.u ** 2, axis=1))
    assert abs(np.sum(vg.w * g) / (2 * np.pi) ** 1.5 - 1.0) <= 1e-12
    second = np.sum(vg.w * g * vg.u[:, 0] ** 2) / (2 * np.pi) ** 1.5
    assert abs(second - 1.0) <= 1e-12                          # unit variance


def test_node_ordering():
    vg = VelocityGrid((3, 4, 5), (0.0, 0.0, 0.0), (2.0, 3.0, 4.0))
    k1, k2, k3 = 2, 1, 3
    k = k1 + 3 * (k2 + 4 * k3)
    assert np.allclose(vg.u[k], [k1 * 1.0, k2 * 1.0, k3 * 1.0])
    assert np.isclose(vg.w[k], vg.w1d[0][k1] * vg.w1d[1][k2] * vg.w1d[2][k3])
