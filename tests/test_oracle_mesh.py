"""Pins of the box mesh (oracle/mesh.py): element and node numbering,
neighbours across periodic and closed faces, node placement and the affine
Jacobian (the tensor Gauss quadrature with it integrates the box's volume and
linear functions exactly)."""
import numpy as np

from oracle.fr import FR1D
from oracle.mesh import BoxMesh


def test_neighbours_wrap_on_periodic_axes_and_stop_at_closed_ones():
    m = BoxMesh((3, 4, 2), (0.0, 0.0, 0.0), (3.0, 2.0, 1.0), (True, False, True))
    e = m.index(0, 0, 1)
    assert m.coords(e) == (0, 0, 1)
    assert m.neighbour(e, 0, -1) == m.index(2, 0, 1)           # periodic wrap
    assert m.neighbour(e, 0, 1) == m.index(1, 0, 1)
    assert m.neighbour(e, 1, -1) == -1                         # closed axis
    assert m.neighbour(e, 1, 1) == m.index(0, 1, 1)
    assert m.neighbour(e, 2, 1) == m.index(0, 0, 0)            # periodic wrap in the third axis
    for d in range(3):
        for side in (-1, 1):
            nb = m.neighbours(d, side)
            inner = nb >= 0
            back = m.neighbours(d, -side)[nb[inner]]
            assert np.array_equal(back, np.arange(m.n_elem)[inner])   # the relation is symmetric


def test_node_placement_and_quadrature_of_the_affine_map():
    lo, hi = np.array([-1.0, 0.5, 2.0]), np.array([2.0, 1.5, 6.0])
    m = BoxMesh((3, 2, 4), lo, hi, (False, False, False))
    fr = FR1D(2)
    x = m.node_coords(fr.xi)                                   # [e, s, 3]
    q = 3
    e = m.index(1, 1, 2)
    s = 2 + q * (0 + q * 1)                                    # i1 = 2, i2 = 0, i3 = 1
    h = (hi - lo) / np.array([3, 2, 4])
    want = lo + (np.array([1, 1, 2]) + 0.5 * (fr.xi[[2, 0, 1]] + 1.0)) * h
    assert np.allclose(x[e, s], want, rtol=0, atol=1e-14)
    W = np.einsum("i,j,k->kji", fr.wq, fr.wq, fr.wq).reshape(-1)   # node s = i1 + q (i2 + q i3)
    vol = np.prod(hi - lo)
    assert abs(m.n_elem * m.jacobian() * np.sum(W) - vol) <= 1e-13 * vol
    lin = 2.0 + x @ np.array([0.3, -0.7, 0.2])
    exact = vol * (2.0 + np.dot([0.3, -0.7, 0.2], 0.5 * (lo + hi)))
    assert abs(m.jacobian() * np.sum(lin * W[None, :]) - exact) <= 1e-12 * abs(exact)
