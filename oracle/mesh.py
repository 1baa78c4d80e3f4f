"""Uniform affine hexahedral box mesh (test infrastructure).

Paper, section "Numerical method": the spatial domain is split into N_e
non-overlapping elements, each carrying N_s = (p+1)^3 solution nodes.  Here
the elements are the cells of a uniform n1 x n2 x n3 box, element
e = e1 + n1 (e2 + n2 e3), and each axis is either periodic or closed by
Dirichlet faces (a prescribed exterior state, section "Implementation &
problem setup": boundary conditions are weak, through the Riemann flux).

Solution node s = i1 + (p+1) (i2 + (p+1) i3) inside an element, so an array
f[..., e, s] reshaped to [..., Ne, p+1, p+1, p+1] is indexed [..., e, i3, i2, i1].
"""
import numpy as np


class BoxMesh:
    def __init__(self, n, lo, hi, periodic):
        self.n = tuple(int(v) for v in n)
        self.lo = np.asarray(lo, dtype=np.float64)
        self.hi = np.asarray(hi, dtype=np.float64)
        self.periodic = tuple(bool(v) for v in periodic)
        if any(v < 1 for v in self.n):
            raise ValueError("each mesh axis needs at least one element")
        self.h = (self.hi - self.lo) / np.asarray(self.n)
        self.n_elem = self.n[0] * self.n[1] * self.n[2]

    def index(self, e1, e2, e3):
        return e1 + self.n[0] * (e2 + self.n[1] * e3)

    def coords(self, e):
        n1, n2, _ = self.n
        return e % n1, (e // n1) % n2, e // (n1 * n2)

    def neighbour(self, e, d, side):
        """Element across face (d, side) of e, side -1 or +1; -1 if it is a boundary."""
        c = list(self.coords(e))
        c[d] += side
        if c[d] < 0 or c[d] >= self.n[d]:
            if not self.periodic[d]:
                return -1
            c[d] %= self.n[d]
        return self.index(*c)

    def neighbours(self, d, side):
        return np.array([self.neighbour(e, d, side) for e in range(self.n_elem)], dtype=np.int64)

    def node_coords(self, xi):
        """Physical coordinates x[e, s, 3] of the solution nodes given 1-D nodes xi."""
        q = len(xi)
        i3, i2, i1 = np.meshgrid(np.arange(q), np.arange(q), np.arange(q), indexing="ij")
        loc = [xi[i1.ravel()], xi[i2.ravel()], xi[i3.ravel()]]
        out = np.empty((self.n_elem, q ** 3, 3))
        for e in range(self.n_elem):
            c = self.coords(e)
            for d in range(3):
                corner = self.lo[d] + c[d] * self.h[d]
                out[e, :, d] = corner + 0.5 * (loc[d] + 1.0) * self.h[d]
        return out

    def jacobian(self):
        """|J_e| = prod_d h_d / 2 of the affine map from [-1,1]^3."""
        return float(np.prod(self.h / 2.0))
