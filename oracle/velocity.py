"""Discrete velocity grid and trapezoid weights (test infrastructure).

Paper, section "Numerical method": the velocity domain is a box discretised by
a uniform Cartesian grid of nodes; the discrete integration operator M has
strictly positive entries and is the trapezoidal rule on the uniform grid.

Ordering: velocity node k = k1 + n1 (k2 + n2 k3), the u1 index fastest, so a
velocity array reshaped C-order to [n3, n2, n1] is indexed [k3, k2, k1].
"""
import numpy as np


class VelocityGrid:
    def __init__(self, n, lo, hi, weights=None):
        self.n = tuple(int(v) for v in n)
        self.lo = np.asarray(lo, dtype=np.float64)
        self.hi = np.asarray(hi, dtype=np.float64)
        if any(v < 2 for v in self.n):
            raise ValueError("each velocity axis needs at least 2 nodes")
        self.h = (self.hi - self.lo) / (np.asarray(self.n) - 1)
        self.axes = [self.lo[d] + np.arange(self.n[d]) * self.h[d] for d in range(3)]
        # 1-D trapezoid weights h {1/2, 1, ..., 1, 1/2}
        self.w1d = []
        for d in range(3):
            w = np.full(self.n[d], self.h[d])
            w[0] *= 0.5
            w[-1] *= 0.5
            self.w1d.append(w)
        n1, n2, n3 = self.n
        k3, k2, k1 = np.meshgrid(np.arange(n3), np.arange(n2), np.arange(n1), indexing="ij")
        k1, k2, k3 = k1.ravel(), k2.ravel(), k3.ravel()
        # u[k, d]: the 3 components of velocity node k
        self.u = np.stack([self.axes[0][k1], self.axes[1][k2], self.axes[2][k3]], axis=1)
        if weights is None:
            self.w = self.w1d[0][k1] * self.w1d[1][k2] * self.w1d[2][k3]
        else:
            self.w = np.asarray(weights, dtype=np.float64).copy()
            if self.w.shape != (self.size,) or np.any(self.w <= 0):
                raise ValueError("weights must be strictly positive, one per node")

    def index3(self):
        """[k1, k2, k3] index arrays of every node k = k1 + n1 (k2 + n2 k3)."""
        k = np.arange(self.size)
        return [k % self.n[0], (k // self.n[0]) % self.n[1], k // (self.n[0] * self.n[1])]

    @property
    def size(self):
        return self.n[0] * self.n[1] * self.n[2]

    @property
    def volume(self):
        return float(np.prod(self.hi - self.lo))
