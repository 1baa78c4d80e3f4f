"""Shock and sonic-surface quantities from the macroscopic fields (host).

The paper reads its flow fields through the shock standoff, the sonic
surface and the degree of non-equilibrium (section "Results").  bgk_macro
gives, per solution point, rho, U, theta, p, Mach, lambda, ||grad rho|| and
Kn_GLL; this module extracts from them, along lines of nodes that run
through the structured mesh in its first index direction (the radial
direction of the sphere O-grid, the shock-normal direction of the normal
shock):
  * mach_crossings: the points where Mach passes through 1 (linear
    interpolation between neighbouring nodes) -- the sonic surface;
  * max_gradient_position: the position of the largest ||grad rho|| on a
    line, refined by a parabola through it and its neighbours -- the shock;
  * max_slope_thickness: (rho_2 - rho_1) / max ||grad rho||, the classical
    shock thickness.
"""
import numpy as np


def first_axis_lines(wl):
    """Point indices of every node line running through the mesh along its
    first index direction: [n_lines, n1 (p+1)], nodes ordered by element and
    node index along that direction.  Lines are indexed by (e2, e3, i2, i3)."""
    q = wl.p + 1
    n1, n2, n3 = wl.mesh_n
    Ns = q ** 3
    lines = []
    for e3 in range(n3):
        for e2 in range(n2):
            for i3 in range(q):
                for i2 in range(q):
                    pts = [((e1 + n1 * (e2 + n2 * e3)) * Ns + i1 + q * (i2 + q * i3))
                           for e1 in range(n1) for i1 in range(q)]
                    lines.append(pts)
    return np.asarray(lines, dtype=np.int64)


def mach_crossings(x, mach, lines):
    """Mach = 1 crossings along each line: list of (line index, point [3]) by
    linear interpolation in the node positions x[P, 3]."""
    out = []
    for li, pts in enumerate(lines):
        sup = mach[pts] >= 1.0
        for j in np.nonzero(sup[:-1] != sup[1:])[0]:
            a, b = pts[j], pts[j + 1]
            t = (1.0 - mach[a]) / (mach[b] - mach[a])
            out.append((li, x[a] + t * (x[b] - x[a])))
    return out


def max_gradient_position(x, grad_rho, line):
    """Position along a line (arc length from its first node) and point of the
    largest ||grad rho||, refined by the vertex of the parabola through the
    maximum and its two neighbours (in arc length)."""
    pts = np.asarray(line)
    seg = np.linalg.norm(np.diff(x[pts], axis=0), axis=1)
    s = np.concatenate([[0.0], np.cumsum(seg)])
    g = grad_rho[pts]
    j = int(np.argmax(g))
    if 0 < j < len(pts) - 1:
        s0, s1, s2 = s[j - 1], s[j], s[j + 1]
        g0, g1, g2 = g[j - 1], g[j], g[j + 1]
        den = (s0 - s1) * (s0 - s2) * (s1 - s2)
        A = (s2 * (g1 - g0) + s1 * (g0 - g2) + s0 * (g2 - g1)) / den
        B = (s2 * s2 * (g0 - g1) + s1 * s1 * (g2 - g0) + s0 * s0 * (g1 - g2)) / den
        if A < 0.0:
            sv = -B / (2.0 * A)
            if s0 <= sv <= s2:
                k = j - 1 if sv < s1 else j
                t = (sv - s[k]) / (s[k + 1] - s[k])
                return sv, x[pts[k]] + t * (x[pts[k + 1]] - x[pts[k]])
    return s[j], x[pts[j]]


def max_slope_thickness(rho1, rho2, grad_rho_max):
    """(rho_2 - rho_1) / max ||grad rho||."""
    return abs(rho2 - rho1) / grad_rho_max
