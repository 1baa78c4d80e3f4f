"""1-D flux-reconstruction operators (test infrastructure; see oracle/__init__).

Paper, section "Numerical method": the solution in each element is a nodal
polynomial of degree p on N_s solution nodes, and the flux is corrected with
functions h that recover the nodal discontinuous Galerkin method (Huynh 2007).
On tensor-product (hex) elements every operator is a tensor product of the
1-D operators built here.  Solution nodes are the p+1 Gauss--Legendre points
on [-1, 1]; the flux nodes of a face are the face's tensor Gauss--Legendre
points, so every flux node sits at the end of one line of solution nodes.
"""
import numpy as np


def legendre(n, x):
    """P_n(x) and P_n'(x) by Bonnet's three-term recurrence.

    (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1};  P'_{k+1} = P'_{k-1} + (2k+1) P_k.
    """
    x = np.asarray(x, dtype=np.float64)
    p_prev, p = np.ones_like(x), x.copy()
    dp_prev, dp = np.zeros_like(x), np.ones_like(x)
    if n == 0:
        return p_prev, dp_prev
    for k in range(1, n):
        p_next = ((2 * k + 1) * x * p - k * p_prev) / (k + 1)
        dp_next = dp_prev + (2 * k + 1) * p
        p_prev, p = p, p_next
        dp_prev, dp = dp, dp_next
    return p, dp


def gauss_legendre(n):
    """Nodes and weights of the n-point Gauss--Legendre rule on [-1, 1].

    Nodes are the roots of P_n, found by Newton's method from Tricomi's
    estimate cos(pi (i + 3/4) / (n + 1/2)); weights 2 / ((1 - x^2) P_n'(x)^2).
    """
    i = np.arange(n, dtype=np.float64)
    x = np.cos(np.pi * (i + 0.75) / (n + 0.5))
    for _ in range(100):
        p, dp = legendre(n, x)
        dx = p / dp
        x = x - dx
        if np.max(np.abs(dx)) < 1e-16:
            break
    p, dp = legendre(n, x)
    w = 2.0 / ((1.0 - x * x) * dp * dp)
    order = np.argsort(x)
    return x[order], w[order]


def lagrange_values(xi, x):
    """l_j(x) for the Lagrange basis on nodes xi; returns [len(x), len(xi)]."""
    xi = np.asarray(xi, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = len(xi)
    out = np.ones((len(x), n))
    for j in range(n):
        for m in range(n):
            if m != j:
                out[:, j] *= (x - xi[m]) / (xi[j] - xi[m])
    return out


def lagrange_derivatives(xi, x):
    """l_j'(x) = sum_{m != j} 1/(xi_j - xi_m) prod_{r != j, m} (x - xi_r)/(xi_j - xi_r)."""
    xi = np.asarray(xi, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = len(xi)
    out = np.zeros((len(x), n))
    for j in range(n):
        for m in range(n):
            if m == j:
                continue
            term = np.full(len(x), 1.0 / (xi[j] - xi[m]))
            for r in range(n):
                if r != j and r != m:
                    term *= (x - xi[r]) / (xi[j] - xi[r])
            out[:, j] += term
    return out


def correction_left(p, x):
    """g_L(x) = ((-1)^(p+1) / 2) (P_{p+1}(x) - P_p(x)) and its derivative.

    The right Radau polynomial of degree p+1: g_L(-1) = 1, g_L(1) = 0.  With
    solution nodes at the Gauss points this choice makes FR identical to the
    nodal DG method, which is the recovery the paper asks of h.
    """
    a, da = legendre(p + 1, x)
    b, db = legendre(p, x)
    s = 0.5 * (-1.0) ** (p + 1)
    return s * (a - b), s * (da - db)


def correction_right(p, x):
    """g_R(x) = g_L(-x) = (P_{p+1}(x) + P_p(x)) / 2 and its derivative."""
    a, da = legendre(p + 1, x)
    b, db = legendre(p, x)
    return 0.5 * (a + b), 0.5 * (da + db)


class FR1D:
    """All 1-D operators of an order-p FR element on Gauss--Legendre nodes.

    Attributes
    ----------
    xi, wq    solution nodes and quadrature weights (p+1)
    D         D[i, j] = l_j'(xi_i), the nodal derivative
    l_minus   l_j(-1), interpolation to the left flux node of a line
    l_plus    l_j(+1), interpolation to the right flux node of a line
    dgL, dgR  g_L'(xi_i), g_R'(xi_i), the correction-function derivatives
    """

    def __init__(self, p):
        if p < 0:
            raise ValueError("order p must be >= 0")
        self.p = p
        self.xi, self.wq = gauss_legendre(p + 1)
        self.D = lagrange_derivatives(self.xi, self.xi)
        self.l_minus = lagrange_values(self.xi, -1.0)[0]
        self.l_plus = lagrange_values(self.xi, 1.0)[0]
        self.dgL = correction_left(p, self.xi)[1]
        self.dgR = correction_right(p, self.xi)[1]

