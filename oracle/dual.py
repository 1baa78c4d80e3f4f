"""Second, independent route to the Pr = 1 discrete Maxwellian (test pin only).

Paper, "Numerical method": for BGK (Pr = 1, delta = 0) Mieussens' modified
equilibrium is the unique function of the form g = exp(alpha . psi),
psi = [1, u, |u|^2/2], whose discrete moments equal those of f; it is also
the minimiser of the discrete entropy under those constraints.  Its
Lagrange multipliers minimise the strictly convex dual

    Phi(alpha) = sum_k w_k exp(alpha . psi_k) - alpha . Q,

whose gradient is the compatibility residual and whose Hessian
sum_k w_k psi_k psi_k^T g_k is positive definite.  This module minimises Phi
with a damped (Armijo backtracking) Newton iteration, point by point.  It
shares nothing with the primitive-variable Newton of oracle.bgk except the
data it is given, so agreement of the two pins the Q' solve.
"""
import numpy as np


def discrete_maxwellian_dual(Q, vg, tol=1e-15, max_iter=200):
    """g[Nu] = exp(alpha . psi) with sum w psi g = Q, for one point.

    Q = (rho, rho U_1..3, E) with E = sum w |u|^2/2 f (delta = 0).
    Returns (g, alpha, iterations).
    """
    u, w = vg.u, vg.w
    psi = np.concatenate([np.ones((len(w), 1)), u, 0.5 * np.sum(u * u, axis=1)[:, None]], axis=1)
    rho = Q[0]
    U = Q[1:4] / rho
    theta = (2.0 / 3.0) * (Q[4] - 0.5 * rho * U @ U) / rho
    alpha = np.concatenate([[np.log(rho / (2 * np.pi * theta) ** 1.5) - U @ U / (2 * theta)],
                            U / theta, [-1.0 / theta]])

    def phi(a):
        return np.sum(w * np.exp(psi @ a)) - a @ Q

    scale = np.array([rho, rho * np.sqrt(theta), rho * np.sqrt(theta), rho * np.sqrt(theta), Q[4]])
    it = 0
    for it in range(max_iter):
        g = np.exp(psi @ alpha)
        grad = psi.T @ (w * g) - Q
        if np.max(np.abs(grad) / scale) <= tol:
            break
        H = (psi * (w * g)[:, None]).T @ psi
        step = -np.linalg.solve(H, grad)
        t, f0, slope = 1.0, phi(alpha), grad @ step
        while phi(alpha + t * step) > f0 + 1e-4 * t * slope and t > 1e-12:
            t *= 0.5
        new = alpha + t * step
        if np.array_equal(new, alpha):
            break
        alpha = new
    return np.exp(psi @ alpha), alpha, it
