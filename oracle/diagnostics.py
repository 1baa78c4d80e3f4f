"""Macroscopic post-processing of a solution (test infrastructure).

Paper, section "Results": the degree of non-equilibrium is measured by the
density gradient-length local Knudsen number
    Kn_GLL = lambda ||grad rho||_2 / rho,   lambda = (mu(theta)/rho) sqrt(pi/(2 theta)),
with continuum breakdown expected above 0.05; shock profiles and the sonic
surface use the macroscopic fields.  Per solution point this returns
    rho, U_1, U_2, U_3, theta, p, Mach = |U|/sqrt(gamma theta), lambda,
    ||grad rho||_2, Kn_GLL.

grad rho is the FR gradient of the nodal density polynomial (the paper
solves with FR; its gradient is not spelled out): along each reference
direction and line of nodes the corrected polynomial
    rho~(xi) = rho(xi) + (rho^I_L - rho_L) g_L(xi) + (rho^I_R - rho_R) g_R(xi)
matches the common interface values rho^I at both ends, with the central
common value rho^I = (rho^- + rho^+)/2 at interior faces, at a Dirichlet
face the average with the face state's density, and at a specular face the
element's own trace (its mirror image has the same density);
d/dx_d = (2/h_d) d/dxi_d.
"""
import numpy as np

from . import bgk


def macro_fields(problem, m):
    """[P, 10] fields of the moments m[P, 11] on problem's mesh (points e-major)."""
    gas, mesh, fr, q = problem.gas, problem.mesh, problem.fr, problem.q
    rho, U, E, theta, pres, Pi = bgk.macroscopic(m, gas)
    Ne = mesh.n_elem
    mach = np.sqrt(np.sum(U * U, axis=1) / (gas.gamma * theta))
    lam = gas.viscosity(theta) / rho * np.sqrt(np.pi / (2.0 * theta))
    r6 = rho.reshape(Ne, q, q, q)                    # [e, i3, i2, i1]
    grad = np.zeros((Ne, q, q, q, 3))
    for d in range(3):
        ax = 3 - d                                   # axis of i_{d+1}
        rl = np.moveaxis(r6, ax, -1)                 # line index last: [e, a, b, i]
        drl = np.einsum("ij,...j->...i", fr.D, rl)
        tr_L = np.einsum("j,...j->...", fr.l_minus, rl)
        tr_R = np.einsum("j,...j->...", fr.l_plus, rl)
        for side, tr_own, tr_other, dg in ((-1, tr_L, tr_R, fr.dgL), (1, tr_R, tr_L, fr.dgR)):
            nb = problem.nbr[(d, side)]
            outer = np.empty_like(tr_own)
            inner = nb >= 0
            outer[inner] = tr_other[nb[inner]]
            if np.any(~inner):
                # a specular face mirrors the element: its own trace is the exterior density
                outer[~inner] = (tr_own[~inner] if (d, side) in problem.specular
                                 else problem.dirichlet[(d, side)][0])
            common = 0.5 * (tr_own + outer)
            drl = drl + (common - tr_own)[..., None] * dg
        grad[..., d] = np.moveaxis((2.0 / mesh.h[d]) * drl, -1, ax)
    gnorm = np.sqrt(np.sum(grad * grad, axis=-1)).reshape(-1)
    kn = lam * gnorm / rho
    return np.stack([rho, U[:, 0], U[:, 1], U[:, 2], theta, pres, mach, lam, gnorm, kn], axis=1)


def macro_fields_curved(problem, m):
    """[P, 10] fields of the moments m[P, 11] on a curvilinear mesh (points
    e-major; problem is an oracle.curved.CurvedProblem).

    The gradient of the mapped density polynomial by the chain rule,
        grad rho = (1/J) sum_d S^d d rho~/d xi_d,   S^d = J grad xi_d,
    with d rho~/d xi_d the same FR-corrected line derivative as on the box
    (central common value at interior faces, the face state's density
    averaged in at a Dirichlet face).  At a diffuse wall or a collapsed face
    the common value is the element's own trace: neither prescribes a
    density.  On an affine box S^d/J = (2/h_d) e_d and this is macro_fields."""
    gas, mesh, fr, q = problem.gas, problem.mesh, problem.fr, problem.q
    rho, U, E, theta, pres, Pi = bgk.macroscopic(m, gas)
    Ne = mesh.n_elem
    mach = np.sqrt(np.sum(U * U, axis=1) / (gas.gamma * theta))
    lam = gas.viscosity(theta) / rho * np.sqrt(np.pi / (2.0 * theta))
    r6 = rho.reshape(Ne, q, q, q)                    # [e, i3, i2, i1]
    dxi = np.zeros((Ne, 3, q, q, q))
    for d in range(3):
        ax = 3 - d                                   # axis of i_{d+1}
        rl = np.moveaxis(r6, ax, -1)                 # line index last: [e, a, b, i]
        drl = np.einsum("ij,...j->...i", fr.D, rl)
        tr_L = np.einsum("j,...j->...", fr.l_minus, rl)
        tr_R = np.einsum("j,...j->...", fr.l_plus, rl)
        for side, tr_own, tr_other, dg in ((-1, tr_L, tr_R, fr.dgL), (1, tr_R, tr_L, fr.dgR)):
            nb = mesh.nbr[(d, side)]
            outer = np.empty_like(tr_own)
            inner = nb >= 0
            outer[inner] = tr_other[nb[inner]]
            if np.any(~inner):
                outer[~inner] = (problem.dirichlet[(d, side)][0] if (d, side) in problem.dirichlet
                                 else tr_own[~inner])
            common = 0.5 * (tr_own + outer)
            drl = drl + (common - tr_own)[..., None] * dg
        dxi[:, d] = np.moveaxis(drl, -1, ax)
    grad = np.einsum("ednabc,edabc->eabcn", mesh.S, dxi) / mesh.J[..., None]
    gnorm = np.sqrt(np.sum(grad * grad, axis=-1)).reshape(-1)
    kn = lam * gnorm / rho
    return np.stack([rho, U[:, 0], U[:, 1], U[:, 2], theta, pres, mach, lam, gnorm, kn], axis=1)
