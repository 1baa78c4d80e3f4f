"""BGK source of the reduced F/G system, with the conservative Q' solve.

Test infrastructure (see oracle/__init__).  Paper, section "Governing
equations" and the discrete-velocity part of "Numerical method":

* moments Q = (rho, rho U, E) of f against the collision invariants
  psi = [1, u, u.u/2 + zeta]; with the reduced distributions F = int f dzeta
  and G = int zeta f dzeta this reads rho = sum w F, rho U = sum w u F,
  E = sum w (u.u/2) F + sum w G  (the momentum row of that equation prints
  u.u; only the vector u is dimensionally consistent and is used);
* primitives: P = (gamma - 1)(E - rho U.U/2), theta = P / rho, with
  gamma = (5 + delta)/(3 + delta) (3 translational + delta internal degrees
  of freedom; the paper names gamma but does not write it as a function of
  delta);
* pressure tensor Pi_ij = int F (u_i - U_i)(u_j - U_j) du;
* ES temperature tensor T = theta/Pr I + (1 - 1/Pr) Pi/rho;
* collision time tau = mu / (Pr P), Sutherland
  mu = mu_ref (theta/theta_ref)^(3/2) (theta_ref + theta_S)/(theta + theta_S);
* ES-BGK equilibrium g_u = rho / sqrt(det(2 pi T)) exp(-(u-U)^T T^-1 (u-U)/2),
  the G equilibrium (delta theta / 2) g_u, source (g - f)/tau per component;
* discrete compatibility: the equilibrium actually used is g(Q'), the
  Gaussian around a modified state whose discrete moments under the
  trapezoid weights equal those of f; found by Newton's method.

Reading of the modified state for ES-BGK and delta > 0 (the paper gives the
d+2 dimensional system only in words): the unknowns are q' = (rho', U',
theta'); Pi/rho is that of f and held fixed; T'(theta') = theta'/Pr I +
(1 - 1/Pr) Pi/rho; the equations are
    sum_k w_k g_k(q')                            = rho
    sum_k w_k u_k g_k(q')                        = rho U
    sum_k w_k (|u_k|^2/2 + delta theta'/2) g_k(q') = E,
so mass, momentum and total energy of (F, G) are conserved exactly by the
source.  tau is computed from the state of f (not of Q').

Tensor variant (the paper's remark that ES-BGK may need a nonlinear solve of
marginally higher dimension when the velocity grid lacks symmetry, section
"Numerical method"; a reading, monatomic gas): the equilibrium is the
discrete Gaussian g = exp(b0 + b.c + sum_{i<=j} b_ij c_i c_j), c = u - U, whose
discrete moments against phi = (1, c, c_i c_j (i <= j)) equal (rho, 0, rho T)
with T the ES target tensor above: 10 unknowns and 10 equations.  The trace
of the second-moment rows is the energy, so mass, momentum and energy are
conserved, and the discrete stress of g equals rho T exactly (the d+2 solve
above matches only its trace).  Newton on the natural parameters b, whose
Jacobian sum w phi phi^T g is symmetric positive definite (the equations are
the gradient of the strictly convex sum w exp(b.phi) - b.(rho, 0, rho T)),
so the solution is unique.

Moment slots (11, shared with the C-ABI layout of raw moments):
    0: sum w F      1..3: sum w u_d F     4..6: sum w u_d^2 F
    7: sum w u1 u2 F  8: sum w u1 u3 F  9: sum w u2 u3 F   10: sum w G
"""
import numpy as np

PAIRS = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]


class Gas:
    """Gas parameters: internal dof delta, Prandtl Pr, Sutherland law.

    theta_S < 0 selects a constant viscosity mu = mu_ref.
    """

    def __init__(self, delta=0.0, Pr=1.0, mu_ref=0.1, theta_ref=1.0, theta_S=-1.0, es_tensor=False):
        if delta < 0:
            raise ValueError("delta must be >= 0")
        if es_tensor and delta > 0:
            raise ValueError("the tensor variant is for a monatomic gas (delta = 0)")
        self.es_tensor = bool(es_tensor)
        self.delta = float(delta)
        self.Pr = float(Pr)
        self.mu_ref = float(mu_ref)
        self.theta_ref = float(theta_ref)
        self.theta_S = float(theta_S)

    @property
    def gamma(self):
        return (5.0 + self.delta) / (3.0 + self.delta)

    @property
    def n_comp(self):
        return 2 if self.delta > 0 else 1

    def viscosity(self, theta):
        if self.theta_S < 0:
            return np.full_like(np.asarray(theta, dtype=np.float64), self.mu_ref)
        r = theta / self.theta_ref
        return self.mu_ref * r ** 1.5 * (self.theta_ref + self.theta_S) / (theta + self.theta_S)


def raw_moments(F, G, vg):
    """Raw moments m[P, 11] of F[Nu, P] (and G[Nu, P] or None) under weights w."""
    w, u = vg.w, vg.u
    P = F.shape[1]
    m = np.zeros((P, 11))
    m[:, 0] = np.sum(w[:, None] * F, axis=0)
    for d in range(3):
        m[:, 1 + d] = np.sum((w * u[:, d])[:, None] * F, axis=0)
    for j, (a, b) in enumerate(PAIRS):
        m[:, 4 + j] = np.sum((w * u[:, a] * u[:, b])[:, None] * F, axis=0)
    if G is not None:
        m[:, 10] = np.sum(w[:, None] * G, axis=0)
    return m


def macroscopic(m, gas):
    """rho, U[P,3], E, theta, P, Pi[P,3,3] from raw moments (section Governing equations)."""
    rho = m[:, 0]
    U = m[:, 1:4] / rho[:, None]
    E = 0.5 * (m[:, 4] + m[:, 5] + m[:, 6]) + m[:, 10]
    pres = (gas.gamma - 1.0) * (E - 0.5 * rho * np.sum(U * U, axis=1))
    theta = pres / rho
    Pi = np.zeros((len(rho), 3, 3))
    for j, (a, b) in enumerate(PAIRS):
        Pi[:, a, b] = m[:, 4 + j] - rho * U[:, a] * U[:, b]
        Pi[:, b, a] = Pi[:, a, b]
    return rho, U, E, theta, pres, Pi


def collision_time(theta, pres, gas):
    """tau = mu(theta) / (Pr P)."""
    return gas.viscosity(theta) / (gas.Pr * pres)


def temperature_tensor(theta, Pi_over_rho, Pr):
    """T = theta/Pr I + (1 - 1/Pr) Pi/rho, batched over points."""
    T = (1.0 - 1.0 / Pr) * Pi_over_rho
    for d in range(3):
        T[:, d, d] += theta / Pr
    return T


def gaussian(u, rho, U, T):
    """g_u[Nu, P] = rho / sqrt(det(2 pi T)) exp(-(u-U)^T T^-1 (u-U) / 2)."""
    A = np.linalg.inv(T)                                   # [P,3,3]
    c = u[:, None, :] - U[None, :, :]                      # [Nu,P,3]
    quad = np.einsum("kpi,pij,kpj->kp", c, A, c)
    norm = rho / np.sqrt(np.linalg.det(2.0 * np.pi * T))
    return norm[None, :] * np.exp(-0.5 * quad)


def _spd(T):
    """Leading principal minors of symmetric 3x3 matrices all positive."""
    a = T[:, 0, 0]
    b = T[:, 0, 0] * T[:, 1, 1] - T[:, 0, 1] * T[:, 1, 0]
    c = np.linalg.det(T)
    return (a > 0) & (b > 0) & (c > 0)


def scaled_residual(R, rho, theta, E):
    """max(|R_rho|/rho, |R_rhoU|_inf/(rho sqrt(theta)), |R_E|/E) per point."""
    return np.maximum.reduce([
        np.abs(R[:, 0]) / rho,
        np.max(np.abs(R[:, 1:4]), axis=1) / (rho * np.sqrt(theta)),
        np.abs(R[:, 4]) / np.abs(E),
    ])


def compatibility_residual(x, Q, B, gas, vg):
    """R(q') = sum_k w_k psi~_k g_k(q') - Q and the analytic Jacobian dR/dq'.

    x[P,5] = (rho', U'_1..3, theta'); B = (1 - 1/Pr) Pi/rho of f.
    """
    w, u, Pr, delta = vg.w, vg.u, gas.Pr, gas.delta
    rho_p, U_p, th_p = x[:, 0], x[:, 1:4], x[:, 4]
    T = B.copy()
    for d in range(3):
        T[:, d, d] += th_p / Pr
    A = np.linalg.inv(T)
    g = gaussian(u, rho_p, U_p, T)                          # [Nu,P]
    c = u[:, None, :] - U_p[None, :, :]                     # [Nu,P,3]
    Ac = np.einsum("pij,kpj->kpi", A, c)                    # [Nu,P,3]
    # psi~ rows: 1, u_1..3, |u|^2/2 + delta theta'/2
    psi = np.empty((5,) + g.shape)
    psi[0] = 1.0
    for d in range(3):
        psi[1 + d] = u[:, d][:, None]
    psi[4] = 0.5 * np.sum(u * u, axis=1)[:, None] + 0.5 * delta * th_p[None, :]
    wg = w[:, None] * g
    R = np.stack([np.sum(psi[i] * wg, axis=0) for i in range(5)], axis=1) - Q
    # dg/dq' columns
    dg = np.empty((5,) + g.shape)
    dg[0] = g / rho_p[None, :]
    for d in range(3):
        dg[1 + d] = g * Ac[:, :, d]
    trA = np.trace(A, axis1=1, axis2=2)
    dg[4] = g * (np.sum(Ac * Ac, axis=2) - trA[None, :]) / (2.0 * Pr)
    J = np.empty((len(rho_p), 5, 5))
    for i in range(5):
        for j in range(5):
            J[:, i, j] = np.sum(w[:, None] * psi[i] * dg[j], axis=0)
    J[:, 4, 4] += 0.5 * delta * np.sum(wg, axis=0)
    return R, J


def solve_qprime(m, gas, vg, guess=None, tol=1e-13, max_iter=50):
    """Newton's method for the modified state q' of every point.

    m[P,11] raw moments of f.  guess[P,5] optional initial q'
    (default: the primitive state q = (rho, U, theta) of f).
    Returns (qp[P,5], iters[P], converged[P], final scaled residual[P]).
    A step is halved while it would make rho' or theta' non-positive or T'
    not positive definite.
    """
    rho, U, E, theta, pres, Pi = macroscopic(m, gas)
    Q = np.concatenate([rho[:, None], m[:, 1:4], E[:, None]], axis=1)
    B = (1.0 - 1.0 / gas.Pr) * Pi / rho[:, None, None]
    if guess is None:
        x = np.concatenate([rho[:, None], U, theta[:, None]], axis=1)
    else:
        x = np.array(guess, dtype=np.float64, copy=True)
    P = len(rho)
    iters = np.zeros(P, dtype=np.int64)
    done = np.zeros(P, dtype=bool)
    res = np.full(P, np.inf)
    for it in range(max_iter + 1):
        act = np.nonzero(~done)[0]
        if len(act) == 0:
            break
        R, J = compatibility_residual(x[act], Q[act], B[act], gas, vg)
        r = scaled_residual(R, rho[act], theta[act], E[act])
        res[act] = r
        conv = r <= tol
        done[act[conv]] = True
        if it == max_iter:
            break
        upd = act[~conv]
        if len(upd) == 0:
            break
        dx = np.linalg.solve(J[~conv], -R[~conv][:, :, None])[:, :, 0]
        lam = np.ones(len(upd))
        for _ in range(60):
            xt = x[upd] + lam[:, None] * dx
            T = B[upd].copy()
            for d in range(3):
                T[:, d, d] += xt[:, 4] / gas.Pr
            ok = (xt[:, 0] > 0) & (xt[:, 4] > 0) & _spd(T)
            if np.all(ok):
                break
            lam = np.where(ok, lam, 0.5 * lam)
        x[upd] = x[upd] + lam[:, None] * dx
        iters[upd] += 1
    return x, iters, done, res


# phi = (1, c1, c2, c3, c1^2, c2^2, c3^2, c1 c2, c1 c3, c2 c3) as exponents (p1, p2, p3)
TENSOR_PHI = [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (2, 0, 0), (0, 2, 0), (0, 0, 2),
              (1, 1, 0), (1, 0, 1), (0, 1, 1)]


def _phi(c):
    """phi[10, Nu, P] of c[Nu, P, 3]."""
    return np.stack([c[..., 0] ** a * c[..., 1] ** b * c[..., 2] ** d for a, b, d in TENSOR_PHI])


def tensor_targets(m, gas):
    """(rho, 0, rho T_ij) per point [P, 10] in the frame c = u - U, the centre U."""
    rho, U, E, theta, pres, Pi = macroscopic(m, gas)
    T = temperature_tensor(theta, Pi / rho[:, None, None], gas.Pr)
    t = np.zeros((len(rho), 10))
    t[:, 0] = rho
    for a, (i, j) in enumerate(PAIRS):
        t[:, 4 + a] = rho * T[:, i, j]
    return t, U, rho, theta


def tensor_residual(b, t, U, vg):
    """R = sum_k w phi g - t and J = sum_k w phi phi^T g for natural parameters b[P, 10]."""
    c = vg.u[:, None, :] - U[None, :, :]                  # [Nu, P, 3]
    ph = _phi(c)                                         # [10, Nu, P]
    g = np.exp(np.einsum("pa,akp->kp", b, ph))
    wg = vg.w[:, None] * g
    R = np.einsum("akp,kp->pa", ph, wg) - t
    J = np.einsum("akp,bkp,kp->pab", ph, ph, wg)
    return R, J, g


def _tensor_params(b):
    """(A = T'^-1 [P,3,3], spd[P]) of the quadratic part of b."""
    A = np.zeros((len(b), 3, 3))
    for a, (i, j) in enumerate(PAIRS):
        if i == j:
            A[:, i, i] = -2.0 * b[:, 4 + a]
        else:
            A[:, i, j] = A[:, j, i] = -b[:, 4 + a]
    return A, _spd(A)


def solve_qprime_tensor(m, gas, vg, tol=1e-13, max_iter=50):
    """Newton on the natural parameters of the tensor variant, from the
    continuous Gaussian (rho, U, T) of f.  Returns (b[P,10], U[P,3], iters,
    converged, final scaled residual); the scaled residual is
    max(|R_0|/rho, |R_c|_inf/(rho sqrt(theta)), |R_cc|_inf/(rho theta)).  A
    step is halved while the quadratic form would not be negative definite."""
    t, U, rho, theta = tensor_targets(m, gas)
    T = np.zeros((len(rho), 3, 3))
    for a, (i, j) in enumerate(PAIRS):
        T[:, i, j] = T[:, j, i] = t[:, 4 + a] / rho
    A = np.linalg.inv(T)
    b = np.zeros((len(rho), 10))
    b[:, 0] = np.log(rho / np.sqrt(np.linalg.det(2.0 * np.pi * T)))
    for a, (i, j) in enumerate(PAIRS):
        b[:, 4 + a] = -0.5 * A[:, i, i] if i == j else -A[:, i, j]
    P = len(rho)
    iters = np.zeros(P, dtype=np.int64)
    done = np.zeros(P, dtype=bool)
    res = np.full(P, np.inf)
    for it in range(max_iter + 1):
        act = np.nonzero(~done)[0]
        if len(act) == 0:
            break
        R, J, _ = tensor_residual(b[act], t[act], U[act], vg)
        r = np.maximum.reduce([np.abs(R[:, 0]) / rho[act],
                               np.max(np.abs(R[:, 1:4]), axis=1) / (rho[act] * np.sqrt(theta[act])),
                               np.max(np.abs(R[:, 4:]), axis=1) / (rho[act] * theta[act])])
        res[act] = r
        conv = r <= tol
        done[act[conv]] = True
        if it == max_iter:
            break
        upd = act[~conv]
        if len(upd) == 0:
            break
        db = np.linalg.solve(J[~conv], -R[~conv][:, :, None])[:, :, 0]
        lam = np.ones(len(upd))
        for _ in range(60):
            _, ok = _tensor_params(b[upd] + lam[:, None] * db)
            if np.all(ok):
                break
            lam = np.where(ok, lam, 0.5 * lam)
        b[upd] = b[upd] + lam[:, None] * db
        iters[upd] += 1
    return b, U, iters, done, res


def tensor_equilibrium(b, U, vg):
    """g[Nu, P] = exp(b . phi(u - U))."""
    c = vg.u[:, None, :] - U[None, :, :]
    return np.exp(np.einsum("pa,akp->kp", b, _phi(c)))


def equilibrium(qp, m, gas, vg):
    """F_eq = g_u(q'), G_eq = (delta theta'/2) g_u(q'), each [Nu, P]."""
    rho, U, E, theta, pres, Pi = macroscopic(m, gas)
    B = (1.0 - 1.0 / gas.Pr) * Pi / rho[:, None, None]
    T = B.copy()
    for d in range(3):
        T[:, d, d] += qp[:, 4] / gas.Pr
    g = gaussian(vg.u, qp[:, 0], qp[:, 1:4], T)
    G_eq = 0.5 * gas.delta * qp[:, 4][None, :] * g if gas.n_comp == 2 else None
    return g, G_eq


def bgk_source(F, G, gas, vg, guess=None, tol=1e-13, max_iter=50):
    """S = (g' - f) / tau for F (and G).  F, G are [Nu, P].

    Returns (S_F, S_G or None, info) with info = dict(qp, iters, converged, tau, m).
    """
    m = raw_moments(F, G, vg)
    rho, U, E, theta, pres, Pi = macroscopic(m, gas)
    tau = collision_time(theta, pres, gas)
    if gas.es_tensor:
        b, Uc, iters, conv, res = solve_qprime_tensor(m, gas, vg, tol=tol, max_iter=max_iter)
        g = tensor_equilibrium(b, Uc, vg)
        S_F = (g - F) / tau[None, :]
        info = dict(b=b, iters=iters, converged=conv, residual=res, tau=tau, m=m)
        return S_F, None, info
    qp, iters, conv, res = solve_qprime(m, gas, vg, guess=guess, tol=tol, max_iter=max_iter)
    g, Gg = equilibrium(qp, m, gas, vg)
    S_F = (g - F) / tau[None, :]
    S_G = (Gg - G) / tau[None, :] if G is not None else None
    info = dict(qp=qp, iters=iters, converged=conv, residual=res, tau=tau, m=m)
    return S_F, S_G, info


def maxwellian(vg, rho, U, theta):
    """Isotropic Maxwellian sampled at the velocity nodes: [Nu, P] (T = theta I)."""
    T = np.zeros((len(rho), 3, 3))
    for d in range(3):
        T[:, d, d] = theta
    return gaussian(vg.u, np.asarray(rho, dtype=np.float64), np.asarray(U, dtype=np.float64), T)
