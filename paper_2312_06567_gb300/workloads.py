"""Seeded synthetic workloads: problem definitions and input generators.

This module holds problem data only -- sizes, gas parameters, the analytic
macroscopic initial fields and seeded random test states -- and none of the
solver's arithmetic.  It is the one module that both the CUDA path's callers
and the CPU oracle's tests draw inputs from.

No public dataset, mesh or checkpoint stands behind these problems; they are
analytic stand-ins with the structure of the paper's workloads (hex elements,
uniform Cartesian velocity grids, Maxwellian initial data, a normal shock for
the hypersonic physics).

Layout conventions (shared by every caller):
  element  e = e1 + n1 (e2 + n2 e3)
  node     s = i1 + (p+1) (i2 + (p+1) i3)   (Gauss--Legendre nodes per axis)
  velocity k = k1 + n1 (k2 + n2 k3)         (uniform nodes per axis)
  state    f[c][k][e][s], c = 0 for F, 1 for G (delta > 0 only)
"""
import math
from dataclasses import dataclass, field

import numpy as np
from numpy.polynomial.legendre import leggauss


def mu_from_knudsen(kn, theta_ref=1.0, rho_ref=1.0, length=1.0):
    """mu_ref from a Knudsen number via the hard-sphere-like mean free path
    lambda = (mu/rho) sqrt(pi/(2 theta)) used by the paper's Kn_GLL."""
    return kn * rho_ref * length * math.sqrt(2.0 * theta_ref / math.pi)


def normal_shock_states(mach, gamma, rho1=1.0, theta1=1.0):
    """Upstream and downstream (rho, u, theta) of a stationary normal shock
    (Rankine--Hugoniot relations; sound speed sqrt(gamma theta))."""
    u1 = mach * math.sqrt(gamma * theta1)
    m2 = mach * mach
    rho2 = rho1 * (gamma + 1.0) * m2 / ((gamma - 1.0) * m2 + 2.0)
    p1 = rho1 * theta1
    p2 = p1 * (1.0 + 2.0 * gamma / (gamma + 1.0) * (m2 - 1.0))
    u2 = u1 * rho1 / rho2
    return (rho1, u1, theta1), (rho2, u2, p2 / rho2)


@dataclass
class Workload:
    name: str
    mesh_n: tuple
    mesh_lo: tuple
    mesh_hi: tuple
    periodic: tuple
    p: int
    vel_n: tuple
    vel_lo: tuple
    vel_hi: tuple
    delta: float
    Pr: float
    mu_ref: float
    theta_ref: float
    theta_S: float
    cfl: float
    steps: int
    init: object = None                     # x[..., 3] -> (rho, U[..., 3], theta)
    dirichlet: dict = field(default_factory=dict)   # {(d, side): (rho, U(3), theta)}
    specular: tuple = ()                    # ((d, side), ...) specular (symmetry) faces
    # curvilinear meshes: mapping(t[..., 3]) -> x[..., 3] of the normalised lattice
    # coordinates t in [0, 1]^3 (element e1 spans t1 in [e1/n1, (e1+1)/n1]); None = the
    # uniform box mesh_lo..mesh_hi
    mapping: object = None
    diffuse: dict = field(default_factory=dict)     # {(d, side): (U_w(3), theta_w)} diffuse walls
    closed: tuple = ()                      # ((d, side), ...) collapsed faces (no flux)
    h_min_override: float = None            # smallest node spacing of a curvilinear mesh
    es_tensor: bool = False                 # ES equilibrium matching the full target stress (delta = 0)

    @property
    def n_elem(self):
        return self.mesh_n[0] * self.mesh_n[1] * self.mesh_n[2]

    @property
    def n_sol(self):
        return (self.p + 1) ** 3

    @property
    def n_vel(self):
        return self.vel_n[0] * self.vel_n[1] * self.vel_n[2]

    @property
    def n_comp(self):
        return 2 if self.delta > 0 else 1

    @property
    def dof(self):
        return self.n_elem * self.n_sol * self.n_vel

    def h_min(self):
        if self.h_min_override is not None:
            return self.h_min_override
        return min((self.mesh_hi[d] - self.mesh_lo[d]) / self.mesh_n[d] for d in range(3))

    def u_max(self):
        return max(max(abs(self.vel_lo[d]), abs(self.vel_hi[d])) for d in range(3))

    def dt(self):
        """dt = CFL h_min / (u_max (2p+1))."""
        return self.cfl * self.h_min() / (self.u_max() * (2 * self.p + 1))

    def replace(self, **kw):
        d = dict(self.__dict__)
        d.update(kw)
        return Workload(**d)


# ---- analytic initial fields ---------------------------------------------
def _init_sine_density(x):
    rho = 1.0 + 0.1 * np.sin(2.0 * np.pi * x[..., 0])
    return rho, np.zeros(x.shape), np.ones(x.shape[:-1])


def _init_taylor_green(x, mach=0.1):
    X, Y, Z = x[..., 0], x[..., 1], x[..., 2]
    U = np.stack([mach * np.sin(X) * np.cos(Y) * np.cos(Z),
                  -mach * np.cos(X) * np.sin(Y) * np.cos(Z),
                  np.zeros_like(X)], axis=-1)
    P = 1.0 + mach * mach / 16.0 * (np.cos(2 * X) + np.cos(2 * Y)) * (np.cos(2 * Z) + 2.0)
    theta = np.ones_like(X)
    return P / theta, U, theta


def _shock_init(width, s1, s2):
    def init(x):
        blend = 0.5 * (1.0 + np.tanh(x[..., 0] / width))
        rho = s1[0] + (s2[0] - s1[0]) * blend
        ux = s1[1] + (s2[1] - s1[1]) * blend
        theta = s1[2] + (s2[2] - s1[2]) * blend
        U = np.zeros(x.shape)
        U[..., 0] = ux
        return rho, U, theta
    return init


THETA_S_RATIO = 110.4 / 203.0      # Sutherland 110.4 K over a 203 K freestream


def periodic_sine_box():
    """Small plain-method case: [0,1]^3, 4^3 hex, p=1, 8^3 velocities on [-6,6]^3,
    BGK (Pr=1), monatomic, Kn=0.1, rho = 1 + 0.1 sin(2 pi x), U = 0, theta = 1."""
    return Workload("periodic_sine_box_4x4x4_p1_u8", (4, 4, 4), (0, 0, 0), (1, 1, 1),
                    (True, True, True), 1, (8, 8, 8), (-6, -6, -6), (6, 6, 6),
                    0.0, 1.0, mu_from_knudsen(0.1), 1.0, THETA_S_RATIO, 0.1, 10,
                    init=_init_sine_density)


def taylor_green_box():
    """Throughput case: [0,2pi]^3, 16^3 hex, p=3, 24^3 velocities on [-5,5]^3,
    ES-BGK Pr=2/3, monatomic, Kn=0.01, Taylor--Green field at M=0.1, theta=1."""
    two_pi = 2.0 * math.pi
    return Workload("taylor_green_16x16x16_p3_u24", (16, 16, 16), (0, 0, 0),
                    (two_pi, two_pi, two_pi), (True, True, True), 3, (24, 24, 24),
                    (-5, -5, -5), (5, 5, 5), 0.0, 2.0 / 3.0, mu_from_knudsen(0.01), 1.0,
                    THETA_S_RATIO, 0.1, 100, init=_init_taylor_green)


def normal_shock_tube(mach=8.0, width=2.0):
    """Hypersonic normal shock: [-20,40]x[0,1]^2 mean free paths, 64x4x4 hex, p=2,
    32^3 velocities on [-30,30]x[-15,15]^2, diatomic delta=2 (F and G), ES-BGK
    Pr=0.72, Sutherland with mu_ref from lambda_1 = 1; M=8 upstream at theta=1,
    Rankine--Hugoniot downstream (gamma=1.4), tanh blend of width 2 at x=0;
    Dirichlet x-ends, periodic y and z."""
    s1, s2 = normal_shock_states(mach, 1.4)
    dirichlet = {(0, -1): (s1[0], (s1[1], 0.0, 0.0), s1[2]),
                 (0, 1): (s2[0], (s2[1], 0.0, 0.0), s2[2])}
    return Workload("normal_shock_64x4x4_p2_u32_d2", (64, 4, 4), (-20, 0, 0), (40, 1, 1),
                    (False, True, True), 2, (32, 32, 32), (-30, -15, -15), (30, 15, 15),
                    2.0, 0.72, mu_from_knudsen(1.0), 1.0, THETA_S_RATIO, 0.1, 2000,
                    init=_shock_init(width, s1, s2), dirichlet=dirichlet)


def _wavy(amp):
    """Periodic warp of the unit cube: x = t + amp sin(2 pi t1) sin(2 pi t2) sin(2 pi t3)
    on every coordinate (a smooth curvilinear mesh of the periodic unit box)."""
    def mapping(t):
        w = amp * np.sin(2 * np.pi * t[..., 0]) * np.sin(2 * np.pi * t[..., 1]) * np.sin(2 * np.pi * t[..., 2])
        return t + w[..., None]
    return mapping


def wavy_periodic_box(p=2, n=(3, 3, 3), vel_n=(8, 8, 8), amp=0.05, Pr=1.0):
    """Curvilinear periodic case: the unit cube warped by _wavy, p, n hex, velocities
    on [-6,6]^3, monatomic, Kn=0.1, rho = 1 + 0.1 sin(2 pi x), U = 0, theta = 1."""
    return Workload("wavy_periodic_box_%dx%dx%d_p%d" % (n + (p,)), tuple(n), (0, 0, 0), (1, 1, 1),
                    (True, True, True), p, tuple(vel_n), (-6, -6, -6), (6, 6, 6),
                    0.0, Pr, mu_from_knudsen(0.1), 1.0, THETA_S_RATIO, 0.1, 10,
                    init=_init_sine_density, mapping=_wavy(amp),
                    h_min_override=(1.0 - 8.0 * amp) / max(n))


def _sphere_shell(r_in, r_out, ratio, n_r):
    """Latitude--longitude shell: t1 -> radius (geometric stretch `ratio` per radial
    element), t2 -> polar angle in [0, pi] (poles on the z axis), t3 -> azimuth."""
    def mapping(t):
        tr = t[..., 0] * n_r
        r = r_in + (r_out - r_in) * (ratio ** tr - 1.0) / (ratio ** n_r - 1.0)
        th = np.pi * t[..., 1]
        ph = 2.0 * np.pi * t[..., 2]
        return np.stack([r * np.sin(th) * np.cos(ph), r * np.sin(th) * np.sin(ph), r * np.cos(th)], axis=-1)
    return mapping


def sphere_ogrid(n=(12, 24, 24), p=1, vel_n=(40, 40, 40), umax=35.0, mach=22.7, kn=8e-4,
                 theta_w=0.1):
    """Blunt-body case: latitude--longitude O-grid around a sphere of diameter 1
    (r in [0.5, 4], radial stretch 1.15 per element), polar axis z perpendicular to
    the freestream along +x.  Diatomic delta=2, ES-BGK Pr=0.72, Sutherland, mu_ref
    from Kn_D; freestream Maxwellian at M (gamma=1.4, theta=1); diffuse wall at
    theta_w on the sphere, Dirichlet freestream at r=4, collapsed (no-flux) faces at
    the poles, periodic azimuth."""
    u_inf = mach * math.sqrt(1.4)
    free = (1.0, (u_inf, 0.0, 0.0), 1.0)
    mapping = _sphere_shell(0.5, 4.0, 1.15, n[0])

    def init(x):
        U = np.zeros(x.shape)
        U[..., 0] = u_inf
        return np.ones(x.shape[:-1]), U, np.ones(x.shape[:-1])
    # node spacing bound: the azimuthal extent at the first Gauss node off the pole
    xi0 = leggauss(p + 1)[0][0]
    th0 = np.pi / n[1] * 0.5 * (1.0 + xi0)
    dr0 = (4.0 - 0.5) * (1.15 - 1.0) / (1.15 ** n[0] - 1.0)
    h_min = min(0.5 * math.sin(th0) * 2.0 * math.pi / n[2], dr0) / (p + 1)
    return Workload("sphere_ogrid_%dx%dx%d_p%d_u%d_d2" % (n + (p, vel_n[0])), tuple(n), (0, 0, 0), (1, 1, 1),
                    (False, False, True), p, tuple(vel_n), (-umax,) * 3, (umax,) * 3,
                    2.0, 0.72, mu_from_knudsen(kn), 1.0, THETA_S_RATIO, 0.1, 500, init=init,
                    dirichlet={(0, 1): free}, diffuse={(0, -1): ((0.0, 0.0, 0.0), theta_w)},
                    closed=((1, -1), (1, 1)), mapping=mapping, h_min_override=h_min)


# ---- sampled inputs --------------------------------------------------------
def gll_nodes(q):
    """Gauss--Lobatto--Legendre nodes on [-1, 1] (the endpoints and the roots of
    P'_{q-1}), used to sample a mapping on element boundaries."""
    if q == 2:
        return np.array([-1.0, 1.0])
    inner = np.sort(np.polynomial.legendre.Legendre.basis(q - 1).deriv().roots().real)
    return np.concatenate([[-1.0], inner, [1.0]])


def _lagrange_matrix(src, dst):
    """L[i, j] = l_j(dst_i) for the Lagrange basis on the nodes src."""
    L = np.ones((len(dst), len(src)))
    for j in range(len(src)):
        for m in range(len(src)):
            if m != j:
                L[:, j] *= (dst - src[m]) / (src[j] - src[m])
    return L


def node_positions(wl):
    """Solution node coordinates x[Ne, Ns, 3] (numpy's Gauss--Legendre nodes).
    Curvilinear meshes: each element's mapping is the tensor interpolant of degree
    p of wl.mapping sampled at the element's Gauss--Lobatto points (shared by
    neighbouring elements, so the geometry is continuous), evaluated at the
    Gauss--Legendre nodes."""
    q = wl.p + 1
    xi = leggauss(q)[0]
    if wl.mapping is not None:
        return _mapped_node_positions(wl, xi)
    i3, i2, i1 = np.meshgrid(np.arange(q), np.arange(q), np.arange(q), indexing="ij")
    loc = [xi[i1.ravel()], xi[i2.ravel()], xi[i3.ravel()]]
    n1, n2, n3 = wl.mesh_n
    e = np.arange(wl.n_elem)
    c = [e % n1, (e // n1) % n2, e // (n1 * n2)]
    x = np.empty((wl.n_elem, q ** 3, 3))
    for d in range(3):
        h = (wl.mesh_hi[d] - wl.mesh_lo[d]) / wl.mesh_n[d]
        x[:, :, d] = wl.mesh_lo[d] + (c[d][:, None] + 0.5 * (loc[d][None, :] + 1.0)) * h
    return x


def _mapped_node_positions(wl, xi):
    q = wl.p + 1
    eta = gll_nodes(q)
    L = _lagrange_matrix(eta, xi)                              # [gl, gll]
    n1, n2, n3 = wl.mesh_n
    e = np.arange(wl.n_elem)
    c = np.stack([e % n1, (e // n1) % n2, e // (n1 * n2)], axis=1).astype(np.float64)
    nn = np.asarray(wl.mesh_n, dtype=np.float64)
    g3, g2, g1 = np.meshgrid(eta, eta, eta, indexing="ij")     # [i3, i2, i1]
    loc = np.stack([g1, g2, g3], axis=-1)                      # GLL points, [q, q, q, 3]
    t = (c[:, None, None, None, :] + 0.5 * (loc[None] + 1.0)) / nn
    X = wl.mapping(t)                                          # [Ne, q, q, q, 3] at GLL points
    X = np.einsum("ai,bj,ck,eijkn->eabcn", L, L, L, X)         # at GL nodes, [e, i3, i2, i1]
    return X.reshape(wl.n_elem, q ** 3, 3)


def velocity_nodes(wl):
    """u[Nu, 3] in the k = k1 + n1 (k2 + n2 k3) order."""
    ax = [np.linspace(wl.vel_lo[d], wl.vel_hi[d], wl.vel_n[d]) for d in range(3)]
    k3, k2, k1 = np.meshgrid(*(np.arange(wl.vel_n[d]) for d in (2, 1, 0)), indexing="ij")
    return np.stack([ax[0][k1.ravel()], ax[1][k2.ravel()], ax[2][k3.ravel()]], axis=1)


def gaussian_samples(u, rho, U, cov):
    """rho / sqrt(det(2 pi cov)) exp(-(u-U)^T cov^-1 (u-U)/2) for every (velocity,
    point): u[Nu,3], rho[P], U[P,3], cov[P,3,3] -> [Nu, P].  Initial-data sampler."""
    inv = np.linalg.inv(cov)
    c = u[:, None, :] - U[None, :, :]
    quad = np.einsum("kpi,pij,kpj->kp", c, inv, c)
    return (rho / np.sqrt(np.linalg.det(2.0 * np.pi * cov)))[None, :] * np.exp(-0.5 * quad)


def maxwellian_state(wl, x=None, fields=None):
    """f[C, Nu, Ne, Ns] = the isotropic Maxwellian of the initial field at each node
    (G = delta theta / 2 F)."""
    if x is None:
        x = node_positions(wl)
    rho, U, theta = fields if fields is not None else wl.init(x)
    P = wl.n_elem * wl.n_sol
    rho, U, theta = (np.broadcast_to(rho, x.shape[:-1]).reshape(P),
                     np.broadcast_to(U, x.shape).reshape(P, 3),
                     np.broadcast_to(theta, x.shape[:-1]).reshape(P))
    cov = theta[:, None, None] * np.eye(3)[None]
    F = gaussian_samples(velocity_nodes(wl), rho, U, cov)
    f = np.empty((wl.n_comp, wl.n_vel, wl.n_elem, wl.n_sol))
    f[0] = F.reshape(wl.n_vel, wl.n_elem, wl.n_sol)
    if wl.n_comp == 2:
        f[1] = (0.5 * wl.delta * theta)[None, :].reshape(1, wl.n_elem, wl.n_sol) * f[0]
    return f


def random_anisotropic_state(wl, seed, spread=0.3, bimodal=0.3):
    """Seeded non-equilibrium state: at every node a mixture of two Gaussians with
    random means and random SPD covariances around the initial field, so that
    Pi/rho is anisotropic and the element data are discontinuous."""
    rng = np.random.default_rng(seed)
    x = node_positions(wl)
    rho, U, theta = wl.init(x)
    P = wl.n_elem * wl.n_sol
    rho = np.broadcast_to(rho, x.shape[:-1]).reshape(P) * (1 + 0.2 * rng.uniform(-1, 1, P))
    U = np.broadcast_to(U, x.shape).reshape(P, 3) + 0.3 * rng.standard_normal((P, 3))
    theta = np.broadcast_to(theta, x.shape[:-1]).reshape(P) * (1 + 0.3 * rng.uniform(-1, 1, P))
    u = velocity_nodes(wl)
    total = np.zeros((wl.n_vel, P))
    for part, frac in ((0, 1.0 - bimodal), (1, bimodal)):
        a = rng.standard_normal((P, 3, 3)) * spread
        cov = theta[:, None, None] * (np.eye(3)[None] + np.einsum("pij,pkj->pik", a, a))
        shift = 0.0 if part == 0 else 0.8 * np.sqrt(theta)[:, None] * rng.standard_normal((P, 3))
        total += frac * gaussian_samples(u, rho, U + shift, cov)
    f = np.empty((wl.n_comp, wl.n_vel, wl.n_elem, wl.n_sol))
    f[0] = total.reshape(wl.n_vel, wl.n_elem, wl.n_sol)
    if wl.n_comp == 2:
        z = 0.5 * wl.delta * theta * (1 + 0.2 * rng.uniform(-1, 1, P))
        f[1] = z.reshape(1, wl.n_elem, wl.n_sol) * f[0]
    return f


def mixture_params(wl, x, elem):
    """Per-point parameters of a deterministic non-equilibrium state for states
    too large for the seeded generators: at every node a mixture
    3/4 N(U, diag s) + 1/4 N(U + a, 0.6 theta I) around the initial field, with
    smooth anisotropic s(x), a shifted second mean a(x), density and
    temperature modulations and a per-element density jump (discontinuous
    element data).  x[P, 3] node coordinates, elem[P] element indices."""
    rho, U, theta = wl.init(x)
    P = x.shape[0]
    rho = np.broadcast_to(rho, (P,)).astype(np.float64)
    U = np.broadcast_to(U, (P, 3)).astype(np.float64)
    theta = np.broadcast_to(theta, (P,)).astype(np.float64)
    s1, s2, s3 = x[:, 0], x[:, 1], x[:, 2]
    n1, n2 = wl.mesh_n[0], wl.mesh_n[1]
    e1, e2, e3 = elem % n1, (elem // n1) % n2, elem // (n1 * n2)
    jump = 1.0 + 0.025 * (((e1 + 2 * e2 + 3 * e3) % 5) - 2)
    rho = rho * (1.0 + 0.15 * np.sin(3.0 * s1 + 2.0 * s2 - s3)) * jump
    theta = theta * (1.0 + 0.2 * np.cos(2.0 * s1 - s2 + 3.0 * s3))
    var1 = theta[:, None] * (1.0 + 0.3 * np.sin(np.stack([s1, s2 + 1.0, s3 + 2.0], axis=1)))
    mean2 = U + 0.25 * np.sqrt(theta)[:, None] * np.sin(np.stack([s2 + 2.0 * s3, s3 + 2.0 * s1, s1 + 2.0 * s2], axis=1))
    var2 = np.repeat((0.6 * theta)[:, None], 3, axis=1)
    norm1 = 0.75 * rho / np.sqrt((2.0 * np.pi) ** 3 * var1[:, 0] * var1[:, 1] * var1[:, 2])
    norm2 = 0.25 * rho / np.sqrt((2.0 * np.pi) ** 3 * var2[:, 0] * var2[:, 1] * var2[:, 2])
    gfac = 0.5 * wl.delta * theta
    return dict(mean1=U, var1=var1, norm1=norm1, mean2=mean2, var2=var2, norm2=norm2, gfac=gfac)


def mixture_values(par, u, exp):
    """F[len(u), P] of the mixture_params state at velocities u[Nu, 3]; the
    arrays may be numpy or torch (exp is the matching exponential)."""
    out = 0.0
    for mean, var, norm in ((par["mean1"], par["var1"], par["norm1"]), (par["mean2"], par["var2"], par["norm2"])):
        q = 0.0
        for d in range(3):
            c = u[:, d:d + 1] - mean[None, :, d]
            q = q + c * c / var[None, :, d]
        out = out + norm[None, :] * exp(-0.5 * q)
    return out


def reduced(wl, mesh_n=None, vel_n=None):
    """Same physics and domain with fewer elements and/or velocity nodes."""
    kw = {}
    if mesh_n is not None:
        kw["mesh_n"] = tuple(mesh_n)
    if vel_n is not None:
        kw["vel_n"] = tuple(vel_n)
    return wl.replace(name=wl.name + "_reduced", **kw)
