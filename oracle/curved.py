"""FR residual on curvilinear hexahedra, diffuse walls and collapsed faces
(test infrastructure: only the tests, the smoke check and the benchmark's CPU
baseline use this module; the CUDA path never imports it).

Paper, section "Numerical method": F(x) = u f(x) + sum_i [F^I_i - f(x^f_i)
u.n_i] h_i(x) with outward normals n_i at the flux nodes and the upwind
common flux F^I.  On a curved element this is applied to the equation mapped
to the reference cube (the standard FR treatment of curved elements; the
paper states the physical-space form only):

    J d_t f + sum_d d/dxi_d (Ft_d) = J S,    Ft_d = (u . S^d) f,
    S^d = J dxi_d/dx  (the contravariant metric vectors times J).

Readings of the discrete metric terms (the paper is silent on them):
  - geometry: per element, the nodal interpolant of degree p of the
    solution-node coordinates x_s;
  - S^d in the conservative curl form (Kopriva 2006),
        (S^i)_n = -[curl_xi I(X_l grad_xi X_m)]_i,   (n, m, l) cyclic,
    with the interpolant I and the derivatives taken on the element's
    Gauss--Lobatto--Legendre (GLL) points (which include the faces), and the
    resulting polynomial of degree p evaluated at the solution nodes.  Its
    divergence vanishes identically (the divergence of a curl), and its trace
    on a face depends only on X and its tangential derivatives on that face,
    which neighbouring elements share when the geometry is continuous: then
    a uniform state has zero residual exactly (free-stream preservation);
    J = det(dX/dxi) of the interpolant at the solution nodes;
  - face vectors at the flux nodes: the trace of each side's S^d polynomial,
    averaged over the two sides of an interior face (a no-op for continuous
    geometry), so the common flux is single-valued and the scheme conserves
    exactly; a boundary face takes its own trace.  On affine elements this is
    the analytic face normal times the face's area scale.

Along each reference direction d and each line of p+1 nodes, with a_j =
u.S^d_j, Ft_j = a_j f_j and A_R, A_L = u.S_face at the line's right (+xi_d)
and left faces (both oriented along +xi_d):
    right face: F^I = A_R f^- if A_R > 0 else A_R f^+,  J_R = F^I - sum_j l_j(+1) Ft_j
    left face:  outward u_n = -A_L, F^I_out = u_n (f^- if u_n > 0 else f^+),
                J_L = -F^I_out - sum_j l_j(-1) Ft_j        (+xi orientation)
    dFt/dxi(xi_i) = sum_j D_ij Ft_j + J_R g_R'(xi_i) + J_L g_L'(xi_i)
and div = (1/J) sum_d dFt_d/dxi.  Unlike the affine case, an outflow face
contributes as well (the trace of a_j f_j is not A times the trace of f).

Boundary faces (section "Implementation & problem setup": all weak through
the Riemann flux):
  - Dirichlet: the exterior state is a prescribed Maxwellian;
  - diffuse wall (reading; details are in a companion paper): at each flux
    node the exterior state of the velocities entering the gas (u_n < 0,
    n the outward normal of the gas) is rho_w M(u; U_w, theta_w) (G:
    delta theta_w / 2 times it), with rho_w set so that no mass crosses the
    node: rho_w = -sum_{u_n>0} w u_n F^- / sum_{u_n<0} w u_n M(u; U_w, theta_w);
  - closed: a collapsed face of zero area (the poles of a latitude--longitude
    grid); no flux crosses it, F^I = 0.
"""
import numpy as np

from . import bgk
from .fr import FR1D
from .mesh import BoxMesh

_CYC = ((0, 1, 2), (1, 2, 0), (2, 0, 1))        # (n, m, l) cyclic


def gll_points(q):
    """Gauss--Lobatto--Legendre points: -1, the roots of P'_{q-1}, +1."""
    if q == 2:
        return np.array([-1.0, 1.0])
    inner = np.sort(np.polynomial.legendre.Legendre.basis(q - 1).deriv().roots().real)
    return np.concatenate([[-1.0], inner, [1.0]])


def lagrange_values(src, dst):
    """L[i, j] = l_j(dst_i), l_j the Lagrange basis on the points src."""
    L = np.ones((len(dst), len(src)))
    for j in range(len(src)):
        for m in range(len(src)):
            if m != j:
                L[:, j] *= (dst - src[m]) / (src[j] - src[m])
    return L


def lagrange_derivative(src):
    """D[i, j] = l_j'(src_i): barycentric weights b_j = 1 / prod_{m != j}(x_j - x_m),
    D_ij = (b_j / b_i) / (x_i - x_j) off the diagonal, rows summing to zero."""
    q = len(src)
    b = np.array([1.0 / np.prod([src[j] - src[m] for m in range(q) if m != j]) for j in range(q)])
    D = np.zeros((q, q))
    for i in range(q):
        for j in range(q):
            if i != j:
                D[i, j] = (b[j] / b[i]) / (src[i] - src[j])
        D[i, i] = -np.sum(D[i])
    return D


def _apply3(g, L):
    """Apply the 1-D matrix L along the three node axes of g[e, i3, i2, i1, ...]."""
    for ax in (1, 2, 3):
        h = np.moveaxis(g, ax, -1)
        g = np.moveaxis(np.einsum("ij,...j->...i", L, h), -1, ax)
    return g


def _dxi(g, j, D):
    """Reference derivative along xi_j of nodal values g[e, i3, i2, i1, ...]."""
    ax = 3 - j
    h = np.moveaxis(g, ax, -1)
    return np.moveaxis(np.einsum("ij,...j->...i", D, h), -1, ax)


def curl_metrics(x6, fr):
    """S[e, i, n, i3, i2, i1] = (J a^i)_n and J[e, i3, i2, i1] at the solution
    nodes from their coordinates x6[e, i3, i2, i1, 3]: the curl form on the GLL
    points, evaluated at the Gauss nodes."""
    eta = gll_points(len(fr.xi))
    DL = lagrange_derivative(eta)
    XL = _apply3(x6, lagrange_values(fr.xi, eta))                         # X at the GLL points
    dX = [[_dxi(XL[..., n], j, DL) for n in range(3)] for j in range(3)]  # dX[j][n] = d_j X_n
    SL = np.zeros(x6.shape[:1] + (3, 3) + x6.shape[1:4])
    for n, m, l in _CYC:
        # V_j = X_l d_j X_m at the GLL points (nodal values of its interpolant)
        V = [XL[..., l] * dX[j][m] for j in range(3)]
        for i, j, k in _CYC:
            SL[:, i, n] = -(_dxi(V[k], j, DL) - _dxi(V[j], k, DL))
    to_gauss = lagrange_values(eta, fr.xi)
    S = np.moveaxis(_apply3(np.moveaxis(SL, (1, 2), (-2, -1)), to_gauss), (-2, -1), (1, 2))
    dXg = [[_dxi(x6[..., n], j, fr.D) for n in range(3)] for j in range(3)]
    Jm = np.stack([np.stack([dXg[j][n] for j in range(3)], axis=-1) for n in range(3)], axis=-2)
    J = np.linalg.det(Jm)                      # det[d X_n / d xi_j]
    return S, J


class CurvedMesh:
    """Structured hex topology (BoxMesh element numbering, neighbours and
    periodicity) with curvilinear elements given by their node coordinates
    x[Ne, Ns, 3] at the tensor Gauss--Legendre nodes of order p."""

    def __init__(self, n, periodic, x, p):
        self.topo = BoxMesh(n, (0.0, 0.0, 0.0), (1.0, 1.0, 1.0), periodic)
        self.n, self.periodic, self.n_elem = self.topo.n, self.topo.periodic, self.topo.n_elem
        self.fr = FR1D(p)
        q = p + 1
        self.q = q
        x = np.asarray(x, dtype=np.float64)
        if x.shape != (self.n_elem, q ** 3, 3):
            raise ValueError("node coordinates must be [Ne, (p+1)^3, 3]")
        self.x = x
        x6 = x.reshape(self.n_elem, q, q, q, 3)
        self.S, self.J = curl_metrics(x6, self.fr)
        if np.any(self.J <= 0):
            raise ValueError("non-positive Jacobian at a solution node")
        self.nbr = {(d, s): self.topo.neighbours(d, s) for d in range(3) for s in (-1, 1)}
        self.face = {}                          # (d, side) -> [Ne, q, q, 3], oriented +xi_d
        own = {}
        for d in range(3):
            Sd = np.moveaxis(self.S[:, d], 1, -1)                  # [e, i3, i2, i1, n]
            Sl = np.moveaxis(Sd, 3 - d, -1)                        # line index last
            own[(d, -1)] = np.einsum("j,...j->...", self.fr.l_minus, Sl)
            own[(d, 1)] = np.einsum("j,...j->...", self.fr.l_plus, Sl)
        for d in range(3):
            for side in (-1, 1):
                nb = self.nbr[(d, side)]
                v = own[(d, side)].copy()
                inner = nb >= 0
                v[inner] = 0.5 * (v[inner] + own[(d, -side)][nb[inner]])
                self.face[(d, side)] = v

    def node_weights(self):
        """W_s J_s per node [Ne, Ns]: the quadrature of the totals."""
        W1 = self.fr.wq
        W = np.einsum("i,j,k->ijk", W1, W1, W1)
        return (W[None] * self.J).reshape(self.n_elem, -1)


class CurvedProblem:
    """FR + discrete-velocity BGK on a CurvedMesh.

    dirichlet: {(d, side): (rho, U(3), theta)}; diffuse: {(d, side): (U_w(3),
    theta_w)}; closed: faces with no flux.  Every non-periodic face needs one of
    the three (or the exterior hook of the tests: exterior(d, side, fm) -> f^+
    traces [C, Nu, Ne, q, q])."""

    def __init__(self, mesh, vg, gas, dirichlet=None, diffuse=None, closed=(), exterior=None):
        self.mesh, self.vg, self.gas = mesh, vg, gas
        self.fr, self.q, self.p = mesh.fr, mesh.q, mesh.q - 1
        self.Ns = self.q ** 3
        self.dirichlet = dict(dirichlet or {})
        self.diffuse = dict(diffuse or {})
        self.closed = set(closed)
        self.exterior = exterior
        for d in range(3):
            if not mesh.periodic[d] and exterior is None:
                for side in (-1, 1):
                    kinds = [(d, side) in self.dirichlet, (d, side) in self.diffuse, (d, side) in self.closed]
                    if sum(kinds) != 1:
                        raise ValueError("face (%d, %d) needs exactly one boundary kind" % (d, side))

    @property
    def shape(self):
        return (self.gas.n_comp, self.vg.size, self.mesh.n_elem, self.Ns)

    def _maxwellian_comps(self, rho, U, theta):
        F = bgk.maxwellian(self.vg, np.array([rho]), np.array([U], dtype=np.float64), np.array([theta]))[:, 0]
        comps = [F]
        if self.gas.n_comp == 2:
            comps.append(0.5 * self.gas.delta * theta * F)
        return np.stack(comps)                                    # [C, Nu]

    def wall_density(self, d, side, fm):
        """rho_w[Ne, q, q] of a diffuse face from the interior F traces fm[C, Nu, Ne, q, q]."""
        U_w, theta_w = self.diffuse[(d, side)]
        M = self._maxwellian_comps(1.0, U_w, theta_w)[0]           # [Nu]
        un = side * np.einsum("kn,eabn->keab", self.vg.u, self.mesh.face[(d, side)])
        w = self.vg.w[:, None, None, None]
        num = np.sum(np.where(un > 0, w * un * fm[0], 0.0), axis=0)
        den = np.sum(np.where(un < 0, w * un * M[:, None, None, None], 0.0), axis=0)
        return -num / den

    def divergence(self, f):
        """div(u_k f) at every solution node [C, Nu, Ne, Ns]."""
        C, Nu, Ne, Ns = f.shape
        q, fr, mesh = self.q, self.fr, self.mesh
        u = self.vg.u
        f6 = f.reshape(C, Nu, Ne, q, q, q)
        acc = np.zeros_like(f6)
        for d in range(3):
            ax = 5 - d
            a = np.einsum("kn,enabc->keabc", u, mesh.S[:, d])[None]      # [1, Nu, Ne, i3, i2, i1]
            fl = np.moveaxis(f6, ax, -1)
            Fl = np.moveaxis(a * f6, ax, -1)
            dF = np.einsum("ij,...j->...i", fr.D, Fl)
            fm = {-1: np.einsum("j,...j->...", fr.l_minus, fl), 1: np.einsum("j,...j->...", fr.l_plus, fl)}
            Ft = {-1: np.einsum("j,...j->...", fr.l_minus, Fl), 1: np.einsum("j,...j->...", fr.l_plus, Fl)}
            A = {s: np.einsum("kn,eabn->keab", u, mesh.face[(d, s)])[None] for s in (-1, 1)}
            FI_out = {}
            for side in (-1, 1):
                un = side * A[side]                                       # outward normal velocity
                nb = mesh.nbr[(d, side)]
                inner = nb >= 0
                fp = np.empty_like(fm[side])
                fp[:, :, inner] = fm[-side][:, :, nb[inner]]
                closed = np.zeros(Ne, dtype=bool)
                if np.any(~inner):
                    if self.exterior is not None:
                        fp[:, :, ~inner] = self.exterior(d, side, fm[side])[:, :, ~inner]
                    elif (d, side) in self.closed:
                        closed = ~inner
                        fp[:, :, ~inner] = 0.0
                    elif (d, side) in self.diffuse:
                        U_w, theta_w = self.diffuse[(d, side)]
                        rho_w = self.wall_density(d, side, fm[side])      # [Ne, q, q]
                        Mc = self._maxwellian_comps(1.0, U_w, theta_w)    # [C, Nu]
                        ext = Mc[:, :, None, None, None] * rho_w[None, None]
                        fp[:, :, ~inner] = ext[:, :, ~inner]
                    else:
                        st = self._maxwellian_comps(*self.dirichlet[(d, side)])
                        fp[:, :, ~inner] = st[:, :, None, None, None]
                F = np.where(un > 0, un * fm[side], un * fp)
                F[:, :, closed] = 0.0
                FI_out[side] = F
            J_R = FI_out[1] - Ft[1]
            J_L = -FI_out[-1] - Ft[-1]
            dxi = dF + J_R[..., None] * fr.dgR + J_L[..., None] * fr.dgL
            acc += np.moveaxis(dxi, -1, ax)
        J = mesh.J[None, None]                                            # [1, 1, e, i3, i2, i1]
        return (acc / J).reshape(C, Nu, Ne, Ns)

    def rhs(self, f, advect=True, collide=True, guess=None, tol=1e-13, max_iter=50):
        C, Nu, Ne, Ns = f.shape
        R = np.zeros_like(f)
        if advect:
            R -= self.divergence(f)
        info = None
        if collide:
            F = f[0].reshape(Nu, Ne * Ns)
            G = f[1].reshape(Nu, Ne * Ns) if C == 2 else None
            S_F, S_G, info = bgk.bgk_source(F, G, self.gas, self.vg, guess=guess, tol=tol, max_iter=max_iter)
            R[0] += S_F.reshape(Nu, Ne, Ns)
            if C == 2:
                R[1] += S_G.reshape(Nu, Ne, Ns)
        return R, info

    def stage(self, f_n, f_s, a, b, dt, **kw):
        R, info = self.rhs(f_s, **kw)
        return a * f_n + b * (f_s + dt * R), info

    def step(self, f, dt, **kw):
        f1, i1 = self.stage(f, f, 0.0, 1.0, dt, **kw)
        f2, i2 = self.stage(f, f1, 0.75, 0.25, dt, **kw)
        f3, i3 = self.stage(f, f2, 1.0 / 3.0, 2.0 / 3.0, dt, **kw)
        return f3, [i1, i2, i3]

    def totals(self, f):
        """(rho, rho U, E) totals: sum_e sum_s W_s J_s sum_k w_k psi_k f."""
        C = f.shape[0]
        Wx = self.mesh.node_weights()
        w, u = self.vg.w, self.vg.u
        F = np.einsum("kes,es->k", f[0], Wx)
        out = np.zeros(5)
        out[0] = np.sum(w * F)
        for d in range(3):
            out[1 + d] = np.sum(w * u[:, d] * F)
        out[4] = np.sum(w * 0.5 * np.sum(u * u, axis=1) * F)
        if C == 2:
            out[4] += np.sum(w * np.einsum("kes,es->k", f[1], Wx))
        return out


def problem_from_workload(wl, x, exterior=None):
    """CurvedProblem of a workload (duck-typed: sizes, gas and boundary faces)
    on the node coordinates x[Ne, Ns, 3]."""
    from .velocity import VelocityGrid
    mesh = CurvedMesh(wl.mesh_n, wl.periodic, x, wl.p)
    vg = VelocityGrid(wl.vel_n, wl.vel_lo, wl.vel_hi)
    gas = bgk.Gas(delta=wl.delta, Pr=wl.Pr, mu_ref=wl.mu_ref, theta_ref=wl.theta_ref, theta_S=wl.theta_S,
                  es_tensor=getattr(wl, "es_tensor", False))
    return CurvedProblem(mesh, vg, gas, dirichlet=wl.dirichlet, diffuse=getattr(wl, "diffuse", {}),
                         closed=getattr(wl, "closed", ()), exterior=exterior)


def element_residual(p, vg, gas, x27, f27, with_source=False, guess=None, tol=1e-13, max_iter=50):
    """R(f) = -div(u f) + S(f) of one curvilinear element from its 3x3x3 block.

    x27[27, Ns, 3] are the node coordinates and f27[C, Nu, 27, Ns] the state of
    the element (block index 13) and its neighbours in the order
    e = i1 + 3 (i2 + 3 i3); the face vectors of the element's faces are the
    averages over both sides as in the whole mesh, and the block's outer faces
    see a zero exterior state, which affects the outer elements only.  Used to
    check single elements of states too large for the whole-mesh routines.
    Returns R[C, Nu, Ns] (and the source part S[C, Nu, Ns] with with_source)."""
    mesh = CurvedMesh((3, 3, 3), (False, False, False), x27, p)
    prob = CurvedProblem(mesh, vg, gas, exterior=lambda d, side, fm: np.zeros_like(fm))
    div = prob.divergence(f27)[:, :, 13, :]
    C = f27.shape[0]
    F = f27[0, :, 13, :]
    G = f27[1, :, 13, :] if C == 2 else None
    S_F, S_G, _ = bgk.bgk_source(F, G, gas, vg, guess=guess, tol=tol, max_iter=max_iter)
    S = np.stack([S_F] + ([S_G] if C == 2 else []))
    R = S - div
    return (R, S) if with_source else R
