"""FR residual, SSP-RK3 stage and diagnostics (test infrastructure).

Paper, section "Numerical method": for every discrete velocity u_k the
distribution obeys a linear advection d_t f + div(u_k f) = S, coupled across
velocities only by the BGK source S.  Inside each element f is the nodal
polynomial on the solution nodes; the flux u_k f is corrected with the
upwind common flux at the flux nodes:

    F(x) = u_k f(x) + sum_i [F^I_i - f(x^f_i) u_k.n_i] h_i(x),
    F^I_i = u_n f^-_i if u_n > 0 else u_n f^+_i,    u_n = u_k . n_i,

with h the DG-recovering correction function.  On a hex with tensor
Gauss--Legendre nodes this is, along each reference direction d and each
line of p+1 nodes, the 1-D FR derivative
    dF/dxi (xi_i) = u_d sum_j D_ij f_j + J_R g_R'(xi_i) - J_L g_L'(xi_i),
where J_R, J_L are the normal jumps F^I - u_n f^- at the right (+e_d) and
left (-e_d) flux nodes of the line; the left face's outward normal is -e_d,
which flips the sign of its jump in the +xi orientation.  The affine map
scales d/dx_d = (2/h_d) d/dxi_d, and R(f) = -div F + S.

Boundary conditions (section "Implementation & problem setup") are weak: a
boundary face sees an exterior state f^+.  A Dirichlet face's exterior state
is the Maxwellian of a prescribed (rho, U, theta) (for G: delta theta/2
times it), the same at every flux node of the face.  A specular (symmetry)
face reflects the particles: its exterior state at velocity u is the
element's own trace at the mirrored velocity u - 2 (u.n) n, i.e. with the
face's normal component negated (the velocity grid must be symmetric in that
axis so the mirrored velocity is a node).

Time integration: the paper only says "explicit"; the stage is the
Shu--Osher three-stage SSP Runge--Kutta scheme,
    f1 = f + dt R(f),  f2 = 3/4 f + 1/4 (f1 + dt R(f1)),
    f^{n+1} = 1/3 f + 2/3 (f2 + dt R(f2)).
"""
import numpy as np

from . import bgk
from .fr import FR1D


class Problem:
    """An FR + discrete-velocity BGK problem on a box mesh.

    dirichlet: dict {(d, side): (rho, (U1, U2, U3), theta)} for the
    non-periodic sides (side = -1 or +1).
    exterior: optional callable (d, side, fm) -> f^+ face traces replacing
    the Dirichlet state (used by the tests to prescribe exact data); fm is
    the interior trace array [C, Nu, Ne, q, q] of that side.
    specular: the non-periodic faces (d, side) that reflect specularly.
    """

    def __init__(self, mesh, p, vg, gas, dirichlet=None, exterior=None, specular=()):
        self.mesh, self.p, self.vg, self.gas = mesh, p, vg, gas
        self.fr = FR1D(p)
        self.q = p + 1
        self.Ns = self.q ** 3
        self.dirichlet = dict(dirichlet or {})
        self.exterior = exterior
        self.specular = set(specular)
        for d in range(3):
            if not mesh.periodic[d] and exterior is None:
                for side in (-1, 1):
                    if (d, side) not in self.dirichlet and (d, side) not in self.specular:
                        raise ValueError("missing boundary state for face (%d, %d)" % (d, side))
        self.mirror = {}
        for d, side in self.specular:
            if not np.isclose(vg.lo[d], -vg.hi[d]):
                raise ValueError("specular face needs a velocity grid symmetric in axis %d" % d)
            j = vg.index3()
            j[d] = vg.n[d] - 1 - j[d]
            self.mirror[d] = j[0] + vg.n[0] * (j[1] + vg.n[1] * j[2])
        self.nbr = {(d, s): mesh.neighbours(d, s) for d in range(3) for s in (-1, 1)}

    @property
    def shape(self):
        return (self.gas.n_comp, self.vg.size, self.mesh.n_elem, self.Ns)

    # -- advection ---------------------------------------------------------
    def _dirichlet_state(self, d, side):
        rho, U, theta = self.dirichlet[(d, side)]
        F = bgk.maxwellian(self.vg, np.array([rho]), np.array([U], dtype=np.float64),
                           np.array([theta]))[:, 0]
        comps = [F]
        if self.gas.n_comp == 2:
            comps.append(0.5 * self.gas.delta * theta * F)
        return np.stack(comps)                                      # [C, Nu]

    def divergence(self, f):
        """div(u_k f) at every solution node by FR with upwind flux: [C,Nu,Ne,Ns]."""
        C, Nu, Ne, Ns = f.shape
        q, fr = self.q, self.fr
        f6 = f.reshape(C, Nu, Ne, q, q, q)             # [..., i3, i2, i1]
        div = np.zeros_like(f6)
        for d in range(3):
            ax = 5 - d                                  # axis of the line index i_{d+1}
            ud = self.vg.u[:, d].reshape(1, Nu, 1, 1, 1)
            fl = np.moveaxis(f6, ax, -1)                # line index last
            dfl = np.einsum("ij,...j->...i", fr.D, fl)
            fm_L = np.einsum("j,...j->...", fr.l_minus, fl)   # [C,Nu,Ne,q,q]
            fm_R = np.einsum("j,...j->...", fr.l_plus, fl)
            fp_L = np.empty_like(fm_L)
            fp_R = np.empty_like(fm_R)
            for side, fm, fp, other in ((-1, fm_L, fp_L, fm_R), (1, fm_R, fp_R, fm_L)):
                nb = self.nbr[(d, side)]
                inner = nb >= 0
                fp[:, :, inner] = other[:, :, nb[inner]]
                if np.any(~inner):
                    if self.exterior is not None:
                        ext = self.exterior(d, side, fm)
                        fp[:, :, ~inner] = ext[:, :, ~inner]
                    elif (d, side) in self.specular:
                        # the element's own trace on this face at the mirrored velocity
                        fp[:, :, ~inner] = fm[:, self.mirror[d]][:, :, ~inner]
                    else:
                        st = self._dirichlet_state(d, side)        # [C, Nu]
                        fp[:, :, ~inner] = st[:, :, None, None, None]
            # outward normal +e_d on the right face, -e_d on the left face
            un_R, un_L = ud, -ud
            FI_R = np.where(un_R > 0, un_R * fm_R, un_R * fp_R)
            FI_L = np.where(un_L > 0, un_L * fm_L, un_L * fp_L)
            J_R = FI_R - un_R * fm_R
            J_L = FI_L - un_L * fm_L
            dxi = ud[..., None] * dfl + J_R[..., None] * fr.dgR - J_L[..., None] * fr.dgL
            div += np.moveaxis((2.0 / self.mesh.h[d]) * dxi, -1, ax)
        return div.reshape(C, Nu, Ne, Ns)

    # -- full residual -----------------------------------------------------
    def rhs(self, f, advect=True, collide=True, guess=None, tol=1e-13, max_iter=50):
        """R(f) = -div(u f) + S(f) and the source info (None if collide=False)."""
        C, Nu, Ne, Ns = f.shape
        R = np.zeros_like(f)
        if advect:
            R -= self.divergence(f)
        info = None
        if collide:
            F = f[0].reshape(Nu, Ne * Ns)
            G = f[1].reshape(Nu, Ne * Ns) if C == 2 else None
            S_F, S_G, info = bgk.bgk_source(F, G, self.gas, self.vg, guess=guess,
                                            tol=tol, max_iter=max_iter)
            R[0] += S_F.reshape(Nu, Ne, Ns)
            if C == 2:
                R[1] += S_G.reshape(Nu, Ne, Ns)
        return R, info

    def stage(self, f_n, f_s, a, b, dt, **kw):
        """a f_n + b (f_s + dt R(f_s)): one Shu--Osher stage."""
        R, info = self.rhs(f_s, **kw)
        return a * f_n + b * (f_s + dt * R), info

    def step(self, f, dt, **kw):
        """One SSP-RK3 step; returns (f^{n+1}, list of the three source infos)."""
        f1, i1 = self.stage(f, f, 0.0, 1.0, dt, **kw)
        f2, i2 = self.stage(f, f1, 0.75, 0.25, dt, **kw)
        f3, i3 = self.stage(f, f2, 1.0 / 3.0, 2.0 / 3.0, dt, **kw)
        return f3, [i1, i2, i3]

    # -- diagnostics -------------------------------------------------------
    def _node_weights(self):
        W1 = self.fr.wq
        W = np.einsum("i,j,k->ijk", W1, W1, W1).reshape(-1)    # [i3,i2,i1] order
        return W * self.mesh.jacobian()

    def totals(self, f):
        """Domain totals of (rho, rho U, E): sum_e sum_s W_s |J| sum_k w_k psi_k f."""
        C, Nu, Ne, Ns = f.shape
        Wx = self._node_weights()
        w, u = self.vg.w, self.vg.u
        F = np.einsum("kes,s->k", f[0], Wx)
        out = np.zeros(5)
        out[0] = np.sum(w * F)
        for d in range(3):
            out[1 + d] = np.sum(w * u[:, d] * F)
        out[4] = np.sum(w * 0.5 * np.sum(u * u, axis=1) * F)
        if C == 2:
            out[4] += np.sum(w * np.einsum("kes,s->k", f[1], Wx))
        return out

    def entropy(self, f):
        """Discrete entropy H = sum W |J| sum_k w_k F ln F (F > 0 required)."""
        Wx = self._node_weights()
        F = f[0]
        return float(np.sum(self.vg.w[:, None, None] * Wx[None, None, :] * F * np.log(F)))

    def l2(self, f):
        """sum W |J| sum_k w_k f^2 over all components."""
        Wx = self._node_weights()
        return float(np.sum(self.vg.w[None, :, None, None] * Wx * f * f))


def element_residual(h, p, vg, gas, f27, guess=None, tol=1e-13, max_iter=50, with_source=False):
    """R(f) = -div(u f) + S(f) of one element from its 3x3x3 block of elements.

    f27[C, Nu, 27, Ns] holds the element (block index 13) and its neighbours in
    the order e = i1 + 3 (i2 + 3 i3); only the six face neighbours enter the
    element's residual (the upwind flux couples face neighbours only, and S is
    local).  The block is evaluated as a 3x3x3 box of spacing h whose outer
    faces see a zero exterior state, which affects the outer elements only.
    Used to check single elements of states too large for the whole-mesh
    routines.  Returns R[C, Nu, Ns] (and the source part S[C, Nu, Ns] with
    with_source).
    """
    from .mesh import BoxMesh
    mesh = BoxMesh((3, 3, 3), (0.0, 0.0, 0.0), tuple(3.0 * np.asarray(h, dtype=np.float64)), (False, False, False))
    prob = Problem(mesh, p, vg, gas, exterior=lambda d, side, fm: np.zeros_like(fm))
    div = prob.divergence(f27)[:, :, 13, :]
    C, Nu = f27.shape[:2]
    F = f27[0, :, 13, :]
    G = f27[1, :, 13, :] if C == 2 else None
    S_F, S_G, _ = bgk.bgk_source(F, G, gas, vg, guess=guess, tol=tol, max_iter=max_iter)
    S = np.stack([S_F] + ([S_G] if C == 2 else []))
    R = S - div
    return (R, S) if with_source else R


def slab_residual(h, n_yz, p, vg, gas, dirichlet, f3, target, with_source=False, tol=1e-13, max_iter=50):
    """R(f) = -div(u f) + S(f) of one first-axis slab of elements (the n2 x n3
    elements at one first-axis index) of a mesh that is periodic in its second
    and third directions, from three consecutive slabs.

    f3[C, Nu, 3 n2 n3, Ns] holds the slabs in mesh order (element
    e = i1 + 3 (i2 + n2 i3), i1 = 0, 1, 2); the sub-box of spacing h has
    Dirichlet first-axis faces with the given states.  The residual of slab
    `target` is exact when target = 1 (both first-axis neighbours present)
    and when the target's outer face is the full mesh's own Dirichlet face
    (target 0 at the low end, 2 at the high end).  Used to check slabs of
    states too large for the whole-mesh routines.  Returns R[C, Nu, n2 n3, Ns]
    (and the source part S with with_source)."""
    from .mesh import BoxMesh
    n2, n3 = n_yz
    hh = np.asarray(h, dtype=np.float64)
    mesh = BoxMesh((3, n2, n3), (0.0, 0.0, 0.0), (3.0 * hh[0], n2 * hh[1], n3 * hh[2]), (False, True, True))
    prob = Problem(mesh, p, vg, gas, dirichlet=dirichlet)
    div = prob.divergence(f3)
    C, Nu = f3.shape[:2]
    sel = np.array([target + 3 * (i2 + n2 * i3) for i3 in range(n3) for i2 in range(n2)])
    div = div[:, :, sel, :]
    F = f3[0][:, sel, :].reshape(Nu, -1)
    G = f3[1][:, sel, :].reshape(Nu, -1) if C == 2 else None
    S_F, S_G, _ = bgk.bgk_source(F, G, gas, vg, tol=tol, max_iter=max_iter)
    S = np.stack([S_F] + ([S_G] if C == 2 else [])).reshape(div.shape)
    R = S - div
    return (R, S) if with_source else R


def cfl_dt(mesh, vg, p, cfl):
    """dt = CFL h_min / (u_max (2p + 1)) (the paper gives only the explicit scheme)."""
    umax = float(np.max(np.abs(vg.u)))
    return cfl * float(np.min(mesh.h)) / (umax * (2 * p + 1))


def problem_from_workload(wl, exterior=None):
    """Build a Problem from a workload definition (duck-typed: sizes and gas only)."""
    from .mesh import BoxMesh
    from .velocity import VelocityGrid
    mesh = BoxMesh(wl.mesh_n, wl.mesh_lo, wl.mesh_hi, wl.periodic)
    vg = VelocityGrid(wl.vel_n, wl.vel_lo, wl.vel_hi)
    gas = bgk.Gas(delta=wl.delta, Pr=wl.Pr, mu_ref=wl.mu_ref, theta_ref=wl.theta_ref,
                  theta_S=wl.theta_S,
                  es_tensor=getattr(wl, "es_tensor", False))
    return Problem(mesh, wl.p, vg, gas, dirichlet=wl.dirichlet, exterior=exterior,
                   specular=getattr(wl, "specular", ()))
