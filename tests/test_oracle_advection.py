"""Pins of the oracle's FR advection: polynomial exactness, equivalence with an
independently written strong-form nodal DG residual, collisionless closed form
with its convergence order, L2 stability and discrete conservation."""
import numpy as np
import pytest
from numpy.polynomial import polynomial as npoly
from numpy.polynomial.legendre import leggauss

from oracle import bgk, stage
from oracle.mesh import BoxMesh
from oracle.velocity import VelocityGrid


def _problem(mesh_n, p, vel_n=(2, 3, 2), vlo=(-1.5, -1.2, -0.7), vhi=(1.5, 1.2, 0.9),
             periodic=(True, True, True), exterior=None, lo=(0, 0, 0), hi=(1, 0.8, 1.3)):
    mesh = BoxMesh(mesh_n, lo, hi, periodic)
    vg = VelocityGrid(vel_n, vlo, vhi)
    gas = bgk.Gas(delta=0.0, Pr=1.0, mu_ref=0.1)
    return stage.Problem(mesh, p, vg, gas, exterior=exterior)


def _poly(x, u, p):
    """A velocity-dependent polynomial of degree <= p in each coordinate, and its
    advective derivative u . grad."""
    X, Y, Z = x[..., 0], x[..., 1], x[..., 2]
    a = 1.0 + 0.3 * u[:, 0] - 0.2 * u[:, 1] * u[:, 2]
    b = 0.5 - 0.1 * u[:, 2]
    a, b = a[:, None, None], b[:, None, None]
    if p == 1:
        val = a + b * X * Y - 0.7 * Y * Z + 0.2 * X * Y * Z
        gx = b * Y + 0.2 * Y * Z
        gy = b * X - 0.7 * Z + 0.2 * X * Z
        gz = -0.7 * Y + 0.2 * X * Y + 0 * b
    else:
        val = a + b * X * X * Y - 0.7 * Y * Z * Z + 0.2 * X * X * Y * Y * Z * Z
        gx = 2 * b * X * Y + 0.4 * X * Y * Y * Z * Z
        gy = b * X * X - 0.7 * Z * Z + 0.4 * X * X * Y * Z * Z
        gz = -1.4 * Y * Z + 0.4 * X * X * Y * Y * Z + 0 * b
    ud = [u[:, d][:, None, None] for d in range(3)]
    return val, ud[0] * gx + ud[1] * gy + ud[2] * gz


@pytest.mark.parametrize("p", [1, 2])
def test_polynomial_exactness(p):
    """With data in Q_p and the exact exterior state every jump vanishes and
    the FR divergence equals u . grad f at the nodes."""
    holder = {}

    def exterior(d, side, fm):
        pb = holder["pb"]
        q = pb.q
        x = pb.mesh.node_coords(pb.fr.xi).reshape(pb.mesh.n_elem, q, q, q, 3)
        xl = np.moveaxis(x, 3 - d, -2)                     # [Ne, a, b, line, 3]
        xf = xl[..., 0, :].copy()
        e = np.arange(pb.mesh.n_elem)
        c = np.array([pb.mesh.coords(i)[d] for i in e])
        xf[..., d] = (pb.mesh.lo[d] + (c + (side + 1) / 2) * pb.mesh.h[d])[:, None, None]
        val, _ = _poly(xf.reshape(-1, 3)[None], pb.vg.u, p)
        return val.reshape(1, pb.vg.size, pb.mesh.n_elem, q, q)

    pb = _problem((3, 2, 2), p, periodic=(False, False, False), exterior=exterior)
    holder["pb"] = pb
    x = pb.mesh.node_coords(pb.fr.xi)
    val, adv = _poly(x.reshape(-1, 3)[None], pb.vg.u, p)
    f = val.reshape(1, pb.vg.size, pb.mesh.n_elem, pb.Ns)
    div = pb.divergence(f)
    ref = adv.reshape(div.shape)
    assert np.max(np.abs(div - ref)) <= 1e-12 * np.max(np.abs(ref))


def _lagrange_1d(xi):
    """Monomial coefficients of the Lagrange basis on nodes xi (Vandermonde solve)."""
    V = npoly.polyvander(xi, len(xi) - 1)
    return np.linalg.inv(V)          # column j = coefficients of l_j


def _dg_residual(pb, f):
    """Strong/weak-form nodal DG residual -div, written independently:
    M du/dt = sum_d u_d int dphi/dx_d f  -  sum_faces int phi F^I_n dS,
    with exact Gauss quadrature (p+3 points) and an explicit mass matrix."""
    q = pb.q
    xi = leggauss(q)[0]
    C = _lagrange_1d(xi)
    xq, wq = leggauss(q + 2)
    Lq = np.stack([npoly.polyval(xq, C[:, j]) for j in range(q)], axis=1)       # [nq, q]
    dC = np.stack([npoly.polyder(C[:, j]) for j in range(q)], axis=1)
    dLq = np.stack([npoly.polyval(xq, dC[:, j]) for j in range(q)], axis=1)
    M1 = Lq.T @ (wq[:, None] * Lq)
    S1 = dLq.T @ (wq[:, None] * Lq)                 # S1[a, b] = int l_a' l_b
    em = np.array([npoly.polyval(-1.0, C[:, j]) for j in range(q)])
    ep = np.array([npoly.polyval(1.0, C[:, j]) for j in range(q)])
    h = pb.mesh.h
    J = np.prod(h / 2)
    kron3 = lambda a3, a2, a1: np.kron(a3, np.kron(a2, a1))
    M3 = J * kron3(M1, M1, M1)
    K = [kron3(M1, M1, S1), kron3(M1, S1, M1), kron3(S1, M1, M1)]
    n1, n2, n3 = pb.mesh.n
    Ne, Nu = pb.mesh.n_elem, pb.vg.size
    u = pb.vg.u
    fe = f[0]                                        # [Nu, Ne, Ns]
    # traces at the 6 faces, face values indexed by the two tangential nodes
    f6 = fe.reshape(Nu, Ne, q, q, q)
    out = np.zeros_like(fe)
    for e in range(Ne):
        c = [e % n1, (e // n1) % n2, e // (n1 * n2)]
        rhs = np.zeros((Nu, q ** 3))
        for d in range(3):
            rhs += (u[:, d] * (2 / h[d]) * J)[:, None] * (fe[:, e] @ K[d].T)
        for d in range(3):
            ax = 4 - d                                # line axis in [Nu, i3, i2, i1]
            Jf = J * 2 / h[d]
            for side, own, other in ((-1, em, ep), (1, ep, em)):
                cc = list(c)
                cc[d] = (cc[d] + side) % pb.mesh.n[d]
                en = cc[0] + n1 * (cc[1] + n2 * cc[2])
                fm = np.tensordot(np.moveaxis(f6[:, e], ax - 1, -1), own, axes=([3], [0]))
                fp = np.tensordot(np.moveaxis(f6[:, en], ax - 1, -1), other, axes=([3], [0]))
                un = side * u[:, d][:, None, None]
                FI = np.where(un > 0, un * fm, un * fp)      # [Nu, a, b]
                # int phi_s F^I dS: own trace value of the line basis times face mass
                Mf = np.kron(M1, M1)                            # acts on (a, b)
                proj = (FI.reshape(Nu, q * q) @ Mf.T).reshape(Nu, q, q)
                vol = np.zeros((Nu, q, q, q))
                line = own
                # place line basis along axis d
                if d == 0:
                    vol = proj[:, :, :, None] * line[None, None, None, :]
                elif d == 1:
                    vol = proj[:, :, None, :] * line[None, None, :, None]
                else:
                    vol = proj[:, None, :, :] * line[None, :, None, None]
                rhs -= Jf * vol.reshape(Nu, q ** 3)
        out[:, e] = np.linalg.solve(M3, rhs.T).T
    return out


@pytest.mark.parametrize("p", [1, 2])
def test_fr_equals_nodal_dg(p):
    """FR with the Radau (g_DG) correction on Gauss nodes reproduces nodal DG
    (Huynh 2007) on random discontinuous data: pins sign and scale of the lift."""
    pb = _problem((3, 2, 2), p)
    rng = np.random.default_rng(7)
    f = rng.uniform(0.5, 1.5, (1, pb.vg.size, pb.mesh.n_elem, pb.Ns))
    ours = -pb.divergence(f)[0]
    dg = _dg_residual(pb, f)
    assert np.max(np.abs(ours - dg)) <= 1e-12 * np.max(np.abs(dg))


@pytest.mark.parametrize("p,rate", [(1, 1.5), (2, 2.5)])
def test_collisionless_closed_form_converges(p, rate):
    """Source off: f_k(x, t) = f_k(x - u_k t, 0) for sinusoidal data; the nodal
    max error falls at least like h^(p+1/2) and the L2 energy never grows."""
    errs = []
    for n in (4, 8, 16):
        pb = _problem((n, 1, 1), p, vel_n=(2, 2, 2), vlo=(-1, -1, -1), vhi=(1, 1, 1),
                      hi=(1, 1, 1))
        x = pb.mesh.node_coords(pb.fr.xi)[..., 0]        # [Ne, Ns]
        s = 1 + 0.1 * np.arange(pb.vg.size)
        u1 = pb.vg.u[:, 0]
        f = (1 + 0.5 * np.sin(2 * np.pi * x)[None] * s[:, None, None])[None]
        T = 0.1
        dt = 0.1 * pb.mesh.h[0] / (2 * p + 1)
        nsteps = int(np.ceil(T / dt))
        dt = T / nsteps
        e_prev = pb.l2(f)
        for _ in range(nsteps):
            f, _ = pb.step(f, dt, collide=False)
            e_now = pb.l2(f)
            assert e_now <= e_prev * (1 + 1e-14)
            e_prev = e_now
        exact = 1 + 0.5 * np.sin(2 * np.pi * (x[None] - u1[:, None, None] * T)) * s[:, None, None]
        errs.append(np.max(np.abs(f[0] - exact)))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates >= rate), (errs, rates)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_advection_conserves_totals_periodic(p):
    """sum_e sum_s W_s |J| div_s telescopes to zero on a periodic mesh."""
    pb = _problem((3, 2, 2), p)
    rng = np.random.default_rng(3 + p)
    f = rng.uniform(0.1, 2.0, (1, pb.vg.size, pb.mesh.n_elem, pb.Ns))
    div = pb.divergence(f)
    tot = pb.totals(div)
    scale = np.max(np.abs(pb.totals(np.abs(div))))
    assert np.all(np.abs(tot) <= 1e-14 * scale)


def test_element_residual_from_its_block_equals_the_whole_mesh():
    """The single-element residual evaluated on a 3x3x3 block (the element and
    its neighbours, periodic wrap taken by the caller) equals the whole-mesh
    residual at that element: advection and BGK source, ES with G."""
    from oracle import stage as ost
    from paper_2312_06567_gb300 import workloads as W
    wl = W.reduced(W.normal_shock_tube(mach=3.0), mesh_n=(4, 3, 5), vel_n=(13, 9, 11)).replace(
        p=2, periodic=(True, True, True), dirichlet=None, vel_lo=(-9.0, -8.0, -8.0), vel_hi=(11.0, 8.0, 8.0))
    pb = ost.problem_from_workload(wl)
    f = W.random_anisotropic_state(wl, seed=21)
    R, _ = pb.rhs(f)
    n1, n2, n3 = wl.mesh_n
    for e in (0, 17, wl.n_elem - 1):
        c = (e % n1, (e // n1) % n2, e // (n1 * n2))
        idx = [((c[0] + d1) % n1) + n1 * (((c[1] + d2) % n2) + n2 * ((c[2] + d3) % n3))
               for d3 in (-1, 0, 1) for d2 in (-1, 0, 1) for d1 in (-1, 0, 1)]
        Re = ost.element_residual(pb.mesh.h, wl.p, pb.vg, pb.gas, f[:, :, idx, :])
        scale = np.abs(R[:, :, e, :]).max()
        assert np.max(np.abs(Re - R[:, :, e, :])) <= 1e-13 * scale


def test_slab_residual_from_three_slabs_equals_the_whole_mesh():
    """The residual of one first-axis slab evaluated from three consecutive
    slabs (the normal shock's layout: Dirichlet first-axis ends, periodic in
    the other two) equals the whole-mesh residual at both Dirichlet ends and
    in the interior: advection (incl. the Dirichlet exterior state) and the
    ES source with G."""
    from oracle import stage as ost
    from paper_2312_06567_gb300 import workloads as W
    wl = W.reduced(W.normal_shock_tube(mach=3.0), mesh_n=(6, 2, 3), vel_n=(13, 9, 11)).replace(
        p=2, vel_lo=(-9.0, -8.0, -8.0), vel_hi=(11.0, 8.0, 8.0))
    pb = ost.problem_from_workload(wl)
    f = W.random_anisotropic_state(wl, seed=23)
    R, _ = pb.rhs(f)
    n1, n2, n3 = wl.mesh_n
    for e1 in (0, 3, n1 - 1):
        first = min(max(e1 - 1, 0), n1 - 3)
        idx = [first + d1 + n1 * (i2 + n2 * i3) for i3 in range(n3) for i2 in range(n2) for d1 in range(3)]
        Rs = ost.slab_residual(pb.mesh.h, (n2, n3), wl.p, pb.vg, pb.gas, wl.dirichlet, f[:, :, idx, :], e1 - first)
        sel = [e1 + n1 * (i2 + n2 * i3) for i3 in range(n3) for i2 in range(n2)]
        scale = np.abs(R[:, :, sel, :]).max()
        assert np.max(np.abs(Rs - R[:, :, sel, :])) <= 1e-13 * scale, e1


def _mirror_case(p=2, with_g=True):
    """A box [0, L] x [0,1]^2 with specular faces at x = 0 and x = L, and the
    periodic doubled box [-L, L] holding the mirror image of the data."""
    from oracle import stage as ost
    from paper_2312_06567_gb300 import workloads as W
    base = W.reduced(W.normal_shock_tube(mach=3.0), mesh_n=(3, 2, 1), vel_n=(8, 7, 6)).replace(
        p=p, vel_lo=(-9.0, -8.0, -8.0), vel_hi=(9.0, 8.0, 8.0), mesh_lo=(0.0, 0.0, 0.0), mesh_hi=(3.0, 1.0, 1.0),
        delta=2.0 if with_g else 0.0)
    half = base.replace(periodic=(False, True, True), dirichlet={}, specular=((0, -1), (0, 1)))
    full = base.replace(mesh_n=(6, 2, 1), mesh_lo=(-3.0, 0.0, 0.0), mesh_hi=(3.0, 1.0, 1.0),
                        periodic=(True, True, True), dirichlet={}, specular=())
    return ost.problem_from_workload(half), ost.problem_from_workload(full), half


def test_specular_faces_equal_the_mirrored_periodic_domain():
    """FR with specular walls at x = 0 and x = L on [0, L] gives exactly the
    residual that the periodic domain [-L, L] gives on [0, L] when its data
    are the mirror image f(-x, R u) of the half-domain data: the exterior
    state of the reflecting face is what the mirrored neighbour presents."""
    from paper_2312_06567_gb300 import workloads as W
    ph, pf, half = _mirror_case()
    f = W.random_anisotropic_state(half, seed=31)                       # [C, Nu, 6 elems, Ns]
    C, Nu, Ne, Ns = f.shape
    q = half.p + 1
    mir = ph.mirror[0]
    # element e = e1 + 3 e2 (n = (3, 2, 1)); the full box has e1' = e1 + 3 on [0, L] and the
    # mirror image e1' = 2 - e1 on [-L, 0], nodes mirrored along x (i1 -> q - 1 - i1)
    g = np.empty((C, Nu, 12, Ns))
    f6 = f.reshape(C, Nu, 2, 3, q, q, q)                             # [c, k, e2, e1, i3, i2, i1]
    full = np.empty((C, Nu, 2, 6, q, q, q))
    full[:, :, :, 3:] = f6
    full[:, :, :, :3] = f6[:, mir][:, :, :, ::-1, :, :, ::-1]
    g = full.reshape(C, Nu, 12, Ns)
    Rh, _ = ph.rhs(f)
    Rf, _ = pf.rhs(g)
    Rf6 = Rf.reshape(C, Nu, 2, 6, Ns)[:, :, :, 3:].reshape(C, Nu, 6, Ns)
    assert np.max(np.abs(Rh - Rf6)) <= 1e-12 * np.max(np.abs(Rh))


def test_specular_walls_conserve_mass_energy_and_tangential_momentum():
    from paper_2312_06567_gb300 import workloads as W
    ph, _, half = _mirror_case()
    f = W.random_anisotropic_state(half, seed=32)
    t0 = ph.totals(f)
    f1, _ = ph.step(f, half.dt())
    t1 = ph.totals(f1)
    scale = np.abs(t0).max()
    for i in (0, 2, 3, 4):                                   # mass, tangential momenta, energy
        assert abs(t1[i] - t0[i]) <= 1e-13 * scale, i
    assert abs(t1[1] - t0[1]) > 1e-10 * scale                # the walls push on the normal momentum
