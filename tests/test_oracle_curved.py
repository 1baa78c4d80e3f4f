"""Pins of the curvilinear oracle (metric terms, transformed FR residual,
diffuse walls, collapsed faces) against closed forms, the affine oracle and
exact conservation laws."""
import numpy as np
import pytest

from oracle import bgk, curved, stage
from oracle.fr import FR1D
from oracle.velocity import VelocityGrid
from paper_2312_06567_gb300 import workloads as W


def _affine_mapping(M, b):
    M = np.asarray(M, dtype=np.float64)

    def mapping(t):
        return t @ M.T + b
    return mapping


M_SHEAR = np.array([[1.0, 0.3, -0.2], [0.1, 0.8, 0.25], [-0.15, 0.2, 1.2]])


def _wl_mapped(mapping, n, p, periodic=(True, True, True), vel_n=(3, 4, 3), **kw):
    base = W.wavy_periodic_box(p=p, n=n, vel_n=vel_n)
    return base.replace(mapping=mapping, periodic=periodic, **kw)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_affine_metrics_are_the_cofactor_columns(p):
    """x = M t + b: J a^i = d_j X x d_k X with d_j X = M[:, j] / (2 n_j), and
    J = det(d X / d xi), at every node (closed form)."""
    n = (2, 3, 2)
    wl = _wl_mapped(_affine_mapping(M_SHEAR, np.array([0.3, -1.0, 2.0])), n, p)
    x = W.node_positions(wl)
    mesh = curved.CurvedMesh(n, wl.periodic, x, p)
    cols = [M_SHEAR[:, j] / (2.0 * n[j]) for j in range(3)]
    exact = [np.cross(cols[1], cols[2]), np.cross(cols[2], cols[0]), np.cross(cols[0], cols[1])]
    for i in range(3):
        got = mesh.S[:, i].reshape(mesh.n_elem, 3, -1)
        assert np.max(np.abs(got - exact[i][None, :, None])) <= 1e-12 * np.max(np.abs(exact[i]))
    detJ = np.linalg.det(np.stack(cols, axis=1))
    assert np.max(np.abs(mesh.J - detJ)) <= 1e-15


def test_trilinear_metrics_equal_the_cross_product_form_for_p2():
    """Trilinear elements (corners on a sphere shell), p = 2: X_l d_j X_m has
    degree <= 2 per direction, so the curl form is exact and equals the cross
    products d_2 X x d_3 X (and cyclic) of the trilinear map at the nodes."""
    p, n = 2, (2, 3, 4)
    ogrid = W.sphere_ogrid(n=n, p=1)
    xi = FR1D(p).xi
    q = p + 1
    x = np.empty((ogrid.n_elem, q ** 3, 3))
    exact = np.empty((ogrid.n_elem, 3, 3, q ** 3))
    n1, n2 = n[0], n[1]
    g3, g2, g1 = np.meshgrid(xi, xi, xi, indexing="ij")
    loc = np.stack([g1.ravel(), g2.ravel(), g3.ravel()], axis=1)            # [s, 3]
    for e in range(ogrid.n_elem):
        c = np.array([e % n1, (e // n1) % n2, e // (n1 * n2)], dtype=np.float64)
        corners = {}
        for a in (0, 1):
            for b in (0, 1):
                for cc in (0, 1):
                    t = (c + np.array([a, b, cc])) / np.asarray(n, dtype=np.float64)
                    corners[(a, b, cc)] = ogrid.mapping(t)
        X = np.zeros((q ** 3, 3))
        dX = np.zeros((3, q ** 3, 3))
        for (a, b, cc), v in corners.items():
            s = [(1 + (2 * a - 1) * loc[:, 0]) / 2, (1 + (2 * b - 1) * loc[:, 1]) / 2,
                 (1 + (2 * cc - 1) * loc[:, 2]) / 2]
            ds = [(2 * a - 1) / 2.0, (2 * b - 1) / 2.0, (2 * cc - 1) / 2.0]
            X += (s[0] * s[1] * s[2])[:, None] * v
            dX[0] += (ds[0] * s[1] * s[2])[:, None] * v
            dX[1] += (s[0] * ds[1] * s[2])[:, None] * v
            dX[2] += (s[0] * s[1] * ds[2])[:, None] * v
        x[e] = X
        exact[e, 0] = np.cross(dX[1], dX[2]).T
        exact[e, 1] = np.cross(dX[2], dX[0]).T
        exact[e, 2] = np.cross(dX[0], dX[1]).T
    mesh = curved.CurvedMesh(n, (False, False, True), x, p)
    got = mesh.S.reshape(ogrid.n_elem, 3, 3, -1)
    assert np.max(np.abs(got - exact)) <= 1e-13 * np.max(np.abs(exact))


@pytest.mark.parametrize("p", [1, 2, 3])
def test_discrete_metric_identity(p):
    """sum_i D_i S^i = 0 at every node of a curved mesh (the curl form)."""
    wl = W.wavy_periodic_box(p=p, n=(2, 3, 2), amp=0.08)
    mesh = curved.CurvedMesh(wl.mesh_n, wl.periodic, W.node_positions(wl), p)
    div = sum(curved._dxi(np.moveaxis(mesh.S[:, i], 1, -1), i, mesh.fr.D) for i in range(3))
    assert np.max(np.abs(div)) <= 1e-13 * np.max(np.abs(mesh.S))


def test_shell_volume_converges():
    """sum_e sum_s W_s J_s tends to the shell volume 4/3 pi (4^3 - 0.5^3) under
    refinement (p = 2: third-order geometry)."""
    exact = 4.0 / 3.0 * np.pi * (4.0 ** 3 - 0.5 ** 3)
    errs = []
    for k in (1, 2, 4):
        wl = W.sphere_ogrid(n=(3 * k, 4 * k, 8 * k), p=2)
        mesh = curved.CurvedMesh(wl.mesh_n, wl.periodic, W.node_positions(wl), wl.p)
        errs.append(abs(mesh.node_weights().sum() - exact) / exact)
    assert errs[2] < 2e-3
    assert errs[0] / errs[1] > 6.0 and errs[1] / errs[2] > 6.0, errs


def _shock_wl(p, mesh_n=(3, 2, 2), vel_n=(13, 9, 11), periodic=(False, True, True)):
    wl = W.reduced(W.normal_shock_tube(mach=3.0), mesh_n=mesh_n, vel_n=vel_n).replace(
        p=p, vel_lo=(-9.0, -8.0, -8.0), vel_hi=(11.0, 8.0, 8.0), periodic=periodic)
    if all(periodic):
        wl = wl.replace(dirichlet={})
    return wl


@pytest.mark.parametrize("p,periodic", [(1, (False, True, True)), (2, (False, True, True)),
                                        (3, (True, True, True))])
def test_axis_aligned_box_equals_the_affine_oracle(p, periodic):
    """The box given as node coordinates: residual (advection, Dirichlet faces,
    ES-BGK source with G) equal to the affine oracle's."""
    wl = _shock_wl(p, periodic=periodic)
    f = W.random_anisotropic_state(wl, seed=40 + p)
    Ra, _ = stage.problem_from_workload(wl).rhs(f)
    Rc, _ = curved.problem_from_workload(wl, W.node_positions(wl)).rhs(f)
    assert np.max(np.abs(Rc - Ra)) <= 1e-12 * np.max(np.abs(Ra))


@pytest.mark.parametrize("p", [1, 2])
def test_sheared_mesh_polynomial_exactness(p):
    """On a sheared affine mesh, data linear in x with the exact exterior state:
    div = u . grad f exactly at every node (pins the orientation of S)."""
    n = (2, 2, 3)
    wl = _wl_mapped(_affine_mapping(M_SHEAR, np.zeros(3)), n, p, periodic=(False, False, False),
                    vel_n=(3, 3, 2))
    x = W.node_positions(wl)
    vg = VelocityGrid(wl.vel_n, wl.vel_lo, wl.vel_hi)
    rng = np.random.default_rng(5)
    c0 = rng.uniform(1, 2, vg.size)
    b = rng.uniform(-1, 1, (vg.size, 3))
    mesh = curved.CurvedMesh(n, wl.periodic, x, p)
    q = p + 1
    x6 = x.reshape(mesh.n_elem, q, q, q, 3)

    def value(xx):
        return c0.reshape((-1,) + (1,) * (xx.ndim - 1)) + np.einsum("kn,...n->k...", b, xx)

    def exterior(d, side, fm):
        xl = np.moveaxis(x6, 3 - d, -2)                       # [e, a, b, line, 3]
        lw = mesh.fr.l_plus if side > 0 else mesh.fr.l_minus
        xf = np.einsum("j,eabjn->eabn", lw, xl)              # face points (affine: exact)
        return value(xf)[None]

    gas = bgk.Gas(delta=0.0, Pr=1.0, mu_ref=0.1)
    pb = curved.CurvedProblem(mesh, vg, gas, exterior=exterior)
    f = value(x)[None]
    div = pb.divergence(f)[0]
    exact = np.einsum("kn,kn->k", vg.u, b)[:, None, None] * np.ones_like(div)
    assert np.max(np.abs(div - exact)) <= 1e-12 * np.max(np.abs(exact))


@pytest.mark.parametrize("p", [1, 2, 3])
def test_curved_periodic_step_conserves_totals(p):
    """Full SSP-RK3 step (advection and ES-BGK source) on the warped periodic
    mesh: mass, momentum and energy totals to 1e-13."""
    wl = W.wavy_periodic_box(p=p, n=(2, 2, 3), vel_n=(9, 8, 7), amp=0.07, Pr=2.0 / 3.0)
    pb = curved.problem_from_workload(wl, W.node_positions(wl))
    f = W.random_anisotropic_state(wl, seed=11 + p)
    t0 = pb.totals(f)
    f1, _ = pb.step(f, wl.dt())
    t1 = pb.totals(f1)
    scale = pb.totals(np.abs(f))
    scale[1:4] = np.max(scale)
    assert np.all(np.abs(t1 - t0) <= 1e-13 * np.abs(scale)), (t1 - t0) / scale


def _skew_warp(t):
    w = np.sin(2 * np.pi * t[..., 0] + 0.4) * np.sin(2 * np.pi * t[..., 1] + 1.1) * np.sin(2 * np.pi * t[..., 2] + 2.3)
    return t + np.stack([0.05 * w, -0.04 * w, 0.03 * w], axis=-1)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_free_stream_is_preserved_exactly(p):
    """A uniform state on a warped (continuous) curvilinear mesh has zero
    advective residual: the metric divergence vanishes and both sides of every
    face see the same metric trace."""
    wl = W.wavy_periodic_box(p=p, n=(3, 2, 4), vel_n=(3, 2, 2)).replace(mapping=_skew_warp)
    pb = curved.problem_from_workload(wl, W.node_positions(wl))
    f = np.ones(pb.shape)
    scale = np.max(np.abs(pb.vg.u)) * np.max(np.abs(pb.mesh.S)) / np.min(pb.mesh.J)
    assert np.max(np.abs(pb.divergence(f))) <= 1e-12 * scale
    for d in range(3):
        Sd = np.moveaxis(pb.mesh.S[:, d], 1, -1)
        own = np.einsum("j,...j->...", pb.fr.l_plus, np.moveaxis(Sd, 3 - d, -1))
        assert np.max(np.abs(own - pb.mesh.face[(d, 1)])) <= 1e-13 * np.max(np.abs(pb.mesh.S))


def _stretch_shear(t):
    """Periodic curvilinear map whose x depends on t1 alone (so data depending on
    x only need refinement along t1), with y and z sheared and bent."""
    s1 = np.sin(2 * np.pi * t[..., 0])
    return np.stack([t[..., 0] + 0.05 * s1, t[..., 1] + 0.05 * s1,
                     t[..., 2] + 0.04 * np.cos(2 * np.pi * t[..., 0]) + 0.03 * np.sin(2 * np.pi * t[..., 1])], axis=-1)


@pytest.mark.parametrize("p,rate", [(1, 1.5), (2, 2.5)])
def test_collisionless_closed_form_converges_on_curved_mesh(p, rate):
    """Source off: f_k(x, t) = f_k(x - u_k t, 0) for sinusoidal data on a
    stretched and sheared periodic mesh; the nodal max error falls at least
    like h^(p+1/2)."""
    errs = []
    for n in (8, 16, 32):
        wl = W.wavy_periodic_box(p=p, n=(n, 2, 2), vel_n=(2, 2, 2)).replace(
            vel_lo=(-1, -1, -1), vel_hi=(1, 1, 1), mapping=_stretch_shear)
        x = W.node_positions(wl)
        pb = curved.problem_from_workload(wl, x)
        s = 1 + 0.1 * np.arange(pb.vg.size)
        u1 = pb.vg.u[:, 0]
        f = (1 + 0.5 * np.sin(2 * np.pi * x[..., 0])[None] * s[:, None, None])[None]
        T = 0.1
        dt = 0.05 * (1.0 / n) / (2 * p + 1)
        nsteps = int(np.ceil(T / dt))
        dt = T / nsteps
        for _ in range(nsteps):
            f, _ = pb.step(f, dt, collide=False)
        exact = 1 + 0.5 * np.sin(2 * np.pi * (x[None, ..., 0] - u1[:, None, None] * T)) * s[:, None, None]
        errs.append(np.max(np.abs(f[0] - exact)))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates >= rate), (errs, rates)


def _channel(p, walls, theta_w=1.0, delta=0.0, mapping=None, vel=(8, 7, 6), n=(3, 2, 2)):
    wl = W.wavy_periodic_box(p=p, n=n, vel_n=vel).replace(
        periodic=(False, True, True), delta=delta, vel_lo=(-6.0, -6.0, -6.0), vel_hi=(6.0, 6.0, 6.0),
        diffuse={(0, s): ((0.0, 0.0, 0.0), theta_w) for s in walls}, mapping=mapping)
    return wl


@pytest.mark.parametrize("delta,slide", [(0.0, 0.0), (2.0, 0.0), (2.0, 0.7)])
def test_gas_at_the_wall_state_is_steady(delta, slide):
    """Diffuse walls at (U_w, theta_w) around a uniform Maxwellian at (U_w,
    theta_w), U_w tangential (Pr = 1, grid symmetric in the normal axis):
    rho_w = rho, no jumps, q' = q, R = 0."""
    U_w = (0.0, slide, 0.0)
    wl = _channel(2, (-1, 1), theta_w=0.8, delta=delta, mapping=_affine_mapping(np.diag([1.0, 0.7, 1.1]), np.zeros(3)))
    wl = wl.replace(diffuse={k: (U_w, th) for k, (_, th) in wl.diffuse.items()})
    x = W.node_positions(wl)
    pb = curved.problem_from_workload(wl, x)
    U = np.zeros(x.shape)
    U[..., 1] = slide
    f = W.maxwellian_state(wl, x, fields=(np.full(x.shape[:-1], 1.3), U, np.full(x.shape[:-1], 0.8)))
    R, _ = pb.rhs(f)
    assert np.max(np.abs(R)) <= 1e-13 * np.max(np.abs(f)) * 10.0


@pytest.mark.parametrize("p", [1, 2])
def test_diffuse_walls_conserve_mass_and_exchange_energy(p):
    """Curved channel with diffuse walls at both ends of the first axis: no mass
    crosses a wall node, so the mass total is conserved through a full step
    (source included); a wall colder than the gas removes energy."""
    bend = lambda t: np.stack([t[..., 0] + 0.05 * np.sin(2 * np.pi * t[..., 1]) * np.cos(2 * np.pi * t[..., 2]),
                               t[..., 1] + 0.04 * np.sin(np.pi * t[..., 0]), t[..., 2]], axis=-1)
    wl = _channel(p, (-1, 1), theta_w=0.3, delta=2.0, mapping=bend)
    x = W.node_positions(wl)
    pb = curved.problem_from_workload(wl, x)
    f = W.random_anisotropic_state(wl, seed=60 + p)
    t0 = pb.totals(f)
    f1, _ = pb.step(f, wl.dt())
    t1 = pb.totals(f1)
    assert abs(t1[0] - t0[0]) <= 1e-13 * t0[0]
    assert t1[4] < t0[4] * (1 - 1e-6)


def test_wall_density_balances_the_outgoing_mass_flux():
    """rho_w at every wall node makes sum_k w u_n f (outgoing interior trace,
    incoming wall Maxwellian) vanish."""
    wl = _channel(2, (-1, 1), theta_w=0.5, mapping=None).replace(mapping=W._wavy(0.06))
    x = W.node_positions(wl)
    pb = curved.problem_from_workload(wl, x)
    f = W.random_anisotropic_state(wl, seed=70)
    q = pb.q
    fl = np.moveaxis(f.reshape(f.shape[:3] + (q, q, q)), 5, -1)
    fm = np.einsum("j,...j->...", pb.fr.l_minus, fl)
    rho_w = pb.wall_density(0, -1, fm)
    U_w, th = pb.diffuse[(0, -1)]
    M = bgk.maxwellian(pb.vg, np.array([1.0]), np.array([U_w]), np.array([th]))[:, 0]
    un = -np.einsum("kn,eabn->keab", pb.vg.u, pb.mesh.face[(0, -1)])
    wall = pb.mesh.nbr[(0, -1)] < 0
    trace = np.where(un > 0, fm[0], M[:, None, None, None] * rho_w[None])
    flux = np.einsum("k,keab->eab", pb.vg.w, un * trace)[wall]
    scale = np.einsum("k,keab->eab", pb.vg.w, np.abs(un) * np.abs(trace))[wall]
    assert np.all(np.abs(flux) <= 1e-14 * scale)


@pytest.mark.parametrize("theta_g,theta_w", [(1.0, 0.5), (0.6, 1.4)])
def test_wall_density_tends_to_the_half_space_flux_balance(theta_g, theta_w):
    """Gas at rest at (rho_g, theta_g) against a wall at theta_w: the mass
    carried toward the wall by a half-Maxwellian is rho sqrt(theta / 2 pi), so
    the balance gives rho_w = rho_g sqrt(theta_g / theta_w) (kinetic theory,
    independent of the discretisation).  On symmetric grids with a node at
    u_n = 0 the discrete rho_w converges to it at second order in the normal
    velocity spacing (the one-sided sums have a kink at u_n = 0)."""
    errs = []
    for n1 in (17, 33, 65):
        wl = W.wavy_periodic_box(p=1, n=(2, 1, 1), vel_n=(n1, 21, 21)).replace(
            periodic=(False, True, True), delta=0.0, vel_lo=(-7.0, -7.0, -7.0), vel_hi=(7.0, 7.0, 7.0),
            diffuse={(0, s): ((0.0, 0.0, 0.0), theta_w) for s in (-1, 1)}, mapping=None)
        x = W.node_positions(wl)
        pb = curved.problem_from_workload(wl, x)
        f = W.maxwellian_state(wl, x, fields=(np.full(x.shape[:-1], 1.3), np.zeros(x.shape),
                                              np.full(x.shape[:-1], theta_g)))
        q = pb.q
        fl = np.moveaxis(f.reshape(f.shape[:3] + (q, q, q)), 5, -1)
        fm = np.einsum("j,...j->...", pb.fr.l_minus, fl)
        rho_w = pb.wall_density(0, -1, fm)[pb.mesh.nbr[(0, -1)] < 0]
        exact = 1.3 * np.sqrt(theta_g / theta_w)
        errs.append(float(np.max(np.abs(rho_w - exact))) / exact)
    assert errs[-1] <= 5e-3, errs
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates >= 1.9), (errs, rates)


def test_closed_faces_conserve_every_total():
    """No flux crosses a closed face: a box closed at both ends of the first
    axis conserves all five totals through a full step."""
    wl = _shock_wl(2).replace(dirichlet={}, closed=((0, -1), (0, 1)))
    pb = curved.problem_from_workload(wl, W.node_positions(wl))
    f = W.random_anisotropic_state(wl, seed=80)
    t0 = pb.totals(f)
    f1, _ = pb.step(f, wl.dt())
    t1 = pb.totals(f1)
    scale = np.max(np.abs(pb.totals(np.abs(f))))
    assert np.all(np.abs(t1 - t0) <= 1e-13 * scale)


def test_ogrid_geometry_and_one_step():
    """The sphere O-grid: positive Jacobian at every node (pole elements
    included), pole face vectors much smaller than the others, and one full
    step from the freestream stays finite and positive in mass."""
    wl = W.sphere_ogrid(n=(2, 4, 4), vel_n=(6, 6, 6), umax=6.0, mach=1.5)
    x = W.node_positions(wl)
    pb = curved.problem_from_workload(wl, x)
    assert np.all(pb.mesh.J > 0)
    pole = np.abs(pb.mesh.face[(1, -1)][pb.mesh.nbr[(1, -1)] < 0]).max()
    assert pole < 0.05 * np.abs(pb.mesh.face[(0, 1)]).max()
    f = W.maxwellian_state(wl, x)
    f1, infos = pb.step(f, wl.dt())
    assert np.all(np.isfinite(f1))
    assert pb.totals(f1)[0] > 0


def test_curved_element_residual_from_its_block_equals_the_whole_mesh():
    """The single-element residual of a curvilinear element on its 3x3x3 block
    (node coordinates and state of the block) equals the whole-mesh residual
    at that element: the sphere O-grid (periodic azimuth wrap included), F and G."""
    wl = W.sphere_ogrid(n=(4, 5, 6), vel_n=(8, 7, 7), umax=6.0, mach=1.2, kn=0.05)
    x = W.node_positions(wl)
    pb = curved.problem_from_workload(wl, x)
    f = W.random_anisotropic_state(wl, seed=90, spread=0.2)
    R, _ = pb.rhs(f)
    n1, n2, n3 = wl.mesh_n
    for c in ((1, 2, 0), (2, 3, 5), (2, 1, 3)):
        e = c[0] + n1 * (c[1] + n2 * c[2])
        idx = [(c[0] + d1) + n1 * ((c[1] + d2) + n2 * ((c[2] + d3) % n3))
               for d3 in (-1, 0, 1) for d2 in (-1, 0, 1) for d1 in (-1, 0, 1)]
        Re = curved.element_residual(wl.p, pb.vg, pb.gas, x[idx], f[:, :, idx, :])
        scale = np.abs(R[:, :, e, :]).max()
        assert np.max(np.abs(Re - R[:, :, e, :])) <= 1e-13 * scale


@pytest.mark.parametrize("make", [lambda: W.sphere_ogrid(n=(3, 4, 6), p=2),
                                  lambda: W.wavy_periodic_box(p=3, n=(2, 3, 2), amp=0.06)])
def test_workload_geometry_is_continuous_across_faces(make):
    """The generators sample the analytic map at each element's GLL points, so
    the degree-p interpolants of neighbouring elements agree on their shared
    face (the continuity that exact free-stream preservation rests on); periodic
    translations of the box are removed before comparing."""
    wl = make()
    x = W.node_positions(wl)
    q = wl.p + 1
    fr = FR1D(wl.p)
    x6 = x.reshape(wl.n_elem, q, q, q, 3)
    mesh = curved.CurvedMesh(wl.mesh_n, wl.periodic, x, wl.p)
    for d in range(3):
        xl = np.moveaxis(x6, 3 - d, -2)                       # [e, a, b, line, 3]
        hi = np.einsum("j,eabjn->eabn", fr.l_plus, xl)
        lo = np.einsum("j,eabjn->eabn", fr.l_minus, xl)
        nb = mesh.nbr[(d, 1)]
        inner = nb >= 0
        jump = hi[inner] - lo[nb[inner]]
        if wl.mapping is not None and wl.name.startswith("wavy"):
            jump -= np.round(jump)                             # the unit period of the box
        assert np.max(np.abs(jump)) <= 1e-12 * np.max(np.abs(x)), (d, np.max(np.abs(jump)))
