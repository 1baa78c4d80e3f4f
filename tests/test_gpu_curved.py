"""Curvilinear meshes, diffuse walls and closed faces on the GPU against the
oracle: the residual and one SSP-RK3 step (FP64 within 1e-12, mixed within
1e-5 of the per-velocity scale; moments within 1e-5 of the point's scale),
exact free-stream preservation and conservation, the wall's zero mass flux,
the sphere O-grid, and the configurations the library declines."""
import numpy as np
import pytest

from oracle import bgk as obgk
from oracle import curved
from paper_2312_06567_gb300 import workloads as W

from test_gpu_parity import moment_err, slab_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib(libbgk, cuda_device):
    from paper_2312_06567_gb300 import bgk
    return bgk


def _skew_warp(t):
    w = np.sin(2 * np.pi * t[..., 0] + 0.4) * np.sin(2 * np.pi * t[..., 1] + 1.1) * np.sin(2 * np.pi * t[..., 2] + 2.3)
    return t + np.stack([0.05 * w, -0.04 * w, 0.03 * w], axis=-1)


def _bend(t):
    return np.stack([t[..., 0] + 0.05 * np.sin(2 * np.pi * t[..., 1]) * np.cos(2 * np.pi * t[..., 2]),
                     t[..., 1] + 0.04 * np.sin(np.pi * t[..., 0]), t[..., 2]], axis=-1)


def _warped_es(p, n=(3, 2, 2), vel_n=(10, 9, 8)):
    return W.wavy_periodic_box(p=p, n=n, vel_n=vel_n, Pr=2.0 / 3.0).replace(mapping=_skew_warp)


def _channel(p, delta=2.0, theta_w=0.4, vel_n=(12, 9, 8)):
    return W.wavy_periodic_box(p=p, n=(3, 2, 2), vel_n=vel_n).replace(
        periodic=(False, True, True), delta=delta, Pr=0.72, mapping=_bend,
        vel_lo=(-7.0, -6.0, -6.0), vel_hi=(7.0, 6.0, 6.0),
        diffuse={(0, -1): ((0.0, 0.3, 0.0), theta_w), (0, 1): ((0.0, 0.0, 0.0), 1.5 * theta_w)})


def _ogrid(p=1):
    return W.sphere_ogrid(n=(2, 4, 4), p=p, vel_n=(10, 9, 9), umax=7.0, mach=2.0, kn=0.05)


def _closed_box(p=2):
    return W.reduced(W.normal_shock_tube(mach=3.0), mesh_n=(3, 2, 2), vel_n=(13, 9, 11)).replace(
        p=p, vel_lo=(-9.0, -8.0, -8.0), vel_hi=(11.0, 8.0, 8.0), dirichlet={}, closed=((0, -1), (0, 1)))


CASES = {
    "warped_es_p1": lambda: _warped_es(1),
    "warped_es_p2": lambda: _warped_es(2),
    "warped_es_p3": lambda: _warped_es(3, n=(2, 2, 2)),
    "channel_diffuse_fg_p2": lambda: _channel(2),
    "ogrid_p1": lambda: _ogrid(1),
    "closed_box_p2": lambda: _closed_box(2),
}


def _problem(wl):
    return curved.problem_from_workload(wl, W.node_positions(wl))


def _state(wl, seed):
    if wl.mapping is not None and wl.name.startswith("sphere"):
        # random mixture around the freestream: the O-grid's poles take no data
        return W.random_anisotropic_state(wl, seed=seed, spread=0.2)
    return W.random_anisotropic_state(wl, seed=seed)


def _rate(pb):
    """Per velocity: max over nodes of sum_d |u . S^d| / J (the advection rate)."""
    a = np.abs(np.einsum("kn,ednabc->kdeabc", pb.vg.u, pb.mesh.S)).sum(axis=1)
    return (a / pb.mesh.J[None]).reshape(pb.vg.size, -1).max(axis=1)


def _rhs_err(r_gpu, r_ora, f, pb, S):
    C, Nu = f.shape[:2]
    scale = np.abs(f).reshape(C, Nu, -1).max(axis=2) * _rate(pb)[None, :] + np.abs(S).reshape(C, Nu, -1).max(axis=2)
    d = np.abs(r_gpu - r_ora).reshape(C, Nu, -1).max(axis=2)
    return float(np.max(d / np.maximum(scale, 1e-300)))


@pytest.mark.parametrize("name", list(CASES))
def test_fp64_rhs_and_step_match_oracle(lib, name):
    wl = CASES[name]()
    pb = _problem(wl)
    f = _state(wl, seed=51)
    r_ora, info = pb.rhs(f)
    S = r_ora + pb.divergence(f)
    f1_ora, _ = pb.step(f, wl.dt())
    with lib.Solver(wl, lib.BGK_FP64) as s:
        assert np.allclose(s.node_coords(), W.node_positions(wl), rtol=0.0, atol=1e-13)
        s.set_state(f)
        r = s.rhs(f)
        assert s.step(wl.dt(), 1) == lib.BGK_OK
        f1 = s.get_state()
        t_gpu = s.totals()
    assert _rhs_err(r, r_ora, f, pb, S) <= 1e-12
    assert slab_err(f1, f1_ora) <= 1e-12
    t_ora = pb.totals(f1_ora)
    assert np.all(np.abs(t_gpu - t_ora) <= 1e-12 * np.max(np.abs(pb.totals(np.abs(f1_ora)))))


@pytest.mark.parametrize("name", list(CASES))
def test_mixed_rhs_step_and_moments_match_oracle(lib, name):
    wl = CASES[name]()
    pb = _problem(wl)
    f32 = _state(wl, seed=52).astype(np.float32)
    f = f32.astype(np.float64)
    r_ora, info = pb.rhs(f)
    S = r_ora + pb.divergence(f)
    f1_ora, _ = pb.step(f, wl.dt())
    m1_ora = obgk.raw_moments(f1_ora[0].reshape(wl.n_vel, -1),
                              f1_ora[1].reshape(wl.n_vel, -1) if wl.n_comp == 2 else None, pb.vg)
    for fp32_sums in (False, True):
        with lib.Solver(wl, lib.BGK_MIXED) as s:
            s.set_qprime_engine(fp32_sums)
            s.set_state(f32)
            r = s.rhs(f32).astype(np.float64)
            assert s.step(wl.dt(), 1) == lib.BGK_OK
            f1 = s.get_state().astype(np.float64)
            m1 = s.moments()
        if not fp32_sums:
            assert _rhs_err(r, r_ora, f, pb, S) <= 1e-5
            assert slab_err(f1, f1_ora) <= 1e-5
        assert moment_err(m1, m1_ora, wl.delta) <= 1e-5


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_free_stream_is_preserved(lib, precision):
    """A uniform Maxwellian on the warped periodic mesh stays uniform: the
    residual is zero up to rounding (FP64 1e-12, FP32 1e-5 of u f S/J)."""
    wl = _warped_es(2, vel_n=(8, 8, 8)).replace(Pr=1.0)
    pb = _problem(wl)
    x = W.node_positions(wl)
    f = W.maxwellian_state(wl, x, fields=(np.full(x.shape[:-1], 1.2), np.zeros(x.shape), np.full(x.shape[:-1], 0.9)))
    prec = lib.BGK_FP64 if precision == "fp64" else lib.BGK_MIXED
    dt = np.float64 if precision == "fp64" else np.float32
    with lib.Solver(wl, prec) as s:
        s.set_state(f.astype(dt))
        r = s.rhs(f.astype(dt)).astype(np.float64)
    scale = np.abs(f).reshape(wl.n_vel, -1).max(axis=1) * _rate(pb)
    err = np.abs(r[0]).reshape(wl.n_vel, -1).max(axis=1) / scale
    assert float(err.max()) <= (1e-12 if precision == "fp64" else 1e-5)


def test_warped_periodic_fp64_step_conserves_totals(lib):
    """Three FP64 steps on the warped periodic mesh: totals kept to 1e-12."""
    wl = _warped_es(3, n=(3, 3, 2), vel_n=(10, 9, 8))
    f = _state(wl, seed=53)
    with lib.Solver(wl, lib.BGK_FP64) as s:
        s.set_state(f)
        t0 = s.totals()
        scale = np.max(np.abs(t0))
        for _ in range(3):
            assert s.step(wl.dt(), 1) == lib.BGK_OK
            t1 = s.totals()
            assert np.all(np.abs(t1 - t0) <= 1e-12 * scale), (t1 - t0) / scale
            t0 = t1


def _residual_rates(lib, wl, f, curvy):
    """|sum W_x sum_k w psi R| dt / sum W_x sum_k w |psi f| of the mixed residual
    for psi = 1, u1, u3, |u|^2/2 (+ G), with the quadrature the stage conserves
    (W_s / (1/J)_32 on the curvilinear path, W_s |J| on the box)."""
    with lib.Solver(wl, lib.BGK_MIXED) as s:
        s.set_state(f)
        r = s.rhs(f).astype(np.float64)
    pb = _problem(wl)
    W3 = np.einsum("i,j,k->ijk", pb.fr.wq, pb.fr.wq, pb.fr.wq).reshape(-1)[None]
    J = pb.mesh.J.reshape(wl.n_elem, -1)
    Wx = W3 / (1.0 / J).astype(np.float32).astype(np.float64) if curvy else W3 * J
    w, u = pb.vg.w, pb.vg.u
    fd = f.astype(np.float64)
    out = []
    for psis in ((np.ones(len(w)), None), (u[:, 0], None), (u[:, 2], None),
                 (0.5 * np.sum(u * u, axis=1), np.ones(len(w)))):
        rate = sum(np.einsum("k,kes,es->", w * ps, r[c], Wx) for c, ps in enumerate(psis[:wl.n_comp]) if ps is not None)
        tot = sum(np.einsum("k,kes,es->", w * np.abs(ps), np.abs(fd[c]), Wx)
                  for c, ps in enumerate(psis[:wl.n_comp]) if ps is not None)
        out.append(abs(rate) * wl.dt() / tot)
    return np.array(out)


@pytest.mark.parametrize("name", ["warped_es_p1", "warped_es_p3", "closed_box_p2"])
def test_mixed_residual_is_conservative_for_smooth_data(lib, name):
    """Totals of the mixed residual of a smooth state (the Maxwellian of the
    case's initial field) within 5e-11 of their scale per time step, half the
    mixed form's drift bound: the advection telescopes exactly for the stored
    FP32 coefficients and its sums act on deviations; what remains is the
    FP32 rounding of the metric-variation term u.(S_face - S_node) f (a few
    1e-11 in momentum on the warped mesh) and of the FP32 equilibrium."""
    wl = CASES[name]()
    x = W.node_positions(wl)
    f = W.maxwellian_state(wl, x).astype(np.float32)
    r = _residual_rates(lib, wl, f, True)
    assert np.all(r <= 5e-11), r


@pytest.mark.parametrize("p", [1, 2, 3])
def test_mixed_residual_conservation_matches_the_affine_kernels(lib, p):
    """Random discontinuous states on the box: the curvilinear path (the box
    given as a mapping) conserves as well as the affine kernels do -- its
    worst total within twice theirs, whose floor here (up to ~2e-10) is set
    by the FP32 source of such states."""
    wl = W.reduced(W.normal_shock_tube(mach=3.0), mesh_n=(3, 2, 2), vel_n=(13, 9, 11)).replace(
        p=p, vel_lo=(-9.0, -8.0, -8.0), vel_hi=(11.0, 8.0, 8.0), periodic=(True, True, True), dirichlet={})
    lo, hi = np.asarray(wl.mesh_lo, dtype=np.float64), np.asarray(wl.mesh_hi, dtype=np.float64)
    wc = wl.replace(mapping=lambda t: lo + t * (hi - lo))
    for seed in (56, 57):
        f = W.random_anisotropic_state(wl, seed=seed).astype(np.float32)
        ra = _residual_rates(lib, wl, f, False)
        rc = _residual_rates(lib, wc, f, True)
        assert rc.max() <= max(2.0 * ra.max(), 2e-11), (rc, ra)


def test_mixed_conservation_drift_at_scale(lib):
    """2.3e8 DOF of the Taylor--Green physics on the warped 8x8x4 mesh (p=3,
    24^3 velocities, ES-BGK): mass, momentum and energy drift <= 1e-10 of
    their scale per step, FP64 totals of the stored FP32 state over 4 steps."""
    base = W.reduced(W.taylor_green_box(), mesh_n=(8, 8, 4))
    two_pi = 2.0 * np.pi
    wl = base.replace(mapping=lambda t: two_pi * _skew_warp(t), h_min_override=two_pi * 0.7 / 8)
    n = 4
    with lib.Solver(wl, lib.BGK_MIXED) as s:
        x = s.node_coords()
        rho, U, theta = wl.init(x)
        q = np.concatenate([rho.reshape(-1, 1), U.reshape(-1, 3), theta.reshape(-1, 1)], axis=1)
        s.set_maxwellian(q)
        t0 = s.totals()
        assert s.step(wl.dt(), n) == lib.BGK_OK
        s.set_state(s.get_state())
        t1 = s.totals()
    scale = np.array([t0[0]] * 4 + [t0[4]])
    assert np.all(np.abs(t1 - t0) / scale / n <= 1e-10), (t1 - t0) / scale / n


def test_diffuse_walls_conserve_mass_on_gpu(lib):
    """No mass crosses a diffuse wall: the mass total is kept through steps;
    the colder walls remove energy."""
    wl = _channel(2, theta_w=0.3)
    f = _state(wl, seed=54)
    with lib.Solver(wl, lib.BGK_FP64) as s:
        s.set_state(f)
        t0 = s.totals()
        for _ in range(2):
            assert s.step(wl.dt(), 1) == lib.BGK_OK
        t1 = s.totals()
    assert abs(t1[0] - t0[0]) <= 2e-12 * t0[0]
    assert t1[4] < t0[4]


def test_ogrid_graph_replay_matches_direct_launches(lib):
    """The sphere O-grid (wall, farfield, poles, periodic azimuth), mixed form:
    graph replay of the wall + Q' + stage launches is bit-identical to direct
    launches, and the direct launches run the wall kernel once per stage."""
    wl = _ogrid(1)
    x = W.node_positions(wl)
    rho, U, theta = wl.init(x)
    q = np.concatenate([np.broadcast_to(rho, x.shape[:-1]).reshape(-1, 1), U.reshape(-1, 3),
                        np.broadcast_to(theta, x.shape[:-1]).reshape(-1, 1)], axis=1)
    outs = []
    for graphs in (False, True):
        with lib.Solver(wl, lib.BGK_MIXED) as s:
            s.set_maxwellian(q)
            s.set_graphs(graphs)
            if not graphs:
                s.profile(True)
            assert s.step(wl.dt(), 3) == lib.BGK_OK
            if not graphs:
                prof = s.profile_read()
                assert prof["wall"][1] == 9 and prof["stage"][1] == 9
            outs.append(s.get_state())
    assert np.array_equal(outs[0], outs[1])
    assert np.all(np.isfinite(outs[0]))


def test_curvilinear_declines_what_it_does_not_support(lib):
    wl = _channel(2)
    with lib.Solver(wl, lib.BGK_MIXED) as s:
        s.set_state(_state(wl, seed=55).astype(np.float32))
        for v in ("async", "line", "line_wide", "half", "half_wide"):
            with pytest.raises(RuntimeError):
                s.set_stage_kernel(v, 4)
        s.set_stage_kernel("plain", 4)
        v, d, ms = s.tune_stage(wl.dt(), reps=1)
        assert v in ("auto", "plain")
        # the macroscopic diagnostics take the metric terms (not declined)
        assert np.all(np.isfinite(s.macro()))
