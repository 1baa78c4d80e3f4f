"""Parity at the sphere O-grid's full size (12x24x24 hex, p=1, 40^3
velocities, F and G: 3.54e9 DOF) on sampled elements, mixed form in the
benchmark's launch configuration.

The state (a deterministic non-equilibrium mixture around the freestream) is
generated on the device in FP64 per velocity chunk and stored in FP32; the
3x3x3 element blocks around a few sampled elements (a periodic-azimuth wrap,
an inner element, one next to the farfield layer) are generated on the host
from the same per-point parameters.  The GPU computes the residual and a
Runge--Kutta stage of the whole state; the oracle computes the sampled
elements from their blocks (curved.element_residual, pinned against the
whole-mesh residual).  The mixed form's contract, the moments of the stage
output within 1e-5 of the point's scale, holds; the residual and the output
are compared velocity by velocity too, at 5e-5 of max|f| over the element's
block times its advection rate plus max|S|: the FP32 Newton engine stops at a
scaled residual of 1e-6 and the exact moment correction's basis (1, c,
|c|^2/2) absorbs a theta' error only for an isotropic T', so with this state's
ES anisotropy (+-30%) and velocity tails where |c|^2/(2 theta) reaches ~30, a
few 1e-5 of the equilibrium's shape remain (the box's full-size test, with
milder tails, meets 1e-5 there).  The FP64 form does not fit
beside the test's buffers at this size (3 x 57 GB of context state plus the
input, residual and stage output) and is covered at smaller sizes."""
import numpy as np
import pytest

from oracle import bgk as obgk
from oracle import curved
from oracle.velocity import VelocityGrid
from paper_2312_06567_gb300 import workloads as W

pytestmark = pytest.mark.gpu

CELLS = ((1, 5, 0), (6, 12, 13), (10, 20, 23))          # (radial, polar, azimuth) indices


@pytest.fixture(scope="module")
def lib(libbgk, cuda_device):
    from paper_2312_06567_gb300 import bgk
    return bgk


def _block(wl, c):
    n1, n2, n3 = wl.mesh_n
    return [(c[0] + d1) + n1 * ((c[1] + d2) + n2 * ((c[2] + d3) % n3))
            for d3 in (-1, 0, 1) for d2 in (-1, 0, 1) for d1 in (-1, 0, 1)]


@pytest.fixture(scope="module")
def ogrid_state(cuda_device):
    import torch
    wl = W.sphere_ogrid()
    free = torch.cuda.mem_get_info()[0]
    if free < 200e9:
        pytest.skip("needs ~200 GB of free device memory, %.0f GB free" % (free / 1e9))
    x = W.node_positions(wl)
    xf = x.reshape(-1, 3)
    P = xf.shape[0]
    elem = np.repeat(np.arange(wl.n_elem), wl.n_sol)
    par = W.mixture_params(wl, xf, elem)
    u = W.velocity_nodes(wl)
    host = {}
    for c in CELLS:
        blk = _block(wl, c)
        pts = (np.asarray(blk)[:, None] * wl.n_sol + np.arange(wl.n_sol)[None, :]).ravel()
        sub = {k: v[pts] for k, v in par.items()}
        F = W.mixture_values(sub, u, np.exp)
        host[c] = (blk, np.stack([F, sub["gfac"][None, :] * F]), x[blk])
    dpar = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in par.items()}
    du = torch.from_numpy(u).cuda()
    f32 = torch.empty((2, wl.n_vel, P), dtype=torch.float32, device="cuda")
    step = 256
    for k0 in range(0, wl.n_vel, step):
        k1 = min(wl.n_vel, k0 + step)
        F = W.mixture_values(dpar, du[k0:k1], torch.exp)
        f32[0, k0:k1] = F.float()
        f32[1, k0:k1] = (dpar["gfac"][None, :] * F).float()
        del F
    del dpar
    torch.cuda.empty_cache()
    yield wl, f32.view(2, wl.n_vel, wl.n_elem, wl.n_sol), host
    del f32
    torch.cuda.empty_cache()


def test_ogrid_full_size_mixed_residual_and_stage_on_sampled_elements(lib, ogrid_state):
    import torch
    wl, f, host = ogrid_state
    dt = wl.dt()
    with lib.Solver(wl, lib.BGK_MIXED) as s:
        s.set_state(f)
        s.tune_stage(dt, reps=1)
        r = torch.empty_like(f)
        s.rhs(f, r)
        out = torch.empty_like(f)
        s.stage(f, f, out, 0.75, 0.25, 0.25 * dt)
    vg = VelocityGrid(wl.vel_n, wl.vel_lo, wl.vel_hi)
    gas = obgk.Gas(delta=wl.delta, Pr=wl.Pr, mu_ref=wl.mu_ref, theta_ref=wl.theta_ref, theta_S=wl.theta_S)
    for c, (blk, fblk, x27) in host.items():
        e = c[0] + wl.mesh_n[0] * (c[1] + wl.mesh_n[1] * c[2])
        f27 = fblk.reshape(2, wl.n_vel, 27, wl.n_sol).astype(np.float32).astype(np.float64)
        R, S = curved.element_residual(wl.p, vg, gas, x27, f27, with_source=True)
        mesh = curved.CurvedMesh((3, 3, 3), (False,) * 3, x27, wl.p)
        a = np.abs(np.einsum("kn,dnabc->kdabc", vg.u, mesh.S[13])).sum(axis=1)
        adv = (a / mesh.J[13][None]).reshape(wl.n_vel, -1).max(axis=1)
        fe = f27[:, :, 13, :]
        # the upwind flux brings in the face neighbours' traces, which in the
        # velocity tails of this state (its mean is 27 thermal speeds off the
        # grid centre) can exceed the element's own f by orders of magnitude:
        # the advection scale takes max|f| over the block.  In the far tails
        # the FP32 state underflows to 0 (and so does the oracle's source): the
        # scale there is floored at 1e-25 of the largest one, far below FP32
        # resolution relative to it
        fnb = np.abs(f27).reshape(2, wl.n_vel, -1).max(axis=2)
        scale = fnb * adv[None, :] + np.abs(S).max(axis=2)
        scale = np.maximum(scale, 1e-25 * scale.max())
        r_e = r[:, :, e, :].double().cpu().numpy()
        err = float(np.max(np.abs(r_e - R).max(axis=2) / scale))
        assert err <= 5e-5, (c, err)
        o_e = out[:, :, e, :].double().cpu().numpy()
        o_ora = fe + (0.25 * dt) * R
        sc = np.abs(fe).max(axis=2) + 0.25 * dt * (np.abs(R).max(axis=2) + np.abs(S).max(axis=2))
        sc = np.maximum(sc, 1e-25 * sc.max())
        assert float(np.max(np.abs(o_e - o_ora).max(axis=2) / sc)) <= 5e-5, c
        # the mixed form's contract: per point |d rho|/rho, |d rho U|_inf /
        # (rho sqrt(theta)), |d E|/E of the stage output within 1e-5 (at this
        # speed the raw second moments are ~700 rho theta, so their FP32
        # storage rounding alone is ~1e-5 of rho theta: they are not compared
        # slot by slot)
        m_e = obgk.raw_moments(o_e[0], o_e[1], vg)
        m_o = obgk.raw_moments(o_ora[0], o_ora[1], vg)
        rho, U, E, th, _, _ = obgk.macroscopic(m_o, gas)
        rho_e, U_e, E_e, _, _, _ = obgk.macroscopic(m_e, gas)
        q_err = max(np.max(np.abs(rho_e - rho) / rho),
                    np.max(np.abs(rho_e[:, None] * U_e - rho[:, None] * U).max(axis=1) / (rho * np.sqrt(th))),
                    np.max(np.abs(E_e - E) / E))
        assert q_err <= 1e-5, (c, q_err)
