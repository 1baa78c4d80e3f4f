"""The asynchronous-copy mixed-form stage kernel against the plain one.

Both kernels evaluate the same FP32 expressions in the same order (the
deviation-form FR advection, the corrected FP32 equilibrium, the Runge--Kutta
update and the error-free moment epilogue); only the way the operands reach
the threads differs (bulk copies into a shared-memory ring instead of
per-thread loads).  So their states and moments must agree bit for bit, for
every copy-ring depth, on ragged element runs (first mesh axis not a multiple
of the run length), Dirichlet faces, two-component (F, G) states and the
Runge--Kutta stages with and without f^n.  The plain kernel is itself checked
against the FP64 oracle in test_gpu_mixed.py.
"""
import numpy as np
import pytest

from paper_2312_06567_gb300 import workloads as W

from test_gpu_parity import _mild_es_box, _mild_shock

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib(libbgk, cuda_device):
    from paper_2312_06567_gb300 import bgk
    return bgk


ASYNC_CASES = {
    # Q = 2: 32-element runs, all rows shorter than a run
    "sine_box_p1": lambda: W.periodic_sine_box(),
    "ragged_p1_dirichlet_x": lambda: _mild_shock(mesh_n=(3, 1, 2), vel_n=(13, 9, 11)).replace(p=1),
    # Q = 4: 4-element runs; rows of 3 (one short run) and of 6 (a full and a short run)
    "tgv_es_p3_ragged": lambda: _mild_es_box(),
    "tgv_es_p3_two_runs": lambda: _mild_es_box(mesh_n=(6, 3, 2), vel_n=(9, 8, 7)),
    "shock_fg_p3_dirichlet": lambda: _mild_shock(mesh_n=(6, 1, 1), vel_n=(16, 10, 9)).replace(p=3),
    "shock_fg_p3_dirichlet_3d": lambda: _mild_shock(mesh_n=(5, 2, 3), vel_n=(12, 9, 8)).replace(p=3),
}


def _run(lib, wl, f0, variant, depth, steps):
    with lib.Solver(wl, lib.BGK_MIXED) as s:
        s.set_stage_kernel(variant, depth)
        s.set_state(f0)
        r = s.rhs(f0)
        assert s.step(wl.dt(), steps) == lib.BGK_OK
        return r, s.get_state(), s.moments()


@pytest.mark.parametrize("name", list(ASYNC_CASES))
def test_async_stage_is_bitwise_plain_stage(lib, name):
    wl = ASYNC_CASES[name]()
    f0 = W.random_anisotropic_state(wl, seed=5).astype(np.float32)
    r_p, f_p, m_p = _run(lib, wl, f0, "plain", 6, 2)
    for depth in (2, 3, 6, 16):
        r_a, f_a, m_a = _run(lib, wl, f0, "async", depth, 2)
        assert np.array_equal(r_a, r_p), (name, depth, float(np.max(np.abs(r_a - r_p))))
        assert np.array_equal(f_a, f_p), (name, depth, float(np.max(np.abs(f_a - f_p))))
        assert np.array_equal(m_a, m_p), (name, depth, float(np.max(np.abs(m_a - m_p))))


def test_async_stage_entry_point_with_fn(lib):
    """bgk_stage with f^n (a != 0) on caller buffers: async == plain."""
    wl = ASYNC_CASES["tgv_es_p3_two_runs"]()
    fn = W.random_anisotropic_state(wl, seed=6).astype(np.float32)
    fs = W.random_anisotropic_state(wl, seed=7).astype(np.float32)
    outs = []
    for variant in ("plain", "async"):
        with lib.Solver(wl, lib.BGK_MIXED) as s:
            s.set_stage_kernel(variant, 4)
            s.set_state(fs)          # the Q' solve reads the moments of f_in itself
            import torch
            dn = torch.from_numpy(fn).cuda()
            ds = torch.from_numpy(fs).cuda()
            do = torch.empty_like(ds)
            s.stage(dn, ds, do, 0.75, 0.25, 0.25 * wl.dt())
            outs.append(do.cpu().numpy())
    assert np.array_equal(outs[0], outs[1])


def test_async_stage_unsupported_configurations(lib):
    # p = 2: element slabs of 27 floats are not whole 16-byte units
    wl = _mild_shock()
    with lib.Solver(wl, lib.BGK_MIXED) as s:
        with pytest.raises(RuntimeError):
            s.set_stage_kernel("async", 6)
        s.set_stage_kernel("auto", 6)           # falls back to the plain kernel
        with pytest.raises(RuntimeError):
            s.set_stage_kernel("auto", 1)       # depth out of range
        with pytest.raises(RuntimeError):
            s.set_stage_kernel("auto", 17)
    with lib.Solver(ASYNC_CASES["sine_box_p1"](), lib.BGK_FP64) as s:
        with pytest.raises(RuntimeError):
            s.set_stage_kernel("async", 6)


def test_async_stage_bitwise_at_scale(lib):
    """2.3e8 DOF of the Taylor--Green physics (8x8x4 hex, p=3, 24^3
    velocities), the configuration the benchmark's stage kernel runs in:
    one SSP-RK3 step, async == plain for every state value and moment."""
    import torch
    wl = W.reduced(W.taylor_green_box(), mesh_n=(8, 8, 4))
    res = []
    for variant in ("plain", "async"):
        with lib.Solver(wl, lib.BGK_MIXED) as s:
            s.set_stage_kernel(variant, 6)
            x = s.node_coords()
            rho, U, theta = wl.init(x)
            q = np.concatenate([rho.reshape(-1, 1), U.reshape(-1, 3), theta.reshape(-1, 1)], axis=1)
            s.set_maxwellian(q)
            assert s.step(wl.dt(), 1) == lib.BGK_OK
            f = torch.empty(s.shape, dtype=torch.float32, device="cuda")
            s.get_state(f)
            res.append((f, s.moments()))
    assert torch.equal(res[0][0], res[1][0])
    assert np.array_equal(res[0][1], res[1][1])
