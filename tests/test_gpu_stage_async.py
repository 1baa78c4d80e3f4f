"""The asynchronous-copy mixed-form stage kernels against the plain one.

All variants evaluate the same FP32 expressions in the same order for every
point (the deviation-form FR advection, the corrected FP32 equilibrium, the
Runge--Kutta update and the error-free moment epilogue); only the way the
operands reach the threads (bulk copies into a shared-memory ring instead of
per-thread loads) and the work mapping (one node or one first-axis node line
per thread) differ.  So their states and moments must agree bit for bit, for
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


VARIANTS = ("async", "line", "line_wide", "half", "half_wide")

ASYNC_CASES = {
    # Q = 2: 32-element runs, all rows shorter than a run
    "sine_box_p1": lambda: W.periodic_sine_box(),
    "ragged_p1_dirichlet_x": lambda: _mild_shock(mesh_n=(3, 1, 2), vel_n=(13, 9, 11)).replace(p=1),
    # Q = 4: 4-element runs; rows of 3 (one short run) and of 6 (a full and a short run)
    "tgv_es_p3_ragged": lambda: _mild_es_box(),
    "tgv_es_p3_two_runs": lambda: _mild_es_box(mesh_n=(6, 3, 2), vel_n=(9, 8, 7)),
    "shock_fg_p3_dirichlet": lambda: _mild_shock(mesh_n=(6, 1, 1), vel_n=(16, 10, 9)).replace(p=3),
    "shock_fg_p3_dirichlet_3d": lambda: _mild_shock(mesh_n=(5, 2, 3), vel_n=(12, 9, 8)).replace(p=3),
    # Q = 3 (the line mapping on rows of whole 4-element groups): 16-element runs
    # with 4-element halo copies; one short run, a full and a short run, F/G with
    # Dirichlet x-ends, and a periodic single-component box
    "shock_fg_p2_rows8": lambda: _mild_shock(mesh_n=(8, 1, 2), vel_n=(13, 9, 8)),
    "shock_fg_p2_two_runs": lambda: _mild_shock(mesh_n=(20, 1, 1), vel_n=(12, 9, 8)),
    "es_box_p2_periodic": lambda: _mild_es_box(mesh_n=(4, 2, 2), p=2, vel_n=(9, 8, 7)),
}


def _smem_bytes(variant, q, C, depth):
    """Shared memory of an asynchronous stage kernel (the launcher's formula);
    a configuration above 200 KB is refused by design (and every variant but
    the line mapping at q = 3)."""
    ns = q ** 3
    if q == 3:
        if variant != "line":
            return 1 << 30
        eb, nq = 16, (7 if C == 2 else 6)
        nct = (eb * 9 + 31) // 32 * 32
        return depth * C * (4 * eb + 8) * ns * 4 + 3 * 2 * nq * nct * 4 + 16 * depth
    if variant == "async":
        eb = 256 // ns
        nct = eb * ns
        return depth * C * (4 * eb + 2) * ns * 4 + (11 * 8 + 14 * 4) * nct + 16 * depth
    wide = variant.endswith("_wide")
    eb = (4 if q == 4 else 16) * (2 if wide else 1)
    npt = q if variant.startswith("line") else q // 2
    nct = eb * q * q * (q // npt)
    nq = 7 if C == 2 else 6
    return depth * C * (4 * eb + 2) * ns * 4 + npt * 2 * nq * nct * 4 + 16 * depth


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
    for variant in VARIANTS:
        for depth in (2, 3, 6, 16):
            if _smem_bytes(variant, wl.p + 1, wl.n_comp, depth) > 200 * 1024:
                with pytest.raises(RuntimeError):
                    _run(lib, wl, f0, variant, depth, 2)
                continue
            r_a, f_a, m_a = _run(lib, wl, f0, variant, depth, 2)
            tag = (name, variant, depth)
            assert np.array_equal(r_a, r_p), (tag, float(np.max(np.abs(r_a - r_p))))
            assert np.array_equal(f_a, f_p), (tag, float(np.max(np.abs(f_a - f_p))))
            assert np.array_equal(m_a, m_p), (tag, float(np.max(np.abs(m_a - m_p))))


def test_async_stage_entry_point_with_fn(lib):
    """bgk_stage with f^n (a != 0) on caller buffers: async == plain."""
    wl = ASYNC_CASES["tgv_es_p3_two_runs"]()
    fn = W.random_anisotropic_state(wl, seed=6).astype(np.float32)
    fs = W.random_anisotropic_state(wl, seed=7).astype(np.float32)
    outs = []
    for variant in ("plain",) + VARIANTS:
        with lib.Solver(wl, lib.BGK_MIXED) as s:
            s.set_stage_kernel(variant, 4)
            s.set_state(fs)          # the Q' solve reads the moments of f_in itself
            import torch
            dn = torch.from_numpy(fn).cuda()
            ds = torch.from_numpy(fs).cuda()
            do = torch.empty_like(ds)
            s.stage(dn, ds, do, 0.75, 0.25, 0.25 * wl.dt())
            outs.append(do.cpu().numpy())
    for o in outs[1:]:
        assert np.array_equal(outs[0], o)


def test_async_stage_unsupported_configurations(lib):
    # p = 2 on rows of 6 elements: element slabs of 27 floats, rows not whole
    # 4-element (16-byte) groups
    wl = _mild_shock()
    with lib.Solver(wl, lib.BGK_MIXED) as s:
        for variant in VARIANTS:
            with pytest.raises(RuntimeError):
                s.set_stage_kernel(variant, 6)
        s.set_stage_kernel("auto", 6)           # falls back to the plain kernel
        with pytest.raises(RuntimeError):
            s.set_stage_kernel("auto", 1)       # depth out of range
        with pytest.raises(RuntimeError):
            s.set_stage_kernel("auto", 17)
    with lib.Solver(ASYNC_CASES["sine_box_p1"](), lib.BGK_FP64) as s:
        for variant in VARIANTS:
            with pytest.raises(RuntimeError):
                s.set_stage_kernel(variant, 6)


def test_async_stage_bitwise_at_scale(lib):
    """2.3e8 DOF of the Taylor--Green physics (8x8x4 hex, p=3, 24^3
    velocities), the configuration the benchmark's stage kernel runs in:
    one SSP-RK3 step, async == plain for every state value and moment."""
    import torch
    wl = W.reduced(W.taylor_green_box(), mesh_n=(8, 8, 4))
    res = []
    for variant in ("plain",) + VARIANTS:
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
    for f, m in res[1:]:
        assert torch.equal(res[0][0], f)
        assert np.array_equal(res[0][1], m)


def test_tuner_keeps_state_and_picks_a_supported_kernel(lib):
    wl = ASYNC_CASES["tgv_es_p3_two_runs"]()
    f0 = W.random_anisotropic_state(wl, seed=8).astype(np.float32)
    with lib.Solver(wl, lib.BGK_MIXED) as s:
        s.set_state(f0)
        v, d, ms = s.tune_stage(wl.dt(), reps=1)
        assert v in ("plain",) + VARIANTS and 2 <= d <= 16 and ms > 0.0
        assert np.array_equal(s.get_state(), f0)
        assert s.step(wl.dt(), 1) == lib.BGK_OK
        f1 = s.get_state()
    _, f_p, _ = _run(lib, wl, f0, "plain", 6, 1)
    assert np.array_equal(f1, f_p)


def test_velocity_blocking_changes_only_the_last_bits(lib):
    """bgk_set_velocity_blocks regroups the moment partials (and the stage
    grid); two steps agree with the default blocking within the mixed form's
    1e-5, and the blocking is reported back; counts above the maximum are
    refused."""
    wl = ASYNC_CASES["tgv_es_p3_two_runs"]()
    f0 = W.random_anisotropic_state(wl, seed=9).astype(np.float32)
    outs = {}
    for n in (0, 1, 3, 5):
        with lib.Solver(wl, lib.BGK_MIXED) as s:
            s.set_stage_kernel("line", 2)
            nb, per, mx = s.velocity_blocks()
            assert 1 <= nb <= mx and per % wl.vel_n[0] == 0 and nb * per >= wl.n_vel
            if n:
                s.set_velocity_blocks(n)
                nb, per, _ = s.velocity_blocks()
                lines = wl.n_vel // wl.vel_n[0]
                assert per == -(-lines // n) * wl.vel_n[0] and nb == -(-wl.n_vel // per)
            with pytest.raises(RuntimeError):
                s.set_velocity_blocks(mx + 1)
            s.set_state(f0)
            assert s.step(wl.dt(), 2) == lib.BGK_OK
            outs[n] = (s.get_state().astype(np.float64), s.moments())
    f_ref, m_ref = outs[0]
    scale = np.abs(f_ref).reshape(f_ref.shape[0], f_ref.shape[1], -1).max(axis=2)[:, :, None, None]
    for n, (f, m) in outs.items():
        assert np.max(np.abs(f - f_ref) / np.maximum(scale, 1e-300)) <= 1e-5, n
        assert np.max(np.abs(m - m_ref) / np.maximum(np.abs(m_ref).max(axis=0), 1e-300)) <= 1e-5, n
