"""bgk_moments_noalloc against bgk_moments and the oracle (GPU, through the C-ABI).

The no-allocation entry point serves callers that cannot call cudaMalloc (a
framework that already holds the whole memory pool, an allocation-free
real-time loop, a plugin host that forbids allocation) and so cannot create a
solver context; it keeps its scratch in a fixed device array inside the
library.  This file is collected last so that a run that stops at the first
failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_2312_06567_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _moment_scale(m, delta):
    """Per-slot scales rho, rho sqrt(theta), rho theta (the parity tests' moment scale)."""
    rho = m[:, 0]
    U = m[:, 1:4] / rho[:, None]
    E = 0.5 * (m[:, 4] + m[:, 5] + m[:, 6]) + m[:, 10]
    theta = (2.0 / (3.0 + delta)) * (E - 0.5 * rho * np.sum(U * U, axis=1)) / rho
    r, rs, rt = rho, rho * np.sqrt(theta), rho * theta
    return np.stack([r, rs, rs, rs, rt, rt, rt, rt, rt, rt, np.maximum(m[:, 10], rt)], axis=1)


def _oracle_moments(wl, f):
    from oracle import bgk as obgk
    from oracle.velocity import VelocityGrid
    vg = VelocityGrid(wl.vel_n, wl.vel_lo, wl.vel_hi)
    C, Nu = f.shape[:2]
    F = f[0].reshape(Nu, -1)
    G = f[1].reshape(Nu, -1) if C == 2 else None
    return obgk.raw_moments(F, G, vg)


def _check_two_calls(wl, cuda_device, seeds=(1, 2), with_oracle=True):
    import torch
    from paper_2312_06567_gb300 import bgk

    _, vgrid, _ = bgk.descriptors(wl)
    P = wl.n_elem * wl.n_sol
    m_dev = torch.empty((P, 11), dtype=torch.float64, device=cuda_device)
    stream = torch.cuda.current_stream()
    with bgk.Solver(wl) as s:
        for seed in seeds:                      # calls in a row, different states
            f = W.random_anisotropic_state(wl, seed=seed)
            s.set_state(f)
            ref = s.moments()
            f_dev = torch.from_numpy(f).to(cuda_device)
            m_dev.fill_(np.nan)
            bgk.moments_noalloc(vgrid, f_dev, wl.n_comp, P, m_dev, stream)
            torch.cuda.synchronize()
            got = m_dev.cpu().numpy()
            assert np.all(np.isfinite(got))
            scale = _moment_scale(ref, wl.delta)
            assert np.max(np.abs(got - ref) / scale) <= 1e-13
            if with_oracle:
                ora = _oracle_moments(wl, f)
                assert np.max(np.abs(got - ora) / scale) <= 1e-13
            if wl.n_comp == 1:
                assert np.all(got[:, 10] == 0.0)


def test_noalloc_moments_match_context_moments_on_two_calls(libbgk, cuda_device):
    """F and G (delta = 2): two calls in a row equal bgk_moments and the oracle."""
    wl = W.reduced(W.normal_shock_tube(mach=3.0), mesh_n=(5, 1, 2), vel_n=(13, 9, 10)).replace(
        vel_lo=(-9.0, -8.0, -8.0), vel_hi=(11.0, 8.0, 8.0))
    _check_two_calls(wl, cuda_device)


def test_noalloc_moments_single_component(libbgk, cuda_device):
    """F only (delta = 0): slot 10 stays exactly zero; two calls in a row."""
    wl = W.reduced(W.taylor_green_box(), mesh_n=(3, 2, 2), vel_n=(9, 8, 7)).replace(p=2)
    _check_two_calls(wl, cuda_device)


def test_noalloc_moments_at_the_scratch_limit(libbgk, cuda_device):
    """185,600 points (11 * n_points within 2.6% of the 2^21-double scratch, so a
    single velocity block) on a 4^3 velocity grid, two calls in a row."""
    wl = W.reduced(W.taylor_green_box(), mesh_n=(29, 10, 10), vel_n=(4, 4, 4))
    assert wl.n_elem * wl.n_sol == 185600
    _check_two_calls(wl, cuda_device, with_oracle=False)


def test_noalloc_rejects_sizes_beyond_its_scratch(libbgk, cuda_device):
    """The library itself refuses more points than its scratch holds (host
    check, before any launch), whatever the buffers."""
    import torch
    from paper_2312_06567_gb300 import bgk

    wl = W.periodic_sine_box()
    _, vgrid, _ = bgk.descriptors(wl)
    too_many = (1 << 21) // 11 + 1
    f = torch.zeros(1, dtype=torch.float64, device=cuda_device)
    m = torch.zeros(1, dtype=torch.float64, device=cuda_device)
    st = libbgk.bgk_moments_noalloc(ctypes.byref(vgrid), ctypes.c_void_p(f.data_ptr()), 1, too_many,
                                    ctypes.c_void_p(m.data_ptr()), None)
    assert st == bgk.BGK_EINVAL
