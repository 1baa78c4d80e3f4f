"""bgk_moments_noalloc against bgk_moments (GPU, through the C-ABI).

The no-allocation entry point serves callers that cannot call cudaMalloc and
so cannot create a solver context; it keeps its scratch in a fixed device
array inside the library.  This file is collected last so that a run that
stops at the first failure has already run every other test.
"""
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


def test_noalloc_moments_match_context_moments_on_two_calls(libbgk, cuda_device):
    import torch
    from paper_2312_06567_gb300 import bgk

    wl = W.reduced(W.normal_shock_tube(mach=3.0), mesh_n=(5, 1, 2), vel_n=(13, 9, 10)).replace(
        vel_lo=(-9.0, -8.0, -8.0), vel_hi=(11.0, 8.0, 8.0))
    _, vgrid, _ = bgk.descriptors(wl)
    P = wl.n_elem * wl.n_sol
    m_dev = torch.empty((P, 11), dtype=torch.float64, device=cuda_device)
    stream = torch.cuda.current_stream()
    with bgk.Solver(wl) as s:
        for seed in (1, 2):                     # two calls in a row, different states
            f = W.random_anisotropic_state(wl, seed=seed)
            s.set_state(f)
            ref = s.moments()
            f_dev = torch.from_numpy(f).to(cuda_device)
            m_dev.fill_(np.nan)
            bgk.moments_noalloc(vgrid, f_dev, wl.n_comp, P, m_dev, stream)
            torch.cuda.synchronize()
            got = m_dev.cpu().numpy()
            assert np.all(np.isfinite(got))
            assert np.max(np.abs(got - ref) / _moment_scale(ref, wl.delta)) <= 1e-13


def test_noalloc_rejects_sizes_beyond_its_scratch(libbgk, cuda_device):
    import torch
    from paper_2312_06567_gb300 import bgk

    wl = W.periodic_sine_box()
    _, vgrid, _ = bgk.descriptors(wl)
    too_many = (1 << 21) // 11 + 1
    f = torch.zeros(1, dtype=torch.float64, device=cuda_device)
    m = torch.zeros(1, dtype=torch.float64, device=cuda_device)
    with pytest.raises(bgk.BGKError) as ei:
        bgk.moments_noalloc(vgrid, f, 1, too_many, m)
    assert ei.value.status == bgk.BGK_EINVAL
