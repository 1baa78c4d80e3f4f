"""The discrete entropy output of bgk_totals against the FP64 oracle (GPU).

H = sum_e sum_s W_s |J| sum_k w_k F ln F (section "Numerical method": the
discrete-velocity BGK relaxation satisfies a discrete H-theorem).  The library
sums F ln F per point in FP64 on the GPU and weighs the points on the host;
the oracle is a plain numpy sum.  Pin P8: on the periodic sine box (4^3
elements, p = 1, 8^3 velocities, 10 SSP-RK3 steps) the oracle's entropy falls
by about 1e-7 of |H| per step, so the library's must not rise.
"""
import numpy as np
import pytest

from oracle import stage as ostage
from paper_2312_06567_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib(libbgk, cuda_device):
    from paper_2312_06567_gb300 import bgk
    return bgk


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_entropy_of_a_random_state_matches_oracle(lib, prec):
    wl = W.reduced(W.taylor_green_box(), mesh_n=(3, 2, 2), vel_n=(9, 8, 7)).replace(p=2)
    f = W.random_anisotropic_state(wl, seed=5)
    pb = ostage.problem_from_workload(wl)
    with lib.Solver(wl, lib.BGK_FP64 if prec == "fp64" else lib.BGK_MIXED) as s:
        s.set_state(f)
        stored = s.get_state().astype(np.float64)   # the FP32-rounded state in the mixed form
        H = s.entropy()
    ref = pb.entropy(stored)
    assert abs(H - ref) <= 1e-13 * abs(ref)


def test_entropy_is_nan_when_some_f_is_not_positive(lib):
    wl = W.reduced(W.taylor_green_box(), mesh_n=(2, 1, 1), vel_n=(6, 6, 6)).replace(p=1)
    f = W.random_anisotropic_state(wl, seed=6)
    f[0, 7, 1, 3] = 0.0
    with lib.Solver(wl) as s:
        s.set_state(f)
        assert np.isnan(s.entropy())
        assert np.all(np.isfinite(s.totals()))


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_entropy_does_not_increase_on_the_sine_box(lib, prec):
    """P8 on the full small configuration: H non-increasing over its 10 steps,
    and in the FP64 form equal to the oracle's H after every step (1e-13)."""
    wl = W.periodic_sine_box()
    pb = ostage.problem_from_workload(wl)
    f = W.maxwellian_state(wl)
    dt = wl.dt()
    with lib.Solver(wl, lib.BGK_FP64 if prec == "fp64" else lib.BGK_MIXED) as s:
        s.set_state(f)
        H = [s.entropy()]
        for _ in range(wl.steps):
            assert s.step(dt, 1) == lib.BGK_OK
            H.append(s.entropy())
    H = np.array(H)
    assert np.all(np.isfinite(H))
    assert np.all(np.diff(H) <= 1e-12 * abs(H[0])), np.diff(H) / abs(H[0])
    # the decrease is real, not round-off: about 1e-7 of |H| per step
    assert H[-1] < H[0] - 5e-7 * abs(H[0])
    if prec == "fp64":
        fo = f
        for n in range(wl.steps):
            fo, _ = pb.step(fo, dt)
            assert abs(H[n + 1] - pb.entropy(fo)) <= 1e-13 * abs(H[0])
