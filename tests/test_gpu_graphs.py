"""bgk_step as CUDA-graph replays against direct launches.

A captured step replays the same six launches with the same arguments, so
states, moments and Newton statistics must agree bit for bit; a change of
anything baked into the kernel arguments (here dt and the Newton settings)
must trigger a new capture rather than replaying stale arguments.
"""
import numpy as np
import pytest

from paper_2312_06567_gb300 import workloads as W

from test_gpu_parity import _mild_es_box

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib(libbgk, cuda_device):
    from paper_2312_06567_gb300 import bgk
    return bgk


def _run(lib, wl, prec, f0, graphs, schedule):
    with lib.Solver(wl, prec) as s:
        s.set_graphs(graphs)
        s.set_state(f0)
        for dt, n, tol in schedule:
            s.set_newton(tol=tol)
            assert s.step(dt, n) == lib.BGK_OK
        return s.get_state(), s.moments(), s.stats()


@pytest.mark.parametrize("prec_name", ["BGK_MIXED", "BGK_FP64"])
def test_graph_steps_are_bitwise_direct_steps(lib, prec_name):
    prec = getattr(lib, prec_name)
    wl = _mild_es_box(mesh_n=(4, 2, 2))
    f0 = W.random_anisotropic_state(wl, seed=3)
    f0 = f0.astype(np.float32 if prec == lib.BGK_MIXED else np.float64)
    dt = wl.dt()
    # odd and even step counts exercise both buffer parities; dt and tol changes force recaptures
    schedule = [(dt, 3, 1e-13), (0.5 * dt, 2, 1e-13), (0.5 * dt, 1, 1e-12)]
    fa, ma, sa = _run(lib, wl, prec, f0, False, schedule)
    fb, mb, sb = _run(lib, wl, prec, f0, True, schedule)
    assert np.array_equal(fa, fb)
    assert np.array_equal(ma, mb)
    assert sa == sb


def test_graphs_off_while_profiling(lib):
    """Profiling times each kernel, so steps run as direct launches then."""
    wl = _mild_es_box(mesh_n=(2, 2, 2))
    f0 = W.random_anisotropic_state(wl, seed=4).astype(np.float32)
    with lib.Solver(wl, lib.BGK_MIXED) as s:
        s.set_graphs(True)
        s.set_state(f0)
        s.profile(True)
        assert s.step(wl.dt(), 2) == lib.BGK_OK
        prof = s.profile_read()
        s.profile(False)
    assert prof["qprime"][1] == 6 and prof["stage"][1] == 6
