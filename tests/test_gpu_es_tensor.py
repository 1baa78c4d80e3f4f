"""The tensor variant of the discrete ES equilibrium on the GPU against the
oracle: residual and one SSP-RK3 step (FP64 within 1e-12; mixed within 1e-5
of the per-velocity scale, moments within 1e-5), conservation, graph replay,
and the configurations it declines."""
import numpy as np
import pytest

from oracle import bgk as obgk
from oracle import stage as ostage
from paper_2312_06567_gb300 import workloads as W

from test_gpu_parity import moment_err, rhs_err, slab_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib(libbgk, cuda_device):
    from paper_2312_06567_gb300 import bgk
    return bgk


def _case(p=3, mesh_n=(3, 2, 2), vel_n=(10, 9, 8)):
    return W.reduced(W.taylor_green_box(), mesh_n=mesh_n, vel_n=vel_n).replace(p=p, es_tensor=True)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_tensor_rhs_and_step_match_oracle(lib, p):
    wl = _case(p=p)
    pb = ostage.problem_from_workload(wl)
    f = W.random_anisotropic_state(wl, seed=71)
    r_ora, info = pb.rhs(f)
    assert np.all(info["converged"])
    f1_ora, _ = pb.step(f, wl.dt())
    with lib.Solver(wl, lib.BGK_FP64) as s:
        s.set_state(f)
        r = s.rhs(f)
        assert s.step(wl.dt(), 1) == lib.BGK_OK
        f1 = s.get_state()
    assert rhs_err(r, r_ora, f, wl, info["tau"].min()) <= 1e-12
    assert slab_err(f1, f1_ora) <= 1e-12
    # the d+2 equilibrium differs from it by far more than the tolerance
    r5, _ = ostage.problem_from_workload(wl.replace(es_tensor=False)).rhs(f)
    assert rhs_err(r5, r_ora, f, wl, info["tau"].min()) > 1e-9


@pytest.mark.parametrize("fp32_sums", [False, True])
def test_tensor_mixed_form_matches_oracle(lib, fp32_sums):
    wl = _case(p=3)
    pb = ostage.problem_from_workload(wl)
    f32 = W.random_anisotropic_state(wl, seed=72).astype(np.float32)
    f = f32.astype(np.float64)
    r_ora, info = pb.rhs(f)
    f1_ora, _ = pb.step(f, wl.dt())
    m1_ora = obgk.raw_moments(f1_ora[0].reshape(wl.n_vel, -1), None, pb.vg)
    with lib.Solver(wl, lib.BGK_MIXED) as s:
        s.set_qprime_engine(fp32_sums)
        s.set_state(f32)
        r = s.rhs(f32).astype(np.float64)
        assert s.step(wl.dt(), 1) == lib.BGK_OK
        f1 = s.get_state().astype(np.float64)
        m1 = s.moments()
    assert rhs_err(r, r_ora, f, wl, info["tau"].min()) <= 1e-5
    assert slab_err(f1, f1_ora) <= 1e-5
    assert moment_err(m1, m1_ora) <= 1e-5


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_tensor_steps_conserve_and_graphs_replay_bitwise(lib, precision):
    wl = _case(p=3, mesh_n=(3, 3, 2))
    f = W.random_anisotropic_state(wl, seed=73)
    prec = lib.BGK_FP64 if precision == "fp64" else lib.BGK_MIXED
    dt = np.float64 if precision == "fp64" else np.float32
    outs = []
    for graphs in (False, True):
        with lib.Solver(wl, prec) as s:
            s.set_state(f.astype(dt))
            s.set_graphs(graphs)
            t0 = s.totals()
            assert s.step(wl.dt(), 3) == lib.BGK_OK
            s.set_state(s.get_state())
            t1 = s.totals()
            outs.append(s.get_state())
        scale = np.array([t0[0]] * 4 + [t0[4]])
        bar = 1e-12 if precision == "fp64" else 2e-9
        assert np.all(np.abs(t1 - t0) / scale / 3 <= bar), (t1 - t0) / scale
    assert np.array_equal(outs[0], outs[1])


def test_tensor_variant_declined_for_polyatomic_gas(lib):
    wl = W.reduced(W.normal_shock_tube(mach=3.0), mesh_n=(3, 1, 1), vel_n=(13, 9, 11)).replace(p=1)
    with lib.Solver(wl, lib.BGK_FP64) as s:
        with pytest.raises(RuntimeError):
            s.set_es_tensor(True)
