"""Macroscopic post-processing (bgk_macro: fields, FR density gradient,
Kn_GLL) against the oracle's macro_fields on the same state, FP64 and mixed
forms, periodic and Dirichlet faces, F/G; and after a step, where the
moments come from the stage's own epilogue."""
import numpy as np
import pytest

from oracle import bgk as obgk
from oracle import diagnostics as odiag
from oracle import stage as ostage
from paper_2312_06567_gb300 import workloads as W

from test_gpu_parity import CASES

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib(libbgk, cuda_device):
    from paper_2312_06567_gb300 import bgk
    return bgk


def _oracle(wl, pb, f):
    m = obgk.raw_moments(f[0].reshape(wl.n_vel, -1), f[1].reshape(wl.n_vel, -1) if wl.n_comp == 2 else None, pb.vg)
    return odiag.macro_fields(pb, m)


def _err(a, b):
    sc = np.maximum(np.abs(b).max(axis=0), 1e-300)
    return float(np.max(np.abs(a - b) / sc[None, :]))


@pytest.mark.parametrize("name", ["sine_box_p1", "tgv_es_p3_ragged", "shock_fg_p2_dirichlet", "ragged_p1_dirichlet_x"])
@pytest.mark.parametrize("form", ["fp64", "mixed"])
def test_macro_fields_match_oracle(lib, name, form):
    wl = CASES[name]()
    pb = ostage.problem_from_workload(wl)
    f = W.random_anisotropic_state(wl, seed=13)
    prec = lib.BGK_FP64 if form == "fp64" else lib.BGK_MIXED
    if form == "mixed":
        f = f.astype(np.float32)
    with lib.Solver(wl, prec) as s:
        s.set_state(f)
        out = s.macro()
        assert s.step(wl.dt(), 1) == lib.BGK_OK
        f1 = s.get_state()
        out1 = s.macro()
    tol = 1e-12 if form == "fp64" else 1e-11
    assert _err(out, _oracle(wl, pb, f.astype(np.float64))) <= tol
    assert _err(out1, _oracle(wl, pb, f1.astype(np.float64))) <= tol


@pytest.mark.parametrize("case", ["wavy", "ogrid"])
@pytest.mark.parametrize("form", ["fp64", "mixed"])
def test_curvilinear_macro_fields_match_oracle(lib, case, form):
    """bgk_macro on curvilinear meshes (chain rule through the metric terms)
    against the oracle's macro_fields_curved: a warped periodic box and a
    reduced sphere O-grid (diffuse wall, collapsed poles, Dirichlet farfield,
    where the paper's continuum-breakdown diagnostic matters)."""
    from oracle import curved
    if case == "wavy":
        wl = W.wavy_periodic_box(p=2, n=(3, 2, 2), vel_n=(8, 7, 6))
    else:
        wl = W.reduced(W.sphere_ogrid(), mesh_n=(3, 4, 6), vel_n=(9, 8, 8))
    x = W.node_positions(wl)
    pb = curved.problem_from_workload(wl, x)
    f = W.random_anisotropic_state(wl, seed=17)
    prec = lib.BGK_FP64 if form == "fp64" else lib.BGK_MIXED
    if form == "mixed":
        f = f.astype(np.float32)
    with lib.Solver(wl, prec) as s:
        s.set_state(f)
        out = s.macro()
    fd = f.astype(np.float64)
    m = obgk.raw_moments(fd[0].reshape(wl.n_vel, -1), fd[1].reshape(wl.n_vel, -1) if wl.n_comp == 2 else None,
                         pb.vg)
    ref = odiag.macro_fields_curved(pb, m)
    tol = 1e-12 if form == "fp64" else 1e-11
    assert _err(out, ref) <= tol
    assert np.all(out[:, 9] >= 0.0)
