"""Velocity shards of libbgk (GPU, through the C-ABI) against the unsharded context.

Two or three shard contexts on one GPU stand for the ranks of a sharded run:
per stage each writes its partial raw moments, the test sums them (what the
all-reduce does across GPUs) and hands the sum to every shard.  Nothing
waits on another context: the calls are sequential on one stream.  The
gathered state must equal the unsharded context's: FP64 form within 1e-12
after two steps (the moments are summed in another order, nothing else
differs), mixed form within 1e-5 (the FP32 Newton engine may stop at another
iterate when its input moves by an ulp), and the gathered totals conserved."""
import numpy as np
import pytest

from paper_2312_06567_gb300 import workloads as W
from paper_2312_06567_gb300.shard import ShardedStepper, velocity_slabs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib(libbgk, cuda_device):
    from paper_2312_06567_gb300 import bgk
    return bgk


def _slab_err(a, b):
    C, Nu = b.shape[:2]
    d = np.abs(a - b).reshape(C * Nu, -1).max(axis=1)
    s = np.abs(b).reshape(C * Nu, -1).max(axis=1)
    return float(np.max(d / np.maximum(s, 1e-300)))


def _run(lib, wl, prec, n_shards, steps, f0):
    import torch
    dt = wl.dt()
    n12 = wl.vel_n[0] * wl.vel_n[1]
    slabs = velocity_slabs(wl.vel_n[2], n_shards)
    shards = [lib.Solver(wl, prec, shard=sl) for sl in slabs]
    try:
        for sh, (lo, hi) in zip(shards, slabs):
            sh.set_state(f0[:, lo * n12:hi * n12])
        P = shards[0].n_points
        ms = [torch.empty((11, P), dtype=torch.float64, device="cuda") for _ in shards]
        tot0 = sum(sh.totals() for sh in shards)
        for _ in range(steps):
            for stage in range(3):
                for sh, m in zip(shards, ms):
                    sh.shard_partials(m)
                total = sum(ms[1:], ms[0].clone())
                for sh in shards:
                    assert sh.shard_stage(total, stage, dt) == lib.BGK_OK
        tot1 = sum(sh.totals() for sh in shards)
        f = np.concatenate([sh.get_state() for sh in shards], axis=1)
    finally:
        for sh in shards:
            sh.destroy()
    return f, tot0, tot1


@pytest.mark.parametrize("case,prec,tol,n_shards", [
    ("box", "fp64", 1e-12, 2), ("box", "fp64", 1e-12, 3), ("shock", "fp64", 1e-12, 2),
    ("box", "mixed", 1e-5, 2), ("shock", "mixed", 1e-5, 3)])
def test_shards_equal_the_unsharded_context(lib, case, prec, tol, n_shards):
    if case == "box":
        wl = W.reduced(W.taylor_green_box(), mesh_n=(3, 2, 2), vel_n=(9, 8, 12)).replace(p=2)
    else:
        wl = W.reduced(W.normal_shock_tube(mach=3.0), mesh_n=(4, 1, 2), vel_n=(13, 9, 12)).replace(
            p=2, vel_lo=(-9.0, -8.0, -8.0), vel_hi=(11.0, 8.0, 8.0))
    p = lib.BGK_FP64 if prec == "fp64" else lib.BGK_MIXED
    f0 = W.random_anisotropic_state(wl, seed=41)
    if prec == "mixed":
        f0 = f0.astype(np.float32)
    dt = wl.dt()
    with lib.Solver(wl, p) as s:
        s.set_state(f0)
        t0 = s.totals()
        assert s.step(dt, 2) == lib.BGK_OK
        ref = s.get_state()
        t1 = s.totals()
    got, g0, g1 = _run(lib, wl, p, n_shards, 2, f0)
    assert _slab_err(got.astype(np.float64), ref.astype(np.float64)) <= tol
    # the shards' totals add up to the whole context's, and are conserved as
    # well as its own on a periodic box
    scale = np.array([abs(t0[0])] * 4 + [abs(t0[4])])
    assert np.max(np.abs(g0 - t0) / scale) <= 1e-13
    if case == "box":
        assert np.max(np.abs(g1 - g0) / scale) <= (1e-12 if prec == "fp64" else 1e-9)


def test_sharded_stepper_drives_library_shards(lib):
    """ShardedStepper (the multi-rank host loop) on one rank with a one-shard
    'all-reduce' (the identity): the whole grid in one shard context equals
    the plain context bit for bit."""
    import torch
    wl = W.reduced(W.taylor_green_box(), mesh_n=(3, 2, 2), vel_n=(9, 8, 12)).replace(p=2)
    f0 = W.random_anisotropic_state(wl, seed=41)
    dt = wl.dt()
    with lib.Solver(wl) as s:
        s.set_state(f0)
        assert s.step(dt, 2) == lib.BGK_OK
        ref = s.get_state()
    with lib.Solver(wl, shard=(0, wl.vel_n[2])) as s:
        s.set_state(f0)
        m = torch.empty((11, s.n_points), dtype=torch.float64, device="cuda")
        assert ShardedStepper(s, m, lambda t: None).step(dt, 2) == 0
        got = s.get_state()
    assert np.array_equal(got, ref)


def test_shard_rejects_what_it_cannot_do(lib):
    wl = W.reduced(W.taylor_green_box(), mesh_n=(2, 1, 1), vel_n=(6, 6, 6)).replace(p=1)
    with pytest.raises(lib.BGKError):
        lib.Solver(wl, shard=(0, 1))              # one plane
    with pytest.raises(lib.BGKError):
        lib.Solver(wl, shard=(4, 7))              # past the axis
    with lib.Solver(wl, shard=(0, 3)) as s:
        s.set_state(W.random_anisotropic_state(wl, seed=1)[:, :6 * 6 * 3])
        with pytest.raises(lib.BGKError):
            s.step(wl.dt(), 1)
        with pytest.raises(lib.BGKError):
            s.macro()
