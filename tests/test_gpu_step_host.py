"""Pipelined host-to-host stepping (bgk_step_host) against the plain
set_state / step / get_state sequence (GPU, through the C-ABI).

Five independent inputs go through the pipeline back to back (each call's
input copy and the earlier results' output copies overlap the compute; five
calls rotate every state buffer through every role); every result must equal
the sequential one bit for bit (the same kernels in the same order), in both
forms, with one and with two steps per call, and the context's state after the
sync is the last result.  Ordinary stepping keeps working on the rotated
buffers, and the pipeline keeps working after it."""
import numpy as np
import pytest

from paper_2312_06567_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib(libbgk, cuda_device):
    from paper_2312_06567_gb300 import bgk
    return bgk


@pytest.mark.parametrize("form,n_steps,pinned", [("mixed", 1, True), ("fp64", 2, True), ("mixed", 2, False)])
def test_pipelined_host_steps_equal_sequential_ones(lib, form, n_steps, pinned):
    import torch
    wl = W.reduced(W.taylor_green_box(), mesh_n=(3, 2, 2), vel_n=(9, 8, 12)).replace(p=2)
    prec = lib.BGK_FP64 if form == "fp64" else lib.BGK_MIXED
    dt_np = np.float64 if form == "fp64" else np.float32
    ins = [W.random_anisotropic_state(wl, seed=60 + i).astype(dt_np) for i in range(5)]
    dt = wl.dt()
    with lib.Solver(wl, prec) as s:
        ref = []
        for f in ins:
            s.set_state(f)
            assert s.step(dt, n_steps) == lib.BGK_OK
            ref.append(s.get_state())
    with lib.Solver(wl, prec) as s:
        if pinned:
            tdt = torch.float64 if form == "fp64" else torch.float32
            hin = [torch.from_numpy(f).pin_memory() for f in ins]
            hout = [torch.empty(s.shape, dtype=tdt, pin_memory=True) for _ in ins]
        else:
            hin = ins
            hout = [np.empty(s.shape, dtype=dt_np) for _ in ins]
        for a, b in zip(hin, hout):
            s.step_host(a, b, dt, n_steps)
        assert s.step_host_sync() == lib.BGK_OK
        outs = [np.asarray(b) for b in hout]
        last = s.get_state()
        outs = [o.copy() for o in outs]
        # ordinary stepping on the rotated buffers (CUDA graphs keyed on them)
        s.set_state(ins[1])
        assert s.step(dt, n_steps) == lib.BGK_OK
        plain = s.get_state()
        # the pipeline keeps going after an ordinary call
        s.set_state(ins[0])
        for a, b in zip(hin[:3], hout[:3]):
            s.step_host(a, b, dt, n_steps)
        assert s.step_host_sync() == lib.BGK_OK
        again = [np.asarray(b).copy() for b in hout[:3]]
    for o, r in zip(outs, ref):
        assert np.array_equal(o, r)
    assert np.array_equal(last, ref[-1])
    assert np.array_equal(plain, ref[1])
    for o, r in zip(again, ref[:3]):
        assert np.array_equal(o, r)
