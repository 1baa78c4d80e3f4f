"""Bounded waits of the copy-ring stage kernels on the GPU (through the C-ABI).

The test entry bgk_test_ring_stall makes every block's copy ring stop after a
few velocities, so the consumers wait for a stage buffer that is never filled
-- a wait on a flag that nothing sets.  The wait gives up after the
shortened limit (10 ms instead of about 2 s), the kernel lets its issued
copies land, records its timeout status and returns; the step reports
BGK_ETIMEOUT, and the same context, the stall lifted, steps normally again
with results bit-identical to a context that never stalled.  No fault, trap
or hang is involved: every wait in these kernels ends by construction."""
import time

import numpy as np
import pytest

from paper_2312_06567_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib(libbgk, cuda_device):
    from paper_2312_06567_gb300 import bgk
    return bgk


@pytest.mark.parametrize("variant", ["line", "async", "half"])
def test_ring_wait_gives_up_reports_timeout_and_context_recovers(lib, variant):
    wl = W.reduced(W.taylor_green_box(), mesh_n=(4, 4, 2))
    f = W.random_anisotropic_state(wl, seed=7).astype(np.float32)
    dt = wl.dt()
    with lib.Solver(wl, lib.BGK_MIXED) as ref:
        ref.set_stage_kernel(variant, 2)
        ref.set_state(f)
        assert ref.step(dt, 1) == lib.BGK_OK
        want = ref.get_state()
    with lib.Solver(wl, lib.BGK_MIXED) as s:
        s.set_stage_kernel(variant, 2)
        s.set_state(f)
        s.test_ring_stall(5, 0.01)
        t0 = time.time()
        with pytest.raises(lib.BGKError) as err:
            s.step(dt, 1)
        assert err.value.status == lib.BGK_ETIMEOUT
        assert time.time() - t0 < 5.0                  # the shortened limit, not 2 s per wait
        s.test_ring_stall(0)
        s.set_state(f)
        assert s.step(dt, 1) == lib.BGK_OK
        assert np.array_equal(s.get_state(), want)
