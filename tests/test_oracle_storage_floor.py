"""The FP32 storage floor of conservation on the sine box (CPU, oracle only).

The oracle's SSP-RK3 stages are exact up to FP64 rounding and conserve mass,
momentum and energy to ~1e-16 per step on this periodic box.  Rounding each
stage's result once to FP32 -- what storing the state in FP32 does and
nothing more -- already moves the totals by more than 1e-10 per step here:
the box's 512 points hold only 8 distinct states (the density varies along x
alone), so one rounding per stored value does not average out over the
points.  No FP32-storage scheme that rounds each value once can do better on
this workload; the GPU mixed form is held to this floor
(tests/test_gpu_mixed.py)."""
import numpy as np

from oracle import stage as ostage
from paper_2312_06567_gb300 import workloads as W


def test_fp32_storage_rounding_alone_exceeds_1e10_per_step_on_the_sine_box():
    wl = W.periodic_sine_box()
    pb = ostage.problem_from_workload(wl)
    dt = wl.dt()
    f0 = W.maxwellian_state(wl).astype(np.float32).astype(np.float64)
    t0 = pb.totals(f0)
    scale = np.array([t0[0]] * 4 + [t0[4]])
    r32 = lambda x: x.astype(np.float32).astype(np.float64)
    f, g = f0.copy(), f0.copy()
    worst = 0.0
    for n in range(1, 4):
        f1, _ = pb.stage(f, f, 0.0, 1.0, dt)
        f1 = r32(f1)
        f2, _ = pb.stage(f, f1, 0.75, 0.25, dt)
        f2 = r32(f2)
        f3, _ = pb.stage(f, f2, 1.0 / 3.0, 2.0 / 3.0, dt)
        f = r32(f3)
        worst = max(worst, float(np.max(np.abs(pb.totals(f) - t0) / scale)) / n)
        g, _ = pb.step(g, dt)
        assert np.max(np.abs(pb.totals(g) - t0) / scale) <= 1e-14 * n
    assert worst >= 5e-10
