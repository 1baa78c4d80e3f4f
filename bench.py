#!/usr/bin/env python
"""Throughput of the Boltzmann--ES-BGK FR stage: DOF-updates/s per RK stage.

Workload: the Taylor--Green periodic box (16^3 hex, p=3, 24^3 velocities on
[-5,5]^3, ES-BGK Pr=2/3, Kn=0.01, M=0.1), N_e N_s N_u = 3.62e9 DOF, f
initialised on the device to the Maxwellian of the Taylor--Green field.  A
step is one SSP-RK3 step = 3 stages; value = DOF x 3 K / (timed seconds),
summed over ranks (independent replicas, weak scaling).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload NAME] [--forms fp64,fp64_learned,mixed,mixed_learned]
                  [--stage-kernel tune|auto|plain|async|line|...] [--depth S]
                  [--no-graphs] [--velocity-blocks N] [--e2e-steps E] [--no-cpu-baseline]
                  [--no-tc-probe] [--tc-probe-panels N] [--no-other-workloads]

Workloads: taylor_green (default), sine_box, normal_shock, sphere_ogrid and
smaller copies of the box and the O-grid for profiling.  The line carries the
headline form (mixed + learned guess) at the top level and the other forms
under their names, the dominant kernel's roofline, the clocks sampled during
the timed steps, the end-to-end number through host buffers (with the copies'
bandwidth), the oracle's CPU baseline (one process and all cores), the
tensor-core FR-operator probe, the learned guess's held-out check and batched
inference, and -- for the default Taylor--Green run -- the normal shock and the
sphere O-grid (mixed + learned guess) nested under other_workloads.

--impl reference times the FP64 CPU oracle (the method written out plainly,
test infrastructure) on the host cores on a bounded sample of the same
workload (one element, all 13,824 velocities per stage).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_2312_06567_gb300 import workloads as W  # noqa: E402

METRIC = "DOF-updates/s per RK stage (Ne*Ns*Nu)"
UNIT = "DOF-updates/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--forms", default="fp64,fp64_learned,mixed,mixed_learned")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--workload", default="taylor_green", choices=sorted(WORKLOADS))
    ap.add_argument("--stage-kernel", default="tune", choices=["tune", "auto", "plain", "async", "line", "line_wide", "half", "half_wide"],
                    help="mixed-form stage kernel; 'tune' times the candidates on the workload (untimed)")
    ap.add_argument("--depth", type=int, default=6, help="copy-ring depth of the async stage kernel")
    ap.add_argument("--no-graphs", action="store_true", help="time direct launches instead of CUDA-graph replays")
    ap.add_argument("--velocity-blocks", type=int, default=0,
                    help="velocity blocks of the stage grid (0: the context's choice, tuned with --stage-kernel tune)")
    ap.add_argument("--no-tc-probe", action="store_true", help="skip the tensor-core FR-operator probe")
    ap.add_argument("--no-other-workloads", action="store_true",
                    help="skip the normal shock and sphere O-grid lines nested in the default run")
    ap.add_argument("--tc-probe-panels", type=int, default=1 << 20,
                    help="panels (48 velocities x 64 nodes, 12 KB each) the tensor-core probe streams")
    return ap.parse_args()


def _tg_small():
    """Same physics as the Taylor--Green box on 8x8x4 elements (2.3e8 DOF): the
    size used for ncu captures (a few GB on the device)."""
    return W.reduced(W.taylor_green_box(), mesh_n=(8, 8, 4))


def _shock():
    return W.normal_shock_tube()


def _shock_small():
    """The normal shock physics on 16x4x4 elements (2.3e8 DOF, F and G): the size
    used for ncu captures of its stage kernel."""
    return W.reduced(W.normal_shock_tube(), mesh_n=(16, 4, 4))


def _ogrid_small():
    """The sphere O-grid physics on 6x12x12 elements (4.4e8 DOF): the size used
    for ncu captures of the curvilinear kernels."""
    return W.sphere_ogrid(n=(6, 12, 12))


def _ogrid_tiny():
    """4x8x8 elements (1.3e8 DOF, 3 GB of state): a small case for full ncu captures."""
    return W.sphere_ogrid(n=(4, 8, 8))


WORKLOADS = {"taylor_green": W.taylor_green_box, "taylor_green_8x8x4": _tg_small,
             "normal_shock": _shock, "normal_shock_16x4x4": _shock_small, "sine_box": W.periodic_sine_box,
             "sphere_ogrid": W.sphere_ogrid, "sphere_ogrid_6x12x12": _ogrid_small,
             "sphere_ogrid_4x8x8": _ogrid_tiny}


def _sample_mesh(wl):
    """Elements of the oracle's sample: one element of the box; a 1x4x4 shell
    of a curvilinear mesh (one element would fold the mapping onto itself)."""
    return (1, 4, 4) if wl.mapping is not None else (1, 1, 1)


# ---------------------------------------------------------------------------
def oracle_stage_sample(wl, mesh_n=None):
    """One oracle stage on a reduced-N_e copy of the workload (same p, N_u and
    physics; per-DOF work does not depend on N_e).  Returns (DOF, wall s, cpu s)."""
    sw = W.reduced(wl, mesh_n=mesh_n or _sample_mesh(wl))
    if sw.mapping is not None:
        from oracle import curved
        x = W.node_positions(sw)
        pb = curved.problem_from_workload(sw, x)
        f = W.maxwellian_state(sw, x)
    else:
        from oracle import stage as ostage
        pb = ostage.problem_from_workload(sw)
        f = W.maxwellian_state(sw)
    t0, c0 = time.perf_counter(), time.process_time()
    pb.stage(f, f, 0.0, 1.0, sw.dt())
    return sw.dof, time.perf_counter() - t0, time.process_time() - c0


def cpu_baseline(wl, target_s=12.0):
    dof, wall, cpu = oracle_stage_sample(wl)
    n = max(1, int(target_s / max(wall, 1e-3)))
    tot_dof, tot_wall, tot_cpu = dof, wall, cpu
    for _ in range(n - 1):
        d, w_, c = oracle_stage_sample(wl)
        tot_dof += d
        tot_wall += w_
        tot_cpu += c
    return {"value": tot_dof / tot_wall, "unit": UNIT, "cores": round(tot_cpu / tot_wall, 2),
            "kind": "oracle", "stages": n,
            "sample": "%d oracle stage(s) of the workload reduced to %s elements (%d nodes x %d "
                      "velocities = %d DOF each), %.1f s wall" % (n, "x".join(map(str, _sample_mesh(wl))),
                                                                   dof // wl.n_vel, wl.n_vel, dof, tot_wall)}


def _oracle_worker_ready(_):
    """Warm-up task of the all-cores pool: import the oracle before the clock."""
    from oracle import curved, stage  # noqa: F401
    time.sleep(0.05)
    return os.getpid()


def _oracle_worker(job):
    """One process of the all-cores timing: `reps` oracle stages of the named
    workload's sample.  Returns (DOF, wall s, cpu s)."""
    name, reps = job
    wl = WORKLOADS[name]()
    tot = [0, 0.0, 0.0]
    for _ in range(reps):
        d, w_, c = oracle_stage_sample(wl)
        tot[0] += d
        tot[1] += w_
        tot[2] += c
    return tuple(tot)


def cpu_baseline_all_cores(name, reps, procs=None):
    """The oracle as it stands on every host core: one spawned process per core
    (BLAS held to one thread each), each running `reps` stages of its own copy
    of the sample; DOF-updates/s of all of them over the batch's wall time,
    with the processes started and the oracle imported before the clock.
    Waits are bounded (a lost worker raises multiprocessing.TimeoutError)."""
    import multiprocessing as mp
    procs = procs or len(os.sched_getaffinity(0))
    keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
    saved = {k: os.environ.get(k) for k in keys}
    for k in keys:
        os.environ[k] = "1"
    try:
        with mp.get_context("spawn").Pool(procs) as pool:      # leaving the block terminates the workers
            pool.map_async(_oracle_worker_ready, range(4 * procs), chunksize=1).get(timeout=60)
            t0 = time.perf_counter()
            res = pool.map_async(_oracle_worker, [(name, reps)] * procs, chunksize=1).get(timeout=300)
            wall = time.perf_counter() - t0
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    dof = sum(r[0] for r in res)
    cpu = sum(r[2] for r in res)
    return {"value": dof / wall, "unit": UNIT, "processes": procs, "cores": round(cpu / wall, 2),
            "sample": "%d processes x %d oracle stage(s) of the same sample, %.1f s wall" % (procs, reps, wall)}


# ---------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms in the background."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.out = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.out, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            self.out.close()
            os.unlink(self.out.name)
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        self.out.flush()
        with open(self.out.name) as fh:
            lines = fh.readlines()
        self.out.close()
        os.unlink(self.out.name)
        return summarize_clocks(lines)


def summarize_clocks(lines):
    """Median SM clock, the largest max clock and the throttle reasons seen in
    nvidia-smi CSV rows of ClockSampler.FIELDS (no header, no units); rows
    with fewer fields are skipped, non-numeric clocks ("[N/A]") ignored."""
    rows = []
    for line in lines:
        parts = [p.strip() for p in line.split(",")]
        if len(parts) >= 9:
            rows.append(parts)
    if not rows:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
    sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
    mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
    return {"sm_mhz": statistics.median(sm) if sm else None,
            "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
            "samples": len(rows)}


# ---------------------------------------------------------------------------
# Algorithmic work per DOF: the method's arithmetic and bytes, not the kernels' instruction counts.
def stage_flops_per_dof(p, C):
    """Flops of the fused stage per DOF: FR per component (sum-factorised
    derivative, inflow trace, lift, metric scaling) 6(p+1) + 5 + 12 + 9/(p+1) + 6;
    equilibrium + source + RK 26 (+4 for G) with the exp lattice-factorised to
    3 multiplies; moment epilogue 22 (+2 for G)."""
    q = p + 1
    fr = 6 * q + 5 + 12 + 9.0 / q + 6
    return C * fr + 26 + 3 + 4 * (C - 1) + 22 + 2 * (C - 1)


def qprime_flops_per_dof_eval(n1):
    """Flops of one residual + Jacobian evaluation per velocity in the
    line-separable organisation: ratio recurrence 2, five line sums 10, and
    per line (n1 velocities) the fold into 35 moments (70 + 30 for the
    prefactors) plus two exps and a division counted at 3 flops each."""
    return 12.0 + (70.0 + 30.0 + 9.0) / n1


def drift_is_conservation(wl):
    """True when every face is periodic or collapsed: only then are mass,
    momentum and energy closed, so the totals' change per step measures
    conservation (Dirichlet faces carry flux, diffuse walls exchange momentum
    and energy, specular faces change the normal momentum)."""
    for d in range(3):
        if wl.periodic[d]:
            continue
        for side in (-1, 1):
            if (d, side) not in tuple(wl.closed):
                return False
    return True


def max_over_ranks(x, world, device=None):
    """The largest x over the ranks (the slowest rank's time; x itself on one
    rank).  Works with any torch.distributed backend (gloo needs device=None)."""
    if world <= 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, dof, steps, ms):
    """DOF-updates/s per RK stage of the whole job: every rank advances its own
    replica (weak scaling), 3 stages per step, over the slowest rank's time."""
    return world * dof * 3 * steps / (ms * 1e-3)


def run_ours(args, rank, world, dev):
    import torch
    from paper_2312_06567_gb300 import bgk

    wl = WORKLOADS[args.workload]()
    dt = wl.dt()
    stream = torch.cuda.current_stream()
    results = {}
    peaks = {}
    if rank == 0:
        for k in ("fp64_fma", "fp64_exp", "fp32_fma", "fp32_exp2"):
            peaks[k] = bgk.probe_peak(k)
        if wl.p == 3 and not args.no_tc_probe:
            # the p = 3 FR element operator streamed through tcgen05 MMAs
            # (by default 2^20 panels = 3.2e9 element-node-velocity DOF,
            # 12.9 GB of split operands), measured beside the stage it would feed
            try:
                peaks["tensor_fr_probe"] = bgk.probe_tc(args.tc_probe_panels)
            except Exception as exc:
                peaks["tensor_fr_probe"] = {"unavailable": "%s: %s" % (type(exc).__name__, exc)}
    forms = [f for f in args.forms.split(",") if f]
    headline = next((f for f in ("mixed_learned", "mixed", "fp64") if f in forms), forms[0])
    for form in forms:
        prec = bgk.BGK_FP64 if form.startswith("fp64") else bgk.BGK_MIXED
        learned = form.endswith("_learned")
        s = bgk.Solver(wl, prec, stream=stream)
        x = s.node_coords()
        rho, U, theta = wl.init(x)
        rho, U, theta = (np.broadcast_to(rho, x.shape[:-1]), np.broadcast_to(U, x.shape),
                         np.broadcast_to(theta, x.shape[:-1]))
        q = np.concatenate([rho.reshape(-1, 1), U.reshape(-1, 3), theta.reshape(-1, 1)], axis=1)
        s.set_maxwellian(q)
        tuned = None
        if args.stage_kernel == "tune" or prec == bgk.BGK_MIXED:
            if args.stage_kernel == "tune":
                # (the FP64 form has one stage kernel: only its velocity blocking is tuned)
                v, d, tms = s.tune_stage(dt, reps=3 if prec == bgk.BGK_MIXED else 1)
                tuned = {"variant": v, "depth": d, "ms_per_stage": tms}
            else:
                s.set_stage_kernel(args.stage_kernel, args.depth)
                tuned = {"variant": args.stage_kernel, "depth": args.depth}
            if args.velocity_blocks > 0:
                s.set_velocity_blocks(args.velocity_blocks)
            nvb, per_blk, _ = s.velocity_blocks()
            tuned["velocity_blocks"] = nvb
            tuned["velocities_per_block"] = per_blk
        train = None
        if learned:
            # warm-up steps log the solver's own (features, Delta) pairs; the
            # network is trained on them (outside the timed region) and the
            # timed steps start Newton from its guess
            s.mlp_log(True, 3 * wl.n_elem * wl.n_sol * args.warmup + 1)
        for _ in range(args.warmup):
            s.step(dt, 1)
        torch.cuda.synchronize()
        if learned:
            s.mlp_log(False)
            s.stats()
            t0 = time.perf_counter()
            loss = s.mlp_train(epochs=8, batch=4096, lr=2e-3, seed=0, bf16=True)
            torch.cuda.synchronize()
            train = {"seconds": time.perf_counter() - t0, "final_loss": loss, "epochs": 8,
                     "batch": 4096, "pairs": 3 * wl.n_elem * wl.n_sol * args.warmup,
                     "precision": "bf16 operands, fp32 accumulate, fp32 master weights"}
            s.set_guess(1, bf16=True)
            s.mlp_stats()
        if not args.no_graphs:
            # capture the step graphs of both buffer parities (untimed)
            s.set_graphs(True)
            s.step(dt, 2)
        s.stats()
        tot0 = s.totals()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        clocks = ClockSampler(dev.index if dev.index is not None else 0)
        clocks.start()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.nvtx.range_push("timed")        # lets a profiler select the timed region
        e0.record(stream)
        st = s.step(dt, args.steps)
        e1.record(stream)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        ck = clocks.stop()
        ms = e0.elapsed_time(e1)
        mean_it, max_it, res = s.stats()
        tot1 = s.totals()
        scale = np.array([tot0[0]] * 4 + [tot0[4]])
        drift = float(np.max(np.abs(tot1 - tot0) / scale)) / args.steps
        mac = s.macro()                                 # Kn_GLL etc. of the final state (untimed)
        diag = {"kn_gll_max": float(mac[:, 9].max()), "mach_max": float(mac[:, 6].max()),
                "breakdown_fraction": float(np.mean(mac[:, 9] > 0.05))}
        diag.update(shock_diagnostics(wl, mac))
        # per-kernel times: one more step with direct launches and an event
        # pair around each kernel (outside the timed region)
        s.profile(True)
        s.step(dt, 1)
        prof = s.profile_read()
        s.profile(False)
        s.stats()
        ms = max_over_ranks(ms, world, dev)
        # e2e: host pinned state in, one step, state out, through the C-ABI
        e2e = None
        if args.e2e_steps > 0 and form == headline:
            tdt = torch.float64 if prec == bgk.BGK_FP64 else torch.float32
            h_in = torch.empty(s.shape, dtype=tdt, pin_memory=True)
            h_out = torch.empty(s.shape, dtype=tdt, pin_memory=True)
            s.get_state(h_in)
            nbytes = h_in.numel() * h_in.element_size()
            # (1) sequential: set_state, step, get_state, each returning after its work
            s.set_state(h_in); s.step(dt, 1); s.get_state(h_out)      # untimed first round trip
            torch.cuda.synchronize()
            t_in = t_step = t_out = 0.0
            t0 = time.perf_counter()
            for _ in range(args.e2e_steps):
                ta = time.perf_counter()
                s.set_state(h_in)                   # returns after the copy (host memory)
                tb = time.perf_counter()
                s.step(dt, 1)
                torch.cuda.synchronize()
                tc = time.perf_counter()
                s.get_state(h_out)                  # returns after the copy
                td = time.perf_counter()
                t_in += tb - ta
                t_step += tc - tb
                t_out += td - tc
            torch.cuda.synchronize()
            seq_s = max_over_ranks(time.perf_counter() - t0, world, dev)
            # (2) pipelined: bgk_step_host, the copies of neighbouring steps overlapping the compute
            s.step_host(h_in, h_out, dt, 1)
            s.step_host_sync()                      # untimed: the pipeline's buffer and streams
            n_pipe = max(args.e2e_steps, 4)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(n_pipe):
                s.step_host(h_in, h_out, dt, 1)
            s.step_host_sync()
            pipe_s = max_over_ranks(time.perf_counter() - t0, world, dev)
            e2e = {"value": job_throughput(world, wl.dof, n_pipe, 1e3 * pipe_s), "unit": UNIT,
                   "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
                   "steps": n_pipe,
                   "api": "bgk_step_host (host in, host out, every step) + bgk_step_host_sync",
                   "sequential": {"value": job_throughput(world, wl.dof, args.e2e_steps, 1e3 * seq_s),
                                  "h2d_gbs": nbytes * args.e2e_steps / t_in / 1e9,
                                  "d2h_gbs": nbytes * args.e2e_steps / t_out / 1e9,
                                  "step_ms": 1e3 * t_step / args.e2e_steps,
                                  "api": "bgk_set_state, bgk_step, bgk_get_state"}}
            del h_in, h_out
        newton = dict(mean_iters=mean_it, max_iters=max_it, max_residual=res)
        if learned:
            newton["guess_fallbacks"] = s.mlp_stats()
            newton["training"] = train
        if learned:
            newton["held_out"] = held_out_guess(s, wl, dt, torch)
            if prec == bgk.BGK_MIXED:
                newton["inference"] = inference_throughput(s, torch, stream)
        results[form] = dict(ms=ms, status=bgk.STATUS_NAMES[st], prof=prof, clocks=ck,
                             newton=newton, e2e=e2e, drift=drift, stage_kernel=tuned, diagnostics=diag)
        s.destroy()
        torch.cuda.empty_cache()
    return wl, results, peaks


def shock_diagnostics(wl, mac):
    """Shock and sonic-surface quantities of the final state (postprocess):
    the number of Mach = 1 crossings along the first-axis node lines, the
    max-slope shock thickness where a shock is set up (the normal shock), and
    the shock standoff on the stagnation line of the sphere O-grid."""
    from paper_2312_06567_gb300 import postprocess as pp
    x = W.node_positions(wl).reshape(-1, 3)
    lines = pp.first_axis_lines(wl)
    out = {"sonic_crossings": len(pp.mach_crossings(x, mac[:, 6], lines))}
    if wl.dirichlet and (0, -1) in wl.dirichlet and (0, 1) in wl.dirichlet and wl.mapping is None:
        r1, r2 = wl.dirichlet[(0, -1)][0], wl.dirichlet[(0, 1)][0]
        out["shock_thickness_max_slope"] = pp.max_slope_thickness(r1, r2, float(mac[:, 8].max()))
    if wl.mapping is not None and wl.diffuse:
        # the line whose nodes point most nearly against the freestream (+x)
        xn = x[lines[:, 0]]
        j = int(np.argmax(-xn[:, 0] / np.linalg.norm(xn, axis=1)))
        sv, pt = pp.max_gradient_position(x, mac[:, 8], lines[j])
        r_body = float(np.linalg.norm(wl.mapping(np.array([[0.0, 0.5, 0.5]]))[0]))    # the wall's radius
        out["stagnation_line_shock_radius"] = float(np.linalg.norm(pt))
        out["shock_standoff"] = float(np.linalg.norm(pt)) - r_body
    return out


def held_out_guess(s, wl, dt, torch):
    """The trained guess on a state it was not trained on (untimed): the
    current state with an anisotropic, density- and temperature-changing
    perturbation, f (1 + 0.15 (u1^2 - u2^2)/25 + 0.1 u3/5), one step from q and
    one from the guess.  Newton updates per solve both ways, the guesses
    discarded, and the largest difference of the two results."""
    f = torch.empty(s.shape, dtype=torch.float64 if s.precision == 0 else torch.float32, device="cuda")
    s.get_state(f)
    u = torch.from_numpy(W.velocity_nodes(wl)).to(device="cuda", dtype=f.dtype)
    fac = 1.0 + 0.15 * (u[:, 0] ** 2 - u[:, 1] ** 2) / 25.0 + 0.1 * u[:, 2] / 5.0
    f.mul_(fac.view(1, -1, 1, 1).clamp_min(0.2))
    out = {}
    res = []
    for mode in (0, 1):
        s.set_guess(mode, bf16=True)
        s.set_state(f)
        s.stats()
        s.mlp_stats()
        s.step(dt, 1)
        mean_it, max_it, r = s.stats()
        out["from_q" if mode == 0 else "learned"] = {"mean_iters": mean_it, "max_iters": max_it,
                                                     "max_residual": r}
        if mode:
            out["learned"]["guess_fallbacks"] = s.mlp_stats()
        g = torch.empty_like(f)
        s.get_state(g)
        res.append(g)
    scale = res[0].abs().amax(dim=(0, 2, 3)).clamp_min(1e-300)
    out["max_rel_diff"] = float(((res[1] - res[0]).abs().amax(dim=(0, 2, 3)) / scale).max())
    out["state"] = "the benchmark state after the timed steps times (1 + 0.15 (u1^2-u2^2)/25 + 0.1 u3/5)"
    del f, res
    return out


def inference_throughput(s, torch, stream, sizes=(1000000, 10000000), reps=5):
    """bgk_mlp_infer (tensor cores) on batches resampled (seed 1) from the
    logged training features: points per second at each batch size."""
    pairs = s.mlp_log_read(1 << 22)
    if len(pairs) == 0:
        return None
    rng = np.random.default_rng(1)
    out = {}
    for B in sizes:
        x = torch.from_numpy(np.ascontiguousarray(pairs[rng.integers(0, len(pairs), B), :9])).cuda()
        d = torch.empty((B, 5), dtype=torch.float32, device="cuda")
        s.mlp_infer(x, d)                            # warm-up
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            s.mlp_infer(x, d)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        flops = 2.0 * (9 * 64 + 64 * 64 + 64 * 5) * B
        out[str(B)] = {"ms": ms, "points_per_s": B / (ms * 1e-3), "tflops": flops / (ms * 1e-3) / 1e12}
        del x, d
    out["kernel"] = "tcgen05 kind::f16, BF16 in, FP32 accumulate, 128 points per MMA tile"
    return out


def stage_bytes_per_dof(C, elem):
    """Algorithmic HBM bytes per DOF of one stage, averaged over the three
    SSP-RK3 stages: read f_s and write f_out (stage 1), plus read f^n (2, 3)."""
    return C * elem * (2 + 3 + 3) / 3.0


def qprime_ops_per_dof_eval_fp32(n1):
    """FP32 operations of one evaluation per velocity in the FP32-sum engine:
    ratio recurrence 2, on-the-fly monomials 3, five line sums 5, weight
    select 1; per line (n1 velocities) the fold into 35 moments (35 FMA = 70
    flops + 30 for prefactors) and the anchors."""
    return 2 * (2 + 3 + 5 + 1) + (70.0 + 30.0 + 9.0) / n1


def kernel_rooflines(wl, r, peaks, form):
    """Per-kernel roofline of one form: algorithmic work / event-timed launch
    duration against the pipe or memory that bounds it."""
    prof = r["prof"]
    out = {}
    evals = r["newton"]["mean_iters"] + 1.0           # updates + the converged check
    ms_s = prof["stage"][0] / max(prof["stage"][1], 1)
    ms_q = prof["qprime"][0] / max(prof["qprime"][1], 1)
    if form.startswith("fp64"):
        fl = wl.dof * stage_flops_per_dof(wl.p, wl.n_comp)
        out["stage"] = {"bound": "alu", "kernel": "stage", "pipe": "fp64", "achieved": fl / (ms_s * 1e-3) / 1e12,
                        "peak": peaks["fp64_fma"] / 1e12, "unit": "TFLOP/s", "ms": ms_s}
        fl = wl.dof * evals * qprime_flops_per_dof_eval(wl.vel_n[0])
        out["qprime"] = {"bound": "alu", "kernel": "qprime", "pipe": "fp64", "achieved": fl / (ms_q * 1e-3) / 1e12,
                         "peak": peaks["fp64_fma"] / 1e12, "unit": "TFLOP/s", "ms": ms_q}
    else:
        by = wl.dof * stage_bytes_per_dof(wl.n_comp, 4)
        out["stage"] = {"bound": "hbm", "kernel": "stage", "achieved": by / (ms_s * 1e-3) / 1e9,
                        "peak": peaks["hbm_gbs"], "unit": "GB/s", "ms": ms_s}
        fl = wl.dof * evals * qprime_ops_per_dof_eval_fp32(wl.vel_n[0])
        out["qprime"] = {"bound": "alu", "kernel": "qprime", "pipe": "fp32", "achieved": fl / (ms_q * 1e-3) / 1e12,
                         "peak": peaks["fp32_fma"] / 1e12, "unit": "TFLOP/s", "ms": ms_q}
    for v in out.values():
        v["frac"] = v["achieved"] / v["peak"]
        v["traffic"] = None
    return out


# DRAM bytes per DOF of a stage launch, mean over the three stages of a step,
# from ncu captures (dram__bytes_read.sum + dram__bytes_write.sum) of a stage
# that reads f^n (the second), with the first stage's f^n read (4 B/DOF per
# component) taken off for the mean: the line kernels on the Taylor--Green
# physics at 8x8x4 elements, p = 3, 24^3 velocities (4-element runs 12.75 B/DOF
# captured, 8-element runs 12.77), and on the normal shock physics at 16x4x4
# elements, p = 2, F and G (25.21 B/DOF).
# Valid for those kernels as they stand; traffic per DOF does not depend on N_e.
# Keys: (variant, p, components).
MEASURED_STAGE_TRAFFIC_PER_DOF = {("line", 3, 1): 11.42, ("line_wide", 3, 1): 11.44, ("line", 2, 2): 22.54}


def tensor_probe_summary(tc, wl, peaks):
    """The tensor-core FR-operator probe next to the stage: its rate, the time
    the own-element operator of all three directions alone would take for the
    whole state at that rate (split operands resident in HBM, no conversion,
    no epilogue), and its arithmetic against FP64."""
    if "unavailable" in tc:
        return tc
    bf16 = _measured_bf16()
    out = {"tflops": tc["flops"] / 1e12, "dof_per_s": tc["dof_per_s"],
           "operand_gbs": tc["bytes_per_s"] / 1e9, "ms": tc["ms"],
           "ms_per_stage_equiv": 1e3 * wl.dof / tc["dof_per_s"],
           "max_rel_err": tc["max_rel_err"], "bias": tc["bias"],
           "shape": "M=64 N=48 K=16 kind::f16 (BF16 in, FP32 accumulate), 36 MMAs per 48 velocities x 64 nodes",
           "split": "bf16 hi + lo, three products (hi.hi + lo.hi + hi.lo)"}
    if bf16:
        out["frac_of_bf16_peak"] = tc["flops"] / (bf16 * 1e12)
        out["bf16_peak_tflops"] = bf16
    return out


def _measured_bf16():
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops"])
    except (OSError, KeyError, ValueError):
        return None


def dominant_roofline(rl):
    k = max(rl, key=lambda n: rl[n]["ms"])
    d = dict(rl[k])
    d["peak_source"] = ("MEASURED_PEAKS.json hbm_gbs" if d["bound"] == "hbm"
                        else "measured %s FMA throughput (bgk_probe_peak) on this GPU" % d.get("pipe", ""))
    return d


def _measured_hbm():
    """Measured HBM copy bandwidth of this GPU (MEASURED_PEAKS.json, a STREAM-style
    copy), else 6.8 TB/s, an earlier copy measurement on a GB300."""
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6800.0


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    wl = WORKLOADS[args.workload]()

    if args.impl == "reference":
        if rank != 0:
            return
        times, dofs, cpus = [], [], []
        for i in range(args.warmup + args.steps):
            d, w_, c = oracle_stage_sample(wl)
            if i >= args.warmup:
                times.append(w_)
                dofs.append(d)
                cpus.append(c)
        v = sum(dofs) / sum(times)
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT,
                "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": wl.name, "sample": "%s elements x %d nodes x %d velocities "
                           "per step (one oracle stage)" % ("x".join(map(str, _sample_mesh(wl))), wl.n_sol, wl.n_vel)},
                "cpu_baseline": {"kind": "oracle", "cores": round(sum(cpus) / sum(times), 2),
                                 "sample": "one oracle stage on %s elements per step" % "x".join(map(str, _sample_mesh(wl))),
                                 "value": v, "unit": UNIT},
                "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    import torch
    if world > 1:
        torch.distributed.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    wl, results, peaks = run_ours(args, rank, world, dev)
    if rank != 0:
        return
    peaks["hbm_gbs"] = _measured_hbm()
    line = compose_line(args, wl, results, peaks, world)
    if world == 1 and args.workload == "taylor_green" and not args.no_other_workloads:
        # the normal shock and the sphere O-grid at full size, mixed form + learned
        # guess, beside the headline (their own clocks and kernel times)
        line["other_workloads"] = {}
        for name in ("normal_shock", "sphere_ogrid"):
            sub = argparse.Namespace(**vars(args))
            sub.workload, sub.forms, sub.e2e_steps, sub.steps, sub.no_tc_probe = name, "mixed_learned", 0, 2, True
            try:
                wl2, res2, pk2 = run_ours(sub, rank, world, dev)
                pk2["hbm_gbs"] = peaks["hbm_gbs"]
                l2 = compose_line(sub, wl2, res2, pk2, world)
                line["other_workloads"][name] = {
                    k: l2[k] for k in ("value", "ms_per_step", "config", "kernels_ms_per_step", "roofline", "clocks",
                                       "conservation_drift_per_step", "drift_is_conservation", "newton",
                                       "stage_kernel", "diagnostics", "status")}
            except Exception as exc:
                line["other_workloads"][name] = {"unavailable": "%s: %s" % (type(exc).__name__, exc)}
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(wl)
        try:
            line["cpu_baseline"]["all_cores"] = cpu_baseline_all_cores(args.workload,
                                                                       line["cpu_baseline"]["stages"])
        except Exception as exc:             # the line is printed whatever the host's process limits
            line["cpu_baseline"]["all_cores"] = {"unavailable": "%s: %s" % (type(exc).__name__, exc)}
    print(json.dumps(line))


def compose_line(args, wl, results, peaks, world):
    """The benchmark's JSON line from the per-form results of run_ours: the
    headline form (mixed + learned guess, else mixed, else FP64) at the top
    level, the other forms under their names."""
    main_form = next((f for f in ("mixed_learned", "mixed", "fp64") if f in results), list(results)[0])
    r = results[main_form]
    ms_per_step = r["ms"] / args.steps
    value = job_throughput(world, wl.dof, args.steps, r["ms"])
    launches = sum(v[1] for v in r["prof"].values()) * args.steps     # the profiled step x timed steps
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if main_form == "fp64" else "f32+f64" + ("+bf16" if "learned" in main_form else ""),
        "data": "synthetic",
        "config": {"workload": wl.name, "dof": wl.dof, "elements": wl.n_elem, "order": wl.p,
                   "velocities": wl.n_vel, "form": main_form, "parallelism": "replicas",
                   "l2": "inputs larger than L2 (state %.1f GB per copy)" %
                         (wl.dof * wl.n_comp * (8 if main_form == "fp64" else 4) / 1e9)},
        "clocks": r["clocks"],
        "e2e": r["e2e"],
        "conservation_drift_per_step": r["drift"],
        "drift_is_conservation": drift_is_conservation(wl),
        "gpu_launches": launches,
        "kernels_ms_per_step": {k: v[0] for k, v in r["prof"].items()},
        "launch": "cuda graph replay" if not args.no_graphs else "direct launches",
        "component_updates_per_s": value * wl.n_comp,
        "newton": r["newton"],
        "stage_kernel": r["stage_kernel"],
        "diagnostics": r["diagnostics"],
        "status": r["status"],
        "peaks_measured": peaks,
    }
    rl = kernel_rooflines(wl, r, peaks, main_form)
    sk = ((r.get("stage_kernel") or {}).get("variant"), wl.p, wl.n_comp)
    if sk in MEASURED_STAGE_TRAFFIC_PER_DOF and "stage" in rl:
        rl["stage"]["traffic"] = MEASURED_STAGE_TRAFFIC_PER_DOF[sk] * wl.dof
    line["roofline"] = dominant_roofline(rl)
    line["roofline_kernels"] = rl
    tc = peaks.pop("tensor_fr_probe", None)
    if tc is not None:
        line["tensor_fr_probe"] = tensor_probe_summary(tc, wl, peaks)
    for form, rr in results.items():
        if form != main_form:
            line[form] = {"value": job_throughput(world, wl.dof, args.steps, rr["ms"]),
                          "ms_per_step": rr["ms"] / args.steps,
                          "kernels_ms_per_step": {k: v[0] for k, v in rr["prof"].items()},
                          "newton": rr["newton"], "e2e": rr["e2e"],
                          "conservation_drift_per_step": rr["drift"],
                          "roofline_kernels": kernel_rooflines(wl, rr, peaks, form),
                          "stage_kernel": rr["stage_kernel"], "clocks": rr["clocks"]}
    return line


if __name__ == "__main__":
    main()
