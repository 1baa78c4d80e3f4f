"""The velocity-sharded step's host logic on CPU ranks (gloo, world size 2).

Each rank holds one slab of third-axis velocity planes (velocity_slabs) and
steps it with ShardedStepper, the same code that drives libbgk shards: per
stage, the slab's partial raw moments, an all-reduce over the ranks, the
stage from the summed moments.  The rank's shard here is a stand-in built
from the oracle (partial moments of its velocities with the whole grid's
weights; Q' from the summed moments over the whole grid; FR advection and
the BGK source on its own velocities), so the test runs without a GPU.  The
gathered state must equal the unsharded oracle step to 1e-12."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _workload():
    from paper_2312_06567_gb300 import workloads as W
    return W.reduced(W.normal_shock_tube(mach=3.0), mesh_n=(3, 1, 2), vel_n=(13, 9, 10)).replace(
        p=1, vel_lo=(-9.0, -8.0, -8.0), vel_hi=(11.0, 8.0, 8.0))


class OracleShard:
    """Stand-in for a libbgk shard: the oracle on the velocities of one slab."""

    def __init__(self, wl, f_slab, lo, hi):
        import torch
        from oracle import bgk as obgk
        from oracle import stage as ostage
        from oracle.velocity import VelocityGrid
        self.torch, self.obgk = torch, obgk
        self.full = ostage.problem_from_workload(wl)
        self.vg = self.full.vg
        n1, n2 = wl.vel_n[0], wl.vel_n[1]
        self.sel = np.arange(lo * n1 * n2, hi * n1 * n2)          # this slab's velocities
        h3 = (wl.vel_hi[2] - wl.vel_lo[2]) / (wl.vel_n[2] - 1)
        self.vslab = VelocityGrid((n1, n2, hi - lo), (wl.vel_lo[0], wl.vel_lo[1], wl.vel_lo[2] + lo * h3),
                                  (wl.vel_hi[0], wl.vel_hi[1], wl.vel_lo[2] + (hi - 1) * h3))
        self.slab = ostage.Problem(self.full.mesh, wl.p, self.vslab, self.full.gas, dirichlet=wl.dirichlet)
        self.fn = f_slab.copy()
        self.fs = f_slab.copy()
        self.n_points = wl.n_elem * wl.n_sol

    def _partials(self, f):
        C, Nu = f.shape[:2]
        w, u = self.vg.w[self.sel], self.vg.u[self.sel]
        F = f[0].reshape(Nu, -1)
        m = np.zeros((11, F.shape[1]))
        m[0] = w @ F
        for d in range(3):
            m[1 + d] = (w * u[:, d]) @ F
        for j, (a, b) in enumerate(((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))):
            m[4 + j] = (w * u[:, a] * u[:, b]) @ F
        if C == 2:
            m[10] = w @ f[1].reshape(Nu, -1)
        return m

    def shard_partials(self, m):
        m.copy_(self.torch.from_numpy(self._partials(self.fs)))

    def shard_stage(self, m, stage, dt):
        obgk, gas = self.obgk, self.full.gas
        mm = m.numpy().T.copy()                                  # [P, 11], summed over the shards
        rho, U, E, theta, pres, Pi = obgk.macroscopic(mm, gas)
        tau = obgk.collision_time(theta, pres, gas)
        qp, _, conv, _ = obgk.solve_qprime(mm, gas, self.vg)     # the whole grid
        assert np.all(conv)
        g, Gg = obgk.equilibrium(qp, mm, gas, self.vslab)        # at this slab's velocities
        f = self.fs
        C, Nu = f.shape[:2]
        S = [(g - f[0].reshape(Nu, -1)) / tau[None, :]]
        if C == 2:
            S.append((Gg - f[1].reshape(Nu, -1)) / tau[None, :])
        R = np.stack(S).reshape(f.shape) - self.slab.divergence(f)
        a, b = ((0.0, 1.0), (0.75, 0.25), (1.0 / 3.0, 2.0 / 3.0))[stage]
        out = a * self.fn + b * (f + dt * R)
        if stage == 2:
            self.fn = out.copy()
        self.fs = out
        return 0


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    from paper_2312_06567_gb300 import workloads as W
    from paper_2312_06567_gb300.shard import ShardedStepper, velocity_slabs
    dist.init_process_group("gloo", rank=rank, world_size=world)
    wl = _workload()
    f = W.random_anisotropic_state(wl, seed=31)
    lo, hi = velocity_slabs(wl.vel_n[2], world)[rank]
    n12 = wl.vel_n[0] * wl.vel_n[1]
    shard = OracleShard(wl, f[:, lo * n12:hi * n12], lo, hi)
    m = torch.zeros((11, shard.n_points), dtype=torch.float64)
    stepper = ShardedStepper(shard, m, lambda t: dist.all_reduce(t))
    assert stepper.step(wl.dt(), 2) == 0
    parts = [None] * world
    dist.all_gather_object(parts, (lo, shard.fn))
    if rank == 0:
        q.put(parts)
    dist.barrier()
    dist.destroy_process_group()


def test_velocity_slabs_cover_the_axis():
    from paper_2312_06567_gb300.shard import velocity_slabs
    for n3, world in ((24, 2), (24, 5), (40, 8), (8, 4)):
        sl = velocity_slabs(n3, world)
        assert sl[0][0] == 0 and sl[-1][1] == n3 and len(sl) == world
        assert all(a[1] == b[0] for a, b in zip(sl, sl[1:]))
        sizes = [hi - lo for lo, hi in sl]
        assert min(sizes) >= 2 and max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        velocity_slabs(7, 4)


def test_two_rank_sharded_step_equals_the_unsharded_oracle():
    import torch.multiprocessing as mp
    from oracle import stage as ostage
    from paper_2312_06567_gb300 import workloads as W
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    parts = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    wl = _workload()
    f = W.random_anisotropic_state(wl, seed=31)
    pb = ostage.problem_from_workload(wl)
    ref = f
    for _ in range(2):
        ref, _ = pb.step(ref, wl.dt())
    got = np.concatenate([fp for _, fp in sorted(parts, key=lambda t: t[0])], axis=1)
    C, Nu = ref.shape[:2]
    err = np.abs(got - ref).reshape(C * Nu, -1).max(1) / np.abs(ref).reshape(C * Nu, -1).max(1)
    assert float(err.max()) <= 1e-12
