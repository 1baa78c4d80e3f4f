"""Velocity-sharded SSP-RK3 stepping across ranks (one GPU per rank).

The discrete-velocity BGK method couples velocities only through the moments
of f (section "Numerical method"): the FR advection of each velocity is
independent, and the BGK source needs Q of the whole velocity set.  A shard
(bgk_create_shard) holds a slab of third-axis velocity planes; each stage the
ranks sum their partial raw moments (11 doubles per point) with one
all-reduce, then every rank solves Q' for every point over the whole grid and
advances its own velocities.  No other data moves between ranks.

This module is the host logic: how the planes are split and the order of the
calls.  The collective is passed in (torch.distributed.all_reduce on a
process group, or any callable that sums a tensor over the ranks in place).
"""


def velocity_slabs(n3, world):
    """Split the n3 third-axis velocity planes into `world` contiguous slabs
    [lo, hi) of near-equal size (the first n3 % world slabs one plane larger),
    each of at least two planes."""
    if world < 1 or n3 < 2 * world:
        raise ValueError("need at least two velocity planes per shard (n3=%d, world=%d)" % (n3, world))
    base, extra = divmod(n3, world)
    out, lo = [], 0
    for r in range(world):
        hi = lo + base + (1 if r < extra else 0)
        out.append((lo, hi))
        lo = hi
    return out


class ShardedStepper:
    """Steps one shard in lockstep with the others.

    shard: an object with n_points, shard_partials(m) and shard_stage(m, stage, dt)
           (a bgk.Solver created with shard=(lo, hi), or a stand-in);
    m: the exchange tensor [11, n_points] float64 on the shard's device;
    all_reduce: callable summing m over all ranks in place.
    """

    def __init__(self, shard, m, all_reduce):
        self.shard = shard
        self.m = m
        self.all_reduce = all_reduce

    def step(self, dt, n_steps=1):
        """n_steps SSP-RK3 steps; returns the last non-OK status (or 0)."""
        status = 0
        for _ in range(n_steps):
            for stage in range(3):
                self.shard.shard_partials(self.m)
                self.all_reduce(self.m)
                st = self.shard.shard_stage(self.m, stage, dt)
                if st:
                    status = st
        return status
