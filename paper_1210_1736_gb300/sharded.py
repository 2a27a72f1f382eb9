"""One nested-grid step of a particle set sharded across processes.

Each process owns a disjoint part of the particles and a full copy of the
grids (one GPU each).  The paper parallelises its solver by splitting the
FFT into slabs across processes (Sec. 2.2.3); here the grids fit on every
GPU, so only the particles are split and the step needs two exchanges, both
element-wise sums of int64 buffers, exact and independent of the order in
which the processes' parts are added:

1. the centre-of-mass accumulators of the recentring (Sec. 2.1), after each
   process has added its particles' integer sums;
2. the densities of every mass set (Sec. 2.1, Eq. eqn:cell), after each
   process has deposited its particles.

Then every process solves the same potentials (replicated, identical) and
kicks and drifts its own particles.  The result equals the single-process
step bit for bit.

A context here is anything with the methods recentre_sums(p),
recentre_apply(), deposit(p), exchange_buffers() -> (rho, csum), solve() and
kick_drift(p, dt), such as pm.Context.  The sums use torch.distributed: on
device tensors directly (NCCL), or through host copies for a CPU backend
(gloo).
"""
from __future__ import annotations


class ShardedStep:
    def __init__(self, ctx, group=None):
        import torch.distributed as dist
        self.ctx = ctx
        self.group = group
        self.rho, self.csum = ctx.exchange_buffers()
        self.host = dist.get_backend(group) != "nccl" and self.rho.device.type != "cpu"

    def _sum(self, t):
        import torch.distributed as dist
        if self.host:
            h = t.cpu()
            dist.all_reduce(h, op=dist.ReduceOp.SUM, group=self.group)
            t.copy_(h)
        else:
            dist.all_reduce(t, op=dist.ReduceOp.SUM, group=self.group)

    def deposit(self, p, recentre=True):
        """Recentre (unless recentre is False) and deposit, with the sums
        across processes: afterwards every process holds the centres and
        densities of all particles."""
        if recentre:
            self.ctx.recentre_sums(p)
            self._sum(self.csum)
            self.ctx.recentre_apply()
        self.ctx.deposit(p)
        self._sum(self.rho)

    def step(self, p, dt, nsteps=1):
        """nsteps leap-frog steps of this process's particles p."""
        for _ in range(nsteps):
            self.deposit(p)
            self.ctx.solve()
            self.ctx.kick_drift(p, dt)
