"""One rank of the sharded-step tests, launched by torch.distributed.run
(gloo, rendezvous on 127.0.0.1).  Rank r takes the particles r, r + W, ...
of the two-galaxy test system and steps them with ShardedStep.

  _sharded_worker.py oracle OUT   the context is OracleShard (CPU, the oracle)
  _sharded_worker.py gpu OUT      the context is the library's (cuda:0)

Each rank writes its particles' final state to OUT.rank.npz."""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import numpy as np  # noqa: E402
import torch  # noqa: E402
import torch.distributed as dist  # noqa: E402

import oracle as O  # noqa: E402
from paper_1210_1736_gb300 import workloads as W  # noqa: E402
from paper_1210_1736_gb300.sharded import ShardedStep  # noqa: E402

STEPS = 3


class OracleShard:
    """The context interface of ShardedStep computed by the oracle on CPU
    tensors: the exchange buffers hold every mass set's int64 density
    (flattened in set order) and the per-galaxy integer centre-of-mass sums."""

    def __init__(self, system, centres):
        self.system = system
        self.centres = np.array(centres, dtype=np.float64)
        self.sets = [(g, k, geom) for g, gal in enumerate(system.galaxies) for k, geom, _, _ in O.mass_sets(gal)]
        self.rho = torch.zeros(sum(int(np.prod(geom.shape)) for _, _, geom in self.sets), dtype=torch.int64)
        self.csum = torch.zeros(4 * len(system.galaxies), dtype=torch.int64)
        self.s = O.fixed_shift(system.mass_bound)

    def exchange_buffers(self):
        return self.rho, self.csum

    def recentre_sums(self, p):
        p.centres = self.centres
        self.csum += torch.from_numpy(O.recentre_sums(p, self.system).ravel())

    def recentre_apply(self):
        self.centres = O.recentre_apply(self.centres, self.csum.numpy().reshape(-1, 4), self.system)
        self.csum.zero_()

    def deposit(self, p):
        p.centres = self.centres
        flags, own = O.classify(p, self.system)
        rho, p.flags, self.s = O.deposit(p, self.system, flags, own)
        self.rho.copy_(torch.from_numpy(np.concatenate([rho[g][k].ravel() for g, k, _ in self.sets])))

    def solve(self):
        rho, off = [dict() for _ in self.system.galaxies], 0
        for g, k, geom in self.sets:
            n = int(np.prod(geom.shape))
            rho[g][k] = self.rho[off:off + n].numpy().reshape(geom.shape)
            off += n
        self.phi = O.solve_all(rho, self.system, self.s)

    def kick_drift(self, p, dt):
        acc = O.accelerations(p, self.system, self.phi, p.flags)
        live = (p.flags & O.FLAG_LOST) == 0
        p.vel = O.kick(p.vel, acc, dt, live)
        p.pos = O.drift(p.pos, p.vel, dt, live)


def main():
    mode, out = sys.argv[1], sys.argv[2]
    rank, world = int(os.environ["RANK"]), int(os.environ["WORLD_SIZE"])
    dist.init_process_group("gloo")
    w = W.merger_small(precision="fp64")
    mine = np.arange(rank, len(w["m"]), world)
    dt = w["dt"]
    if mode == "oracle":
        ww = dict(w)
        system = O.system_from_workload(ww, O.mass_bound(w["m"]))
        state = O.state_from_workload(ww)
        p = O.State(state.pos[:, mine], state.vel[:, mine], state.m[mine], state.gal[mine], state.flags[mine],
                    state.centres)
        sh = ShardedStep(OracleShard(system, state.centres))
        sh.step(p, dt, STEPS)
        np.savez(f"{out}.{rank}.npz", idx=mine, pos=p.pos, vel=p.vel, flags=p.flags, centres=sh.ctx.centres)
    else:
        from paper_1210_1736_gb300 import pm
        torch.cuda.set_device(0)
        ctx = pm.Context(w, O.mass_bound(w["m"]))
        parts = pm.Particles(w["pos"][:, mine], w["vel"][:, mine], w["m"][mine], w["gal"][mine], precision="fp64")
        sh = ShardedStep(ctx)
        sh.deposit(parts, recentre=False)      # leap-frog start at t = 0
        ctx.solve()
        ctx.kick(parts, -0.5 * dt)
        sh.step(parts, dt, STEPS)
        torch.cuda.synchronize()
        pos, vel, flags = parts.host()
        np.savez(f"{out}.{rank}.npz", idx=mine, pos=pos, vel=vel, flags=flags, centres=ctx.centres())
        ctx.close()
    dist.barrier()
    dist.destroy_process_group()


if __name__ == "__main__":
    main()
