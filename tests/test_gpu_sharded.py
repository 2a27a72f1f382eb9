"""The particle-sharded step through the library: two processes (gloo
ranks, both on the one GPU a test gets, the int64 sums through host
copies) each step half of the two-galaxy test system with ShardedStep; the
result must equal the single-process graph-replayed step bit for bit, since
the summed densities and centre-of-mass sums are exact integers and every
later kernel sees the same inputs."""
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_1210_1736_gb300 import workloads as W
from tests._harness import gpu_setup, require_cuda
from tests.test_multirank_host import ROOT, _free_port

pytestmark = pytest.mark.gpu


def test_two_rank_sharded_steps_equal_single_process(tmp_path):
    torch = require_cuda()
    out = str(tmp_path / "shard")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.join("tests", "_sharded_worker.py"), "gpu", out]
    r = subprocess.run(cmd, cwd=ROOT, env=dict(os.environ, OMP_NUM_THREADS="1"), capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]

    w = W.merger_small(precision="fp64")
    dt = w["dt"]
    ctx, parts = gpu_setup(w)
    ctx.deposit(parts)
    ctx.solve()
    ctx.kick(parts, -0.5 * dt)
    ctx.step(parts, dt, 3)
    torch.cuda.synchronize()
    pos, vel, flags = parts.host()
    n = len(w["m"])
    got_pos, got_vel, got_flags = np.zeros((3, n)), np.zeros((3, n)), np.zeros(n, np.int64)
    for rank in range(2):
        d = np.load(f"{out}.{rank}.npz")
        got_pos[:, d["idx"]], got_vel[:, d["idx"]], got_flags[d["idx"]] = d["pos"], d["vel"], d["flags"]
        assert np.array_equal(d["centres"], ctx.centres())
    assert np.array_equal(got_flags & 1, flags & 1)
    assert np.array_equal(got_pos, pos)
    assert np.array_equal(got_vel, vel)
    ctx.close()
