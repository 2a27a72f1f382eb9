"""The particle-sharded step (paper_1210_1736_gb300.sharded) on CPU: two gloo
ranks launched as the multi-GPU bench is (torch.distributed.run, rendezvous
on 127.0.0.1), each stepping half of the two-galaxy test system, with the
oracle standing in for the library behind the same context interface.  The
two int64 sums (centre-of-mass accumulators, densities) must make the
sharded steps equal the single-process oracle steps bit for bit."""
import os

import numpy as np

import oracle as O
from paper_1210_1736_gb300 import workloads as W
from tests.test_multirank_host import ROOT, _launch


def test_two_rank_sharded_oracle_steps_equal_single_process(tmp_path):
    out = str(tmp_path / "shard")
    r = _launch([os.path.join("tests", "_sharded_worker.py"), "oracle", out], timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    w = W.merger_small(precision="fp64")
    system = O.system_from_workload(w, O.mass_bound(w["m"]))
    state = O.state_from_workload(w)
    for _ in range(3):
        state = O.step(state, system, w["dt"])
    n = len(state.m)
    pos, vel, flags = np.zeros((3, n)), np.zeros((3, n)), np.zeros(n, np.int64)
    for rank in range(2):
        d = np.load(f"{out}.{rank}.npz")
        pos[:, d["idx"]], vel[:, d["idx"]], flags[d["idx"]] = d["pos"], d["vel"], d["flags"]
        assert np.array_equal(d["centres"], state.centres)
    assert np.array_equal(pos, state.pos)
    assert np.array_equal(vel, state.vel)
    assert np.array_equal(flags, state.flags)
