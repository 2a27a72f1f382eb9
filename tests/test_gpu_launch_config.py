"""The solve's launch configurations (same-shape pairs batched per launch or
one launch per pair; one branch stream per unit or two staggered lanes),
which the context chooses by timing, give the same potentials and the same
trajectory bit for bit: only the grouping of the launches and the order of
independent chains differ, never the arithmetic of a pair."""
import numpy as np
import pytest

from paper_1210_1736_gb300 import workloads as W
from tests._harness import gpu_setup, oracle_setup
from tests.test_gpu_parity import _sets

pytestmark = pytest.mark.gpu

CONFIGS = [(1, 0), (1, 1), (0, 0), (0, 1)]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_launch_configs_bit_identical(precision):
    import torch
    w = W.merger_small(precision=precision)
    system, _ = oracle_setup(w)
    sets = list(_sets(system))
    ref = None
    for batched, sched in CONFIGS:
        ctx, parts = gpu_setup(w)
        ctx.set_launch_config(batched, sched)
        assert ctx.info()["batched"] == batched
        ctx.deposit(parts)
        ctx.solve()
        torch.cuda.synchronize()
        phi = [ctx.potential(g, k) for g, k in sets]
        ctx.step(parts, w["dt"], 3)
        pos, vel, flags = parts.host()
        out = (phi, pos, vel, flags)
        if ref is None:
            ref = out
        else:
            for a, b in zip(ref[0], out[0]):
                assert np.array_equal(a, b), (batched, sched)
            for a, b in zip(ref[1:], out[1:]):
                assert np.array_equal(a, b), (batched, sched)
        ctx.close()


def test_launch_config_rejects_other_values():
    w = W.merger_small(precision="fp32")
    ctx, _ = gpu_setup(w)
    from paper_1210_1736_gb300 import pm
    with pytest.raises(pm.PMError):
        ctx.set_launch_config(2, 0)
    with pytest.raises(pm.PMError):
        ctx.set_launch_config(1, -1)
    ctx.close()
