"""The spatial sort (pm_sort / pm_set_sort_interval) through the C ABI.

Sorting is a locality optimisation: it must permute every particle array
consistently, order particles by (galaxy, region, cell), and leave every
physical result unchanged (bit-exact density with plain or warp-aggregated
atomics; stepped trajectories equal as a set of particle states).
"""
import numpy as np
import pytest

import oracle as O
from paper_1210_1736_gb300 import workloads as W
from tests._harness import gpu_setup, oracle_setup, require_cuda

pytestmark = pytest.mark.gpu

FIELDS = ("x", "y", "z", "vx", "vy", "vz", "m", "gal", "flags")


def _host(parts):
    return {k: getattr(parts, k).cpu().numpy().copy() for k in FIELDS}


def _expected_keys(w, system, state):
    """(galaxy, region, cell of that region's grid) for every particle, from
    the oracle's classification, in a comparable integer form."""
    flags, own = O.classify(state, system)
    key = np.zeros(len(state.m), dtype=np.int64)
    for g, gal in enumerate(system.galaxies):
        sel = state.gal == g
        for reg, geom, cen in ((0, gal.fine, state.centres[g]), (1, gal.medium, state.centres[g]),
                               (2, gal.coarse, system.sys_centre)):
            s2 = sel & (own == reg) & ((flags & 1) == 0)
            if geom is None or not np.any(s2):
                continue
            (a, b, c), ok = O.grid_cells(state.pos[:, s2], cen, geom, system.split)
            key[s2] = ((g * 3 + reg) << 40) + (c * geom.ny + b) * geom.nx + a
    key[(flags & 1) != 0] = np.iinfo(np.int64).max
    return key


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_sort_permutes_consistently_and_orders_by_cell(precision):
    torch = require_cuda()
    w = W.galaxy_small(precision=precision)
    ctx, parts = gpu_setup(w)
    ctx.deposit(parts)
    before = _host(parts)
    rho0 = [ctx.density(0, k) for k in range(1, 6)]
    perm = torch.empty(parts.n, dtype=torch.int64, device="cuda")
    ctx.sort(parts, perm)
    torch.cuda.synchronize()
    after = _host(parts)
    pm_ = perm.cpu().numpy()
    assert np.array_equal(np.sort(pm_), np.arange(parts.n))
    for k in FIELDS:
        assert np.array_equal(after[k], before[k][pm_]), k
    # order: non-decreasing (galaxy, region, cell) by the oracle's classification
    system, state = oracle_setup(w, pos=np.stack([after["x"], after["y"], after["z"]]).astype(np.float64),
                                 vel=np.stack([after["vx"], after["vy"], after["vz"]]).astype(np.float64),
                                 m=after["m"].astype(np.float64), gal=after["gal"])
    keys = _expected_keys(w, system, state)
    assert np.all(np.diff(keys) >= 0)
    # density unchanged, plain atomics and warp-aggregated atomics
    for interval in (0, 1):
        ctx.set_sort_interval(interval)
        ctx.deposit(parts)
        for k in range(1, 6):
            assert np.array_equal(ctx.density(0, k), rho0[k - 1])


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_step_with_periodic_sort_equals_unsorted(precision):
    require_cuda()
    w = W.galaxy_small(precision=precision)
    ctxA, pA = gpu_setup(w)
    ctxB, pB = gpu_setup(w)
    ctxB.set_sort_interval(2)
    ctxA.step(pA, w["dt"], 7)
    ctxB.step(pB, w["dt"], 7)
    a, b = _host(pA), _host(pB)
    rows = lambda h: np.stack([h[k].astype(np.float64) for k in FIELDS], axis=1)  # noqa: E731
    ra, rb = rows(a), rows(b)
    ra = ra[np.lexsort(ra.T[::-1])]
    rb = rb[np.lexsort(rb.T[::-1])]
    assert np.array_equal(ra, rb)
    assert np.array_equal(ctxA.centres(), ctxB.centres())
