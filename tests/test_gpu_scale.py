"""Parity at the workloads' structure and size limits: two galaxies with their
own nested grids (the merger layout), the largest grids (256^3, every
transform of length 512) checked on every density cell and on sampled
potential cells that the oracle sums directly (Eq. eq:poisson), and the FP32
forces of the full-size merger (4.1M particles) and large (16.5M particles)
workloads on sampled particles."""
import os

import numpy as np
import pytest

import oracle as O
from paper_1210_1736_gb300 import workloads as W
from tests._harness import (gpu_setup, oracle_fields, oracle_setup, rel_force_errors,
                            require_cuda)
from tests.test_gpu_parity import _compare_density_and_flags, _phi_rel, _phi_stored, _sets

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_merger_two_galaxies(precision):
    """Galaxy (32^3, 32^3 q=0.8, 32x32x8) + satellite (16^3 x 3): ten mass
    sets, four pair transforms per galaxy pair layout, forces summed over
    both galaxies by the combination rule."""
    w = W.merger_small(precision=precision)
    ctx, parts = gpu_setup(w)
    system, state = oracle_setup(w)
    rho, phi, flags, own, s = oracle_fields(system, state)
    ctx.deposit(parts)
    ctx.solve()
    acc = ctx.force(parts)
    import torch
    torch.cuda.synchronize()
    a_gpu = np.stack([a.cpu().numpy().astype(np.float64) for a in acc])
    _compare_density_and_flags(ctx, parts, system, rho, flags)
    a_ref = O.accelerations(state, system, phi, flags)
    rms, mx = rel_force_errors(a_gpu, a_ref, (flags & 1) == 0)
    if precision == "fp64":
        assert _phi_rel(ctx, system, phi) < 1e-12
        assert mx < 1e-12, (rms, mx)
    else:
        assert _phi_rel(ctx, system, phi) < 2e-6
        assert rms < 2e-5 and mx < 1e-4, (rms, mx)


def test_merger_steps_fp64():
    """Five full steps with both galaxies recentring (FP64)."""
    w = W.merger_small(precision="fp64")
    ctx, parts = gpu_setup(w)
    system, state = oracle_setup(w)
    for _ in range(5):
        state = O.step(state, system, w["dt"])
    ctx.step(parts, w["dt"], 5)
    pos, vel, flags = parts.host()
    assert np.array_equal(flags & 1, state.flags & 1)
    live = (state.flags & 1) == 0
    # a last-bit difference can flip a particle's cell (O(l^2) force change);
    # allow a handful of such particles
    bad = np.sum(np.max(np.abs(pos - state.pos)[:, live], axis=0) > 1e-9)
    assert bad <= max(3, live.sum() // 10000), bad
    # centres are quantised at 2^-24 R_core by the exact integer sums
    assert np.max(np.abs(ctx.centres() - state.centres)) < 1e-6


def _sampled_potential_check(ctx, system, rho, s, nsample, tol, seed):
    rng = np.random.default_rng(seed)
    worst = 0.0
    fields = {(g, k): ctx.potential(g, k).astype(np.float64) for g, k in _sets(system)}
    gscale = {}
    for (g, k), f in fields.items():   # errors relative to the galaxy's largest potential
        gscale[g] = max(gscale.get(g, 0.0), np.max(np.abs(f)))
    for g, k in _sets(system):
        geom = dict((kk, gg) for kk, gg, _, _ in O.mass_sets(system.galaxies[g]))[k]
        got = fields[(g, k)]
        scale = gscale[g]
        cells = list(zip(rng.integers(0, geom.nz, nsample), rng.integers(0, geom.ny, nsample),
                         rng.integers(0, geom.nx, nsample)))
        # plus the cells of the heaviest density (the deepest potential)
        kk, jj, ii = np.unravel_index(np.argmax(rho[g][k]), rho[g][k].shape)
        cells.append((kk, jj, ii))
        ref = O.potential_at(O.rho_real(rho[g][k], s), geom, system.G, system.h000, cells)
        if k in (2, 4) and (k + 1) in rho[g]:   # stored combined with the partner grid
            ref = ref + O.potential_at(O.rho_real(rho[g][k + 1], s), geom, system.G, system.h000, cells)
        err = np.max(np.abs(np.array([got[c] for c in cells]) - ref)) / scale
        worst = max(worst, err)
    print(f"sampled potential: worst rel err {worst:.3e}")
    assert worst < tol


def test_box_256_largest_transforms():
    """1M-particle Plummer sphere on one 256^3 grid (transforms of 512 on
    every axis): every density cell bit-exact, 64 sampled potential cells."""
    w = W.big_box()
    ctx, parts = gpu_setup(w)
    system, state = oracle_setup(w)
    flags, own = O.classify(state, system)
    rho, flags, s = O.deposit(state, system, flags, own)
    ctx.deposit(parts)
    ctx.solve()
    _compare_density_and_flags(ctx, parts, system, rho, flags)
    _sampled_potential_check(ctx, system, rho, s, 64, 2e-6, 1)


def test_galaxy_256_nested_largest_grids():
    """2M-particle galaxy on 256^3, flattened 256^3 and 256x256x64 grids
    (the large-run layout): all five densities bit-exact, sampled potentials."""
    w = W.galaxy_256()
    ctx, parts = gpu_setup(w)
    system, state = oracle_setup(w)
    flags, own = O.classify(state, system)
    rho, flags, s = O.deposit(state, system, flags, own)
    ctx.deposit(parts)
    ctx.solve()
    _compare_density_and_flags(ctx, parts, system, rho, flags)
    _sampled_potential_check(ctx, system, rho, s, 24, 2e-6, 2)


@pytest.mark.parametrize("name", ["merger_4m", "large_16m"])
def test_fp32_forces_full_size(name):
    """The full-size workloads in FP32: every density cell bit-exact and
    every lost flag equal; forces (Eq. eqn:diff by the combination rule) on
    every satellite particle and a uniform sample of 400k particles against
    the oracle: RMS error < 2e-5 and largest error < 1e-4 of the RMS force
    (reading r14; the RMS force and the RMS error from the uniform sample)."""
    import torch
    require_cuda()
    O.set_fft_workers(os.cpu_count())
    try:
        w = getattr(W, name)()
        ctx, parts = gpu_setup(w)
        ctx.deposit(parts)
        ctx.solve()
        acc = ctx.force(parts)
        torch.cuda.synchronize()
        a_gpu = np.stack([a.cpu().numpy().astype(np.float64) for a in acc])
        system, state = oracle_setup(w)
        flags, own = O.classify(state, system)
        rho, flags, s = O.deposit(state, system, flags, own)
        _compare_density_and_flags(ctx, parts, system, rho, flags)
        ctx.close()
        del parts
        phi = O.solve_all(rho, system, s)
        n = len(state.m)
        rng = np.random.default_rng(7)
        uni = rng.choice(n, 400_000, replace=False)
        sat = np.nonzero(np.asarray(w["comp"]) == W.COMP_SATELLITE)[0]
        idx = np.union1d(uni, sat)
        sub = O.State(state.pos[:, idx], state.vel[:, idx], state.m[idx], state.gal[idx], flags[idx],
                      state.centres)
        a_ref = O.accelerations(sub, system, phi, flags[idx])
        live = (flags[idx] & 1) == 0
        in_uni = np.isin(idx, uni)
        d = np.sqrt(np.sum((a_gpu[:, idx] - a_ref) ** 2, axis=0))
        f = np.sqrt(np.sum(a_ref ** 2, axis=0))
        rms_ref = np.sqrt(np.mean(f[live & in_uni] ** 2))
        rms = np.sqrt(np.mean(d[live & in_uni] ** 2)) / rms_ref
        mx = np.max(d[live]) / rms_ref
        mx_sat = np.max(d[live & ~in_uni], initial=0.0) / rms_ref
        print(f"{name}: force error rms {rms:.3e} max {mx:.3e} (satellites {mx_sat:.3e}), "
              f"{int(live.sum())} particles")
        assert rms < 2e-5 and mx < 1e-4, (rms, mx)
    finally:
        O.set_fft_workers(None)
