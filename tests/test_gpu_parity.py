"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Density: bit-exact (int64).  Potentials and forces: FP64 path within 1e-12
relative, FP32 path within 2e-5 RMS and 1e-4 max relative (RMS-normalised,
per particle), plus drift of energy and angular momentum.  Sizes span several
tiles with ragged tails; the full 1M-particle workload is checked on all
density cells and on sampled particles.
"""
import numpy as np
import pytest

import oracle as O
from paper_1210_1736_gb300 import workloads as W
from tests._harness import (cast, gpu_setup, oracle_fields, oracle_setup,
                            rel_force_errors, require_cuda)

pytestmark = pytest.mark.gpu


def _sets(system):
    out = []
    for g, gal in enumerate(system.galaxies):
        for k, _, _, _ in O.mass_sets(gal):
            out.append((g, k))
    return out


def _gpu_fields(ctx, parts):
    ctx.deposit(parts)
    ctx.solve()
    acc = ctx.force(parts)
    import torch
    torch.cuda.synchronize()
    return np.stack([a.cpu().numpy().astype(np.float64) for a in acc])


def _compare_density_and_flags(ctx, parts, system, rho, flags):
    for g, k in _sets(system):
        got = ctx.density(g, k)
        assert np.array_equal(got, rho[g][k]), f"density of grid {k} (galaxy {g}) differs"
    _, _, gflags = parts.host()
    assert np.array_equal(gflags & 1, flags & 1), "lost flags differ"


def _phi_stored(phi, g, k):
    """The library keeps the potentials combined as the force stencils read
    them: grid 2 holds Phi_2 + Phi_3, grid 4 holds Phi_4 + Phi_5."""
    if k in (2, 4) and (k + 1) in phi[g]:
        return phi[g][k] + phi[g][k + 1]
    return phi[g][k]


def _phi_rel(ctx, system, phi):
    """Worst potential error relative to the galaxy's largest stored
    potential: a set can be empty (a satellite with no outer particles) while
    its pair partner is not, and then rounding of the shared transform is the
    only content of its part."""
    worst = 0.0
    sets = _sets(system)
    scale = {}
    for g, k in sets:
        scale[g] = max(scale.get(g, 0.0), np.max(np.abs(_phi_stored(phi, g, k))))
    for g, k in sets:
        got = ctx.potential(g, k).astype(np.float64)
        ref = _phi_stored(phi, g, k)
        worst = max(worst, np.max(np.abs(got - ref)) / max(scale[g], 1e-300))
    return worst


# --------------------------------------------------------------------- FP64 --

def test_plummer32_fp64_density_potential_force():
    w = W.plummer32()
    ctx, parts = gpu_setup(w)
    system, state = oracle_setup(w)
    rho, phi, flags, own, s = oracle_fields(system, state)
    a_gpu = _gpu_fields(ctx, parts)
    _compare_density_and_flags(ctx, parts, system, rho, flags)
    assert _phi_rel(ctx, system, phi) < 1e-12
    a_ref = O.accelerations(state, system, phi, flags)
    live = (flags & 1) == 0
    rms, mx = rel_force_errors(a_gpu, a_ref, live)
    assert mx < 1e-12, (rms, mx)


def test_plummer32_fp64_ten_steps():
    """Plummer sphere of 65,536 particles on one 32^3 grid: 10 leap-frog
    steps, dt = 0.01, FP64 trajectories."""
    w = W.plummer32()
    ctx, parts = gpu_setup(w)
    system, state = oracle_setup(w)
    dt = w["dt"]
    for _ in range(w["steps"]):
        state = O.step(state, system, dt)
    ctx.step(parts, dt, w["steps"])
    pos, vel, flags = parts.host()
    assert np.array_equal(flags & 1, state.flags & 1)
    live = (state.flags & 1) == 0
    dpos = np.max(np.abs(pos - state.pos)[:, live], axis=0)
    scale = np.max(np.abs(state.pos[:, live]))
    # a cell flip from a last-bit difference can move a particle's force by
    # O(l^2) terms; allow a handful of such particles
    bad = np.sum(dpos > 1e-11 * scale)
    assert bad <= max(3, live.sum() // 10000), (bad, dpos.max())


@pytest.mark.parametrize("shape", [(256, 16, 8, 1.0), (8, 256, 16, 1.0), (16, 8, 256, 1.0),
                                   (64, 32, 128, 0.25)])
def test_fp64_potential_all_transform_lengths(shape):
    """Every transform length 16..512 on each axis, FP64, random masses; the
    last case has flattened cells (l_z = l_xy / 4)."""
    nx, ny, nz, q = shape
    rng = np.random.default_rng(hash(shape) % 2**32)
    n = 4000
    l = 0.1
    half = np.array([nx, ny, nz]) / 2 - 3
    pos = (rng.uniform(-1, 1, (3, n)) * half[:, None]) * np.array([[l], [l], [l * q]])
    w = dict(name="box", precision="fp64", dt=0.01,
             system=dict(r_sys=1e9, sys_centre=(0.0, 0.0, 0.0), G=1.0, h000=1.0),
             galaxies=[dict(coarse=(nx, ny, nz, l * (nx - 4) / 2, q), medium=None, fine=None,
                            r_core=0.0, r_out=0.0, centre=(0.0, 0.0, 0.0), recentre=False)],
             pos=pos, vel=np.zeros_like(pos), m=rng.uniform(0.5, 2.0, n),
             gal=np.zeros(n, np.int32))
    ctx, parts = gpu_setup(w)
    system, state = oracle_setup(w)
    rho, phi, flags, own, s = oracle_fields(system, state)
    a_gpu = _gpu_fields(ctx, parts)
    _compare_density_and_flags(ctx, parts, system, rho, flags)
    assert _phi_rel(ctx, system, phi) < 1e-12
    a_ref = O.accelerations(state, system, phi, flags)
    rms, mx = rel_force_errors(a_gpu, a_ref, (flags & 1) == 0)
    assert mx < 1e-11, (rms, mx)


# --------------------------------------------------------------------- FP32 --

@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_galaxy_small_nested(precision):
    """Three nested geometries (32^3, flattened 32^3, 32x32x8), five grids."""
    w = W.galaxy_small(precision=precision)
    ctx, parts = gpu_setup(w)
    system, state = oracle_setup(w)
    rho, phi, flags, own, s = oracle_fields(system, state)
    a_gpu = _gpu_fields(ctx, parts)
    _compare_density_and_flags(ctx, parts, system, rho, flags)
    a_ref = O.accelerations(state, system, phi, flags)
    rms, mx = rel_force_errors(a_gpu, a_ref, (flags & 1) == 0)
    if precision == "fp64":
        assert _phi_rel(ctx, system, phi) < 1e-12
        assert mx < 1e-12, (rms, mx)
    else:
        assert _phi_rel(ctx, system, phi) < 2e-6
        assert rms < 2e-5 and mx < 1e-4, (rms, mx)


def test_galaxy_1m_full_size():
    """The 1M-particle disc-bulge-halo workload at full size (128^3,
    flattened 128^3, 128x128x32): every density cell bit-exact, FP32 forces
    of 4096 sampled particles against the oracle."""
    w = W.galaxy_1m()
    ctx, parts = gpu_setup(w)
    system, state = oracle_setup(w)
    rho, phi, flags, own, s = oracle_fields(system, state)
    a_gpu = _gpu_fields(ctx, parts)
    _compare_density_and_flags(ctx, parts, system, rho, flags)
    assert _phi_rel(ctx, system, phi) < 2e-6
    rng = np.random.default_rng(5)
    live = np.flatnonzero((flags & 1) == 0)
    idx = np.sort(rng.choice(live, 4096, replace=False))
    sub = O.State(pos=state.pos[:, idx], vel=state.vel[:, idx], m=state.m[idx], gal=state.gal[idx],
                  flags=flags[idx], centres=state.centres)
    a_ref = O.accelerations(sub, system, phi, flags[idx])
    rms, mx = rel_force_errors(a_gpu[:, idx], a_ref, np.ones(len(idx), bool))
    assert rms < 2e-5 and mx < 1e-4, (rms, mx)


def test_recentre_bit_exact():
    w = W.galaxy_small(precision="fp32")
    rng = np.random.default_rng(3)
    pos = w["pos"] + np.array([[0.05], [-0.03], [0.02]]) + rng.normal(0, 1e-3, w["pos"].shape)
    ctx, parts = gpu_setup(w, pos=pos)
    system, state = oracle_setup(w, pos=pos)
    ctx.recentre(parts)
    got = ctx.centres()
    ref = O.recentre(state, system)
    assert np.array_equal(got, ref), (got, ref)


def test_step_galaxy_small_fp32_short():
    """Five full steps (recentre, deposit, solve, kick-drift) FP32 vs FP64."""
    w = W.galaxy_small(precision="fp32")
    ctx, parts = gpu_setup(w)
    system, state = oracle_setup(w)
    for _ in range(5):
        state = O.step(state, system, w["dt"])
    ctx.step(parts, w["dt"], 5)
    pos, vel, flags = parts.host()
    live = (state.flags & 1) == 0
    assert np.array_equal(flags & 1, state.flags & 1)
    dv = np.sqrt(np.sum((vel - state.vel)[:, live] ** 2, axis=0))
    vscale = np.sqrt(np.mean(np.sum(state.vel[:, live] ** 2, axis=0)))
    assert np.sqrt(np.mean(dv**2)) < 1e-5 * vscale
    assert np.max(np.abs(ctx.centres() - state.centres)) < 1e-5


def test_step_graph_cache_alternating_sets():
    """The context keeps the captured steps of its four most recently stepped
    particle sets and replaces the least recently used.  Steps alternating
    over five sets on one context (so captures are evicted and retaken)
    equal each set stepped alone, bit for bit: with a fixed grid centre and
    no sorting the sets share no state that changes their results."""
    w = W.plummer32()
    dt = w["dt"]
    ctx, _ = gpu_setup(w)
    rng = np.random.default_rng(5)
    sets = []
    for _ in range(5):
        pos = w["pos"] + rng.normal(0, 1e-3, w["pos"].shape)
        sets.append(pm_particles_like(w, pos))
    order = [0, 1, 2, 3, 0, 4, 1, 2, 2, 3, 4, 0, 1]
    for i in order:
        ctx.step(sets[i][0], dt, 1)
    counts = [order.count(i) for i in range(5)]
    for i, (parts, pos) in enumerate(sets):
        ref_ctx, ref = gpu_setup(w, pos=pos)
        ref_ctx.step(ref, dt, counts[i])
        for a, b in zip(parts.host(), ref.host()):
            assert np.array_equal(a, b)


def pm_particles_like(w, pos):
    from paper_1210_1736_gb300 import pm
    return pm.Particles(cast(w, pos), cast(w, w["vel"]), cast(w, w["m"]), w["gal"], precision=w["precision"]), pos


# ------------------------------------------------------------- edge cases --

def test_empty_particle_set():
    w = W.galaxy_small(precision="fp32")
    e = np.zeros((3, 0))
    ctx, parts = gpu_setup(w, pos=e, vel=e, m=np.zeros(0) + 1.0, gal=np.zeros(0, np.int32))
    ctx.deposit(parts)
    ctx.solve()
    ctx.step(parts, 0.01, 2)
    for k in range(1, 6):
        assert not ctx.density(0, k).any()
        assert not ctx.potential(0, k).any()


def test_all_lost_and_nonfinite():
    w = W.galaxy_small(precision="fp32")
    n = 1000
    rng = np.random.default_rng(9)
    pos = rng.uniform(40, 50, (3, n))
    pos[0, :10] = np.nan
    pos[1, 10:20] = np.inf
    vel = np.zeros((3, n))
    m = np.full(n, 1e-3)
    ctx, parts = gpu_setup(w, pos=pos, vel=vel, m=m, gal=np.zeros(n, np.int32))
    ctx.step(parts, 0.01, 3)
    assert ctx.count_lost(parts) == n
    p2, _, _ = parts.host()
    assert np.array_equal(np.isnan(p2), np.isnan(pos.astype(np.float32)))
    fin = np.isfinite(pos)
    assert np.array_equal(p2[fin], pos.astype(np.float32).astype(np.float64)[fin])
    for k in range(1, 6):
        assert not ctx.density(0, k).any()


def test_cell_edge_ties_bit_exact():
    """Particles exactly on cell faces (u + 1/2 integral) follow floor(u+1/2)."""
    w = W.plummer32()
    l = 0.25
    rng = np.random.default_rng(11)
    n = 5000
    cells = rng.integers(-12, 12, (3, n)).astype(np.float64)
    pos = (cells + 0.5) * l
    pos[:, ::3] = cells[:, ::3] * l
    m = np.full(n, 1.0 / n)
    ctx, parts = gpu_setup(w, pos=pos, vel=np.zeros_like(pos), m=m, gal=np.zeros(n, np.int32))
    system, state = oracle_setup(w, pos=pos, vel=np.zeros_like(pos), m=m, gal=np.zeros(n, np.int32))
    rho, phi, flags, own, s = oracle_fields(system, state)
    ctx.deposit(parts)
    _compare_density_and_flags(ctx, parts, system, rho, flags)


def _ulp_nudged(x, k, dtype):
    """x moved by k units in the last place of dtype (elementwise)."""
    x = np.asarray(x, dtype=dtype)
    out = x.copy()
    for step in range(int(np.max(np.abs(k))) if np.size(k) else 0):
        move = np.abs(k) > step
        out[move] = np.nextafter(out[move], np.where(k[move] > 0, np.inf, -np.inf).astype(dtype))
    return out


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_region_and_box_boundaries_bit_exact(precision):
    """Particles within a few units in the last place of every decision
    boundary of the nested geometry: the spheres R_core, R_out and R_sys,
    and both edges of the usable box (cells 2 .. n-3) of each grid on each
    axis (the cell length is 2R/(n-4); the box spans offsets -R(n-3)/(n-4)
    .. R(n-5)/(n-4) from its centre).  Region, cell and lost decisions --
    hence every density and the lost flags -- must be bit-exact with the
    oracle, which takes them with the same canonical FP32 offsets."""
    w = W.galaxy_small(precision=precision)
    g, sysd = w["galaxies"][0], w["system"]
    dtype = np.float32 if precision == "fp32" else np.float64
    rng = np.random.default_rng(23)
    pts = []
    # spheres about the (initial) galaxy centre, which is the origin
    for R in (g["r_core"], g["r_out"], sysd["r_sys"]):
        u = rng.normal(size=(3, 900))
        u /= np.linalg.norm(u, axis=0)
        pts.append(_ulp_nudged(u * R, rng.integers(-3, 4, (3, 900)), dtype))
    # usable-box edges of each grid (all three centred on the origin here)
    for key in ("coarse", "medium", "fine"):
        n3 = g[key][:3]
        R, q = g[key][3], g[key][4]
        l_xy = 2.0 * R / (n3[0] - 4)
        for ax in range(3):
            n = n3[ax]
            l = l_xy if ax < 2 else q * l_xy
            for edge in ((1.5 - n / 2) * l, (n / 2 - 2.5) * l):
                p = rng.uniform(-0.3, 0.3, (3, 300)) * min(R, 0.9 * g["r_core"])
                p[ax] = edge
                k = np.zeros((3, 300), dtype=np.int64)
                k[ax] = rng.integers(-3, 4, 300)
                pts.append(_ulp_nudged(p, k, dtype))
    pos = np.concatenate(pts, axis=1).astype(np.float64)
    n = pos.shape[1]
    m = np.full(n, 1.0 / n)
    gal = np.zeros(n, np.int32)
    ctx, parts = gpu_setup(w, pos=pos, vel=np.zeros_like(pos), m=m, gal=gal)
    system, state = oracle_setup(w, pos=pos, vel=np.zeros_like(pos), m=m, gal=gal)
    rho, phi, flags, own, s = oracle_fields(system, state)
    ctx.deposit(parts)
    _compare_density_and_flags(ctx, parts, system, rho, flags)
    lost = flags & 1
    assert 0 < lost.sum() < n                 # both sides of R_sys are represented


def test_bounded_wait_expiry_reported():
    """Failure detection without a GPU fault: one block waits, with the
    bounded wait the FFT passes use for their tensor copies, on a barrier
    nothing arrives at.  The wait gives up at its limit (about 2 s), the
    block sets the device error flag and the host reads PM_E_TIMEOUT.  The
    flag is cleared again: the same context then deposits and solves without
    error, with results equal to a fresh context's."""
    import time
    from paper_1210_1736_gb300 import pm
    w = W.galaxy_small(precision="fp32")
    ctx, parts = gpu_setup(w)
    t0 = time.perf_counter()
    assert ctx.selftest_wait_expiry() == pm.PM_E_TIMEOUT
    assert time.perf_counter() - t0 > 1.5
    ctx.deposit(parts)
    ctx.solve()
    ctx2, p2 = gpu_setup(w)
    ctx2.deposit(p2)
    ctx2.solve()
    for k in range(1, 6):
        assert np.array_equal(ctx.density(0, k), ctx2.density(0, k))
        assert np.array_equal(ctx.potential(0, k), ctx2.potential(0, k))


def test_deposit_deterministic_repeat():
    w = W.galaxy_small(precision="fp32")
    ctx, parts = gpu_setup(w)
    ctx.deposit(parts)
    first = [ctx.density(0, k) for k in range(1, 6)]
    for _ in range(3):
        ctx.deposit(parts)
        for k in range(1, 6):
            assert np.array_equal(ctx.density(0, k), first[k - 1])


# ----------------------------------------------------------------- drift --

@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_energy_angular_momentum_drift_100_steps(precision):
    """100 steps of the nested small galaxy: the relative drifts of E and |L|
    match the oracle's (within 1e-12 on the FP64 path, 1e-6 on FP32)."""
    w = W.galaxy_small(precision=precision)
    dt = w["dt"]
    ctx, parts = gpu_setup(w)
    system, state = oracle_setup(w)
    state = O.half_kick_start(state, system, dt)
    d0 = O.diagnostics(state, system, dt)
    for _ in range(100):
        state = O.step(state, system, dt)
    d1 = O.diagnostics(state, system, dt)

    ctx.deposit(parts)
    ctx.solve()
    ctx.kick(parts, -0.5 * dt)
    g0 = ctx.diagnostics(parts, dt)
    ctx.step(parts, dt, 100)
    g1 = ctx.diagnostics(parts, dt)

    dE_ref = (d1["E"] - d0["E"]) / abs(d0["E"])
    dE_gpu = (g1["E"] - g0["E"]) / abs(g0["E"])
    Lr0, Lr1 = np.linalg.norm(d0["L"]), np.linalg.norm(d1["L"])
    Lg0, Lg1 = np.linalg.norm(g0["L"]), np.linalg.norm(g1["L"])
    dL_ref = (Lr1 - Lr0) / Lr0
    dL_gpu = (Lg1 - Lg0) / Lg0
    tol = 1e-12 if precision == "fp64" else 1e-6
    print(f"{precision}: dE oracle {dE_ref:.3e} gpu {dE_gpu:.3e}; dL oracle {dL_ref:.3e} gpu {dL_gpu:.3e}")
    assert abs(g0["E"] - d0["E"]) < (1e-12 if precision == "fp64" else 1e-5) * abs(d0["E"])
    assert abs(dE_gpu - dE_ref) < tol, (dE_gpu, dE_ref)
    assert abs(dL_gpu - dL_ref) < tol, (dL_gpu, dL_ref)


def test_energy_angular_momentum_drift_100_steps_galaxy_1m():
    """The 1M-particle galaxy (128^3, 128^3 q = 1/4, 128x128x32), FP32,
    100 steps: the relative drifts of E and |L| match the oracle's within
    1e-6 (the oracle's FFTs on all host cores)."""
    import os
    O.set_fft_workers(os.cpu_count())
    try:
        w = W.galaxy_1m(precision="fp32")
        dt = w["dt"]
        ctx, parts = gpu_setup(w)
        ctx.deposit(parts)
        ctx.solve()
        ctx.kick(parts, -0.5 * dt)
        g0 = ctx.diagnostics(parts, dt)
        ctx.step(parts, dt, 100)
        g1 = ctx.diagnostics(parts, dt)
        ctx.close()
        system, state = oracle_setup(w)
        state = O.half_kick_start(state, system, dt)
        d0 = O.diagnostics(state, system, dt)
        for _ in range(100):
            state = O.step(state, system, dt)
        d1 = O.diagnostics(state, system, dt)
    finally:
        O.set_fft_workers(None)
    dE_ref = (d1["E"] - d0["E"]) / abs(d0["E"])
    dE_gpu = (g1["E"] - g0["E"]) / abs(g0["E"])
    dL_ref = (np.linalg.norm(d1["L"]) - np.linalg.norm(d0["L"])) / np.linalg.norm(d0["L"])
    dL_gpu = (np.linalg.norm(g1["L"]) - np.linalg.norm(g0["L"])) / np.linalg.norm(g0["L"])
    print(f"galaxy_1m: dE oracle {dE_ref:.3e} gpu {dE_gpu:.3e}; dL oracle {dL_ref:.3e} gpu {dL_gpu:.3e}")
    assert abs(g0["E"] - d0["E"]) < 1e-5 * abs(d0["E"])
    assert abs(dE_gpu - dE_ref) < 1e-6, (dE_gpu, dE_ref)
    assert abs(dL_gpu - dL_ref) < 1e-6, (dL_gpu, dL_ref)
