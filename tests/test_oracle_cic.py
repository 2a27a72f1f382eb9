"""Pins of the CIC variant and of its adjoint in the oracle (CPU only).

The variant's forward is pinned by properties that trilinear assignment and
the central-difference field fix exactly: partition of unity, the first mass
moment, momentum conservation on one grid, and the Newtonian far field.  The
adjoint is pinned by directional finite differences of the oracle's own
forward map (FP64), for positions and masses, on a two-galaxy nested system."""
import numpy as np
import pytest

import oracle as O
from oracle import pm_cic as C
from paper_1210_1736_gb300 import workloads as W

RNG = np.random.default_rng(20121003)


def _one_grid_system(g, precision="fp64"):
    gal = O.Galaxy(coarse=g, medium=None, fine=None, r_core=0.0, r_out=0.0,
                   centre=(0.0, 0.0, 0.0), recentre=False)
    return O.System(galaxies=[gal], r_sys=1e9, sys_centre=(0.0, 0.0, 0.0), G=1.0, h000=1.0,
                    mass_bound=1e3, precision=precision)


def _state(pos, m, gal=None, centres=((0.0, 0.0, 0.0),)):
    n = pos.shape[1]
    return O.State(pos=pos.astype(np.float64), vel=np.zeros((3, n)), m=m.astype(np.float64),
                   gal=np.zeros(n, np.int64) if gal is None else gal,
                   flags=np.zeros(n, np.int64), centres=np.array(centres, dtype=np.float64))


def _acc(st, sysm):
    flags, own = O.classify(st, sysm)
    rho, flags = C.cic_deposit(st, sysm, flags, own)
    return C.cic_accelerations(st, sysm, C.cic_solve(rho, sysm), flags)


def test_weights_partition_of_unity():
    frac = RNG.uniform(0, 1, (3, 1000))
    ws = C.cic_weights(frac)
    assert np.allclose(sum(W for W, _ in ws.values()), 1.0, atol=1e-15)
    assert np.allclose(sum(dW for _, dW in ws.values()), 0.0, atol=1e-15)


def test_deposit_conserves_mass_and_first_moment():
    """Trilinear weights reproduce constants and linear functions exactly:
    sum_c rho_c = M and sum_c rho_c x_c = sum_i m_i x_i on every grid."""
    g = O.Geometry(16, 16, 8, 0.3, 0.15)
    sysm = _one_grid_system(g)
    n = 400
    pos = np.stack([RNG.uniform(-1.8, 1.5, n), RNG.uniform(-1.8, 1.5, n), RNG.uniform(-0.35, 0.2, n)])
    m = RNG.uniform(0.5, 1.5, n)
    st = _state(pos, m)
    rho, flags = C.cic_deposit(st, sysm)
    assert not np.any(flags & O.FLAG_LOST)
    grid = rho[0][5]
    assert abs(grid.sum() - m.sum()) < 1e-12 * m.sum()
    k, j, i = np.meshgrid(np.arange(g.nz), np.arange(g.ny), np.arange(g.nx), indexing="ij")
    xc = [(i - g.nx // 2) * g.l_xy, (j - g.ny // 2) * g.l_xy, (k - g.nz // 2) * g.l_z]
    for d in range(3):
        assert abs((grid * xc[d]).sum() - (m * pos[d]).sum()) < 1e-12 * np.abs(m * pos[d]).sum()


def test_momentum_conservation_one_grid():
    """Same weights for assignment and interpolation, an antisymmetric
    difference and a symmetric convolution: sum m a = 0 to rounding, for
    particles anywhere in their cells (unlike NGP + Taylor terms)."""
    g = O.Geometry(32, 32, 16, 0.2, 0.1)
    sysm = _one_grid_system(g)
    n = 300
    pos = np.stack([RNG.uniform(-2.4, 2.4, n), RNG.uniform(-2.4, 2.4, n), RNG.uniform(-0.5, 0.5, n)])
    m = RNG.uniform(0.5, 1.5, n)
    acc = _acc(_state(pos, m), sysm)
    tot = (m * acc).sum(axis=1)
    assert np.max(np.abs(tot)) < 1e-13 * (m * np.abs(acc)).sum()


@pytest.mark.parametrize("q", [1.0, 0.5])
def test_newton_far_field(q):
    l = 0.05
    g = O.Geometry(64, 64, int(64 / q), l, q * l)
    sysm = _one_grid_system(g)
    rng = np.random.default_rng(7)
    for _ in range(4):
        src = rng.uniform(-0.2, 0.2, 3)
        d = rng.normal(size=3)
        d = d / np.linalg.norm(d) * 1.2
        pos = np.stack([src, src + d], axis=1)
        acc = _acc(_state(pos, np.array([3.0, 1e-6])), sysm)[:, 1]
        newton = -3.0 * d / np.linalg.norm(d) ** 3
        assert np.linalg.norm(acc - newton) < 0.01 * np.linalg.norm(newton)


def _small_merger(precision="fp64", n_gal=1500, n_sat=300):
    w = W.merger_small(precision=precision)
    gal = np.asarray(w["gal"])
    rng = np.random.default_rng(5)
    idx = np.concatenate([rng.choice(np.nonzero(gal == 0)[0], n_gal, replace=False),
                          rng.choice(np.nonzero(gal == 1)[0], n_sat, replace=False)])
    w = dict(w, pos=w["pos"][:, idx], vel=w["vel"][:, idx], m=w["m"][idx], gal=gal[idx])
    return O.system_from_workload(w), O.state_from_workload(w)


def _acc_state(st, sysm):
    flags, own = O.classify(st, sysm)
    rho, flags = C.cic_deposit(st, sysm, flags, own)
    phi = C.cic_solve(rho, sysm)
    return C.cic_accelerations(st, sysm, phi, flags), phi, flags, own


def _regions(st, sysm):
    return [O.region(st.pos, gal, st.centres[h], sysm.split) for h, gal in enumerate(sysm.galaxies)]


def test_vjp_positions_matches_finite_differences():
    """<u, a(x + h e) - a(x - h e)> / 2h = <u^T da/dx, e>, a two-galaxy system
    with all five mass sets populated; h small enough that no particle
    changes region or CIC cell."""
    sysm, st = _small_merger()
    a0, phi, flags, own = _acc_state(st, sysm)
    live = (flags & O.FLAG_LOST) == 0
    assert live.all()
    u = RNG.normal(size=a0.shape)
    gx, gm = C.cic_vjp(st, sysm, phi, flags, own, u)
    for trial in range(3):
        e = RNG.normal(size=st.pos.shape)
        h = 1e-7
        sp, sm = st.copy(), st.copy()
        sp.pos = st.pos + h * e
        sm.pos = st.pos - h * e
        for a, b in zip(_regions(sp, sysm), _regions(sm, sysm)):
            assert np.array_equal(a, b)
        ap = _acc_state(sp, sysm)[0]
        am = _acc_state(sm, sysm)[0]
        fd = np.sum(u * (ap - am)) / (2 * h)
        ad = np.sum(gx * e)
        assert abs(fd - ad) < 1e-6 * abs(ad), (fd, ad)


def test_vjp_masses_matches_finite_differences():
    """a is linear in the masses, so the central difference is exact up to
    rounding."""
    sysm, st = _small_merger()
    a0, phi, flags, own = _acc_state(st, sysm)
    u = RNG.normal(size=a0.shape)
    gx, gm = C.cic_vjp(st, sysm, phi, flags, own, u)
    e = RNG.normal(size=st.m.shape) * st.m
    h = 1e-3
    sp, sm = st.copy(), st.copy()
    sp.m = st.m + h * e
    sm.m = st.m - h * e
    fd = np.sum(u * (_acc_state(sp, sysm)[0] - _acc_state(sm, sysm)[0])) / (2 * h)
    ad = np.sum(gm * e)
    assert abs(fd - ad) < 1e-9 * abs(ad), (fd, ad)


def test_planted_mistake_in_adjoint_is_caught(monkeypatch):
    """A sign error in the transposed difference must fail the position pin."""
    sysm, st = _small_merger(n_gal=600, n_sat=150)
    a0, phi, flags, own = _acc_state(st, sysm)
    u = RNG.normal(size=a0.shape)
    good = C.cic_vjp(st, sysm, phi, flags, own, u)[0]
    orig = C.grid_accel_T
    monkeypatch.setattr(C, "grid_accel_T", lambda f, g: -orig(f, g))
    bad = C.cic_vjp(st, sysm, phi, flags, own, u)[0]
    e = RNG.normal(size=st.pos.shape)
    h = 1e-7
    sp, sm = st.copy(), st.copy()
    sp.pos = st.pos + h * e
    sm.pos = st.pos - h * e
    fd = np.sum(u * (_acc_state(sp, sysm)[0] - _acc_state(sm, sysm)[0])) / (2 * h)
    assert abs(fd - np.sum(good * e)) < 1e-6 * abs(fd)
    assert abs(fd - np.sum(bad * e)) > 1e-3 * abs(fd)


def test_step_matches_kick_drift_of_accelerations():
    sysm, st = _small_merger(n_gal=600, n_sat=150)
    a, _, flags, _ = _acc_state(st, sysm)
    nxt = C.cic_step(st, sysm, 0.01)
    assert np.allclose(nxt.vel, st.vel + 0.01 * a, rtol=0, atol=1e-15)
    assert np.allclose(nxt.pos, st.pos + 0.01 * nxt.vel, rtol=0, atol=1e-15)


def test_trajectory_vjp_matches_central_differences():
    """The transpose of the whole leap-frog map (cic_trajectory_vjp, the
    per-step vector-Jacobian products chained newest first) against central
    differences of the oracle's own forward map (cic_trajectory), 4 steps of
    the two-galaxy system with the satellite inside the disc: directional
    derivatives along the satellite's positions, velocities and masses for a
    random cotangent of (x_T, v_T)."""
    from paper_1210_1736_gb300 import workloads as W
    w = W.merger_small(precision="fp64", r_apo=3.0)
    system = O.system_from_workload(w, 1.25 * O.mass_bound(w["m"]))
    st0 = O.state_from_workload(w)
    steps, dt = 4, w["dt"]
    xT, vT, tape = C.cic_trajectory(st0, system, dt, steps)
    rng = np.random.default_rng(1)
    lx, lv = rng.normal(size=xT.shape), rng.normal(size=vT.shape)
    gx, gv, gm = C.cic_trajectory_vjp(tape, system, dt, lx, lv)

    def J(dx=0.0, dv=0.0, dm=0.0):
        s = st0.copy()
        s.pos, s.vel, s.m = s.pos + dx, s.vel + dv, s.m + dm
        x, v, _ = C.cic_trajectory(s, system, dt, steps)
        return np.sum(lx * x) + np.sum(lv * v)

    sat = np.asarray(w["comp"]) == W.COMP_SATELLITE
    d = np.array([0.3, -0.5, 0.2])[:, None] * sat[None, :]
    h = 1e-8
    fx = (J(dx=h * d) - J(dx=-h * d)) / (2 * h)
    fv = (J(dv=h * d) - J(dv=-h * d)) / (2 * h)
    dm = st0.m * sat
    fm = (J(dm=1e-6 * dm) - J(dm=-1e-6 * dm)) / 2e-6
    assert np.sum(gx * d) == pytest.approx(fx, rel=1e-5)
    assert np.sum(gv * d) == pytest.approx(fv, rel=1e-5)
    assert np.sum(gm * dm) == pytest.approx(fm, rel=1e-5)
