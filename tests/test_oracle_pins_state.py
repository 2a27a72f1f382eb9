"""Pins of the oracle's recentring, energy and angular momentum, potential at
a particle, lost flags and canonical cell index, each against what the paper
and plain mathematics fix rather than against the oracle's own arithmetic.

* recentre (Sec. 2.1, grids 1-3 follow the galaxy by its centre of mass):
  exactly the centre of a symmetric cloud; within the stated quantisation
  bound of the plain FP64 centre of mass of a random cloud; light particles
  kept to 20 bits.
* diagnostics (Sec. 6.4 quantities): K and L = I omega of a rigid rotation;
  W of two particles written out from Eq. (eqn:greens); the half kick to the
  synchronised time.
* phi_at_particle / accel_from_grid: exact on a linear field, flattened cells.
* lost_mask (Sec. 2.1 lost particles): particles just inside and outside
  R_sys and both usable-box edges of two coarse grids of different sizes.
* canonical cell index (Eq. eqn:cell, nearest integer): both FP32 offset rules
  disagree with the exact nearest integer only within a few FP32 ulps of a
  cell face.
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np
import pytest

import oracle as O


def _system(gals, r_sys=50.0, sys_centre=(0.0, 0.0, 0.0), G=1.0, h000=1.0, mb=1.0, precision="fp64"):
    return O.System(galaxies=gals, r_sys=r_sys, sys_centre=sys_centre, G=G, h000=h000, mass_bound=mb,
                    precision=precision)


def _galaxy(r_core=1.5, recentre=True):
    g = O.Geometry(32, 32, 32, O.cell_length(20.0, 32), O.cell_length(20.0, 32))
    return O.Galaxy(coarse=g, r_core=r_core, r_out=4 * r_core, recentre=recentre)


def _state(pos, m, gal, centres, flags=None, vel=None):
    n = pos.shape[1]
    return O.State(pos=np.asarray(pos, np.float64), vel=np.zeros((3, n)) if vel is None else vel,
                   m=np.asarray(m, np.float64), gal=np.asarray(gal, np.int64),
                   flags=np.zeros(n, np.int64) if flags is None else flags,
                   centres=np.asarray(centres, np.float64))


# ----------------------------------------------------------------- recentre ---

def test_recentre_symmetric_cloud_gives_its_centre_exactly():
    """Pairs c0 +- d of equal mass around c0 (all numbers exact in FP32): the
    centre of mass is c0 exactly.  Heavy particles outside R_core of the
    previous centre, particles of another galaxy and lost particles inside it
    must all be left out."""
    rng = np.random.default_rng(1)
    c_prev = np.array([2.0 ** -6, 0.0, -(2.0 ** -7)])
    c0 = c_prev + np.array([2.0 ** -8, -3 * 2.0 ** -9, 2.0 ** -10])
    d = np.round(rng.uniform(-0.6, 0.6, (3, 500)) * 2 ** 20) / 2 ** 20
    pos = np.concatenate([c0[:, None] + d, c0[:, None] - d], axis=1)
    n = pos.shape[1]
    m = np.full(n, 1.0 / 4096)
    gal = np.zeros(n, np.int64)
    # decoys: far and heavy (outside R_core = 1.5), another galaxy's, lost
    far = np.array([[3.0, 0.0], [0.0, -2.5], [0.0, 0.0]])
    other = c0[:, None] + np.array([[0.3], [0.0], [0.0]])
    lost = c0[:, None] + np.array([[0.0], [0.4], [0.0]])
    pos = np.concatenate([pos, far, other, lost], axis=1)
    m = np.concatenate([m, [5.0, 5.0], [3.0], [3.0]])
    gal = np.concatenate([gal, [0, 0], [1], [0]])
    flags = np.zeros(len(m), np.int64)
    flags[-1] = O.FLAG_LOST
    system = _system([_galaxy(), _galaxy(recentre=False)], mb=O.mass_bound(m))
    st = _state(pos, m, gal, [c_prev, [0.0, 0.0, 0.0]], flags=flags)
    new = O.recentre(st, system)
    assert np.array_equal(new[0], c0)
    assert np.array_equal(new[1], [0.0, 0.0, 0.0])      # not a recentring galaxy


def _plain_com(pos, m, c, r_core):
    d = pos - c[:, None]
    inside = np.sum(d * d, axis=0) < r_core * r_core
    return (m[inside][None, :] * pos[:, inside]).sum(axis=1) / m[inside].sum(), inside


def _quantisation_bound(system, gal, pos, m, c, inside):
    """|integer centre - FP64 centre of mass| <= half the offset quantum
    2^-(sD+1) + the FP32 rounding of offsets 2^-24 R_core + the mass
    truncation 2 R_core sum_i 2^(26-s) / M (weights floor(q / 2^26))."""
    s = O.fixed_shift(system.mass_bound)
    f, e = math.frexp(gal.r_core)
    sD = 24 - (e - 1 if f == 0.5 else e)
    M = m[inside].sum()
    return 2.0 ** -(sD + 1) + 2.0 ** -24 * gal.r_core + 2 * gal.r_core * inside.sum() * 2.0 ** (26 - s) / M


@pytest.mark.parametrize("split", [False, True])
def test_recentre_within_bound_of_plain_centre_of_mass(split):
    rng = np.random.default_rng(2)
    c = np.array([0.37, -1.21, 0.05])
    n = 20000
    r = 2.2 * rng.random(n) ** 0.8
    u = rng.normal(size=(3, n))
    pos = c[:, None] + 0.9 * np.array([[1.1], [0.7], [0.4]]) + r * u / np.linalg.norm(u, axis=0)
    # keep clear of the selection sphere's surface (FP32 r^2 there)
    dist = np.linalg.norm(pos - c[:, None], axis=0)
    pos = pos[:, np.abs(dist - 1.5) > 1e-4]
    if split:
        pos = pos.astype(np.float32).astype(np.float64)
    m = rng.uniform(0.5, 2.0, pos.shape[1]) / pos.shape[1]
    gal = _galaxy()
    system = _system([gal], mb=O.mass_bound(m), precision="fp32" if split else "fp64")
    new = O.recentre(_state(pos, m, np.zeros(len(m)), [c]), system)[0]
    com, inside = _plain_com(pos, m, c, gal.r_core)
    bound = _quantisation_bound(system, gal, pos, m, c, inside)
    assert np.max(np.abs(new - com)) <= bound, (new - com, bound)
    # the pin is tight against real mistakes: the centre moved by ~0.5
    assert np.linalg.norm(com - c) > 0.1 and bound < 1e-5


def test_recentre_keeps_light_particles():
    """Masses 2^20 times the weight quantum 2^(26-s): the integer weights keep
    them to one part in 2^20, so the centre follows the plain centre of mass
    of a cloud whose light part carries half the mass to within 1e-6."""
    rng = np.random.default_rng(3)
    c = np.zeros(3)
    heavy = np.array([[-0.8, 0.1], [0.2, -0.3], [0.0, 0.5]])
    n_l = 4096
    light = np.array([[0.7], [0.0], [-0.2]]) + 0.3 * rng.uniform(-1, 1, (3, n_l))
    pos = np.concatenate([heavy, light], axis=1)
    s = O.fixed_shift(1.0)
    w_q = 2.0 ** (26 - s)
    m_l = w_q * (2 ** 20 + rng.integers(0, 2 ** 19, n_l)) + 0.4 * w_q   # fractional weights truncate
    m = np.concatenate([[0.5 * m_l.sum(), 0.5 * m_l.sum()], m_l])
    m *= 1.0 / m.sum()
    gal = _galaxy()
    system = _system([gal], mb=1.0)
    new = O.recentre(_state(pos, m, np.zeros(len(m)), [c]), system)[0]
    com, inside = _plain_com(pos, m, c, gal.r_core)
    assert inside.all()
    assert np.max(np.abs(new - com)) < 1e-6 * gal.r_core


# -------------------------------------------------------------- diagnostics ---

def _box_system(q=1.0, G=1.0, h000=1.0, mb=4.0, N=32, l=0.25):
    g = O.Geometry(N, N, N, l, q * l)
    return _system([O.Galaxy(coarse=g)], r_sys=1e6, G=G, h000=h000, mb=mb), g


def test_kinetic_energy_and_angular_momentum_of_a_rigid_rotation():
    """Particles on rings in the plane z = 0 turning rigidly at omega about z,
    with dt = 0 (v(t) = v): K = omega^2 I / 2, L = (0, 0, I omega),
    I = sum m (x^2 + y^2)."""
    system, g = _box_system()
    rng = np.random.default_rng(4)
    n = 300
    R = rng.uniform(0.2, 2.5, n)
    ph = rng.uniform(0, 2 * np.pi, n)
    pos = np.stack([R * np.cos(ph), R * np.sin(ph), np.zeros(n)])
    om = 0.7
    vel = np.stack([-om * pos[1], om * pos[0], np.zeros(n)])
    m = rng.uniform(0.5, 1.5, n) / n
    d = O.diagnostics(_state(pos, m, np.zeros(n), [[0, 0, 0]], vel=vel), system, 0.0)
    I = float(np.sum(m * R * R))
    assert d["n_live"] == n
    assert d["K"] == pytest.approx(0.5 * om * om * I, rel=1e-13)
    assert np.allclose(d["L"], [0.0, 0.0, om * I], rtol=1e-13, atol=1e-16)
    assert d["E"] == pytest.approx(d["K"] + d["W"], rel=1e-14)


@pytest.mark.parametrize("q,h000", [(1.0, 1.0), (0.5, 0.7)])
def test_potential_energy_of_two_particles(q, h000):
    """Two particles at cell centres p1, p2 of one grid (Delta = 0):
    Phi(p1) = G/l (m1 h000 + m2 H(p2 - p1)), Phi(p2) likewise, so
    W = -1/2 G/l [h000 (m1^2 + m2^2) + 2 m1 m2 H],
    H = [di^2 + dj^2 + (q dk)^2]^(-1/2) (Eq. eqn:greens, flattened)."""
    G = 1.3
    system, g = _box_system(q=q, G=G, h000=h000)
    p1, p2 = np.array([13, 15, 16]), np.array([19, 11, 21])
    centre = lambda p: np.array([(p[0] - g.nx // 2) * g.l_xy, (p[1] - g.ny // 2) * g.l_xy,  # noqa: E731
                                 (p[2] - g.nz // 2) * g.l_z])
    pos = np.stack([centre(p1), centre(p2)], axis=1)
    m1, m2 = 0.75, 0.375
    d = O.diagnostics(_state(pos, [m1, m2], [0, 0], [[0, 0, 0]]), system, 0.0)
    dp = p2 - p1
    H = 1.0 / math.sqrt(dp[0] ** 2 + dp[1] ** 2 + (q * dp[2]) ** 2)
    W = -0.5 * G / g.l_xy * (h000 * (m1 * m1 + m2 * m2) + 2 * m1 * m2 * H)
    assert d["W"] == pytest.approx(W, rel=1e-12)
    assert d["K"] == 0.0


def test_diagnostics_synchronise_velocities_by_half_a_kick():
    """v(t) = v(t - dt/2) + dt/2 a(t): with v stored as -dt/2 a the
    synchronised velocities vanish (K = 0, L = 0), and with v = 0 they are
    dt/2 a (K = dt^2/8 sum m a^2)."""
    system, g = _box_system()
    rng = np.random.default_rng(5)
    n = 200
    pos = rng.uniform(-2.5, 2.5, (3, n))
    m = rng.uniform(0.5, 1.5, n) / n
    st = _state(pos, m, np.zeros(n), [[0, 0, 0]])
    flags, own = O.classify(st, system)
    rho, flags, s = O.deposit(st, system, flags, own)
    a = O.accelerations(st, system, O.solve_all(rho, system, s), flags)
    dt = 0.1
    d0 = O.diagnostics(st, system, dt)
    assert d0["K"] == pytest.approx(dt * dt / 8 * float(np.sum(m * np.sum(a * a, axis=0))), rel=1e-12)
    st.vel = -0.5 * dt * a
    d1 = O.diagnostics(st, system, dt)
    assert abs(d1["K"]) < 1e-25 and np.all(np.abs(d1["L"]) < 1e-15)
    assert d1["W"] == d0["W"]


def test_potential_and_force_at_a_particle_on_a_linear_field():
    """On Phi = a0 + bx X + by Y + bz Z of the cell centres (X = i l_xy,
    Y = j l_xy, Z = k l_z; flattened cells) the potential at a particle is the
    field at its position and the acceleration is (bx, by, bz), exactly up to
    rounding: central differences are exact on linear functions and the
    second differences vanish."""
    g = O.Geometry(16, 16, 16, 0.3, 0.075)
    a0, bx, by, bz = 2.0, -0.7, 0.4, 1.9
    k, j, i = np.meshgrid(np.arange(16), np.arange(16), np.arange(16), indexing="ij")
    phi = a0 + bx * i * g.l_xy + by * j * g.l_xy + bz * k * g.l_z
    rng = np.random.default_rng(6)
    n = 50
    ci, cj, ck = (rng.integers(2, 14, n) for _ in range(3))
    delta = rng.uniform(-0.5, 0.5, (3, n)) * np.array([[g.l_xy], [g.l_xy], [g.l_z]])
    want = a0 + bx * (ci * g.l_xy + delta[0]) + by * (cj * g.l_xy + delta[1]) + bz * (ck * g.l_z + delta[2])
    assert np.allclose(O.phi_at_particle(phi, g, ci, cj, ck, delta), want, rtol=1e-13, atol=1e-13)
    acc = O.accel_from_grid(phi, g, ci, cj, ck, delta)
    assert np.allclose(acc, np.array([[bx], [by], [bz]]) * np.ones(n), rtol=1e-12, atol=1e-12)


# --------------------------------------------------------------- lost flags ---

def test_lost_mask_against_the_definition():
    """Lost iff r >= R_sys from the system centre, or outside the usable box
    (cells 2 .. N-3, i.e. X - c in [-(N/2 - 1.5) l, (N/2 - 2.5) l)) of any
    galaxy's coarse grid.  Points are placed 1e-5 (relative) on either side
    of every such surface, far beyond FP32 rounding."""
    sc = np.array([0.3, -0.2, 0.1])
    g0 = O.Geometry(32, 32, 32, 8.0 / 28, 8.0 / 28)          # box half-widths ~4
    g1 = O.Geometry(16, 32, 16, 1.0 / 3, 0.5 / 3)            # a smaller, flattened box
    r_sys = 3.1
    system = _system([O.Galaxy(coarse=g0), O.Galaxy(coarse=g1)], r_sys=r_sys, sys_centre=tuple(sc))
    pts, want = [], []
    eps = 1e-5
    # the box edges of each grid, along each axis, on both sides
    for g in (g0, g1):
        for ax in range(3):
            n_ax = (g.nx, g.ny, g.nz)[ax]
            l_ax = (g.l_xy, g.l_xy, g.l_z)[ax]
            for edge in (-(n_ax / 2 - 1.5) * l_ax, (n_ax / 2 - 2.5) * l_ax):
                for side in (-1, 1):
                    p = np.zeros(3)
                    p[ax] = edge * (1 + side * eps)
                    pts.append(sc + p)
    # the system sphere, in random directions, on both sides
    rng = np.random.default_rng(7)
    for _ in range(40):
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        for side in (-1, 1):
            pts.append(sc + u * r_sys * (1 + side * eps))
    pts.extend(sc + rng.uniform(-3.5, 3.5, (400, 3)))
    pos = np.array(pts).T

    def inside_box(g):
        ok = np.ones(pos.shape[1], bool)
        for ax, (n_ax, l_ax) in enumerate(((g.nx, g.l_xy), (g.ny, g.l_xy), (g.nz, g.l_z))):
            x = pos[ax] - sc[ax]
            ok &= (x >= -(n_ax / 2 - 1.5) * l_ax) & (x < (n_ax / 2 - 2.5) * l_ax)
        return ok

    r = np.linalg.norm(pos - sc[:, None], axis=0)
    want = (r >= r_sys) | ~inside_box(g0) | ~inside_box(g1)
    assert 0 < want.sum() < len(want)
    assert np.array_equal(O.lost_mask(pos, system), want)
    # lost stays lost (Sec. 2.1: lost particles never return)
    st = _state(pos, np.full(pos.shape[1], 1e-3), np.zeros(pos.shape[1]), [[0, 0, 0], [0, 0, 0]],
                flags=np.full(pos.shape[1], O.FLAG_LOST))
    flags, _ = O.classify(st, system)
    assert np.all(flags & O.FLAG_LOST)


# ---------------------------------------------------- canonical cell index ---

def _exact_u(x, c, l, n):
    return (Fraction(float(x)) - Fraction(float(c))) / Fraction(float(l)) + Fraction(n // 2)


@pytest.mark.parametrize("split", [False, True])
def test_canonical_cell_index_matches_nearest_integer_away_from_faces(split):
    """a = [ (x - c)/l + N/2 ] (Eq. eqn:cell, nearest integer as floor(u+1/2)):
    the canonical FP32 evaluation (unsplit: fl32(x - c) from FP64; split:
    fl32(fl32(x - c_hi) - c_lo) for FP32 positions) gives the exact nearest
    integer except where the exact u lies within a few FP32 ulps of a cell
    face u = a + 1/2."""
    rng = np.random.default_rng(8 + split)
    n, N = 200000, 128
    l = O.cell_length(6.0, N)
    c = 3.0 + rng.uniform(-1, 1)
    x = c + rng.uniform(-(N / 2 - 2) * l, (N / 2 - 2) * l, n)
    # a quarter of the points exactly on, or next to, cell faces
    k = n // 4
    faces = c + (rng.integers(4, N - 4, k) - N // 2 + 0.5) * l
    x[:k] = faces * (1 + rng.integers(-3, 4, k) * 2.0 ** -52)
    if split:
        x = x.astype(np.float32).astype(np.float64)
    a = O.cell_index(O.offset_f32(x, c, split), l, N)
    gamma = np.longdouble(1) / np.longdouble(l)
    u = (np.longdouble(x) - np.longdouble(c)) * gamma + np.longdouble(N // 2)
    a_ex = np.floor(u + np.longdouble(0.5)).astype(np.int64)
    close = np.abs((u + np.longdouble(0.5)) - np.round(u + np.longdouble(0.5))) < np.longdouble(1e-9)
    for idx in np.nonzero(close)[0]:                       # decide the near-ties exactly
        ue = _exact_u(x[idx], c, l, N)
        a_ex[idx] = math.floor(ue + Fraction(1, 2))
    bad = np.nonzero(a != a_ex)[0]
    ulp = np.spacing(np.float32(N))                          # FP32 ulp of u ~ N/2 .. N
    for idx in bad:
        dist_face = abs(float(_exact_u(x[idx], c, l, N) + Fraction(1, 2) - round(_exact_u(x[idx], c, l, N)
                                                                                  + Fraction(1, 2))))
        assert dist_face <= 4 * ulp, (idx, dist_face, ulp)
    # points on a face split either way; uniform points almost never differ
    assert np.count_nonzero(bad >= k) <= 1e-3 * (n - k)


def test_split_and_unsplit_offsets_agree_away_from_faces():
    """For FP32 positions the two canonical offset rules differ by at most an
    FP32 rounding of the offset, so they choose different cells only within
    a few FP32 ulps of a face."""
    rng = np.random.default_rng(10)
    N = 256
    l = O.cell_length(32.0, N)
    c = rng.uniform(-5, 5)
    x = (c + rng.uniform(-(N / 2 - 2) * l, (N / 2 - 2) * l, 300000)).astype(np.float32).astype(np.float64)
    d0, d1 = O.offset_f32(x, c, False), O.offset_f32(x, c, True)
    assert np.all(np.abs(d0.astype(np.float64) - d1.astype(np.float64)) <= np.spacing(np.abs(d0)))
    a0, a1 = O.cell_index(d0, l, N), O.cell_index(d1, l, N)
    bad = np.nonzero(a0 != a1)[0]
    u = (x - c) / l + N // 2
    dist = np.abs(u + 0.5 - np.round(u + 0.5))
    assert np.all(dist[bad] <= 4 * np.spacing(np.float32(N)))
