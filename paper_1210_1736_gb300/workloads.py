"""Named synthetic workloads: grid layout (cells, radii, flattening) plus seeded
particles.  Pure data and sampling; no particle-mesh arithmetic.

A geometry is given as ``(nx, ny, nz, R, q)``: nx*ny*nz active cells whose
usable part spans the diameter 2R in x and y, with cells flattened by q in z.
Each side (library and oracle) derives the cell lengths itself.

Workloads
---------
plummer32   65,536-particle Plummer sphere (M = a = G = 1) truncated at
            r = 3.375 a, single 32^3 grid of cell length 0.25 (grid side 8a),
            FP64, dt = 0.01, 10 steps.
galaxy_1m   disc (400k) + Hernquist bulge (100k) + truncated NFW halo (500k);
            grids: coarse 128^3 (R_sys = 32), medium 128^3 flattened q = 1/4
            (R_out = 6), fine 128x128x32 (R_core = 1.5); dt = 0.01.
galaxy_small  the same model scaled to 48k particles on 32^3 / 32^3 (q = 0.8,
            the smallest admissible at N = 32) / 32x32x8 grids (fast enough for
            the oracle inside a test).
merger_4m   galaxy scaled to 4M particles plus a 100k Plummer satellite; six
            geometries (galaxy 128^3, 128^3, 256x256x32; satellite 64^3 x 3).
large_16m   16M-particle galaxy on 256^3 / 256^3 / 256x256x64 grids plus two
            250k Plummer satellites with 128^3 grids.
merger_small, big_box, galaxy_256: test-size and largest-grid cases.
"""
from __future__ import annotations

import numpy as np

from . import synth

GALAXY_RADII = dict(r_core=1.5, r_out=6.0, r_sys=32.0)


def _galaxy_spec(n_c, n_m, n_f, q_m=0.25, centre=(0.0, 0.0, 0.0)):
    R = GALAXY_RADII
    return dict(
        coarse=(n_c, n_c, n_c, R["r_sys"], 1.0),
        medium=(n_m, n_m, n_m, R["r_out"], q_m),
        fine=(n_f[0], n_f[1], n_f[2], R["r_core"], 1.0),
        r_core=R["r_core"], r_out=R["r_out"], centre=centre, recentre=True)


def plummer32(seed_id=0):
    rng = synth.rng_for(seed_id, 0)
    pos, vel, m = synth.plummer(65536, rng, M=1.0, a=1.0, r_trunc=3.375)
    n = pos.shape[1]
    return dict(
        name="plummer32", precision="fp64", dt=0.01, steps=10,
        system=dict(r_sys=3.5, sys_centre=(0.0, 0.0, 0.0), G=1.0, h000=1.0),
        galaxies=[dict(coarse=(32, 32, 32, 3.5, 1.0), medium=None, fine=None,
                       r_core=0.0, r_out=0.0, centre=(0.0, 0.0, 0.0), recentre=False)],
        pos=pos, vel=vel, m=m, gal=np.zeros(n, dtype=np.int32))


COMP_DISC, COMP_BULGE, COMP_HALO, COMP_SATELLITE = 0, 1, 2, 3


def _components(nd, nb, nh):
    return np.concatenate([np.full(nd, COMP_DISC, np.int8), np.full(nb, COMP_BULGE, np.int8),
                           np.full(nh, COMP_HALO, np.int8)])


def _galaxy_particles(n_total, seed_id):
    """Disc, bulge and halo particles (40/10/50 per cent) and their component
    labels, unscrambled."""
    nd, nb = int(round(0.4 * n_total)), int(round(0.1 * n_total))
    nh = n_total - nd - nb
    pos, vel, m = synth.galaxy(nd, nb, nh, synth.rng_for(seed_id, 1),
                               synth.rng_for(seed_id, 2), synth.rng_for(seed_id, 3))
    return pos, vel, m, _components(nd, nb, nh)


def galaxy(n_total=1_000_000, n_c=128, n_m=128, n_f=(128, 128, 32), seed_id=1,
           precision="fp32", name=None, q_m=0.25):
    pos, vel, m, comp = _galaxy_particles(n_total, seed_id)
    pos, vel, m, comp = synth.scramble(synth.rng_for(seed_id, 9), pos, vel, m, comp)
    n = pos.shape[1]
    return dict(
        name=name or f"galaxy_{n_total}", precision=precision, dt=0.01, steps=100,
        system=dict(r_sys=GALAXY_RADII["r_sys"], sys_centre=(0.0, 0.0, 0.0), G=1.0, h000=1.0),
        galaxies=[_galaxy_spec(n_c, n_m, n_f, q_m=q_m)],
        pos=pos, vel=vel, m=m, gal=np.zeros(n, dtype=np.int32), comp=comp)


def galaxy_1m(precision="fp32"):
    return galaxy(1_000_000, 128, 128, (128, 128, 32), seed_id=1, precision=precision,
                  name="galaxy_1m")


def galaxy_small(precision="fp32", n_total=48_000, seed_id=11):
    # q_crit(N=32) = 4/28 * 32/6 = 0.76 for these radii: the medium grid is
    # flattened by 0.8 here (1/4 needs N >= 128)
    return galaxy(n_total, 32, 32, (32, 32, 8), seed_id=seed_id, precision=precision,
                  name="galaxy_small", q_m=0.8)


def _satellite(pos_g, m_g, n_sat, rng, M, a, R_A, phase, inc_deg, ns, e=0.5):
    """Plummer satellite (truncated at 10a) at apocentre R_A in the disc plane
    at azimuth `phase`, orbit eccentricity e and inclination inc_deg; the
    apocentre speed is the point-mass value sqrt(G M(<R_A) (1 - e) / R_A)
    (the construction of Sec. 6.1 of the paper)."""
    ps, vs, ms = synth.plummer(n_sat, rng, M=M, a=a, r_trunc=10 * a)
    inc = np.deg2rad(inc_deg)
    m_enc = float(m_g[np.linalg.norm(pos_g, axis=0) < R_A].sum())
    v_apo = np.sqrt(m_enc * (1 - e) / R_A)
    c, s = np.cos(phase), np.sin(phase)
    centre = (R_A * c, R_A * s, 0.0)
    ps = ps + np.array(centre)[:, None]
    vs = vs + np.array([[-s * v_apo * np.cos(inc)], [c * v_apo * np.cos(inc)], [v_apo * np.sin(inc)]])
    spec = dict(coarse=(ns, ns, ns, GALAXY_RADII["r_sys"], 1.0),
                medium=(ns, ns, ns, 10 * a, 1.0), fine=(ns, ns, ns, 2.5 * a, 1.0),
                r_core=2.5 * a, r_out=10 * a, centre=centre, recentre=True)
    return ps, vs, ms, spec


def _with_satellites(pos, vel, m, comp, gal_spec, sats, seed_id, precision, name, steps):
    allpos, allvel, allm, allc = [pos], [vel], [m], [comp]
    gal = [np.zeros(pos.shape[1], np.int32)]
    specs = [gal_spec]
    for k, (ps, vs, ms, spec) in enumerate(sats):
        allpos.append(ps); allvel.append(vs); allm.append(ms)
        allc.append(np.full(ps.shape[1], COMP_SATELLITE, np.int8))
        gal.append(np.full(ps.shape[1], k + 1, np.int32))
        specs.append(spec)
    allpos, allvel, allm, gal, allc = synth.scramble(
        synth.rng_for(seed_id, 9), np.concatenate(allpos, axis=1), np.concatenate(allvel, axis=1),
        np.concatenate(allm), np.concatenate(gal), np.concatenate(allc))
    return dict(
        name=name, precision=precision, dt=0.01, steps=steps,
        system=dict(r_sys=GALAXY_RADII["r_sys"], sys_centre=(0.0, 0.0, 0.0), G=1.0, h000=1.0),
        galaxies=specs, pos=allpos, vel=allvel, m=allm, gal=gal, comp=allc)


def merger(n_gal=4_000_000, n_sat=100_000, grids=((128,), (128,), (256, 256, 32), (64,)),
           seed_id=2, precision="fp32", name="merger_4m", q_m=0.25, sat_m=0.1, steps=500, r_apo=8.0):
    """Galaxy plus a Plummer satellite (M = 0.1 M_disc, a = 0.05) at apocentre
    8 R_d on an orbit of eccentricity 0.5, inclined 30 degrees."""
    pos, vel, m, comp = _galaxy_particles(n_gal, seed_id)
    sat = _satellite(pos, m, n_sat, synth.rng_for(seed_id, 4), sat_m, 0.05, r_apo, 0.0, 30.0, grids[3][0])
    return _with_satellites(pos, vel, m, comp, _galaxy_spec(grids[0][0], grids[1][0], grids[2], q_m=q_m), [sat],
                            seed_id, precision, name, steps)


def merger_4m(precision="fp32"):
    return merger(precision=precision)


def large_16m(precision="fp32", seed_id=4):
    """16M-particle galaxy (6M disc, 2M bulge, 8M halo, the model of
    galaxy_1m) on 256^3, 256^3 (q = 1/4) and 256x256x64 grids, plus two
    250k-particle Plummer satellites (M = 0.1, a = 0.05) with 128^3 grids."""
    pos, vel, m = synth.galaxy(6_000_000, 2_000_000, 8_000_000, synth.rng_for(seed_id, 1),
                               synth.rng_for(seed_id, 2), synth.rng_for(seed_id, 3))
    comp = _components(6_000_000, 2_000_000, 8_000_000)
    sats = [_satellite(pos, m, 250_000, synth.rng_for(seed_id, 4), 0.1, 0.05, 8.0, 0.0, 30.0, 128),
            _satellite(pos, m, 250_000, synth.rng_for(seed_id, 5), 0.1, 0.05, 6.0, 2.0, -45.0, 128)]
    return _with_satellites(pos, vel, m, comp, _galaxy_spec(256, 256, (256, 256, 64)), sats, seed_id, precision,
                            "large_16m", 1000)


def adjoint_1m(precision="fp32"):
    """Differentiable-run workload: the 1M-particle galaxy (grids 128^3,
    128^3 q = 1/4, 128x128x32) plus a 20k-particle Plummer satellite
    (M = 0.05, a = 0.05, 64^3 grids) at apocentre 8 R_d; 200 steps."""
    return merger(n_gal=1_000_000, n_sat=20_000, grids=((128,), (128,), (128, 128, 32), (64,)), seed_id=3,
                  precision=precision, name="adjoint_1m", sat_m=0.05, steps=200)


def merger_small(precision="fp32", seed_id=12, r_apo=8.0):
    """Two galaxies at test size: the small galaxy (24k particles) and a 4k
    Plummer satellite with its own 16^3 grids, on an inclined orbit with
    apocentre r_apo."""
    return merger(n_gal=24_000, n_sat=4_000, grids=((32,), (32,), (32, 32, 8), (16,)), seed_id=seed_id,
                  precision=precision, name="merger_small", q_m=0.8, r_apo=r_apo)


def big_box(n=1_000_000, N=256, precision="fp32", seed_id=13):
    """Plummer sphere (M = 1, a = 1, r <= 10) on one N^3 grid of side 24:
    the largest transform length (2N = 512) on every axis."""
    rng = synth.rng_for(seed_id, 0)
    pos, vel, m = synth.plummer(n, rng, M=1.0, a=1.0, r_trunc=10.0)
    R = 12.0 * (N - 4) / N
    return dict(
        name=f"box{N}", precision=precision, dt=0.01, steps=10,
        system=dict(r_sys=11.0, sys_centre=(0.0, 0.0, 0.0), G=1.0, h000=1.0),
        galaxies=[dict(coarse=(N, N, N, R, 1.0), medium=None, fine=None,
                       r_core=0.0, r_out=0.0, centre=(0.0, 0.0, 0.0), recentre=False)],
        pos=pos, vel=vel, m=m, gal=np.zeros(pos.shape[1], dtype=np.int32))


def galaxy_256(n_total=2_000_000, precision="fp32", seed_id=14):
    """The disc-bulge-halo galaxy on the large grids: coarse and medium 256^3,
    fine 256x256x64 (all padded to 512 along x and y)."""
    return galaxy(n_total, 256, 256, (256, 256, 64), seed_id=seed_id, precision=precision,
                  name="galaxy_256", q_m=0.25)


def mass_bound(m):
    """Upper bound on sum |m| handed to both sides (fixes the fixed-point scale);
    1 for an empty set."""
    s = float(np.abs(np.asarray(m, dtype=np.float64)).sum())
    return s if s > 0 else 1.0
