"""Seeded synthetic initial conditions (positions, velocities, masses).

This module holds only sampling of the galaxy components named in the
workloads (Plummer sphere, exponential sech^2 disc, Hernquist bulge, truncated
NFW halo) from a PCG64 stream; it contains none of the particle-mesh step's
arithmetic and is shared by the tests, the benchmark and the smoke check.
Units: G = 1.  All arrays are float64; callers cast to the path precision.

Seeds follow one rule: seed = 20121003 + 1000 * workload + component.
"""
from __future__ import annotations

import numpy as np

BASE_SEED = 20121003


def rng_for(workload: int, component: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(BASE_SEED + 1000 * workload + component))


def _isotropic(rng, r):
    cth = rng.uniform(-1.0, 1.0, len(r))
    sth = np.sqrt(1.0 - cth * cth)
    ph = rng.uniform(0.0, 2.0 * np.pi, len(r))
    return np.stack([r * sth * np.cos(ph), r * sth * np.sin(ph), r * cth])


def plummer(n, rng, M=1.0, a=1.0, r_trunc=None):
    """Plummer sphere rho = 3M/(4 pi a^3) (1 + r^2/a^2)^(-5/2) (paper Sec. 3.2).

    Radii by the inverse of M(r)/M = r^3/(r^2+a^2)^(3/2), optionally truncated
    at r_trunc (the sample then carries the enclosed mass M(r_trunc)).
    Isotropic velocities from the Plummer distribution function by the
    Aarseth-Henon-Wielen (1974) rejection step.  Returns pos, vel, mass (per
    particle) with the sample's total mass."""
    frac = 1.0
    if r_trunc is not None:
        x = r_trunc / a
        frac = x**3 / (1.0 + x * x) ** 1.5
    u = rng.uniform(0.0, frac, n)
    u = np.clip(u, 1e-12, None)
    r = a / np.sqrt(u ** (-2.0 / 3.0) - 1.0)
    pos = _isotropic(rng, r)
    # velocity modulus q * v_esc with g(q) ~ q^2 (1 - q^2)^(7/2)
    q = np.empty(n)
    todo = np.arange(n)
    while len(todo):
        qq = rng.uniform(0.0, 1.0, len(todo))
        yy = rng.uniform(0.0, 0.1, len(todo))
        ok = yy < qq * qq * (1.0 - qq * qq) ** 3.5
        q[todo[ok]] = qq[ok]
        todo = todo[~ok]
    vesc = np.sqrt(2.0 * M) * (r * r + a * a) ** -0.25
    vel = _isotropic(rng, q * vesc)
    m = np.full(n, M * frac / n)
    return pos, vel, m


def _inv_cdf(cdf_r, cdf_v, u):
    return np.interp(u, cdf_v, cdf_r)


def _enclosed_total(r, comps):
    return sum(c(r) for c in comps)


def galaxy(n_disc, n_bulge, n_halo, rng_disc, rng_bulge, rng_halo,
           M_d=1.0, R_d=1.0, z0=0.1, R_cut=5.0, Q=1.5,
           M_b=0.25, a_b=0.2, M_h=10.0, r_s=3.0, r_max=30.0):
    """Disc-bulge-halo model (paper Sec. 3.1 components, workload parameters).

    Disc: Sigma ~ exp(-R/R_d) for R <= R_cut, sech^2(z/z0) vertically
    (|z| <= 10 z0); rotation from the spherical enclosed mass with an
    asymmetric-drift correction, sigma_R from the Toomre Q, sigma_z^2 =
    pi G Sigma z0.  Bulge: Hernquist (a_b) cut at 14 a_b.  Halo: NFW (r_s)
    truncated at r_max.  Bulge and halo velocities: isotropic Jeans equation in
    the spherical total mass.  Returns pos, vel, m (float64)."""
    rr = np.concatenate([[0.0], np.geomspace(1e-5, 2 * r_max, 8000)])

    # --- enclosed masses (spherical) ---
    def m_disc(r):
        x = np.minimum(r, R_cut) / R_d
        return M_d * (1 - (1 + x) * np.exp(-x)) / (1 - (1 + R_cut / R_d) * np.exp(-R_cut / R_d))

    b_cut = 14.0 * a_b

    def m_bulge(r):
        rc = np.minimum(r, b_cut)
        return M_b * (rc / (rc + a_b)) ** 2 / (b_cut / (b_cut + a_b)) ** 2

    def mu(x):
        return np.log1p(x) - x / (1 + x)

    def m_halo(r):
        return M_h * mu(np.minimum(r, r_max) / r_s) / mu(r_max / r_s)

    comps = [m_disc, m_bulge, m_halo]
    Mtot = _enclosed_total(rr, comps)

    # --- disc ---
    R_tab = np.linspace(0, R_cut, 20001)
    F = m_disc(R_tab) / M_d
    R = _inv_cdf(R_tab, F, rng_disc.uniform(0, 1, n_disc))
    t10 = np.tanh(10.0)
    z = z0 * np.arctanh(rng_disc.uniform(-t10, t10, n_disc))
    ph = rng_disc.uniform(0, 2 * np.pi, n_disc)
    Rs = np.maximum(R, 1e-3)
    vc2 = np.interp(Rs, rr, Mtot) / Rs
    Om2 = vc2 / Rs**2
    dR = 1e-3
    vc2p = np.interp(Rs + dR, rr, Mtot) / (Rs + dR)
    Om2p = vc2p / (Rs + dR) ** 2
    kap2 = np.maximum(Rs * (Om2p - Om2) / dR + 4 * Om2, 1e-8)
    Sigma = M_d / (2 * np.pi * R_d**2) * np.exp(-R / R_d)
    sR = np.minimum(Q * 3.36 * Sigma / np.sqrt(kap2), 0.5 * np.sqrt(vc2))
    sz = np.sqrt(np.pi * Sigma * z0)
    sph = sR * np.sqrt(np.clip(kap2 / (4 * Om2), 0.0, 1.0))
    vphi_mean = np.sqrt(np.maximum(vc2 + sR**2 * (1 - kap2 / (4 * Om2) - 2 * R / R_d), 0.0))
    vR = rng_disc.normal(0, 1, n_disc) * sR
    vph = vphi_mean + rng_disc.normal(0, 1, n_disc) * sph
    vz = rng_disc.normal(0, 1, n_disc) * sz
    c, s = np.cos(ph), np.sin(ph)
    pos_d = np.stack([R * c, R * s, z])
    vel_d = np.stack([vR * c - vph * s, vR * s + vph * c, vz])

    # --- Jeans dispersion for a spherical component ---
    def jeans(rho_fn, r_out):
        grid = np.geomspace(1e-4, r_out, 4000)
        integrand = rho_fn(grid) * np.interp(grid, rr, Mtot) / grid**2
        # cumulative integral from r to r_out
        seg = 0.5 * (integrand[1:] + integrand[:-1]) * np.diff(grid)
        tail = np.concatenate([np.cumsum(seg[::-1])[::-1], [0.0]])
        sig2 = tail / np.maximum(rho_fn(grid), 1e-300)
        return grid, np.maximum(sig2, 0.0)

    # --- bulge (Hernquist, cut at 14 a) ---
    ub = rng_bulge.uniform(0, (b_cut / (b_cut + a_b)) ** 2, n_bulge)
    su = np.sqrt(ub)
    rb = a_b * su / (1 - su)
    pos_b = _isotropic(rng_bulge, rb)
    g_b, s2_b = jeans(lambda r: 1.0 / (r * (r + a_b) ** 3), b_cut)
    sb = np.sqrt(np.interp(rb, g_b, s2_b))
    vel_b = rng_bulge.normal(0, 1, (3, n_bulge)) * sb

    # --- halo (NFW truncated at r_max) ---
    r_tab = np.geomspace(1e-4, r_max, 20001)
    Fh = mu(r_tab / r_s) / mu(r_max / r_s)
    rh = _inv_cdf(r_tab, Fh, rng_halo.uniform(Fh[0], 1.0, n_halo))
    pos_h = _isotropic(rng_halo, rh)
    g_h, s2_h = jeans(lambda r: 1.0 / ((r / r_s) * (1 + r / r_s) ** 2), r_max)
    sh = np.sqrt(np.interp(rh, g_h, s2_h))
    vel_h = rng_halo.normal(0, 1, (3, n_halo)) * sh

    pos = np.concatenate([pos_d, pos_b, pos_h], axis=1)
    vel = np.concatenate([vel_d, vel_b, vel_h], axis=1)
    m = np.concatenate([np.full(n_disc, M_d / max(n_disc, 1)),
                        np.full(n_bulge, M_b / max(n_bulge, 1)),
                        np.full(n_halo, M_h / max(n_halo, 1))])
    return pos, vel, m


def scramble(rng, *arrays):
    """One random permutation applied to every array's last axis (mixes the
    components so no launch sees them sorted by kind)."""
    n = arrays[0].shape[-1]
    p = rng.permutation(n)
    return [a[..., p] for a in arrays]
