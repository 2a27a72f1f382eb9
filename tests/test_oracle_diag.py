"""Pins of the oracle's disc diagnostics (Sec. 6 quantities), CPU only:
closed forms of constructed particle sets and the sech^2 thickness."""
import numpy as np

from oracle import pm_diag as D

RNG = np.random.default_rng(61)


def _run(pos, vel, m, nbins=5, nring=3, mmax=3, r_ring=3.0, r0=1.0, dr=0.5, select=None, centre=(0, 0, 0)):
    n = pos.shape[1]
    select = np.ones(n, bool) if select is None else select
    return D.disc_diagnostics(pos, vel, m, select, np.ones(n, bool), np.array(centre, float), nbins, nring, mmax,
                              r_ring, r0, dr)


def test_equal_number_bins():
    n = 1003
    R = RNG.uniform(0.1, 4, n)
    ph = RNG.uniform(0, 2 * np.pi, n)
    pos = np.stack([R * np.cos(ph), R * np.sin(ph), np.zeros(n)])
    out = _run(pos, np.zeros((3, n)), np.ones(n), nbins=7)
    counts = out[7:6 + 4 * 7:4]
    assert counts.sum() == n
    assert set(counts.astype(int)) <= {n // 7, n // 7 + 1}
    Rbar = out[6:6 + 4 * 7:4]
    assert np.all(np.diff(Rbar) > 0)


def test_sech2_thickness():
    """z = z0 atanh(2u - 1) has the sech^2(z/z0) profile of the disc, whose
    RMS is z0 pi / sqrt(12)."""
    n, z0 = 200_000, 0.1
    R = RNG.uniform(0.5, 4, n)
    ph = RNG.uniform(0, 2 * np.pi, n)
    z = z0 * np.arctanh(2 * RNG.uniform(0, 1, n) - 1)
    pos = np.stack([R * np.cos(ph), R * np.sin(ph), z])
    out = _run(pos, np.zeros((3, n)), np.ones(n), nbins=4)
    rms = out[8:6 + 16:4]
    assert np.all(np.abs(rms / (z0 * np.pi / np.sqrt(12)) - 1) < 0.02)


def test_heat_of_flat_rotation_is_random_motion_only():
    """v = v0 e_phi + (v_R, v_z) noise with v0 the same at every radius: the
    binned circular velocity is v0 + mean noise, so E_heat equals the kinetic
    energy about that mean exactly (any interpolation of a constant)."""
    n = 5000
    R = RNG.uniform(0.2, 4, n)
    ph = RNG.uniform(0, 2 * np.pi, n)
    pos = np.stack([R * np.cos(ph), R * np.sin(ph), RNG.normal(0, 0.1, n)])
    v0 = 0.7
    vR = RNG.normal(0, 0.05, n)
    vz = RNG.normal(0, 0.03, n)
    vel = np.stack([vR * np.cos(ph) - v0 * np.sin(ph), vR * np.sin(ph) + v0 * np.cos(ph), vz])
    m = RNG.uniform(0.5, 1.5, n)
    out = _run(pos, vel, m, nbins=1)
    assert abs(out[6 + 3] - v0) < 1e-12
    exp = 0.5 * np.sum(m * (vR ** 2 + vz ** 2))
    assert abs(out[1] - exp) < 1e-12 * exp


def test_fourier_modes_of_a_weighted_ring():
    """J particles equally spaced in phi at one radius with masses
    1 + eps cos(2 phi): A~_2 = eps J / (2 S), every other mode 0."""
    J, eps, Rr = 64, 0.3, 1.2
    ph = 2 * np.pi * np.arange(J) / J
    pos = np.stack([Rr * np.cos(ph), Rr * np.sin(ph), np.zeros(J)])
    m = 1 + eps * np.cos(2 * ph)
    out = _run(pos, np.zeros((3, J)), m, nring=3, mmax=3, r_ring=3.0)
    S = np.pi * (2.0 ** 2 - 1.0 ** 2)        # ring 1 spans [1, 2)
    A = out[6 + 4 * 5:].reshape(3, 3, 2)
    assert abs(A[1, 1, 0] - eps * J / (2 * S)) < 1e-12
    rest = A.copy()
    rest[1, 1, 0] = 0
    assert np.max(np.abs(rest)) < 1e-12


def test_annulus_dispersions_of_symmetric_velocities():
    """Pairs (+a, -a) in v_R, (+b, -b) in v_z and v0 +- c in v_phi give
    sigma_R = a, sigma_z = b, sigma_phi = c exactly; particles outside the
    annulus do not count."""
    n = 400
    R = np.concatenate([RNG.uniform(0.6, 1.4, n), RNG.uniform(2.0, 3.0, n)])
    ph = RNG.uniform(0, 2 * np.pi, 2 * n)
    a, b, c, v0 = 0.11, 0.05, 0.07, 0.6
    s = np.where(np.arange(2 * n) % 2 == 0, 1.0, -1.0)
    vR, vz, vphi = s * a, s * b, v0 + s * c
    vel = np.stack([vR * np.cos(ph) - vphi * np.sin(ph), vR * np.sin(ph) + vphi * np.cos(ph), vz])
    pos = np.stack([R * np.cos(ph), R * np.sin(ph), np.zeros(2 * n)])
    out = _run(pos, vel, np.ones(2 * n), r0=1.0, dr=0.45)
    assert out[5] == n
    assert np.allclose(out[2:5], [a, c, b], rtol=1e-12)


def test_selection_and_centre():
    n = 300
    R = RNG.uniform(0.2, 2, n)
    ph = RNG.uniform(0, 2 * np.pi, n)
    c = np.array([5.0, -2.0, 0.3])
    pos = np.stack([R * np.cos(ph), R * np.sin(ph), RNG.normal(0, 0.1, n)]) + c[:, None]
    sel = np.arange(n) % 3 != 0
    out = _run(pos, np.zeros((3, n)), np.ones(n), select=sel, centre=c)
    ref = _run(pos[:, sel] - c[:, None], np.zeros((3, sel.sum())), np.ones(sel.sum()))
    assert out[0] == sel.sum()
    assert np.allclose(out, ref, rtol=1e-12, atol=1e-14)
