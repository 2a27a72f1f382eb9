"""Plain FP64 CPU reference of the disc diagnostics of the paper's Sec. 6
(thickness, heat, velocity dispersions, Fourier modes).

TEST INFRASTRUCTURE ONLY, like ``oracle.pm_oracle``.

Quantities, for the selected (disc) particles that are not lost, with
positions and velocities relative to a centre c (x, y in the disc plane):
R = sqrt(dx^2 + dy^2), phi = atan2(dy, dx), v_R = (dx vx + dy vy)/R,
v_phi = (dx vy - dy vx)/R.

* Radial bins of equal particle numbers (Sec. 6: thickness figure and the
  heat definition): with n selected particles and B bins, the edges are the
  order statistics e_k = (R^2) of rank floor(k n / B) (0-based, ascending),
  k = 1..B-1, and a particle is in bin #{k : e_k <= R^2}.  Per bin: mean R,
  count, sqrt(<z^2>) (RMS of z, the thickness measure) and the mean v_phi
  (the binned circular velocity).
* E_heat = sum_i m_i |v_i - vbar_c(R_i) e_phi|^2 / 2 (Sec. 6 heat increase),
  vbar_c interpolated linearly in R between the bins' mean radii and held
  constant beyond the first and last.
* Annulus r0 - dr <= R < r0 + dr ("the region around 8 kpc"): mass-weighted
  dispersions sigma_R, sigma_phi, sigma_z and the annulus mass; sigma_z /
  sigma_R and sigma_tot^2 = sigma_R^2 + sigma_phi^2 + sigma_z^2 follow.
* Fourier modes (Sec. 6 comparison with higher resolution): in nring rings of
  equal width on [0, r_ring), A~_m = (1/S) sum_j M_j exp(-i m phi_j) with S
  the ring's area, m = 1..mmax.

Output vector (the layout of the library's pm_disc_diagnostics):
[n, E_heat, sigma_R, sigma_phi, sigma_z, annulus mass,
 (mean R, count, sqrt<z^2>, mean v_phi) per bin,
 (Re A~_m, Im A~_m) per ring and m = 1..mmax]."""
from __future__ import annotations

import numpy as np

__all__ = ["disc_diagnostics", "diag_layout"]


def diag_layout(nbins, nring, mmax):
    return 6 + 4 * nbins + 2 * nring * mmax


def disc_diagnostics(pos, vel, m, select, live, centre, nbins, nring, mmax, r_ring, r0, dr):
    sel = np.asarray(select, dtype=bool) & np.asarray(live, dtype=bool)
    dx = pos[0, sel] - centre[0]
    dy = pos[1, sel] - centre[1]
    dz = pos[2, sel] - centre[2]
    vx, vy, vz = vel[0, sel], vel[1, sel], vel[2, sel]
    mm = m[sel]
    n = int(sel.sum())
    out = np.zeros(diag_layout(nbins, nring, mmax))
    out[0] = n
    if n == 0:
        return out
    R2 = dx * dx + dy * dy
    R = np.sqrt(R2)
    with np.errstate(invalid="ignore", divide="ignore"):
        vR = np.where(R > 0, (dx * vx + dy * vy) / R, 0.0)
        vphi = np.where(R > 0, (dx * vy - dy * vx) / R, 0.0)

    # equal-number bins from order statistics of R^2
    order = np.sort(R2)
    edges = np.array([order[(k * n) // nbins] for k in range(1, nbins)])
    b = np.searchsorted(edges, R2, side="right")
    Rbar = np.zeros(nbins)
    vc = np.zeros(nbins)
    for k in range(nbins):
        inb = b == k
        cnt = int(inb.sum())
        base = 6 + 4 * k
        out[base + 1] = cnt
        if cnt:
            Rbar[k] = R[inb].mean()
            vc[k] = vphi[inb].mean()
            out[base] = Rbar[k]
            out[base + 2] = np.sqrt(np.mean(dz[inb] ** 2))
            out[base + 3] = vc[k]
    filled = out[7:6 + 4 * nbins:4] > 0
    vbar = np.interp(R, Rbar[filled], vc[filled])
    # |v - vbar e_phi|^2 = v_R^2 + (v_phi - vbar)^2 + v_z^2
    out[1] = 0.5 * np.sum(mm * (vR ** 2 + (vphi - vbar) ** 2 + vz ** 2))

    ann = (R >= r0 - dr) & (R < r0 + dr)
    M = mm[ann].sum()
    out[5] = M
    if M > 0:
        def disp(v):
            mean = np.sum(mm[ann] * v[ann]) / M
            return np.sqrt(max(np.sum(mm[ann] * v[ann] ** 2) / M - mean * mean, 0.0))
        out[2], out[3], out[4] = disp(vR), disp(vphi), disp(vz)

    phi = np.arctan2(dy, dx)
    width = r_ring / nring
    ring = np.floor(R / width).astype(np.int64)
    for r in range(nring):
        inr = (ring == r) & (R < r_ring) & (R > 0)
        S = np.pi * (((r + 1) * width) ** 2 - (r * width) ** 2)
        for mode in range(1, mmax + 1):
            A = np.sum(mm[inr] * np.exp(-1j * mode * phi[inr])) / S
            o = 6 + 4 * nbins + 2 * (r * mmax + mode - 1)
            out[o], out[o + 1] = A.real, A.imag
    return out
