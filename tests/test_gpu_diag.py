"""Disc diagnostics (Sec. 6 quantities) on the GPU against the FP64 oracle:
the bin populations are exact (edges are exact order statistics of R^2),
the sums agree to FP64 summation-order rounding."""
import numpy as np
import pytest

from oracle import pm_diag as D
from paper_1210_1736_gb300 import workloads as W
from tests._harness import gpu_setup

pytestmark = pytest.mark.gpu


def _compare(w, steps, nbins=20, nring=10, mmax=4, r_ring=5.0, r0=3.2, dr=0.4, use_select=True):
    import torch
    ctx, parts = gpu_setup(w)
    if steps:
        ctx.deposit(parts)
        ctx.solve()
        ctx.kick(parts, -0.5 * w["dt"])
        ctx.step(parts, w["dt"], steps)
    ctx.deposit(parts)          # lost flags at the current positions
    torch.cuda.synchronize()
    disc = np.asarray(w["comp"]) == W.COMP_DISC
    sel = torch.tensor(disc, device="cuda") if use_select else None
    got = ctx.disc_diagnostics(parts, sel, gal=0, nbins=nbins, nring=nring, mmax=mmax, r_ring=r_ring, r0=r0,
                               dr=dr)["raw"]
    pos, vel, flags = parts.host()
    m = parts.m.cpu().numpy().astype(np.float64)
    select = disc if use_select else (np.asarray(w["gal"]) == 0)
    ref = D.disc_diagnostics(pos, vel, m, select, (flags & 1) == 0, ctx.centres()[0], nbins, nring, mmax, r_ring,
                             r0, dr)
    counts = slice(7, 6 + 4 * nbins, 4)
    assert np.array_equal(got[counts], ref[counts])
    assert got[0] == ref[0]
    scale = np.abs(ref) + 1e-300
    rel = np.abs(got - ref) / scale
    rel[np.abs(ref) < 1e-12 * np.max(np.abs(ref[6 + 4 * nbins:]), initial=1e-300)] = 0   # empty-ish modes
    print(f"diagnostics: n {int(ref[0])}, E_heat {ref[1]:.6e}, sigma_z/sigma_R {ref[4] / ref[2]:.4f}, "
          f"worst rel err {rel.max():.3e}")
    assert rel.max() < 1e-9
    return ref


def test_disc_diagnostics_galaxy_1m_fp32():
    """The 1M-particle galaxy's 400k disc particles at t = 0 and after 10
    steps (FP32 positions, FP64 sums)."""
    ref = _compare(W.galaxy_1m(), 0)
    assert 0.3 < ref[4] / ref[2] < 1.0
    _compare(W.galaxy_1m(), 10)


def test_disc_diagnostics_fp64_and_galaxy_selection():
    """FP64 context, every particle of galaxy 0 (no selection array), odd bin
    and ring counts, after 5 steps."""
    _compare(W.galaxy_small(precision="fp64"), 5, nbins=7, nring=3, mmax=5, r_ring=4.0, r0=2.0, dr=0.5,
             use_select=False)
