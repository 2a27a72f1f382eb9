"""The fine grid's two difference-field convolutions (the spectral factors
H-hat (D_x + i D_y) and H-hat (D_z + i) of Eq. eqn:diff's forward
differences) from one forward z transform, through both H-hat sources of
that path (the tile's staged rows at z lengths 128 and 256, the thread-major
table at 64 and below): nested galaxies with fine grids of 32 x 32 x 64,
16 x 16 x 128, 32 x 32 x 32 and 16 x 16 x 16 cells against the oracle, FP64
and FP32."""
import numpy as np
import pytest

import oracle as O
from paper_1210_1736_gb300 import workloads as W
from tests._harness import gpu_setup, oracle_fields, oracle_setup, rel_force_errors
from tests.test_gpu_parity import _compare_density_and_flags, _gpu_fields, _phi_rel

pytestmark = pytest.mark.gpu


def _galaxy_with_fine(fine, precision):
    w = W.galaxy(24_000, 32, 32, (16, 16, 8), seed_id=21, precision=precision, name="galaxy_fine", q_m=0.8)
    g = dict(w["galaxies"][0])
    g["fine"] = (fine[0], fine[1], fine[2], g["r_core"], fine[3])
    w["galaxies"] = [g]
    return w


@pytest.mark.parametrize("fine", [(32, 32, 64, 0.25), (16, 16, 128, 0.1), (32, 32, 32, 0.5), (16, 16, 16, 1.0)])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_fused_difference_fields(precision, fine):
    w = _galaxy_with_fine(fine, precision)
    ctx, parts = gpu_setup(w)
    system, state = oracle_setup(w)
    rho, phi, flags, own, s = oracle_fields(system, state)
    assert np.count_nonzero(rho[0][1]) > 500   # grid 1 holds mass
    a_gpu = _gpu_fields(ctx, parts)
    _compare_density_and_flags(ctx, parts, system, rho, flags)
    a_ref = O.accelerations(state, system, phi, flags)
    rms, mx = rel_force_errors(a_gpu, a_ref, (flags & 1) == 0)
    prel = _phi_rel(ctx, system, phi)
    print(f"fine {fine} {precision}: phi {prel:.2e} force rms {rms:.2e} max {mx:.2e}")
    if precision == "fp64":
        assert prel < 1e-12
        assert mx < 1e-11, (rms, mx)
    else:
        assert prel < 2e-6
        assert rms < 2e-5 and mx < 1e-4, (rms, mx)
    ctx.close()
