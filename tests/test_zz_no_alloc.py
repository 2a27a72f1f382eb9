"""pm_potential_static, the allocation-free potential solve, against pm_solve.

Callers that cannot allocate device memory (a host application whose device
memory is pre-partitioned by its own pool, a plugin that may not allocate
after start-up) use pm_potential_static; its result must be the one the
context path gives for the same density, and an expired bounded wait inside
it must reach the caller (NaN output, PM_E_TIMEOUT from
pm_potential_static_status).  This file is collected last so that a run stopping at the
first failure has run every other test first.
"""
import ctypes as C

import numpy as np
import pytest

from paper_1210_1736_gb300 import pm, workloads as W
from tests._harness import gpu_setup, require_cuda

pytestmark = pytest.mark.gpu


def _static_call(torch, rho_dev, phi_dev, g, G, h000, shift, precision):
    rc = pm.lib().pm_potential_static(
        C.c_void_p(rho_dev.data_ptr()), C.c_void_p(phi_dev.data_ptr()),
        g.nx, g.ny, g.nz, g.l_xy, g.l_z, G, h000, shift,
        pm.PM_FP32 if precision == "fp32" else pm.PM_FP64,
        C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == pm.PM_OK, pm.lib().pm_last_error()


def _single_grid(nx, ny, nz, q, precision, n=20000, seed=0):
    rng = np.random.default_rng(seed)
    l = 0.1
    half = np.array([nx, ny, nz]) / 2 - 3
    pos = rng.uniform(-1, 1, (3, n)) * half[:, None] * np.array([[l], [l], [l * q]])
    return dict(name="grid", precision=precision, dt=0.01,
                system=dict(r_sys=1e9, sys_centre=(0.0, 0.0, 0.0), G=1.3, h000=1.0),
                galaxies=[dict(coarse=(nx, ny, nz, l * (nx - 4) / 2, q), medium=None, fine=None,
                               r_core=0.0, r_out=0.0, centre=(0.0, 0.0, 0.0), recentre=False)],
                pos=pos, vel=np.zeros_like(pos), m=rng.uniform(0.5, 2.0, n), gal=np.zeros(n, np.int32))


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_static_potential_matches_context_path(precision):
    torch = require_cuda()
    tol = 2e-6 if precision == "fp32" else 1e-12
    dt = torch.float32 if precision == "fp32" else torch.float64
    # 64^3: z transforms of length 128, whose tiles stage their H-hat rows by
    # a bulk copy into the static scratch
    cases = [_single_grid(32, 32, 32, 1.0, precision, seed=1),
             _single_grid(64, 32, 16, 0.5, precision, seed=2),
             _single_grid(64, 64, 64, 1.0, precision, seed=4),
             W.plummer32() if precision == "fp64" else _single_grid(128, 128, 32, 1.0, precision, seed=3)]
    for w in cases:
        ctx, parts = gpu_setup(w)
        ctx.deposit(parts)
        ctx.solve()
        rho = ctx.density(0, 5)
        ref = ctx.potential(0, 5).astype(np.float64)
        shift = ctx.info()["shift"]
        g = ctx.gals[0].coarse
        rho_dev = torch.from_numpy(rho).cuda()
        for call in range(2):  # two calls in a row share (and reuse) the scratch
            phi_dev = torch.full(rho.shape, float("nan"), dtype=dt, device="cuda")
            _static_call(torch, rho_dev, phi_dev, g, ctx.sys.G, ctx.sys.h000, shift, precision)
            torch.cuda.synchronize()
            got = phi_dev.cpu().numpy().astype(np.float64)
            err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
            assert err < tol, (w["name"], g.nx, g.ny, g.nz, call, err)
        assert pm.lib().pm_potential_static_status(C.c_void_p(torch.cuda.current_stream().cuda_stream)) == pm.PM_OK
        ctx.close()


def test_static_potential_rejects_oversize_grid():
    torch = require_cuda()
    rho = torch.zeros(8, dtype=torch.int64, device="cuda")
    phi = torch.zeros(8, dtype=torch.float32, device="cuda")
    rc = pm.lib().pm_potential_static(C.c_void_p(rho.data_ptr()), C.c_void_p(phi.data_ptr()),
                                      128, 128, 128, 0.1, 0.1, 1.0, 1.0, 40, pm.PM_FP32, None)
    assert rc == pm.PM_E_ARG
    assert b"static scratch holds" in pm.lib().pm_last_error()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_static_expired_wait_reaches_the_caller(precision):
    """A bounded wait that expires (one block waits 2 s on a barrier nothing
    arrives at; no fault) leaves NaN in the output and PM_E_TIMEOUT in the
    status query, which clears it; the next solve is unaffected."""
    torch = require_cuda()
    dt = torch.float32 if precision == "fp32" else torch.float64
    prec = pm.PM_FP32 if precision == "fp32" else pm.PM_FP64
    st = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    phi = torch.zeros(4096, dtype=dt, device="cuda")
    assert pm.lib().pm_potential_static_status(st) == pm.PM_OK
    assert pm.lib().pm_static_selftest_wait_expiry(C.c_void_p(phi.data_ptr()), phi.numel(), prec, st) == pm.PM_OK
    assert pm.lib().pm_potential_static_status(st) == pm.PM_E_TIMEOUT
    assert b"time limit" in pm.lib().pm_last_error()
    assert bool(torch.isnan(phi).all())
    assert pm.lib().pm_potential_static_status(st) == pm.PM_OK   # cleared by the query

    w = _single_grid(32, 32, 16, 1.0, precision, seed=5)
    ctx, parts = gpu_setup(w)
    ctx.deposit(parts)
    ctx.solve()
    rho = ctx.density(0, 5)
    ref = ctx.potential(0, 5).astype(np.float64)
    g = ctx.gals[0].coarse
    out = torch.full(rho.shape, float("nan"), dtype=dt, device="cuda")
    _static_call(torch, torch.from_numpy(rho).cuda(), out, g, ctx.sys.G, ctx.sys.h000, ctx.info()["shift"], precision)
    assert pm.lib().pm_potential_static_status(st) == pm.PM_OK
    got = out.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) < (2e-6 if precision == "fp32" else 1e-12)
    ctx.close()
