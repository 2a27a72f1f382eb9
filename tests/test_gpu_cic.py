"""CIC variant and its adjoint on the GPU: forward parity with the FP64
oracle, the vector-Jacobian product against the oracle's, and gradients of
whole trajectories (autograd.Function with checkpointed recomputation)
against central finite differences of the FP64 instantiation."""
import numpy as np
import pytest

import oracle as O
from oracle import pm_cic as OC
from paper_1210_1736_gb300 import pm, workloads as W
from tests._harness import gpu_setup, oracle_setup, rel_force_errors

pytestmark = pytest.mark.gpu


def _oracle_cic(system, state):
    flags, own = O.classify(state, system)
    rho, flags = OC.cic_deposit(state, system, flags, own)
    phi = OC.cic_solve(rho, system)
    return rho, phi, flags, own, OC.cic_accelerations(state, system, phi, flags)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_cic_forward_matches_oracle(precision):
    """Two galaxies, all mass sets: CIC densities (fixed point, each cell share
    rounded) and accelerations against the FP64 oracle."""
    w = W.merger_small(precision=precision)
    ctx, parts = gpu_setup(w)
    system, state = oracle_setup(w)
    rho, phi, flags, own, a_ref = _oracle_cic(system, state)
    ctx.cic_deposit(parts)
    ctx.solve()
    acc = ctx.cic_force(parts)
    a_gpu = np.stack([a.cpu().numpy().astype(np.float64) for a in acc])
    _, _, gflags = parts.host()
    assert np.array_equal(gflags & 1, flags & 1)
    s = ctx.info()["shift"]
    rel = 1e-10 if precision == "fp64" else 1e-5
    for g, per in enumerate(rho):
        for k, ref in per.items():
            got = np.ldexp(ctx.density(g, k).astype(np.float64), -s)
            assert np.max(np.abs(got - ref)) <= rel * max(np.max(np.abs(ref)), 1e-30), (g, k)
    rms, mx = rel_force_errors(a_gpu, a_ref, (flags & 1) == 0)
    if precision == "fp64":
        assert mx < 1e-9
    else:
        assert rms < 2e-5 and mx < 1e-4


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_cic_vjp_matches_oracle(precision):
    """u^T da/dx and u^T da/dm for a random cotangent u, against the oracle's
    adjoint (itself pinned by finite differences on the CPU)."""
    import torch
    w = W.merger_small(precision=precision)
    ctx, parts = gpu_setup(w)
    system, state = oracle_setup(w)
    rho, phi, flags, own, _ = _oracle_cic(system, state)
    dt = np.float32 if precision == "fp32" else np.float64
    u = np.random.default_rng(3).normal(size=state.pos.shape).astype(dt)
    gx_ref, gm_ref = OC.cic_vjp(state, system, phi, flags, own, u.astype(np.float64))
    ctx.cic_deposit(parts)
    ctx.solve()
    ut = torch.tensor(u, device="cuda")
    gx = torch.zeros_like(ut)
    gm = torch.zeros(ut.shape[1], dtype=ut.dtype, device="cuda")
    ctx.cic_vjp(parts, ut, gx, gm)
    ex, em = _rel(gx.cpu().numpy().astype(np.float64), gx_ref), _rel(gm.cpu().numpy().astype(np.float64), gm_ref)
    print(f"vjp {precision}: positions {ex:.3e}, masses {em:.3e}")
    tol = 1e-9 if precision == "fp64" else 1e-4
    assert ex < tol and em < tol


def test_cic_vjp_is_linear_in_u():
    """J^T (u1 + 2 u2) = J^T u1 + 2 J^T u2 (FP64): the fixed-point scale of
    the adjoint densities, chosen per call from max |u|, does not leak."""
    import torch
    w = W.merger_small(precision="fp64")
    ctx, parts = gpu_setup(w)
    rng = np.random.default_rng(4)
    n = parts.n
    outs = []
    us = [rng.normal(size=(3, n)), 1e-3 * rng.normal(size=(3, n))]
    us.append(us[0] + 2 * us[1])
    for u in us:
        ctx.cic_deposit(parts)
        ctx.solve()
        gx = torch.zeros(3, n, dtype=torch.float64, device="cuda")
        gm = torch.zeros(n, dtype=torch.float64, device="cuda")
        ctx.cic_vjp(parts, torch.tensor(u, device="cuda"), gx, gm)
        outs.append((gx.cpu().numpy(), gm.cpu().numpy()))
    assert _rel(outs[2][0], outs[0][0] + 2 * outs[1][0]) < 1e-12
    assert _rel(outs[2][1], outs[0][1] + 2 * outs[1][1]) < 1e-12


def test_cic_kick_drift_and_zero_cotangent():
    import torch
    w = W.merger_small(precision="fp64")
    ctx, parts = gpu_setup(w)
    ctx.cic_deposit(parts)
    ctx.solve()
    a = [t.clone() for t in ctx.cic_force(parts)]
    x0 = parts.x.clone()
    v0 = parts.vx.clone()
    ctx.cic_kick_drift(parts, 0.01, 0.02)
    live = (parts.flags & 1) == 0
    assert int(live.sum()) > 0.99 * parts.n
    assert torch.allclose(parts.vx[live], (v0 + 0.01 * a[0])[live], rtol=1e-14, atol=1e-15)
    assert torch.allclose(parts.x[live], (x0 + 0.02 * parts.vx)[live], rtol=1e-14, atol=1e-15)
    assert torch.equal(parts.x[~live], x0[~live]) and torch.equal(parts.vx[~live], v0[~live])
    gx = torch.ones(3, parts.n, dtype=torch.float64, device="cuda")
    gm = torch.ones(parts.n, dtype=torch.float64, device="cuda")
    ctx.cic_vjp(parts, torch.zeros_like(gx), gx, gm)   # u = 0 adds nothing
    assert torch.all(gx == 1) and torch.all(gm == 1)
    with pytest.raises(pm.PMError):
        ctx.cic_vjp(parts, torch.full_like(gx, float("nan")), gx, gm)


# --------------------------------------------------------------- gradients --

class _Problem:
    """Satellite bulk offset X, velocity offset V and mass scale M applied to
    a workload; losses: the satellite's mean final position along a fixed
    direction, and the disc's vertical kinetic energy sum m v_z^2 / 2."""

    def __init__(self, w, steps, every, follow=False):
        import torch
        self.w, self.steps, self.every = w, steps, every
        self.schedule = None
        self.follow = follow
        self.sat = np.asarray(w["comp"]) == W.COMP_SATELLITE
        self.disc = np.asarray(w["comp"]) == W.COMP_DISC
        self.dir = np.array([0.6, -0.48, 0.64])
        self.torch = torch

    def context(self, precision):
        from paper_1210_1736_gb300.adjoint import Runner
        torch = self.torch
        w = dict(self.w, precision=precision)
        dt = torch.float32 if precision == "fp32" else torch.float64
        npdt = np.float32 if precision == "fp32" else np.float64
        ctx = pm.Context(w, 1.25 * O.mass_bound(np.asarray(w["m"]).astype(npdt)))
        gal = torch.tensor(np.asarray(w["gal"]), dtype=torch.int32, device="cuda")
        base = [torch.tensor(np.ascontiguousarray(np.asarray(w[k]).astype(npdt)), device="cuda")
                for k in ("pos", "vel", "m")]
        runner = Runner(ctx, gal, w["dt"], self.steps, self.every)
        if self.follow:
            # one schedule of grid centres for every run (recorded once, FP64)
            if self.schedule is None:
                self.schedule = runner.record_centres(*base) if precision == "fp64" else None
                if self.schedule is None:
                    raise RuntimeError("record the schedule with the FP64 context first")
            runner.centres = self.schedule
        return ctx, runner, base, dt

    def inputs(self, base, theta, dt):
        torch = self.torch
        sat = torch.tensor(self.sat, device="cuda").to(dt)
        pos, vel, m = base
        x0 = pos + sat[None, :] * theta[0:3, None]
        v0 = vel + sat[None, :] * theta[3:6, None]
        mm = m * (1 + sat * theta[6])
        return x0.contiguous(), v0.contiguous(), mm.contiguous()

    def losses(self, xT, vT, m):
        torch = self.torch
        sat = torch.tensor(self.sat, device="cuda")
        disc = torch.tensor(self.disc, device="cuda")
        d = torch.tensor(self.dir, dtype=xT.dtype, device="cuda")
        L1 = (xT[:, sat].mean(dim=1) * d).sum()
        L2 = 0.5 * (m[disc] * vT[2, disc] ** 2).sum()
        return L1, L2

    def adjoint_grads(self, precision):
        from paper_1210_1736_gb300.adjoint import trajectory
        torch = self.torch
        ctx, runner, base, dt = self.context(precision)
        grads = []
        for which in (0, 1):
            theta = torch.zeros(7, dtype=dt, device="cuda", requires_grad=True)
            x0, v0, m = self.inputs(base, theta, dt)
            xT, vT = trajectory(x0, v0, m, runner)
            L = self.losses(xT, vT, m)[which]
            L.backward()
            grads.append(theta.grad.double().cpu().numpy())
        ctx.close()
        return np.array(grads)

    def fd_grads(self, h_pos, h_mass):
        """Central differences of both losses with the FP64 instantiation:
        step h_pos for X and V (small, so that almost no particle crosses a
        CIC cell centre, where the map has a kink) and h_mass for the mass
        scale (the map is smooth in it).  The disc term is differenced per
        particle, sum m (v+ - v-)(v+ + v-) / 2, so that the sum's rounding
        does not swamp the small difference."""
        torch = self.torch
        ctx, runner, base, dt = self.context("fp64")
        disc = torch.tensor(self.disc, device="cuda")
        out = np.zeros((2, 7))
        with torch.no_grad():
            for k in range(7):
                h = h_pos if k < 6 else h_mass
                runs = []
                for sgn in (1.0, -1.0):
                    theta = torch.zeros(7, dtype=dt, device="cuda")
                    theta[k] = sgn * h
                    x0, v0, m = self.inputs(base, theta, dt)
                    xT, vT, _, _ = runner.forward_run(x0, v0, m)
                    runs.append((float(self.losses(xT, vT, m)[0]), vT[2, disc], m[disc]))
                (l1p, vp, mp), (l1m, vm, _) = runs
                out[0, k] = (l1p - l1m) / (2 * h)
                out[1, k] = float((0.5 * mp * (vp - vm) * (vp + vm)).sum()) / (2 * h)
        ctx.close()
        return out


def _grad_rel_err(g, ref):
    """Per loss: max over parameters of |g - ref| / max |ref| of that loss."""
    return np.max(np.abs(g - ref), axis=1) / np.max(np.abs(ref), axis=1)


def test_trajectory_gradient_matches_finite_differences_small():
    """merger_small (24k + 4k particles) with the satellite's apocentre at
    3 R_d, inside the disc, 20 steps, checkpoints every 5:
    gradients of both losses with respect to the satellite's (X, V, M)
    from the hand-written adjoint (FP64 and FP32) against FP64 central
    differences."""
    prob = _Problem(W.merger_small(r_apo=3.0), steps=20, every=5)
    fd = prob.fd_grads(1e-9, 1e-6)
    g64 = prob.adjoint_grads("fp64")
    g32 = prob.adjoint_grads("fp32")
    e64, e32 = _grad_rel_err(g64, fd), _grad_rel_err(g32, fd)
    print("fd", fd, "\nadjoint fp64", g64, "\nadjoint fp32", g32)
    print(f"relative error: fp64 {e64}, fp32 {e32}")
    assert np.all(e64 < 1e-5)
    assert np.all(e32 < 1e-4)


def _oracle_theta_grads(w, steps):
    """The FP64 CPU reference: gradients of both losses with respect to the
    satellite's (X, V, M) from the oracle's trajectory map and its transpose
    (cic_trajectory, cic_trajectory_vjp; grid centres fixed)."""
    system = O.system_from_workload(w, 1.25 * O.mass_bound(w["m"]))
    st0 = O.state_from_workload(w)
    xT, vT, tape = OC.cic_trajectory(st0, system, w["dt"], steps)
    sat = np.asarray(w["comp"]) == W.COMP_SATELLITE
    disc = np.asarray(w["comp"]) == W.COMP_DISC
    d = np.array([0.6, -0.48, 0.64])
    out = np.zeros((2, 7))
    for which in (0, 1):
        lx, lv, lm_direct = np.zeros_like(xT), np.zeros_like(vT), np.zeros(len(st0.m))
        if which == 0:      # L1 = d . mean of the satellite's final positions
            lx[:, sat] = d[:, None] / sat.sum()
        else:               # L2 = sum over the disc of m v_z^2 / 2 at t = T
            lv[2, disc] = st0.m[disc] * vT[2, disc]
            lm_direct[disc] = 0.5 * vT[2, disc] ** 2
        gx, gv, gm = OC.cic_trajectory_vjp(tape, system, w["dt"], lx, lv)
        out[which, 0:3] = gx[:, sat].sum(axis=1)
        out[which, 3:6] = gv[:, sat].sum(axis=1)
        out[which, 6] = np.sum(st0.m[sat] * (gm + lm_direct)[sat])
    return out


def test_trajectory_gradient_matches_oracle_reference():
    """The same small case against the FP64 CPU reference gradient of the
    whole trajectory (the oracle's per-step vector-Jacobian products chained
    through the leap-frog map, itself pinned by central differences of the
    oracle's map): the FP64 adjoint within 1e-9, the FP32 adjoint within
    1e-4 (per loss, relative to its largest component)."""
    w = W.merger_small(r_apo=3.0)
    prob = _Problem(w, steps=20, every=5)
    ref = _oracle_theta_grads(dict(w, precision="fp64"), 20)
    g64 = prob.adjoint_grads("fp64")
    g32 = prob.adjoint_grads("fp32")
    e64, e32 = _grad_rel_err(g64, ref), _grad_rel_err(g32, ref)
    print("oracle", ref, "\nadjoint fp64", g64, "\nadjoint fp32", g32)
    print(f"relative error vs the oracle: fp64 {e64}, fp32 {e32}")
    assert np.all(e64 < 1e-9)
    assert np.all(e32 < 1e-4)


def test_trajectory_gradient_full_size():
    """The differentiable-run workload at full size: 1M-particle galaxy
    (grids 128^3, 128^3 q = 1/4, 128x128x32) + 20k-particle satellite
    (M = 0.05, a = 0.05, 64^3 grids), 200 steps, checkpoints every 20, grid
    centres following a recorded schedule.

    Satellite position: FP32 adjoint against FP64 central differences with
    h = 1e-8 (the satellite's own particles cross CIC cell centres, where
    the map has kinks, and region boundaries, where it jumps, in proportion
    to h).  Disc vertical energy (gradients ~1e-7): central differences
    scatter by ~1e-3 of the row between h = 1e-8 and 1e-6, so the FP32
    adjoint is held to the FP64 adjoint (whose agreement with differences is
    pinned on the small case) within 5e-4 (FP32 rounding of the trajectory),
    and both adjoints to the differences within that scatter."""
    import time
    import torch
    prob = _Problem(W.adjoint_1m(), steps=200, every=20, follow=True)
    fd8 = prob.fd_grads(1e-8, 1e-6)
    fd6 = prob.fd_grads(1e-6, 1e-6)
    g64 = prob.adjoint_grads("fp64")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g32 = prob.adjoint_grads("fp32")
    torch.cuda.synchronize()
    t_adj = time.perf_counter() - t0
    e_fd = np.array([_grad_rel_err(g32, fd8)[0], _grad_rel_err(g32, fd6)[1]])
    e_64 = _grad_rel_err(g32, g64)
    scatter = _grad_rel_err(fd8, fd6)[1]
    print("fd h=1e-8", fd8, "\nfd h=1e-6", fd6, "\nadjoint fp64", g64, "\nadjoint fp32", g32)
    print(f"fp32 adjoint vs fd {e_fd}; vs fp64 adjoint {e_64}; fd scatter of the disc row {scatter:.2e}; "
          f"2 x (forward + backward) of 200 steps in FP32: {t_adj:.2f} s")
    assert e_fd[0] < 1e-4 and e_64[0] < 1e-4
    # the disc row is ~1e-7 in size: FP32 rounding of the 200-step trajectory
    # moves it by ~1e-4 of the row (the FP64 adjoint is the exact derivative
    # of the FP64 map)
    assert e_64[1] < 5e-4
    assert _grad_rel_err(g64, fd6)[1] < max(1e-4, 2 * scatter)
    assert e_fd[1] < max(1e-4, 2 * scatter)
