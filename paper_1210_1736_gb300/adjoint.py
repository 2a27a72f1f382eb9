"""Differentiable CIC trajectories: a torch.autograd.Function over many
leap-frog steps of the CIC variant, with a hand-written adjoint.

Every forward and backward operation runs in the library's kernels
(pm_cic_deposit, pm_solve, pm_cic_kick_drift, pm_cic_vjp); PyTorch only holds
the tensors and the checkpoints.

The map (positions and velocities synchronised at t = 0 and t = T = steps*dt):
    V    = v0 - dt/2 a(x0)                      (leap-frog start, Sec. 2.1)
    V    = V + dt a(x_t);  x_{t+1} = x_t + dt V   t = 0 .. steps-1
    v_T  = V + dt/2 a(x_T)
with a the CIC acceleration at fixed grid centres.  Its adjoint, from the
cotangents (lx, lv) of (x_T, v_T):
    lV = lv;  lx += J_x(x_T)^T (dt/2 lv);  lm += J_m(x_T)^T (dt/2 lv)
    per step, newest first:  mu = lV + dt lx;  lx += J_x(x_t)^T (dt mu);
                             lm += J_m(x_t)^T (dt mu);  lV = mu
    start:  lv0 = lV;  lx += J_x(x_0)^T (-dt/2 lV);  lm += ...
where J^T u is pm_cic_vjp.  The forward keeps (x, V, flags) every `every`
steps; the backward recomputes each segment's positions from its checkpoint
and walks it in reverse (one deposit + solve + vjp per step).
"""
from __future__ import annotations

import numpy as np
import torch

from . import pm


class Runner:
    """Fixed data of a differentiable run: the context (its grids), galaxy
    ids, time step, step count, checkpoint interval and the grid centres.

    centres: None keeps the context's centres for the whole run; otherwise an
    array (steps + 1, ngal, 3) of centres used for the force at x_t, a
    schedule fixed in advance (e.g. by record_centres) and therefore a
    constant of the differentiated map."""

    def __init__(self, ctx: "pm.Context", gal: torch.Tensor, dt: float, steps: int, every: int = 20,
                 centres=None):
        if ctx.precision not in ("fp32", "fp64"):
            raise ValueError("unknown precision")
        self.ctx, self.gal, self.dt, self.steps, self.every = ctx, gal, float(dt), int(steps), max(1, int(every))
        self.centres = None if centres is None else np.asarray(centres, dtype=np.float64)
        if self.centres is not None and self.centres.shape[0] != self.steps + 1:
            raise ValueError("centre schedule needs steps + 1 entries")

    def particles(self, x, v, m, flags):
        return pm.Particles.from_tensors(x, v, m, self.gal, flags)

    def accel_field(self, p, t):
        """Deposit and solve at p's positions x_t (potentials then current)."""
        if self.centres is not None:
            self.ctx.set_centres(self.centres[t])
        self.ctx.cic_deposit(p)
        self.ctx.solve()

    def vjp(self, p, t, u, gx, gm):
        self.accel_field(p, t)
        self.ctx.cic_vjp(p, u.contiguous(), gx, gm)

    def record_centres(self, x0, v0, m):
        """Runs the trajectory once, moving the grid centres by the library's
        recentring (centre of mass within R_core, Sec. 2.1) before every force
        evaluation, and keeps them as this runner's schedule."""
        dt = self.dt
        x = x0.detach().clone().contiguous()
        v = v0.detach().clone().contiguous()
        m = m.detach().contiguous()
        p = self.particles(x, v, m, torch.zeros(m.shape[0], dtype=torch.int32, device=m.device))
        sched = []
        saved, self.centres = self.centres, None
        try:
            for t in range(self.steps + 1):
                self.ctx.recentre(p)
                sched.append(self.ctx.centres())
                self.accel_field(p, t)
                if t < self.steps:
                    self.ctx.cic_kick_drift(p, 0.5 * dt if t == 0 else dt, dt)
        finally:
            self.centres = saved
        self.centres = np.array(sched)
        return self.centres

    def forward_run(self, x0, v0, m):
        """Returns x_T, v_T, the final flags and the checkpoints."""
        dt = self.dt
        x = x0.detach().clone().contiguous()
        v = v0.detach().clone().contiguous()
        m = m.detach().contiguous()
        flags = torch.zeros(m.shape[0], dtype=torch.int32, device=m.device)
        p = self.particles(x, v, m, flags)
        self.accel_field(p, 0)
        self.ctx.cic_kick_drift(p, -0.5 * dt, 0.0)
        ckpts = []
        for t in range(self.steps):
            if t % self.every == 0:
                ckpts.append((t, x.clone(), v.clone(), flags.clone()))
            self.accel_field(p, t)
            self.ctx.cic_kick_drift(p, dt, dt)
        self.accel_field(p, self.steps)
        self.ctx.cic_kick_drift(p, 0.5 * dt, 0.0)
        return x, v, flags, ckpts


class CICTrajectory(torch.autograd.Function):
    """(x0 (3, n), v0 (3, n), m (n,)) -> (x_T, v_T), differentiable in all three."""

    @staticmethod
    def forward(fctx, x0, v0, m, runner: Runner):
        xT, vT, flags, ckpts = runner.forward_run(x0, v0, m)
        fctx.runner = runner
        fctx.ckpts = ckpts
        fctx.x_T = xT
        fctx.flags_T = flags
        fctx.m = m.detach().contiguous()
        fctx.x0 = x0.detach().contiguous()
        return xT.clone(), vT.clone()

    @staticmethod
    def backward(fctx, gxT, gvT):
        R = fctx.runner
        dt = R.dt
        m = fctx.m
        dev, dtype = m.device, m.dtype
        lx = torch.zeros(3, m.shape[0], dtype=dtype, device=dev) if gxT is None else gxT.detach().clone().contiguous()
        lV = torch.zeros_like(lx) if gvT is None else gvT.detach().clone().contiguous()
        lm = torch.zeros_like(m)
        scratch_v = torch.zeros_like(lx)
        # end kick at x_T
        pT = R.particles(fctx.x_T, scratch_v, m, fctx.flags_T.clone())
        R.vjp(pT, R.steps, 0.5 * dt * lV, lx, lm)
        # steps, newest segment first
        for t0, xc, vc, fc in reversed(fctx.ckpts):
            t1 = min(t0 + R.every, R.steps)
            xs, fs = [], []
            x, v, f = xc.clone(), vc.clone(), fc.clone()
            p = R.particles(x, v, m, f)
            for t in range(t0, t1):
                R.accel_field(p, t)        # deposit flags particles lost at x_t
                xs.append(x.clone())
                fs.append(f.clone())
                R.ctx.cic_kick_drift(p, dt, dt)
            for k in range(len(xs) - 1, -1, -1):
                mu = lV + dt * lx
                pk = R.particles(xs[k], scratch_v, m, fs[k])
                R.vjp(pk, t0 + k, dt * mu, lx, lm)
                lV = mu
        # leap-frog start at x_0
        p0 = R.particles(fctx.x0.clone(), scratch_v, m, torch.zeros_like(fctx.flags_T))
        R.vjp(p0, 0, -0.5 * dt * lV, lx, lm)
        return lx, lV, lm, None


def trajectory(x0, v0, m, runner: Runner):
    """x_T, v_T of the CIC run from (x0, v0, m); differentiable."""
    return CICTrajectory.apply(x0, v0, m, runner)
