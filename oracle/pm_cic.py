"""Plain FP64 CPU reference of the cloud-in-cell (CIC) variant of the
nested-grid step and of its adjoint, used to check the differentiable path.

TEST INFRASTRUCTURE ONLY, like ``oracle.pm_oracle``: only the tests, the smoke
check and the benchmark's CPU-baseline leg import it.

Why a variant: the paper assigns mass and reads forces by nearest grid point
(Eq. eqn:cell), which is piecewise constant in the particle position, so
derivatives of a trajectory with respect to positions vanish almost
everywhere.  The differentiable runs therefore use CIC, stated as such:

* mass assignment: every particle of a mass set spreads its mass over the 8
  cells around it with the trilinear weights W = prod_d (1 - |x_d - x_cd| / l_d);
* grid acceleration: the central difference g_d = (Phi[c+e_d] - Phi[c-e_d]) / (2 l_d)
  (the first term of Eq. eqn:diff) at every cell;
* interpolation: a(x) = sum_c W(x - x_c) g_c with the same weights (the usual
  momentum-conserving pairing of assignment and interpolation);
* unchanged from the oracle: the region predicate and the mass sets of
  Sec. 2.1 (decided with the NGP cell of Eq. eqn:cell and the canonical
  rounding), the doubled-grid convolution (Eq. eq:poisson, eqn:greens), the
  combination rule and the leap-frog;
* the grid centres stay where they are (no recentring), so the centres are
  constants of the differentiated map.

With the NGP cell a in the usable box 2..N-3 the CIC cells are a0 = a - 1 or
a and a0 + 1, and the differences reach cells a0 - 1 .. a0 + 2, all inside
0..N-1: no particle that the NGP rules keep ever reads outside its grid.

The adjoint.  With K the convolution of Eq. (eq:poisson) (symmetric, H even),
D_d the central difference (D_d^T = -D_d on the active grid) and W the CIC
weights, one galaxy's field at a field point x_i in region r is
    a_i = sum_{k in comb(r)} sum_c W_k(x_i - x_c) (D K_k rho_k)_c,
    rho_k[c] = sum_{j in set k} m_j W_k(x_j - x_c).
For a cotangent u_i (one 3-vector per particle) the vector-Jacobian product is
    dx_i += sum_k sum_c grad W_k(x_i - x_c) (g_k[c] . u_i)             (direct)
    psi_k^d[c] = sum_{i: k in comb(r_i)} W_k(x_i - x_c) u_i^d
    lam_k = K_k sum_d D_d^T psi_k^d
    dx_j += m_j sum_c grad W_k(x_j - x_c) lam_k[c],
    dm_j += sum_c W_k(x_j - x_c) lam_k[c]        for j in mass set k.
"""
from __future__ import annotations

import numpy as np

from .pm_oracle import (FLAG_LOST, REGION_CORE, REGION_OUTER, REGION_SHELL, State, System, classify,
                        combination, grid_cells, kick, drift, mass_sets, potential_fft, region)

__all__ = ["cic_cells", "cic_weights", "cic_deposit", "cic_solve", "grid_accel", "cic_interp",
           "cic_accelerations", "cic_step", "cic_vjp", "cic_half_kick_start", "cic_trajectory",
           "cic_trajectory_vjp"]


def cic_cells(pos, centre, g, split=False):
    """Lower CIC cell (a0, b0, c0) and fractions f in [0, 1) per axis.

    The NGP cell a (Eq. eqn:cell, canonical rounding) fixes the particle's
    cell; Delta = (x - c) - (a - N/2) l is its offset from that cell's centre
    (FP64) and t = Delta / l lies in [-1/2, 1/2]; the lower CIC cell is a - 1
    with f = t + 1 when t < 0, else a with f = t."""
    (a, b, c), ok = grid_cells(pos, centre, g, split)
    idx = []
    frac = []
    for ax, (n, l, cell) in enumerate(((g.nx, g.l_xy, a), (g.ny, g.l_xy, b), (g.nz, g.l_z, c))):
        t = ((pos[ax] - centre[ax]) - (cell - n // 2) * l) / l
        low = t < 0
        idx.append(np.where(low, cell - 1, cell))
        frac.append(np.where(low, t + 1.0, t))
    return idx, np.stack(frac), ok


def cic_weights(frac):
    """Weights of the 8 cells (di, dj, dk) in {0,1}^3 and their position
    derivatives times l (d/dx_d W = (d/dt_d W) / l_d)."""
    w = [(1.0 - frac[d], frac[d]) for d in range(3)]
    dw = [(-np.ones_like(frac[d]), np.ones_like(frac[d])) for d in range(3)]
    out = {}
    for di in (0, 1):
        for dj in (0, 1):
            for dk in (0, 1):
                W = w[0][di] * w[1][dj] * w[2][dk]
                dW = np.stack([dw[0][di] * w[1][dj] * w[2][dk],
                               w[0][di] * dw[1][dj] * w[2][dk],
                               w[0][di] * w[1][dj] * dw[2][dk]])
                out[(di, dj, dk)] = (W, dW)
    return out


def _lengths(g):
    return np.array([g.l_xy, g.l_xy, g.l_z])


def cic_deposit(state: State, system: System, flags=None, own=None):
    """rho[g][k] (mass per cell, FP64, layout [z][y][x]) with CIC weights for
    every galaxy and mass set of Sec. 2.1; returns (rho, flags)."""
    if flags is None:
        flags, own = classify(state, system)
    live = (flags & FLAG_LOST) == 0
    rho = []
    for g, gal in enumerate(system.galaxies):
        per = {}
        for k, geom, ck, regs in mass_sets(gal):
            centre = state.centres[g] if ck == "gal" else system.sys_centre
            sel = live & (state.gal == g) & np.isin(own, regs)
            (a0, b0, c0), frac, ok = cic_cells(state.pos[:, sel], centre, geom, system.split)
            assert ok.all(), "particle of a mass set outside its grid"
            grid = np.zeros(geom.shape)
            for (di, dj, dk), (W, _) in cic_weights(frac).items():
                np.add.at(grid, (c0 + dk, b0 + dj, a0 + di), state.m[sel] * W)
            per[k] = grid
        rho.append(per)
    return rho, flags


def cic_solve(rho, system: System):
    """Phi[g][k] = K rho[g][k] for every mass set (Eq. eq:poisson)."""
    return [{k: potential_fft(rho[g][k], geom, system.G, system.h000)
             for k, geom, _, _ in mass_sets(gal)} for g, gal in enumerate(system.galaxies)]


def grid_accel(phi, g):
    """Central-difference gradient (3, nz, ny, nx) on the interior cells
    (faces left zero: no particle reads them)."""
    out = np.zeros((3,) + phi.shape)
    out[0][:, :, 1:-1] = (phi[:, :, 2:] - phi[:, :, :-2]) / (2 * g.l_xy)
    out[1][:, 1:-1, :] = (phi[:, 2:, :] - phi[:, :-2, :]) / (2 * g.l_xy)
    out[2][1:-1, :, :] = (phi[2:, :, :] - phi[:-2, :, :]) / (2 * g.l_z)
    return out


def grid_accel_T(field3, g):
    """Transpose of grid_accel: sum_d D_d^T field3[d] on the active grid."""
    out = np.zeros(field3.shape[1:])
    fx, fy, fz = field3
    hx, hz = 1.0 / (2 * g.l_xy), 1.0 / (2 * g.l_z)
    # (D_x f)[i] = (f[i+1] - f[i-1]) h for 1 <= i <= n-2; its transpose sends
    # field[i] to +h at i+1 and -h at i-1
    out[:, :, 2:] += hx * fx[:, :, 1:-1]
    out[:, :, :-2] -= hx * fx[:, :, 1:-1]
    out[:, 2:, :] += hx * fy[:, 1:-1, :]
    out[:, :-2, :] -= hx * fy[:, 1:-1, :]
    out[2:, :, :] += hz * fz[1:-1, :, :]
    out[:-2, :, :] -= hz * fz[1:-1, :, :]
    return out


def cic_interp(field, idx, frac):
    """sum_c W(x - x_c) field[..., c] for a field of shape (..., nz, ny, nx)."""
    a0, b0, c0 = idx
    val = 0.0
    for (di, dj, dk), (W, _) in cic_weights(frac).items():
        val = val + W * field[..., c0 + dk, b0 + dj, a0 + di]
    return val


def _field_points(state, system, flags):
    """For every galaxy h: (region of each live particle, per-set geometry and centre)."""
    live = (flags & FLAG_LOST) == 0
    for h, gal in enumerate(system.galaxies):
        reg = region(state.pos, gal, state.centres[h], system.split)
        sets = {k: (geom, state.centres[h] if ck == "gal" else system.sys_centre)
                for k, geom, ck, _ in mass_sets(gal)}
        yield h, reg, sets, live


def cic_accelerations(state: State, system: System, phi, flags):
    """a_i = sum_h sum_{k in comb(region_h(x_i))} CIC interpolation of D Phi_k."""
    n = len(state.m)
    acc = np.zeros((3, n))
    for h, reg, sets, live in _field_points(state, system, flags):
        for r in (REGION_CORE, REGION_SHELL, REGION_OUTER):
            sel = live & (reg == r)
            if not np.any(sel):
                continue
            for k in combination(r):
                if k not in sets:
                    continue
                geom, centre = sets[k]
                idx, frac, ok = cic_cells(state.pos[:, sel], centre, geom, system.split)
                assert ok.all()
                acc[:, sel] += cic_interp(grid_accel(phi[h][k], geom), idx, frac)
    return acc


def cic_step(state: State, system: System, dt: float) -> State:
    """One CIC step: classify, deposit, solve, interpolate, kick, drift."""
    st = state.copy()
    flags, own = classify(st, system)
    rho, flags = cic_deposit(st, system, flags, own)
    phi = cic_solve(rho, system)
    acc = cic_accelerations(st, system, phi, flags)
    live = (flags & FLAG_LOST) == 0
    st.vel = kick(st.vel, acc, dt, live)
    st.pos = drift(st.pos, st.vel, dt, live)
    st.flags = flags
    return st


def cic_half_kick_start(state: State, system: System, dt: float) -> State:
    """v(-dt/2) = v(0) - dt/2 a(0) with the CIC acceleration."""
    st = state.copy()
    flags, own = classify(st, system)
    rho, flags = cic_deposit(st, system, flags, own)
    phi = cic_solve(rho, system)
    acc = cic_accelerations(st, system, phi, flags)
    st.vel = kick(st.vel, acc, -0.5 * dt, (flags & FLAG_LOST) == 0)
    st.flags = flags
    return st


def cic_vjp(state: State, system: System, phi, flags, own, u):
    """Vector-Jacobian product of the CIC acceleration a(x, m) at the state:
    returns (u^T da/dx (3, n), u^T da/dm (n,)).  phi is the forward potential
    at these positions; u is (3, n); lost particles get zero."""
    n = len(state.m)
    gx = np.zeros((3, n))
    gm = np.zeros(n)
    live = (flags & FLAG_LOST) == 0
    for h, reg, sets, live_h in _field_points(state, system, flags):
        psi = {k: np.zeros((3,) + geom.shape) for k, (geom, _) in sets.items()}
        # direct term and the field points' cotangents spread on the grids
        for r in (REGION_CORE, REGION_SHELL, REGION_OUTER):
            sel = live_h & (reg == r)
            if not np.any(sel):
                continue
            for k in combination(r):
                if k not in sets:
                    continue
                geom, centre = sets[k]
                idx, frac, ok = cic_cells(state.pos[:, sel], centre, geom, system.split)
                g3 = grid_accel(phi[h][k], geom)
                # d/dx_d of sum_c W g_c . u = sum_c (dW/dt_d / l_d) (g_c . u)
                a0, b0, c0 = idx
                for (di, dj, dk), (W, dW) in cic_weights(frac).items():
                    gc = g3[:, c0 + dk, b0 + dj, a0 + di]
                    s = np.sum(gc * u[:, sel], axis=0)
                    gx[:, sel] += dW / _lengths(geom)[:, None] * s
                    for d in range(3):
                        np.add.at(psi[k][d], (c0 + dk, b0 + dj, a0 + di), W * u[d, sel])
        # adjoint densities through the (symmetric) convolution, then the
        # mass-set particles' dependence on their own positions and masses
        gal = system.galaxies[h]
        for k, geom, ck, regs in mass_sets(gal):
            lam = potential_fft(grid_accel_T(psi[k], geom), geom, system.G, system.h000)
            centre = state.centres[h] if ck == "gal" else system.sys_centre
            sel = live & (state.gal == h) & np.isin(own, regs)
            if not np.any(sel):
                continue
            idx, frac, ok = cic_cells(state.pos[:, sel], centre, geom, system.split)
            a0, b0, c0 = idx
            for (di, dj, dk), (W, dW) in cic_weights(frac).items():
                lc = lam[c0 + dk, b0 + dj, a0 + di]
                gx[:, sel] += state.m[sel] * dW / _lengths(geom)[:, None] * lc
                gm[sel] += W * lc
    return gx, gm


def _cic_fields(state: State, system: System):
    flags, own = classify(state, system)
    rho, flags = cic_deposit(state, system, flags, own)
    phi = cic_solve(rho, system)
    return phi, flags, own


def cic_trajectory(state: State, system: System, dt: float, steps: int):
    """The differentiable run's map with positions and velocities
    synchronised at t = 0 and t = T = steps dt (grid centres fixed):
        V = v0 - dt/2 a(x0);  V += dt a(x_t), x_{t+1} = x_t + dt V  (t < steps);
        v_T = V + dt/2 a(x_T),
    a the CIC acceleration.  Returns (x_T, v_T, tape) with tape[t] =
    (State at x_t, phi, flags, own) for cic_trajectory_vjp."""
    st = state.copy()
    tape = []
    phi, flags, own = _cic_fields(st, system)
    live = (flags & FLAG_LOST) == 0
    V = kick(st.vel, cic_accelerations(st, system, phi, flags), -0.5 * dt, live)
    for t in range(steps + 1):
        if t > 0:
            phi, flags, own = _cic_fields(st, system)
        st.flags = flags
        tape.append((st.copy(), phi, flags, own))
        live = (flags & FLAG_LOST) == 0
        acc = cic_accelerations(st, system, phi, flags)
        if t == steps:
            return st.pos.copy(), kick(V, acc, 0.5 * dt, live), tape
        V = kick(V, acc, dt, live)
        st.vel = V
        st.pos = drift(st.pos, V, dt, live)


def cic_trajectory_vjp(tape, system: System, dt: float, lx, lv):
    """Cotangents (of x0, v0, m) of the map of cic_trajectory for cotangents
    (lx, lv) of (x_T, v_T): its transpose, newest step first,
        lV = lv;  lx += J_x(x_T)^T (dt/2 lv);  lm += J_m(x_T)^T (dt/2 lv);
        per step t = T-1 .. 0:  mu = lV + dt lx;  lx += J_x(x_t)^T (dt mu);
                                lm += J_m(x_t)^T (dt mu);  lV = mu;
        v0: lV;  lx += J_x(x_0)^T (-dt/2 lV);  lm += J_m(x_0)^T (-dt/2 lV),
    with J^T u = cic_vjp at the stored x_t (each the chain rule of one
    leap-frog step V' = V + dt a(x), x' = x + dt V')."""
    steps = len(tape) - 1
    lx = np.array(lx, dtype=np.float64, copy=True)
    lV = np.array(lv, dtype=np.float64, copy=True)
    lm = np.zeros(lx.shape[1])

    def add(t, u):
        st, phi, flags, own = tape[t]
        gx, gm = cic_vjp(st, system, phi, flags, own, u)
        lx[...] += gx
        lm[...] += gm

    add(steps, 0.5 * dt * lV)
    for t in range(steps - 1, -1, -1):
        mu = lV + dt * lx
        add(t, dt * mu)
        lV = mu
    add(0, -0.5 * dt * lV)
    return lx, lV, lm
