"""Plain FP64 CPU reference ("the oracle") for the nested-grid particle-mesh
gravity step of Superbox-10 (Bien, Brandt & Just 2012, MNRAS).

TEST INFRASTRUCTURE ONLY.  The tests, the smoke check and the benchmark's
CPU-baseline leg are the only code allowed to import this module.  The product
path (the CUDA library and its binding) never does, and shares no code with it.

Everything here is written for a reader checking it against the paper by eye:
numpy arrays, float64 throughout, no blocking, fusion or reordering.  numpy's
FFT serves as a library step (it only accelerates the exact doubled-grid
convolution); ``potential_direct`` is the plain O(cells^2) sum it replaces.

Where the paper is silent the readings below are used (each is listed with its
reason in the design notes of the repository):

* H(0,0,0) = h000 (default 1, in units of 1/l_xy): with it an isolated particle
  on a cubic grid feels exactly zero self-force under Eq. (eqn:diff).
* "Nearest integer" in Eq. (eqn:cell) is floor(u + 1/2); cells are 0-based and
  cell N/2 is centred on the grid centre.
* The cell index is evaluated by one canonical rounding sequence so that the
  GPU path assigns every particle to the same cell: the offset from a centre c
  is d = fl32(x - c) (one FP64 subtraction, rounded) for FP64 systems, and
  d = fl32(fl32(x32 - c_hi) - c_lo) with c_hi = fl32(c), c_lo = fl32(c - c_hi)
  for FP32 systems (positions are FP32 numbers there; the rule needs no FP64
  arithmetic per particle); then u = fl32(fl32(d gamma) + N/2) and
  a = floor(fl32(u + 1/2)), no fused multiply-add.  This is the only non-FP64
  arithmetic in this module.
* Masses are deposited as 64-bit fixed point, q = rint(m * 2^s),
  s = 62 - ceil(log2(mass_bound)); integer sums make the density exact.
* Flattened grids (Sec. 2.2.2): cell lengths l_xy, l_xy, l_z = q*l_xy and
  H = [i^2 + j^2 + (q k)^2]^(-1/2) in units of 1/l_xy.
* Delta in Eq. (eqn:diff) is the physical offset from the cell centre.
* Sign convention of Eq. (eq:poisson): Phi = +G sum rho H is positive and the
  acceleration is +grad Phi; the potential energy is W = -1/2 sum m Phi.
* Mass sets (Sec. 2.1, grids 1-5) and the potential combination rule use one
  region predicate: C (core) = r < R_core and inside the usable boxes of grid 1
  and grid 2; S (shell) = not C, r < R_out and inside the usable box of grid 2;
  O = the rest.  A particle is lost when it leaves the usable box of any coarse
  grid or r_sys >= R_sys, and stays lost.
* Recentring (Sec. 2.1: grids 1-3 follow the galaxy, centre of mass as the
  stated alternative to the density maximum): centre of mass of the galaxy's
  own live particles inside R_core of the previous centre, accumulated in exact
  integer fixed point so that the result does not depend on summation order.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from functools import lru_cache

import numpy as np

__all__ = [
    "Geometry", "Galaxy", "System", "cell_length", "q_crit", "fixed_shift", "mass_bound",
    "quantize_mass", "offset_f32", "cell_index", "in_box", "region",
    "classify", "deposit", "green_doubled", "green_hat", "potential_fft",
    "potential_direct", "accel_from_grid", "phi_at_particle",
    "accelerations", "kick", "drift", "recentre", "recentre_sums", "recentre_apply", "step", "diagnostics",
    "State", "solve_all", "rho_real", "mass_sets", "combination", "lost_mask",
    "grid_cells", "r2_f32", "half_kick_start", "potential_at", "REGION_CORE", "REGION_SHELL",
    "REGION_OUTER", "FLAG_LOST", "set_fft_workers",
]

REGION_CORE, REGION_SHELL, REGION_OUTER = 0, 1, 2
FLAG_LOST = 1


# ---------------------------------------------------------------------------
# Grid geometry (Sec. 2.1, Eq. eqn:cell; Sec. 2.2.2; Sec. 4.1, Table 3)
# ---------------------------------------------------------------------------

def cell_length(R: float, N: int, q: float = 1.0) -> float:
    """Cell length of a grid whose usable N-4 cells span the diameter 2R.

    Sec. 2.1 (two empty boundary cells, N-4 usable cells per dimension) and
    Sec. 4.1 / Table 3 (vertical resolution for flattening q and N cells, with
    R_out = 28 kpc): l = 2 R q / (N - 4).
    """
    return 2.0 * R * q / (N - 4)


def q_crit(r_core: float, r_out: float, r_sys: float, N: int) -> float:
    """Smallest admissible flattening of grids 2 and 3 (Sec. 2.2.2)."""
    return max(r_core / r_out, 4.0 / (N - 4) * r_sys / r_out)


@dataclass(frozen=True)
class Geometry:
    """One grid: nx*ny*nz active cells of lengths l_xy, l_xy, l_z.

    The flattening of Sec. 2.2.2 is q = l_z / l_xy.  The isolated-boundary
    work grid is 2nx*2ny*2nz (Sec. 2.1, doubling trick).
    """
    nx: int
    ny: int
    nz: int
    l_xy: float
    l_z: float

    @property
    def q(self) -> float:
        return self.l_z / self.l_xy

    @property
    def shape(self):  # array layout [z][y][x], x fastest
        return (self.nz, self.ny, self.nx)


@dataclass
class Galaxy:
    """Grids 1 (fine), 2/3 (medium) and 4/5 (coarse) of one galaxy (Sec. 2.1)."""
    coarse: Geometry
    medium: Geometry | None = None
    fine: Geometry | None = None
    r_core: float = 0.0
    r_out: float = 0.0
    centre: tuple = (0.0, 0.0, 0.0)
    recentre: bool = False


@dataclass
class System:
    galaxies: list
    r_sys: float
    sys_centre: tuple = (0.0, 0.0, 0.0)
    G: float = 1.0
    h000: float = 1.0
    mass_bound: float = 1.0
    precision: str = "fp64"    # selects the canonical offset rule (FP32 systems)

    @property
    def split(self) -> bool:
        return self.precision == "fp32"


# ---------------------------------------------------------------------------
# Fixed-point mass (exact deposit)
# ---------------------------------------------------------------------------

def fixed_shift(mass_bound: float) -> int:
    """s = 62 - ceil(log2(mass_bound)): any sum of masses below the bound fits
    in a signed 64-bit integer with one bit of headroom."""
    f, e = math.frexp(mass_bound)       # mass_bound = f * 2^e, 0.5 <= f < 1
    ceil_log2 = e - 1 if f == 0.5 else e
    return 62 - ceil_log2


def mass_bound(m) -> float:
    """The bound sum |m_i| that fixes the fixed-point scale (1 for no mass)."""
    b = float(np.sum(np.abs(np.asarray(m, dtype=np.float64))))
    return b if b > 0 else 1.0


def quantize_mass(m, s: int) -> np.ndarray:
    """q_i = rint(m_i * 2^s) (round half to even), int64."""
    return np.rint(np.ldexp(np.asarray(m, dtype=np.float64), s)).astype(np.int64)


# ---------------------------------------------------------------------------
# Cell assignment, Eq. (eqn:cell), with the canonical rounding sequence
# ---------------------------------------------------------------------------

def offset_f32(x, c: float, split: bool = False) -> np.ndarray:
    """Canonical FP32 offset of x from c: fl32(x - c) in FP64 (split=False),
    or fl32(fl32(x32 - c_hi) - c_lo) with c = c_hi + c_lo (split=True)."""
    if not split:
        return (np.asarray(x, dtype=np.float64) - np.float64(c)).astype(np.float32)
    c_hi = np.float32(c)
    c_lo = np.float32(np.float64(c) - np.float64(c_hi))
    x32 = np.asarray(x, dtype=np.float64).astype(np.float32)
    return ((x32 - c_hi).astype(np.float32) - c_lo).astype(np.float32)


def cell_index(d32: np.ndarray, l: float, n: int) -> np.ndarray:
    """a = [gamma x + N/2] (Eq. eqn:cell) with gamma = 1/l, nearest integer as
    floor(u + 1/2), evaluated as fl32(fl32(d*gamma) + N/2) then fl32(u + 1/2)."""
    gamma = np.float32(1.0 / l)
    u = (d32 * gamma).astype(np.float32)
    u = (u + np.float32(n // 2)).astype(np.float32)
    return np.floor((u + np.float32(0.5)).astype(np.float32)).astype(np.int64)


def in_box(idx: np.ndarray, n: int) -> np.ndarray:
    """Usable cells leave two empty cells at each boundary (Sec. 2.1):
    2 <= a <= N - 3."""
    return (idx >= 2) & (idx <= n - 3)


def r2_f32(dx, dy, dz) -> np.ndarray:
    """Squared distance from the three FP32 offsets, FP32, no fused multiply-add."""
    return ((dx * dx).astype(np.float32) + (dy * dy).astype(np.float32)
            ).astype(np.float32) + (dz * dz).astype(np.float32)


def grid_cells(pos, centre, g: Geometry, split: bool = False):
    """Cell indices (a, b, c) of positions in geometry g centred on `centre`,
    and the usable-box mask."""
    d = [offset_f32(pos[k], centre[k], split) for k in range(3)]
    a = cell_index(d[0], g.l_xy, g.nx)
    b = cell_index(d[1], g.l_xy, g.ny)
    c = cell_index(d[2], g.l_z, g.nz)
    ok = in_box(a, g.nx) & in_box(b, g.ny) & in_box(c, g.nz)
    return (a, b, c), ok


def region(pos, gal: Galaxy, centre, split: bool = False) -> np.ndarray:
    """Region of each position relative to one galaxy (Sec. 2.1 list of grids
    and potential combination rule): 0 core, 1 shell, 2 outer."""
    d = [offset_f32(pos[k], centre[k], split) for k in range(3)]
    r2 = r2_f32(*d)
    n = len(pos[0])
    reg = np.full(n, REGION_OUTER, dtype=np.int64)
    in_g2 = np.zeros(n, dtype=bool)
    if gal.medium is not None:
        _, in_g2 = grid_cells(pos, centre, gal.medium, split)
    core = np.zeros(n, dtype=bool)
    if gal.fine is not None and gal.medium is not None:
        _, in_g1 = grid_cells(pos, centre, gal.fine, split)
        core = (r2 < np.float32(gal.r_core * gal.r_core)) & in_g1 & in_g2
    shell = (~core) & (r2 < np.float32(gal.r_out * gal.r_out)) & in_g2
    reg[core] = REGION_CORE
    reg[shell] = REGION_SHELL
    return reg


def lost_mask(pos, system: System) -> np.ndarray:
    """Particles outside R_sys or outside the usable box of any coarse grid are
    lost (Sec. 2.1)."""
    d = [offset_f32(pos[k], system.sys_centre[k], system.split) for k in range(3)]
    lost = ~(r2_f32(*d) < np.float32(system.r_sys * system.r_sys))
    for gal in system.galaxies:
        _, ok = grid_cells(pos, system.sys_centre, gal.coarse, system.split)
        lost |= ~ok
    return lost


@dataclass
class State:
    """Particle state; v is the half-step velocity v(t - dt/2) (Sec. 2.1)."""
    pos: np.ndarray            # (3, n) float64
    vel: np.ndarray            # (3, n) float64
    m: np.ndarray              # (n,) float64
    gal: np.ndarray            # (n,) int64
    flags: np.ndarray          # (n,) int64, bit 0 = lost
    centres: np.ndarray        # (ngal, 3) float64, centres of grids 1-3

    def copy(self):
        return State(self.pos.copy(), self.vel.copy(), self.m.copy(),
                     self.gal.copy(), self.flags.copy(), self.centres.copy())


def classify(state: State, system: System):
    """Lost flags (sticky) and, per particle, its region in its own galaxy."""
    lost = ((state.flags & FLAG_LOST) != 0) | lost_mask(state.pos, system)
    flags = np.where(lost, state.flags | FLAG_LOST, state.flags)
    own = np.full(len(state.m), REGION_OUTER, dtype=np.int64)
    for g, gal in enumerate(system.galaxies):
        sel = state.gal == g
        if np.any(sel):
            own[sel] = region(state.pos[:, sel], gal, state.centres[g], system.split)
    return flags, own


# ---------------------------------------------------------------------------
# Mass assignment (Sec. 2.1 rho = mass per cell; Sec. 2.2.1 individual masses)
# ---------------------------------------------------------------------------

def mass_sets(gal: Galaxy):
    """(set number, geometry, centre kind, regions) for grids 1..5 (Sec. 2.1)."""
    sets = []
    if gal.fine is not None and gal.medium is not None:
        sets.append((1, gal.fine, "gal", (REGION_CORE,)))
    if gal.medium is not None:
        sets.append((2, gal.medium, "gal", (REGION_CORE,)))
        sets.append((3, gal.medium, "gal", (REGION_SHELL,)))
        sets.append((4, gal.coarse, "sys", (REGION_CORE, REGION_SHELL)))
    sets.append((5, gal.coarse, "sys", (REGION_OUTER,)))
    return sets


def deposit(state: State, system: System, flags=None, own=None):
    """Integer densities rho[g][k] (int64, layout [z][y][x]) for every galaxy g
    and mass set k; returns (rho, flags, shift)."""
    if flags is None:
        flags, own = classify(state, system)
    s = fixed_shift(system.mass_bound)
    q = quantize_mass(state.m, s)
    live = (flags & FLAG_LOST) == 0
    rho = []
    for g, gal in enumerate(system.galaxies):
        per = {}
        for k, geom, ck, regs in mass_sets(gal):
            centre = state.centres[g] if ck == "gal" else system.sys_centre
            sel = live & (state.gal == g) & np.isin(own, regs)
            (a, b, c), ok = grid_cells(state.pos[:, sel], centre, geom, system.split)
            assert ok.all(), "particle of a mass set outside its grid"
            grid = np.zeros(geom.shape, dtype=np.int64)
            np.add.at(grid, (c, b, a), q[sel])
            per[k] = grid
        rho.append(per)
    return rho, flags, s


# ---------------------------------------------------------------------------
# Potential: Eq. (eq:poisson), (eqn:greens), doubling (eq:symmetry)
# ---------------------------------------------------------------------------

def green_doubled(g: Geometry, h000: float) -> np.ndarray:
    """H on the 2nz*2ny*2nx grid, even-extended per Eq. (eq:symmetry):
    H[a] uses the distance min(a, 2N - a) along each axis; flattened form
    [i^2 + j^2 + (q k)^2]^(-1/2) in units of 1/l_xy; H(0,0,0) = h000."""
    i = np.arange(2 * g.nx); i = np.minimum(i, 2 * g.nx - i).astype(np.float64)
    j = np.arange(2 * g.ny); j = np.minimum(j, 2 * g.ny - j).astype(np.float64)
    k = np.arange(2 * g.nz); k = np.minimum(k, 2 * g.nz - k).astype(np.float64)
    r2 = (k[:, None, None] * g.q) ** 2 + j[None, :, None] ** 2 + i[None, None, :] ** 2
    with np.errstate(divide="ignore"):
        H = 1.0 / np.sqrt(r2)
    H[0, 0, 0] = h000
    return H


_FFT_WORKERS = None


def set_fft_workers(n):
    """Threads of the library FFT behind potential_fft and green_hat: None
    (the default) uses numpy's single-threaded FFT, n > 1 scipy.fft with n
    threads (the same pocketfft algorithm; results agree to rounding).  The
    arithmetic of the method is unchanged; large test workloads use it."""
    global _FFT_WORKERS
    _FFT_WORKERS = n if (n is not None and n > 1) else None


def _rfftn(x):
    if _FFT_WORKERS is None:
        return np.fft.rfftn(x)
    import scipy.fft
    return scipy.fft.rfftn(x, workers=_FFT_WORKERS)


def _irfftn(x, shape):
    if _FFT_WORKERS is None:
        return np.fft.irfftn(x, s=shape, axes=(0, 1, 2))
    import scipy.fft
    return scipy.fft.irfftn(x, s=shape, axes=(0, 1, 2), workers=_FFT_WORKERS)


@lru_cache(maxsize=16)
def green_hat(g: Geometry, h000: float) -> np.ndarray:
    """DFT of the doubled H (real-input half spectrum)."""
    return _rfftn(green_doubled(g, h000))


def rho_real(rho_int: np.ndarray, s: int) -> np.ndarray:
    """Fixed-point density back to mass per cell, FP64."""
    return np.ldexp(rho_int.astype(np.float64), -s)


def potential_fft(rho: np.ndarray, g: Geometry, G: float, h000: float) -> np.ndarray:
    """Phi = G/l_xy * IDFT(DFT(rho_pad) * DFT(H)) / (2nx 2ny 2nz), active part.

    Sec. 2.1: zero-pad the active N^3 region into the doubled grid, transform,
    multiply by H-hat, transform back; the result is exact in the active region
    (Eastwood & Brownrigg 1979).  `rho` is mass per cell (float64)."""
    pad = np.zeros((2 * g.nz, 2 * g.ny, 2 * g.nx))
    pad[: g.nz, : g.ny, : g.nx] = rho
    conv = _irfftn(_rfftn(pad) * green_hat(g, h000), pad.shape)
    return (G / g.l_xy) * conv[: g.nz, : g.ny, : g.nx]


def potential_direct(rho: np.ndarray, g: Geometry, G: float, h000: float) -> np.ndarray:
    """Eq. (eq:poisson) as the plain sum over all cell pairs (small grids only)."""
    cz, cy, cx = np.meshgrid(np.arange(g.nz), np.arange(g.ny), np.arange(g.nx), indexing="ij")
    cells = np.stack([cx.ravel(), cy.ravel(), cz.ravel()], axis=1).astype(np.float64)
    dx = cells[:, None, 0] - cells[None, :, 0]
    dy = cells[:, None, 1] - cells[None, :, 1]
    dz = (cells[:, None, 2] - cells[None, :, 2]) * g.q
    r2 = dx * dx + dy * dy + dz * dz
    with np.errstate(divide="ignore"):
        H = 1.0 / np.sqrt(r2)
    H[r2 == 0] = h000
    phi = (G / g.l_xy) * (H @ rho.ravel())
    return phi.reshape(g.shape)


def potential_at(rho: np.ndarray, g: Geometry, G: float, h000: float, cells) -> np.ndarray:
    """Eq. (eq:poisson) evaluated at selected cells only, as the plain sum over
    the occupied cells of rho (any grid size): Phi[a] = G/l_xy sum rho H."""
    occ = np.nonzero(rho)
    w = rho[occ]
    cz, cy, cx = (np.asarray(c, dtype=np.float64) for c in occ)
    out = np.empty(len(cells))
    for n, (k, j, i) in enumerate(cells):
        dx = cx - i
        dy = cy - j
        dz = (cz - k) * g.q
        r2 = dx * dx + dy * dy + dz * dz
        with np.errstate(divide="ignore"):
            H = np.where(r2 > 0, 1.0 / np.sqrt(np.where(r2 > 0, r2, 1.0)), h000)
        out[n] = (G / g.l_xy) * np.sum(w * H)
    return out


def solve_all(rho, system: System, s: int):
    """Phi[g][k] for every mass set."""
    out = []
    for g, gal in enumerate(system.galaxies):
        per = {}
        for k, geom, _, _ in mass_sets(gal):
            per[k] = potential_fft(rho_real(rho[g][k], s), geom, system.G, system.h000)
        out.append(per)
    return out


# ---------------------------------------------------------------------------
# Forces: Eq. (eqn:diff) and the potential combination rule (Sec. 2.1)
# ---------------------------------------------------------------------------

def _cell_and_delta(pos, centre, g: Geometry, split: bool = False):
    (a, b, c), ok = grid_cells(pos, centre, g, split)
    delta = np.stack([
        (pos[0] - centre[0]) - (a - g.nx // 2) * g.l_xy,
        (pos[1] - centre[1]) - (b - g.ny // 2) * g.l_xy,
        (pos[2] - centre[2]) - (c - g.nz // 2) * g.l_z,
    ])
    return (a, b, c), delta, ok


def accel_from_grid(phi: np.ndarray, g: Geometry, i, j, k, delta) -> np.ndarray:
    """Eq. (eqn:diff): central difference plus first-order Taylor terms, for
    all three components (a_y, a_z by cyclic permutation), cell lengths
    l_x = l_y = l_xy and l_z (Sec. 2.2.2)."""
    P = lambda di, dj, dk: phi[k + dk, j + dj, i + di]  # noqa: E731  layout [z][y][x]
    lx = ly = g.l_xy
    lz = g.l_z
    dx, dy, dz = delta
    c = P(0, 0, 0)
    ax = ((P(1, 0, 0) - P(-1, 0, 0)) / (2 * lx)
          + (P(1, 0, 0) + P(-1, 0, 0) - 2 * c) / lx**2 * dx
          + (P(1, 1, 0) - P(-1, 1, 0) + P(-1, -1, 0) - P(1, -1, 0)) / (4 * lx * ly) * dy
          + (P(1, 0, 1) - P(-1, 0, 1) + P(-1, 0, -1) - P(1, 0, -1)) / (4 * lx * lz) * dz)
    ay = ((P(0, 1, 0) - P(0, -1, 0)) / (2 * ly)
          + (P(0, 1, 0) + P(0, -1, 0) - 2 * c) / ly**2 * dy
          + (P(0, 1, 1) - P(0, -1, 1) + P(0, -1, -1) - P(0, 1, -1)) / (4 * ly * lz) * dz
          + (P(1, 1, 0) - P(1, -1, 0) + P(-1, -1, 0) - P(-1, 1, 0)) / (4 * ly * lx) * dx)
    az = ((P(0, 0, 1) - P(0, 0, -1)) / (2 * lz)
          + (P(0, 0, 1) + P(0, 0, -1) - 2 * c) / lz**2 * dz
          + (P(1, 0, 1) - P(1, 0, -1) + P(-1, 0, -1) - P(-1, 0, 1)) / (4 * lz * lx) * dx
          + (P(0, 1, 1) - P(0, 1, -1) + P(0, -1, -1) - P(0, -1, 1)) / (4 * lz * ly) * dy)
    return np.stack([ax, ay, az])


def phi_at_particle(phi: np.ndarray, g: Geometry, i, j, k, delta) -> np.ndarray:
    """Potential at the particle: cell value plus the first-order Taylor term
    with the central-difference gradient (used only for the energy)."""
    P = lambda di, dj, dk: phi[k + dk, j + dj, i + di]  # noqa: E731
    return (P(0, 0, 0)
            + (P(1, 0, 0) - P(-1, 0, 0)) / (2 * g.l_xy) * delta[0]
            + (P(0, 1, 0) - P(0, -1, 0)) / (2 * g.l_xy) * delta[1]
            + (P(0, 0, 1) - P(0, 0, -1)) / (2 * g.l_z) * delta[2])


def combination(reg: int):
    """Grids whose potentials are summed for a field point in a region of one
    galaxy (Sec. 2.1): core 1+3+5, shell 2+3+5, outside 4+5."""
    return {REGION_CORE: (1, 3, 5), REGION_SHELL: (2, 3, 5), REGION_OUTER: (4, 5)}[reg]


def accelerations(state: State, system: System, phi, flags, with_phi=False):
    """Acceleration (and optionally potential) of every live particle, summed
    over galaxies by the combination rule; lost particles get zero."""
    n = len(state.m)
    acc = np.zeros((3, n))
    pot = np.zeros(n)
    live = (flags & FLAG_LOST) == 0
    pos = state.pos
    for h, gal in enumerate(system.galaxies):
        reg = region(pos, gal, state.centres[h], system.split)
        sets = {k: (geom, ck) for k, geom, ck, _ in mass_sets(gal)}
        for r in (REGION_CORE, REGION_SHELL, REGION_OUTER):
            sel = live & (reg == r)
            if not np.any(sel):
                continue
            for k in combination(r):
                if k not in sets:
                    continue
                geom, ck = sets[k]
                centre = state.centres[h] if ck == "gal" else system.sys_centre
                (a, b, c), delta, ok = _cell_and_delta(pos[:, sel], centre, geom, system.split)
                assert ok.all(), "field point outside the grid chosen for it"
                acc[:, sel] += accel_from_grid(phi[h][k], geom, a, b, c, delta)
                if with_phi:
                    pot[sel] += phi_at_particle(phi[h][k], geom, a, b, c, delta)
    return (acc, pot) if with_phi else acc


# ---------------------------------------------------------------------------
# Leap-frog (Sec. 2.1), recentring (Sec. 2.1), one full step
# ---------------------------------------------------------------------------

def kick(vel, acc, dt, live):
    """v(t + dt/2) = v(t - dt/2) + dt a(t)."""
    return np.where(live, vel + dt * acc, vel)


def drift(pos, vel, dt, live):
    """x(t + dt) = x(t) + dt v(t + dt/2)."""
    return np.where(live, pos + dt * vel, pos)


def recentre_sums(state: State, system: System) -> np.ndarray:
    """Integer sums of the centre of mass of each recentred galaxy's live
    particles within R_core of its current centre: per galaxy
    (sum w, sum w D_x, sum w D_y, sum w D_z) with weights w = q >> 26 (q the
    deposit's fixed-point mass) and offsets D = rint(d 2^sD), |d| < R_core <=
    2^(24 - sD).  Integer sums do not depend on order, so the sums of
    disjoint parts of the particles add up to the sums of all of them.
    Returns an int64 array (ngal, 4); zeros for galaxies not recentred."""
    s = fixed_shift(system.mass_bound)
    q = quantize_mass(state.m, s) >> 26
    out = np.zeros((len(system.galaxies), 4), dtype=np.int64)
    live = (state.flags & FLAG_LOST) == 0
    for g, gal in enumerate(system.galaxies):
        if not gal.recentre or gal.r_core <= 0:
            continue
        sD = _offset_shift(gal.r_core)
        sel = live & (state.gal == g)
        d = [offset_f32(state.pos[k, sel], state.centres[g, k], system.split) for k in range(3)]
        inside = r2_f32(*d) < np.float32(gal.r_core * gal.r_core)
        w = q[sel][inside]
        out[g, 0] = int(w.sum())
        for k in range(3):
            D = np.rint(np.ldexp(d[k][inside].astype(np.float64), sD)).astype(np.int64)
            out[g, 1 + k] = int((w * D).sum())
    return out


def _offset_shift(r_core: float) -> int:
    """sD = 24 - ceil(log2 R_core): offsets below R_core times 2^sD stay
    below 2^24."""
    f, e = math.frexp(r_core)
    return 24 - (e - 1 if f == 0.5 else e)


def recentre_apply(centres: np.ndarray, sums: np.ndarray, system: System) -> np.ndarray:
    """New centres c + (sum w D / sum w) 2^-sD for every galaxy whose summed
    weight is positive; the others keep theirs."""
    new = np.array(centres, dtype=np.float64, copy=True)
    for g, gal in enumerate(system.galaxies):
        M = int(sums[g, 0])
        if not gal.recentre or gal.r_core <= 0 or M <= 0:
            continue
        sD = _offset_shift(gal.r_core)
        for k in range(3):
            new[g, k] = centres[g, k] + math.ldexp(float(int(sums[g, 1 + k])) / float(M), -sD)
    return new


def recentre(state: State, system: System) -> np.ndarray:
    """New centres of grids 1-3 (Sec. 2.1, the centre of mass as the stated
    alternative to the density maximum): centre of mass of each recentred
    galaxy's live particles within R_core of its current centre, from the
    exact integer sums of recentre_sums."""
    return recentre_apply(state.centres, recentre_sums(state, system), system)


def step(state: State, system: System, dt: float) -> State:
    """One nested-grid step: recentre, classify, deposit, solve every mass set,
    force by the combination rule, kick and drift (Sec. 2.1)."""
    st = state.copy()
    st.centres = recentre(st, system)
    flags, own = classify(st, system)
    rho, flags, s = deposit(st, system, flags, own)
    phi = solve_all(rho, system, s)
    acc = accelerations(st, system, phi, flags)
    live = (flags & FLAG_LOST) == 0
    st.vel = kick(st.vel, acc, dt, live)
    st.pos = drift(st.pos, st.vel, dt, live)
    st.flags = flags
    return st


def diagnostics(state: State, system: System, dt: float):
    """Energy and angular momentum at the synchronised time t of a state that
    holds v(t - dt/2): v(t) = v(t - dt/2) + dt/2 a(t); K = sum m v^2 / 2,
    W = -1/2 sum m Phi(x), L = sum m x cross v (live particles; Sec. 6.4
    quantities).  Returns dict with K, W, E, L (3,), n_live."""
    flags, own = classify(state, system)
    rho, flags, s = deposit(state, system, flags, own)
    phi = solve_all(rho, system, s)
    acc, pot = accelerations(state, system, phi, flags, with_phi=True)
    live = (flags & FLAG_LOST) == 0
    v = state.vel + 0.5 * dt * acc
    m = np.where(live, state.m, 0.0)
    K = 0.5 * float(np.sum(m * np.sum(v * v, axis=0)))
    W = -0.5 * float(np.sum(m * pot))
    L = np.sum(m * np.cross(state.pos.T, v.T).T, axis=1)
    return {"K": K, "W": W, "E": K + W, "L": L, "n_live": int(live.sum())}


def half_kick_start(state: State, system: System, dt: float) -> State:
    """Leap-frog start: v(-dt/2) = v(0) - dt/2 a(0) (positions unchanged)."""
    st = state.copy()
    flags, own = classify(st, system)
    rho, flags, s = deposit(st, system, flags, own)
    phi = solve_all(rho, system, s)
    acc = accelerations(st, system, phi, flags)
    st.vel = kick(st.vel, acc, -0.5 * dt, (flags & FLAG_LOST) == 0)
    st.flags = flags
    return st
