"""ctypes binding of libpm (include/pm.h): argument marshalling only.

Every step of the particle-mesh path runs in the library's CUDA kernels; this
module only turns Python/PyTorch objects into the C structs and pointers the
C ABI takes.  There is no fallback: if libpm.so is missing, importing the
library raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpm.so")

PM_OK, PM_E_ARG, PM_E_QCRIT, PM_E_NESTING, PM_E_OVERFLOW, PM_E_CUDA, PM_E_STATE = 0, -1, -2, -3, -4, -5, -6
PM_E_TIMEOUT = -7
PM_FP32, PM_FP64 = 1, 2
PM_FLAG_LOST = 1
PM_MAX_GALAXIES = 8

# Names declared in include/pm.h, with (restype, argtypes).
_vp = C.c_void_p
_SIGS = {}


class pm_geometry(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("l_xy", C.c_double), ("l_z", C.c_double)]


class pm_galaxy(C.Structure):
    _fields_ = [("coarse", pm_geometry), ("medium", pm_geometry), ("fine", pm_geometry),
                ("r_core", C.c_double), ("r_out", C.c_double),
                ("centre", C.c_double * 3), ("recentre", C.c_int32)]


class pm_system(C.Structure):
    _fields_ = [("precision", C.c_int32), ("ngal", C.c_int32),
                ("G", C.c_double), ("h000", C.c_double), ("r_sys", C.c_double),
                ("sys_centre", C.c_double * 3), ("mass_bound", C.c_double)]


class pm_particles(C.Structure):
    _fields_ = [("x", _vp), ("y", _vp), ("z", _vp), ("vx", _vp), ("vy", _vp), ("vz", _vp),
                ("m", _vp), ("gal", _vp), ("flags", _vp), ("n", C.c_int64)]


class pm_disc_query(C.Structure):
    _fields_ = [("gal", C.c_int32), ("nbins", C.c_int32), ("nring", C.c_int32), ("mmax", C.c_int32),
                ("r_ring", C.c_double), ("r0", C.c_double), ("dr", C.c_double)]


_P = C.POINTER
_SIGS.update({
    "pm_cell_length": (C.c_double, [C.c_double, C.c_int32, C.c_double]),
    "pm_q_crit": (C.c_double, [C.c_double, C.c_double, C.c_double, C.c_int32]),
    "pm_fixed_shift": (C.c_int32, [C.c_double]),
    "pm_last_error": (C.c_char_p, []),
    "pm_create_grids": (C.c_int, [_P(pm_system), _P(pm_galaxy), _vp, _P(_vp)]),
    "pm_destroy": (None, [_vp]),
    "pm_set_stream": (C.c_int, [_vp, _vp]),
    "pm_recentre": (C.c_int, [_vp, _P(pm_particles)]),
    "pm_deposit": (C.c_int, [_vp, _P(pm_particles)]),
    "pm_solve": (C.c_int, [_vp]),
    "pm_force": (C.c_int, [_vp, _P(pm_particles), _vp, _vp, _vp]),
    "pm_kick": (C.c_int, [_vp, _P(pm_particles), C.c_double]),
    "pm_step": (C.c_int, [_vp, _P(pm_particles), C.c_double, C.c_int32]),
    "pm_diagnostics": (C.c_int, [_vp, _P(pm_particles), C.c_double, _P(C.c_double)]),
    "pm_get_density": (C.c_int, [_vp, C.c_int32, C.c_int32, _vp]),
    "pm_get_potential": (C.c_int, [_vp, C.c_int32, C.c_int32, _vp]),
    "pm_get_centres": (C.c_int, [_vp, _P(C.c_double)]),
    "pm_set_centres": (C.c_int, [_vp, _P(C.c_double)]),
    "pm_count_lost": (C.c_int, [_vp, _P(pm_particles), _P(C.c_int64)]),
    "pm_info": (C.c_int, [_vp, _P(C.c_int64)]),
    "pm_set_launch_config": (C.c_int, [_vp, C.c_int32, C.c_int32]),
    "pm_step_timed": (C.c_int, [_vp, _P(pm_particles), C.c_double, C.c_int32, _P(C.c_float)]),
    "pm_sort": (C.c_int, [_vp, _P(pm_particles), _vp]),
    "pm_set_sort_interval": (C.c_int, [_vp, C.c_int32]),
    "pm_potential_static": (C.c_int, [_vp, _vp, C.c_int32, C.c_int32, C.c_int32, C.c_double, C.c_double,
                                      C.c_double, C.c_double, C.c_int32, C.c_int32, _vp]),
    "pm_potential_static_status": (C.c_int, [_vp]),
    "pm_static_selftest_wait_expiry": (C.c_int, [_vp, C.c_int64, C.c_int32, _vp]),
    "pm_disc_diagnostics": (C.c_int, [_vp, _P(pm_particles), _vp, _P(pm_disc_query), _P(C.c_double)]),
    "pm_cic_deposit": (C.c_int, [_vp, _P(pm_particles)]),
    "pm_cic_force": (C.c_int, [_vp, _P(pm_particles), _vp, _vp, _vp]),
    "pm_cic_kick_drift": (C.c_int, [_vp, _P(pm_particles), C.c_double, C.c_double]),
    "pm_cic_vjp": (C.c_int, [_vp, _P(pm_particles), _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "pm_selftest_wait_expiry": (C.c_int, [_vp]),
    "pm_recentre_sums": (C.c_int, [_vp, _P(pm_particles)]),
    "pm_recentre_apply": (C.c_int, [_vp]),
    "pm_exchange_buffers": (C.c_int, [_vp, _P(_vp), _P(C.c_int64), _P(_vp), _P(C.c_int64)]),
    "pm_kick_drift": (C.c_int, [_vp, _P(pm_particles), C.c_double]),
})

_lib = None


def lib():
    """The loaded libpm.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libpm.so not found at {LIB_PATH}: build it with "
                              "`python -m paper_1210_1736_gb300.build` (no CPU fallback exists)")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class PMError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"pm error {code}: {msg}")
        self.code = code


def _check(rc):
    if rc != PM_OK:
        raise PMError(rc, lib().pm_last_error().decode())
    return rc


def cell_length(R, N, q=1.0):
    return lib().pm_cell_length(float(R), int(N), float(q))


def q_crit(r_core, r_out, r_sys, N):
    return lib().pm_q_crit(float(r_core), float(r_out), float(r_sys), int(N))


def fixed_shift(mass_bound):
    return lib().pm_fixed_shift(float(mass_bound))


def geometry(spec):
    """(nx, ny, nz, R, q) -> pm_geometry with l_xy = 2R/(nx-4), l_z = q l_xy;
    None -> absent geometry."""
    g = pm_geometry()
    if spec is None:
        return g
    nx, ny, nz, R, q = spec
    g.nx, g.ny, g.nz = int(nx), int(ny), int(nz)
    g.l_xy = cell_length(R, nx, 1.0)
    g.l_z = float(q) * g.l_xy
    return g


def describe(workload, mass_bound):
    """pm_system and pm_galaxy[] of a workload dict (see workloads.py)."""
    gals = (pm_galaxy * PM_MAX_GALAXIES)()
    for i, g in enumerate(workload["galaxies"]):
        gals[i].coarse = geometry(g["coarse"])
        gals[i].medium = geometry(g.get("medium"))
        gals[i].fine = geometry(g.get("fine"))
        gals[i].r_core = float(g["r_core"])
        gals[i].r_out = float(g["r_out"])
        for k in range(3):
            gals[i].centre[k] = float(g["centre"][k])
        gals[i].recentre = 1 if g["recentre"] else 0
    s = workload["system"]
    sysd = pm_system()
    sysd.precision = PM_FP32 if workload["precision"] == "fp32" else PM_FP64
    sysd.ngal = len(workload["galaxies"])
    sysd.G = float(s["G"])
    sysd.h000 = float(s["h000"])
    sysd.r_sys = float(s["r_sys"])
    for k in range(3):
        sysd.sys_centre[k] = float(s["sys_centre"][k])
    sysd.mass_bound = float(mass_bound)
    return sysd, gals


class Particles:
    """Device-resident structure-of-arrays particle set (torch tensors)."""

    def __init__(self, pos, vel, m, gal, precision="fp32", device="cuda"):
        import torch
        dt = torch.float32 if precision == "fp32" else torch.float64
        self.dtype = dt
        pos = np.asarray(pos)
        vel = np.asarray(vel)
        self.x, self.y, self.z = (torch.as_tensor(np.ascontiguousarray(pos[k]), dtype=dt).to(device) for k in range(3))
        self.vx, self.vy, self.vz = (torch.as_tensor(np.ascontiguousarray(vel[k]), dtype=dt).to(device) for k in range(3))
        self.m = torch.as_tensor(np.ascontiguousarray(m), dtype=dt).to(device)
        self.gal = torch.as_tensor(np.ascontiguousarray(gal), dtype=torch.int32).to(device)
        self.flags = torch.zeros(len(self.m), dtype=torch.int32, device=device)
        self.n = len(self.m)

    @classmethod
    def from_tensors(cls, pos, vel, m, gal, flags=None):
        """Wraps device tensors without copying: pos and vel (3, n) contiguous,
        m (n,), gal int32 (n,), flags int32 (n,) (zeros if None)."""
        import torch
        self = cls.__new__(cls)
        self.dtype = pos.dtype
        self.x, self.y, self.z = pos[0], pos[1], pos[2]
        self.vx, self.vy, self.vz = vel[0], vel[1], vel[2]
        self.m = m
        self.gal = gal
        self.flags = torch.zeros(m.shape[0], dtype=torch.int32, device=m.device) if flags is None else flags
        self.n = int(m.shape[0])
        for t in (self.x, self.y, self.z, self.vx, self.vy, self.vz, self.m, self.gal, self.flags):
            if not t.is_contiguous():
                raise ValueError("particle arrays must be contiguous")
        return self

    def struct(self):
        p = pm_particles()
        for k in ("x", "y", "z", "vx", "vy", "vz", "m", "gal", "flags"):
            setattr(p, k, getattr(self, k).data_ptr())
        p.n = self.n
        return p

    def host(self):
        import torch  # noqa: F401
        pos = np.stack([t.cpu().numpy().astype(np.float64) for t in (self.x, self.y, self.z)])
        vel = np.stack([t.cpu().numpy().astype(np.float64) for t in (self.vx, self.vy, self.vz)])
        return pos, vel, self.flags.cpu().numpy().astype(np.int64)


class _DeviceArray:
    """An int64 device buffer owned by the library, exposed to torch through
    the CUDA array interface (no copy)."""

    def __init__(self, ptr, n):
        self.__cuda_array_interface__ = {"shape": (int(n),), "typestr": "<i8", "data": (int(ptr), False),
                                         "version": 3, "strides": None}


class Context:
    """One pm_ctx: the grids, H-hat tables and work buffers of a system."""

    def __init__(self, workload, mass_bound, stream=None):
        import torch
        self.workload = workload
        self.sys, self.gals = describe(workload, mass_bound)
        self.precision = workload["precision"]
        self.np_dtype = np.float32 if self.precision == "fp32" else np.float64
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        h = _vp()
        _check(lib().pm_create_grids(C.byref(self.sys), self.gals, _vp(stream), C.byref(h)))
        self.h = h
        self.shapes = {}
        for gi, g in enumerate(workload["galaxies"]):
            specs = {1: g.get("fine"), 2: g.get("medium"), 3: g.get("medium"), 4: g["coarse"], 5: g["coarse"]}
            for k, sp in specs.items():
                if sp is None or (k in (1,) and g.get("medium") is None) or (k == 4 and g.get("medium") is None):
                    continue
                self.shapes[(gi, k)] = (int(sp[2]), int(sp[1]), int(sp[0]))

    def close(self):
        if getattr(self, "h", None):
            lib().pm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream):
        _check(lib().pm_set_stream(self.h, _vp(stream)))

    def recentre(self, p):
        _check(lib().pm_recentre(self.h, C.byref(p.struct())))

    def recentre_sums(self, p):
        _check(lib().pm_recentre_sums(self.h, C.byref(p.struct())))

    def recentre_apply(self):
        _check(lib().pm_recentre_apply(self.h))

    def exchange_buffers(self):
        """(rho, csum): int64 device tensors viewing the context's density
        block and centre-of-mass accumulators, without copying."""
        import torch
        rp, rb, cp, cb = _vp(), C.c_int64(), _vp(), C.c_int64()
        _check(lib().pm_exchange_buffers(self.h, C.byref(rp), C.byref(rb), C.byref(cp), C.byref(cb)))
        dev = torch.cuda.current_device()
        return (torch.as_tensor(_DeviceArray(rp.value, rb.value // 8), device=f"cuda:{dev}"),
                torch.as_tensor(_DeviceArray(cp.value, cb.value // 8), device=f"cuda:{dev}"))

    def kick_drift(self, p, dt):
        _check(lib().pm_kick_drift(self.h, C.byref(p.struct()), float(dt)))

    def deposit(self, p):
        _check(lib().pm_deposit(self.h, C.byref(p.struct())))

    def solve(self):
        _check(lib().pm_solve(self.h))

    def force(self, p):
        import torch
        a = [torch.empty(p.n, dtype=p.dtype, device=p.x.device) for _ in range(3)]
        _check(lib().pm_force(self.h, C.byref(p.struct()), a[0].data_ptr(), a[1].data_ptr(), a[2].data_ptr()))
        return a

    def kick(self, p, dt):
        _check(lib().pm_kick(self.h, C.byref(p.struct()), float(dt)))

    # CIC variant (differentiable runs; see include/pm.h)
    def cic_deposit(self, p):
        _check(lib().pm_cic_deposit(self.h, C.byref(p.struct())))

    def cic_force(self, p):
        import torch
        a = [torch.empty(p.n, dtype=p.dtype, device=p.x.device) for _ in range(3)]
        _check(lib().pm_cic_force(self.h, C.byref(p.struct()), a[0].data_ptr(), a[1].data_ptr(), a[2].data_ptr()))
        return a

    def cic_kick_drift(self, p, dt_kick, dt_drift):
        _check(lib().pm_cic_kick_drift(self.h, C.byref(p.struct()), float(dt_kick), float(dt_drift)))

    def cic_vjp(self, p, u, gx, gm):
        """Adds u^T da/dx to gx (3, n) and u^T da/dm to gm (n,) (device
        tensors of the context precision); u is (3, n)."""
        for t in (u, gx, gm):
            if not t.is_contiguous() or t.dtype != p.dtype:
                raise ValueError("cotangent and gradient tensors must be contiguous, context precision")
        _check(lib().pm_cic_vjp(self.h, C.byref(p.struct()), u[0].data_ptr(), u[1].data_ptr(), u[2].data_ptr(),
                                gx[0].data_ptr(), gx[1].data_ptr(), gx[2].data_ptr(), gm.data_ptr()))

    def step(self, p, dt, nsteps=1):
        _check(lib().pm_step(self.h, C.byref(p.struct()), float(dt), int(nsteps)))

    def sort(self, p, perm=None):
        """Spatially sort p's arrays in place; perm (int64 device tensor of
        length n, optional) receives perm[new] = old."""
        _check(lib().pm_sort(self.h, C.byref(p.struct()), None if perm is None else perm.data_ptr()))

    def set_sort_interval(self, k):
        _check(lib().pm_set_sort_interval(self.h, int(k)))

    def step_timed(self, p, dt, nsteps=1):
        out = (C.c_float * 10)()
        _check(lib().pm_step_timed(self.h, C.byref(p.struct()), float(dt), int(nsteps), out))
        return list(out)

    def diagnostics(self, p, dt):
        out = (C.c_double * 8)()
        _check(lib().pm_diagnostics(self.h, C.byref(p.struct()), float(dt), out))
        return {"K": out[0], "W": out[1], "E": out[2], "L": np.array(out[3:6]), "n_live": int(out[6])}

    def disc_diagnostics(self, p, select=None, gal=0, nbins=20, nring=10, mmax=4, r_ring=5.0, r0=3.2, dr=0.4):
        """Sec. 6 disc quantities (see pm_disc_diagnostics in include/pm.h);
        select: device uint8/bool tensor (nonzero = take) or None for every
        particle of galaxy `gal`.  Returns a dict of numpy values."""
        q = pm_disc_query(int(gal), int(nbins), int(nring), int(mmax), float(r_ring), float(r0), float(dr))
        nout = 6 + 4 * nbins + 2 * nring * mmax
        out = (C.c_double * nout)()
        sp = None
        if select is not None:
            import torch
            sel = select.to(torch.uint8).contiguous()
            sp = sel.data_ptr()
        _check(lib().pm_disc_diagnostics(self.h, C.byref(p.struct()), sp, C.byref(q), out))
        a = np.array(out)
        bins = a[6:6 + 4 * nbins].reshape(nbins, 4)
        A = a[6 + 4 * nbins:].reshape(nring, mmax, 2)
        sR, sphi, sz = a[2], a[3], a[4]
        return {"raw": a, "n": int(a[0]), "E_heat": a[1], "sigma_R": sR, "sigma_phi": sphi, "sigma_z": sz,
                "sigma_z_over_R": sz / sR if sR > 0 else float("nan"), "sigma_tot2": sR ** 2 + sphi ** 2 + sz ** 2,
                "annulus_mass": a[5], "R_mean": bins[:, 0], "count": bins[:, 1], "z_rms": bins[:, 2],
                "v_c": bins[:, 3], "A": A[..., 0] + 1j * A[..., 1]}

    def density(self, gal, k):
        a = np.empty(self.shapes[(gal, k)], dtype=np.int64)
        _check(lib().pm_get_density(self.h, gal, k, a.ctypes.data))
        return a

    def potential(self, gal, k):
        a = np.empty(self.shapes[(gal, k)], dtype=self.np_dtype)
        _check(lib().pm_get_potential(self.h, gal, k, a.ctypes.data))
        return a

    def centres(self):
        n = self.sys.ngal
        out = (C.c_double * (3 * n))()
        _check(lib().pm_get_centres(self.h, out))
        return np.array(out).reshape(n, 3)

    def set_centres(self, c):
        c = np.ascontiguousarray(np.asarray(c, dtype=np.float64).ravel())
        _check(lib().pm_set_centres(self.h, c.ctypes.data_as(_P(C.c_double))))

    def count_lost(self, p):
        out = C.c_int64()
        _check(lib().pm_count_lost(self.h, C.byref(p.struct()), C.byref(out)))
        return out.value

    def selftest_wait_expiry(self):
        """Status of the bounded-wait self-test (PM_E_TIMEOUT is the expected
        result: the wait gave up and the host saw it); see include/pm.h."""
        return int(lib().pm_selftest_wait_expiry(self.h))

    def set_launch_config(self, batched, schedule):
        """The solve's launch grouping (batched 1/0) and branch schedule
        (0/1) in place of the ones timed fastest at creation."""
        _check(lib().pm_set_launch_config(self.h, int(batched), int(schedule)))

    def info(self):
        out = (C.c_int64 * 6)()
        _check(lib().pm_info(self.h, out))
        return {"shift": out[0], "nsets": out[1], "ngeom": out[2], "bytes": out[3], "solve_schedule": out[4],
                "batched": out[5]}
