"""Plain FP64 CPU reference of the nested-grid particle-mesh step.

TEST INFRASTRUCTURE: imported only by tests/, the smoke check and the
benchmark's CPU-baseline leg; the product path never imports it.
"""
from .pm_oracle import *  # noqa: F401,F403
from .pm_cic import *  # noqa: F401,F403
from .pm_diag import *  # noqa: F401,F403
from .pm_oracle import Geometry, Galaxy, System, State, cell_length, mass_bound
import numpy as np


def geometry_from_spec(spec):
    """(nx, ny, nz, R, q) -> Geometry with l_xy = 2R/(nx-4), l_z = q l_xy."""
    if spec is None:
        return None
    nx, ny, nz, R, q = spec
    l_xy = cell_length(R, nx)
    return Geometry(nx, ny, nz, l_xy, q * l_xy)


def system_from_workload(w, mb=None):
    """System of a workload dict; mb: the mass bound (default: the oracle's
    own sum |m| of the workload's masses)."""
    gals = []
    for g in w["galaxies"]:
        gals.append(Galaxy(coarse=geometry_from_spec(g["coarse"]),
                           medium=geometry_from_spec(g.get("medium")),
                           fine=geometry_from_spec(g.get("fine")),
                           r_core=g["r_core"], r_out=g["r_out"],
                           centre=tuple(g["centre"]), recentre=bool(g["recentre"])))
    s = w["system"]
    return System(galaxies=gals, r_sys=s["r_sys"], sys_centre=tuple(s["sys_centre"]),
                  G=s["G"], h000=s["h000"], mass_bound=mass_bound(w["m"]) if mb is None else float(mb),
                  precision=w.get("precision", "fp64"))


def state_from_workload(w, pos=None, vel=None, m=None):
    """FP64 state holding exactly the values the path sees (cast through the
    path precision first, so both sides start from identical numbers)."""
    dt = np.float32 if w["precision"] == "fp32" else np.float64
    pos = np.asarray(w["pos"] if pos is None else pos).astype(dt).astype(np.float64)
    vel = np.asarray(w["vel"] if vel is None else vel).astype(dt).astype(np.float64)
    m = np.asarray(w["m"] if m is None else m).astype(dt).astype(np.float64)
    n = pos.shape[1]
    cents = np.array([g["centre"] for g in w["galaxies"]], dtype=np.float64)
    return State(pos=pos, vel=vel, m=m, gal=np.asarray(w["gal"]).astype(np.int64),
                 flags=np.zeros(n, dtype=np.int64), centres=cents)
