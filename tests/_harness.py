"""Shared helpers of the parity tests: run one workload through the library
(C ABI via the ctypes binding) and through the oracle on identical inputs."""
from __future__ import annotations

import numpy as np

import oracle as O
from paper_1210_1736_gb300 import pm


def require_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch


def cast(w, a):
    dt = np.float32 if w["precision"] == "fp32" else np.float64
    return np.asarray(a).astype(dt)


def gpu_setup(w, pos=None, vel=None, m=None, gal=None):
    """Context + device particles holding exactly the oracle's numbers."""
    require_cuda()
    pos = w["pos"] if pos is None else pos
    vel = w["vel"] if vel is None else vel
    m = w["m"] if m is None else m
    gal = w["gal"] if gal is None else gal
    # the same bound goes to both sides (it fixes the fixed-point scale)
    mb = O.mass_bound(cast(w, m))
    ctx = pm.Context(w, mb)
    parts = pm.Particles(cast(w, pos), cast(w, vel), cast(w, m), gal, precision=w["precision"])
    return ctx, parts


def oracle_setup(w, pos=None, vel=None, m=None, gal=None):
    pos = w["pos"] if pos is None else pos
    vel = w["vel"] if vel is None else vel
    m = w["m"] if m is None else m
    ww = dict(w)
    ww["m"] = cast(w, m)
    if gal is not None:
        ww["gal"] = gal
    system = O.system_from_workload(ww, O.mass_bound(ww["m"]))
    state = O.state_from_workload(ww, pos=pos, vel=vel, m=m)
    return system, state


def oracle_fields(system, state):
    flags, own = O.classify(state, system)
    rho, flags, s = O.deposit(state, system, flags, own)
    phi = O.solve_all(rho, system, s)
    return rho, phi, flags, own, s


def rel_force_errors(a_gpu, a_ref, live):
    d = (a_gpu - a_ref)[:, live]
    ref = a_ref[:, live]
    rms_ref = np.sqrt(np.mean(np.sum(ref * ref, axis=0)))
    rms = np.sqrt(np.mean(np.sum(d * d, axis=0))) / rms_ref
    mx = np.max(np.sqrt(np.sum(d * d, axis=0))) / rms_ref
    print(f"force error: rms {rms:.3e} max {mx:.3e} (RMS-normalised, {d.shape[1]} particles)")
    return rms, mx
