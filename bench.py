#!/usr/bin/env python
"""Benchmark of the nested-grid particle-mesh step (Superbox-10) on GB300.

One step = recentre + deposit + (x, y, z-convolve, y, x) FFT passes on every
grid + force/kick-drift, FP32 with int64 fixed-point density.  The default
workload is the largest: a 16M-particle disc-bulge-halo galaxy on 256^3,
256^3 (q = 1/4) and 256x256x64 grids plus two 250k-particle satellites with
128^3 grids.  The same line reports the 1M-particle galaxy and the 4M-particle
merger (extra_workloads).  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 (torchrun): every rank steps its own independent galaxy (weak scaling,
no collective on the data path); rank 0 prints.  --impl reference times the
FP64 CPU oracle (the only reference this method has) on the host cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-steps/s per nested-grid step; FFT-convolve GB/s vs HBM peak"
UNIT = "particle-steps/s"
WORKLOAD = "large_16m"
EXTRA_WORKLOADS = ("galaxy_1m", "merger_4m")
WORKLOAD_DESC = {
    "galaxy_1m": "galaxy_1m: 1M particles (400k exp. disc, 100k Hernquist bulge, 500k truncated NFW halo); "
                 "grids coarse 128^3, medium 128^3 q=1/4, fine 128x128x32; dt=0.01",
    "merger_4m": "merger_4m: 4M-particle galaxy + 100k Plummer satellite; galaxy grids 128^3, 128^3 q=1/4, "
                 "256x256x32; satellite grids 64^3 x 3; dt=0.01",
    "large_16m": "large_16m: 16M-particle galaxy + two 250k Plummer satellites; galaxy grids 256^3, 256^3 q=1/4, "
                 "256x256x64; satellite grids 128^3 x 3 each; dt=0.01",
    "galaxy_256": "galaxy_256: 2M-particle galaxy on the large run's grids 256^3, 256^3 q=1/4, 256x256x64; dt=0.01 "
                  "(profiling size)",
}
PHASES = ["recentre", "deposit", "fft_x_fwd", "fft_y_fwd", "fft_z_conv", "fft_y_inv", "fft_x_inv", "force_kick_drift"]
SORT_PHASE = 9


def env_rank():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))


def slowest_rank_ms(ms, world, device):
    """The job's time is its slowest rank's: the maximum over ranks of a
    per-rank time in ms (all ranks call it; device: where the process group's
    backend takes tensors, "cuda" for NCCL, "cpu" for gloo)."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world, n, steps, ms):
    """Whole-job particle-steps/s: every rank advances its own n particles
    for `steps` steps (weak scaling) in the job time ms."""
    return world * n * steps / (ms / 1e3)


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_source_hash():
    """Hash of the kernel sources' code: comments and whitespace are left
    out, so that only a change of the compiled code invalidates counters
    stored against it."""
    import re
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1210_1736_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        if f.endswith((".cu", ".cuh", ".h")):
            text = open(os.path.join(csrc, f), encoding="utf-8").read()
            text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
            text = re.sub(r"//[^\n]*", " ", text)
            h.update(f.encode() + b"\0" + " ".join(text.split()).encode())
    return h.hexdigest()[:16]


def ncu_traffic(phase, workload):
    """DRAM bytes per step of a phase from the committed ncu summary, if it
    was taken on the current kernel sources and this workload (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    if d.get("source_hash") != kernel_source_hash() or d.get("workload") != workload:
        return None
    return d.get("phases", {}).get(phase)


def fp64_comparison(w, host, m32, n_steps):
    """The same workload through the FP64 instantiation of the same kernels:
    its step time, and the FP32 path's force error against it at the
    initial state (FP64 forces match the oracle to ~1e-14)."""
    import torch
    from paper_1210_1736_gb300 import pm
    from paper_1210_1736_gb300.workloads import mass_bound
    dt = w["dt"]
    mb = mass_bound(m32)
    w32 = dict(w, precision="fp32")
    w64 = dict(w, precision="fp64")
    ctx32 = pm.Context(w32, mb)
    p32 = pm.Particles(host["pos"], host["vel"], m32, w["gal"])
    ctx32.deposit(p32)
    ctx32.solve()
    a32 = [a.double() for a in ctx32.force(p32)]
    ctx32.close()
    del p32
    ctx64 = pm.Context(w64, mb)
    p64 = pm.Particles(host["pos"].astype(np.float64), host["vel"].astype(np.float64),
                       m32.astype(np.float64), w["gal"], precision="fp64")
    ctx64.deposit(p64)
    ctx64.solve()
    a64 = ctx64.force(p64)
    torch.cuda.synchronize()
    live = (p64.flags & 1) == 0
    d2 = sum(((x - y)[live] ** 2) for x, y in zip(a32, a64))
    f2 = sum((y[live] ** 2) for y in a64)
    rms_ref = float(torch.sqrt(f2.mean()))
    rms = float(torch.sqrt(d2.mean())) / rms_ref
    mx = float(torch.sqrt(d2.max())) / rms_ref
    # where the largest errors sit: per galaxy
    gal = torch.as_tensor(w["gal"], device=d2.device)[live]
    by_gal = {}
    for g in range(len(w["galaxies"])):
        sel = gal == g
        if bool(sel.any()):
            by_gal[str(g)] = {"rms": float(torch.sqrt(d2[sel].mean())) / rms_ref,
                              "max": float(torch.sqrt(d2[sel].max())) / rms_ref}
    ctx64.kick(p64, -0.5 * dt)
    ctx64.step(p64, dt, 2)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    ctx64.step(p64, dt, n_steps)
    e1.record()
    torch.cuda.synchronize()
    ms64 = e0.elapsed_time(e1) / n_steps
    ctx64.close()
    del p64, a64, a32
    torch.cuda.empty_cache()
    return {"ms_per_step": ms64, "steps": n_steps, "fp32_force_err_rms": rms, "fp32_force_err_max": mx,
            "fp32_force_err_by_galaxy": by_gal,
            "note": "FP64 build of the same kernels (graph-replayed steps); force errors relative to the "
                    "RMS force over live particles at the initial state (by galaxy: the same measure over "
                    "that galaxy's particles)"}


class Clocks:
    """nvidia-smi clock/throttle sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        time.sleep(0.25)
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = []
        for line in open(self.f.name):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.f.name)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for _, _, r in rows for n, v in zip(names, r) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def phase_bytes(w, n, esz):
    """Algorithmic HBM bytes per step of each phase (byte model): spectra are
    complex of 2*esz bytes; per mass set A = nx ny nz, S1 = (nx+1) ny nz,
    S2 = (nx+1) 2ny nz; H-hat read once per geometry launch.  Grid 1 (the
    fine grid, solved for its difference fields) is counted as two real
    fields' chains from the z pass on (z: 4 S2, y inverse: 2 (S2 + S1), x
    inverse: 2 S1 reads and four real fields fx, fy, fz, Phi_1 written),
    below the R2C minimum for the four real fields it produces from one
    spectrum (z: one read and four writes, 5 S2; y inverse: 4 (S2 + S1); x
    inverse: 4 S1 + 4 A), so its fractions are understated, not inflated."""
    cz = 2 * esz
    b = dict.fromkeys(PHASES, 0.0)
    geoms = {}
    A_total = 0
    for g in w["galaxies"]:
        sets = [("coarse", 2 if g.get("medium") else 1)]
        if g.get("medium"):
            sets.append(("medium", 2))
            if g.get("fine"):
                sets.append(("fine", 1))
        for key, count in sets:
            nx, ny, nz = g[key][:3]
            geoms[tuple(g[key])] = (nx, ny, nz)
            A = nx * ny * nz
            S1 = (nx + 1) * ny * nz
            S2 = 2 * S1
            A_total += A * count
            diff = key == "fine"
            b["fft_x_fwd"] += count * (8 * A + cz * S1)
            b["fft_y_fwd"] += count * (cz * S1 + cz * S2)
            b["fft_z_conv"] += count * (2 * cz * S2) * (2 if diff else 1)
            b["fft_y_inv"] += count * (cz * S2 + cz * S1) * (2 if diff else 1)
            b["fft_x_inv"] += count * (cz * S1 * (2 if diff else 1) + esz * A * (4 if diff else 1))
    for nx, ny, nz in geoms.values():
        b["fft_z_conv"] += esz * (nx + 1) * (ny + 1) * (nz + 1)
    b["recentre"] = n * (4 * esz + 8)
    b["deposit"] = n * (4 * esz + 8) + 8 * A_total
    b["force_kick_drift"] = n * (12 * esz + 4)
    b["spatial_sort"] = 0.0
    return b


def phase_hbm_fracs(phase_ms, pb, peak):
    """Each phase's byte-model bytes per step over its time per step, as a
    fraction of the HBM peak (GB/s).  The particle phases count only their
    streamed particle bytes (the gathers and atomics that L2 serves are not
    in the model), so theirs are lower bounds; phases without a byte model
    (the spatial sort) are left out."""
    return {p: pb[p] / (t / 1e3) / 1e9 / peak for p, t in phase_ms.items() if pb.get(p) and t > 0}


def bench_config(w, workload, n, world):
    """The `config` object of the JSON line, identical in both arms."""
    geoms = {tuple(g[k]) for g in w["galaxies"] for k in ("coarse", "medium", "fine") if g.get(k)}
    ws = sum(phase_bytes(w, n, 4).values())
    return {"workload": WORKLOAD_DESC[workload], "particles_per_gpu": n, "galaxies": len(w["galaxies"]),
            "geometries": len(geoms),
            "l2": f"algorithmic bytes per step ~{ws / 1e9:.2f} GB > 129 MB L2 (inputs larger than L2, no flush)",
            "parallelism": f"{world} independent replicas" if world > 1 else "1 GPU"}


def fft_pairs(w):
    """FFT launches per pass: one per pair of mass sets sharing a transform
    (per galaxy: grids 4+5, or 5 alone; grids 2+3; grid 1)."""
    n = 0
    for g in w["galaxies"]:
        n += 1
        if g.get("medium"):
            n += 1
            if g.get("fine"):
                n += 1
    return n


def fused_diff(spec):
    """A fine grid whose two difference-field z products come from one
    forward transform in one launch (z length up to 64, or 128 and 256 with
    the tile's H-hat rows staged: FP32 tile columns 4096 / L <= nx), as the
    library plans it."""
    nx, nz = spec[0], spec[2]
    return nz <= 32 or (nz in (64, 128) and min(4096 // (2 * nz), 256) <= nx)


def fft_launches(w, batched=True):
    """FFT launches per step: the pairs of mass sets of all galaxies are
    grouped by grid shape (nx, ny, nz) and each pass of a shape is one launch
    per 8 pairs; a fine grid (grid 1, solved for its difference fields) adds
    a second work array to the y and x inverse passes and one z pass of its
    own (two where its two products are not fused, see fused_diff)."""
    shapes = {}
    for g in w["galaxies"]:
        pairs = [(g["coarse"], False)]
        if g.get("medium"):
            pairs.append((g["medium"], False))
            if g.get("fine"):
                pairs.append((g["fine"], True))
        for spec, diff in pairs:
            p, d = shapes.get(tuple(spec[:3]), (0, 0))
            shapes[tuple(spec[:3])] = (p + 1, d + int(diff))
    zd = {s: (1 if fused_diff(s) else 2) for s in shapes}   # z launches per batch of fine grids
    if not batched:   # a launch per pair: five passes, two or three more for a fine grid
        return sum(5 * p + (zd[s] + 1) * d for s, (p, d) in shapes.items())
    up = lambda k: (k + 7) // 8  # noqa: E731
    n = 0
    for s, (p, d) in shapes.items():
        n += 2 * up(p)                                   # x and y forward
        n += up(p - d) + (zd[s] * up(d) if d else 0)     # z: plain, then the difference-field pass(es)
        n += 2 * up(p + d)                               # y and x inverse over both work arrays
    return n


def launches(w, steps, sort_every, batched=True):
    """Kernels of `steps` graph steps: recentre and its centre update, deposit,
    the FFT passes (batched or per pair, as the context chose), force/
    kick-drift; every sort_every-th step adds the six kernels of the spatial
    sort."""
    per_step = 2 + 1 + fft_launches(w, batched) + 1
    sorts = (steps + sort_every - 1) // sort_every if sort_every > 0 else 0
    return per_step * steps + 6 * sorts


def request_block_from(parts):
    """One request's particle state as a pinned host block (9, n) float32,
    copied from a device particle set: x, y, z, vx, vy, vz, m, galaxy id and
    flags (the last two as int32), in the set's current (spatially sorted)
    order."""
    import torch
    hbuf = torch.empty((9, parts.n), dtype=torch.float32).pin_memory()
    for k, t in enumerate((parts.x, parts.y, parts.z, parts.vx, parts.vy, parts.vz, parts.m)):
        hbuf[k].copy_(t)
    hbuf[7].view(torch.int32).copy_(parts.gal)
    hbuf[8].view(torch.int32).copy_(parts.flags)
    return hbuf


def request_block(host, m32, gal):
    """One request's particle state as a pinned host block (9, n) float32:
    x, y, z, vx, vy, vz, m, galaxy id and flags (the last two as int32)."""
    import torch
    n = len(m32)
    hbuf = torch.empty((9, n), dtype=torch.float32).pin_memory()
    for k, a in enumerate((host["pos"][0], host["pos"][1], host["pos"][2], host["vel"][0], host["vel"][1],
                           host["vel"][2], m32)):
        hbuf[k].copy_(torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)))
    hbuf[7].view(torch.int32).copy_(torch.from_numpy(np.asarray(gal, dtype=np.int32)))
    hbuf[8].view(torch.int32).zero_()
    return hbuf


class RequestPipeline:
    """One-step requests whose particle state lives in pinned host memory,
    through the C ABI: each request's state goes up as one block, one step
    runs, and the updated positions and velocities (6, n) come back as one
    block.  With overlap the requests rotate over NB device buffers, so the
    upload of request k+1 and the download of request k-1 run on their own
    streams while request k steps (the library keeps the captured step of
    each buffer); a buffer is refilled only after its previous download has
    read it.  Without overlap each request's upload, step and download run in
    sequence on one buffer."""
    NB = 3

    def __init__(self, ctx, hbuf, dt, nout=NB):
        """nout: host result blocks (request k lands in hout[k % nout]; at
        least NB)."""
        import torch
        from paper_1210_1736_gb300 import pm
        self.ctx, self.hbuf, self.dt = ctx, hbuf, dt
        n = hbuf.shape[1]
        self.hout = [torch.empty((6, n), dtype=torch.float32).pin_memory() for _ in range(max(nout, self.NB))]
        self.dbuf = [torch.empty((9, n), dtype=torch.float32, device="cuda") for _ in range(self.NB)]
        self.pe = [pm.Particles.from_tensors(d[0:3], d[3:6], d[6], d[7].view(torch.int32), d[8].view(torch.int32))
                   for d in self.dbuf]
        self.h2d_bytes = hbuf.numel() * hbuf.element_size()
        self.d2h_bytes = self.hout[0].numel() * self.hout[0].element_size()
        self.main = torch.cuda.current_stream()
        self.up, self.down = torch.cuda.Stream(), torch.cuda.Stream()
        self.ev_up = [torch.cuda.Event() for _ in range(self.NB)]
        self.ev_step = [torch.cuda.Event() for _ in range(self.NB)]
        self.ev_down = [torch.cuda.Event() for _ in range(self.NB)]
        self.reset()

    def reset(self):
        """Marks every buffer free (its download events as done)."""
        for e in self.ev_down:
            e.record(self.main)

    def request(self, k, overlap=True):
        """Enqueues request k; returns the index o of the host block hout[o]
        that receives its result (complete once the launching stream has
        passed join())."""
        import torch
        b = k % self.NB if overlap else 0
        o = k % len(self.hout)
        if overlap:
            with torch.cuda.stream(self.up):
                self.up.wait_event(self.ev_down[b])   # request k-NB's download has read dbuf[b]
                self.dbuf[b].copy_(self.hbuf, non_blocking=True)
                self.ev_up[b].record(self.up)
            self.main.wait_event(self.ev_up[b])
            self.ctx.step(self.pe[b], self.dt, 1)
            self.ev_step[b].record(self.main)
            with torch.cuda.stream(self.down):
                self.down.wait_event(self.ev_step[b])
                self.hout[o].copy_(self.dbuf[b][0:6], non_blocking=True)
                self.ev_down[b].record(self.down)
        else:
            self.dbuf[b].copy_(self.hbuf, non_blocking=True)
            self.ctx.step(self.pe[b], self.dt, 1)
            self.hout[o].copy_(self.dbuf[b][0:6], non_blocking=True)
            self.ev_down[b].record(self.main)
        return o

    def join(self):
        """The launching stream waits for every download enqueued so far."""
        for e in self.ev_down:
            self.main.wait_event(e)


def device_phases(ctx, parts, w, n, dt, K):
    """Per-phase device times (the step's kernels launched with CUDA events
    between phases on the launching stream, K steps), the algorithmic bytes
    of each phase, and the convolution span as the step runs it (all
    geometries' pass chains on their branch streams, overlapping)."""
    import torch
    ph = ctx.step_timed(parts, dt, K)
    phase_ms = {p: ph[i] / K for i, p in enumerate(PHASES)}
    phase_ms["spatial_sort"] = ph[SORT_PHASE] / K
    pb = phase_bytes(w, n, 4)
    fft_phases = PHASES[2:7]
    dom = max(PHASES, key=lambda p: phase_ms[p])
    conv_ms = sum(phase_ms[p] for p in fft_phases)
    conv_gbs = sum(pb[p] for p in fft_phases) / (conv_ms / 1e3) / 1e9
    ctx.solve()
    torch.cuda.synchronize()
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    Ks = max(10, min(K, 200))
    s0.record()
    for _ in range(Ks):
        ctx.solve()
    s1.record()
    torch.cuda.synchronize()
    span_ms = s0.elapsed_time(s1) / Ks
    span_gbs = sum(pb[p] for p in fft_phases) / (span_ms / 1e3) / 1e9
    return {"phase_ms": phase_ms, "pb": pb, "dom": dom, "conv_ms": conv_ms, "conv_gbs": conv_gbs,
            "span_ms": span_ms, "span_gbs": span_gbs}


def extra_workload(name, K, Wm, sort_every, fp64_steps):
    """Step rate, phase roofline and convolution span of another workload
    with the same kernels (and, with fp64_steps, the FP64 comparison)."""
    import torch
    from paper_1210_1736_gb300 import pm, workloads as W
    from paper_1210_1736_gb300.workloads import mass_bound
    w = getattr(W, name)()
    dt = w["dt"]
    m32 = w["m"].astype(np.float32)
    host = dict(pos=w["pos"].astype(np.float32), vel=w["vel"].astype(np.float32), m=m32, gal=w["gal"])
    fp64 = fp64_comparison(w, host, m32, fp64_steps) if fp64_steps > 0 else None
    ctx = pm.Context(w, mass_bound(m32))
    parts = pm.Particles(host["pos"], host["vel"], m32, w["gal"])
    n = parts.n
    ctx.deposit(parts)
    ctx.solve()
    ctx.kick(parts, -0.5 * dt)
    ctx.set_sort_interval(sort_every)
    ctx.step(parts, dt, Wm)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    ctx.step(parts, dt, K)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / K
    dm = device_phases(ctx, parts, w, n, dt, K)
    peak, _ = peaks()
    z = dm["phase_ms"]["fft_z_conv"]
    out = {"workload": WORKLOAD_DESC[name], "particles": n, "steps": K, "value": n / (ms / 1e3),
           "unit": UNIT, "ms_per_step": ms,
           "fft_z_conv": {"ms_per_step": z, "frac": dm["pb"]["fft_z_conv"] / (z / 1e3) / 1e9 / peak},
           "fft_convolve": {"frac": dm["conv_gbs"] / peak, "span_frac": dm["span_gbs"] / peak,
                            "span_ms_per_step": dm["span_ms"]},
           "step_bound_frac": sum(dm["pb"].values()) / (peak * 1e9) * 1e3 / ms,
           "solve_schedule": ctx.info()["solve_schedule"], "batched": ctx.info()["batched"],
           "phase_ms_per_step": dm["phase_ms"], "phase_hbm_frac": phase_hbm_fracs(dm["phase_ms"], dm["pb"], peak)}
    if fp64 is not None:
        fp64["speedup_fp32"] = fp64["ms_per_step"] / ms
        out["fp64_path"] = fp64
    ctx.close()
    del parts
    torch.cuda.empty_cache()
    return out


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_1210_1736_gb300 import pm, workloads as W
    from paper_1210_1736_gb300.workloads import mass_bound

    rank, local, world = env_rank()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    w = getattr(W, args.workload)()
    dt = w["dt"]
    m32 = w["m"].astype(np.float32)
    host = dict(pos=w["pos"].astype(np.float32), vel=w["vel"].astype(np.float32), m=m32, gal=w["gal"])
    fp64 = fp64_comparison(w, host, m32, args.fp64_steps) if args.fp64_steps > 0 else None
    ctx = pm.Context(w, mass_bound(m32))
    parts = pm.Particles(host["pos"], host["vel"], m32, w["gal"])
    n = parts.n
    K, Wm = args.steps, args.warmup

    ctx.deposit(parts)
    ctx.solve()
    ctx.kick(parts, -0.5 * dt)
    ctx.set_sort_interval(args.sort_every)
    ctx.step(parts, dt, Wm)
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # ---- device-resident timed region (graph replays) ----
    clk = Clocks(local)
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    ctx.step(parts, dt, K)
    e1.record()
    barrier()
    clocks = clk.stop()
    ms = slowest_rank_ms(e0.elapsed_time(e1), world, "cuda")
    value = job_rate(world, n, K, ms)

    # ---- per-phase device times and the convolution span ----
    dm = device_phases(ctx, parts, w, n, dt, K)
    phase_ms, pb, dom = dm["phase_ms"], dm["pb"], dm["dom"]
    peak, peak_kind = peaks()
    achieved = pb[dom] / (phase_ms[dom] / 1e3) / 1e9

    # ---- end to end through the C ABI with host buffers (RequestPipeline) ----
    # every request carries the state as the device-resident run left it:
    # spatially sorted, as a client that keeps the library's particle order
    # sends it
    hbuf = request_block_from(parts)
    pipe = RequestPipeline(ctx, hbuf, dt)
    h2d, d2h = pipe.h2d_bytes, pipe.d2h_bytes
    Ke = max(1, min(K, 200))

    def e2e_run(overlap):
        pipe.reset()
        # untimed: every buffer's captured steps (with and without the sort
        # of every args.sort_every-th step) are made here
        for k in range(pipe.NB * max(1, args.sort_every)):
            pipe.request(k, overlap)
        torch.cuda.synchronize()
        barrier()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(pipe.main)
        for k in range(Ke):
            pipe.request(k, overlap)
        pipe.join()
        f1.record(pipe.main)
        barrier()
        return job_rate(world, n, Ke, slowest_rank_ms(f0.elapsed_time(f1), world, "cuda"))

    e2e_serial = e2e_run(False)
    e2e = e2e_run(True)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": Wm,
        "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic (seeded disc-bulge-halo galaxy, random order)",
        "config": bench_config(w, args.workload, n, world),
        "spatial_sort_every": args.sort_every,
        "solve_schedule": ({0: "one branch per unit", 1: "two staggered lanes",
                            -1: "single unit"}[ctx.info()["solve_schedule"]] +
                           ("; units: grid shapes, same-shape pairs batched per launch" if ctx.info()["batched"]
                            else "; units: geometries, one launch per pair")),
        "device_bytes": ctx.info()["bytes"],
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": ncu_traffic(dom, args.workload)},
        "step_bound": {"algorithmic_bytes": sum(pb.values()),
                       "min_ms_per_step": sum(pb.values()) / (peak * 1e9) * 1e3,
                       "frac": sum(pb.values()) / (peak * 1e9) * 1e3 / (ms / K),
                       "note": "whole step by the byte model (every phase's algorithmic HBM bytes) at the "
                               "measured copy bandwidth, against the graph-replayed step"},
        "fft_convolve": {"gbs": dm["conv_gbs"], "frac": dm["conv_gbs"] / peak, "ms_per_step": dm["conv_ms"],
                         "span_gbs": dm["span_gbs"], "span_frac": dm["span_gbs"] / peak,
                         "span_ms_per_step": dm["span_ms"],
                         "note": "gbs/frac: the five pass phases timed one after another; span: pm_solve as "
                                 "the step runs it (geometry chains overlapping), byte model over time"},
        "phase_ms_per_step": phase_ms,
        "phase_hbm_frac": phase_hbm_fracs(phase_ms, pb, peak),
        "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "steps": Ke, "serial_value": e2e_serial,
                "pipeline": "one-step requests rotating over three device buffers: upload of k+1 and download "
                            "of k-1 on their own streams overlap the step of k; serial_value without the overlap; "
                            "each request uploads the full particle state (spatially sorted, as the device-resident "
                            "run left it) and downloads positions and velocities"},
        "gpu_launches": launches(w, K, args.sort_every, bool(ctx.info()["batched"])),
        "clocks": clocks,
    }
    if fp64 is not None:
        fp64["speedup_fp32"] = fp64["ms_per_step"] / (ms / K)
        line["fp64_path"] = fp64
    ctx.close()
    del pipe, parts
    torch.cuda.empty_cache()
    if rank == 0 and world == 1:
        extras = [x for x in args.extra_workloads.split(",") if x and x != "none" and x != args.workload]
        line["extra_workloads"] = {x: extra_workload(x, K, Wm, args.sort_every,
                                                     args.fp64_steps if x == "galaxy_1m" else 0)
                                   for x in extras}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = oracle_sampled_rate(w, args.workload, 3)
    if world > 1:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)


def oracle_sampled_rate(w, workload, steps):
    """The FP64 oracle, as it stands, timed on bounded samples of its step.

    With S mass sets, sampled step k runs the per-particle work of one full
    step (recentre sums, classification, deposit, forces by the combination
    rule, kick, drift) on particle slice k mod S of S equal slices, plus the
    doubled-grid convolution of one mass set, taken in an order that visits
    every distinct geometry first.  A full step's time is estimated as S x
    the mean slice time plus, for every mass set, the mean time measured for
    its geometry's convolution (an FFT's cost does not depend on the data).
    Forces use zero potentials of the right shapes (the gathers cost the
    same).  At least one step per distinct geometry is run."""
    import oracle as O
    ww = dict(w)
    ww["m"] = w["m"].astype(np.float32)
    system = O.system_from_workload(ww)
    state = O.state_from_workload(ww)
    sets = []
    for g, gal in enumerate(system.galaxies):
        for k, geom, _, _ in O.mass_sets(gal):
            sets.append((g, k, geom))
            O.green_hat(geom, system.h000)      # H-hat tables: set-up, outside the clock (as the library's)
    first, rest, seen = [], [], set()
    for x in sets:
        (rest if x[2] in seen else first).append(x)
        seen.add(x[2])
    order = first + rest
    S = len(sets)
    phi0 = [{k: np.zeros(geom.shape) for gg, k, geom in sets if gg == g} for g in range(len(system.galaxies))]
    n = len(state.m)
    bounds = np.linspace(0, n, S + 1).astype(np.int64)
    t_part, t_conv = [], {}
    nrun = max(steps, len(first))
    for k in range(nrun):
        a, b = bounds[k % S], bounds[k % S + 1]
        sub = O.State(state.pos[:, a:b].copy(), state.vel[:, a:b].copy(), state.m[a:b].copy(),
                      state.gal[a:b].copy(), state.flags[a:b].copy(), state.centres.copy())
        g, kk, geom = order[k % S]
        t0 = time.perf_counter()
        sub.centres = O.recentre(sub, system)
        flags, own = O.classify(sub, system)
        rho, flags, sh = O.deposit(sub, system, flags, own)
        acc = O.accelerations(sub, system, phi0, flags)
        live = (flags & O.FLAG_LOST) == 0
        sub.vel = O.kick(sub.vel, acc, w["dt"], live)
        sub.pos = O.drift(sub.pos, sub.vel, w["dt"], live)
        t1 = time.perf_counter()
        O.potential_fft(O.rho_real(rho[g][kk], sh), geom, system.G, system.h000)
        t2 = time.perf_counter()
        t_part.append(t1 - t0)
        t_conv.setdefault(geom, []).append(t2 - t1)
    tp = S * float(np.mean(t_part))
    tc = sum(float(np.mean(t_conv[geom])) for _, _, geom in sets)
    total = tp + tc
    return {"value": n / total, "unit": UNIT, "cores": 1, "host_nproc": os.cpu_count(), "kind": "oracle",
            "steps_sampled": nrun, "est_s_per_step": total,
            "sample": f"{nrun} sampled step(s) of {workload} ({n} particles, {S} mass sets): each the "
                      f"per-particle work of a step on 1/{S} of the particles plus one mass set's doubled-grid "
                      f"convolution; full step estimated at {total:.1f} s = {tp:.1f} s particle work + "
                      f"{tc:.1f} s convolutions; single-threaded numpy FP64 on one of the host's "
                      f"{os.cpu_count()} cores (H-hat tables built before timing)"}


REF_SAMPLES = 20


def run_reference(args):
    from paper_1210_1736_gb300 import workloads as W
    rank, _, world = env_rank()
    if rank != 0:
        return
    w = getattr(W, args.workload)()
    # at most REF_SAMPLES sampled oracle steps (at least one per distinct
    # geometry), whatever --steps asks for: a sampled large_16m step takes a
    # few seconds on one host core, and the run must end within minutes
    cb = oracle_sampled_rate(w, args.workload, max(1, min(args.steps, REF_SAMPLES)))
    line = {"metric": METRIC, "value": cb["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic (seeded disc-bulge-halo galaxy)", "impl": "reference",
            "config": bench_config(w, args.workload, len(w["m"]), world),
            "note": "the oracle needs no warm-up (no compilation, no caches beyond the H-hat tables, which "
                    "are built before timing); each timed step is a bounded sample of a full step (see "
                    "cpu_baseline.sample), and at most %d such samples run whatever --steps asks for" % REF_SAMPLES,
            "cpu_baseline": cb,
            "e2e": {"value": cb["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(WORKLOAD_DESC))
    ap.add_argument("--extra-workloads", default=",".join(EXTRA_WORKLOADS),
                    help="comma-separated workloads also measured (rank 0, N = 1), reported in extra_workloads "
                         "('none' or '': no others)")
    ap.add_argument("--fp64-steps", type=int, default=5,
                    help="steps timed on the FP64 instantiation for comparison (0: skip)")
    ap.add_argument("--sort-every", type=int, default=10,
                    help="re-sort particles by cell every k steps inside the timed steps (0: never)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
