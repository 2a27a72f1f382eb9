"""Host logic of bench.py (CPU): the byte model behind the roofline numbers,
the count of kernel launches it claims, and the rule that a stored DRAM
traffic figure is used only on the kernel code it was captured on.

Byte model per mass set of A = nx ny nz active cells (8-byte complex
spectra, S1 = (nx+1) ny nz): x forward 8A + 8 S1, y forward 8 S1 + 16 S1,
z convolve 2 x 16 S1 (+ the H-hat octant once per geometry), y inverse
16 S1 + 8 S1, x inverse 8 S1 + 4A -- in all 12 A + 96 S1, i.e. about 108 A."""
import numpy as np

import bench
from paper_1210_1736_gb300 import workloads as W


def _one_set(n):
    return dict(galaxies=[dict(coarse=(n, n, n, 10.0, 1.0), medium=None, fine=None)])


def test_byte_model_of_one_set():
    for n in (32, 128):
        A, S1 = n ** 3, (n + 1) * n * n
        b = bench.phase_bytes(_one_set(n), 0, 4)
        fft = sum(b[p] for p in ("fft_x_fwd", "fft_y_fwd", "fft_z_conv", "fft_y_inv", "fft_x_inv"))
        hhat = 4 * (n + 1) ** 3
        assert fft == 12 * A + 96 * S1 + hhat
        assert abs(fft - hhat - 108 * A) <= 96 * A / n + 1


def test_byte_model_counts_pairs_and_particles():
    spec = dict(galaxies=[dict(coarse=(128, 128, 128, 32.0, 1.0), medium=(128, 128, 128, 6.0, 0.25),
                               fine=(128, 128, 32, 1.5, 1.0))])
    n = 1000
    b = bench.phase_bytes(spec, n, 4)
    A2, A1 = 128 ** 3, 128 * 128 * 32
    # five mass sets: two on each 128^3 geometry, one on the fine grid
    assert b["deposit"] == n * 24 + 8 * (4 * A2 + A1)
    assert b["force_kick_drift"] == n * 52
    assert b["recentre"] == n * 24


def test_launch_count_per_pair():
    assert bench.fft_pairs(_one_set(32)) == 1
    g = W.galaxy_small()
    assert bench.fft_pairs(g) == 3
    # galaxy_small: shapes 32^3 (coarse and medium pairs) and 32x32x8 (the
    # fine grid): x, y forward 2 + 2, z 1 + 1, y, x inverse 2 + 2 -> 10;
    # per step also recentre (2), deposit (1), force (1); six sort kernels
    # every sort_every-th step
    assert bench.fft_launches(g) == 10
    assert bench.launches(g, 10, 0) == 10 * (2 + 1 + 10 + 1)
    assert bench.launches(g, 10, 5) == 10 * 14 + 2 * 6
    # large_16m: the satellites' six 128^3 pairs (two of them fine grids)
    # share launches: x 1, y 1, z 1 + 1 (both difference fields of the two
    # fine grids in one launch), y inverse 1, x inverse 1; the galaxy's
    # 256x256x64 fine grid: x, y 2, z 1 (fused), y, x inverse 2
    spec = dict(galaxies=[
        dict(coarse=(256, 256, 256, 32, 1), medium=(256, 256, 256, 6, 0.25), fine=(256, 256, 64, 1.5, 1)),
        dict(coarse=(128, 128, 128, 32, 1), medium=(128, 128, 128, 0.5, 1), fine=(128, 128, 128, 0.125, 1)),
        dict(coarse=(128, 128, 128, 32, 1), medium=(128, 128, 128, 0.5, 1), fine=(128, 128, 128, 0.125, 1))])
    assert bench.fused_diff((256, 256, 64)) and bench.fused_diff((128, 128, 128))
    assert bench.fused_diff((32, 32, 8)) and bench.fused_diff((128, 128, 32))
    assert not bench.fused_diff((16, 16, 64))   # 32 tile columns > nx: two launches
    assert not bench.fused_diff((256, 256, 256))   # length 512: two launches
    assert bench.fft_launches(spec) == (2 + 1 + 2) + (2 + 1 + 2) + (2 + 2 + 2)
    # unbatched: five launches per pair and two more per fused fine grid
    # (three where the two difference-field products take two launches)
    assert bench.fft_launches(spec, batched=False) == 5 * 9 + 2 * 3
    assert bench.fft_launches(W.galaxy_small(), batched=False) == 5 * 3 + 2


def test_grid1_counted_below_its_r2c_minimum():
    # grid 1 gives four real fields (fx, fy, fz, Phi_1) from one spectrum;
    # the byte model counts its z, y-inverse and x-inverse passes as two
    # real fields' chains, below the R2C minimum of four
    base = dict(coarse=(64, 64, 64, 32.0, 1.0), medium=(64, 64, 64, 6.0, 0.25))
    with1 = bench.phase_bytes(dict(galaxies=[dict(base, fine=(64, 64, 16, 1.5, 1.0))]), 0, 4)
    without = bench.phase_bytes(dict(galaxies=[dict(base, fine=None)]), 0, 4)
    nx, ny, nz = 64, 64, 16
    A, S1 = nx * ny * nz, (nx + 1) * ny * nz
    S2 = 2 * S1
    hhat = 4 * (nx + 1) * (ny + 1) * (nz + 1)
    d = {p: with1[p] - without[p] for p in with1}
    assert d["fft_z_conv"] - hhat == 4 * 8 * S2 < 5 * 8 * S2
    assert d["fft_y_inv"] == 2 * 8 * (S2 + S1) < 4 * 8 * (S2 + S1)
    assert d["fft_x_inv"] == 2 * 8 * S1 + 4 * 4 * A < 4 * 8 * S1 + 4 * 4 * A


def test_traffic_record_follows_the_kernel_code(tmp_path, monkeypatch):
    # the stored DRAM traffic is used only while the kernel sources' code is
    # the one it was captured on: comments do not count, code does
    import json
    import os
    import shutil
    csrc = os.path.join(tmp_path, "paper_1210_1736_gb300", "csrc")
    shutil.copytree(os.path.join(bench.ROOT, "paper_1210_1736_gb300", "csrc"), csrc)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.kernel_source_hash()
    os.makedirs(os.path.join(tmp_path, "profiles"))
    rec = dict(source_hash=h0, workload="large_16m", phases=dict(fft_z_conv=1.5e9))
    json.dump(rec, open(os.path.join(tmp_path, "profiles", "traffic.json"), "w"))
    assert bench.ncu_traffic("fft_z_conv", "large_16m") == 1.5e9
    assert bench.ncu_traffic("fft_z_conv", "galaxy_1m") is None
    f = os.path.join(csrc, "pm_passes.cuh")
    src = open(f).read()
    open(f, "w").write(src + "\n// a comment\n/* and a\n   block comment */\n")
    assert bench.kernel_source_hash() == h0
    assert bench.ncu_traffic("fft_z_conv", "large_16m") == 1.5e9
    open(f, "w").write(src + "\nstatic const int pm_unused_constant = 1;\n")
    assert bench.kernel_source_hash() != h0
    assert bench.ncu_traffic("fft_z_conv", "large_16m") is None


def test_phase_fractions():
    # 6.7934 GB in 1 ms is the measured copy bandwidth exactly; a phase
    # without bytes (the sort) or without time is left out
    f = bench.phase_hbm_fracs({"fft_x_fwd": 1.0, "fft_y_fwd": 2.0, "spatial_sort": 0.1, "deposit": 0.0},
                              {"fft_x_fwd": 6.7934e9, "fft_y_fwd": 6.7934e9, "spatial_sort": 0.0,
                               "deposit": 1e9}, 6793.4)
    assert set(f) == {"fft_x_fwd", "fft_y_fwd"}
    assert abs(f["fft_x_fwd"] - 1.0) < 1e-12 and abs(f["fft_y_fwd"] - 0.5) < 1e-12
