"""The multi-process path of bench.py on CPU: two ranks launched as the
N-GPU bench is (torch.distributed.run, one process per rank, rendezvous on
127.0.0.1), with the gloo backend.  The job time is the slowest rank's time
and the job rate counts every rank's particles (weak scaling: each rank
steps its own galaxy, no collective on the data path).  The reference arm
under the same launcher runs on rank 0 only and prints one line."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _launch(args, timeout):
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port())] + args
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="", OMP_NUM_THREADS="1")
    return subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=timeout)


def _json_lines(out):
    """Every JSON object in the ranks' shared output, in order."""
    dec, objs, i = json.JSONDecoder(), [], out.find("{")
    while i >= 0:
        obj, end = dec.raw_decode(out, i)
        objs.append(obj)
        i = out.find("{", end)
    return objs


def test_two_ranks_combine_times_as_the_bench_does():
    r = _launch([os.path.join("tests", "_multirank_worker.py")], timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = sorted(_json_lines(r.stdout), key=lambda d: d["rank"])
    assert [d["rank"] for d in lines] == [0, 1]
    assert [d["local"] for d in lines] == [0, 1]
    for d in lines:
        assert d["world"] == 2
        assert d["ms"] == 5.0                              # the slower rank's time
        assert d["value"] == pytest.approx(2 * 1000 * 10 / 5e-3)


def test_reference_arm_runs_on_rank_zero_only():
    r = _launch(["bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0",
                 "--workload", "galaxy_1m"], timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _json_lines(r.stdout)
    assert len(lines) == 1
    d = lines[0]
    assert d["impl"] == "reference" and d["n_gpus"] == 2
    assert d["cpu_baseline"]["kind"] == "oracle" and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0
