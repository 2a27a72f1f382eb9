"""The end-to-end request pipeline of bench.py: one-step requests whose state
lives in pinned host memory, rotating over three device buffers with their
uploads and downloads on their own streams, give request by request the same
results, bit for bit, as the same requests run one after another on one
buffer (so the streams' ordering around each step is right)."""
import numpy as np
import pytest

import bench
from paper_1210_1736_gb300 import workloads as W
from tests._harness import gpu_setup, require_cuda

pytestmark = pytest.mark.gpu


def test_pipelined_requests_equal_serial():
    torch = require_cuda()
    w = W.galaxy_small(precision="fp32")
    m32 = w["m"].astype(np.float32)
    host = dict(pos=w["pos"].astype(np.float32), vel=w["vel"].astype(np.float32))
    hbuf = bench.request_block(host, m32, w["gal"])
    R = 9
    results = {}
    for overlap in (False, True):
        ctx, _ = gpu_setup(w)
        pipe = bench.RequestPipeline(ctx, hbuf, w["dt"], nout=R)
        slots = [pipe.request(k, overlap) for k in range(R)]
        pipe.join()
        torch.cuda.synchronize()
        results[overlap] = [pipe.hout[o].clone() for o in slots]
        ctx.close()
    assert len(set(slots)) == R
    for k, (a, b) in enumerate(zip(results[False], results[True])):
        assert torch.equal(a, b), f"request {k} differs"
    # the requests did something: the positions moved
    assert not torch.equal(results[True][0][0], hbuf[0])
