"""One rank of the two-process host test (launched by torch.distributed.run
with the gloo backend on CPU): each rank reports a different step time, the
ranks combine them with the bench's own rules, and each prints what it got."""
import json
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import torch.distributed as dist  # noqa: E402

import bench  # noqa: E402


def main():
    rank, local, world = bench.env_rank()
    dist.init_process_group("gloo")
    my_ms = 3.0 + 2.0 * rank                 # rank 1 is the slower one
    ms = bench.slowest_rank_ms(my_ms, world, "cpu")
    value = bench.job_rate(world, 1000, 10, ms)
    dist.barrier()
    dist.destroy_process_group()
    # one write per line: the ranks share the launcher's stdout
    sys.stdout.write(json.dumps({"rank": rank, "local": local, "world": world, "ms": ms, "value": value}) + "\n")
    sys.stdout.flush()


if __name__ == "__main__":
    main()
