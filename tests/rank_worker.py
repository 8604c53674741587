"""One rank of the CPU test of bench.py's replica aggregation (launched by
torch.distributed.run in tests/test_bench_ranks.py; not a test module)."""
import json
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import torch.distributed as dist  # noqa: E402

import bench  # noqa: E402


def main():
    ws, rank, _ = bench._dist()
    dist.init_process_group("gloo")
    # rank r took 1 + r seconds for 100 (r + 1) pivots
    elapsed, iters = bench.aggregate_ranks(1.0 + rank, 100 * (rank + 1), ws, "cpu")
    # one file per rank: lines printed by two ranks into one pipe can interleave
    with open(os.path.join(sys.argv[1], f"rank{rank}.json"), "w") as f:
        json.dump({"rank": rank, "elapsed": elapsed, "iters": iters}, f)
    dist.barrier()
    dist.destroy_process_group()


if __name__ == "__main__":
    main()
