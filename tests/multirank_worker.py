"""One gloo rank for tests/test_bench_cpu.py: joins the process group from
RANK / WORLD_SIZE / MASTER_ADDR / MASTER_PORT, runs bench.py's rank reduction
on rank-dependent timings and prints the result as JSON."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import torch.distributed as dist  # noqa: E402

import bench  # noqa: E402


def main():
    rank, world = int(os.environ["RANK"]), int(os.environ["WORLD_SIZE"])
    dist.init_process_group("gloo")
    t_step, t_e2e = 1.0 + rank, 10.0 * (world - rank)  # the slowest rank differs per quantity
    t_step, t_e2e = bench.reduce_max([t_step, t_e2e], world)
    print(json.dumps({"rank": rank, "t_step": t_step, "t_e2e": t_e2e,
                      "value": bench.job_throughput(630, world, t_step)}), flush=True)
    dist.barrier()
    dist.destroy_process_group()


if __name__ == "__main__":
    main()
