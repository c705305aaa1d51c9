"""Run by tests/test_bench_contract.py under torchrun (gloo, CPU): each rank
reduces its own value with bench.reduce_max and prints the result."""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import torch.distributed as dist  # noqa: E402

import bench  # noqa: E402

dist.init_process_group("gloo")
rank = dist.get_rank()
# one write per line: the two ranks share the pipe
sys.stdout.write(f"rank {rank} max {bench.reduce_max(1.0 + rank, dist, 'cpu')}\n")
sys.stdout.flush()
dist.barrier()
dist.destroy_process_group()
