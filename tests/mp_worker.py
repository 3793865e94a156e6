"""Rank program for tests/test_multiprocess.py (run under torch.distributed.run, gloo)."""
import json
import os
import sys

import torch
import torch.distributed as dist

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402

dist.init_process_group("gloo")
rank = dist.get_rank()
got = bench.max_over_ranks([1.0 + rank, 5.0 - rank, float(rank)])
bench.barrier(torch)
print(json.dumps({"rank": rank, "max": got}), flush=True)
dist.destroy_process_group()
