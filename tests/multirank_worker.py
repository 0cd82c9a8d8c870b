"""Worker for the two-rank CPU test: run under torch.distributed.run with the gloo backend."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import torch.distributed as dist  # noqa: E402

import bench  # noqa: E402

dist.init_process_group("gloo")
rank, world = dist.get_rank(), dist.get_world_size()
dist.barrier()
mx = bench.max_over_ranks(10.0 * (rank + 1), world)
print(json.dumps({"rank": rank, "world": world, "max": mx}), flush=True)
dist.barrier()
dist.destroy_process_group()
