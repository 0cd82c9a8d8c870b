"""The bench's multi-rank timing path on two gloo ranks (CPU): every replica reports the
slowest rank's time."""
import json
import os
import re
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))


def test_max_over_ranks_two_gloo_ranks():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", "29531", os.path.join(HERE, "multirank_worker.py")]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=240)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [json.loads(m) for m in re.findall(r'\{"rank"[^{}]*\}', r.stdout)]
    assert sorted(l["rank"] for l in lines) == [0, 1]
    assert all(l["world"] == 2 and l["max"] == 20.0 for l in lines)


def test_max_over_ranks_single_rank_is_identity():
    sys.path.insert(0, os.path.dirname(HERE))
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
