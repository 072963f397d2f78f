"""The multi-rank path of bench.py on CPU: two gloo ranks (no GPU), the
barrier and the max-over-ranks timing the JSON line reports."""
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import os, sys
sys.path.insert(0, {root!r})
import bench
world, rank, local = bench.dist_setup(None, backend="gloo")
assert world == 2 and rank in (0, 1)
bench.barrier(world)
got = bench.max_over_ranks(10.0 + rank, world)
assert got == 11.0, got
import torch.distributed as dist
dist.destroy_process_group()
print("rank", rank, "ok")
"""


def test_two_gloo_ranks_barrier_and_max(tmp_path):
    script = tmp_path / "worker.py"
    script.write_text(WORKER.format(root=ROOT))
    env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT="29517", WORLD_SIZE="2")
    procs = []
    for r in range(2):
        e = dict(env, RANK=str(r), LOCAL_RANK=str(r))
        procs.append(subprocess.Popen([sys.executable, str(script)], env=e,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = [p.communicate(timeout=120) for p in procs]
    for p, (out, err) in zip(procs, outs):
        assert p.returncode == 0, err
        assert "ok" in out
