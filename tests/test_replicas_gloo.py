"""The multi-rank bench path (one independent replica per rank, slowest rank's
time, whole-job rate) with world size 2 on the gloo backend, on CPU."""
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import os, sys
sys.path.insert(0, {root!r})
import torch.distributed as dist
import bench
dist.init_process_group("gloo")
rank, world = dist.get_rank(), dist.get_world_size()
t = bench.reduce_max(1.5 + rank, dist)        # rank 1 is the slowest
assert t == 1.5 + world - 1, t
rate = bench.job_rate(world, 4096 * 2048, 200, t)
if rank == 0:
    print("OK", t, rate)
dist.barrier()
dist.destroy_process_group()
"""


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_two_rank_max_time_and_job_rate(tmp_path):
    script = tmp_path / "worker.py"
    script.write_text(WORKER.format(root=ROOT))
    port = free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                   WORLD_SIZE="2", LOCAL_RANK=str(rank))
        procs.append(subprocess.Popen([sys.executable, str(script)], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True))
    outs = [p.communicate(timeout=120)[0] for p in procs]
    assert all(p.returncode == 0 for p in procs), outs
    ok = [o for o in outs if o.startswith("OK")]
    assert len(ok) == 1
    t, rate = map(float, ok[0].split()[1:])
    assert t == 2.5
    assert abs(rate - 2 * 4096 * 2048 * 200 / 2.5 / 1e6) < 1e-6 * rate


def test_single_rank_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max(3.25) == 3.25
    assert abs(bench.job_rate(1, 100, 10, 1e-3) - 1.0) < 1e-12
