"""The bench's replicas-only multi-GPU aggregation on two gloo ranks (CPU): each rank reports its
own solves and time; the job value is the total over ranks divided by the slowest rank's time."""
import os
import socket
import subprocess
import sys
import textwrap

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = textwrap.dedent("""
    import os, sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo")
    rank, world = dist.get_rank(), dist.get_world_size()
    # rank r solved 64 * (r + 1) solves in 1000 * (r + 1) ms
    value, ms = bench.aggregate_ranks(64.0 * (rank + 1), 1000.0 * (rank + 1), world)
    assert abs(ms - 2000.0) < 1e-9, ms
    assert abs(value - (64.0 + 128.0) / 2.0) < 1e-9, value
    dist.barrier()
    dist.destroy_process_group()
    print("rank", rank, "ok")
""").replace("ROOT", repr(ROOT))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_replicas_aggregate_over_two_gloo_ranks():
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE="2", LOCAL_RANK=str(r),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", WORKER], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = [p.communicate(timeout=240) for p in procs]
    for p, (o, e) in zip(procs, outs):
        assert p.returncode == 0, o + e
        assert "ok" in o


def test_single_rank_aggregate():
    sys.path.insert(0, ROOT)
    import bench
    v, ms = bench.aggregate_ranks(128.0, 2000.0, 1)
    assert v == 64.0 and ms == 2000.0
