"""The multi-process path of bench.py on CPU (torch.distributed gloo, two
ranks, 127.0.0.1): each rank runs an independent replica, the job's time is
the slowest rank's (a max all-reduce every rank receives), and the job's
throughput counts all ranks' cell updates over that time.  A non-zero rank
of the reference arm exits at once without output (rank 0 alone prints)."""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

RANK_SCRIPT = r"""
import json, os, sys
sys.path.insert(0, sys.argv[1])
import bench
world, rank, local, dist = bench.replica_context("gloo")
ms = 10.0 + 5.0 * rank            # rank 1 is the slower replica
m = bench.max_over_ranks(ms, dist, "cpu")
v = bench.job_mlups(world, 1000000, m)
dist.barrier()
print(json.dumps({"rank": rank, "local": local, "world": world, "ms_max": m, "mlups": v}))
dist.destroy_process_group()
"""


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_replicas_share_the_slowest_time():
    port = free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE="2", RANK=str(r),
                   LOCAL_RANK=str(r))
        procs.append(subprocess.Popen([sys.executable, "-c", RANK_SCRIPT, ROOT], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    out = []
    for p in procs:
        o, e = p.communicate(timeout=180)
        assert p.returncode == 0, e[-2000:]
        out.append(json.loads(o.strip().splitlines()[-1]))
    out.sort(key=lambda d: d["rank"])
    assert [d["rank"] for d in out] == [0, 1] and [d["local"] for d in out] == [0, 1]
    for d in out:
        assert d["world"] == 2
        assert d["ms_max"] == 15.0
        assert abs(d["mlups"] - 2 * 1000000 / 0.015 / 1e6) < 1e-9


def test_reference_arm_on_a_non_zero_rank_exits_quietly():
    env = dict(os.environ, WORLD_SIZE="2", RANK="1", LOCAL_RANK="1")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2"], env=env,
                       capture_output=True, text=True, timeout=120)
    assert p.returncode == 0, p.stderr[-2000:]
    assert p.stdout.strip() == ""
