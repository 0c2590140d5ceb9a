"""The bench's multi-rank path on the CPU (two gloo ranks): every rank runs its
own replica, rank 0 reports the frames of all ranks over the slowest rank's
time; the reference arm's other ranks exit without work."""
import os
import socket
import subprocess
import sys
import textwrap

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = textwrap.dedent("""
    import json, os, sys
    sys.path.insert(0, os.environ["REPO"])
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo")
    rank = dist.get_rank()
    slow = bench.max_over_ranks([10.0 * (rank + 1), 7.0 - rank], "cpu")
    ws, r, local = bench.dist_env()
    print(json.dumps({"rank": rank, "env": [ws, r, local], "slowest": slow,
                      "rate": bench.whole_job_rate(30, ws, slow[0])}))
    dist.barrier()
    dist.destroy_process_group()
""")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _env(rank, ws, port):
    env = dict(os.environ, REPO=ROOT, RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(ws),
               MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    env.pop("CUDA_VISIBLE_DEVICES", None)
    return env


def test_two_gloo_ranks_take_the_slowest_time():
    import json
    port = _free_port()
    procs = [subprocess.Popen([sys.executable, "-c", WORKER], env=_env(r, 2, port), stdout=subprocess.PIPE,
                              stderr=subprocess.PIPE, text=True) for r in range(2)]
    outs = [p.communicate(timeout=120) for p in procs]
    assert all(p.returncode == 0 for p in procs), [o[1][-500:] for o in outs]
    res = sorted((json.loads(o[0].strip().splitlines()[-1]) for o in outs), key=lambda d: d["rank"])
    for d in res:
        assert d["env"] == [2, d["rank"], d["rank"]]
        assert d["slowest"] == [20.0, 7.0]  # the max over ranks, elementwise
        assert abs(d["rate"] - 2 * 30 / 0.020) < 1e-9  # both ranks' frames over the slowest time


def test_reference_arm_other_ranks_exit_without_work():
    env = _env(1, 2, _free_port())
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference"], env=env,
                       capture_output=True, text=True, timeout=120)
    assert p.returncode == 0, p.stderr[-500:]
    assert p.stdout.strip() == ""
