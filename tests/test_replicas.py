"""The N > 1 path of bench.py on the CPU: two gloo ranks.

The solver runs as independent replicas (nothing is exchanged on the data
path); what N > 1 adds is host logic: the rank environment, the maximum of
the timings over ranks, the whole-job rate, and that only rank 0 reports."""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

RANK_CODE = r"""
import json, sys
sys.path.insert(0, sys.argv[1])
import torch.distributed as dist
import bench
ws, rank, local = bench.dist_env()
dist.init_process_group("gloo", rank=rank, world_size=ws)
mine = [10.0 + rank, 20.0 - rank, 3.0 * (rank + 1)]
got = bench.max_over_ranks(mine, dist)
print(json.dumps(dict(env=[ws, rank, local], got=got, rate=bench.whole_job_rate(ws, 48, 10, got[0]))))
dist.destroy_process_group()
"""


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _env(rank, ws, port):
    env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
               WORLD_SIZE=str(ws), LOCAL_RANK=str(rank), OMP_NUM_THREADS="1")
    env.pop("CUDA_VISIBLE_DEVICES", None)
    return env


def test_two_ranks_take_the_slowest_rank_time():
    ws, port = 2, _free_port()
    procs = [subprocess.Popen([sys.executable, "-c", RANK_CODE, ROOT], env=_env(r, ws, port),
                              stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True) for r in range(ws)]
    outs = []
    try:
        for p in procs:
            out, err = p.communicate(timeout=180)
            assert p.returncode == 0, err[-2000:]
            outs.append(json.loads(out.strip().splitlines()[-1]))
    finally:
        for p in procs:
            if p.poll() is None:
                p.kill()
    for rank, o in enumerate(outs):
        assert o["env"] == [ws, rank, rank]
        assert o["got"] == [11.0, 20.0, 6.0]          # element-wise max over the two ranks
        assert o["rate"] == ws * 48 * 50 * 10 / (11.0 / 1e3)


def test_reference_arm_reports_on_rank_zero_only():
    """Under torchrun the reference arm runs on rank 0; other ranks exit 0 silently
    (before any oracle work)."""
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "3"], env=_env(1, 2, _free_port()), capture_output=True,
                       text=True, timeout=120)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""
