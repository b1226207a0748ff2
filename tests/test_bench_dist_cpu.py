"""The multi-process path of the benchmark on CPU: two ranks over gloo (no
GPU).  Each replica sorts its own keys; the job's time is the slowest
rank's; the job's value counts every rank's bytes; the reference arm prints
one line from rank 0 and nothing from the others."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


WORKER = r'''
import os, sys, json
sys.path.insert(0, sys.argv[1])
import torch.distributed as dist
import bench
dist.init_process_group("gloo", rank=int(os.environ["RANK"]), world_size=int(os.environ["WORLD_SIZE"]))
rank, world, local = bench.dist_env()
t = bench.max_over_ranks(1.5 + 2.0 * rank, world, "cpu")   # rank 1 is the slow one
print(json.dumps({"rank": rank, "world": world, "max": t, "seed": bench.rank_seed(rank),
                  "gbs": bench.job_gbs(world, 36 * (1 << 20), t / 1e3)}))
dist.barrier()
dist.destroy_process_group()
'''


def run_ranks(script, extra_args, world=2, timeout=240):
    port = str(free_port())
    procs = []
    for r in range(world):
        env = dict(os.environ, RANK=str(r), LOCAL_RANK=str(r), WORLD_SIZE=str(world),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=port, CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable, "-c", script] + extra_args, env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True,
                                      cwd=ROOT))
    outs = []
    for p in procs:
        o, e = p.communicate(timeout=timeout)
        assert p.returncode == 0, e
        outs.append(o)
    return outs


def test_two_rank_max_and_job_value():
    outs = run_ranks(WORKER, [ROOT])
    lines = [json.loads(o.strip().splitlines()[-1]) for o in outs]
    assert [l["rank"] for l in lines] == [0, 1]
    for l in lines:
        assert l["world"] == 2
        assert l["max"] == 3.5                       # the slowest rank's time
        assert abs(l["gbs"] - 2 * 36 * (1 << 20) / 3.5e-3 / 1e9) < 1e-9
    assert lines[0]["seed"] != lines[1]["seed"]      # each replica sorts its own keys


REF = r'''
import os, sys
sys.path.insert(0, sys.argv[1])
import torch.distributed as dist
dist.init_process_group("gloo", rank=int(os.environ["RANK"]), world_size=int(os.environ["WORLD_SIZE"]))
sys.argv = ["bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0",
            "--ref-sample", "65536"]
import bench
bench.main()
dist.barrier()
dist.destroy_process_group()
'''


def test_reference_arm_prints_on_rank0_only():
    outs = run_ranks(REF, [ROOT])
    line = json.loads(outs[0].strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["unit"] == "GB/s"
    assert line["cpu_baseline"]["kind"] == "oracle" and line["e2e"]["h2d_bytes_per_step"] == 0
    assert outs[1].strip() == ""
