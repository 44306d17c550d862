"""The N > 1 path of bench.py on the CPU: two gloo ranks.  One apply does not
shard, so N GPUs run N independent replicas; what crosses ranks is the
barrier around the timed region, the maximum of the timings over ranks and
rank 0 alone printing the line."""

import argparse
import json
import os
import socket
import subprocess
import sys

import torch.multiprocessing as mp

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group(backend="gloo")
    try:
        bench.barrier(world)
        # rank r reports r + 1 seconds: every rank must see the slowest one
        out.put((rank, bench.max_over_ranks(float(rank + 1), world)))
        bench.barrier(world)
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_on_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert got == {0: 2.0, 1: 2.0}


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(3.5, 1) == 3.5
    bench.barrier(1)


def test_reference_arm_under_torchrun_prints_one_line_from_rank_0():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2", "--master-addr",
           "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference", "--gpus", "2", "--steps", "2",
           "--warmup", "1", "--grid", "16"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=300, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"


def test_whole_job_value_counts_every_rank():
    """Weak scaling: each rank applies the operator `steps` times in the
    (max over ranks) timed region, so the job's rate is world x steps / time."""
    a = argparse.Namespace(gpus=2, steps=10, warmup=3, impl="gff", increments=0, cpu_applies=0, grid=128)
    raw = {"ms64": 30.0, "ms32": 4.0, "msd": 31.0, "k64": [1.2, 0.9, 0.9], "k32": [0.18, 0.06, 0.07],
           "e2e_s": 0.05, "xbytes": 9 * 128 ** 3 * 8, "clocks": None, "increment": None, "cpu": None}
    one = bench.build_line(a, 1, raw, {"hbm_gbs": 6800.0}, "measured")
    two = bench.build_line(a, 2, raw, {"hbm_gbs": 6800.0}, "measured")
    assert two["n_gpus"] == 2 and two["scaling"] == "weak"
    assert abs(two["value"] - 2 * one["value"]) < 1e-9
    assert abs(two["e2e"]["value"] - 2 * one["e2e"]["value"]) < 1e-9
    assert abs(two["variants"]["fp32_apply"]["value"] - 2 * one["variants"]["fp32_apply"]["value"]) < 1e-9
