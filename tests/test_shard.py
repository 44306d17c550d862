"""Independent RVEs over the ranks of a job: the assignment every rank computes
alike, and the one gather of per-RVE results at the end (two gloo ranks on the
CPU; no GPU)."""

import math
import os
import socket

import torch.multiprocessing as mp

from paper_1806_10599_gb300 import shard
from rve_inputs import batch_rves


def test_cost_model_is_n_log_n():
    assert shard.rve_cost(4) == 64 * 6
    assert shard.rve_cost((2, 4, 8)) == 64 * 6
    assert shard.rve_cost(96) > shard.rve_cost(80) > shard.rve_cost(64)


def test_every_rve_on_exactly_one_rank_and_balanced():
    shapes = [n for n, _, _ in batch_rves()]
    costs = [shard.rve_cost(s) for s in shapes]
    for world in (1, 2, 3, 4, 8, 40):
        parts = shard.assign(shapes, world)
        assert len(parts) == world
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(shapes)))
        loads = [sum(costs[i] for i in p) for p in parts]
        # greedy longest-processing-time bound: no rank exceeds the mean load by more than one RVE's cost
        assert max(loads) <= sum(costs) / world + max(costs) + 1e-9
        assert parts == shard.assign(shapes, world)  # deterministic: every rank gets the same answer
    # one rank: everything, in order
    assert shard.assign(shapes, 1) == [list(range(len(shapes)))]


def test_lpt_on_a_hand_case():
    # costs 384 (64 voxels), 160 (32), 64 (16), 64 (16): rank 0 takes the largest, rank 1 the rest (288 < 384)
    shapes = [(4, 4, 4), (4, 4, 2), (4, 2, 2), (2, 2, 4)]
    assert [shard.rve_cost(s) for s in shapes] == [384, 160, 64, 64]
    assert shard.assign(shapes, 2) == [[0], [1, 2, 3]]
    assert shard.assign(shapes, 3) == [[0], [1], [2, 3]]


def test_merge_restores_the_global_order():
    parts = [[0, 3], [1, 2]]
    assert shard.merge([["a", "d"], ["b", "c"]], parts, 4) == ["a", "b", "c", "d"]
    try:
        shard.merge([["a"], ["b", "c"]], parts, 4)
    except ValueError:
        pass
    else:
        raise AssertionError("a short result list must be refused")


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group(backend="gloo")
    try:
        shapes = [n for n, _, _ in batch_rves()]
        parts = shard.assign(shapes, world)
        # each rank "solves" its RVEs: a stand-in result that names the RVE and the rank
        mine = [("rve", i, rank, math.sqrt(i)) for i in parts[rank]]
        got = shard.gather_to_rank0(mine, world)
        if rank == 0:
            out.put(shard.merge(got, parts, len(shapes)))
        else:
            assert got is None
    finally:
        dist.destroy_process_group()


def test_results_gathered_on_rank_0_from_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    merged = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    shapes = [n for n, _, _ in batch_rves()]
    parts = shard.assign(shapes, 2)
    owner = {i: r for r, p in enumerate(parts) for i in p}
    assert [m[1] for m in merged] == list(range(len(shapes)))
    assert all(m[2] == owner[m[1]] for m in merged)
    assert {m[2] for m in merged} == {0, 1}


class _FakeLib:
    """Stands in for the library in the bench's batch measurement: each RVE
    "solves" instantly and reports its edge length as its Fatemi-Socie maximum."""

    GFF_WARM_EXTRAPOLATE = 3
    GFF_MAT_CP_FCC = 2

    class _Rep:
        newton_iters = 2
        cuts = 0

    def make_options(self, **kw):
        return kw

    def make_material(self, kind):
        return kind

    def create_rve(self, ms, mats, opts):
        return {"n": ms[1]}

    def gff_set_warm_start(self, h, u, mode):
        pass

    def gff_autotune(self, h):
        pass

    def gff_destroy(self, h):
        pass

    def gff_batch_run(self, hs, dt, Fbar, mask, Pbar, cycle_start=None, raise_on_error=True):
        import numpy as np

        return None, [[self._Rep() for _ in dt] for _ in hs], np.zeros(len(hs), np.int32)

    def gff_get_fips(self, h, ngrains):
        return None, None, [h["n"] / 100.0]

    def gff_run_history(self, h, dt, Fbar, mask, Pbar, cycle_start=None):
        return None, []


def _bench_rank(rank, world, port, out):
    import types

    import torch.distributed as dist

    import bench
    import rve_inputs

    rve_inputs.polycrystal = lambda n, ng, seed: ("ms", n)  # no microstructure needed by the stand-in
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group(backend="gloo")
    try:
        torch_stub = types.SimpleNamespace(cuda=types.SimpleNamespace(synchronize=lambda: None))
        res = bench.time_batch(_FakeLib(), torch_stub, 4, 2, 1, world, rank)
        if rank == 0:
            out.put(res)
    finally:
        dist.destroy_process_group()


def test_bench_batch_spreads_the_rves_over_two_gloo_ranks():
    """bench.py's batch measurement under two ranks: each rank builds and runs
    only its share, rank 0 reports every RVE's result in the global order."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_bench_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = q.get(timeout=180)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    specs = batch_rves()
    assert "error" not in res, res
    assert res["ranks"] == 2 and sum(res["rves_per_rank"]) == len(specs) and min(res["rves_per_rank"]) > 0
    assert res["cycle"]["fatemi_socie_max_per_rve"] == [n / 100.0 for n, _, _ in specs]
    assert res["cycle"]["status"] == [0] * len(specs) and res["cycle"]["newton_mean"] == 2.0
    assert res["cycle"]["s_per_increment_batched"] >= 0
    assert "batched_speedup_first_2" in res
