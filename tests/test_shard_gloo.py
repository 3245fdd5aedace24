"""Multi-rank bookkeeping of the batched workload on CPU (gloo, world size 2)."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_1810_09299_gb300 import shard, workloads as W


def test_assign_cases_partitions_and_balances():
    sizes = [c["nr"] * c["nz"] for c in W.batched_cases(64, seed=7)]
    for world in (1, 2, 3, 4, 8):
        parts = [shard.assign_cases(sizes, world, r) for r in range(world)]
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(sizes)))
        loads = [sum(sizes[i] for i in p) for p in parts]
        assert max(loads) - min(loads) <= max(sizes)
    with pytest.raises(ValueError):
        shard.assign_cases(sizes, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sizes = [c["nr"] * c["nz"] for c in W.batched_cases(16, seed=3)]
    mine = shard.assign_cases(sizes, world, rank)
    local_nodes = sum(sizes[i] for i in mine)
    local_ms = 10.0 + 5.0 * rank  # rank 1 is the slow one
    mlups, ms, nodes = shard.job_throughput(local_nodes, 20, local_ms, dist)
    out[rank] = (mlups, ms, nodes, local_nodes)
    dist.barrier()
    dist.destroy_process_group()


def test_job_throughput_two_gloo_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    total = sum(c["nr"] * c["nz"] for c in W.batched_cases(16, seed=3))
    for r in range(world):
        mlups, ms, nodes, _ = out[r]
        assert ms == 15.0                       # max over ranks
        assert nodes == total                   # every case counted once
        assert abs(mlups - total * 20 / 15e-3 / 1e6) < 1e-9
    assert out[0][3] + out[1][3] == total


def test_single_rank_fallback():
    mlups, ms, nodes = shard.job_throughput(1000, 10, 2.0, None)
    assert (ms, nodes) == (2.0, 1000) and abs(mlups - 5.0) < 1e-12


def _sim_worker(rank, world, port, steps, out):
    """Each rank advances its share of a small batch on the FP64 oracle (the
    CPU stand-in for its GPU) and reports each case's diagnostics and its own
    measured time; the job's throughput comes from those times."""
    import time

    import torch.distributed as dist

    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    oracle.set_threads(1)
    cases = [c for _, c in sorted(W.small_cases().items())]
    sizes = [c["nr"] * c["nz"] for c in cases]
    mine = shard.assign_cases(sizes, world, rank)
    t0 = time.perf_counter()
    diags = {}
    for i in mine:
        o = oracle.Oracle(dict(cases[i], precision="fp64")).init(W.initial_phi(cases[i]))
        o.step(steps)
        diags[i] = o.diagnostics()
    local_ms = (time.perf_counter() - t0) * 1e3
    local_nodes = sum(sizes[i] for i in mine)
    mlups, ms, nodes = shard.job_throughput(local_nodes, steps, local_ms, dist)
    gathered = [None] * world
    dist.all_gather_object(gathered, local_ms)
    out[rank] = (diags, local_ms, mlups, ms, nodes, gathered)
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_batch_equals_single_rank_run():
    """World size 2: the union of the ranks' per-case diagnostics equals the
    single-rank run bit for bit, every case is advanced exactly once, and the
    job throughput is all nodes over the slowest rank's measured time."""
    import oracle

    world, steps = 2, 30
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_sim_worker, args=(r, world, port, steps, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    cases = [c for _, c in sorted(W.small_cases().items())]
    union = {}
    for r in range(world):
        for i, d in out[r][0].items():
            assert i not in union, "a case advanced on two ranks"
            union[i] = d
    assert sorted(union) == list(range(len(cases)))
    for i, c in enumerate(cases):
        ref = oracle.Oracle(dict(c, precision="fp64")).init(W.initial_phi(c)).step(steps).diagnostics()
        assert union[i] == ref, i
    times = out[0][5]
    total = sum(c["nr"] * c["nz"] for c in cases)
    for r in range(world):
        _, local_ms, mlups, ms, nodes, _ = out[r]
        assert ms == max(times) and nodes == total
        assert abs(mlups - total * steps / (ms * 1e-3) / 1e6) < 1e-9 * mlups
