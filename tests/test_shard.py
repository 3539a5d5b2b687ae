"""Multi-rank host logic on CPU: the work partition, and the result gather and timing
reduction over a world-size-2 gloo process group (127.0.0.1)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1706_07413_b300 import shard


def test_instance_work_matches_step_rule():
    w = shard.instance_work([1025, 4097], 1.0)
    # dt = 1 / ceil(1 / (0.5 h)), h = pi / (2 (N - 1)): 1304 steps at N = 1025, 5216 at N = 4097
    assert w[0] == 1025 * 1304 and w[1] == 4097 * 5216


def test_partition_is_balanced_and_complete():
    rng = np.random.default_rng(0)
    work = rng.choice([1.0, 4.0, 16.0], size=193) * rng.uniform(0.5, 1.5, size=193)
    for world in (1, 2, 3, 8):
        parts = shard.partition(work, world)
        assert sorted(i for p in parts for i in p) == list(range(work.size))
        loads = [work[p].sum() for p in parts]
        assert max(loads) - min(loads) <= work.max() + 1e-9   # LPT bound
        for p in parts:
            assert p == sorted(p)


def test_partition_single_instance_and_empty_ranks():
    assert shard.partition([5.0], 4) == [[0], [], [], []]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        work = np.arange(1, 12, dtype=np.float64) ** 2
        parts = shard.partition(work, world)
        mine = parts[rank]
        # every rank "computes" per-instance results: 10 * index + rank marker in column 2
        local = np.stack([10.0 * np.asarray(mine), np.full(len(mine), float(rank))], axis=1)
        res = shard.gather_results(local, mine, work.size, dist, group=dist.new_group(backend="gloo"))
        t, w = shard.reduce_timing(0.5 + rank, float(work[mine].sum()), dist)
        q.put((rank, None if res is None else res.tolist(), t, w))
    finally:
        dist.destroy_process_group()


def test_gather_and_timing_over_gloo_world_size_2():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = {}
    for _ in procs:
        r, res, t, w = q.get(timeout=120)
        out[r] = (res, t, w)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    work = np.arange(1, 12, dtype=np.float64) ** 2
    parts = shard.partition(work, 2)
    res = np.asarray(out[0][0])
    assert out[1][0] is None
    assert np.array_equal(res[:, 0], 10.0 * np.arange(work.size))
    for r in range(2):
        assert np.all(res[parts[r], 1] == r)
        assert out[r][1] == 1.5 and out[r][2] == work.sum()


def test_bench_splits_one_global_batch_over_the_ranks():
    """bench.py under torchrun: each rank's share of a workload is a piece of one global batch of
    B x world instances (one seed), the shares partition it, and one rank gets the N = 1 batch."""
    import importlib.util
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(root, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    one, idx1, _ = bench.workload_insts("amp_scan", 0, 1)
    assert idx1 == list(range(256)) and [it.eps for it in one] == [it.eps for it in bench.W.amp_scan()]
    for name in ("amp_scan", "uneven"):
        shares = [bench.workload_insts(name, r, 2) for r in range(2)]
        allidx = sorted(i for s in shares for i in s[1])
        assert allidx == list(range(2 * len(one if name == "amp_scan" else bench.W.uneven())))
        assert abs(len(shares[0][0]) - len(shares[1][0])) <= (0 if name == "amp_scan" else 40)
        glob = bench.WORKLOADS[name][0](B=len(allidx), seed=bench.WORKLOADS[name][2])
        for insts, idx, _ in shares:
            assert [it.N for it in insts] == [glob[i].N for i in idx]
