"""Host logic of the multi-rank batched run: the cost-balanced partition of independent
systems and the max-over-ranks timing, on CPU (gloo, world size 2)."""
import itertools
import os
import socket

import pytest

from paper_2601_18838_gb300 import shard


def _brute_opt(costs, m):
    best = float("inf")
    for assign in itertools.product(range(m), repeat=len(costs)):
        loads = [0.0] * m
        for c, r in zip(costs, assign):
            loads[r] += c
        best = min(best, max(loads))
    return best


def test_partition_covers_each_system_once():
    costs = [shard.system_cost(K, n) for K, n in [(32, 2000), (64, 50000), (48, 9000), (96, 3000), (32, 40000)] * 7]
    for m in (1, 2, 3, 4, 8, 64, 100):
        parts = shard.partition_lpt(costs, m)
        assert len(parts) == m
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(costs)))
        assert parts == shard.partition_lpt(costs, m)      # deterministic


@pytest.mark.parametrize("seed", range(6))
def test_lpt_within_graham_bound(seed):
    import numpy as np
    rng = np.random.default_rng(seed)
    costs = list(rng.uniform(1.0, 10.0, size=7))
    for m in (2, 3):
        got = shard.makespan(costs, shard.partition_lpt(costs, m))
        opt = _brute_opt(costs, m)
        assert got <= (4.0 / 3.0 - 1.0 / (3 * m)) * opt + 1e-12


def test_cost_orders_mesh_and_particles():
    assert shard.system_cost(64, 1000) > shard.system_cost(32, 1000)
    assert shard.system_cost(32, 50000) > shard.system_cost(32, 2000)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out_dir):
    import torch
    import torch.distributed as dist
    from paper_2601_18838_gb300 import shard as sh
    from paper_2601_18838_gb300 import workloads
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=ws)
    systems = workloads.batched()
    parts = sh.partition_lpt([sh.system_cost(s.K, s.n) for s in systems], ws)
    mine = parts[rank]
    gathered = [None] * ws
    dist.all_gather_object(gathered, mine)
    t = torch.tensor([float(1 + rank)], dtype=torch.float64)   # stand-in for each rank's timed ms
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as fh:
        fh.write(repr((gathered, t.item(), len(systems))))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_sharding_gloo(tmp_path):
    import torch.multiprocessing as mp
    ws = 2
    mp.start_processes(_worker, args=(ws, _free_port(), str(tmp_path)), nprocs=ws, join=True, start_method="spawn")
    res = [eval(open(tmp_path / f"r{r}.txt").read()) for r in range(ws)]
    gathered, tmax, n = res[0]
    assert all(r == res[0] for r in res)                     # every rank agrees
    flat = sorted(i for p in gathered for i in p)
    assert flat == list(range(n))                             # disjoint and complete
    assert tmax == float(ws)                                  # max over ranks
    from paper_2601_18838_gb300 import workloads
    systems = workloads.batched()
    costs = [shard.system_cost(s.K, s.n) for s in systems]
    loads = [sum(costs[i] for i in p) for p in gathered]
    assert max(loads) <= 1.05 * sum(costs) / ws + max(costs)  # balanced to within one system
