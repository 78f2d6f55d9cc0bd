"""The multi-rank path on CPU: query sharding, the cost-balanced split of uneven batch
instances, max-over-ranks timing and the gathers of results, with world_size 2 gloo ranks
solving their shards with the oracle.  The gathered result must equal the single-rank
solve bit for bit (each query and each instance is independent)."""
import os
import socket

import numpy as np
import pytest

import oracle
from paper_2510_02635_gb300 import shard
from paper_2510_02635_gb300 import workloads as W

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")

W_SMALL = W.Workload("shard_test", "ac_manufactured", d=24, sigma=1.0, T=0.5, N=3, M=96, Q=5,
                     seed=8, x0_law="normal_1/d")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _solve(w, q):
    x0 = W.inputs(w)["x0"][q]
    r = oracle.solve(oracle.Problem(w.kind, w.d, w.sigma, w.T, w.N, w.M), x0, w.seed, q)
    return np.concatenate([[r["u0"]], r["grad"]])


def _worker(rank, world, port, out_path):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    first, count = shard.query_shard(W_SMALL.Q, rank, world)
    local = np.stack([_solve(W_SMALL, q) for q in range(first, first + count)])
    full = shard.gather_queries(local, W_SMALL.Q)
    t = shard.max_over_ranks(1.0 + rank)
    if rank == 0:
        np.save(out_path, full)
        with open(out_path + ".t", "w") as fh:
            fh.write(repr(t))
    dist.destroy_process_group()


def test_query_shard_partitions_exactly():
    for q, world in [(16, 1), (16, 2), (5, 2), (7, 4), (3, 8)]:
        got = [shard.query_shard(q, r, world) for r in range(world)]
        assert sum(c for _, c in got) == q
        assert [f for f, _ in got] == list(np.cumsum([0] + [c for _, c in got])[:-1])


def test_two_gloo_ranks_equal_single_rank(tmp_path):
    import torch.multiprocessing as mp
    out = str(tmp_path / "full.npy")
    mp.start_processes(_worker, args=(2, _free_port(), out), nprocs=2, join=True,
                       start_method="spawn")
    full = np.load(out)
    ref = np.stack([_solve(W_SMALL, q) for q in range(W_SMALL.Q)])
    assert np.array_equal(full, ref)
    assert float(open(out + ".t").read()) == 2.0


# uneven instances (d, M, N, kind differ), small enough for the oracle
def _small_batch():
    out = []
    for i, (d, M, N) in enumerate([(12, 40, 2), (30, 120, 3), (7, 24, 4), (40, 96, 2),
                                   (18, 64, 3), (5, 16, 2), (25, 200, 2), (9, 30, 3)]):
        kind, sigma, T = (("ac_manufactured", 1.0, 0.5) if i % 2 == 0
                          else ("logistic_grad", float(d), 1.0))
        out.append(W.Workload(f"shard_batch_{i}", kind, d=d, sigma=sigma, T=T, N=N, M=M, Q=1,
                              seed=9, x0_law="normal_1/d", extra={"index": i}))
    return out


def _solve_instance(w, i):
    x0 = W.inputs(w)["x0"][0]
    r = oracle.solve(oracle.Problem(w.kind, w.d, w.sigma, w.T, w.N, w.M), x0, w.seed, i)
    return np.concatenate([[r["u0"]], r["grad"]])


def _batch_worker(rank, world, port, out_path):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    batch = _small_batch()
    mine = shard.cost_shard(batch, world)[rank]
    local = {i: _solve_instance(batch[i], i) for i in mine}
    full = shard.gather_instances(local, len(batch))
    if rank == 0:
        np.save(out_path, np.concatenate(full))
    dist.destroy_process_group()


def test_cost_shard_covers_and_balances_the_512_instance_batch():
    """The 512-instance uneven batch over 2, 4 and 8 ranks: every instance exactly once,
    and the most loaded rank within 1% of the mean load (largest-first list scheduling;
    the largest single instance is far below a rank's share)."""
    batch = W.batch_instances()
    costs = np.array([shard.instance_cost(w) for w in batch])
    for world in (1, 2, 4, 8):
        parts = shard.cost_shard(batch, world)
        assert sorted(i for p in parts for i in p) == list(range(len(batch)))
        loads = np.array([costs[p].sum() for p in parts])
        assert loads.max() <= 1.01 * loads.mean()
    assert shard.cost_shard(batch, 4) == shard.cost_shard(list(batch), 4)   # deterministic


def test_two_gloo_ranks_cost_sharded_batch_equal_single_rank(tmp_path):
    import torch.multiprocessing as mp
    out = str(tmp_path / "batch.npy")
    mp.start_processes(_batch_worker, args=(2, _free_port(), out), nprocs=2, join=True,
                       start_method="spawn")
    full = np.load(out)
    ref = np.concatenate([_solve_instance(w, i) for i, w in enumerate(_small_batch())])
    assert np.array_equal(full, ref)
