"""The multi-rank path on CPU: query sharding, max-over-ranks timing and the gather of
results, with world_size 2 gloo ranks solving their shards with the oracle.  The gathered
result must equal the single-rank solve bit for bit (each query is independent)."""
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
