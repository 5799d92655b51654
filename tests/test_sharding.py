"""Multi-rank host logic on CPU (gloo, world_size 2): batch sharding.

Each rank takes its share of a heterogeneous batch, computes it (here with
the CPU oracle, standing in for the rank's GPU), and rank 0 reassembles the
results in batch order from the ranks' records; nothing else is exchanged."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2010_00465_gb300 import inputs, sharding


def test_partition_covers_and_balances():
    ns, _, _ = inputs.batch_shapes(20000, index=3)
    for world in (1, 2, 4, 8):
        parts = sharding.lpt_partition(ns.astype(float) ** 3, world)
        flat = np.sort(np.concatenate([np.array(p, dtype=int) for p in parts]))
        assert np.array_equal(flat, np.arange(len(ns)))
        assert sharding.imbalance(ns, parts) < 1.001
    assert sharding.lpt_partition([5.0, 1.0, 1.0, 1.0, 1.0, 1.0], 2) == [[0], [1, 2, 3, 4, 5]]
    with pytest.raises(ValueError):
        sharding.lpt_partition([1.0], 0)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, count, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    ns, norms, fams = inputs.batch_shapes(count, n_lo=2, n_hi=24, index=5)
    mine = sharding.shard(ns, world, rank)
    records = []
    for i in mine:
        A = inputs.matrix(int(ns[i]), str(fams[i]), float(norms[i]), index=5, sub=i + 1)
        C, S, info = oracle.cossin(A, "single")
        records.append((i, C, S, info["m"], info["s"]))
    gathered = [None] * world
    dist.all_gather_object(gathered, records)
    if rank == 0:
        byidx = {}
        for recs in gathered:
            for rec in recs:
                assert rec[0] not in byidx
                byidx[rec[0]] = rec
        out["indices"] = sorted(byidx)
        # spot check against a single-process computation
        for i in (0, count // 2, count - 1):
            A = inputs.matrix(int(ns[i]), str(fams[i]), float(norms[i]), index=5, sub=i + 1)
            C, S, _ = oracle.cossin(A, "single")
            out[i] = bool(np.array_equal(C, byidx[i][1]) and np.array_equal(S, byidx[i][2]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_shards_reassemble():
    count = 64
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(2, port, count, out), nprocs=2, join=True)
        assert out["indices"] == list(range(count))
        assert out[0] and out[count // 2] and out[count - 1]
