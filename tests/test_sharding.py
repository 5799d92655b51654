"""Multi-rank host logic on CPU (gloo, world_size 2): batch sharding.

Each rank calls ``sharded.run_sharded`` -- the function the GPU ranks call --
with a compute step that runs the CPU oracle on its share (standing in for
the rank's batched GPU launch), and rank 0 reassembles the results in batch
order from the ranks' records; nothing else is exchanged."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2010_00465_gb300 import inputs, sharded, sharding


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


def _oracle_compute(indices, mats):
    import time

    import oracle
    t0 = time.perf_counter()
    res = []
    for A in mats:
        C, S, info = oracle.cossin(A, "single")
        res.append((C, S, info["m"], info["s"]))
    return res, time.perf_counter() - t0


def _make(ns, norms, fams):
    return lambda i: inputs.matrix(int(ns[i]), str(fams[i]), float(norms[i]), index=5, sub=i + 1)


def _worker(rank, world, port, count, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ns, norms, fams = inputs.batch_shapes(count, n_lo=2, n_hi=24, index=5)
    got = sharded.run_sharded(ns, _make(ns, norms, fams), _oracle_compute)
    out["share%d" % rank] = list(got["indices"])
    if rank == 0:
        out["n_all"] = len(got["all"])
        out["seconds_max"] = got["seconds_max"]
        # spot check against a single-process computation
        import oracle
        for i in (0, count // 2, count - 1):
            C, S, _ = oracle.cossin(_make(ns, norms, fams)(i), "single")
            out[i] = bool(np.array_equal(C, got["all"][i][0]) and np.array_equal(S, got["all"][i][1]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_shards_reassemble():
    count = 64
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(2, port, count, out), nprocs=2, join=True)
        ns, _, _ = inputs.batch_shapes(count, n_lo=2, n_hi=24, index=5)
        assert sorted(out["share0"] + out["share1"]) == list(range(count))
        assert out["share0"] == sharding.shard(ns, 2, 0) and out["share1"] == sharding.shard(ns, 2, 1)
        assert out["n_all"] == count and out["seconds_max"] > 0
        assert out[0] and out[count // 2] and out[count - 1]


def test_single_process_runs_the_whole_batch():
    ns, norms, fams = inputs.batch_shapes(6, n_lo=2, n_hi=8, index=6)
    got = sharded.run_sharded(ns, _make(ns, norms, fams), _oracle_compute)
    assert got["indices"] == list(range(6)) and len(got["all"]) == 6


def test_compute_must_cover_its_share():
    ns = np.array([3, 4, 5])
    with pytest.raises(RuntimeError):
        sharded.run_sharded(ns, lambda i: i, lambda idx, xs: ([], 0.0), rank=0, world=1)
