"""Batches of independent matrices over ranks, one process per GPU.

Every matrix of a batch is its own problem, so the ranks exchange nothing
while they compute: each takes its share (``sharding.shard``: greedy
longest-processing-time on n^3), runs it, and the results can be gathered to
rank 0 afterwards (``torch.distributed.gather_object``, over NCCL or gloo).

``run_sharded`` is the host logic every rank calls; what a rank does with its
share is the ``compute`` argument:

  * ``batched_compute``: the persistent batched cos/sin launch (FP32,
    orders <= 256), one graph-captured plan per rank;
  * ``adjoint_compute``: the batched FP64 adjoint of the cos/sin loss;
  * anything else with the same signature (the CPU tests pass the oracle).
"""
from __future__ import annotations

import time

import numpy as np

from . import sharding


def _dist():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        return dist
    return None


def run_sharded(ns, make, compute, *, gather: bool = True, rank: int | None = None, world: int | None = None):
    """Run this rank's share of a batch and optionally gather to rank 0.

    ns       orders of the batch (host array); the batch's cost model is n^3.
    make     make(i) -> the inputs of matrix i (whatever ``compute`` takes).
    compute  compute(indices, inputs) -> (results, seconds): one result per
             index of this rank's share, and the time the rank spent on it.
    Returns a dict: "indices" (this rank's share), "results", "seconds", and on
    rank 0 with gather=True "all" (every result in batch order) and
    "seconds_max" (the slowest rank's time).
    """
    d = _dist()
    if rank is None:
        rank = d.get_rank() if d else 0
    if world is None:
        world = d.get_world_size() if d else 1
    mine = sharding.shard(ns, world, rank)
    inputs = [make(i) for i in mine]
    results, seconds = compute(mine, inputs)
    if len(results) != len(mine):
        raise RuntimeError("compute returned %d results for %d matrices" % (len(results), len(mine)))
    out = {"indices": mine, "results": results, "seconds": seconds}
    if not gather:
        return out
    if d is None or world == 1:
        out["all"] = list(results)
        out["seconds_max"] = seconds
        return out
    payload = (mine, results, seconds)
    got = [None] * world if rank == 0 else None
    d.gather_object(payload, got, dst=0)
    if rank == 0:
        everything = [None] * len(ns)
        slowest = 0.0
        for idx, res, sec in got:
            slowest = max(slowest, sec)
            for i, r in zip(idx, res):
                if everything[i] is not None:
                    raise RuntimeError("matrix %d computed twice" % i)
                everything[i] = r
        if any(r is None for r in everything):
            raise RuntimeError("some matrices were computed by no rank")
        out["all"] = everything
        out["seconds_max"] = slowest
    return out


def batched_compute(reps: int = 3, autotune: bool = True):
    """compute() for FP32 matrices on this rank's GPU: one graph-captured
    persistent plan over the share, timed over ``reps`` replays with CUDA
    events; results are (C, S, m, s) on the host."""
    def compute(indices, mats):
        import torch
        from . import api
        if not mats:
            return [], 0.0
        dev = [torch.as_tensor(np.ascontiguousarray(M), dtype=torch.float32).cuda() for M in mats]
        plan = api.BatchedPlan(dev, autotune=autotune)
        plan.launch()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            plan.launch()
        e1.record()
        torch.cuda.synchronize()
        api.device_status()
        if np.any(plan.status() != 0):
            raise RuntimeError("batched status: %s" % plan.status())
        infos = plan.infos()
        res = [(plan.C[k].cpu().numpy(), plan.S[k].cpu().numpy(), int(infos[k]["m"]), int(infos[k]["s"]))
               for k in range(len(mats))]
        plan.close()
        return res, e0.elapsed_time(e1) / 1e3 / reps
    return compute


def adjoint_compute(prec: str = "fp64"):
    """compute() for (A, G_C, G_S) FP64 triples of one order on this rank's
    GPU: one batched backward call over the share (wall clock around it);
    results are dA on the host."""
    def compute(indices, triples):
        import torch
        from . import api
        if not triples:
            return [], 0.0
        A = torch.as_tensor(np.stack([t[0] for t in triples])).cuda()
        GC = torch.as_tensor(np.stack([t[1] for t in triples])).cuda()
        GS = torch.as_tensor(np.stack([t[2] for t in triples])).cuda()
        api.cossin_backward(A, GC, GS, prec=prec)  # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        dA = api.cossin_backward(A, GC, GS, prec=prec)
        torch.cuda.synchronize()
        sec = time.perf_counter() - t0
        host = dA.cpu().numpy()
        return [host[k] for k in range(len(triples))], sec
    return compute
