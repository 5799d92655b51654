"""Benchmark: simultaneous matrix cos/sin on GB300.

One step = the n = 4096 single-matrix workload: dense N(0,1) matrices with
||A||_1 in {2^-4, 1, 8, 64}, plus a symmetric (A + A^T)/2 and a non-normal
upper-triangular (strict upper part x10) matrix at ||A||_1 = 8, each through
the FP64 path (double table) and, where built, the FP32 path (single table).
Every matrix is an independent problem, so with N GPUs every rank runs the
whole set (weak scaling, no collective on the data path).

Prints one JSON line: the device-timed throughput, the same metric end to
end through the public API with host buffers, the dominant kernel's
roofline, the oracle on the host cores, and the other forms (precisions,
batched, adjoint, c/s) with their errors.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N = 4096
NORMS = [2.0 ** -4, 1.0, 8.0, 64.0]
EXTRA = [("symmetric", 8.0), ("triangular", 8.0)]
METRIC = "cos+sin TFLOP/s & matrices/s (n=4096, batched) at stated error vs FP64 oracle"
WORKLOAD = ("n=4096 single matrices: N(0,1) at ||A||_1 in {2^-4,1,8,64} + symmetric and "
            "upper-triangular(x10) at ||A||_1=8")


def cases(precisions):
    out = []
    for prec in precisions:
        for nrm in NORMS:
            out.append((prec, "normal", nrm))
        for fam, nrm in EXTRA:
            out.append((prec, fam, nrm))
    return out


def make_input(fam, nrm, prec):
    from paper_2010_00465_gb300 import inputs
    A = inputs.matrix(N, fam, nrm, index=1)
    return A.astype(np.float32) if prec == "fp32" else A


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        # raw samples (the JSON line carries their summary); COSSIN_CLOCK_LOG_DIR
        # chooses where they go
        log_dir = os.environ.get("COSSIN_CLOCK_LOG_DIR", os.path.join(ROOT, "_clocks"))
        self.path = os.path.join(log_dir, "clocks_rank%d.csv" % gpu_index)

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.fh,
                stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        busy = [v for v in sm if v >= 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(busy), "sm_max_mhz": max(smax), "samples": len(sm),
                "reasons": sorted(reasons)}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def cpu_baseline(gpu_results=None):
    """The oracle as it stands, on the host cores, on one matrix of the
    headline workload: the n = 4096 N(0,1) FP64 matrix at ||A||_1 = 2^-4
    (double table: 2m = 8, s = 0, 4 products, 0.55 TFLOP), about half a
    minute on 16 cores.  With the GPU results of that matrix (FP64 and FP32
    paths) their relative Frobenius error against this oracle result is
    returned beside the timing (the FP32 path's against the double-table
    oracle, i.e. against the function, at its own single-table (m, s))."""
    import oracle
    oracle.build()
    A = make_input("normal", 2.0 ** -4, "fp64")
    t0 = time.perf_counter()
    Co, So, info = oracle.cossin(A)
    dt = time.perf_counter() - t0
    flops = 2.0 * N ** 3 * info["products"]
    out = {"value": flops / dt / 1e12, "unit": "TFLOP/s", "cores": oracle.threads(), "kind": "oracle",
           "sample": "one oracle cos/sin of the n=%d FP64 N(0,1) matrix at ||A||_1=2^-4 of the headline workload "
                     "((2m, s) = (%d, %d), %d products), %.1f s" % (N, info["m"], info["s"], info["products"], dt),
           "matrices_per_s": 1.0 / dt}
    errs = {}
    for prec, (C, S) in (gpu_results or {}).items():
        Cg = C.double().cpu().numpy()
        Sg = S.double().cpu().numpy()
        errs[prec] = max(float(np.linalg.norm(Cg - Co) / np.linalg.norm(Co)),
                         float(np.linalg.norm(Sg - So) / np.linalg.norm(So)))
    out["gpu_rel_err_vs_this_oracle_result"] = errs
    return out


def run_reference(args):
    """The reference arm: the oracle (the paper's method as a plain FP64 CPU
    program), on the host cores, one n = 2048 N(0,1) FP64 matrix at
    ||A||_1 = 2^-4 per step (the headline workload's family and norm at a
    quarter of its size, 4 products, a few seconds a step)."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    from paper_2010_00465_gb300 import inputs
    oracle.build()
    n = 2048
    A = inputs.matrix(n, "normal", 2.0 ** -4, index=1)
    for _ in range(args.warmup):
        oracle.cossin(A)
    times, flops = [], 0.0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        _, _, info = oracle.cossin(A)
        times.append(time.perf_counter() - t0)
        flops += 2.0 * n ** 3 * info["products"]
    total = sum(times)
    val = flops / total / 1e12
    sample = "one oracle cos/sin of a 2048x2048 FP64 N(0,1) matrix, ||A||_1=2^-4, per step"
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "TFLOP/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "sample": sample},
            "cpu_baseline": {"value": val, "unit": "TFLOP/s", "cores": oracle.threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": val, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precisions", default=None, help="comma list: fp64,fp32")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip the split-precision comparison")
    ap.add_argument("--ncu-case", default=None, choices=["gemm_tf32", "gemm_f64", "norm1", "batched", "batched256", "gemm_emu"],
                    help="run one small launch set for an ncu capture and exit")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.ncu_case:
        return ncu_case(args.ncu_case)

    import torch
    import torch.distributed as dist

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2010_00465_gb300 import api, _lib

    precs = args.precisions.split(",") if args.precisions else ["fp64", "fp32"]
    work = cases(precs)
    # inputs resident in HBM, outputs and workspace preallocated
    dev_in = [torch.from_numpy(make_input(f, r, p)).to(dev) for p, f, r in work]
    outs = [(torch.empty_like(a), torch.empty_like(a)) for a in dev_in]
    wsz = max(api.workspace_size(N, p) for p in precs)
    wsp = torch.empty(wsz, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    infos = []

    case_ms = []

    def step(record=False):
        for (p, f, r), A, (C, S) in zip(work, dev_in, outs):
            if record:
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(torch.cuda.current_stream())
            _, _, info = api.cossin(A, p, workspace=wsp, out=(C, S), return_info=True)
            if record:
                e1.record(torch.cuda.current_stream())
                e1.synchronize()
                case_ms.append(e0.elapsed_time(e1))
                infos.append(info)

    for _ in range(max(args.warmup, 0)):
        step()
    torch.cuda.synchronize()
    flops_per_step = 0.0
    step(record=True)
    torch.cuda.synchronize()
    flops_per_step = sum(i["flops"] for i in infos)
    launches_per_step = sum(launches_of(p, i) for (p, _, _), i in zip(work, infos))

    # the FP64 roofline's denominator, measured on this GPU (register-only FMAs)
    fp64_probe = max(api.fp64_fma_rate() for _ in range(3))
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count

    api.prof_reset()
    api.prof_enable(True)
    with ClockSampler(local) as clk:
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(args.steps):
            step()
        ev1.record(stream)
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
    api.prof_enable(False)
    api.device_status()  # no bounded wait of a tensor-core kernel expired in the timed region
    ms = ev0.elapsed_time(ev1)
    if ws > 1:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    kern = {k: api.prof_read(k) for k in ("norm1", "gemm_f64", "gemm_tf32", "gemm_emu", "other")}

    # end to end through the public API with host buffers (pinned), copies inside
    host_in = [torch.from_numpy(make_input(f, r, p)).pin_memory() for p, f, r in work]
    host_out = [(torch.empty(a.shape, dtype=a.dtype, pin_memory=True),
                 torch.empty(a.shape, dtype=a.dtype, pin_memory=True)) for a in host_in]
    h2d = sum(a.numel() * a.element_size() for a in host_in)
    d2h = 2 * h2d
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_steps = max(1, min(args.steps, 2))
    for _ in range(e2e_steps):
        for (p, _, _), A, o in zip(work, host_in, host_out):
            C, S = api.cossin(A, p, workspace=wsp, out=o)  # results land in pinned host buffers
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0

    # accuracy stated beside the number: the 64 x 64 workload against the oracle,
    # and cos^2 + sin^2 - I at n = 4096
    acc = accuracy(api, dev_in, outs, work)

    # the same workload and metric with the FP64 matrices on the emulated FP64
    # products (CS_FP64_EMU), and how far its results are from the native ones
    alt = None
    if "fp64" in precs and not args.no_forms:
        emu_work = [("fp64_emu" if p == "fp64" else p) for p, _, _ in work]
        wse = torch.empty(max(api.workspace_size(N, p) for p in emu_work), dtype=torch.uint8, device=dev)
        emu_outs = [(torch.empty_like(a), torch.empty_like(a)) for a in dev_in]

        def emu_step():
            for p, A, (C, S) in zip(emu_work, dev_in, emu_outs):
                api.cossin(A, p, workspace=wse, out=(C, S))

        for _ in range(max(args.warmup, 0)):
            emu_step()
        torch.cuda.synchronize()
        ea = torch.cuda.Event(enable_timing=True)
        eb = torch.cuda.Event(enable_timing=True)
        ea.record(stream)
        for _ in range(args.steps):
            emu_step()
        eb.record(stream)
        torch.cuda.synchronize()
        ems = ea.elapsed_time(eb)
        diff = 0.0
        for (p, _, _), (C, S), (Ce, Se) in zip(work, outs, emu_outs):
            if p == "fp64":
                diff = max(diff, float((Ce - C).norm() / C.norm()), float((Se - S).norm() / S.norm()))
        alt = {"value": flops_per_step * args.steps / (ems / 1e3) / 1e12, "unit": "TFLOP/s",
               "ms_per_step": ems / args.steps, "speedup_vs_value": ms / ems,
               "max_rel_diff_vs_native_fp64_results": diff,
               "note": "same 12 matrices and metric; the six FP64 matrices through CS_FP64_EMU (FP64 products "
                       "emulated on the BF16 tensor cores, per-product error below the native FP64 kernel's)"}
        del wse, emu_outs

    total_flops = flops_per_step * args.steps * ws
    value = total_flops / (ms / 1e3) / 1e12
    dominant = max(("gemm_f64", "gemm_emu"), key=lambda k: kern[k][0])
    clocks = clk.summary()
    pk, pk_kind = peaks()
    pk["fp64_probe_tflops"] = fp64_probe
    pk["sm_count"] = sm_count
    roof = roofline(dominant, *kern[dominant], pk, pk_kind, clocks)
    other = "gemm_emu" if dominant == "gemm_f64" else "gemm_f64"
    roof_other = roofline(other, *kern[other], pk, pk_kind, clocks)
    norm_ms, norm_n, norm_bytes = kern["norm1"]
    roof_norm = None
    if norm_n:
        gbs = norm_bytes / (norm_ms / 1e3) / 1e9
        roof_norm = {"bound": "hbm", "achieved": gbs, "peak": pk["hbm_gbs"], "unit": "GB/s",
                     "frac": gbs / pk["hbm_gbs"], "traffic": None,
                     "note": "two kernels per call (column partials + finish); bytes = n^2 x element size"}
    line = {
        "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "+".join("f64" if p == "fp64" else "f32" for p in precs),
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": N, "precisions": precs, "matrices_per_step": len(work),
                   "l2": "inputs > L2: each step reads %d matrices of %d MB and streams GBs of workspace"
                         % (len(work), N * N * 8 // 2 ** 20)},
        "matrices_per_s": len(work) * args.steps * ws / (ms / 1e3),
        "roofline": roof,
        "roofline_other_kernels": {other: roof_other, "norm1": roof_norm},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clocks,
        "e2e": {"value": flops_per_step * e2e_steps / e2e_s / 1e12, "unit": "TFLOP/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "accuracy": acc,
        "alt_fp64_emu": alt,
        "per_case": [{"prec": p, "family": f, "norm1": r, "m": i["m"], "s": i["s"], "products": i["products"],
                      "ms": t, "alg_tflops": i["flops"] / t / 1e9,
                      "rel_diff_vs_fp64_path": acc.get("%s_vs_fp64_path_%s_norm%g" % (p, f, r), 0.0 if p == "fp64" else None)}
                     for (p, f, r), i, t in zip(work, infos, case_ms)],
        "kernels": {k: {"ms": v[0], "launches": v[1], "work": v[2]} for k, v in kern.items()},
    }
    if ws > 1 and not args.no_forms:
        # every matrix of a batch is independent: the batched workload and
        # the adjoint's control workload split over the ranks (no collective
        # while computing; results gathered to rank 0 afterwards)
        sh = sharded_forms()
        if rank == 0:
            line["sharded"] = sh
    if rank == 0 and not args.no_forms:
        line["forms"] = forms(api, wsp)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        head = {p: o for (p, f, r), o in zip(work, outs) if f == "normal" and r == 2.0 ** -4}
        line["cpu_baseline"] = cpu_baseline(head)
        line["accuracy"]["n4096_norm2^-4_rel_err_vs_oracle"] = line["cpu_baseline"]["gpu_rel_err_vs_this_oracle_result"]
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()
    return 0


def sharded_forms(count=20000, adj_count=512, adj_n=128):
    """With N ranks: the 20,000-matrix batched workload and the 512-matrix
    adjoint workload, each split over the ranks by sharding.shard (LPT on
    n^3), each rank's share one batched launch; the time is the slowest
    rank's, the rate the whole batch over it (strong scaling: the batch is
    fixed as N grows)."""
    from paper_2010_00465_gb300 import inputs, sharded
    ns, norms, fams = inputs.batch_shapes(count, index=3)
    make = lambda i: inputs.matrix(int(ns[i]), str(fams[i]), float(norms[i]), index=3, sub=i + 1).astype(np.float32)
    b = sharded.run_sharded(ns, make, sharded.batched_compute())
    A, GC, GS = inputs.hamiltonian_batch(adj_count, adj_n)
    a = sharded.run_sharded(np.full(adj_count, adj_n), lambda i: (A[i], GC[i], GS[i]), sharded.adjoint_compute())
    out = {"scaling": "strong", "partition": "greedy LPT on n^3 (sharding.shard)"}
    if "seconds_max" in b:
        out["batched"] = {"count": count, "ms_slowest_rank": 1e3 * b["seconds_max"],
                          "matrices_per_s": count / b["seconds_max"]}
        out["adjoint"] = {"count": adj_count, "n": adj_n, "ms_slowest_rank": 1e3 * a["seconds_max"],
                          "matrices_per_s": adj_count / a["seconds_max"]}
    return out


def forms(api, wsp):
    """The other precisions at n = 4096 and 8192 against the plain FP64 path on the same
    FP64 input: FP64 with every product emulated on the BF16 tensor cores,
    split precision (Taylor chain as four-pass TF32 products) with native or
    emulated FP64 double-angle products, and split precision on the BF16
    tensor cores alone (four-slice chain products, eight-slice double-angle
    products); each with its relative difference to the FP64 path stated
    beside it."""
    import torch
    from paper_2010_00465_gb300 import inputs
    out = {}
    precs = ("fp64", "fp64_emu", "split_tf32", "split_emu", "split_bf16")
    for n_, nrm in [(N, 1.0), (N, 16.0), (N, 64.0), (2 * N, 1.0), (2 * N, 16.0), (2 * N, 64.0)]:
        A = torch.from_numpy(inputs.matrix(n_, "normal", nrm, index=2)).cuda()
        row = {}
        res = {}
        for prec in precs:
            need = api.workspace_size(n_, prec)
            ws = wsp if wsp.numel() >= need else torch.empty(need, dtype=torch.uint8, device="cuda")
            if n_ == N:  # warm-up (the n = 8192 rows reuse the warmed kernels)
                api.cossin(A, prec, workspace=ws)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            C, S, info = api.cossin(A, prec, workspace=ws, return_info=True)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            res[prec] = (C, S)
            row[prec] = {"ms": ms, "m": info["m"], "s": info["s"], "alg_tflops": info["flops"] / ms / 1e9}
        C64, S64 = res["fp64"]
        for prec in precs[1:]:
            Cp, Sp = res[prec]
            row[prec]["rel_diff_vs_fp64_path"] = max(float((Cp - C64).norm() / C64.norm()),
                                                     float((Sp - S64).norm() / S64.norm()))
            row[prec]["speedup_vs_fp64_path"] = row["fp64"]["ms"] / row[prec]["ms"]
        out["n%d_norm%g" % (n_, nrm)] = row
        del A, res
        torch.cuda.empty_cache()
    return {"n": [N, 2 * N], "family": "normal", "precisions": out, "fp64_emu_product": emu_product_form(api),
            "bf16x4_product": emu_product_form(api, prec="split_bf16"),
            "tf32x4_product": emu_product_form(api, prec="split_tf32"),
            "batched": batched_form(api), "adjoint": adjoint_form(api), "cs": cs_form(api, wsp)}


def emu_product_form(api, reps=5, prec="fp64_emu"):
    """One n = 4096 tensor-core product: on the BF16 tensor cores from 7-bit
    slices, eight (prec "fp64_emu", 36 slice products, FP64-class) or four
    (prec "split_bf16", 10 slice products, FP32-class), or the four-pass TF32
    product of (hi, lo) splits (prec "split_tf32").  The kernel's time from
    its own CUDA events, the work it issues against the tensor peak, the FP64
    rate it stands for, and its difference to the native FP64 product."""
    import torch
    from paper_2010_00465_gb300 import inputs
    pairs = {"fp64_emu": 36, "split_bf16": 10, "split_tf32": 4}[prec]
    X = torch.from_numpy(inputs.matrix(N, "normal", None, index=1)).cuda()
    Y = torch.from_numpy(inputs.matrix(N, "normal", None, index=5)).cuda()
    P = api.matmul(X, Y, prec)
    P64 = api.matmul(X, Y, "fp64")
    torch.cuda.synchronize()
    rel = float((P - P64).norm() / P64.norm())
    del P, P64
    api.prof_reset()
    api.prof_enable(True)
    t0 = time.perf_counter()
    for _ in range(reps):
        api.matmul(X, Y, prec)
    torch.cuda.synchronize()
    call_ms = (time.perf_counter() - t0) * 1e3 / reps
    api.prof_enable(False)
    tf32 = prec == "split_tf32"
    ms, launches, work = api.prof_read("gemm_tf32" if tf32 else "gemm_emu")
    kms = ms / max(launches, 1)
    pk, pk_kind = peaks()
    issued = pairs * 2.0 * N ** 3 / (kms / 1e3) / 1e12
    native = 2.0 * N ** 3
    key = {"fp64_emu": "ozaki_kernel", "split_bf16": "ozaki_kernel_s4", "split_tf32": "gemm_tf32_kernel"}[prec]
    if tf32:
        # TF32 has no measured peak here: the BF16 burst scaled by the nominal
        # dense ratio 1.1 / 2.25 PFLOP/s
        peak = pk["bf16_tflops"] * 1.1 / 2.25
        note = ("4 TF32 passes per product (hi*hi, lo*hi, hi*lo, lo*lo); peak = cuBLAS BF16 burst x 1.1/2.25 "
                "(nominal TF32/BF16 dense ratio), " + pk_kind)
    else:
        peak = pk["bf16_tflops"]
        note = "%d BF16 slice products per product; peak = cuBLAS BF16 burst, " % pairs + pk_kind
    return {"n": N, "prec": prec, "kernel_ms": kms, "call_ms_with_slicing_and_alloc": call_ms,
            "fp64_equivalent_tflops": native / (kms / 1e3) / 1e12, "rel_diff_vs_fp64_product": rel,
            "roofline": {"bound": "tensor", "achieved": issued, "peak": peak, "unit": "TFLOP/s",
                         "frac": issued / peak, "traffic": traffic_of(key), "note": note}}


def cs_form(api, wsp):
    """The Sec. 2.2 variant at n = 4096: c(t^2 A), s(t, A) of A = X^2 (t = 1)
    against cos(X), sin(X) of the cos/sin path, both timed with CUDA events;
    the variant starts from B = A and drops the sine's last product."""
    import torch
    from paper_2010_00465_gb300 import inputs
    out = {}
    for nrm in (1.0, 8.0):
        X = torch.from_numpy(inputs.matrix(N, "normal", nrm, index=4)).cuda()
        A = X @ X
        for prec in ("fp64", "split_tf32"):
            need = api.workspace_size(N, prec)
            ws = wsp if wsp.numel() >= need else torch.empty(need, dtype=torch.uint8, device="cuda")
            row = {}
            res = {}
            for name, call in (("cossin", lambda: api.cossin(X, prec, workspace=ws, return_info=True)),
                               ("cs", lambda: api.cossin_cs(A, 1.0, prec, workspace=ws, return_info=True))):
                call()
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                C, S, info = call()
                e1.record()
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1)
                res[name] = C
                row[name] = {"ms": ms, "m": info["m"], "s": info["s"], "products": info["products"],
                             "alg_tflops": info["flops"] / ms / 1e9}
            row["rel_diff_c_vs_cos"] = float((res["cs"] - res["cossin"]).norm() / res["cossin"].norm())
            row["speedup_vs_cossin"] = row["cossin"]["ms"] / row["cs"]["ms"]
            out["normX%g_%s" % (nrm, prec)] = row
    return out


def adjoint_form(api, count=512, n=128, reps=3):
    """The control workload: 512 FP64 matrices n = 128, A = H0 + sum u_k H_k,
    random cotangents; one batched backward call (forward recomputed with its
    tape, then the reverse pass), with native and with emulated FP64
    products.  Work = 2 n^3 (3 Pi_2m + 6 s) per matrix."""
    import torch
    import oracle
    from paper_2010_00465_gb300 import inputs
    A, GC, GS = inputs.hamiltonian_batch(count, n)
    Ad, GCd, GSd = (torch.from_numpy(x).cuda() for x in (A, GC, GS))
    out = {"count": count, "n": n}
    res = {}
    for prec in ("fp64", "fp64_emu"):
        api.cossin_backward(Ad, GCd, GSd, prec=prec)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            dA, infos = api.cossin_backward(Ad, GCd, GSd, return_info=True, prec=prec)
        torch.cuda.synchronize()
        sec = (time.perf_counter() - t0) / reps
        flops = sum(i["flops"] for i in infos)
        b = 7
        m, s = infos[b]["m"], infos[b]["s"]
        ref = oracle.gradient(A[b], GC[b], GS[b], m, s)
        err = float(np.linalg.norm(dA[b].cpu().numpy() - ref) / np.linalg.norm(ref))
        res[prec] = {"ms_per_call": sec * 1e3, "alg_tflops": flops / sec / 1e12,
                     "rel_err_vs_oracle_block_frechet_matrix7": err}
        out["ms_pairs"] = sorted({(i["m"], i["s"]) for i in infos})
    out.update(res["fp64"])
    out["fp64_emu"] = res["fp64_emu"]
    out["fp64_emu"]["speedup_vs_fp64"] = res["fp64"]["ms_per_call"] / res["fp64_emu"]["ms_per_call"]
    return out


def batched_form(api, count=20000, reps=5):
    """The batched workload: 20,000 FP32 matrices, n log-uniform in [8, 256],
    ||A||_1 log-uniform in [2^-6, 2^6], half symmetric, in one graph-captured
    persistent launch (autotuned).  Against it: the plain FP64 GPU path, one
    cossin call per matrix over the whole batch (each call's 1-norm read is a
    host round trip), timed end to end."""
    import torch
    import oracle
    from paper_2010_00465_gb300 import inputs
    ns, norms, fams = inputs.batch_shapes(count, index=3)
    host = [inputs.matrix(int(ns[i]), str(fams[i]), float(norms[i]), index=3, sub=i + 1).astype(np.float32)
            for i in range(count)]
    dev = [torch.from_numpy(M).cuda() for M in host]
    plan = api.BatchedPlan(dev, autotune=True)
    for _ in range(2):
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
    assert np.all(plan.status() == 0)
    ms = e0.elapsed_time(e1) / reps
    infos = plan.infos()
    flops = float(infos["flops"].sum())
    # accuracy: the largest orders, the largest norms and a random set
    # against the oracle (single table, same (m, s))
    g = inputs.rng(3, 77)
    errs = []
    sample = list(np.argsort(-ns)[:2]) + list(np.argsort(-norms)[:3]) + list(g.choice(count, 6, replace=False))
    for i in sample:
        A = host[i].astype(np.float64)
        Co, So, _ = oracle.cossin(A, "single", m=int(infos[i]["m"]), s=int(infos[i]["s"]))
        C = plan.C[i].double().cpu().numpy()
        S = plan.S[i].double().cpu().numpy()
        errs.append(max(float(np.linalg.norm(C - Co) / np.linalg.norm(Co)),
                        float(np.linalg.norm(S - So) / max(np.linalg.norm(So), 1e-300))))
    variant = plan.variant()
    plan.close()
    # the plain FP64 GPU path on every matrix of the batch
    d64 = [torch.from_numpy(M.astype(np.float64)).cuda() for M in host]
    nmax = int(max(ns))
    flat = torch.empty(2 * nmax * nmax, dtype=torch.float64, device="cuda")
    wsf = torch.empty(api.workspace_size(nmax, "fp64"), dtype=torch.uint8, device="cuda")

    def plain(A):
        n = A.shape[0]
        api.cossin(A, "fp64", workspace=wsf, out=(flat[: n * n].view(n, n), flat[n * n: 2 * n * n].view(n, n)),
                   check_device=False)

    for A in d64[:8]:
        plain(A)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for A in d64:
        plain(A)
    torch.cuda.synchronize()
    t64 = time.perf_counter() - t0
    api.device_status()
    del d64, flat, wsf
    return {"count": count, "ms_per_batch": ms, "matrices_per_s": count / (ms / 1e3),
            "alg_tflops": flops / (ms / 1e3) / 1e12, "alg_gflop_per_batch": flops / 1e9,
            "autotuned_variant": variant,
            "max_rel_err_vs_oracle_sample": max(errs), "sample_size": len(errs),
            "sample": "2 largest orders, 3 largest norms, 6 random",
            "fp64_plain_path_ms": 1e3 * t64,
            "fp64_plain_path_method": "all %d matrices through cossin(fp64), one call each, wall clock" % count,
            "speedup_vs_fp64_plain_path": 1e3 * t64 / ms,
            "roofline": batched_roofline(flops, ms)}


def batched_roofline(flops, ms):
    """The batched kernel against the tensor pipe it issues its products to:
    every product is ten BF16 slice products (four slices per operand, p + q
    <= 3), so the issued work is 10x the algorithmic; the peak is the measured
    sustained BF16 rate.  The kernel is bound by the CUDA-core work around the
    products (slicing, double-float epilogues), which this fraction shows."""
    pk, pk_kind = peaks()
    issued = 10.0 * flops / (ms / 1e3) / 1e12
    return {"bound": "tensor", "achieved": issued, "peak": pk["bf16_tflops_sustained"], "unit": "TFLOP/s",
            "frac": issued / pk["bf16_tflops_sustained"], "traffic": traffic_of("batched_kernel"),
            "kernel": "batched_kernel<128, 512>",
            "note": "10 BF16 slice products per product; peak = sustained bf16, " + pk_kind +
                    "; bound in practice by CUDA-core issue (slicing, double-float epilogues)"}


def ncu_case(name):
    """A few launches of one kernel at n = 4096 (inputs larger than L2) for an
    ncu capture; prints nothing on success."""
    import torch
    from paper_2010_00465_gb300 import api, inputs
    if name == "gemm_tf32":
        # the four-pass TF32 chain of the split form
        A = torch.from_numpy(inputs.matrix(N, "normal", 1.0, index=1)).cuda()
        api.cossin(A, "split_tf32")
    elif name == "batched":
        # 2,000 matrices of the batched workload's distribution, one launch
        ns, norms, fams = inputs.batch_shapes(2000, index=3)
        dev = [torch.from_numpy(inputs.matrix(int(ns[i]), str(fams[i]), float(norms[i]), index=3,
                                              sub=i + 1).astype(np.float32)).cuda() for i in range(2000)]
        plan = api.BatchedPlan(dev, autotune=False)
        plan.launch()
        torch.cuda.synchronize()
        plan.close()
    elif name == "batched256":
        # 304 matrices of order 256 (the largest of the batched workload), one launch
        dev = [torch.from_numpy(inputs.matrix(256, "normal", 8.0, index=3, sub=i + 1).astype(np.float32)).cuda()
               for i in range(304)]
        plan = api.BatchedPlan(dev, autotune=False)
        plan.launch()
        torch.cuda.synchronize()
        plan.close()
    elif name == "gemm_f64":
        # the headline FP64 matrix at ||A||_1 = 2^-4: (2m, s) = (8, 0), four
        # products through the cos/sin workspace (last wave split over K)
        A = torch.from_numpy(inputs.matrix(N, "normal", 2.0 ** -4, index=1)).cuda()
        api.cossin(A, "fp64")
    elif name == "gemm_emu":
        # one n = 4096 FP64 product emulated on the BF16 tensor cores (eight
        # slices), then one four-slice product
        X = torch.from_numpy(inputs.matrix(N, "normal", 1.0, index=1)).cuda()
        api.matmul(X, X, "fp64_emu")
        api.matmul(X, X, "split_bf16")
    else:
        A = torch.from_numpy(inputs.matrix(2 * N, "normal", 1.0, index=1)).cuda()
        api.norm1(A)
    torch.cuda.synchronize()
    return 0


def launches_of(prec, info, n=None):
    """Kernels one cossin call launches: the 1-norm (2); then Pi_2m chain
    products and s double-angle products (one stacked 2n x n x n product each;
    info["products"] counts those twice).  FP64: one or two kernels per
    product (two when the last wave of tiles is split over K, as the library
    reports); FP32: the input conversion, per product the emulated product's
    five slicing kernels, a memset and the product kernel, and the two output
    conversions."""
    s = info["s"]
    chain = info["products"] - 2 * s
    if prec == "fp64":
        from paper_2010_00465_gb300 import api
        n = n or N
        return 2 + chain * api.fp64_product_launches(n, n, n) + s * api.fp64_product_launches(2 * n, n, n)
    return 2 + 1 + 7 * (chain + s) + 2


def traffic_of(kernel):
    """DRAM bytes per launch from the committed ncu summary, only while the
    kernel source is unchanged since the capture (else None)."""
    import hashlib
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    rec = json.load(open(p)).get(kernel)
    if not rec:
        return None
    src = os.path.join(ROOT, rec["source"])
    if not os.path.exists(src) or hashlib.sha256(open(src, "rb").read()).hexdigest()[:16] != rec["sha256_16"]:
        return None
    return rec["read_bytes"] + rec["write_bytes"]


def roofline(kind, ms, launches, work, pk, pk_kind, clocks):
    """achieved = algorithmic flops per launch / average launch time (CUDA
    events around every launch on the launch stream, inside the timed region)."""
    if launches == 0 or ms <= 0:
        return None
    per_launch_s = ms / 1e3 / launches
    achieved = work / launches / per_launch_s / 1e12
    if kind == "gemm_f64":
        # FP64 FMA units: measured by the register-only probe in this run;
        # the nominal 2 FMA/clk/SM x SMs x clock beside it
        mhz = clocks.get("sm_mhz") or 2070.0
        sms = pk.get("sm_count", 152)
        nominal = 2 * 2 * sms * mhz * 1e6 / 1e12
        peak = pk.get("fp64_probe_tflops") or nominal
        return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic_of("gemm_f64_kernel"), "kernel": "gemm_f64_kernel",
                "peak_note": "measured: cossin_fp64_fma_rate (16 independent FP64 FMA chains per thread, %d SMs x 4 "
                             "CTAs x 256 threads, best of 3) in this run, %.4f TFLOP/s; nominal 2 FMA/clk/SM x %d "
                             "SMs x median SM clock under load (%.0f MHz) = %.4f" % (sms, peak, sms, mhz, nominal)}
    if kind == "gemm_emu":
        # the headline step's emulated products are the FP32 path's four-slice
        # BF16 products: 10 slice products per algorithmic product
        bf16 = pk.get("bf16_tflops_sustained", pk.get("bf16_tflops"))
        issued = achieved * 10
        return {"bound": "tensor", "achieved": issued, "peak": bf16, "unit": "TFLOP/s", "frac": issued / bf16,
                "traffic": traffic_of("ozaki_kernel_s4"), "kernel": "ozaki_kernel<4>",
                "peak_note": "%s sustained bf16 (the kernel runs inside a long step); achieved counts the 10 "
                             "BF16 slice products of each product" % pk_kind, "algorithmic_tflops": achieved}
    # TF32 tensor: half the bf16 rate (nominal 1.1 vs 2.25 PFLOP/s); four passes per product
    bf16 = pk.get("bf16_tflops_sustained", pk.get("bf16_tflops"))
    peak = bf16 * 1100.0 / 2250.0
    issued = achieved * 4
    return {"bound": "tensor", "achieved": issued, "peak": peak, "unit": "TFLOP/s", "frac": issued / peak,
            "traffic": traffic_of("gemm_tf32_kernel"), "kernel": "gemm_tf32_kernel",
            "peak_note": "%s sustained bf16 x nominal tf32/bf16 ratio; achieved counts the 4 TF32 passes"
                         % pk_kind, "algorithmic_tflops": achieved}


def accuracy(api, dev_in, outs, work):
    import torch
    import oracle
    from paper_2010_00465_gb300 import inputs
    res = {}
    A = inputs.matrix(64, "normal", 2.0, index=0)
    Co, So, _ = oracle.cossin(A)
    Ad = torch.from_numpy(A).cuda()
    C, S = api.cossin(Ad, "fp64")
    # the 64 x 64 configuration's latency per call (norm, its one host
    # synchronisation, 9 products), median of 50
    ts = []
    for _ in range(50):
        t0 = time.perf_counter()
        api.cossin(Ad, "fp64")
        torch.cuda.synchronize()
        ts.append(time.perf_counter() - t0)
    res["fp64_64x64_latency_us"] = float(np.median(ts) * 1e6)
    # the same call at the C ABI with caller-provided workspace and outputs
    # (no Python-side allocation), median of 200
    import ctypes
    from paper_2010_00465_gb300 import _lib
    L = _lib.lib()
    wsn = torch.empty(api.workspace_size(64, "fp64"), dtype=torch.uint8, device="cuda")
    Cn, Sn = torch.empty_like(Ad), torch.empty_like(Ad)
    info = _lib.CsInfo()
    cargs = (ctypes.c_void_p(Ad.data_ptr()), 64, _lib.CS_FP64, ctypes.c_void_p(Cn.data_ptr()),
             ctypes.c_void_p(Sn.data_ptr()), ctypes.c_void_p(wsn.data_ptr()), wsn.numel(), -1, -1,
             ctypes.byref(info), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    ts = []
    for _ in range(200):
        t0 = time.perf_counter()
        _lib.check(L.cossin_ex(*cargs))
        ts.append(time.perf_counter() - t0)
    res["fp64_64x64_latency_us_c_abi"] = float(np.median(ts) * 1e6)
    res["fp64_64x64_m_s"] = [info.m, info.s]
    t0 = time.perf_counter()
    oracle.cossin(A)
    res["fp64_64x64_oracle_us"] = (time.perf_counter() - t0) * 1e6
    res["fp64_64x64_rel_err_vs_oracle"] = max(
        float(np.linalg.norm(C.cpu().numpy() - Co) / np.linalg.norm(Co)),
        float(np.linalg.norm(S.cpu().numpy() - So) / np.linalg.norm(So)))
    ref = {(f, r): (C, S) for (p, f, r), (C, S) in zip(work, outs) if p == "fp64"}
    for (p, f, r), (C, S) in zip(work, outs):
        if p != "fp64" and (f, r) in ref:
            C64, S64 = ref[(f, r)]
            res["%s_vs_fp64_path_%s_norm%g" % (p, f, r)] = max(
                float((C.double() - C64).norm() / C64.norm()), float((S.double() - S64).norm() / S64.norm()))
    for (p, f, r), Ad, (C, S) in zip(work, dev_in, outs):
        if f == "normal" and r == 64.0:
            Cd, Sd = C.double(), S.double()
            I = torch.eye(N, dtype=torch.float64, device=Cd.device)
            R = Cd @ Cd + Sd @ Sd - I
            res["%s_4096_norm64_pythagoras_residual" % p] = float(
                R.norm() / ((Cd @ Cd).norm() + (Sd @ Sd).norm()))
    return res


if __name__ == "__main__":
    sys.exit(main())
