#!/usr/bin/env python
"""Throughput of block-sparse C = A*B on GB300: time per product and useful GFLOP/s.

Workload (one "step" = one full bsm_multiply: symbolic phase, numeric phase,
exact-zero removal and C's level build, inputs resident in HBM):
  random block-sparse N = 65536, 32 x 32 leaf blocks, every block position
  nonzero with probability 0.02 (uniform placement), entries N(0,1), C = A*B.
Useful flops = 2 * bs^3 per nonzero (A_IK, B_KJ) block pair.

The default run also times, on the same GPU: the split-precision product of
the same operands, the product end to end with host buffers, 64 batched
products, the 20,000-point decay-type product (split BF16x7 and FP8x12 whole,
FP64 on one diagonal quadtree node of C, errors against the oracle on
sampled blocks), and the CPU oracle on bounded samples (one core and every
available core).  The FP64 roofline denominator is measured in the same run
by the library's probe (bsm_probe_fp64).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun every rank runs an independent product of the same size
(weak scaling, no data-path collective); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402
from synth import metrics  # noqa: E402

METRIC = "useful GFLOP/s of C=A*B (2*bs^3 per nonzero block pair), FP64"
WORKLOAD = {"workload": "random block-sparse N=65536, bs=32, block density 0.02, N(0,1)",
            "n": 65536, "bs": 32, "p": 0.02, "global_batch": 1,
            "l2": "inputs larger than L2 (A+B 1.4 GB, C 19 GB)"}


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "of measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "of fallback"


def workload_seeds(rank: int):
    sa = synth.BASE_SEED + 1 + 1000 * rank
    return sa, sa + 7919


WORKLOAD_SEEDS = workload_seeds(0)


def workload(rank: int, n: int, bs: int, p: float):
    sa, sb = workload_seeds(rank)
    A = synth.random_blocks(n, bs, p, sa)
    B = synth.random_blocks(n, bs, p, sb)
    return A, B


# ------------------------------------------------------------- peaks, clocks
def ClockSampler(dev: int):
    from paper_1501_07800_gb300.probe import ClockSampler as CS
    return CS(dev)


def fp64_peak_measured(bsm, seconds: float = 1.0) -> dict:
    """The chip's FP64 peak measured now by the library's probe
    (bsm_probe_fp64 on every SM, best of two launches of about a second each
    for scalar DFMA -- the FP64 kernel's arithmetic -- and for the FP64 tensor
    path, mma.sync m8n8k4), with its clock."""
    from paper_1501_07800_gb300 import probe
    p = probe.fp64_peak(seconds)
    clk = p["clocks"]
    return {"tflops": p["tflops"], "clocks": clk, "runs": p["runs"], "kind": p["kind"],
            "dmma_tflops": p["dmma"], "dfma_tflops": p["dfma"],
            "source": (f"measured in this run by bsm_probe_fp64 "
                       f"(paper_1501_07800_gb300/csrc/bsm_probe.cu, every SM): FP64 peak "
                       f"{p['tflops']:.4f} TFLOP/s ({p['kind']}; DFMA {p['dfma']:.4f}, DMMA "
                       f"m8n8k4 {p['dmma']:.4f}) at median SM clock {clk.get('sm_mhz')} MHz")}


# ------------------------------------------------------------ traffic table
def source_sha(srcs) -> str:
    h = hashlib.sha256()
    for src in srcs:
        h.update(open(os.path.join(ROOT, src), "rb").read())
    return h.hexdigest()[:16]


FP64_SOURCES = ("paper_1501_07800_gb300/csrc/bsm_numeric_fp64.cu",
                "paper_1501_07800_gb300/csrc/bsm_fp64_body.cuh")


def recorded_traffic(kernel: str, srcs):
    """Per-launch DRAM bytes from an ncu capture, valid only while the kernel's
    source files are unchanged since the capture (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p)).get(kernel)
    if not d:
        return None
    return d.get("bytes_per_launch") if d.get("src_sha") == source_sha(srcs) else None


# ------------------------------------------------------------ CPU baseline
def _oracle_rows_worker(n, bs, p, seed_a, seed_b, r0, r1, bar, q):
    """One process of the all-core oracle timing: regenerates the workload from
    its seeds, builds the oracle's trees for A's block rows [r0, r1) and all of
    B, waits for the other processes, and times the product (the unmodified
    oracle; CLOCK_MONOTONIC times, comparable across processes)."""
    import oracle
    A = synth.random_blocks(n, bs, p, seed_a)
    B = synth.random_blocks(n, bs, p, seed_b)
    keep = (A.brow >= r0) & (A.brow < r1)
    As = synth.BlockCOO(A.nrows, A.ncols, A.bs, A.brow[keep], A.bcol[keep], A.vals[keep])
    L = oracle.common_depth(A, B)
    ta, tb = oracle.tree(As, L), oracle.tree(B, L)
    del A
    bar.wait(timeout=900)
    t0 = time.perf_counter()
    P = oracle.multiply_trees(ta, tb)
    q.put((r0, t0, time.perf_counter(), P.triples))


def oracle_all_cores(n, bs, p, seed_a, seed_b, rows_per_proc: int, nproc: int) -> dict:
    """The oracle in `nproc` processes over disjoint ranges of A's block rows
    (the same arithmetic; spawned processes, no GPU): wall time from the first
    start to the last end."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    bar, q = ctx.Barrier(nproc), ctx.Queue()
    procs = [ctx.Process(target=_oracle_rows_worker,
                         args=(n, bs, p, seed_a, seed_b, k * rows_per_proc,
                               (k + 1) * rows_per_proc, bar, q)) for k in range(nproc)]
    for pr in procs:
        pr.start()
    import queue
    res, t_end = [], time.time() + 1800
    try:
        while len(res) < nproc:
            try:
                res.append(q.get(timeout=2))
            except queue.Empty:
                if any(pr.exitcode not in (None, 0) for pr in procs) or time.time() > t_end:
                    raise RuntimeError("an oracle process failed")
    finally:
        for pr in procs:
            pr.join(timeout=30 if len(res) == nproc else 0.1)
            if pr.is_alive():
                pr.terminate()
    t0 = min(x[1] for x in res)
    t1 = max(x[2] for x in res)
    triples = sum(x[3] for x in res)
    return {"seconds": t1 - t0, "triples": triples,
            "gflops": metrics.block_flops(bs, triples) / (t1 - t0) / 1e9}


def cpu_baseline(A, B, decay=None, target_s: float = 12.0):
    """The oracle, as it stands, on bounded samples of the same workload: the
    first R block rows of A times the whole of B on one core, then disjoint
    row ranges in one process per available host core.  With the decay
    product's sampled-block timing, its extrapolated full-product times."""
    import oracle

    L = oracle.common_depth(A, B)
    tb = oracle.tree(B, L)

    def sample(rows):
        keep = A.brow < rows
        As = synth.BlockCOO(A.nrows, A.ncols, A.bs, A.brow[keep], A.bcol[keep], A.vals[keep])
        ta = oracle.tree(As, L)
        t0 = time.perf_counter()
        P = oracle.multiply_trees(ta, tb)
        return P, time.perf_counter() - t0

    rows = 16
    P, dt = sample(rows)  # calibration, then a sample of about target_s
    rows = int(min(A.mb, max(rows, rows * target_s / max(dt, 1e-3))))
    P, dt = sample(rows)
    del tb
    single = metrics.block_flops(A.bs, P.triples) / dt / 1e9
    cores = len(os.sched_getaffinity(0))
    out = {"value": single, "unit": "GFLOP/s", "cores": 1, "cores_available": cores,
           "kind": "oracle",
           "sample": f"first {rows} of {A.mb} block rows of A times all of B "
                     f"({P.triples} block products, {dt:.2f} s single-threaded)",
           "single_thread": {"value": single, "rows": rows, "seconds": dt}}
    if cores > 1:
        # about target_s of wall time in all processes, disjoint row ranges
        per = int(max(1, min(A.mb // cores, rows * target_s / max(dt, 1e-3))))
        sa, sb = WORKLOAD_SEEDS
        allc = oracle_all_cores(A.nrows, A.bs, WORKLOAD["p"], sa, sb, per, cores)
        out.update({"value": allc["gflops"], "cores": cores,
                    "sample": f"{cores} processes, each {per} consecutive block rows of A "
                              f"(rows 0..{cores * per - 1} of {A.mb}) times all of B "
                              f"({allc['triples']} block products, {allc['seconds']:.2f} s wall)",
                    "all_cores": {"value": allc["gflops"], "processes": cores,
                                  "rows_per_process": per, "seconds": allc["seconds"],
                                  "speedup_vs_single": allc["gflops"] / single}})
    if decay is not None and "oracle" in decay:
        o = decay["oracle"]
        scale = out["value"] / single
        out["decay_c2_extrapolated"] = {
            "single_thread_s": o["full_product_s_extrapolated"],
            "all_cores_s": o["full_product_s_extrapolated"] / scale,
            "how": f"oracle time on {o['sampled_blocks']} sampled C blocks of the 20,000-point "
                   f"decay product ({o['gflops']:.2f} GFLOP/s, one thread), extrapolated to "
                   f"its {decay['block_products']} block products by the flop ratio; all cores: "
                   f"divided by the all-core speedup measured on the random product",
            "label": "extrapolated"}
    return out


def run_reference(args):
    """Reference arm: the CPU oracle timed on the host on bounded samples."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle

    n, bs, p = WORKLOAD["n"], WORKLOAD["bs"], WORKLOAD["p"]
    A, B = workload(0, n, bs, p)
    L = oracle.common_depth(A, B)
    tb = oracle.tree(B, L)
    rows = 16
    keep = A.brow < rows
    As = synth.BlockCOO(A.nrows, A.ncols, bs, A.brow[keep], A.bcol[keep], A.vals[keep])
    ta = oracle.tree(As, L)
    for _ in range(args.warmup):
        oracle.multiply_trees(ta, tb)
    times, trip = [], 0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        P = oracle.multiply_trees(ta, tb)
        times.append(time.perf_counter() - t0)
        trip = P.triples
    flops = metrics.block_flops(bs, trip)
    tot = sum(times)
    val = flops * len(times) / tot / 1e9
    sample = f"first {rows} of {A.mb} block rows of A times all of B ({trip} block products)"
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "GFLOP/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot / len(times), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": WORKLOAD,
            "cpu_baseline": {"kind": "oracle", "cores": 1, "sample": sample, "value": val,
                             "unit": "GFLOP/s"},
            "e2e": {"value": val, "unit": "GFLOP/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- GPU arm
def run_gpu(args):
    import torch

    import paper_1501_07800_gb300 as bsm

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    bsm.load()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def allmax(x: float) -> float:
        if dist is None:
            return x
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    def allsum(x: float) -> float:
        if dist is None:
            return x
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        return float(t.item())

    n, bs, p = WORKLOAD["n"], WORKLOAD["bs"], WORKLOAD["p"]
    t0 = time.time()
    # replicas: one product per rank (weak scaling); --shard: one product
    # split by Morton ranges of C over the ranks (strong scaling)
    A, B = workload(0 if args.shard else rank, n, bs, p)
    key_range = None
    if args.shard:
        from paper_1501_07800_gb300 import shard as sh
        L = sh.depth(-(-n // bs))
        key_range = sh.balanced_ranges(A.brow, A.bcol, B.brow, B.bcol, world, L)[rank]
        am, bm = sh.shard_operands(A.brow, A.bcol, B.brow, B.bcol, *key_range, L)
        A = synth.BlockCOO(n, n, bs, A.brow[am], A.bcol[am], A.vals[am])
        B = synth.BlockCOO(n, n, bs, B.brow[bm], B.bcol[bm], B.vals[bm])
        args.no_split = args.no_e2e = args.no_batched = True
    log(f"[rank {rank}] generated A {A.nblk} blocks, B {B.nblk} blocks in {time.time() - t0:.1f} s")
    ga = bsm.bsm_build(n, n, bs, torch.from_numpy(A.brow).to(dev), torch.from_numpy(A.bcol).to(dev),
                       torch.from_numpy(A.vals).to(dev))
    gb = bsm.bsm_build(n, n, bs, torch.from_numpy(B.brow).to(dev), torch.from_numpy(B.bcol).to(dev),
                       torch.from_numpy(B.vals).to(dev))
    torch.cuda.synchronize()

    prec = bsm.BSM_SPLIT_BF16 if args.mode == "split" else bsm.BSM_FP64

    def product():
        if key_range is None:
            return bsm.bsm_multiply(ga, gb, prec=prec)
        return bsm.bsm_multiply_range(ga, gb, key_range[0], key_range[1], prec=prec)

    # the FP64 roofline denominator, measured now on this GPU
    peak = fp64_peak_measured(bsm) if prec == bsm.BSM_FP64 else None
    for _ in range(args.warmup):
        C = product()
        del C
    torch.cuda.synchronize()
    _, triples, nc_sym = bsm.bsm_last_stats()
    flops = metrics.block_flops(bs, triples)

    def timed_steps(k: int, instrumented: bool):
        """k products between events on the stream.  instrumented: per-phase
        timing on -- CUDA events the product records and never waits for,
        read back after each step's end event (outside the step's interval)."""
        bsm.bsm_set_timing(instrumented)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(k)]
        num, nlaunch, nblk = [], 0, 0
        for i in range(k):
            ev[i][0].record(stream)
            C = product()
            ev[i][1].record(stream)
            ms, nl = bsm.bsm_last_phase_ms()
            num.append(ms[1])
            nlaunch += nl
            nblk = C.nblk
            del C
        torch.cuda.synchronize()
        return [x.elapsed_time(y) for x, y in ev], num, nlaunch, nblk

    clocks = ClockSampler(local)
    barrier()
    clocks.start().wait_first()   # nvidia-smi's start-up stays outside the timed steps
    step_ms, numeric_ms, launches, nblk_c = timed_steps(args.steps, True)
    barrier()
    clk = clocks.stop()
    phase_last = [float(x) for x in bsm.bsm_last_phase_ms()[0]]
    # the same steps without any instrumentation: the timing events cost nothing
    plain_ms, _, _, _ = timed_steps(min(args.steps, 3), False)
    bsm.bsm_set_timing(True)
    tot_s = allmax(sum(step_ms) / 1e3)
    total_flops = allsum(flops * args.steps)
    value = total_flops / tot_s / 1e9

    peaks, which = measured_peaks()
    t_num = statistics.mean(numeric_ms) / 1e3
    if prec == bsm.BSM_FP64:
        roofline = {"bound": "alu", "kernel": "k_numeric_fp64 (FP64 DFMA)",
                    "achieved": flops / t_num / 1e12, "peak": peak["tflops"],
                    "unit": "TFLOP/s", "frac": flops / t_num / 1e12 / peak["tflops"],
                    "peak_source": peak["source"], "peak_runs_tflops": peak["runs"],
                    "achieved_from": "useful flops / mean duration of the numeric phase "
                                     "(CUDA events on the product's stream) over the timed steps"}
    else:  # split mode: BF16 digit-pair flops against the bf16 peak
        roofline = {"bound": "tensor", "kernel": "k_numeric_split (tcgen05 kind::f16)",
                    "achieved": flops * 28 / t_num / 1e12, "peak": peaks["bf16_tflops_sustained"],
                    "unit": "TFLOP/s",
                    "frac": flops * 28 / t_num / 1e12 / peaks["bf16_tflops_sustained"],
                    "peak_source": f"{which} bf16 sustained"}
    roofline["traffic"] = recorded_traffic("k_numeric_fp64", FP64_SOURCES)

    # split-precision mode on the same inputs, same timing protocol
    split = split6 = None
    if not args.no_split and args.mode == "fp64":
        split = run_split(bsm, torch, ga, gb, args, stream, flops, triples, A, B, rank)
        # the fewest BF16 slices that keep the error below 1e-11 on this product
        split6 = run_split(bsm, torch, ga, gb, args, stream, flops, triples, A, B, rank,
                           slices=6)

    line = None
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": statistics.mean(step_ms), "higher_is_better": True,
                "scaling": "strong" if args.shard else "weak", "vs_baseline": None,
                "dtype": "f64" if prec == 0 else "bf16x-split", "data": "synthetic",
                "config": dict(WORKLOAD, parallelism=(f"C Morton-range shards x{world}"
                                                      if args.shard else f"replicas{world}")),
                "triples": triples, "c_blocks": nblk_c, "c_blocks_symbolic": nc_sym,
                "phase_ms_last": phase_last, "ms_per_step_uninstrumented":
                    statistics.mean(plain_ms),
                "roofline": roofline, "gpu_launches": launches, "clocks": clk}
        if split is not None:
            line["split_bf16"] = split
        if split6 is not None:
            line["split_bf16x6"] = split6

    # end to end through the public API with host buffers (pinned)
    if not args.no_e2e:
        e2e = run_e2e(bsm, torch, A, B, prec, max(2, min(args.steps, 5)))
        e2e_v = allsum(flops * e2e["steps"]) / allmax(e2e["seconds"]) / 1e9
        if line is not None:
            line["e2e"] = {"value": e2e_v, "unit": "GFLOP/s",
                           "h2d_bytes_per_step": e2e["h2d"], "d2h_bytes_per_step": e2e["d2h"],
                           "ms_per_step": 1e3 * e2e["seconds"] / e2e["steps"],
                           "steps": e2e["steps"], "overlap": e2e["overlap"]}
    if line is not None and not args.no_batched:
        line["batched"] = run_batched(bsm, torch, args, stream)
    if line is not None and world == 1 and not args.no_decay:
        # the decay-type product with 20,000 points (N = 100,000): full split
        # products, FP64 on one diagonal quadtree node of C
        del ga, gb
        bsm.bsm_release_memory()
        torch.cuda.empty_cache()
        line["decay_c2"] = decay_c2(bsm, torch, peak, args)
    if line is not None and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(A, B, line.get("decay_c2"))
    if line is not None:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def decay_c2(bsm, torch, peak, args) -> dict:
    """The electronic-structure-like product A*A with 20,000 points (N =
    100,000, bs 32): split BF16x7 and FP8x12 over the whole product (two timed
    products each after a warm-up), FP64 on the C blocks of the diagonal
    quadtree node [1024, 1536)^2 (its block products' flops against the FP64
    peak), errors against the oracle on 1000 C blocks sampled over all of C
    (plus 200 inside the node), with the clock record."""
    if peak is None:
        peak = fp64_peak_measured(bsm)
    legs = [dict(name="split_bf16x7", prec=bsm.BSM_SPLIT_BF16, slices=7, sym=False),
            dict(name="split_fp8x12", prec=bsm.BSM_SPLIT_FP8, slices=12, sym=False),
            dict(name="fp64_node", prec=bsm.BSM_FP64, slices=0, sym=False, range=(1024, 512),
                 steps=1)]
    clk = ClockSampler(torch.cuda.current_device()).start().wait_first()
    out = decay_product(bsm, torch, 20000, 32, legs, 2, peak=peak)
    out["clocks"] = clk.stop()
    f = out["fp64_node"]
    for k in ("split_bf16x7", "split_fp8x12"):
        # the FP64 time of the whole product at the node's measured rate
        fp64_full_ms = out["block_products"] / f["block_products"] * f["ms_per_product"]
        out[k]["speedup_vs_fp64_at_node_rate"] = fp64_full_ms / out[k]["ms_per_product"]
    return out


def run_split(bsm, torch, ga, gb, args, stream, flops, triples, A, B, rank, slices=7):
    """Split-precision products: time, roofline of the split kernel, and relative
    Frobenius error against the FP64 product (all C blocks) and against the
    oracle's definition on sampled C blocks."""
    prec = bsm.BSM_SPLIT_BF16
    for _ in range(args.warmup):
        C = bsm.bsm_multiply(ga, gb, prec=prec, slices=slices)
        del C
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    num_ms = []
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start().wait_first()
    for i in range(args.steps):
        ev[i][0].record(stream)
        C = bsm.bsm_multiply(ga, gb, prec=prec, slices=slices)
        ev[i][1].record(stream)
        num_ms.append(bsm.bsm_last_phase_ms()[0][1])
        if i < args.steps - 1:
            del C
    torch.cuda.synchronize()
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    # errors
    r1, c1, v1 = bsm.bsm_to_blocks(C, device=True)
    Cd = bsm.bsm_multiply(ga, gb)
    r2, c2, v2 = bsm.bsm_to_blocks(Cd, device=True)
    same = bool(torch.equal(r1, r2) and torch.equal(c1, c2))
    err_fp64 = float(torch.linalg.vector_norm(v1 - v2) / torch.linalg.vector_norm(v2)) if same else None
    err_oracle = None
    if rank == 0:
        import oracle
        L = oracle.common_depth(A, B)
        ta, tb = oracle.tree(A, L), oracle.tree(B, L)
        rng = np.random.default_rng(synth.BASE_SEED)
        pick = rng.choice(int(r1.shape[0]), size=min(200, int(r1.shape[0])), replace=False)
        rr, cc = r1[pick].cpu().numpy(), c1[pick].cpu().numpy()
        got = v1[torch.from_numpy(pick).to(v1.device)].cpu().numpy()
        ref = np.stack([oracle.block_product(ta, tb, i, j)[1] for i, j in zip(rr, cc)])
        err_oracle = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    del C, Cd
    t_num = statistics.mean(num_ms) / 1e3
    peaks, which = measured_peaks()
    pair_flops = flops * slices * (slices + 1) / 2  # BF16 digit-pair products needed
    achieved = pair_flops / t_num / 1e12
    return {"value": flops / (sum(step_ms) / len(step_ms) / 1e3) / 1e9, "unit": "GFLOP/s",
            "ms_per_step": statistics.mean(step_ms), "slices": slices,
            "rel_err_vs_fp64": err_fp64, "rel_err_vs_oracle_200_blocks": err_oracle,
            "numeric_ms": 1e3 * t_num,
            "roofline": {"bound": "tensor", "kernel": "k_numeric_split (tcgen05 kind::f16)",
                         "achieved": achieved, "peak": peaks["bf16_tflops_sustained"],
                         "unit": "TFLOP/s", "frac": achieved / peaks["bf16_tflops_sustained"],
                         "work": "BF16 digit-pair flops: s(s+1)/2 x 2 bs^3 per block product",
                         "peak_source": f"{which} bf16 sustained"},
            "clocks": clk}


def run_batched(bsm, torch, args, stream, nprod=64):
    """64 independent products, N log-uniform in [2048, 32768], block density
    U[0.5%, 10%], bs 32, uniform[-1,1) entries (generated on the device).
    Times the full batched call (symbolic + one persistent numeric launch +
    C assembly) and the autotuned plan replay (numeric phase from a CUDA graph;
    leaf size and launch schedule chosen by measurement), FP64 and split
    BF16x7, and the split result's error against FP64."""
    from synth import device as sd

    dev = torch.device("cuda", torch.cuda.current_device())
    t0 = time.time()
    gen = sd.batched(nprod, synth.BASE_SEED + 3, dev)
    As = [bsm.bsm_build(n, n, 32, r, c, v) for (n, r, c, v), _ in gen]
    Bs = [bsm.bsm_build(n, n, 32, r, c, v) for _, (n, r, c, v) in gen]
    del gen
    torch.cuda.synchronize()
    log(f"batched workload built in {time.time() - t0:.1f} s")
    out = {"workload": f"{nprod} products, N log-uniform [2048, 32768], bs 32, block density "
                       f"U[0.5%, 10%], uniform[-1,1) entries", "products": nprod}

    def timed(fn, steps):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        for i in range(steps):
            ev[i][0].record(stream)
            fn()
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in ev]

    for name, prec in (("fp64", bsm.BSM_FP64), ("split_bf16x7", bsm.BSM_SPLIT_BF16)):
        C = bsm.bsm_multiply_batched(As, Bs, prec=prec)  # warm-up
        del C
        _, triples, ncs = bsm.bsm_last_stats()
        flops = metrics.block_flops(32, triples)
        steps = 2 if prec == bsm.BSM_FP64 else 3

        def full():
            c = bsm.bsm_multiply_batched(As, Bs, prec=prec)
            del c
        full_ms = timed(full, steps)
        full()  # one more call for the phase split (symbolic + work list, numeric, C assembly)
        phases = [float(x) for x in bsm.bsm_last_phase_ms()[0]]
        t1 = time.time()
        # the autotuner picks the leaf size (re-blocked copies of the
        # operands, refreshed at every replay) and the launch schedule
        plan = bsm.bsm_plan_create(As, Bs, prec=prec, autotune=True, autotune_bs=True)
        create_s = time.time() - t1
        order, chunk, ctas, nitems = bsm.bsm_plan_info(plan)
        leaf = bsm.bsm_plan_block_size(plan)
        bsm.bsm_plan_execute(plan)
        replay_ms = timed(lambda: bsm.bsm_plan_execute(plan), steps)
        del plan  # one plan's buffers (all C blocks) at a time
        out[name] = {"full_call_ms": statistics.mean(full_ms), "full_call_phase_ms": phases,
                     "full_call_gflops": flops / (statistics.mean(full_ms) / 1e3) / 1e9,
                     "graph_replay_ms": statistics.mean(replay_ms),
                     "graph_replay_gflops": flops / (statistics.mean(replay_ms) / 1e3) / 1e9,
                     "plan_create_s": create_s, "triples": triples, "work_items": nitems,
                     "autotuned": {"leaf_size": leaf,
                                   "order": "longest-first" if order == 0 else
                                   "product-major Morton", "chunk": chunk, "ctas_per_sm": ctas}}
    # split vs FP64, product by product on every 8th product (bounded memory)
    num = den = 0.0
    for i in range(0, nprod, 8):
        cf = bsm.bsm_multiply(As[i], Bs[i])
        cs = bsm.bsm_multiply(As[i], Bs[i], prec=bsm.BSM_SPLIT_BF16)
        rf, _, vf = bsm.bsm_to_blocks(cf, device=True)
        rs, _, vs = bsm.bsm_to_blocks(cs, device=True)
        del cf, cs
        if rf.shape != rs.shape:
            num = float("nan")
            break
        num += float(torch.sum((vf - vs) ** 2))
        den += float(torch.sum(vf ** 2))
        del rf, rs, vf, vs
    out["split_rel_err_vs_fp64"] = (num / den) ** 0.5 if den > 0 else None
    out["split_err_sample"] = "every 8th product, all C blocks"
    return out


def _morton(i: int, j: int) -> int:
    from paper_1501_07800_gb300 import shard as sh
    return int(sh.morton(i, j))


def decay_product(bsm, torch, npts: int, bs: int, legs, steps: int, node=None,
                  nsample: int = 1000, range_sample: int = 200, peak=None) -> dict:
    """Decay-type product A*A: points uniform in a cube at 0.1 per cubic
    Angstrom, recursive-bisection order, 5 functions per point, A_ij = s_ij
    exp(-0.5 r_ij) dropped below 1e-6 (20,000 points: N = 100,000), generated
    on the device.

    legs: dicts {name, prec, slices, sym, range}; range = (first block, side)
    of a diagonal quadtree node of C (a Morton range, bsm_multiply_range) or
    None for the whole product; sym: the symmetric square (upper triangle of
    A*A from the upper triangle of A).  Each leg is timed over `steps`
    products (split legs after one warm-up product).  C's symbolic structure
    is compared with the block-pattern product (the definition of S_C);
    blocks whose entries all vanish are removed by the product, and on
    `nsample` C blocks sampled uniformly over C (plus `range_sample` inside
    every node range) the values and the presence of each block are compared
    with the oracle's definition, computed from the operand blocks in the
    sampled rows and columns.  The oracle's time on the sampled blocks
    (single-threaded) gives its extrapolated time for the whole product.
    node = (lo, hi): only the operand blocks with a row or a column in
    [lo, hi) are generated (products whose full C would not fit on one GPU);
    every leg then covers the node and the sample is a 32 x 32 grid of it."""
    import ctypes

    import oracle
    from synth import device as sd

    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    t0 = time.time()
    n, r, c, v = sd.decay(npts, bs, synth.BASE_SEED + 2, dev, cross=node)
    nbk = -(-n // bs)
    A = bsm.bsm_build(n, n, bs, r, c, v)
    U = None
    if any(g["sym"] for g in legs):
        up = r <= c
        U = bsm.bsm_build(n, n, bs, r[up].contiguous(), c[up].contiguous(), v[up].contiguous())
        del up
    torch.cuda.synchronize()
    gen_s = time.time() - t0
    nblk = A.nblk
    # C's structure by definition: the block-pattern product of A's stored
    # blocks (the generator's all-zero blocks are not stored); K[i, j] is the
    # number of block products of C block (i, j)
    ar = torch.empty(max(nblk, 1), dtype=torch.int32, device=dev)
    ac = torch.empty(max(nblk, 1), dtype=torch.int32, device=dev)
    cnt = ctypes.c_int64(nblk)
    assert bsm.load().bsm_to_blocks(A.handle, ctypes.byref(cnt), ar.data_ptr(), ac.data_ptr(),
                                    None, 1, stream.cuda_stream) == 0
    Pm = torch.zeros((nbk, nbk), dtype=torch.float32, device=dev)
    Pm[ar[:nblk].long(), ac[:nblk].long()] = 1.0
    del ar, ac
    a0, a1 = node if node is not None else (0, nbk)
    K = Pm[a0:a1] @ Pm[:, a0:a1]   # exact: counts below 2^24
    del Pm
    ci, cj = torch.nonzero(K > 0.5, as_tuple=True)
    nc_def = int(ci.numel())
    g = torch.Generator(device="cpu").manual_seed(synth.BASE_SEED)
    cic, cjc = ci.cpu() + a0, cj.cpu() + a0
    if node is None:
        pick = torch.randperm(nc_def, generator=g)[:nsample]
    else:
        # a grid of 32 block rows x 32 block columns of the node (about 1000
        # blocks) keeps the oracle's restricted operands small
        side = node[1] - node[0]
        gr = node[0] + torch.randperm(side, generator=g)[:32]
        gcl = node[0] + torch.randperm(side, generator=g)[:32]
        pick = torch.nonzero(torch.isin(cic, gr) & torch.isin(cjc, gcl)).flatten()
    picks = [pick]
    for lg in legs:   # extra samples inside every node range of a leg
        if lg.get("range") and node is None:
            lo_b, side = lg["range"]
            inr = torch.nonzero((cic >= lo_b) & (cic < lo_b + side) & (cjc >= lo_b) &
                                (cjc < lo_b + side)).flatten()
            picks.append(inr[torch.randperm(int(inr.numel()), generator=g)[:range_sample]])
    pick = torch.unique(torch.cat(picks))
    si, sj = cic[pick].numpy(), cjc[pick].numpy()
    nprod_s = K[torch.from_numpy(si - a0).to(dev), torch.from_numpy(sj - a0).to(dev)]
    sampled_flops = metrics.block_flops(bs, int(nprod_s.sum().item()))

    def useful(rng, sym):
        """Block products of the leg's C blocks, from the pattern counts."""
        Kr = K
        off = a0
        if rng is not None:
            lo_b, side = rng
            Kr = K[lo_b - a0:lo_b - a0 + side, lo_b - a0:lo_b - a0 + side]
            off = lo_b
        if sym:
            ii = torch.arange(Kr.shape[0], device=dev)[:, None] + off
            jj = torch.arange(Kr.shape[1], device=dev)[None, :] + off
            Kr = torch.where(ii <= jj, Kr, torch.zeros_like(Kr))
        return int(Kr.sum(dtype=torch.float64).item()), int((Kr > 0.5).sum().item())

    total_triples, _ = useful(None, False)
    # oracle operands restricted to the sampled rows (left) and columns (right)
    rows_keep = torch.isin(r, torch.from_numpy(si).to(dev).to(torch.int32))
    cols_keep = torch.isin(c, torch.from_numpy(sj).to(dev).to(torch.int32))
    left = synth.BlockCOO(n, n, bs, r[rows_keep].cpu().numpy(), c[rows_keep].cpu().numpy(),
                          v[rows_keep].cpu().numpy())
    right = synth.BlockCOO(n, n, bs, r[cols_keep].cpu().numpy(), c[cols_keep].cpu().numpy(),
                           v[cols_keep].cpu().numpy())
    del r, c, v, rows_keep, cols_keep
    torch.cuda.empty_cache()
    L = oracle.common_depth(left, right)
    tl, tr = oracle.tree(left, L), oracle.tree(right, L)
    t1 = time.perf_counter()
    refs = [oracle.block_product(tl, tr, i, j) for i, j in zip(si, sj)]
    oracle_s = time.perf_counter() - t1
    ref = np.stack([x[1] for x in refs])
    ref_nonzero = np.array([bool(np.any(x[1] != 0.0)) for x in refs])
    del tl, tr, left, right, refs
    oracle_rate = sampled_flops / oracle_s
    log(f"decay: n={n} blocks={nblk} C(def)={nc_def}; generation {gen_s:.1f} s, "
        f"oracle on {len(si)} blocks {oracle_s:.1f} s")
    out = {"workload": f"decay A*A, {npts} points (N={n}), bs {bs}", "a_blocks": nblk,
           "c_blocks_definition": nc_def, "block_products": total_triples,
           "useful_gflop": metrics.block_flops(bs, total_triples) / 1e9,
           "sampled_blocks": int(len(si)),
           "sampled_blocks_exactly_zero": int((~ref_nonzero).sum()),
           "oracle": {"kind": "oracle", "cores": 1, "sampled_blocks": int(len(si)),
                      "seconds": oracle_s, "gflops": oracle_rate / 1e9,
                      "full_product_s_extrapolated": metrics.block_flops(bs, total_triples)
                      / oracle_rate,
                      "how": "the oracle's single-threaded time on the sampled C blocks, "
                             "extrapolated to the whole product by the flop ratio"}}
    if node is not None:
        out["workload"] += (f": the C blocks of the diagonal quadtree node [{node[0]}, "
                            f"{node[1]})^2 of {nbk}^2 block positions, operands restricted to "
                            f"its rows and columns (bsm_multiply_range)")
    for lg in legs:
        name, prec, nsl, sym = lg["name"], lg["prec"], lg["slices"], lg["sym"]
        rng = lg.get("range")
        if node is not None:
            rng = (node[0], node[1] - node[0])
        key_range = None
        if rng is not None:
            klo = _morton(rng[0], rng[0])
            key_range = (klo, klo + rng[1] * rng[1])
        times = []
        C = None
        warm = 0 if prec == bsm.BSM_FP64 else 1
        for k in range(lg.get("steps", steps) + warm):
            C = None
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            C = (bsm.bsm_sym_square(U, prec=prec, slices=nsl) if sym
                 else bsm.bsm_multiply_range(A, A, *key_range, prec=prec, slices=nsl)
                 if key_range else bsm.bsm_multiply(A, A, prec=prec, slices=nsl))
            e1.record(stream)
            torch.cuda.synchronize()
            if k >= warm:
                times.append(e0.elapsed_time(e1))
        ms, _ = bsm.bsm_last_phase_ms()
        _, triples_run, ncs = bsm.bsm_last_stats()
        triples, nc_leg = useful(rng if node is None else None, sym)
        flops = metrics.block_flops(bs, triples)
        nr, ncol, _, ncb = bsm.bsm_info(C)
        cr = torch.empty(max(ncb, 1), dtype=torch.int32, device=dev)
        cc = torch.empty(max(ncb, 1), dtype=torch.int32, device=dev)
        cnt = ctypes.c_int64(ncb)
        assert bsm.load().bsm_to_blocks(C.handle, ctypes.byref(cnt), cr.data_ptr(),
                                        cc.data_ptr(), None, 1, stream.cuda_stream) == 0
        key_gpu = cr[:ncb].long() * nbk + cc[:ncb].long()   # row-major: ascending
        # the sampled blocks this leg computes; a symmetric result holds
        # (min, max), and C_ji = C_ij^T
        mine = np.ones(len(si), bool)
        if rng is not None and node is None:
            mine = (si >= rng[0]) & (si < rng[0] + rng[1]) & (sj >= rng[0]) & (sj < rng[0] + rng[1])
        lo, hi = (np.minimum(si, sj), np.maximum(si, sj)) if sym else (si, sj)
        want = torch.from_numpy(lo[mine].astype(np.int64) * nbk + hi[mine]).to(dev)
        pos = torch.searchsorted(key_gpu, want).clamp(max=max(ncb - 1, 0))
        present = ((key_gpu[pos] == want).cpu().numpy() if ncb else
                   np.zeros(int(mine.sum()), bool))
        bsm.bsm_release_memory()  # cached pool memory is not PyTorch's to use
        _, _, cv = bsm.bsm_to_blocks(C, device=True)
        got = cv[pos].cpu().numpy() if ncb else np.zeros_like(ref[mine])
        got[~present] = 0.0
        if sym:
            flip = si[mine] > sj[mine]
            got[flip] = got[flip].transpose(0, 2, 1)
        del cv, cr, cc, key_gpu
        err = float(np.linalg.norm(got - ref[mine]) / np.linalg.norm(ref[mine]))
        recut = prec != bsm.BSM_FP64 and bs != 32
        res = {"ms_per_product": statistics.mean(times), "steps": len(times),
               "gflops": flops / (statistics.mean(times) / 1e3) / 1e9,
               "block_products": triples, "phase_ms": [float(x) for x in ms],
               "chunks": bsm.bsm_last_chunks(), "computed_at_bs": 32 if recut else bs,
               "c_blocks_symbolic": ncs, "c_blocks": ncb,
               "symbolic_structure_matches_definition": None if recut else ncs == nc_leg,
               "sampled_presence_matches_oracle": bool(np.array_equal(present,
                                                                      ref_nonzero[mine])),
               "rel_err_vs_oracle_sampled_blocks": err, "sampled_blocks": int(mine.sum())}
        if rng is not None and node is None:
            res["c_range"] = (f"diagonal quadtree node [{rng[0]}, {rng[0] + rng[1]})^2, "
                              f"Morton keys [{key_range[0]}, {key_range[1]})")
        if prec == bsm.BSM_FP64 and peak is not None and ms[1] > 0:
            t_num = ms[1] / 1e3   # the numeric phase of the last timed product
            res["numeric_tflops"] = flops / t_num / 1e12
            res["frac_of_fp64_peak"] = flops / t_num / 1e12 / peak["tflops"]
            res["peak"] = peak["source"]
        out[name] = res
        del C
        bsm.bsm_release_memory()
        torch.cuda.empty_cache()
        log(f"{name}: {res}")
    del A, U, K
    bsm.bsm_release_memory()
    torch.cuda.empty_cache()
    return out


def run_decay(args):
    """--workload decay: the decay-type product A*A with the requested legs
    (one JSON line)."""
    import torch

    import paper_1501_07800_gb300 as bsm

    torch.cuda.set_device(0)
    bsm.load()
    bsm.bsm_set_timing(True)
    npts, bs = args.points, args.bs
    node = None
    if args.node_side:
        S = args.node_side
        nbk_full = -(-(npts * 5) // bs)
        lo_b = args.node_at if args.node_at is not None else (nbk_full // 2) // S * S
        if S & (S - 1) or lo_b % S or lo_b >= nbk_full:
            raise SystemExit("--node-side must be a power of two and --node-at a multiple of it")
        node = (lo_b, min(lo_b + S, nbk_full))
        args.sym = False
    slices = [int(x) for x in args.slices.split(",") if x]
    legs = [dict(name=f"split_bf16x{k}", prec=bsm.BSM_SPLIT_BF16, slices=k, sym=False)
            for k in slices]
    legs += [dict(name=f"split_fp8x{k}", prec=bsm.BSM_SPLIT_FP8, slices=int(k), sym=False)
             for k in args.fp8_slices.split(",") if k]
    if not args.no_fp64:
        fr = None
        if args.fp64_node_side:
            fr = (args.fp64_node_at, args.fp64_node_side)
        legs.append(dict(name="fp64", prec=bsm.BSM_FP64, slices=0, sym=False, range=fr,
                         steps=1))
    if args.sym:
        legs.append(dict(name=f"sym_square_split_bf16x{slices[-1]}", prec=bsm.BSM_SPLIT_BF16,
                         slices=slices[-1], sym=True))
        if not args.no_fp64:
            legs.append(dict(name="sym_square_fp64", prec=bsm.BSM_FP64, slices=0, sym=True,
                             steps=1))
    peak = fp64_peak_measured(bsm) if not args.no_fp64 else None
    out = decay_product(bsm, torch, npts, bs, legs, args.steps, node=node, peak=peak)
    best = f"split_bf16x{max(slices)}" if slices else None
    if best and "fp64" in out and out["fp64"].get("c_range") is None:
        out["split_speedup_vs_fp64"] = out["fp64"]["ms_per_product"] / out[best]["ms_per_product"]
    if args.sym and "sym_square_fp64" in out and "fp64" in out:
        out["sym_square_speedup_vs_full_fp64"] = (out["fp64"]["ms_per_product"] /
                                                  out["sym_square_fp64"]["ms_per_product"])
    print(json.dumps(out), flush=True)
    return 0


def run_decay_nodes(args):
    """--workload decay --all-nodes: the decay-type product A*A over the whole
    of C, one quadtree node of C (side --node-side blocks, row by row) at a
    time, for products whose operands and C do not fit on one GPU together
    (80,000 points, bs 64: A 171 GB, C about 927 GB).  Per node, only the
    operand blocks with a row or a column in the node's rows and columns are
    generated on the device; each split mode computes the node's C blocks
    (bsm_multiply_range, one product per node and mode, timed with CUDA
    events, the first node after a warm-up), and FP64 runs on --fp64-nodes
    nodes (evenly spaced along the diagonal), its time for the whole product
    extrapolated by the block-product ratio.  Errors: against the oracle on a
    grid of 38 block rows x 38 block columns drawn uniformly (every grid
    position in C's structure), from the operand blocks of those rows and
    columns."""
    import ctypes

    import torch

    import oracle
    import paper_1501_07800_gb300 as bsm
    from paper_1501_07800_gb300 import shard as sh
    from synth import device as sd

    torch.cuda.set_device(0)
    bsm.load()
    bsm.bsm_set_timing(True)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    npts, bs, S = args.points, args.bs, args.node_side or 512
    seed = synth.BASE_SEED + 2
    n = npts * 5
    nbk = -(-n // bs)
    pts = synth.decay_points(npts, seed)
    modes = [(f"split_bf16x{k}", bsm.BSM_SPLIT_BF16, int(k)) for k in args.slices.split(",") if k]
    modes += [(f"split_fp8x{k}", bsm.BSM_SPLIT_FP8, int(k)) for k in args.fp8_slices.split(",") if k]
    side_nodes = -(-nbk // S)
    nodes = [(i * S, j * S) for i in range(side_nodes) for j in range(side_nodes)]
    if args.max_nodes:
        nodes = nodes[:args.max_nodes]
    diag = [(i * S, i * S) for i in range(side_nodes)]
    nf = max(0, args.fp64_nodes)
    fp64_nodes = set(diag[(k * len(diag)) // (nf + 1) + len(diag) // (2 * (nf + 1))]
                     for k in range(nf)) if nf else set()
    peak = fp64_peak_measured(bsm) if nf else None

    # the oracle on a grid of block rows x block columns drawn uniformly
    g = torch.Generator(device="cpu").manual_seed(synth.BASE_SEED)
    grows = torch.sort(torch.randperm(nbk, generator=g)[:38]).values
    gcols = torch.sort(torch.randperm(nbk, generator=g)[:38]).values
    rmask = torch.zeros(nbk, dtype=torch.bool, device=dev)
    cmask = torch.zeros(nbk, dtype=torch.bool, device=dev)
    rmask[grows.to(dev)] = True
    cmask[gcols.to(dev)] = True
    t0 = time.time()
    # the candidate blocks of the whole matrix (structure only), once
    cand = sd.decay_blocks(npts, bs, seed, dev, points=pts)
    _, r, c, v = sd.decay(npts, bs, seed, dev, keep=(rmask, cmask), points=pts, blocks=cand)
    lk, rk = rmask[r.long()], cmask[c.long()]
    left = synth.BlockCOO(n, n, bs, r[lk].cpu().numpy(), c[lk].cpu().numpy(), v[lk].cpu().numpy())
    right = synth.BlockCOO(n, n, bs, r[rk].cpu().numpy(), c[rk].cpu().numpy(), v[rk].cpu().numpy())
    del r, c, v, lk, rk
    torch.cuda.empty_cache()
    L = oracle.common_depth(left, right)
    tl, tr = oracle.tree(left, L), oracle.tree(right, L)
    gi, gj = np.meshgrid(grows.numpy(), gcols.numpy(), indexing="ij")
    gi, gj = gi.ravel(), gj.ravel()
    # grid positions in C's structure: some K has A_iK and A_Kj stored
    pa = {}
    for i, k in zip(left.brow, left.bcol):
        pa.setdefault(int(i), set()).add(int(k))
    pb = {}
    for k, j in zip(right.brow, right.bcol):
        pb.setdefault(int(j), set()).add(int(k))
    inc = np.array([bool(pa.get(int(i), set()) & pb.get(int(j), set())) for i, j in zip(gi, gj)])
    gi, gj = gi[inc], gj[inc]
    nprod_grid = sum(len(pa[int(i)] & pb[int(j)]) for i, j in zip(gi, gj))
    t1 = time.perf_counter()
    refs = [oracle.block_product(tl, tr, int(i), int(j)) for i, j in zip(gi, gj)]
    oracle_s = time.perf_counter() - t1
    ref = np.stack([x[1] for x in refs])
    ref_nz = np.array([bool(np.any(x[1] != 0.0)) for x in refs])
    del tl, tr, left, right, refs
    gkey = gi.astype(np.int64) * nbk + gj
    log(f"decay nodes: n={n}, {len(nodes)} nodes of side {S}; oracle on {len(gi)} grid blocks "
        f"{oracle_s:.1f} s (setup {time.time() - t0:.1f} s)")

    acc = {name: {"ms": 0.0, "num": 0.0, "den": 0.0, "presence_ok": True, "blocks": 0,
                  "c_blocks": 0} for name, _, _ in modes}
    # output buffers for a node's C blocks (at most S^2), allocated once
    ob = (torch.empty(S * S, dtype=torch.int32, device=dev),
          torch.empty(S * S, dtype=torch.int32, device=dev),
          torch.empty((S * S, bs, bs), dtype=torch.float64, device=dev))
    fp64 = {"ms": 0.0, "products": 0, "nodes": [], "num": 0.0, "den": 0.0, "numeric_ms": 0.0}
    total_products, gen_s, t_all, prod_s = 0, 0.0, time.time(), 0.0
    for ni, (r0, c0) in enumerate(nodes):
        tg = time.time()
        rm = torch.zeros(nbk, dtype=torch.bool, device=dev)
        cm = torch.zeros(nbk, dtype=torch.bool, device=dev)
        rm[r0:r0 + S] = True
        cm[c0:c0 + S] = True
        _, r, c, v = sd.decay(npts, bs, seed, dev, keep=(rm, cm), points=pts, blocks=cand)
        Ar = bsm.bsm_build(n, n, bs, r, c, v)
        del r, c, v
        # the generator's memory back to the driver; the library keeps its own
        # pool (its peak is reached at the first node and then reused)
        torch.cuda.empty_cache()
        # block products of the node by definition, from the stored blocks
        nb_ = Ar.nblk
        sr = torch.empty(max(nb_, 1), dtype=torch.int32, device=dev)
        sc = torch.empty(max(nb_, 1), dtype=torch.int32, device=dev)
        cnt = ctypes.c_int64(nb_)
        assert bsm.load().bsm_to_blocks(Ar.handle, ctypes.byref(cnt), sr.data_ptr(),
                                        sc.data_ptr(), None, 1, stream.cuda_stream) == 0
        sr, sc = sr[:nb_].long(), sc[:nb_].long()
        lsel, rsel = (sr >= r0) & (sr < r0 + S), (sc >= c0) & (sc < c0 + S)
        Pl = torch.zeros((S, nbk), dtype=torch.float32, device=dev)
        Pr = torch.zeros((nbk, S), dtype=torch.float32, device=dev)
        Pl[sr[lsel] - r0, sc[lsel]] = 1.0
        Pr[sr[rsel], sc[rsel] - c0] = 1.0
        node_products = int((Pl @ Pr).sum(dtype=torch.float64).item())
        del Pl, Pr, sr, sc, lsel, rsel
        total_products += node_products
        torch.cuda.synchronize()
        gen_s += time.time() - tg
        klo = int(sh.morton(r0, c0))
        kr = (klo, klo + S * S)
        sel = (gi >= r0) & (gi < r0 + S) & (gj >= c0) & (gj < c0 + S)
        todo = [(name, prec, sl) for name, prec, sl in modes]
        if (r0, c0) in fp64_nodes:
            todo.append(("fp64", bsm.BSM_FP64, 0))
        for name, prec, sl in todo:
            reps = 2 if ni == 0 and prec != bsm.BSM_FP64 else 1   # first node: a warm-up run
            for k in range(reps):
                C = None
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                C = bsm.bsm_multiply_range(Ar, Ar, kr[0], kr[1], prec=prec, slices=sl)
                e1.record(stream)
                torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            prod_s += ms / 1e3
            ncb = bsm.bsm_info(C)[3]
            nerr = dden = 0.0
            pres_ok = True
            if sel.any() and ncb:
                bsm.bsm_to_blocks(C, device=True, out=ob)
                cr, cc, cv = ob[0][:ncb], ob[1][:ncb], ob[2]
                ck = cr.long() * nbk + cc.long()
                want = torch.from_numpy(gkey[sel]).to(dev)
                pos = torch.searchsorted(ck, want).clamp(max=ncb - 1)
                present = (ck[pos] == want).cpu().numpy()
                got = cv[pos].cpu().numpy()
                got[~present] = 0.0
                nerr = float(np.sum((got - ref[sel]) ** 2))
                dden = float(np.sum(ref[sel] ** 2))
                pres_ok = bool(np.array_equal(present, ref_nz[sel]))
                del cr, cc, cv, ck
            del C
            if name == "fp64":
                fp64["ms"] += ms
                fp64["products"] += node_products
                fp64["nodes"].append([r0, c0])
                fp64["numeric_ms"] += float(bsm.bsm_last_phase_ms()[0][1])
                fp64["num"] += nerr
                fp64["den"] += dden
            else:
                a = acc[name]
                a["ms"] += ms
                a["num"] += nerr
                a["den"] += dden
                a["presence_ok"] &= pres_ok
                a["blocks"] += int(sel.sum())
                a["c_blocks"] += ncb
        del Ar
        if ni % 10 == 0:
            log(f"node {ni + 1}/{len(nodes)} at ({r0}, {c0}): {node_products} block products; "
                f"{time.time() - t_all:.0f} s (operands {gen_s:.0f} s, products {prod_s:.0f} s)")
    flops_total = metrics.block_flops(bs, total_products)
    out = {"workload": f"decay A*A, {npts} points (N={n}), bs {bs}, whole product node by node "
                       f"({len(nodes)} quadtree nodes of C of side {S} blocks)",
           "nodes": len(nodes), "block_products": total_products,
           "useful_pflop": flops_total / 1e15, "operand_generation_s": gen_s,
           "grid": {"rows": 38, "cols": 38, "blocks_in_c": int(len(gi)),
                    "exactly_zero": int((~ref_nz).sum()), "oracle_s": oracle_s,
                    "oracle_block_products": nprod_grid}}
    for name, _, _ in modes:
        a = acc[name]
        out[name] = {"seconds": a["ms"] / 1e3,
                     "useful_tflops": flops_total / (a["ms"] / 1e3) / 1e12,
                     "rel_err_vs_oracle_grid": (a["num"] / a["den"]) ** 0.5 if a["den"] else None,
                     "grid_blocks_compared": a["blocks"],
                     "grid_presence_matches_oracle": a["presence_ok"], "c_blocks": a["c_blocks"]}
    if fp64["products"]:
        rate = metrics.block_flops(bs, fp64["products"]) / (fp64["ms"] / 1e3)
        out["fp64"] = {"nodes": fp64["nodes"], "seconds_measured": fp64["ms"] / 1e3,
                       "block_products_measured": fp64["products"],
                       "useful_tflops": rate / 1e12,
                       "numeric_frac_of_fp64_peak": metrics.block_flops(bs, fp64["products"]) /
                       (fp64["numeric_ms"] / 1e3) / 1e12 / peak["tflops"],
                       "peak": peak["source"],
                       "whole_product_s_extrapolated": flops_total / rate,
                       "label": "extrapolated by the block-product ratio",
                       "rel_err_vs_oracle_grid": (fp64["num"] / fp64["den"]) ** 0.5
                       if fp64["den"] else None}
        for name, _, _ in modes:
            out[name]["speedup_vs_fp64_extrapolated"] = (out["fp64"]["whole_product_s_extrapolated"]
                                                        / out[name]["seconds"])
    oracle_rate = metrics.block_flops(bs, nprod_grid) / oracle_s
    out["oracle_extrapolated"] = {"single_thread_s": flops_total / oracle_rate,
                                  "gflops": oracle_rate / 1e9, "label": "extrapolated",
                                  "how": "the oracle's time on the grid blocks, scaled by the "
                                         "flop ratio"}
    print(json.dumps(out), flush=True)
    return 0


def run_rmat(args):
    """Locality sweep on R-MAT graph matrices (N = 8192, 5 edge draws per row,
    b = c = d = (1 - a) / 3): per-level multiply-task counts of A*A (the
    quantity of Fig. 5, right) and the time of the product, bs 16."""
    import torch

    import paper_1501_07800_gb300 as bsm

    torch.cuda.set_device(0)
    bsm.load()
    stream = torch.cuda.current_stream()
    out = {"workload": "R-MAT A*A, N = 8192, 5 draws per row, bs 16", "sweep": []}
    for a in (0.25, 0.4, 0.55, 0.7, 0.85, 0.95):
        A = synth.rmat(13, a, 16, synth.BASE_SEED + 40)
        M = bsm.bsm_build(A.nrows, A.ncols, A.bs, A.brow, A.bcol, A.vals)
        times = []
        for k in range(args.warmup + args.steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            C = bsm.bsm_multiply(M, M)
            e1.record(stream)
            torch.cuda.synchronize()
            if k >= args.warmup:
                times.append(e0.elapsed_time(e1))
        tasks, triples, _ = bsm.bsm_last_stats()
        row = {"a": a, "a_blocks": A.nblk, "c_blocks": bsm.bsm_info(C)[3],
               "tasks_per_level_root_first": [int(x) for x in tasks], "triples": triples,
               "ms_per_product": statistics.median(times)}
        out["sweep"].append(row)
        log(f"rmat: {row}")
    print(json.dumps(out), flush=True)
    return 0


def run_e2e(bsm, torch, A, B, prec, steps):
    """Host COO in pinned memory -> bsm_build x2 -> bsm_multiply -> C's blocks
    into pinned host buffers, every step, through the public API.  Step i's
    product runs while step i-1's download crosses the host link: each step
    first builds its operands (from the pinned arrays, read in place while the
    link is otherwise idle -- an upload beside a 19 GB download crawls), then
    queues the previous product's download on a copy stream (bsm_to_blocks'
    asynchronous mode: chunked device gathers and copy-engine transfers on the
    library's highest-priority stream), then multiplies.  Two sets of result buffers alternate.  The timed region ends
    when the last download has landed."""
    def pinned(a: np.ndarray) -> np.ndarray:
        t = torch.empty(a.shape, dtype=getattr(torch, str(a.dtype)), pin_memory=True)
        t.numpy()[...] = a
        return t.numpy()

    pa = [pinned(x) for x in (A.brow, A.bcol, A.vals)]
    pb = [pinned(x) for x in (B.brow, B.bcol, B.vals)]
    h2d = sum(x.nbytes for x in pa + pb)
    compute, copy = torch.cuda.Stream(), torch.cuda.Stream()
    bufs = [None, None]       # the caller's result buffers (pinned), one set per parity
    inflight = [None, None]   # (C, event): C stays alive until its download has landed
    state = {"prev": None}    # the last product, not yet queued for download

    def download(C, k):
        if inflight[k] is not None:   # this buffer set's previous download
            inflight[k][1].synchronize()
            inflight[k] = None
        n = C.nblk
        if bufs[k] is None or bufs[k][0].shape[0] < n:
            # allocated in the untimed warm-up steps (one per buffer set)
            bufs[k] = (torch.empty(n, dtype=torch.int32, pin_memory=True).numpy(),
                       torch.empty(n, dtype=torch.int32, pin_memory=True).numpy(),
                       torch.empty((n, A.bs, A.bs), dtype=torch.float64,
                                   pin_memory=True).numpy())
        bsm.bsm_to_blocks(C, out=bufs[k], stream=copy, asynchronous=True)
        ev = torch.cuda.Event()
        ev.record(copy)
        inflight[k] = (C, ev)
        return n * (8 + 8 * A.bs * A.bs)

    def step(i):
        ga = bsm.bsm_build(A.nrows, A.ncols, A.bs, *pa, stream=compute)
        gb = bsm.bsm_build(B.nrows, B.ncols, B.bs, *pb, stream=compute)
        d2h = 0
        if state["prev"] is not None:
            d2h = download(*state["prev"])
        C = bsm.bsm_multiply(ga, gb, prec=prec, stream=compute)
        del ga, gb
        state["prev"] = (C, i % 2)
        return d2h

    def drain():
        d2h = download(*state["prev"])
        state["prev"] = None
        for f in inflight:
            if f is not None:
                f[1].synchronize()
        return d2h

    step(0)   # untimed: sizes and pins both buffer sets
    step(1)
    drain()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    d2h = 0
    for i in range(steps):
        d2h = max(d2h, step(i))
    d2h = max(d2h, drain())
    dt = time.perf_counter() - t0
    inflight[0] = inflight[1] = None
    return {"seconds": dt, "steps": steps, "h2d": h2d, "d2h": d2h,
            "overlap": "each step's product overlaps the previous step's download (chunked "
                       "gather + copy engine on a high-priority stream); uploads run while "
                       "the link is idle"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="bsm", choices=["bsm", "reference"])
    ap.add_argument("--mode", default="fp64", choices=["fp64", "split"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-split", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-decay", action="store_true",
                    help="skip the 20,000-point decay product of the default run")
    ap.add_argument("--workload", default="random", choices=["random", "decay", "rmat"],
                    help="decay: the decay-type A*A product (separate JSON line)")
    ap.add_argument("--points", type=int, default=20000, help="decay workload: number of points")
    ap.add_argument("--bs", type=int, default=32, choices=[16, 32, 64],
                    help="leaf block size (random and decay workloads)")
    ap.add_argument("--slices", default="7", help="decay workload: split slice counts, e.g. 3,5,7")
    ap.add_argument("--fp8-slices", default="", help="decay workload: FP8 split slice counts")
    ap.add_argument("--no-fp64", action="store_true", help="decay workload: skip the FP64 legs")
    ap.add_argument("--fp64-node-side", type=int, default=0,
                    help="decay workload: the FP64 leg on one diagonal quadtree node of C of this "
                         "side (blocks), the split legs on the whole product")
    ap.add_argument("--fp64-node-at", type=int, default=0,
                    help="decay workload: first block row/column of the FP64 leg's node")
    ap.add_argument("--node-side", type=int, default=0,
                    help="decay workload: compute only the C blocks of one diagonal quadtree "
                         "node of this side (blocks, a power of two)")
    ap.add_argument("--node-at", type=int, default=None,
                    help="decay workload: first block row/column of that node")
    ap.add_argument("--all-nodes", action="store_true",
                    help="decay workload: the whole product node by node (side --node-side, "
                         "default 512 blocks)")
    ap.add_argument("--fp64-nodes", type=int, default=1,
                    help="decay --all-nodes: FP64 on this many diagonal nodes")
    ap.add_argument("--max-nodes", type=int, default=0,
                    help="decay --all-nodes: stop after this many nodes (testing)")
    ap.add_argument("--sym", action="store_true",
                    help="decay workload: also the symmetric square from the upper triangle")
    ap.add_argument("--shard", action="store_true",
                    help="split one product over the ranks by Morton ranges of C")
    ap.add_argument("--n", type=int, default=None, help="matrix side (profiling runs only)")
    ap.add_argument("--p", type=float, default=None, help="block density (profiling runs only)")
    args = ap.parse_args()
    if args.n is not None or args.p is not None or args.bs != 32:
        # the random workload at another leaf size (each block position
        # nonzero with the same p at that size), or a reduced profiling case
        WORKLOAD["n"] = args.n or WORKLOAD["n"]
        WORKLOAD["p"] = args.p or WORKLOAD["p"]
        WORKLOAD["bs"] = args.bs
        reduced = args.n is not None or args.p is not None
        WORKLOAD["workload"] = (f"random block-sparse N={WORKLOAD['n']}, bs={args.bs}, block "
                                f"density {WORKLOAD['p']}, N(0,1)"
                                + (" (reduced profiling case)" if reduced else ""))
        if args.bs != 32:
            WORKLOAD["l2"] = "inputs larger than L2 (A+B about 1.4 GB, C over 10 GB)"
    if args.warmup < 3:
        log("warm-up raised to 3 steps")
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "decay" and args.all_nodes:
        return run_decay_nodes(args)
    if args.workload == "decay":
        return run_decay(args)
    if args.workload == "rmat":
        return run_rmat(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
