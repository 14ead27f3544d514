"""Peak rates of the current GPU, measured with the library's probes
(include/bsm_probe.h), with the SM clock sampled during each measurement.

These rates are the roofline denominators of the library's kernels: the FP64
tensor pipe (mma.sync f64, the numeric FP64 kernel's instruction), DFMA, the
tcgen05 BF16 / E4M3 MMA issue rate at M = 128 and the N values the split
kernel uses, and the HBM read rate of 1-D bulk copies.  Each figure is one
launch of about `seconds` (its repetition count calibrated by a short launch
first), timed with CUDA events; `clocks` is the median SM clock nvidia-smi
reported while it ran.

    python -m paper_1501_07800_gb300.probe [--seconds S]

prints one JSON object.
"""
from __future__ import annotations

import argparse
import json
import statistics
import subprocess
import sys
import threading

import paper_1501_07800_gb300 as bsm

FP64_KINDS = {"dmma_m8n8k4": bsm.BSM_PROBE_DMMA_M8N8K4, "dmma_m16n8k4": bsm.BSM_PROBE_DMMA_M16N8K4,
              "dmma_m16n8k8": bsm.BSM_PROBE_DMMA_M16N8K8,
              "dmma_m16n8k16": bsm.BSM_PROBE_DMMA_M16N8K16, "dfma": bsm.BSM_PROBE_DFMA,
              "dmma_and_dfma": bsm.BSM_PROBE_MIXED}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms between
    start() and stop() (read-only queries)."""

    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev: int):
        self.dev = dev
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (FileNotFoundError, OSError):
            self.proc = None
        return self

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def wait_first(self, timeout: float = 2.0):
        """Returns once the sampler has reported (or after `timeout` s), so that
        starting nvidia-smi does not overlap what is sampled next."""
        import time
        t0 = time.perf_counter()
        while self.proc is not None and not self.lines and time.perf_counter() - t0 < timeout:
            time.sleep(0.01)
        return self

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                smax.append(float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _device() -> int:
    import torch
    return torch.cuda.current_device()


def _calibrated(run, seconds: float, iters0: int):
    """run(iters) -> (work, ms); a short launch sizes one of about `seconds`."""
    work, ms = run(iters0)
    iters = max(1, int(iters0 * seconds * 1e3 / max(ms, 1e-3)))
    clk = ClockSampler(_device()).start()
    work, ms = run(iters)
    return work, ms, iters, clk.stop()


def fp64(kind: str = "dmma_m8n8k4", seconds: float = 1.0) -> dict:
    """FP64 rate of one probe kind (TFLOP/s)."""
    work, ms, iters, clk = _calibrated(lambda it: bsm.bsm_probe_fp64(FP64_KINDS[kind], it),
                                       seconds, 2000)
    return {"tflops": work / ms / 1e9, "ms": ms, "iters": iters, "clocks": clk}


def tcgen05(fmt: int, n: int, seconds: float = 0.5, tiles: int = 1, issuers: int = 1) -> dict:
    """tcgen05.mma rate at M = 128 and N = n (TFLOP/s); fmt 0 BF16, 1 E4M3;
    consecutive instructions on `tiles` distinct operand pairs, `issuers`
    issuing threads per SM.  cycles: SM cycles per instruction at the sampled
    clock."""
    work, ms, iters, clk = _calibrated(
        lambda it: bsm.bsm_probe_tcgen05(fmt, n, it, tiles, issuers), seconds, 20000)
    out = {"tflops": work / ms / 1e9, "ms": ms, "iters": iters, "clocks": clk}
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    if clk.get("sm_mhz"):
        per_inst = 2.0 * 128 * n * (16 if fmt == 0 else 32)
        out["cycles_per_instruction"] = per_inst / (work / ms * 1e3 / sms / (clk["sm_mhz"] * 1e6))
    return out


def bulk_copy(nbytes: int = 8 << 30, stage_bytes: int = 32768, stages: int = 4) -> dict:
    """HBM read rate of 1-D bulk copies into shared memory (GB/s)."""
    bsm.bsm_probe_bulk_copy(1 << 28, stage_bytes, stages)  # warm-up
    clk = ClockSampler(_device()).start()
    moved, ms = bsm.bsm_probe_bulk_copy(nbytes, stage_bytes, stages)
    return {"gbs": moved / ms / 1e6, "ms": ms, "bytes": moved, "stage_bytes": stage_bytes,
            "stages": stages, "clocks": clk.stop()}


def fp64_peak(seconds: float = 1.0, repeats: int = 2) -> dict:
    """The chip's FP64 peak: the best of `repeats` launches each of scalar
    DFMA and of the FP64 tensor path (mma.sync m8n8k4), which share one FP64
    pipe; on GB300 DFMA is the faster.  `kind` names the winner, `dmma` gives
    the tensor path's own best."""
    runs = {k: [fp64(k, seconds) for _ in range(repeats)] for k in ("dfma", "dmma_m8n8k4")}
    best = {k: max(v, key=lambda r: r["tflops"]) for k, v in runs.items()}
    kind = max(best, key=lambda k: best[k]["tflops"])
    return dict(best[kind], kind=kind, runs=[r["tflops"] for r in runs[kind]],
                dmma=best["dmma_m8n8k4"]["tflops"], dfma=best["dfma"]["tflops"])


def measure_all(seconds: float = 0.5) -> dict:
    out = {"fp64": {k: fp64(k, seconds) for k in FP64_KINDS}}
    out["tcgen05_bf16"] = {str(n): tcgen05(0, n, seconds) for n in (32, 64, 96, 128, 256)}
    out["tcgen05_e4m3"] = {str(n): tcgen05(1, n, seconds) for n in (32, 64, 96, 128, 256)}
    # distinct operands per instruction, as in the split kernel
    out["tcgen05_bf16_distinct_tiles"] = {str(n): tcgen05(0, n, seconds, tiles=8)
                                          for n in (32, 64, 128)}
    out["tcgen05_e4m3_distinct_tiles"] = {str(n): tcgen05(1, n, seconds, tiles=8)
                                          for n in (32, 64, 128)}
    # issue rate: several threads issuing to their own accumulators
    out["tcgen05_bf16_issuers"] = {f"n{n}_x{k}": tcgen05(0, n, seconds, tiles=8, issuers=k)
                                   for n in (32, 64) for k in (1, 2, 4)}
    out["tcgen05_e4m3_issuers"] = {f"n{n}_x{k}": tcgen05(1, n, seconds, tiles=8, issuers=k)
                                   for n in (32, 64) for k in (1, 2)}
    out["bulk_copy"] = [bulk_copy(stage_bytes=sb, stages=st)
                        for sb, st in ((16384, 4), (32768, 4), (36864, 4), (65536, 3))]
    return out


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--seconds", type=float, default=0.5)
    a = ap.parse_args(argv)
    import torch
    torch.cuda.set_device(0)
    bsm.load()
    out = {"device": torch.cuda.get_device_name(0), "sms":
           torch.cuda.get_device_properties(0).multi_processor_count}
    out.update(measure_all(a.seconds))
    print(json.dumps(out), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
