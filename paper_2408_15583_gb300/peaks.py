"""Measured unit rates of the device in use, through ``pe_probe_units``: FP32
FMA (scalar and the packed FP32x2 form), ``__sinf`` (the PO term's sine
path), FP64 FMA, L2-resident reads and
fire-and-forget 64-bit atomicMin (the splat's update).  They bound the
ALU- and atomic-bound kernels of the path; the FP32 figure is reported beside
the peak derived from the unit counts (SMs x 128 FP32 lanes x 2 flops x SM
clock) at the SM clock sampled during the probes.

``python -m paper_2408_15583_gb300.peaks`` prints one JSON line.
"""
from __future__ import annotations

import json
import shutil
import subprocess
import sys
from typing import Dict, Optional

import torch

from . import _lib

# name: (kind, iterations per thread, unit divisor, unit)
PROBES = {
    "fp32_fma": (0, 100_000, 1e12, "TFLOP/s"),
    "sin": (1, 20_000, 1e9, "G sines/s"),
    "fp64_fma": (2, 2_000, 1e12, "TFLOP/s"),
    "l2_read": (3, 4_000, 1e9, "GB/s"),
    "atomic_min_u64": (4, 1_000, 1e9, "G atomics/s"),
    "fp32x2_fma": (5, 50_000, 1e12, "TFLOP/s"),
}
SCRATCH_BYTES = 32 << 20   # well inside the 129 MB L2
BLOCKS_PER_SM = 8


def _clock_sampler():
    exe = shutil.which("nvidia-smi")
    if exe is None:
        return None
    return subprocess.Popen([exe, "--query-gpu=clocks.sm,clocks.max.sm",
                             "--format=csv,noheader,nounits", "-lms", "100"],
                            stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)


def _clock_stop(p) -> Optional[Dict[str, float]]:
    if p is None:
        return None
    p.terminate()
    try:
        out, _ = p.communicate(timeout=5)
    except subprocess.TimeoutExpired:
        p.kill()
        out, _ = p.communicate()
    sm, mx = [], []
    for line in out.splitlines():
        parts = [x.strip() for x in line.split(",")]
        if len(parts) >= 2:
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                pass
    if not sm:
        return None
    sm.sort()
    return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(mx), "samples": len(sm)}


def measure(device: str = "cuda:0", reps: int = 5, scale: float = 1.0, only=None) -> dict:
    """Best rate over `reps` timed launches of each probe (after one warm-up
    launch), in the units of PROBES.  `scale` shortens every probe; `only`
    names the probes to run (all by default)."""
    lib = _lib.load()
    dev = torch.device(device)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks = sms * BLOCKS_PER_SM
    scratch = torch.zeros(SCRATCH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    sampler = _clock_sampler()
    out = {"sms": sms, "blocks": blocks, "threads_per_block": 256}
    try:
        for name, (kind, n_iter, div, unit) in PROBES.items():
            if only is not None and name not in only:
                continue
            if kind == 3:
                scratch.zero_()
            elif kind == 4:
                scratch.fill_(255)          # keys start at all ones, as in the splat
            n = max(1, int(n_iter * scale))
            best = 0.0
            for r in range(reps + 1):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                ops = lib.pe_probe_units(kind, blocks, n, scratch.data_ptr(), SCRATCH_BYTES,
                                         stream.cuda_stream)
                e1.record(stream)
                if ops < 0:
                    raise RuntimeError(f"pe_probe_units: {lib.pe_last_error().decode()}")
                e1.synchronize()
                if r == 0:
                    continue                # warm-up (L2 fill, clocks)
                ms = e0.elapsed_time(e1)
                best = max(best, ops / (ms / 1e3))
            out[name] = {"value": best / div, "unit": unit, "ops_per_launch": int(ops)}
    finally:
        clocks = _clock_stop(sampler)
    out["clocks"] = clocks
    if clocks and "fp32_fma" in out:
        derived = sms * 128 * 2 * clocks["sm_mhz"] * 1e6 / 1e12
        out["fp32_fma"]["derived_peak_tflops"] = derived
        out["fp32_fma"]["frac_of_derived"] = out["fp32_fma"]["value"] / derived
    return out


def main(argv=None) -> int:
    if not torch.cuda.is_available():
        print(json.dumps({"error": "no CUDA device"}))
        return 1
    print(json.dumps(measure()))
    return 0


if __name__ == "__main__":
    sys.exit(main())
