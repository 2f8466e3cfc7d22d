"""Measured throughput peaks of the pipes the render kernels are bound by.

The render forward and backward are bound by instruction issue (FP32 arithmetic and the
special-function unit), not by HBM, so their roofline denominators are the GPU's FP32
fused-multiply-add rate and its ex2 / rcp rate, measured here with the library's
microbenchmark kernels (ges_peak_run) and CUDA events, together with the FP32 atomic-add
rate into L2 in the backward's accumulator pattern and the SM count read from the device.
"""
from __future__ import annotations

import ctypes
from typing import Dict

import torch

from . import _lib
from .api import _stream

KINDS = {"fp32_fma": 0, "mufu_ex2": 1, "mufu_rcp": 2, "l2_atomic_add": 3}


def run(kind: int, blocks_per_sm: int, iters: int, sink: torch.Tensor) -> int:
    """Launches one microbenchmark kernel on the current stream; returns its operation count."""
    ops = ctypes.c_uint64(0)
    _lib.check(_lib.lib().ges_peak_run(kind, blocks_per_sm, iters, ctypes.c_void_p(sink.data_ptr()),
                                       sink.numel(), _stream(None), ctypes.byref(ops)), "ges_peak_run")
    return int(ops.value)


def _best_rate(kind: int, blocks_per_sm: int, iters: int, sink: torch.Tensor, reps: int) -> float:
    """Operations per second of the fastest of `reps` timed launches (after one warm-up)."""
    run(kind, blocks_per_sm, iters, sink)
    best = 0.0
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ops = run(kind, blocks_per_sm, iters, sink)
        e1.record()
        torch.cuda.synchronize()
        best = max(best, ops / (e0.elapsed_time(e1) / 1e3))
    return best


def measure(reps: int = 5) -> Dict[str, float]:
    """Peaks of this GPU: fp32_tflops (FMA, 2 flops each), mufu_ex2_gops, mufu_rcp_gops,
    l2_atomic_gops (FP32 adds into a 64 MB buffer, which L2 holds), and sm_count."""
    dev = torch.cuda.current_device()
    props = torch.cuda.get_device_properties(dev)
    sink = torch.zeros(16 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 64 MB, 1M lines
    # each launch runs for tens of milliseconds, far above launch overhead
    out = {"sm_count": int(props.multi_processor_count)}
    out["fp32_tflops"] = _best_rate(KINDS["fp32_fma"], 8, 4096, sink, reps) / 1e12
    out["mufu_ex2_gops"] = _best_rate(KINDS["mufu_ex2"], 8, 1024, sink, reps) / 1e9
    out["mufu_rcp_gops"] = _best_rate(KINDS["mufu_rcp"], 8, 1024, sink, reps) / 1e9
    out["l2_atomic_gops"] = _best_rate(KINDS["l2_atomic_add"], 8, 2048, sink, reps) / 1e9
    torch.cuda.synchronize()
    return out


if __name__ == "__main__":
    import json
    print(json.dumps(measure()))
