"""Measured ALU peaks of this GPU (packed FP32 FMA, MUFU exp2, FP64 FMA) from
the library's microbenchmark kernels, timed with CUDA events."""
from __future__ import annotations

import ctypes

import torch

from . import hawkes

KINDS = {0: "ffma2_lane_fma_per_s", 1: "ex2_per_s", 2: "dfma_per_s"}


def _lib():
    L = hawkes.lib()
    if not getattr(L, "_peak_typed", False):
        L.hawkes_peak_ops.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_int]
        L.hawkes_peak_ops.restype = ctypes.c_int64
        L.hawkes_peak_launch.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
        L.hawkes_peak_launch.restype = ctypes.c_int
        L._peak_typed = True
    return L


def measure(device="cuda", reps=5):
    """{kind: best rate over reps} with enough blocks to fill every SM several times."""
    L = _lib()
    dev = torch.device(device)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks = sms * 16
    sink = torch.zeros(1, dtype=torch.float32, device=dev)
    s = torch.cuda.current_stream(dev)
    out = {"sms": sms}
    for which, name in KINDS.items():
        iters = {0: 8192, 1: 2048, 2: 512}[which]
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        best = 0.0
        for i in range(reps + 1):
            ev[0].record(s)
            rc = L.hawkes_peak_launch(which, blocks, iters, ctypes.c_void_p(sink.data_ptr()),
                                      ctypes.c_void_p(s.cuda_stream))
            if rc != hawkes.OK:
                raise hawkes.HawkesError(rc, hawkes.strerror(rc))
            ev[1].record(s)
            ev[1].synchronize()
            if i > 0:
                best = max(best, L.hawkes_peak_ops(which, blocks, iters) / (ev[0].elapsed_time(ev[1]) * 1e-3))
        out[name] = best
    return out
