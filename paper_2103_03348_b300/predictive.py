"""Posterior-predictive simulation over many parameter settings on the GPU
(the forward simulation the paper's Discussion proposes): the binding of
hawkes_predictive.  Every event is drawn by the library's kernel."""
from __future__ import annotations

import ctypes

import torch

from . import hawkes

MAX_CAPACITY = 1 << 24
STATUS_OK, STATUS_OVERFLOW, STATUS_BADPARAM = 0, 1, 2


def _lib():
    L = hawkes.lib()
    if not getattr(L, "_pred_typed", False):
        vp, i64 = ctypes.c_void_p, ctypes.c_int64
        L.hawkes_predictive_workspace_size.argtypes = [i64]
        L.hawkes_predictive_workspace_size.restype = ctypes.c_size_t
        L.hawkes_predictive.argtypes = [vp, vp, vp, vp, i64, vp, i64, vp, i64, i64, ctypes.c_double,
                                        ctypes.c_uint64, ctypes.c_uint32, i64, vp, ctypes.c_size_t,
                                        vp, vp, vp, vp, vp, vp, vp]
        L.hawkes_predictive.restype = ctypes.c_int
        L._pred_typed = True
    return L


def simulate(x, y, t, r_base, seq_idx, q, horizon: float, seed: int, capacity: int, sample_offset: int = 0):
    """Events of (T0, T0 + horizon] for every row of q (device, [S, 6 + M]).

    Returns a dict of device tensors: x, y, t [S, capacity] (rows valid up to
    count), src [S, capacity], count [S], status [S]."""
    L = _lib()
    dev = t.device
    n = t.numel()
    q = q.contiguous()
    s_count = q.shape[0]
    seq = seq_idx.to(device=dev, dtype=torch.int32).contiguous()
    m = seq.numel()
    ws = torch.empty(int(L.hawkes_predictive_workspace_size(n)), dtype=torch.uint8, device=dev)
    f64 = dict(dtype=torch.float64, device=dev)
    out = {"x": torch.empty(s_count, capacity, **f64), "y": torch.empty(s_count, capacity, **f64),
           "t": torch.empty(s_count, capacity, **f64),
           "src": torch.empty(s_count, capacity, dtype=torch.int64, device=dev),
           "count": torch.empty(s_count, dtype=torch.int64, device=dev),
           "status": torch.empty(s_count, dtype=torch.int32, device=dev)}
    p = lambda a: ctypes.c_void_p(a.data_ptr())  # noqa: E731
    rc = L.hawkes_predictive(p(x), p(y), p(t), p(r_base), n, p(seq) if m else None, m, p(q), s_count, q.shape[1],
                             float(horizon), int(seed), int(sample_offset), int(capacity), p(ws),
                             ctypes.c_size_t(ws.numel()), p(out["x"]), p(out["y"]), p(out["t"]), p(out["src"]),
                             p(out["count"]), p(out["status"]),
                             ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream))
    if rc != hawkes.OK:
        raise hawkes.HawkesError(rc, hawkes.strerror(rc))
    return out
