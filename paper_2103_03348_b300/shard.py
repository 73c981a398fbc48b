"""Sharded evaluation of the log-likelihood and its derivatives.

The double sum splits over k shards by 128-event tiles: each shard runs the
row pass (Eq. 1 inner sums) for its target tiles, publishes one record per
tile (partial sums and column weights B / lambda_n) into its slice of an
exchange buffer, and after an all-gather of the slices runs the column pass
(Eqs. 4-5) for its source tiles.  The union of the shards' outputs equals the
unsharded evaluation bit for bit.

`evaluate` runs every shard in sequence on one GPU, each with its own
workspace and exchange buffer (the exchange is a device copy between them);
`allgather_records` is the same exchange between ranks over torch.distributed
(NCCL on GPUs, gloo on CPUs), and `distributed_evaluate` composes the whole
evaluation across the ranks of a process group: each rank's row phase, the
record all-gather, each rank's column phase, and an all-gather of the
per-event entries, so that every rank ends with the unsharded call's outputs.
"""
from __future__ import annotations

import ctypes

import torch
import torch.distributed as dist

from . import hawkes

RECORD_DOUBLES = 16 + 128


def _lib():
    L = hawkes.lib()
    if not getattr(L, "_shard_typed", False):
        vp, i64, sz, ci = ctypes.c_void_p, ctypes.c_int64, ctypes.c_size_t, ctypes.c_int
        L.hawkes_shard_exchange_size.argtypes = [i64]
        L.hawkes_shard_exchange_size.restype = sz
        L.hawkes_shard_range.argtypes = [i64, ci, ci, ctypes.POINTER(i64), ctypes.POINTER(i64),
                                         ctypes.POINTER(sz), ctypes.POINTER(sz)]
        L.hawkes_shard_range.restype = ci
        L.hawkes_shard_rows.argtypes = [vp, vp, vp, vp, i64, vp, ci, ci, ci, ci, vp, sz, vp, sz, vp, vp]
        L.hawkes_shard_rows.restype = ci
        L.hawkes_shard_cols.argtypes = [vp, vp, vp, vp, i64, vp, ci, ci, ci, ci, vp, sz, vp, sz, vp, vp, vp, vp, vp]
        L.hawkes_shard_cols.restype = ci
        L._shard_typed = True
    return L


def _check(rc):
    if rc != hawkes.OK:
        raise hawkes.HawkesError(rc, hawkes.strerror(rc))


def shard_range(n: int, shard: int, n_shards: int):
    """(first_event, end_event, record_first, record_end) of a shard."""
    L = _lib()
    a, b = ctypes.c_int64(), ctypes.c_int64()
    off, nb = ctypes.c_size_t(), ctypes.c_size_t()
    _check(L.hawkes_shard_range(n, shard, n_shards, ctypes.byref(a), ctypes.byref(b), ctypes.byref(off),
                                ctypes.byref(nb)))
    rec = RECORD_DOUBLES * 8
    return a.value, b.value, off.value // rec, (off.value + nb.value) // rec


def n_records(n: int) -> int:
    return int(_lib().hawkes_shard_exchange_size(n)) // (RECORD_DOUBLES * 8)


class Shard:
    """One shard's workspace and exchange buffer (records as a [T, 144] float64 tensor)."""

    def __init__(self, n: int, precision: str, shard: int, n_shards: int, device="cuda"):
        self.n, self.precision, self.shard, self.n_shards = n, precision, shard, n_shards
        self.p = hawkes.PRECISIONS[precision]
        self.ws = torch.empty(hawkes.workspace_size(n, precision), dtype=torch.uint8, device=device)
        self.xbuf = torch.zeros(n_records(n), RECORD_DOUBLES, dtype=torch.float64, device=device)
        self.first, self.end, self.rec0, self.rec1 = shard_range(n, shard, n_shards)
        self.status = torch.zeros((), dtype=torch.int32, device=device)

    def _common(self, x, y, t, r, params, mode):
        pa = (ctypes.c_double * 6)(*[float(v) for v in params])
        return [ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(t.data_ptr()),
                ctypes.c_void_p(r.data_ptr()), self.n, pa, self.p, hawkes.MODES[mode], self.shard, self.n_shards,
                ctypes.c_void_p(self.ws.data_ptr()), ctypes.c_size_t(self.ws.numel())]

    def rows(self, x, y, t, r, params, mode="hess"):
        s = ctypes.c_void_p(torch.cuda.current_stream(x.device).cuda_stream)
        _check(_lib().hawkes_shard_rows(*self._common(x, y, t, r, params, mode),
                                        ctypes.c_void_p(self.xbuf.data_ptr()),
                                        ctypes.c_size_t(self.xbuf.numel() * 8),
                                        ctypes.c_void_p(self.status.data_ptr()), s))

    def cols(self, x, y, t, r, params, out, mode="hess"):
        """Fills out['loglik'] and the shard's entries of out['grad'] / out['hdiag']."""
        s = ctypes.c_void_p(torch.cuda.current_stream(x.device).cuda_stream)
        p = lambda k: ctypes.c_void_p(out[k].data_ptr() if out.get(k) is not None else 0)  # noqa: E731
        _check(_lib().hawkes_shard_cols(*self._common(x, y, t, r, params, mode),
                                        ctypes.c_void_p(self.xbuf.data_ptr()),
                                        ctypes.c_size_t(self.xbuf.numel() * 8),
                                        p("loglik"), p("grad"), p("hdiag"),
                                        ctypes.c_void_p(self.status.data_ptr()), s))


def exchange_local(shards):
    """The all-gather on one device: every shard's records into every buffer."""
    for src in shards:
        sl = slice(src.rec0, src.rec1)
        for dst in shards:
            if dst is not src and src.rec1 > src.rec0:
                dst.xbuf[sl].copy_(src.xbuf[sl])


def allgather_records(xbuf: torch.Tensor, n: int, rank: int, world: int, group=None):
    """The exchange between ranks: all-gather each rank's record slice into
    every rank's xbuf ([T, 144]) over torch.distributed.  Slices differ in
    length by at most one record, so they travel padded to the longest."""
    ranges = [shard_range(n, s, world)[2:] for s in range(world)]
    return _allgather_slices(xbuf, ranges, rank, group)


def evaluate(x, y, t, r, params, precision="fp32c", n_shards=2, mode="hess"):
    """(loglik, grad, hdiag) from n_shards shards run in sequence on one GPU.

    Each shard has its own workspace and exchange buffer, as on separate
    ranks; the outputs are assembled from the shards' disjoint entries."""
    n = t.numel()
    dev = t.device
    shards = [Shard(n, precision, s, n_shards, dev) for s in range(n_shards)]
    for sh in shards:
        sh.rows(x, y, t, r, params, mode)
    exchange_local(shards)
    f64 = dict(dtype=torch.float64, device=dev)
    grad = torch.full((6 + n,), float("nan"), **f64) if mode in ("grad", "hess") else None
    hdiag = torch.full((6 + n,), float("nan"), **f64) if mode == "hess" else None
    ll = None
    statuses = []
    for sh in shards:
        out = {"loglik": torch.empty((), **f64),
               "grad": torch.full((6 + n,), float("nan"), **f64) if grad is not None else None,
               "hdiag": torch.full((6 + n,), float("nan"), **f64) if hdiag is not None else None}
        sh.cols(x, y, t, r, params, out, mode)
        if ll is None:
            ll = out["loglik"]
            if grad is not None:
                grad[:6] = out["grad"][:6]
            if hdiag is not None:
                hdiag[:6] = out["hdiag"][:6]
        sl = slice(6 + sh.first, 6 + sh.end)
        if grad is not None:
            grad[sl] = out["grad"][sl]
        if hdiag is not None:
            hdiag[sl] = out["hdiag"][sl]
        statuses.append(sh.status)
    st = int(torch.stack(statuses).max().item())
    if st != hawkes.OK:
        raise hawkes.HawkesError(st, hawkes.strerror(st))
    return ll, grad, hdiag


def _allgather_slices(full: torch.Tensor, ranges, rank: int, group=None, stage_on_host=False):
    """All-gather the slices full[a:b] that each rank owns (ranges[s] = (a, b))
    into every rank's copy of `full`, padded to the longest slice; with
    stage_on_host the bytes travel through host memory (a gloo group)."""
    longest = max(max(b - a for a, b in ranges), 1)
    a, b = ranges[rank]
    dev = torch.device("cpu") if stage_on_host else full.device
    send = torch.zeros((longest,) + tuple(full.shape[1:]), dtype=full.dtype, device=dev)
    send[: b - a].copy_(full[a:b])
    recv = [torch.empty_like(send) for _ in range(len(ranges))]
    dist.all_gather(recv, send, group=group)
    for s, (a2, b2) in enumerate(ranges):
        if s != rank and b2 > a2:
            full[a2:b2].copy_(recv[s][: b2 - a2])
    return full


def distributed_evaluate(x, y, t, r, params, precision="fp32c", mode="hess", group=None, shard=None):
    """(loglik, grad, hdiag) of the whole problem on every rank of `group`,
    each rank evaluating one shard: its row phase, the all-gather of the
    per-tile records (0.9 MB at 100,000 events), its column phase, then an
    all-gather of the per-event entries (each rank owns a disjoint range).
    The result equals hawkes_hess_diag bit for bit.  Every rank passes the
    same events (replicated) and parameters.  With a gloo group and device
    tensors the exchanged bytes are staged through host memory; with NCCL
    they stay on the device.  shard: an optional Shard of this rank to reuse
    (its workspace and exchange buffer)."""
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    n = t.numel()
    dev = t.device
    host = dist.get_backend(group) == "gloo" and dev.type == "cuda"
    sh = shard if shard is not None else Shard(n, precision, rank, world, dev)
    if (sh.n, sh.shard, sh.n_shards) != (n, rank, world):
        raise ValueError("the shard belongs to another problem or rank")
    sh.rows(x, y, t, r, params, mode)
    rec_ranges = [shard_range(n, s, world)[2:] for s in range(world)]
    if host:
        buf = sh.xbuf.cpu()
        _allgather_slices(buf, rec_ranges, rank, group, stage_on_host=True)
        sh.xbuf.copy_(buf)
    else:
        _allgather_slices(sh.xbuf, rec_ranges, rank, group)
    f64 = dict(dtype=torch.float64, device=dev)
    out = {"loglik": torch.empty((), **f64),
           "grad": torch.zeros(6 + n, **f64) if mode in ("grad", "hess") else None,
           "hdiag": torch.zeros(6 + n, **f64) if mode == "hess" else None}
    sh.cols(x, y, t, r, params, out, mode)
    ev_ranges = [(6 + a, 6 + b) for a, b, _, _ in (shard_range(n, s, world) for s in range(world))]
    for k in ("grad", "hdiag"):
        if out[k] is None:
            continue
        if host:
            v = out[k].cpu()
            _allgather_slices(v, ev_ranges, rank, group, stage_on_host=True)
            out[k].copy_(v)
        else:
            _allgather_slices(out[k], ev_ranges, rank, group)
    st = sh.status.to(torch.int64)
    st = st.cpu() if host else st
    dist.all_reduce(st, op=dist.ReduceOp.MAX, group=group)
    code = int(st.item())
    if code != hawkes.OK:
        raise hawkes.HawkesError(code, hawkes.strerror(code))
    return out["loglik"], out["grad"], out["hdiag"]
