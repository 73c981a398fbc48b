"""Python binding of libhawkes.so (argument marshalling only).

Every step of the computation runs in the CUDA library; this module only turns
torch CUDA tensors into device pointers, the parameter vector into a host
double[6] and the current torch stream into a cudaStream_t, allocates the
caller-owned workspace with torch, and reads back the device status.  There
is no CPU fallback: if the library is missing or no GPU is present the calls
raise.

    ll = loglik(x, y, t, r, params)                      # Eq. 1
    ll, g = grad(x, y, t, r, params)                     # + gradient (6 + N)
    ll, g, h = hess_diag(x, y, t, r, params)             # + Hessian diagonal (6 + N)
    HawkesLogLik.apply(x, y, t, r, params_tensor, "fp32c")   # differentiable scalar

Parameter order: (mu0, tau_x, tau_t, theta0, omega, h); tau_t = inf gives the
paper's purely spatial background.  x, y, t, r are float64 CUDA tensors of
length N sorted by t; r holds the per-event log-rates log theta_n.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libhawkes.so")

FP64, FP32C, FP32C_BAND, FP32C_ST = 0, 1, 2, 3
PRECISIONS = {"fp64": FP64, "fp32c": FP32C, "fp32c_band": FP32C_BAND, "fp32c_st": FP32C_ST, FP64: FP64, FP32C: FP32C,
              FP32C_BAND: FP32C_BAND, FP32C_ST: FP32C_ST}

OK, EINVAL, EUNSORTED, ENONFINITE, EWORKSPACE, ECUDA, EZERO, ESCRATCH = range(8)

_lock = threading.Lock()
_lib = None
_ws_cache: dict = {}


class HawkesError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{msg} (status {code})")
        self.code = code


def lib():
    """Load libhawkes.so once; raise loudly if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"libhawkes.so not built at {LIB_PATH}; run python -m paper_2103_03348_b300.build")
            L = ctypes.CDLL(LIB_PATH)
            vp, dp, ip, i64, sz = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_void_p, ctypes.c_int64, ctypes.c_size_t
            common = [vp, vp, vp, vp, i64, dp, ctypes.c_int, vp, sz]
            L.hawkes_workspace_size.argtypes = [i64, ctypes.c_int]
            L.hawkes_workspace_size.restype = sz
            L.hawkes_loglik.argtypes = common + [vp, ip, vp]
            L.hawkes_loglik.restype = ctypes.c_int
            L.hawkes_grad.argtypes = common + [vp, vp, ip, vp]
            L.hawkes_grad.restype = ctypes.c_int
            L.hawkes_hess_diag.argtypes = common + [vp, vp, vp, ip, vp]
            L.hawkes_hess_diag.restype = ctypes.c_int
            L.hawkes_hess_diag_timed.argtypes = common + [vp, vp, vp, ip, vp, ctypes.POINTER(ctypes.c_void_p)]
            L.hawkes_eval_device_params.argtypes = [vp, vp, vp, vp, i64, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                    vp, sz, vp, vp, vp, ip, vp]
            L.hawkes_eval_device_params.restype = ctypes.c_int
            L.hawkes_eval_rates_subset.argtypes = [vp, vp, vp, vp, i64, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                   vp, i64, vp, sz, vp, vp, vp, vp, vp]
            L.hawkes_eval_rates_subset.restype = ctypes.c_int
            L.hawkes_hess_diag_timed.restype = ctypes.c_int
            L.hawkes_strerror.argtypes = [ctypes.c_int]
            L.hawkes_strerror.restype = ctypes.c_char_p
            L.hawkes_version.argtypes = []
            L.hawkes_version.restype = ctypes.c_char_p
            _lib = L
    return _lib


def strerror(code: int) -> str:
    return lib().hawkes_strerror(int(code)).decode()


def workspace_size(n: int, precision="fp32c") -> int:
    return int(lib().hawkes_workspace_size(int(n), PRECISIONS[precision]))


def kernels_per_call(mode: str, precision="fp32c") -> int:
    """Number of kernels one call launches (memsets excluded)."""
    p = PRECISIONS[precision]
    # FP64: setup, prep, pack, row, combine, epilogue, finalize; FP32C: setup, prep,
    # pack, row, finish (combine, FP64 fix-up of tiny rows, epilogue), finalize
    k = 7 if p == FP64 else 6
    if p == FP32C_ST:
        k += 2  # order: slab sort, gather
    if mode in ("grad", "hess"):
        k += 2  # column pass, column finish
    return k


def _workspace(n: int, precision: int, device) -> torch.Tensor:
    key = (int(n), precision, str(device))
    ws = _ws_cache.get(key)
    if ws is None:
        nbytes = workspace_size(n, precision)
        if nbytes == 0:
            raise HawkesError(EINVAL, "invalid n for workspace")
        ws = torch.empty(nbytes, dtype=torch.uint8, device=device)
        _ws_cache.clear()  # keep one workspace alive at a time
        _ws_cache[key] = ws
    return ws


def _params_array(params):
    if isinstance(params, torch.Tensor):
        vals = [float(v) for v in params.detach().cpu().double().tolist()]
    else:
        vals = [float(v) for v in params]
    if len(vals) != 6:
        raise ValueError("params must hold 6 values (mu0, tau_x, tau_t, theta0, omega, h)")
    return (ctypes.c_double * 6)(*vals)


def _check_events(x, y, t, r):
    for name, a in (("x", x), ("y", y), ("t", t), ("r", r)):
        if not isinstance(a, torch.Tensor) or not a.is_cuda:
            raise TypeError(f"{name} must be a CUDA tensor")
        if a.dtype != torch.float64 or not a.is_contiguous() or a.dim() != 1:
            raise TypeError(f"{name} must be a contiguous 1-D float64 tensor")
    n = t.numel()
    if not (x.numel() == y.numel() == r.numel() == n):
        raise ValueError("x, y, t, r must have the same length")
    if not (x.device == y.device == t.device == r.device):
        raise ValueError("x, y, t, r must be on the same device")
    return n


def _raise_status(code: int):
    if code == OK:
        return
    if code == EZERO:
        raise FloatingPointError(strerror(code))
    if code in (EUNSORTED, ENONFINITE):
        raise ValueError(strerror(code))
    raise HawkesError(code, strerror(code))


MODES = {"loglik": 0, "grad": 1, "hess": 2, "grad_globals": 3, "hess_globals": 4}


REUSE_EVENTS = 16  # HAWKES_MODE_REUSE_EVENTS


def _call(mode: str, x, y, t, r, params, precision="fp32c", stream=None, workspace=None, check=True, out=None,
          phase_events=None, log_params=False, reuse_events=False, rate_idx=None):
    """One evaluation.  params: a 6-sequence or CPU tensor (passed as a host
    vector), or a CUDA float64 tensor whose first six entries are read on the
    device (their logarithms when log_params) with no host round trip.
    reuse_events (device params only): x, y, t and the workspace are those of
    an earlier call, whose event preparation is reused.
    rate_idx (device params, modes grad / hess): a device int32 tensor of the
    sources whose rate entries are wanted; only those entries are written."""
    n = _check_events(x, y, t, r)
    p = PRECISIONS[precision]
    dev = t.device
    ws = workspace if workspace is not None else _workspace(n, p, dev)
    if out is None:
        out = {
            "loglik": torch.empty((), dtype=torch.float64, device=dev),
            "grad": torch.empty(6 + n, dtype=torch.float64, device=dev) if mode != "loglik" else None,
            "hdiag": torch.empty(6 + n, dtype=torch.float64, device=dev) if mode in ("hess", "hess_globals") else None,
            "status": torch.empty((), dtype=torch.int32, device=dev),
        }
    if stream is None:
        stream = torch.cuda.current_stream(dev).cuda_stream
    elif isinstance(stream, torch.cuda.Stream):
        stream = stream.cuda_stream
    L = lib()
    if rate_idx is not None:
        if not (isinstance(params, torch.Tensor) and params.is_cuda) or mode not in ("grad", "hess"):
            raise ValueError("rate_idx needs device params and mode grad or hess")
        if rate_idx.dtype != torch.int32 or rate_idx.dim() != 1 or not rate_idx.is_contiguous() \
                or rate_idx.device != dev:
            raise TypeError("rate_idx must be a contiguous 1-D int32 tensor on the events' device")
    if isinstance(params, torch.Tensor) and params.is_cuda:
        if params.dtype != torch.float64 or not params.is_contiguous() or params.numel() < 6:
            raise TypeError("device params must be a contiguous float64 CUDA tensor with at least 6 entries")
        st_p = ctypes.c_void_p(out["status"].data_ptr())
        ptrs = [ctypes.c_void_p(out[k].data_ptr()) if out.get(k) is not None else ctypes.c_void_p(0)
                for k in ("loglik", "grad", "hdiag")]
        if mode not in ("hess", "hess_globals"):
            ptrs[2] = ctypes.c_void_p(0)
        if mode == "loglik":
            ptrs[1] = ctypes.c_void_p(0)
        common = (ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(t.data_ptr()),
                  ctypes.c_void_p(r.data_ptr()), ctypes.c_int64(n), ctypes.c_void_p(params.data_ptr()),
                  int(bool(log_params)), p, MODES[mode] | (REUSE_EVENTS if reuse_events else 0))
        with torch.cuda.device(dev):
            if rate_idx is not None:
                rc = L.hawkes_eval_rates_subset(*common, ctypes.c_void_p(rate_idx.data_ptr()),
                                                ctypes.c_int64(rate_idx.numel()), ctypes.c_void_p(ws.data_ptr()),
                                                ctypes.c_size_t(ws.numel()), *ptrs, st_p, ctypes.c_void_p(int(stream)))
            else:
                rc = L.hawkes_eval_device_params(*common, ctypes.c_void_p(ws.data_ptr()), ctypes.c_size_t(ws.numel()),
                                                 *ptrs, st_p, ctypes.c_void_p(int(stream)))
        if rc != OK:
            raise HawkesError(rc, strerror(rc))
        if check:
            _raise_status(int(out["status"].item()))
        return out
    pa = _params_array(params)
    args = [ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(t.data_ptr()),
            ctypes.c_void_p(r.data_ptr()), ctypes.c_int64(n), pa, ctypes.c_int(p),
            ctypes.c_void_p(ws.data_ptr()), ctypes.c_size_t(ws.numel())]
    ll_p = ctypes.c_void_p(out["loglik"].data_ptr())
    st_p = ctypes.c_void_p(out["status"].data_ptr())
    s_p = ctypes.c_void_p(int(stream))
    with torch.cuda.device(dev):
        if mode == "loglik":
            rc = L.hawkes_loglik(*args, ll_p, st_p, s_p)
        elif mode == "grad":
            rc = L.hawkes_grad(*args, ll_p, ctypes.c_void_p(out["grad"].data_ptr()), st_p, s_p)
        else:
            g_p = ctypes.c_void_p(out["grad"].data_ptr()) if out.get("grad") is not None else ctypes.c_void_p(0)
            h_p = ctypes.c_void_p(out["hdiag"].data_ptr())
            if phase_events is None:
                rc = L.hawkes_hess_diag(*args, ll_p, g_p, h_p, st_p, s_p)
            else:
                # torch creates events lazily: record each once so that it has a handle
                for e in phase_events:
                    if e.cuda_event == 0:
                        e.record()
                evs = (ctypes.c_void_p * 4)(*[ctypes.c_void_p(e.cuda_event) for e in phase_events])
                rc = L.hawkes_hess_diag_timed(*args, ll_p, g_p, h_p, st_p, s_p, evs)
    if rc != OK:
        raise HawkesError(rc, strerror(rc))
    if check:
        _raise_status(int(out["status"].item()))
    return out


def loglik(x, y, t, r, params, precision="fp32c", **kw):
    """Eq. 1 on the GPU; returns a 0-d float64 CUDA tensor."""
    return _call("loglik", x, y, t, r, params, precision, **kw)["loglik"]


def grad(x, y, t, r, params, precision="fp32c", **kw):
    """(loglik, gradient[6 + N]) on the GPU."""
    o = _call("grad", x, y, t, r, params, precision, **kw)
    return o["loglik"], o["grad"]


def hess_diag(x, y, t, r, params, precision="fp32c", **kw):
    """(loglik, gradient[6 + N], Hessian diagonal[6 + N]) on the GPU."""
    o = _call("hess", x, y, t, r, params, precision, **kw)
    return o["loglik"], o["grad"], o["hdiag"]


class HawkesLogLik(torch.autograd.Function):
    """Differentiable log-likelihood: forward runs the fused row + column passes
    (hawkes_grad) once and keeps the gradient; backward scales it by the
    incoming gradient, with no second pass over the pairs.

    Inputs: x, y, t (no gradient), r (log-rates, [N]) and params (6-vector,
    CPU or CUDA tensor; gradient w.r.t. the raw parameters)."""

    @staticmethod
    def forward(ctx, x, y, t, r, params, precision="fp32c"):
        ll, g = grad(x, y, t, r.detach(), params.detach(), precision)
        ctx.save_for_backward(g)
        ctx.params_device = params.device
        return ll.clone()

    @staticmethod
    def backward(ctx, grad_out):
        (g,) = ctx.saved_tensors
        gr = (grad_out * g[6:]) if ctx.needs_input_grad[3] else None
        gp = (grad_out * g[:6]).to(ctx.params_device) if ctx.needs_input_grad[4] else None
        return None, None, None, gr, gp, None


def version() -> str:
    return lib().hawkes_version().decode()


def st_live_pairs(n: int, workspace: torch.Tensor, stream=None) -> dict:
    """Pairs the HAWKES_FP32C_ST passes evaluate for the evaluation held in
    `workspace` (a hess evaluation of n events in that precision): background
    and excitation pairs of the row pass, pairs of the column pass."""
    L = lib()
    if not getattr(L, "_st_count_typed", False):
        L.hawkes_st_live_pairs.argtypes = [ctypes.c_int64, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p,
                                           ctypes.c_void_p]
        L.hawkes_st_live_pairs.restype = ctypes.c_int
        L._st_count_typed = True
    dev = workspace.device
    counts = torch.zeros(3, dtype=torch.int64, device=dev)
    if stream is None:
        stream = torch.cuda.current_stream(dev).cuda_stream
    elif isinstance(stream, torch.cuda.Stream):
        stream = stream.cuda_stream
    with torch.cuda.device(dev):
        rc = L.hawkes_st_live_pairs(int(n), ctypes.c_void_p(workspace.data_ptr()), ctypes.c_size_t(workspace.numel()),
                                    ctypes.c_void_p(counts.data_ptr()), ctypes.c_void_p(stream))
    _raise_status(rc)
    c = [int(v) for v in counts.cpu().tolist()]
    return {"row_background_pairs": c[0], "row_excitation_pairs": c[1], "column_pairs": c[2]}
