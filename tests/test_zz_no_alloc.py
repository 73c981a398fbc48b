"""hawkes_hess_diag_noalloc: the allocation-free variant for callers that
cannot call cudaMalloc while they evaluate (a plugin whose host program owns
every device allocation, or a loop that cannot afford cudaMalloc's implicit
device synchronisation).  It must give what hawkes_hess_diag gives with a
caller-provided workspace, call after call, although every call reuses the
same library-owned scratch array.

This file is collected last on purpose, so that a run stopping at the first
failure has already run every other test; it passes alone in a fresh process
too (the first call on the device does the one-time address lookup).
"""
import ctypes

import pytest

from paper_2103_03348_b300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _lib():
    from paper_2103_03348_b300 import build, hawkes
    build.build()
    L = hawkes.lib()
    vp = ctypes.c_void_p
    L.hawkes_hess_diag_noalloc.argtypes = [vp, vp, vp, vp, ctypes.c_int64, ctypes.POINTER(ctypes.c_double),
                                           ctypes.c_int, vp, vp, vp, vp, vp]
    L.hawkes_hess_diag_noalloc.restype = ctypes.c_int
    return hawkes, L


def _noalloc(L, x, y, t, r, params, precision):
    n = t.numel()
    dev = t.device
    ll = torch.empty((), dtype=torch.float64, device=dev)
    g = torch.empty(6 + n, dtype=torch.float64, device=dev)
    h = torch.empty(6 + n, dtype=torch.float64, device=dev)
    st = torch.empty((), dtype=torch.int32, device=dev)
    pa = (ctypes.c_double * 6)(*[float(v) for v in params])
    stream = torch.cuda.current_stream(dev).cuda_stream
    p = lambda a: ctypes.c_void_p(a.data_ptr())  # noqa: E731
    rc = L.hawkes_hess_diag_noalloc(p(x), p(y), p(t), p(r), n, pa, precision, p(ll), p(g), p(h), p(st),
                                    ctypes.c_void_p(stream))
    return rc, ll, g, h, st


@pytest.mark.parametrize("precision", [0, 1, 2, 3])
def test_noalloc_matches_workspace_call_twice(precision):
    """Both entry points run the same deterministic kernels on the same inputs,
    so the results must be equal bit for bit, also on the second call, which
    reuses the scratch array the first call filled (a large problem first, then
    a smaller one: stale bytes beyond the smaller one's extent are never read)."""
    hawkes, L = _lib()
    d = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda")  # noqa: E731
    name = ("fp64", "fp32c", "fp32c_band", "fp32c_st")[precision]
    for seed, n in ((31, 4096), (32, 1500)):
        w = synth.make_uniform(seed, n, box=1.0, t_max=1.0, r_sd=0.5, params=(0.5, 0.1, 0.05, 0.3, 10.0, 0.02))
        x, y, t, r = d(w.x), d(w.y), d(w.t), d(w.r)
        rc, ll, g, h, st = _noalloc(L, x, y, t, r, w.params, precision)
        assert rc == hawkes.OK, hawkes.strerror(rc)
        torch.cuda.synchronize()
        assert int(st.item()) == hawkes.OK
        ref_ll, ref_g, ref_h = hawkes.hess_diag(x, y, t, r, w.params, name)
        assert torch.equal(ll, ref_ll) and torch.equal(g, ref_g) and torch.equal(h, ref_h), (name, n)


def test_noalloc_rejects_too_many_events():
    hawkes, L = _lib()
    n = 4097
    z = torch.zeros(n, dtype=torch.float64, device="cuda")
    rc, *_ = _noalloc(L, z, z, z, z, (0.5, 0.1, 0.05, 0.3, 10.0, 0.02), 1)
    assert rc == hawkes.ESCRATCH
    assert "HAWKES_NOALLOC_MAX_EVENTS" in hawkes.strerror(rc)
