"""The C-ABI library loads, exports every symbol include/hawkes.h declares, and
rejects bad arguments synchronously before touching any pointer.  No GPU is
needed: argument checks return before the first CUDA call."""
import ctypes
import math
import os
import re

import pytest

from paper_2103_03348_b300 import build, hawkes

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    build.build()
    return hawkes.lib()


def declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(hawkes_\w+)\s*\(", src)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    assert {"hawkes_loglik", "hawkes_grad", "hawkes_hess_diag", "hawkes_workspace_size",
            "hawkes_strerror"} <= set(names)
    for nm in names:
        assert hasattr(L, nm), nm


def test_strerror_and_version(L):
    for code in range(7):
        assert len(hawkes.strerror(code)) > 5
    assert "unknown" in hawkes.strerror(99)
    assert "sm_103a" in hawkes.version()


def test_workspace_size(L):
    assert hawkes.workspace_size(1, "fp32c") == 0
    assert L.hawkes_workspace_size(2, 7) == 0
    a = hawkes.workspace_size(2000, "fp32c")
    b = hawkes.workspace_size(100_000, "fp32c")
    c = hawkes.workspace_size(100_000, "fp64")
    assert 0 < a < b and c > 0
    assert a % 256 == 0 and b % 256 == 0
    # the workspace for 1e5 events stays far below the GPU's memory
    assert b < 1 << 30


def _call(L, fn, n=10, params=(0.5, 0.1, 0.05, 0.3, 10.0, 0.02), precision=1, ws=4096, ws_bytes=None,
          out=8, status=16, x=1024, nullify=()):
    # fake, never-dereferenced addresses: the checks must reject before any use
    ptr = {"x": x, "y": 2048, "t": 3072, "r": 4096 + 1024, "ws": ws, "out": out, "status": status}
    for k in nullify:
        ptr[k] = 0
    pa = (ctypes.c_double * 6)(*params)
    wsb = ws_bytes if ws_bytes is not None else hawkes.workspace_size(max(n, 2), precision if precision in (0, 1) else 1)
    args = [ctypes.c_void_p(ptr["x"]), ctypes.c_void_p(ptr["y"]), ctypes.c_void_p(ptr["t"]), ctypes.c_void_p(ptr["r"]),
            ctypes.c_int64(n), pa, ctypes.c_int(precision), ctypes.c_void_p(ptr["ws"]), ctypes.c_size_t(wsb)]
    o = ctypes.c_void_p(ptr["out"])
    s = ctypes.c_void_p(ptr["status"])
    if fn == "loglik":
        return L.hawkes_loglik(*args, o, s, None)
    if fn == "grad":
        return L.hawkes_grad(*args, o, o, s, None)
    return L.hawkes_hess_diag(*args, o, o, o, s, None)


@pytest.mark.parametrize("fn", ["loglik", "grad", "hess"])
def test_argument_errors(L, fn):
    EINVAL, EWS = hawkes.EINVAL, hawkes.EWORKSPACE
    assert _call(L, fn, n=1) == EINVAL
    assert _call(L, fn, n=0) == EINVAL
    assert _call(L, fn, n=-5) == EINVAL
    assert _call(L, fn, precision=4) == EINVAL
    for bad in [(0.0, 0.1, 0.05, 0.3, 10.0, 0.02), (0.5, -0.1, 0.05, 0.3, 10.0, 0.02),
                (0.5, 0.1, 0.05, 0.3, math.nan, 0.02), (0.5, 0.1, 0.05, 0.3, 10.0, math.inf),
                (0.5, 0.1, -math.inf, 0.3, 10.0, 0.02), (0.5, 0.1, 0.05, 0.0, 10.0, 0.02)]:
        assert _call(L, fn, params=bad) == EINVAL, bad
    for k in ("x", "ws", "status", "out"):
        assert _call(L, fn, nullify=(k,)) == EINVAL, k
    assert _call(L, fn, ws=4096 + 16) == EINVAL  # workspace not 256-byte aligned
    assert _call(L, fn, ws_bytes=1000) == EWS


def test_hess_diag_accepts_null_loglik_and_grad_only_after_checks(L):
    # hdiag required: NULL hdiag is an argument error
    pa = (ctypes.c_double * 6)(0.5, 0.1, 0.05, 0.3, 10.0, 0.02)
    v = ctypes.c_void_p
    rc = L.hawkes_hess_diag(v(1024), v(2048), v(3072), v(4096), ctypes.c_int64(10), pa, 1, v(4096),
                            ctypes.c_size_t(1 << 30), None, None, None, v(16), None)
    assert rc == hawkes.EINVAL


def test_kernel_count_per_call():
    # FP32C: setup, prep, pack, row, finish, finalize [, column, column finish]
    assert hawkes.kernels_per_call("hess", "fp32c") == 8
    assert hawkes.kernels_per_call("grad", "fp64") == 9
    assert hawkes.kernels_per_call("loglik", "fp32c") == 6
    assert hawkes.kernels_per_call("hess", "fp32c_st") == 10  # and the slab sort and gather


def test_predictive_argument_checks(L):
    """hawkes_predictive refuses bad arguments before touching any pointer."""
    from paper_2103_03348_b300 import predictive
    P = predictive._lib()
    f = ctypes.c_void_p(1 << 20)
    ws = ctypes.c_size_t(1 << 30)
    good = dict(n=100, m=5, ns=4, stride=11, horizon=10.0, cap=1000)

    def call(**kw):
        a = dict(good, **kw)
        return P.hawkes_predictive(f, f, f, f, a["n"], f, a["m"], f, a["ns"], a["stride"], a["horizon"], 1, 0,
                                   a["cap"], f, ws, f, f, f, f, f, f, None)

    assert P.hawkes_predictive_workspace_size(0) == 0
    assert P.hawkes_predictive_workspace_size(100) >= 400
    assert call(n=0) == hawkes.EINVAL
    assert call(m=101) == hawkes.EINVAL
    assert call(stride=10) == hawkes.EINVAL            # q rows shorter than 6 + m
    assert call(horizon=0.0) == hawkes.EINVAL
    assert call(horizon=math.inf) == hawkes.EINVAL
    assert call(cap=0) == hawkes.EINVAL
    assert call(cap=(1 << 24) + 1) == hawkes.EINVAL
    assert call(ns=0) == hawkes.OK                     # nothing to do, nothing launched


def test_peak_microbenchmark_arguments(L):
    from paper_2103_03348_b300 import peaks
    P = peaks._lib()
    assert P.hawkes_peak_ops(0, 10, 104) == 10 * 256 * 104 * 8 * 2
    assert P.hawkes_peak_ops(2, 10, 104) == 10 * 256 * 104 * 8
    assert P.hawkes_peak_ops(3, 10, 104) == 0
    assert P.hawkes_peak_ops(0, 10, 100) == 0  # not a multiple of the unroll
    assert P.hawkes_peak_launch(5, 10, 100, ctypes.c_void_p(8), None) == hawkes.EINVAL
    assert P.hawkes_peak_launch(0, 0, 100, ctypes.c_void_p(8), None) == hawkes.EINVAL
    assert P.hawkes_peak_launch(0, 10, 100, None, None) == hawkes.EINVAL


def test_tree_mass_argument_checks(L):
    """hawkes_tree_mass_factor / _velocity / _momentum refuse bad arguments before any
    CUDA call (the fake pointers below are never dereferenced)."""
    from paper_2103_03348_b300 import tree
    T = tree._lib()
    f = ctypes.c_void_p(1 << 20)
    m = 10
    need = int(T.hawkes_tree_mass_workspace_size(m))
    assert T.hawkes_tree_mass_workspace_size(1) == 0
    assert need >= (6 * (2 * m - 1) + m) * 8
    good = dict(m=m, s2=1.0, rv=0.0, k=16, z0=6, nc=6, eps=0.1, ws=need)

    def vel(vel_=f, q=f, kin=f, **kw):
        a = dict(good, **kw)
        return T.hawkes_tree_mass_velocity(a["m"], f, f, a["nc"], f, a["k"], a["z0"], f, f, vel_, q, a["eps"], kin,
                                           f, ctypes.c_size_t(a["ws"]), None)

    def fac(**kw):
        a = dict(good, **kw)
        return T.hawkes_tree_mass_factor(a["m"], f, f, a["rv"], a["s2"], f, f, f, ctypes.c_size_t(a["ws"]), None)

    def mom(**kw):
        a = dict(good, **kw)
        return T.hawkes_tree_mass_momentum(a["m"], f, f, a["rv"], a["s2"], f, a["nc"], f, a["k"], a["z0"], f, f, f,
                                           f, ctypes.c_size_t(a["ws"]), None)

    for call in (vel, mom, fac):
        assert call(m=1) == hawkes.EINVAL
        assert call(ws=need - 8) == hawkes.EWORKSPACE
    for call in (vel, mom):
        assert call(nc=7) == hawkes.EINVAL              # coupled coordinates overlap the rate block
        assert call(nc=-1) == hawkes.EINVAL
        assert call(nc=9, z0=9, k=20) == hawkes.EINVAL  # more than 8 coupled coordinates
        assert call(k=9) == hawkes.EINVAL               # the block does not fit in the state
        assert call(z0=7) == hawkes.EINVAL              # z0 + m > k
        assert call(z0=-1) == hawkes.EINVAL
    for call in (mom, fac):
        assert call(s2=0.0) == hawkes.EINVAL
        assert call(rv=-1.0) == hawkes.EINVAL
        assert call(rv=math.nan) == hawkes.EINVAL
    assert vel(vel_=None, q=None, kin=None) == hawkes.EINVAL  # nothing to compute
    assert vel(eps=math.inf) == hawkes.EINVAL
